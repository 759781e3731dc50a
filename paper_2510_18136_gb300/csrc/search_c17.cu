// Search kernel instantiation for chunks of 17 samples per lane (windows up to 543 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(17)
NSFRB_INSTANTIATE_PIPE(17, 0)
}  // namespace nsfrb
