// Search kernel instantiation for chunks of 3 samples per lane (windows up to 95 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(3)
NSFRB_INSTANTIATE_PIPE(3, 0)
}  // namespace nsfrb
