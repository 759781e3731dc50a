// Search kernel instantiation for chunks of 9 samples per lane (windows up to 287 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(9)
NSFRB_INSTANTIATE_PIPE(9, 0)
}  // namespace nsfrb
