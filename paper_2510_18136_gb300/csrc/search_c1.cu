// Search kernel instantiation for chunks of 1 samples per lane (windows up to 31 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(1)
NSFRB_INSTANTIATE_PIPE(1, 0)
}  // namespace nsfrb
