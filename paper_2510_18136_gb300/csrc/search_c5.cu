// Search kernel instantiation for chunks of 5 samples per lane (windows up to 159 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(5)
NSFRB_INSTANTIATE_PIPE(5, 0)
}  // namespace nsfrb
