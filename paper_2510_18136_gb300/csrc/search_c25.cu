// Search kernel instantiation for chunks of 25 samples per lane (windows up to 799 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(25)
NSFRB_INSTANTIATE_PIPE(25, 0)
}  // namespace nsfrb
