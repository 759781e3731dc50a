// Search kernel instantiation for chunks of 39 samples per lane (windows of 1216 to 1247 samples).
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(39)
NSFRB_INSTANTIATE_PIPE(39, 0)
}  // namespace nsfrb
