// Search kernel instantiation for chunks of 38 samples per lane (windows up to 1215 samples),
// the sample-pair code path.
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_SEARCH(38)
NSFRB_INSTANTIATE_PIPE(38, 0)
}  // namespace nsfrb
