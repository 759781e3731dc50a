// Barrier-free search kernels for chunks of 38 samples per lane with F16 rows read in
// place (every pixel x DM tile), in a translation unit of their own for a parallel build.
#include "search_impl.cuh"

namespace nsfrb {
NSFRB_INSTANTIATE_PIPE(38, 2)
}  // namespace nsfrb
