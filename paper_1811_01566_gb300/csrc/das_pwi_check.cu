// Tiled DAS launchers for PWI, bounds-checked variants (all RF types, tile configurations
// and staging paths), instantiated in their own translation unit so the
// kernel variants compile in parallel.
#include "das_kernels.cuh"

namespace wf {
template wf_status launch_das_tiled<1, true>(DasArgs&, const Plan&, int, wf_dtype, cudaStream_t);
}  // namespace wf
