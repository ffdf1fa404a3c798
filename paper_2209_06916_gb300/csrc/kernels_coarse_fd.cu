// Coarse-level step kernel, FP32 storage and SL gather with an FP64
// correction solve (MIXED inner cycles on ill-conditioned levels).
#include "coarse_kernel.cuh"

namespace mg {

int launch_coarse(const CoarseParams<float, double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

}  // namespace mg
