// Coarse-level step kernel, FP32 storage and SL gather with an FP32
// correction solve (MIXED inner cycles).
#include "coarse_kernel.cuh"

namespace mg {

int launch_coarse(const CoarseParams<float>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

}  // namespace mg
