// Level-0 SDIRK step kernel, FP32 instantiations (MIXED inner cycles).
#include "sdirk_kernel.cuh"

namespace mg {

int launch_sdirk(const SdirkParams<float>& p, cudaStream_t st) { return launch_sdirk_any(p, st); }

}  // namespace mg
