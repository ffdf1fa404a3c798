// FP32 stage kernel of MIXED inner cycles with per-thread segments:
// instantiations for the odd upwind orders p = 1, 3, 5 and the launch (the
// kernel itself is in sdirk_seg32.cuh).
#include "sdirk_seg32.cuh"

namespace mg {

size_t sdirk_seg32_smem_bytes(int n) {
  const size_t T = (size_t)n / kSeg32Points;
  return 3 * T * (kSeg32Points + 4) * sizeof(float) + 32 * sizeof(double);
}

template <int ST, int C1, int C2, int A1, int A2, int HL, int HR>
static int launch_seg32_t(const SdirkSeg32Params& p, cudaStream_t st) {
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(sdirk_seg32_kernel<ST, C1, C2, A1, A2, HL, HR, kSeg32Points>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (p.K <= 0) return 1;
  const size_t smem = sdirk_seg32_smem_bytes(p.n);
  sdirk_seg32_kernel<ST, C1, C2, A1, A2, HL, HR, kSeg32Points><<<(unsigned)p.K, (unsigned)p.T, smem, st>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <int ST>
static int launch_seg32_s(const SdirkSeg32Params& p, cudaStream_t st) {
  switch (p.c1 * 1000 + p.c2 * 100 + p.a1 * 10 + p.a2) {
    case 1211:  // p = 5
      return launch_seg32_t<ST, 1, 2, 1, 1, 3, 2>(p, st);
    case 1202:
      return launch_seg32_t<ST, 1, 2, 0, 2, 3, 2>(p, st);
    case 1110:  // p = 3
      return launch_seg32_t<ST, 1, 1, 1, 0, 2, 1>(p, st);
    case 210:
      return launch_seg32_t<ST, 0, 2, 1, 0, 2, 1>(p, st);
    case 1000:  // p = 1
      return launch_seg32_t<ST, 1, 0, 0, 0, 1, 0>(p, st);
    default:
      return -1;
  }
}

int launch_sdirk_seg32(const SdirkSeg32Params& p, cudaStream_t st) {
  auto bad_len = [](int w1, int w2) {
    return w1 < 0 || w2 < 0 || w2 > w1 || w1 > kSeg32Points || (w1 & 7) || (w2 & 7);
  };
  if (p.T < 32 || p.T > 256 || (int64_t)p.T * kSeg32Points != p.n || bad_len(p.rc1, p.rc2) ||
      bad_len(p.ra1, p.ra2))
    return -1;
  if (p.stages == 1) return launch_seg32_s<1>(p, st);
  if (p.stages == 3) return launch_seg32_s<3>(p, st);
  return -1;
}

}  // namespace mg
