// Level-0 SDIRK steps with per-thread segments (FP64): instantiations for the
// odd upwind orders p = 1, 3, 5 (recurrence orders (1, 0), (2, 1), (3, 2),
// each split into cascaded sections) and the launch (the kernel itself is in
// sdirk_seg.cuh).
#include "sdirk_seg.cuh"

namespace mg {

size_t sdirk_seg_smem_bytes(int n) {
  const size_t T = (size_t)n / kSegPoints;
  return T * (kSegPoints + 2) * sizeof(double) + 32 * sizeof(double);
}

template <int ST, int C1, int C2, int A1, int A2>
static int launch_seg_t(const SdirkSegParams& p, cudaStream_t st) {
  static std::mutex mu;
  static uint64_t done = 0;
  once_per_device(mu, done, [] {
    cudaFuncSetAttribute(sdirk_seg_kernel<ST, C1, C2, A1, A2, kSegPoints>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (p.K <= 0) return 1;
  const size_t smem = sdirk_seg_smem_bytes(p.n);
  sdirk_seg_kernel<ST, C1, C2, A1, A2, kSegPoints><<<(unsigned)p.K, (unsigned)p.T, smem, st>>>(p);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <int ST>
static int launch_seg_s(const SdirkSegParams& p, cudaStream_t st) {
  // section orders of the odd upwind orders: p = 5 (causal 1 + 2, anticausal
  // two real roots or a complex pair), p = 3 (causal two real roots or a
  // complex pair, anticausal 1), p = 1 (causal 1)
  switch (p.c1 * 1000 + p.c2 * 100 + p.a1 * 10 + p.a2) {
    case 1211:
      return launch_seg_t<ST, 1, 2, 1, 1>(p, st);
    case 1202:
      return launch_seg_t<ST, 1, 2, 0, 2>(p, st);
    case 1110:
      return launch_seg_t<ST, 1, 1, 1, 0>(p, st);
    case 210:
      return launch_seg_t<ST, 0, 2, 1, 0>(p, st);
    case 1000:
      return launch_seg_t<ST, 1, 0, 0, 0>(p, st);
    default:
      return -1;
  }
}

int launch_sdirk_seg(const SdirkSegParams& p, cudaStream_t st) {
  auto bad_len = [](int w1, int w2) { return w1 < 0 || w2 < 0 || w2 > w1 || w1 > kSegPoints || (w1 & 7) || (w2 & 7); };
  if (p.T < 1 || p.T > 128 || (int64_t)p.T * kSegPoints != p.n || bad_len(p.rc1, p.rc2) || bad_len(p.ra1, p.ra2))
    return -1;
  if (p.stages == 1) return launch_seg_s<1>(p, st);
  if (p.stages == 3) return launch_seg_s<3>(p, st);
  return -1;  // two stages: no odd-p pairing uses SDIRK2
}

}  // namespace mg
