// Level-0 SDIRK step kernel, FP64 instantiations, shared-memory size and the
// cluster co-scheduling query (the kernel itself is in sdirk_kernel.cuh).
#include "sdirk_kernel.cuh"

namespace mg {

size_t sdirk_smem_bytes(int npc, int P, int nthr, int nslots, int elem) {
  (void)npc;
  const size_t npad = (size_t)nthr * (size_t)(P + 1);
  return (((size_t)nslots * npad * (size_t)elem + 15) & ~(size_t)15) + ((104 * (size_t)elem + 15) & ~(size_t)15) +
         32 * sizeof(double);
}

int launch_sdirk(const SdirkParams<double>& p, cudaStream_t st) { return launch_sdirk_any(p, st); }

int sdirk_max_cluster(int want, size_t smem, int nthr) {
  configure_sdirk<double, 16, 6>();
  for (int c = want; c >= 1; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c);
    cfg.blockDim = dim3((unsigned)nthr);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, sdirk_kernel<double, 16, 6>, &cfg) == cudaSuccess && nc > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

}  // namespace mg
