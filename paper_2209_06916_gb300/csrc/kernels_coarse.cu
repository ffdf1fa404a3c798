// Coarse-level step kernel, FP64 instantiations, shared-memory size and the
// cluster co-scheduling query (the kernel itself is in coarse_kernel.cuh).
#include "coarse_kernel.cuh"

namespace mg {

size_t coarse_smem_bytes(int npc, int P, int nthr, int elem, int gm_elem) {
  // slots of `elem` bytes; scan buffers budgeted at 8 bytes (FP64 solve);
  // GMRES: the Krylov vector's halo buffer and the reduction area
  (void)npc;
  const size_t npad = (size_t)nthr * (size_t)(P + 1);
  size_t b = ((3 * npad * (size_t)elem + 15) & ~(size_t)15) + ((104 * 8 + 15) & ~(size_t)15) + 32 * sizeof(double);
  if (gm_elem > 0) b += ((npad * (size_t)gm_elem + 15) & ~(size_t)15) + (size_t)kGmSharedDoubles * sizeof(double);
  return b;
}

int launch_coarse(const CoarseParams<double>& p, cudaStream_t st) { return launch_coarse_any(p, st); }

// Largest cluster size <= want (power of two) that can be co-scheduled.
int coarse_max_cluster(int want, size_t smem, int nthr) {
  configure_coarse<double, double, 16, 4, false>();
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
    if (cudaOccupancyMaxActiveClusters(&nc, coarse_kernel<double, double, 16, 4, false>, &cfg) == cudaSuccess && nc > 0)
      return c;
    cudaGetLastError();
  }
  return 1;
}

}  // namespace mg
