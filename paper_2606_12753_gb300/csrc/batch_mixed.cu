// Persistent batch-kernel instantiations and launchers for the mixed form.
#include "batch.cuh"

namespace mhd {

#define MHD_BATCH_TILES(X) X(16, 8) X(8, 8)

cudaError_t batch_launch_mixed(int tx, int ty, unsigned grid, size_t smem, cudaStream_t st, const BatchArgs& ba) {
#define X(TXv, TYv)                                                                          \
  if (tx == TXv && ty == TYv) {                                                              \
    cudaLaunchConfig_t cfg = {};                                                             \
    cfg.gridDim = dim3(grid);                                                                \
    cfg.blockDim = dim3(256);                                                                \
    cfg.dynamicSmemBytes = smem;                                                             \
    cfg.stream = st;                                                                         \
    cudaLaunchAttribute attr[1];                                                             \
    attr[0].id = cudaLaunchAttributeCooperative;                                             \
    attr[0].val.cooperative = 1;                                                             \
    cfg.attrs = attr;                                                                        \
    cfg.numAttrs = 1;                                                                        \
    return cudaLaunchKernelEx(&cfg, batch_kernel<P_MIXED, TXv, TYv>, ba);                    \
  }
  MHD_BATCH_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t batch_set_smem_mixed(int tx, int ty, size_t bytes) {
#define X(TXv, TYv)                                                                                    \
  if (tx == TXv && ty == TYv)                                                                          \
    return cudaFuncSetAttribute(batch_kernel<P_MIXED, TXv, TYv>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                (int)bytes);
  MHD_BATCH_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

int batch_max_blocks_mixed(int tx, int ty, size_t smem) {
  int n = 0;
#define X(TXv, TYv) \
  if (tx == TXv && ty == TYv) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<P_MIXED, TXv, TYv>, 256, smem);
  MHD_BATCH_TILES(X)
#undef X
  return n;
}

}  // namespace mhd
