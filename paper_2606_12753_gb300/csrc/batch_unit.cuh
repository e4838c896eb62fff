// Persistent batch-kernel instantiations and launchers of one precision.
// Included once by each per-precision translation unit, which defines:
//   MHD_UNIT_PREC           P_FP64, P_MIXED or P_FP32
//   MHD_UNIT_FN(name)       name##_fp64, name##_mixed or name##_fp32
//   MHD_BATCH_TILES(X)      the tiles the batch kernel is instantiated for, X(TX, TY)
#include "batch.cuh"

namespace mhd {

cudaError_t MHD_UNIT_FN(batch_launch)(int tx, int ty, unsigned grid, size_t smem, cudaStream_t st,
                                      const BatchArgs& ba) {
#define X(TXv, TYv)                                                                 \
  if (tx == TXv && ty == TYv) {                                                     \
    cudaLaunchConfig_t cfg = {};                                                    \
    cfg.gridDim = dim3(grid);                                                       \
    cfg.blockDim = dim3(256);                                                       \
    cfg.dynamicSmemBytes = smem;                                                    \
    cfg.stream = st;                                                                \
    cudaLaunchAttribute attr[1];                                                    \
    attr[0].id = cudaLaunchAttributeCooperative;                                    \
    attr[0].val.cooperative = 1;                                                    \
    cfg.attrs = attr;                                                               \
    cfg.numAttrs = 1;                                                               \
    return cudaLaunchKernelEx(&cfg, batch_kernel<MHD_UNIT_PREC, TXv, TYv>, ba);     \
  }
  MHD_BATCH_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t MHD_UNIT_FN(batch_set_smem)(int tx, int ty, size_t bytes) {
#define X(TXv, TYv)                                                                            \
  if (tx == TXv && ty == TYv)                                                                  \
    return cudaFuncSetAttribute(batch_kernel<MHD_UNIT_PREC, TXv, TYv>,                         \
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  MHD_BATCH_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

// dynamic shared memory of the batch kernel of a tile (the plain stage layout
// with the unpadded ring and, without a slope phase, the tile's item list;
// 0: not instantiated)
size_t MHD_UNIT_FN(batch_smem_bytes)(int tx, int ty) {
  using R = Prec<MHD_UNIT_PREC>::R;
  using S = Prec<MHD_UNIT_PREC>::S;
#define X(TXv, TYv)                                                                                      \
  if (tx == TXv && ty == TYv)                                                                            \
    return Tile<TXv, TYv, ring_xo<MHD_UNIT_PREC, FM_PLAIN, false>()>::bytes<                             \
        R, S, slopes_in_smem<MHD_UNIT_PREC, FM_PLAIN, TXv, TYv>(),                                       \
        compact_items<MHD_UNIT_PREC, FM_PLAIN, false, TXv, TYv>()>();
  MHD_BATCH_TILES(X)
#undef X
  return 0;
}

int MHD_UNIT_FN(batch_max_blocks)(int tx, int ty, size_t smem) {
  int n = 0;
#define X(TXv, TYv)                                                                                         \
  if (tx == TXv && ty == TYv)                                                                               \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<MHD_UNIT_PREC, TXv, TYv>, 256, smem);
  MHD_BATCH_TILES(X)
#undef X
  return n;
}

}  // namespace mhd
