// Stage-kernel instantiations and launchers of one precision.  Included once
// by each per-precision translation unit, which defines:
//   MHD_UNIT_PREC      P_FP64, P_MIXED or P_FP32
//   MHD_UNIT_FN(name)  name##_fp64, name##_mixed or name##_fp32
//   MHD_TILES(X)       the tiles the plain kernel is instantiated for, X(TX, TY)
#include "stage_impl.cuh"

namespace mhd {

cudaError_t MHD_UNIT_FN(launch_stage)(int stage, int tx, int ty, unsigned nblocks, size_t smem, cudaStream_t st,
                                      const Geo& g, const StageArgs& args, const TmaMaps& tm) {
#define X(TXv, TYv)                                                                                      \
  if (tx == TXv && ty == TYv) {                                                                          \
    constexpr int nt = stage_threads<MHD_UNIT_PREC, TXv, TYv>();                                         \
    if (stage == 1) stage_kernel<MHD_UNIT_PREC, 1, TXv, TYv><<<nblocks, nt, smem, st>>>(g, args, tm);    \
    else stage_kernel<MHD_UNIT_PREC, 2, TXv, TYv><<<nblocks, nt, smem, st>>>(g, args, tm);               \
    return cudaGetLastError();                                                                           \
  }
  MHD_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t MHD_UNIT_FN(set_smem)(int tx, int ty, size_t bytes) {
#define X(TXv, TYv)                                                                                      \
  if (tx == TXv && ty == TYv) {                                                                          \
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<MHD_UNIT_PREC, 1, TXv, TYv>,                       \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);       \
    if (e == cudaSuccess)                                                                                \
      e = cudaFuncSetAttribute(stage_kernel<MHD_UNIT_PREC, 2, TXv, TYv>,                                 \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);                 \
    return e;                                                                                            \
  }
  MHD_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

// dynamic shared memory of the plain kernel of a tile (0: not instantiated)
size_t MHD_UNIT_FN(smem_bytes)(int tx, int ty) {
  using R = Prec<MHD_UNIT_PREC>::R;
  using S = Prec<MHD_UNIT_PREC>::S;
#define X(TXv, TYv)                                                                                      \
  if (tx == TXv && ty == TYv)                                                                            \
    return Tile<TXv, TYv, ring_xo<MHD_UNIT_PREC, FM_PLAIN, true>()>::bytes<                              \
        R, S, slopes_in_smem<MHD_UNIT_PREC, FM_PLAIN, TXv, TYv>()>();
  MHD_TILES(X)
#undef X
  return 0;
}

// characteristic reconstruction (16 x 8 tile) keeps its slopes in shared memory
size_t MHD_UNIT_FN(smem_bytes_char)() {
  return Tile<16, 8, ring_xo<MHD_UNIT_PREC, FM_CHAR, true>()>::bytes<Prec<MHD_UNIT_PREC>::R, Prec<MHD_UNIT_PREC>::S,
                                                               true>();
}

// the learned switch (16 x 8 tile) queues its face items in shared memory
size_t MHD_UNIT_FN(smem_bytes_learned)() {
  return Tile<16, 8, ring_xo<MHD_UNIT_PREC, FM_LEARNED, true>()>::bytes<Prec<MHD_UNIT_PREC>::R,
                                                                  Prec<MHD_UNIT_PREC>::S, false, true>();
}

cudaError_t MHD_UNIT_FN(launch_prims)(unsigned nblocks, cudaStream_t st, const Geo& g, const StageArgs& args) {
  (void)nblocks;   // one CTA per (j, k) row of cells
  prims_kernel<MHD_UNIT_PREC><<<(unsigned)((long long)g.n[1] * g.n[2]), 128, 0, st>>>(g, args);
  return cudaGetLastError();
}

// The learned HLL/HLLD switch is instantiated for the 16 x 8 tile only.
cudaError_t MHD_UNIT_FN(launch_stage_learned)(int stage, unsigned nblocks, size_t smem, cudaStream_t st,
                                              const Geo& g, const StageArgs& args) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  if (stage == 1) stage_kernel_learned<MHD_UNIT_PREC, 1, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else stage_kernel_learned<MHD_UNIT_PREC, 2, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  return cudaGetLastError();
}

cudaError_t MHD_UNIT_FN(set_smem_learned)(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel_learned<MHD_UNIT_PREC, 1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel_learned<MHD_UNIT_PREC, 2, 16, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

// SSP-RK3 stages (ids 3, 4, 5) are instantiated for the 16 x 8 tile only.
cudaError_t MHD_UNIT_FN(launch_stage_rk3)(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                                          const StageArgs& args, const TmaMaps& tm) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  constexpr int nt = stage_threads<MHD_UNIT_PREC, 16, 8>();
  if (stage == ST_RK3_1) stage_kernel<MHD_UNIT_PREC, ST_RK3_1, 16, 8><<<nblocks, nt, smem, st>>>(g, args, tm);
  else if (stage == ST_RK3_2) stage_kernel<MHD_UNIT_PREC, ST_RK3_2, 16, 8><<<nblocks, nt, smem, st>>>(g, args, tm);
  else if (stage == ST_RK3_3) stage_kernel<MHD_UNIT_PREC, ST_RK3_3, 16, 8><<<nblocks, nt, smem, st>>>(g, args, tm);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t MHD_UNIT_FN(set_smem_rk3)(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<MHD_UNIT_PREC, ST_RK3_1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel<MHD_UNIT_PREC, ST_RK3_2, 16, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel<MHD_UNIT_PREC, ST_RK3_3, 16, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

// Characteristic reconstruction (RK2 stages, 16 x 8 tile).
cudaError_t MHD_UNIT_FN(launch_stage_char)(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                                           const StageArgs& args) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  if (stage == 1) stage_kernel_char<MHD_UNIT_PREC, 1, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else if (stage == 2) stage_kernel_char<MHD_UNIT_PREC, 2, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t MHD_UNIT_FN(set_smem_char)(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel_char<MHD_UNIT_PREC, 1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel_char<MHD_UNIT_PREC, 2, 16, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

}  // namespace mhd
