// Stage-kernel instantiations and launchers for the mixed form.
#include "stage_impl.cuh"

namespace mhd {

#define MHD_TILES(X) X(16, 8) X(16, 16) X(32, 8) X(24, 8) X(8, 8)

cudaError_t launch_stage_mixed(int stage, int tx, int ty, unsigned nblocks, size_t smem, cudaStream_t st,
                                 const Geo& g, const StageArgs& args) {
#define X(TXv, TYv)                                                                              \
  if (tx == TXv && ty == TYv) {                                                                  \
    if (stage == 1) stage_kernel<P_MIXED, 1, TXv, TYv><<<nblocks, stage_threads<P_MIXED, TXv, TYv>(), smem, st>>>(g, args);     \
    else stage_kernel<P_MIXED, 2, TXv, TYv><<<nblocks, stage_threads<P_MIXED, TXv, TYv>(), smem, st>>>(g, args);                \
    return cudaGetLastError();                                                                   \
  }
  MHD_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t set_smem_mixed(int tx, int ty, size_t bytes) {
#define X(TXv, TYv)                                                                                        \
  if (tx == TXv && ty == TYv) {                                                                            \
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<P_MIXED, 1, TXv, TYv>,                              \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);         \
    if (e == cudaSuccess)                                                                                  \
      e = cudaFuncSetAttribute(stage_kernel<P_MIXED, 2, TXv, TYv>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)bytes);                                                                \
    return e;                                                                                              \
  }
  MHD_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

size_t smem_bytes_mixed(int tx, int ty) {
  using R = Prec<P_MIXED>::R;
  using S = Prec<P_MIXED>::S;
#define X(TXv, TYv) \
  if (tx == TXv && ty == TYv) return Tile<TXv, TYv>::bytes<R, S, slopes_in_smem<P_MIXED, FM_PLAIN, TXv, TYv>()>();
  MHD_TILES(X)
#undef X
  return 0;
}

// characteristic reconstruction (16 x 8 tile) keeps its slopes in shared memory
size_t smem_bytes_char_mixed() { return Tile<16, 8>::bytes<Prec<P_MIXED>::R, Prec<P_MIXED>::S, true>(); }

cudaError_t launch_prims_mixed(unsigned nblocks, cudaStream_t st, const Geo& g, const StageArgs& args) {
  (void)nblocks;   // one CTA per (j, k) row of cells
  prims_kernel<P_MIXED><<<(unsigned)((long long)g.n[1] * g.n[2]), 128, 0, st>>>(g, args);
  return cudaGetLastError();
}

// The learned HLL/HLLD switch is instantiated for the 16 x 8 tile only.
cudaError_t launch_stage_learned_mixed(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                                   const StageArgs& args) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  if (stage == 1) stage_kernel_learned<P_MIXED, 1, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else stage_kernel_learned<P_MIXED, 2, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  return cudaGetLastError();
}

cudaError_t set_smem_learned_mixed(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel_learned<P_MIXED, 1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel_learned<P_MIXED, 2, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  return e;
}

// SSP-RK3 stages (ids 3, 4, 5) are instantiated for the 16 x 8 tile only.
cudaError_t launch_stage_rk3_mixed(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                                const StageArgs& args) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  if (stage == ST_RK3_1) stage_kernel<P_MIXED, ST_RK3_1, 16, 8><<<nblocks, stage_threads<P_MIXED, 16, 8>(), smem, st>>>(g, args);
  else if (stage == ST_RK3_2) stage_kernel<P_MIXED, ST_RK3_2, 16, 8><<<nblocks, stage_threads<P_MIXED, 16, 8>(), smem, st>>>(g, args);
  else if (stage == ST_RK3_3) stage_kernel<P_MIXED, ST_RK3_3, 16, 8><<<nblocks, stage_threads<P_MIXED, 16, 8>(), smem, st>>>(g, args);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t set_smem_rk3_mixed(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<P_MIXED, ST_RK3_1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel<P_MIXED, ST_RK3_2, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel<P_MIXED, ST_RK3_3, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  return e;
}

// Characteristic reconstruction (RK2 stages, 16 x 8 tile).
cudaError_t launch_stage_char_mixed(int stage, unsigned nblocks, size_t smem, cudaStream_t st, const Geo& g,
                                 const StageArgs& args) {
  if (g.TX != 16 || g.TY != 8) return cudaErrorInvalidValue;
  if (stage == 1) stage_kernel_char<P_MIXED, 1, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else if (stage == 2) stage_kernel_char<P_MIXED, 2, 16, 8><<<nblocks, 256, smem, st>>>(g, args);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t set_smem_char_mixed(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel_char<P_MIXED, 1, 16, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stage_kernel_char<P_MIXED, 2, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  return e;
}

}  // namespace mhd
