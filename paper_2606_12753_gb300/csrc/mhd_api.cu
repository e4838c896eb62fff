// C ABI of the MHD hot path: handle, device buffers, launches, reductions.
#include <cuda.h>   // tensor-map types; the encoder itself is fetched from the driver at run time
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // header-only ranges; no cost unless a profiler is attached
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/mhd_gb300.h"
#include "batch.cuh"

namespace mhd {
cudaError_t launch_stage_fp64(int, int, int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&,
                                const TmaMaps&);
cudaError_t launch_stage_mixed(int, int, int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&,
                                const TmaMaps&);
cudaError_t launch_stage_fp32(int, int, int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&,
                                const TmaMaps&);
cudaError_t set_smem_fp64(int, int, size_t);
cudaError_t set_smem_mixed(int, int, size_t);
cudaError_t set_smem_fp32(int, int, size_t);
size_t smem_bytes_fp64(int, int);
size_t smem_bytes_mixed(int, int);
size_t smem_bytes_fp32(int, int);
size_t smem_bytes_char_fp64();
size_t smem_bytes_learned_fp64();
size_t smem_bytes_char_mixed();
size_t smem_bytes_learned_mixed();
size_t smem_bytes_char_fp32();
size_t smem_bytes_learned_fp32();
cudaError_t launch_stage_learned_fp64(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_stage_learned_mixed(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_stage_learned_fp32(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_stage_rk3_fp64(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&, const TmaMaps&);
cudaError_t launch_stage_rk3_mixed(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&, const TmaMaps&);
cudaError_t launch_stage_rk3_fp32(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&, const TmaMaps&);
cudaError_t set_smem_rk3_fp64(size_t);
cudaError_t set_smem_rk3_mixed(size_t);
cudaError_t set_smem_rk3_fp32(size_t);
cudaError_t launch_stage_char_fp64(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_stage_char_mixed(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_stage_char_fp32(int, unsigned, size_t, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t set_smem_char_fp64(size_t);
cudaError_t set_smem_char_mixed(size_t);
cudaError_t set_smem_char_fp32(size_t);
cudaError_t set_smem_learned_fp64(size_t);
cudaError_t set_smem_learned_mixed(size_t);
cudaError_t set_smem_learned_fp32(size_t);
cudaError_t launch_prims_fp64(unsigned, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_prims_mixed(unsigned, cudaStream_t, const Geo&, const StageArgs&);
cudaError_t launch_prims_fp32(unsigned, cudaStream_t, const Geo&, const StageArgs&);

cudaError_t launch_stage(int prec, int stage, int tx, int ty, unsigned nb, size_t smem, cudaStream_t st,
                         const Geo& g, const StageArgs& a, const TmaMaps* tm) {
  static const TmaMaps no_tma = {};
  const TmaMaps& maps = tm ? *tm : no_tma;
  if (stage >= ST_RK3_1) {
    switch (prec) {
      case P_FP64: return launch_stage_rk3_fp64(stage, nb, smem, st, g, a, maps);
      case P_MIXED: return launch_stage_rk3_mixed(stage, nb, smem, st, g, a, maps);
      default: return launch_stage_rk3_fp32(stage, nb, smem, st, g, a, maps);
    }
  }
  if (g.recon == 1) {
    switch (prec) {
      case P_FP64: return launch_stage_char_fp64(stage, nb, smem, st, g, a);
      case P_MIXED: return launch_stage_char_mixed(stage, nb, smem, st, g, a);
      default: return launch_stage_char_fp32(stage, nb, smem, st, g, a);
    }
  }
  if (g.riemann == 2) {
    // learned switch: needs the network; 16 x 8 tile only
    if (!a.mlp) return cudaErrorInvalidValue;
    switch (prec) {
      case P_FP64: return launch_stage_learned_fp64(stage, nb, smem, st, g, a);
      case P_MIXED: return launch_stage_learned_mixed(stage, nb, smem, st, g, a);
      default: return launch_stage_learned_fp32(stage, nb, smem, st, g, a);
    }
  }
  switch (prec) {
    case P_FP64: return launch_stage_fp64(stage, tx, ty, nb, smem, st, g, a, maps);
    case P_MIXED: return launch_stage_mixed(stage, tx, ty, nb, smem, st, g, a, maps);
    default: return launch_stage_fp32(stage, tx, ty, nb, smem, st, g, a, maps);
  }
}
cudaError_t launch_prims(int prec, unsigned nb, cudaStream_t st, const Geo& g, const StageArgs& a) {
  switch (prec) {
    case P_FP64: return launch_prims_fp64(nb, st, g, a);
    case P_MIXED: return launch_prims_mixed(nb, st, g, a);
    default: return launch_prims_fp32(nb, st, g, a);
  }
}
cudaError_t stage_set_smem_char(int prec, size_t bytes) {
  switch (prec) {
    case P_FP64: return set_smem_char_fp64(bytes);
    case P_MIXED: return set_smem_char_mixed(bytes);
    default: return set_smem_char_fp32(bytes);
  }
}
cudaError_t stage_set_smem_rk3(int prec, size_t bytes) {
  switch (prec) {
    case P_FP64: return set_smem_rk3_fp64(bytes);
    case P_MIXED: return set_smem_rk3_mixed(bytes);
    default: return set_smem_rk3_fp32(bytes);
  }
}
cudaError_t stage_set_smem_learned(int prec, size_t bytes) {
  switch (prec) {
    case P_FP64: return set_smem_learned_fp64(bytes);
    case P_MIXED: return set_smem_learned_mixed(bytes);
    default: return set_smem_learned_fp32(bytes);
  }
}
cudaError_t stage_set_smem(int prec, int tx, int ty, size_t bytes) {
  switch (prec) {
    case P_FP64: return set_smem_fp64(tx, ty, bytes);
    case P_MIXED: return set_smem_mixed(tx, ty, bytes);
    default: return set_smem_fp32(tx, ty, bytes);
  }
}
size_t stage_smem_bytes(int prec, int tx, int ty) {
  switch (prec) {
    case P_FP64: return smem_bytes_fp64(tx, ty);
    case P_MIXED: return smem_bytes_mixed(tx, ty);
    default: return smem_bytes_fp32(tx, ty);
  }
}
bool stage_tile_supported(int prec, int tx, int ty) { return stage_smem_bytes(prec, tx, ty) > 0; }

// Dynamic shared memory of the kernels a configuration launches: the
// characteristic-reconstruction kernels also hold per-cell slopes, the
// learned switch its face queue (and both keep the unpadded ring).
static size_t config_smem_bytes(int prec, int recon, int riemann, int tx, int ty) {
  if (recon == MHD_RECON_CHARACTERISTIC) {
    switch (prec) {
      case P_FP64: return smem_bytes_char_fp64();
      case P_MIXED: return smem_bytes_char_mixed();
      default: return smem_bytes_char_fp32();
    }
  }
  if (riemann == MHD_LEARNED) {
    // the learned kernel and the plain one (the rhs and dump paths) share the handle's size
    size_t l;
    switch (prec) {
      case P_FP64: l = smem_bytes_learned_fp64(); break;
      case P_MIXED: l = smem_bytes_learned_mixed(); break;
      default: l = smem_bytes_learned_fp32(); break;
    }
    const size_t p = stage_smem_bytes(prec, tx, ty);
    return l > p ? l : p;
  }
  return stage_smem_bytes(prec, tx, ty);
}
}  // namespace mhd

using namespace mhd;

struct mhd_handle {
  mhd_config cfg;
  Geo geo;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t elem = 8;          // bytes per state element
  size_t kelem = 8;         // bytes per stage-1 element
  size_t welem = 8;         // bytes per primitive element
  void* U[2] = {nullptr, nullptr};
  void* K1 = nullptr;
  void* Urk[2] = {nullptr, nullptr};        // RK3: the intermediate states U1, U2
  void* W[2] = {nullptr, nullptr};
  unsigned long long* words = nullptr;     // [0,1] CFL words (step parity), [2] reductions, [3] status,
                                           // [4] scratch, [8..] counters
  unsigned int* status = nullptr;
  unsigned long long* counters = nullptr;
  void* pinned = nullptr;                  // host readback buffer
  int cur = 0;                             // U[cur], W[cur] hold the current state
  int parity = 0;                          // words[parity] = CFL max of the current state
  bool prims_valid = false;                // W[cur] and words[parity] match U[cur]
  size_t smem_bytes = 0;
  double last_dt = 0.0;
  int steps = 0;
  bool profiling = false;
  void* mlp = nullptr;                     // copy of the switch network (device)
  float mlp_zt = 0.0f;                     // logit of the switch threshold tau
  std::vector<cudaEvent_t> ev_pool;        // 3 events per recorded step
  size_t ev_used = 0;
  std::string err;
  // host streaming (mhd_stream_step): the state buffers the handle owns (the
  // U pointers rotate over them), the two input slots, the copy streams and
  // the events that order slot reuse between the three streams
  std::vector<void*> owned_states;
  static constexpr int kSlots = 3;         // device states in flight per direction
  void* slot_in[kSlots] = {};
  void* slot_out[kSlots] = {};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_h2d[kSlots] = {}, ev_comp[kSlots] = {}, ev_d2h[kSlots] = {};
  long long nstream = 0;                   // streamed steps since the handle was created
  unsigned long long floors_seen = 0;      // floor hits already reported (MHD_FLOOR_ERROR)
  // TMA maps of the two primitive buffers (plain kernels with 4-byte
  // primitives); the W pointers swap every step, so each map keeps its base
  TmaMaps tmaps[2] = {};
  void* tmap_base[2] = {nullptr, nullptr};
};

// error text of calls without a handle, one per host thread (calls on
// different devices may run on several threads at once)
static thread_local std::string g_create_err;

static int fail(mhd_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_create_err = buf;
  return code;
}

#define CUDA_TRY(h, call)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail((h), MHD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

extern "C" void mhd_default_config(mhd_config* c, int nx, int ny, int nz) {
  memset(c, 0, sizeof *c);
  c->nx = nx; c->ny = ny; c->nz = nz;
  int m = nx > ny ? nx : ny;
  m = m > nz ? m : nz;
  c->dx = c->dy = c->dz = 1.0 / (m > 0 ? m : 1);
  c->gamma = 5.0 / 3.0;
  c->cfl = 0.4;
  c->precision = MHD_FP64;
  c->riemann = MHD_HLLD;
  c->emf = MHD_EMF_UPWIND;
  c->rho_floor = 1e-10;
  c->p_floor = 1e-10;
}

static void default_tile(int prec, int* tx, int* ty, int* tz) {
  if (prec == MHD_FP64) { *tx = 16; *ty = 8; *tz = 32; }
  else { *tx = 16; *ty = 8; *tz = 32; }
}

static void resolve_tile(const mhd_config* c, int* tx, int* ty, int* tz) {
  int dx, dy, dz;
  default_tile(c->precision, &dx, &dy, &dz);
  *tx = c->tile_x ? c->tile_x : dx;
  *ty = c->tile_y ? c->tile_y : dy;
  *tz = c->tile_z ? c->tile_z : dz;
}

static int validate(const mhd_config* c, mhd_handle* h) {
  if (!c) return fail(h, MHD_ERR_INVALID, "null config");
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return fail(h, MHD_ERR_INVALID, "grid must have >= 1 cell per axis");
  if ((long long)c->nx * c->ny * c->nz > (1LL << 33)) return fail(h, MHD_ERR_INVALID, "grid too large");
  int n[3] = {c->nx, c->ny, c->nz};
  double d[3] = {c->dx, c->dy, c->dz};
  for (int a = 0; a < 3; ++a) {
    if (c->bc[a] != MHD_BC_PERIODIC && c->bc[a] != MHD_BC_OUTFLOW)
      return fail(h, MHD_ERR_INVALID, "bc[%d] must be MHD_BC_PERIODIC or MHD_BC_OUTFLOW", a);
    if (c->bc[a] == MHD_BC_OUTFLOW && n[a] < 2) return fail(h, MHD_ERR_INVALID, "an outflow axis needs >= 2 cells");
    if (!(d[a] > 0.0)) return fail(h, MHD_ERR_INVALID, "cell sizes must be positive");
  }
  if (!(c->gamma > 1.0)) return fail(h, MHD_ERR_INVALID, "gamma must exceed 1");
  if (!(c->cfl > 0.0)) return fail(h, MHD_ERR_INVALID, "cfl must be positive");
  if (c->precision < MHD_FP64 || c->precision > MHD_FP32) return fail(h, MHD_ERR_INVALID, "unknown precision");
  if (c->riemann < MHD_HLLD || c->riemann > MHD_LEARNED) return fail(h, MHD_ERR_INVALID, "unknown riemann solver");
  if (c->emf != MHD_EMF_UPWIND && c->emf != MHD_EMF_MEAN) return fail(h, MHD_ERR_INVALID, "unknown emf mode");
  if (!(c->rho_floor > 0.0) || !(c->p_floor > 0.0)) return fail(h, MHD_ERR_INVALID, "floors must be positive");
  if (c->tile_x < 0 || c->tile_y < 0 || c->tile_z < 0) return fail(h, MHD_ERR_INVALID, "tile sizes must be >= 0");
  int tx, ty, tz;
  resolve_tile(c, &tx, &ty, &tz);
  if (tz < 1 || tz > (1 << 20)) return fail(h, MHD_ERR_INVALID, "tile_z out of range");
  if (!stage_tile_supported(c->precision, tx, ty))
    return fail(h, MHD_ERR_INVALID, "tile %dx%d is not instantiated for this precision", tx, ty);
  if (c->riemann == MHD_LEARNED && (tx != 16 || ty != 8))
    return fail(h, MHD_ERR_INVALID, "the learned switch is instantiated for the 16x8 tile only (got %dx%d)", tx, ty);
  if (c->integrator != MHD_RK2 && c->integrator != MHD_RK3) return fail(h, MHD_ERR_INVALID, "unknown integrator");
  if (c->floor_policy != MHD_FLOOR_COUNT && c->floor_policy != MHD_FLOOR_ERROR)
    return fail(h, MHD_ERR_INVALID, "unknown floor policy");
  if (c->plane_copy != MHD_COPY_AUTO && c->plane_copy != MHD_COPY_GATHER)
    return fail(h, MHD_ERR_INVALID, "unknown plane copy mode");
  if (c->integrator == MHD_RK3 && (tx != 16 || ty != 8))
    return fail(h, MHD_ERR_INVALID, "SSP-RK3 is instantiated for the 16x8 tile only (got %dx%d)", tx, ty);
  if (c->integrator == MHD_RK3 && c->riemann == MHD_LEARNED)
    return fail(h, MHD_ERR_INVALID, "the learned switch runs with the RK2 integrator");
  if (c->recon != MHD_RECON_PRIMITIVE && c->recon != MHD_RECON_CHARACTERISTIC)
    return fail(h, MHD_ERR_INVALID, "unknown reconstruction");
  if (c->recon == MHD_RECON_CHARACTERISTIC &&
      (tx != 16 || ty != 8 || c->integrator != MHD_RK2 || c->riemann == MHD_LEARNED))
    return fail(h, MHD_ERR_INVALID, "characteristic reconstruction runs on the 16x8 tile with RK2 and HLLD or HLL");
  if (config_smem_bytes(c->precision, c->recon, c->riemann, tx, ty) > 227 * 1024)
    return fail(h, MHD_ERR_INVALID, "tile %dx%d needs %zu B of shared memory (> 227 KB)", tx, ty,
                config_smem_bytes(c->precision, c->recon, c->riemann, tx, ty));
  return MHD_OK;
}

static void fill_geo(const mhd_config* c, Geo* g) {
  memset(g, 0, sizeof *g);
  g->n[0] = c->nx; g->n[1] = c->ny; g->n[2] = c->nz;
  for (int a = 0; a < 3; ++a) {
    g->bc[a] = c->bc[a];
    g->nf[a] = g->n[a] + (c->bc[a] == MHD_BC_OUTFLOW ? 1 : 0);
  }
  g->inv_d[0] = 1.0 / c->dx; g->inv_d[1] = 1.0 / c->dy; g->inv_d[2] = 1.0 / c->dz;
  for (int a = 0; a < 3; ++a) g->finv_d[a] = (float)g->inv_d[a];
  g->gamma = c->gamma; g->rho_floor = c->rho_floor; g->p_floor = c->p_floor; g->cfl = c->cfl;
  g->emf_mean = c->emf == MHD_EMF_MEAN;
  g->riemann = c->riemann == MHD_HLL ? 1 : (c->riemann == MHD_LEARNED ? 2 : 0);
  g->recon = c->recon == MHD_RECON_CHARACTERISTIC ? 1 : 0;
  g->deadband = c->precision == MHD_FP64 ? 1e-10 : 1e-6;
  if (getenv("MHD_DEADBAND")) g->deadband = atof(getenv("MHD_DEADBAND"));
  g->gm1 = g->gamma - 1.0;
  g->fgamma = (float)g->gamma;
  g->fgm1 = (float)g->gm1;
  g->frho_floor = (float)g->rho_floor;
  g->fp_floor = (float)g->p_floor;
  g->fdeadband = (float)g->deadband;
  resolve_tile(c, &g->TX, &g->TY, &g->TZ);
  g->ntx = (g->n[0] + g->TX - 1) / g->TX;
  g->nty = (g->n[1] + g->TY - 1) / g->TY;
  g->nchunk = (g->n[2] + g->TZ - 1) / g->TZ;
  g->ncell = (long long)g->n[0] * g->n[1] * g->n[2];
  long long o = 5 * g->ncell;
  for (int a = 0; a < 3; ++a) {
    long long cnt = (long long)(a == 0 ? g->nf[0] : g->n[0]) * (a == 1 ? g->nf[1] : g->n[1]) *
                    (a == 2 ? g->nf[2] : g->n[2]);
    g->face_off[a] = o;
    o += cnt;
  }
  g->total = o;
}

// ---- TMA maps -----------------------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    cudaGetLastError();
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// Maps of one primitive buffer: 4D (x, y, z, array) over 11 arrays of n0 x
// n1 x n2 floats; the 8-primitive plane box and the 3-field lower-face box
// of a tile's ring (ring x-offset 4).  Left off (on = 0) where the form has
// no TMA path or the layout breaks a tensor-copy rule (rows of n0 floats
// must be multiples of 16 bytes).
static void build_tma_maps(const mhd_handle* h, void* wbuf, TmaMaps* out) {
  memset(out, 0, sizeof *out);
  const Geo& g = h->geo;
  const mhd_config& c = h->cfg;
  if (c.plane_copy != MHD_COPY_AUTO || c.precision == MHD_FP64 || c.recon != MHD_RECON_PRIMITIVE ||
      c.riemann == MHD_LEARNED)
    return;
  if (g.n[2] < 2 || g.n[0] % 4 != 0 || ((uintptr_t)wbuf & 15u)) return;
  const EncodeTiledFn encode = tensor_map_encoder();
  if (!encode) return;
  const cuuint32_t W = (cuuint32_t)(g.TX + 8), H = (cuuint32_t)(g.TY + 4);
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)NW};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4, (cuuint64_t)g.ncell * 4};
  const cuuint32_t box_p[4] = {W, H, 1, 8}, box_b[4] = {W, H - 2, 1, 3}, es[4] = {1, 1, 1, 1};
  const CUresult r1 = encode(reinterpret_cast<CUtensorMap*>(&out->p), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, wbuf, dims,
                             strides, box_p, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const CUresult r2 = encode(reinterpret_cast<CUtensorMap*>(&out->bn), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, wbuf, dims,
                             strides, box_b, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  out->on = r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

// the maps of the buffer a stage reads its primitives from, or null
static const TmaMaps* tma_for(const mhd_handle* h, const void* win) {
  for (int i = 0; i < 2; ++i)
    if (h->tmaps[i].on && h->tmap_base[i] == win) return &h->tmaps[i];
  return nullptr;
}

// NVTX range over one host entry point (seen by Nsight Systems as the call's
// span on the host timeline; the kernels it enqueues appear beneath it)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static long long face_count(const Geo& g, int d) {
  long long n[3] = {g.n[0], g.n[1], g.n[2]};
  n[d] = g.nf[d];
  return n[0] * n[1] * n[2];
}

extern "C" int mhd_create(const mhd_config* cfg, void* cuda_stream, mhd_handle** out) {
  if (!out) return fail(nullptr, MHD_ERR_INVALID, "null output pointer");
  int rc = validate(cfg, nullptr);
  if (rc) return rc;
  mhd_handle* h = new (std::nothrow) mhd_handle();
  if (!h) return fail(nullptr, MHD_ERR_NOMEM, "host allocation failed");
  h->cfg = *cfg;
  fill_geo(cfg, &h->geo);
  h->stream = (cudaStream_t)cuda_stream;
  h->elem = cfg->precision == MHD_FP32 ? 4 : 8;
  h->kelem = cfg->precision == MHD_FP64 ? 8 : 4;
  h->welem = cfg->precision == MHD_FP64 ? 8 : 4;
  h->smem_bytes = config_smem_bytes(cfg->precision, cfg->recon, cfg->riemann, h->geo.TX, h->geo.TY);
  cudaError_t e = cudaGetDevice(&h->device);
  const size_t bytes = (size_t)h->geo.total * h->elem;
  const size_t kbytes = (size_t)h->geo.total * h->kelem;
  const size_t wbytes = (size_t)h->geo.ncell * NW * h->welem;
  if (e == cudaSuccess) e = cudaMalloc(&h->U[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->U[1], bytes);
  h->owned_states = {h->U[0], h->U[1]};
  if (e == cudaSuccess) e = cudaMalloc(&h->K1, kbytes);
  if (e == cudaSuccess && cfg->integrator == MHD_RK3) e = cudaMalloc(&h->Urk[0], bytes);
  if (e == cudaSuccess && cfg->integrator == MHD_RK3) e = cudaMalloc(&h->Urk[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->W[0], wbytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->W[1], wbytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->words, 64 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 256);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MHD_ERR_NOMEM : MHD_ERR_CUDA;
    fail(nullptr, code, "device allocation of %zu B failed: %s", 2 * bytes + kbytes + 2 * wbytes,
         cudaGetErrorString(e));
    cudaGetLastError();
    mhd_destroy(h);
    return code;
  }
  h->status = (unsigned int*)(h->words + 3);
  h->counters = h->words + 8;
  for (int i = 0; i < 2; ++i) {
    h->tmap_base[i] = h->W[i];
    build_tma_maps(h, h->W[i], &h->tmaps[i]);
  }
  e = cudaMemsetAsync(h->words, 0, 64 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->U[0], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->K1, 0, kbytes, h->stream);
  if (e == cudaSuccess) e = stage_set_smem(cfg->precision, h->geo.TX, h->geo.TY, h->smem_bytes);
  if (e == cudaSuccess && cfg->riemann == MHD_LEARNED) e = stage_set_smem_learned(cfg->precision, h->smem_bytes);
  if (e == cudaSuccess && cfg->integrator == MHD_RK3) e = stage_set_smem_rk3(cfg->precision, h->smem_bytes);
  if (e == cudaSuccess && cfg->recon == MHD_RECON_CHARACTERISTIC)
    e = stage_set_smem_char(cfg->precision, h->smem_bytes);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    fail(nullptr, MHD_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
    cudaGetLastError();
    mhd_destroy(h);
    return MHD_ERR_CUDA;
  }
  *out = h;
  return MHD_OK;
}

extern "C" void mhd_destroy(mhd_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  if (h->s_in) cudaStreamSynchronize(h->s_in);
  if (h->s_out) cudaStreamSynchronize(h->s_out);
  for (void* p : h->owned_states) cudaFree(p);
  for (int p = 0; p < mhd_handle::kSlots; ++p) {
    if (h->ev_h2d[p]) cudaEventDestroy(h->ev_h2d[p]);
    if (h->ev_comp[p]) cudaEventDestroy(h->ev_comp[p]);
    if (h->ev_d2h[p]) cudaEventDestroy(h->ev_d2h[p]);
  }
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  cudaFree(h->K1);
  cudaFree(h->Urk[0]);
  cudaFree(h->Urk[1]);
  cudaFree(h->W[0]);
  cudaFree(h->W[1]);
  cudaFree(h->words);
  cudaFree(h->mlp);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

extern "C" const char* mhd_last_error(const mhd_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

static int copy_arrays(mhd_handle* h, bool in, char* base, size_t elem, void* const* cell, void* const* face,
                       int on_device) {
  if (!cell || !face) return fail(h, MHD_ERR_INVALID, "null state pointer array");
  for (int v = 0; v < 5; ++v)
    if (!cell[v]) return fail(h, MHD_ERR_INVALID, "null cell array %d", v);
  for (int d = 0; d < 3; ++d)
    if (!face[d]) return fail(h, MHD_ERR_INVALID, "null face array %d", d);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  for (int v = 0; v < 5; ++v) {
    char* dev = base + (size_t)v * h->geo.ncell * elem;
    size_t n = (size_t)h->geo.ncell * elem;
    CUDA_TRY(h, in ? cudaMemcpyAsync(dev, cell[v], n, kind, h->stream) : cudaMemcpyAsync(cell[v], dev, n, kind, h->stream));
  }
  for (int d = 0; d < 3; ++d) {
    char* dev = base + (size_t)h->geo.face_off[d] * elem;
    size_t n = (size_t)face_count(h->geo, d) * elem;
    CUDA_TRY(h, in ? cudaMemcpyAsync(dev, face[d], n, kind, h->stream) : cudaMemcpyAsync(face[d], dev, n, kind, h->stream));
  }
  if (!in || !on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MHD_OK;
}

extern "C" int mhd_set_state(mhd_handle* h, const void* const cell[5], const void* const face[3], int on_device) {
  if (!h) return MHD_ERR_INVALID;
  int rc = copy_arrays(h, true, (char*)h->U[h->cur], h->elem, (void* const*)cell, (void* const*)face, on_device);
  if (!rc) h->prims_valid = false;
  return rc;
}

extern "C" int mhd_get_state(mhd_handle* h, void* cell[5], void* face[3], int on_device) {
  if (!h) return MHD_ERR_INVALID;
  return copy_arrays(h, false, (char*)h->U[h->cur], h->elem, cell, face, on_device);
}

static cudaError_t record_event(mhd_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err) return err;
    h->ev_pool.push_back(e);
  }
  return cudaEventRecord(h->ev_pool[h->ev_used++], h->stream);
}

static StageArgs base_args(mhd_handle* h) {
  StageArgs a;
  memset(&a, 0, sizeof a);
  a.status = h->status;
  a.counters = h->counters;
  a.mlp = (const float*)h->mlp;
  a.mlp_zt = h->mlp_zt;
  return a;
}

// Primitives and CFL max of the current state (after set_state).
static cudaError_t ensure_prims(mhd_handle* h) {
  if (h->prims_valid) return cudaSuccess;
  StageArgs a = base_args(h);
  a.U = h->U[h->cur];
  a.Wout = h->W[h->cur];
  a.nextword = h->words + h->parity;
  cudaError_t e = cudaMemsetAsync(h->words + h->parity, 0, sizeof(unsigned long long), h->stream);
  if (e) return e;
  long long n = h->geo.ncell;
  unsigned nb = (unsigned)((n + 255) / 256);
  if (nb > 152u * 16u) nb = 152u * 16u;
  e = launch_prims(h->cfg.precision, nb, h->stream, h->geo, a);
  if (e) return e;
  h->prims_valid = true;
  return cudaSuccess;
}

// One SSP-RK3 step: three stage launches, U^n -> U1 -> U2 -> U^{n+1}.  The
// primitives alternate W[cur] -> W[cur^1] -> W[cur] -> W[cur^1], so W[cur^1]
// holds those of U^{n+1} when cur flips.
static cudaError_t launch_step_rk3(mhd_handle* h, double dt) {
  const Geo& g = h->geo;
  const unsigned nblocks = (unsigned)(g.ntx * g.nty * g.nchunk);
  const int prec = h->cfg.precision;
  StageArgs a = base_args(h);
  a.dt = dt;
  a.dtword = h->words + h->parity;
  a.nextword = h->words + (h->parity ^ 1);
  a.U = h->U[h->cur];
  void* in[3] = {h->U[h->cur], h->Urk[0], h->Urk[1]};
  void* outs[3] = {h->Urk[0], h->Urk[1], h->U[h->cur ^ 1]};
  void* win[3] = {h->W[h->cur], h->W[h->cur ^ 1], h->W[h->cur]};
  void* wout[3] = {h->W[h->cur ^ 1], h->W[h->cur], h->W[h->cur ^ 1]};
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 3; ++s) {
    a.Uin = in[s];
    a.Uout = outs[s];
    a.Win = win[s];
    a.Wout = wout[s];
    if (h->profiling && (e = record_event(h))) return e;
    e = launch_stage(prec, ST_RK3_1 + s, g.TX, g.TY, nblocks, h->smem_bytes, h->stream, g, a, tma_for(h, a.Win));
    if (e) return e;
  }
  if (h->profiling && (e = record_event(h))) return e;
  h->cur ^= 1;
  h->parity ^= 1;
  return cudaSuccess;
}

static cudaError_t launch_step(mhd_handle* h, double dt) {
  const Geo& g = h->geo;
  const unsigned nblocks = (unsigned)(g.ntx * g.nty * g.nchunk);
  const int prec = h->cfg.precision;
  cudaError_t e = ensure_prims(h);
  if (e) return e;
  if (h->cfg.integrator == MHD_RK3) return launch_step_rk3(h, dt);
  StageArgs a = base_args(h);
  a.dt = dt;
  a.dtword = h->words + h->parity;
  a.nextword = h->words + (h->parity ^ 1);
  a.U = h->U[h->cur];
  a.Win = h->W[h->cur];
  a.K1out = h->K1;
  a.Wout = h->W[h->cur ^ 1];
  if (h->profiling && (e = record_event(h))) return e;
  e = launch_stage(prec, 1, g.TX, g.TY, nblocks, h->smem_bytes, h->stream, g, a, tma_for(h, a.Win));
  if (e) return e;
  if (h->profiling && (e = record_event(h))) return e;
  a.K1 = h->K1;
  a.K1out = nullptr;
  a.Win = h->W[h->cur ^ 1];
  a.Wout = h->W[h->cur];     // W(U^n) is dead once stage 1 has read it
  a.Uout = h->U[h->cur ^ 1];
  e = launch_stage(prec, 2, g.TX, g.TY, nblocks, h->smem_bytes, h->stream, g, a, tma_for(h, a.Win));
  if (e) return e;
  if (h->profiling && (e = record_event(h))) return e;
  // U^{n+1} is in U[cur^1] and its primitives in W[cur]: swap the W buffers
  // so that W[new cur] holds them
  void* t = h->W[0];
  h->W[0] = h->W[1];
  h->W[1] = t;
  h->cur ^= 1;
  h->parity ^= 1;
  return cudaSuccess;
}

static int need_switch(mhd_handle* h) {
  if (h->cfg.riemann == MHD_LEARNED && !h->mlp)
    return fail(h, MHD_ERR_INVALID, "riemann is MHD_LEARNED but no network was set (mhd_set_switch)");
  return MHD_OK;
}

static int enqueue_steps(mhd_handle* h, double dt, int nsteps) {
  if (int rc = need_switch(h)) return rc;
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = launch_step(h, dt);
    if (e != cudaSuccess) return fail(h, MHD_ERR_CUDA, "stage launch failed: %s", cudaGetErrorString(e));
    h->steps++;
  }
  return MHD_OK;
}

static int read_words(mhd_handle* h) {
  unsigned long long* hp = (unsigned long long*)h->pinned;
  CUDA_TRY(h, cudaMemcpyAsync(hp, h->words, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MHD_OK;
}

static int check_status(mhd_handle* h) {
  int rc = read_words(h);
  if (rc) return rc;
  unsigned st = *(unsigned*)((unsigned long long*)h->pinned + 3);
  if (st & ST_NONFINITE) return fail(h, MHD_ERR_NONFINITE, "non-finite state value met on the device");
  if (st & ST_TIMEOUT) return fail(h, MHD_ERR_TIMEOUT, "a device wait timed out (barrier or plane copy)");
  if (st & ST_BOUNDS) return fail(h, MHD_ERR_BOUNDS, "a kernel index left its array (bounds-checked build)");
  if (h->cfg.floor_policy == MHD_FLOOR_ERROR) {
    const unsigned long long* hp = (const unsigned long long*)h->pinned;
    unsigned long long hits = hp[8 + C_RHO_FLOOR] + hp[8 + C_P_FLOOR];
    if (hits > h->floors_seen) {
      unsigned long long rho = hp[8 + C_RHO_FLOOR], p = hp[8 + C_P_FLOOR];
      h->floors_seen = hits;
      return fail(h, MHD_ERR_FLOOR, "floors applied: %llu density and %llu pressure hits so far", rho, p);
    }
  }
  return MHD_OK;
}

// ---- host streaming ---------------------------------------------------------

static int stream_setup(mhd_handle* h) {
  if (h->s_in) return MHD_OK;
  const size_t bytes = (size_t)h->geo.total * h->elem;
  cudaError_t e = cudaSuccess;
  constexpr int NS = mhd_handle::kSlots;
  for (int p = 0; p < NS && e == cudaSuccess; ++p) {
    e = cudaMalloc(&h->slot_in[p], bytes);
    if (e == cudaSuccess) h->owned_states.push_back(h->slot_in[p]);
  }
  // the output slots: the handle's own two state buffers and further ones
  for (int p = 0; p < NS && e == cudaSuccess; ++p) {
    if (p < 2) {
      h->slot_out[p] = h->owned_states[p];
    } else {
      e = cudaMalloc(&h->slot_out[p], bytes);
      if (e == cudaSuccess) h->owned_states.push_back(h->slot_out[p]);
    }
  }
  for (int p = 0; p < NS && e == cudaSuccess; ++p) {
    e = cudaEventCreateWithFlags(&h->ev_h2d[p], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[p], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_d2h[p], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    // undo this call's allocations, so that a later call starts afresh
    int code = e == cudaErrorMemoryAllocation ? MHD_ERR_NOMEM : MHD_ERR_CUDA;
    cudaGetLastError();
    for (int p = 0; p < NS; ++p) {
      if (h->ev_h2d[p]) cudaEventDestroy(h->ev_h2d[p]);
      if (h->ev_comp[p]) cudaEventDestroy(h->ev_comp[p]);
      if (h->ev_d2h[p]) cudaEventDestroy(h->ev_d2h[p]);
      h->ev_h2d[p] = h->ev_comp[p] = h->ev_d2h[p] = nullptr;
      h->slot_in[p] = h->slot_out[p] = nullptr;
    }
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    h->s_out = h->s_in = nullptr;
    while (h->owned_states.size() > 2) {   // the first two are the handle's own state buffers
      cudaFree(h->owned_states.back());
      h->owned_states.pop_back();
    }
    return fail(h, code, "streaming setup failed: %s", cudaGetErrorString(e));
  }
  return MHD_OK;
}

static cudaError_t copy_state_async(const mhd_handle* h, bool in, char* dev, void* const* cell, void* const* face,
                                    cudaStream_t st) {
  const cudaMemcpyKind kind = in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 5 && e == cudaSuccess; ++v) {
    char* d = dev + (size_t)v * h->geo.ncell * h->elem;
    const size_t n = (size_t)h->geo.ncell * h->elem;
    e = in ? cudaMemcpyAsync(d, cell[v], n, kind, st) : cudaMemcpyAsync(cell[v], d, n, kind, st);
  }
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    char* d = dev + (size_t)h->geo.face_off[k] * h->elem;
    const size_t n = (size_t)face_count(h->geo, k) * h->elem;
    e = in ? cudaMemcpyAsync(d, face[k], n, kind, st) : cudaMemcpyAsync(face[k], d, n, kind, st);
  }
  return e;
}

extern "C" int mhd_stream_step(mhd_handle* h, const void* const cell_in[5], const void* const face_in[3],
                               void* cell_out[5], void* face_out[3], double dt) {
  NvtxRange nvtx_range("mhd_stream_step");
  if (!h) return MHD_ERR_INVALID;
  if (!cell_in || !face_in || !cell_out || !face_out) return fail(h, MHD_ERR_INVALID, "null state pointer array");
  for (int v = 0; v < 5; ++v)
    if (!cell_in[v] || !cell_out[v]) return fail(h, MHD_ERR_INVALID, "null cell array %d", v);
  for (int k = 0; k < 3; ++k)
    if (!face_in[k] || !face_out[k]) return fail(h, MHD_ERR_INVALID, "null face array %d", k);
  if (dt != dt) return fail(h, MHD_ERR_INVALID, "dt is NaN");
  if (int rc = need_switch(h)) return rc;
  if (int rc = stream_setup(h)) return rc;
  const int p = (int)(h->nstream % mhd_handle::kSlots);
  // input: slot p is free once the step that read it (two back) has run
  CUDA_TRY(h, cudaStreamWaitEvent(h->s_in, h->ev_comp[p], 0));
  CUDA_TRY(h, copy_state_async(h, true, (char*)h->slot_in[p], (void* const*)cell_in, (void* const*)face_in, h->s_in));
  CUDA_TRY(h, cudaEventRecord(h->ev_h2d[p], h->s_in));
  // compute: after the input arrived and the output slot's previous copy-out
  CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_h2d[p], 0));
  CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_d2h[p], 0));
  h->U[h->cur] = h->slot_in[p];
  h->U[h->cur ^ 1] = h->slot_out[p];
  h->prims_valid = false;
  if (int rc = enqueue_steps(h, dt, 1)) return rc;
  if (dt > 0.0) h->last_dt = dt;
  CUDA_TRY(h, cudaEventRecord(h->ev_comp[p], h->stream));
  // output: the new state, now U[cur] = slot_out[p]
  CUDA_TRY(h, cudaStreamWaitEvent(h->s_out, h->ev_comp[p], 0));
  CUDA_TRY(h, copy_state_async(h, false, (char*)h->U[h->cur], cell_out, face_out, h->s_out));
  CUDA_TRY(h, cudaEventRecord(h->ev_d2h[p], h->s_out));
  h->nstream++;
  return MHD_OK;
}

extern "C" int mhd_stream_sync(mhd_handle* h) {
  if (!h) return MHD_ERR_INVALID;
  if (h->s_in) CUDA_TRY(h, cudaStreamSynchronize(h->s_in));
  if (h->s_out) CUDA_TRY(h, cudaStreamSynchronize(h->s_out));
  return check_status(h);
}

extern "C" int mhd_step_async(mhd_handle* h, double dt, int nsteps) {
  NvtxRange nvtx_range("mhd_step_async");
  if (!h) return MHD_ERR_INVALID;
  if (nsteps < 0) return fail(h, MHD_ERR_INVALID, "nsteps must be >= 0");
  if (dt != dt) return fail(h, MHD_ERR_INVALID, "dt is NaN");
  int rc = enqueue_steps(h, dt, nsteps);
  if (!rc && nsteps && dt > 0.0) h->last_dt = dt;
  return rc;
}

extern "C" int mhd_step(mhd_handle* h, double dt, int nsteps) {
  NvtxRange nvtx_range("mhd_step");
  if (!h) return MHD_ERR_INVALID;
  if (nsteps < 0) return fail(h, MHD_ERR_INVALID, "nsteps must be >= 0");
  if (dt != dt) return fail(h, MHD_ERR_INVALID, "dt is NaN");
  int rc = enqueue_steps(h, dt, nsteps);
  if (rc) return rc;
  rc = check_status(h);
  if (nsteps) {
    if (dt > 0.0) {
      h->last_dt = dt;
    } else {
      // the last step used the word of its starting state: parity ^ 1 now
      double m;
      unsigned long long bits = ((unsigned long long*)h->pinned)[h->parity ^ 1];
      memcpy(&m, &bits, sizeof m);
      h->last_dt = m > 0.0 ? h->cfg.cfl / m : 0.0;
    }
  }
  return rc;
}

extern "C" int mhd_rhs(mhd_handle* h, void* cell[5], void* face[3], int on_device) {
  NvtxRange nvtx_range("mhd_rhs");
  if (!h) return MHD_ERR_INVALID;
  if (int rc = need_switch(h)) return rc;
  cudaError_t e = ensure_prims(h);
  if (e) return fail(h, MHD_ERR_CUDA, "primitive recovery failed: %s", cudaGetErrorString(e));
  const Geo& g = h->geo;
  StageArgs a = base_args(h);
  a.dt = 1.0;                               // any dt > 0: only K1 = L(U) is kept
  a.dtword = h->words + h->parity;
  a.nextword = h->words + 4;                // scratch word, not the next step's
  a.U = h->U[h->cur];
  a.Win = h->W[h->cur];
  a.K1out = h->K1;
  a.Wout = nullptr;                         // no primitives of U + dt L
  e = launch_stage(h->cfg.precision, 1, g.TX, g.TY, (unsigned)(g.ntx * g.nty * g.nchunk), h->smem_bytes,
                   h->stream, g, a, tma_for(h, a.Win));
  if (e) return fail(h, MHD_ERR_CUDA, "stage launch failed: %s", cudaGetErrorString(e));
  int rc = copy_arrays(h, false, (char*)h->K1, h->kelem, cell, face, on_device);
  if (rc) return rc;
  return check_status(h);
}

extern "C" int mhd_set_profiling(mhd_handle* h, int on) {
  if (!h) return MHD_ERR_INVALID;
  h->profiling = on != 0;
  return MHD_OK;
}

extern "C" int mhd_get_profile(mhd_handle* h, double ms[3], long long launches[3]) {
  if (!h) return MHD_ERR_INVALID;
  if (!ms || !launches) return fail(h, MHD_ERR_INVALID, "null output pointer");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  const size_t nst = h->cfg.integrator == MHD_RK3 ? 3 : 2;   // events per step: nst + 1
  for (int s = 0; s < 3; ++s) {
    ms[s] = 0.0;
    launches[s] = 0;
  }
  for (size_t i = 0; i + nst + 1 <= h->ev_used; i += nst + 1) {
    for (size_t s = 0; s < nst; ++s) {
      float t = 0.f;
      CUDA_TRY(h, cudaEventElapsedTime(&t, h->ev_pool[i + s], h->ev_pool[i + s + 1]));
      ms[s] += t;
      launches[s]++;
    }
  }
  h->ev_used = 0;
  return MHD_OK;
}

// ------------------------------------------------------------ reductions
// CFL dt of the current state and max |div B|, both in FP64.

template <typename S>
__device__ double face_at(const Geo& g, const S* U, int d, int i, int j, int k) {
  int c[3] = {wrapc(i, g.n[0], g.bc[0]), wrapc(j, g.n[1], g.bc[1]), wrapc(k, g.n[2], g.bc[2])};
  const int raw[3] = {i, j, k};
  const FRef fr = face_ref1(raw[d], g.n[d], g.bc[d]);
  int len[3] = {g.n[0], g.n[1], g.n[2]};
  len[d] = g.nf[d];
  c[d] = fr.a;
  const long long ia = g.face_off[d] + c[0] + (long long)len[0] * (c[1] + (long long)len[1] * c[2]);
  c[d] = fr.b;
  const long long ib = g.face_off[d] + c[0] + (long long)len[0] * (c[1] + (long long)len[1] * c[2]);
  const double f0 = (double)U[ia], f1 = (double)U[ib];
  return f0 + (double)fr.t * (f1 - f0);
}

__device__ __forceinline__ void block_max_atomic(double v, unsigned long long* word) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(word, (unsigned long long)__double_as_longlong(v));
}

template <typename S>
__global__ void __launch_bounds__(256) cfl_kernel(Geo g, const S* U, unsigned long long* word) {
  double m = 0.0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.ncell; s += (long long)gridDim.x * blockDim.x) {
    int i = (int)(s % g.n[0]);
    int j = (int)((s / g.n[0]) % g.n[1]);
    int k = (int)(s / ((long long)g.n[0] * g.n[1]));
    double rho = (double)U[s];
    if (rho < g.rho_floor) rho = g.rho_floor;
    double mx = (double)U[g.ncell + s], my = (double)U[2 * g.ncell + s], mz = (double)U[3 * g.ncell + s];
    double e = (double)U[4 * g.ncell + s];
    double b[3] = {0.5 * (face_at(g, U, 0, i, j, k) + face_at(g, U, 0, i + 1, j, k)),
                   0.5 * (face_at(g, U, 1, i, j, k) + face_at(g, U, 1, i, j + 1, k)),
                   0.5 * (face_at(g, U, 2, i, j, k) + face_at(g, U, 2, i, j, k + 1))};
    double v[3] = {mx / rho, my / rho, mz / rho};
    double p = (g.gamma - 1.0) * (e - 0.5 * (mx * mx + my * my + mz * mz) / rho - 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
    if (p < g.p_floor) p = g.p_floor;
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (g.n[d] <= 1) continue;
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      double w[7] = {rho, v[d], v[t1], v[t2], p, b[t1], b[t2]};
      double cf = fast_speed(w, b[d], g.gamma);
      sum += (fabs(v[d]) + cf) * g.inv_d[d];
    }
    m = fmax(m, sum);
  }
  block_max_atomic(m, word);
}

template <typename S>
__global__ void __launch_bounds__(256) divb_kernel(Geo g, const S* U, unsigned long long* word) {
  double m = 0.0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.ncell; s += (long long)gridDim.x * blockDim.x) {
    int i = (int)(s % g.n[0]);
    int j = (int)((s / g.n[0]) % g.n[1]);
    int k = (int)(s / ((long long)g.n[0] * g.n[1]));
    double div = (face_at(g, U, 0, i + 1, j, k) - face_at(g, U, 0, i, j, k)) * g.inv_d[0] +
                 (face_at(g, U, 1, i, j + 1, k) - face_at(g, U, 1, i, j, k)) * g.inv_d[1] +
                 (face_at(g, U, 2, i, j, k + 1) - face_at(g, U, 2, i, j, k)) * g.inv_d[2];
    m = fmax(m, fabs(div));
  }
  block_max_atomic(m, word);
}

static int reduce_word(mhd_handle* h, bool cfl, double* out) {
  if (!h) return MHD_ERR_INVALID;
  if (!out) return fail(h, MHD_ERR_INVALID, "null output pointer");
  unsigned long long* word = h->words + 2;
  CUDA_TRY(h, cudaMemsetAsync(word, 0, sizeof(unsigned long long), h->stream));
  long long n = h->geo.ncell;
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  if (h->elem == 8) {
    const double* U = (const double*)h->U[h->cur];
    if (cfl) cfl_kernel<double><<<blocks, 256, 0, h->stream>>>(h->geo, U, word);
    else divb_kernel<double><<<blocks, 256, 0, h->stream>>>(h->geo, U, word);
  } else {
    const float* U = (const float*)h->U[h->cur];
    if (cfl) cfl_kernel<float><<<blocks, 256, 0, h->stream>>>(h->geo, U, word);
    else divb_kernel<float><<<blocks, 256, 0, h->stream>>>(h->geo, U, word);
  }
  CUDA_TRY(h, cudaGetLastError());
  unsigned long long* hp = (unsigned long long*)h->pinned;
  CUDA_TRY(h, cudaMemcpyAsync(hp, word, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  double m;
  memcpy(&m, hp, sizeof m);
  *out = cfl ? (m > 0.0 ? h->cfg.cfl / m : 0.0) : m;
  return MHD_OK;
}

extern "C" int mhd_cfl_dt(mhd_handle* h, double* dt_out) { return reduce_word(h, true, dt_out); }
extern "C" int mhd_divb_max(mhd_handle* h, double* out) { return reduce_word(h, false, out); }

extern "C" int mhd_get_stats(mhd_handle* h, mhd_stats* out) {
  if (!h) return MHD_ERR_INVALID;
  if (!out) return fail(h, MHD_ERR_INVALID, "null output pointer");
  int rc = read_words(h);
  if (rc) return rc;
  unsigned long long* hp = (unsigned long long*)h->pinned;
  memset(out, 0, sizeof *out);
  out->status = (int)*(unsigned*)(hp + 3);
  out->rho_floor_hits = (long long)hp[8 + C_RHO_FLOOR];
  out->p_floor_hits = (long long)hp[8 + C_P_FLOOR];
  out->faces_hll = (long long)hp[8 + C_HLL];
  out->faces_hlld = (long long)hp[8 + C_HLLD];
  out->last_dt = h->last_dt;
  out->steps = h->steps;
  out->tma_planes = (long long)hp[8 + C_TMA];
  return MHD_OK;
}

// =====================================================================
// Batched persistent launch
// =====================================================================

namespace mhd {
cudaError_t batch_launch_fp64(int, int, unsigned, size_t, cudaStream_t, const BatchArgs&);
cudaError_t batch_launch_mixed(int, int, unsigned, size_t, cudaStream_t, const BatchArgs&);
cudaError_t batch_launch_fp32(int, int, unsigned, size_t, cudaStream_t, const BatchArgs&);
cudaError_t batch_set_smem_fp64(int, int, size_t);
cudaError_t batch_set_smem_mixed(int, int, size_t);
cudaError_t batch_set_smem_fp32(int, int, size_t);
int batch_max_blocks_fp64(int, int, size_t);
size_t batch_smem_bytes_fp64(int, int);
size_t batch_smem_bytes_mixed(int, int);
size_t batch_smem_bytes_fp32(int, int);
int batch_max_blocks_mixed(int, int, size_t);
int batch_max_blocks_fp32(int, int, size_t);

cudaError_t batch_launch(int prec, int tx, int ty, unsigned grid, size_t smem, cudaStream_t st, const BatchArgs& ba) {
  switch (prec) {
    case P_FP64: return batch_launch_fp64(tx, ty, grid, smem, st, ba);
    case P_MIXED: return batch_launch_mixed(tx, ty, grid, smem, st, ba);
    default: return batch_launch_fp32(tx, ty, grid, smem, st, ba);
  }
}
cudaError_t batch_set_smem(int prec, int tx, int ty, size_t bytes) {
  switch (prec) {
    case P_FP64: return batch_set_smem_fp64(tx, ty, bytes);
    case P_MIXED: return batch_set_smem_mixed(tx, ty, bytes);
    default: return batch_set_smem_fp32(tx, ty, bytes);
  }
}
static size_t batch_smem_bytes(int prec, int tx, int ty) {
  switch (prec) {
    case P_FP64: return batch_smem_bytes_fp64(tx, ty);
    case P_MIXED: return batch_smem_bytes_mixed(tx, ty);
    default: return batch_smem_bytes_fp32(tx, ty);
  }
}
int batch_max_blocks_per_sm(int prec, int tx, int ty, size_t smem) {
  switch (prec) {
    case P_FP64: return batch_max_blocks_fp64(tx, ty, smem);
    case P_MIXED: return batch_max_blocks_mixed(tx, ty, smem);
    default: return batch_max_blocks_fp32(tx, ty, smem);
  }
}
}  // namespace mhd

struct mhd_batch {
  int nbox = 0;
  int prec = 0;
  std::vector<mhd_config> cfg;
  std::vector<BoxDesc> box;          // host mirror
  BoxDesc* dbox = nullptr;           // device copy
  ItemRef* dorder = nullptr;         // device item list, longest first
  size_t dorder_cap = 0;             // its capacity in entries
  std::vector<size_t> ubytes, kbytes, wbytes;
  std::vector<bool> prims_valid;
  void* pool = nullptr;              // all per-box buffers
  unsigned long long* words = nullptr;   // [0..63] general, then 2 per box
  unsigned* bar_count = nullptr;
  unsigned long long* work = nullptr;    // item draws of one launch
  unsigned* status = nullptr;
  unsigned long long* counters = nullptr;
  void* pinned = nullptr;
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap = nullptr;        // private stream for graph capture
  int tx = 16, ty = 8, tz = 32;
  size_t smem = 0;
  unsigned grid = 0;
  long long total_items = 0;
  double timeout_s = 2.0;
  int skip_arrival = 0;
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  double g_dt = 0.0;
  int g_nsteps = -1;
  int steps = 0;
  std::string err;
};

static thread_local std::string g_batch_err;   // error text of batch calls without a handle, per host thread

static int bfail(mhd_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf; else g_batch_err = buf;
  return code;
}

#define BCUDA_TRY(b, call)                                                                \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bfail((b), MHD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

static void drop_graph(mhd_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_nsteps = -1;
}

// Recompute per-box geometry, work items, shared memory and the persistent
// grid for tile (tx, ty, tz), and upload the box table.
static int batch_apply_tile(mhd_batch* b, int tx, int ty, int tz) {
  if (!stage_tile_supported(b->prec, tx, ty) || batch_max_blocks_per_sm(b->prec, tx, ty, 0) < 0)
    return bfail(b, MHD_ERR_INVALID, "tile %dx%d not available for the batch kernel", tx, ty);
  const size_t smem = batch_smem_bytes(b->prec, tx, ty);
  if (smem == 0 || smem > 227 * 1024) return bfail(b, MHD_ERR_INVALID, "tile %dx%d not available", tx, ty);
  cudaError_t e = batch_set_smem(b->prec, tx, ty, smem);
  if (e) return bfail(b, MHD_ERR_INVALID, "tile %dx%d is not instantiated for the batch kernel: %s", tx, ty,
                      cudaGetErrorString(e));
  int per_sm = batch_max_blocks_per_sm(b->prec, tx, ty, smem);
  if (per_sm < 1) return bfail(b, MHD_ERR_INVALID, "tile %dx%d cannot be resident", tx, ty);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long item = 0;
  for (int i = 0; i < b->nbox; ++i) {
    mhd_config c = b->cfg[i];
    c.tile_x = tx; c.tile_y = ty; c.tile_z = tz;
    fill_geo(&c, &b->box[i].g);
    b->box[i].item_begin = item;
    b->box[i].nitems = b->box[i].g.ntx * b->box[i].g.nty * b->box[i].g.nchunk;
    item += b->box[i].nitems;
  }
  b->total_items = item;
  // the item list, longest first: a chunk's cost grows with its planes plus
  // the three-plane prologue of its z-march (ties keep box order)
  std::vector<std::pair<int, ItemRef>> items;
  items.reserve((size_t)item);
  for (int i = 0; i < b->nbox; ++i) {
    const Geo& g = b->box[i].g;
    const int per_chunk = g.ntx * g.nty;
    for (int l = 0; l < b->box[i].nitems; ++l) {
      const int kb = (l / per_chunk) * g.TZ;
      const int ke = kb + g.TZ < g.n[2] ? kb + g.TZ : g.n[2];
      items.push_back({ke - kb + 3, ItemRef{i, l}});
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<int, ItemRef>& x, const std::pair<int, ItemRef>& y) { return x.first > y.first; });
  std::vector<ItemRef> order(items.size());
  for (size_t q = 0; q < items.size(); ++q) order[q] = items[q].second;
  if (order.size() > b->dorder_cap) {
    drop_graph(b);
    cudaFree(b->dorder);
    b->dorder = nullptr;
    b->dorder_cap = 0;
    BCUDA_TRY(b, cudaMalloc(&b->dorder, order.size() * sizeof(ItemRef)));
    b->dorder_cap = order.size();
  }
  BCUDA_TRY(b, cudaMemcpyAsync(b->dorder, order.data(), order.size() * sizeof(ItemRef), cudaMemcpyHostToDevice,
                               b->stream));
  b->tx = tx; b->ty = ty; b->tz = tz;
  b->smem = smem;
  b->grid = (unsigned)(per_sm * nsm);
  BCUDA_TRY(b, cudaMemcpyAsync(b->dbox, b->box.data(), sizeof(BoxDesc) * b->nbox, cudaMemcpyHostToDevice, b->stream));
  BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  drop_graph(b);
  return MHD_OK;
}

extern "C" void mhd_batch_destroy(mhd_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream); else cudaDeviceSynchronize();
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->pool);
  cudaFree(b->words);
  cudaFree(b->dbox);
  cudaFree(b->dorder);
  if (b->pinned) cudaFreeHost(b->pinned);
  delete b;
}

extern "C" const char* mhd_batch_last_error(const mhd_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

extern "C" int mhd_batch_create(int nbox, const mhd_config* cfgs, void* cuda_stream, mhd_batch** out) {
  if (!out || !cfgs || nbox < 1) return bfail(nullptr, MHD_ERR_INVALID, "need nbox >= 1, configs and an output pointer");
  for (int i = 0; i < nbox; ++i) {
    int rc = validate(&cfgs[i], nullptr);
    if (rc) return bfail(nullptr, rc, "box %d: %s", i, g_create_err.c_str());
    if (cfgs[i].precision != cfgs[0].precision || cfgs[i].riemann != cfgs[0].riemann || cfgs[i].emf != cfgs[0].emf)
      return bfail(nullptr, MHD_ERR_INVALID, "all boxes of a batch share precision, Riemann solver and EMF mode");
    if (cfgs[i].riemann == MHD_LEARNED)
      return bfail(nullptr, MHD_ERR_INVALID, "batches solve with HLLD or HLL; the learned switch is single-box only");
    if (cfgs[i].integrator != MHD_RK2)
      return bfail(nullptr, MHD_ERR_INVALID, "batches step with the RK2 integrator; SSP-RK3 is single-box only");
    if (cfgs[i].recon != MHD_RECON_PRIMITIVE)
      return bfail(nullptr, MHD_ERR_INVALID, "batches reconstruct the primitives; characteristic PLM is single-box only");
  }
  mhd_batch* b = new (std::nothrow) mhd_batch();
  if (!b) return bfail(nullptr, MHD_ERR_NOMEM, "host allocation failed");
  b->nbox = nbox;
  b->prec = cfgs[0].precision;
  b->cfg.assign(cfgs, cfgs + nbox);
  b->box.resize(nbox);
  b->prims_valid.assign(nbox, false);
  b->stream = (cudaStream_t)cuda_stream;
  const size_t elem = b->prec == MHD_FP32 ? 4 : 8, kelem = b->prec == MHD_FP64 ? 8 : 4, welem = kelem;
  size_t total = 0;
  auto take = [&](size_t n) { size_t o = total; total += (n + 255) / 256 * 256; return o; };
  std::vector<size_t> off(5 * nbox);
  for (int i = 0; i < nbox; ++i) {
    Geo g;
    fill_geo(&cfgs[i], &g);
    off[5 * i + 0] = take((size_t)g.total * elem);
    off[5 * i + 1] = take((size_t)g.total * elem);
    off[5 * i + 2] = take((size_t)g.total * kelem);
    off[5 * i + 3] = take((size_t)g.ncell * NW * welem);
    off[5 * i + 4] = take((size_t)g.ncell * NW * welem);
    b->ubytes.push_back((size_t)g.total * elem);
    b->kbytes.push_back((size_t)g.total * kelem);
    b->wbytes.push_back((size_t)g.ncell * NW * welem);
  }
  cudaError_t e = cudaMalloc(&b->pool, total);
  if (e == cudaSuccess) e = cudaMalloc(&b->words, (64 + 2 * (size_t)nbox) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->dbox, sizeof(BoxDesc) * nbox);
  if (e == cudaSuccess) e = cudaMallocHost(&b->pinned, 64 * sizeof(unsigned long long) + 8 * (size_t)nbox * 2);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MHD_ERR_NOMEM : MHD_ERR_CUDA;
    bfail(nullptr, code, "batch allocation of %zu B failed: %s", total, cudaGetErrorString(e));
    cudaGetLastError();
    mhd_batch_destroy(b);
    return code;
  }
  b->bar_count = (unsigned*)(b->words + 0);
  b->work = b->words + 1;
  b->status = (unsigned*)(b->words + 3);
  b->counters = b->words + 8;
  char* pool = (char*)b->pool;
  for (int i = 0; i < nbox; ++i) {
    BoxDesc& d = b->box[i];
    memset(&d, 0, sizeof d);
    d.U[0] = pool + off[5 * i + 0];
    d.U[1] = pool + off[5 * i + 1];
    d.K1 = pool + off[5 * i + 2];
    d.W[0] = pool + off[5 * i + 3];
    d.W[1] = pool + off[5 * i + 4];
    d.words = b->words + 64 + 2 * i;
  }
  e = cudaMemsetAsync(b->words, 0, (64 + 2 * (size_t)nbox) * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->pool, 0, total, b->stream);
  if (e != cudaSuccess) {
    bfail(nullptr, MHD_ERR_CUDA, "batch initialisation failed: %s", cudaGetErrorString(e));
    mhd_batch_destroy(b);
    return MHD_ERR_CUDA;
  }
  int tx, ty, tz;
  resolve_tile(&cfgs[0], &tx, &ty, &tz);
  int rc = batch_apply_tile(b, tx, ty, tz);
  if (rc) {
    g_batch_err = b->err;
    mhd_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MHD_OK;
}

static int batch_copy(mhd_batch* b, int i, bool in, void* const* cell, void* const* face, int on_device) {
  if (!b) return MHD_ERR_INVALID;
  if (i < 0 || i >= b->nbox) return bfail(b, MHD_ERR_INVALID, "box index %d out of range", i);
  if (!cell || !face) return bfail(b, MHD_ERR_INVALID, "null state pointer array");
  const Geo& g = b->box[i].g;
  const size_t elem = b->prec == MHD_FP32 ? 4 : 8;
  char* base = (char*)b->box[i].U[b->box[i].cur];
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  for (int v = 0; v < 5; ++v) {
    if (!cell[v]) return bfail(b, MHD_ERR_INVALID, "null cell array %d", v);
    char* dev = base + (size_t)v * g.ncell * elem;
    BCUDA_TRY(b, in ? cudaMemcpyAsync(dev, cell[v], g.ncell * elem, kind, b->stream)
                    : cudaMemcpyAsync(cell[v], dev, g.ncell * elem, kind, b->stream));
  }
  for (int d = 0; d < 3; ++d) {
    if (!face[d]) return bfail(b, MHD_ERR_INVALID, "null face array %d", d);
    char* dev = base + (size_t)g.face_off[d] * elem;
    const size_t n = (size_t)face_count(g, d) * elem;
    BCUDA_TRY(b, in ? cudaMemcpyAsync(dev, face[d], n, kind, b->stream) : cudaMemcpyAsync(face[d], dev, n, kind, b->stream));
  }
  if (!in || !on_device) BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  if (in) b->prims_valid[i] = false;
  return MHD_OK;
}

extern "C" int mhd_batch_set_state(mhd_batch* b, int box, const void* const cell[5], const void* const face[3],
                                   int on_device) {
  return batch_copy(b, box, true, (void* const*)cell, (void* const*)face, on_device);
}

extern "C" int mhd_batch_get_state(mhd_batch* b, int box, void* cell[5], void* face[3], int on_device) {
  return batch_copy(b, box, false, cell, face, on_device);
}

static int batch_ensure_prims(mhd_batch* b) {
  for (int i = 0; i < b->nbox; ++i) {
    if (b->prims_valid[i]) continue;
    BoxDesc& d = b->box[i];
    StageArgs a;
    memset(&a, 0, sizeof a);
    a.status = b->status;
    a.counters = b->counters;
    a.U = d.U[d.cur];
    a.Wout = d.W[0];
    a.nextword = d.words + d.parity;
    BCUDA_TRY(b, cudaMemsetAsync(d.words + d.parity, 0, sizeof(unsigned long long), b->stream));
    unsigned nb = (unsigned)((d.g.ncell + 255) / 256);
    if (nb > 152u * 16u) nb = 152u * 16u;
    BCUDA_TRY(b, launch_prims(b->prec, nb, b->stream, d.g, a));
    b->prims_valid[i] = true;
  }
  return MHD_OK;
}

static BatchArgs batch_args(mhd_batch* b, double dt, int nsteps) {
  BatchArgs ba;
  memset(&ba, 0, sizeof ba);
  ba.boxes = b->dbox;
  ba.nbox = b->nbox;
  ba.total_items = b->total_items;
  ba.order = b->dorder;
  ba.work = b->work;
  ba.nsteps = nsteps;
  ba.dt = dt;
  ba.bar_count = b->bar_count;
  ba.status = b->status;
  ba.counters = b->counters;
  ba.timeout_ns = (unsigned long long)(b->timeout_s * 1e9);
  ba.skip_arrival = b->skip_arrival;
  return ba;
}

// One persistent launch of nsteps steps for every box (enqueue only).
static int batch_enqueue(mhd_batch* b, double dt, int nsteps) {
  int rc = batch_ensure_prims(b);
  if (rc) return rc;
  const BatchArgs ba = batch_args(b, dt, nsteps);
  const bool graph = b->use_graph && !b->skip_arrival;
  if (graph && !(b->gexec && b->g_dt == dt && b->g_nsteps == nsteps)) {
    drop_graph(b);
    cudaGraph_t gr = nullptr;
    BCUDA_TRY(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->words, 0, 2 * sizeof(unsigned long long), b->cap);   // barrier, draws
    if (e == cudaSuccess) e = batch_launch(b->prec, b->tx, b->ty, b->grid, b->smem, b->cap, ba);
    if (e == cudaSuccess) {
      batch_advance<<<(b->nbox + 127) / 128, 128, 0, b->cap>>>(b->dbox, b->nbox, nsteps);
      e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      drop_graph(b);
      cudaGetLastError();
      return bfail(b, MHD_ERR_CUDA, "graph capture of the persistent launch failed: %s", cudaGetErrorString(e));
    }
    b->g_dt = dt;
    b->g_nsteps = nsteps;
  }
  if (graph) {
    BCUDA_TRY(b, cudaGraphLaunch(b->gexec, b->stream));
  } else {
    BCUDA_TRY(b, cudaMemsetAsync(b->words, 0, 2 * sizeof(unsigned long long), b->stream));   // barrier, draws
    BCUDA_TRY(b, batch_launch(b->prec, b->tx, b->ty, b->grid, b->smem, b->stream, ba));
    batch_advance<<<(b->nbox + 127) / 128, 128, 0, b->stream>>>(b->dbox, b->nbox, nsteps);
    BCUDA_TRY(b, cudaGetLastError());
  }
  for (int i = 0; i < b->nbox; ++i) {
    b->box[i].cur = (b->box[i].cur + nsteps) & 1;
    b->box[i].parity = (b->box[i].parity + nsteps) & 1;
  }
  b->steps += nsteps;
  return MHD_OK;
}

static int batch_check(mhd_batch* b) {
  unsigned long long* hp = (unsigned long long*)b->pinned;
  BCUDA_TRY(b, cudaMemcpyAsync(hp, b->words, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
  BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  const unsigned st = *(unsigned*)(hp + 3);
  if (st & (ST_TIMEOUT | ST_NONFINITE | ST_BOUNDS)) {
    // report once, then clear so that the handle can be reused
    BCUDA_TRY(b, cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->stream));
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    if (st & ST_TIMEOUT) return bfail(b, MHD_ERR_TIMEOUT, "device-wide barrier of the persistent launch timed out");
    if (st & ST_BOUNDS) return bfail(b, MHD_ERR_BOUNDS, "a kernel index left its array (bounds-checked build)");
    return bfail(b, MHD_ERR_NONFINITE, "non-finite state value met on the device");
  }
  return MHD_OK;
}

extern "C" int mhd_batch_step_async(mhd_batch* b, double dt, int nsteps) {
  NvtxRange nvtx_range("mhd_batch_step_async");
  if (!b) return MHD_ERR_INVALID;
  if (nsteps < 1) return bfail(b, MHD_ERR_INVALID, "nsteps must be >= 1");
  if (dt != dt) return bfail(b, MHD_ERR_INVALID, "dt is NaN");
  return batch_enqueue(b, dt, nsteps);
}

extern "C" int mhd_batch_step(mhd_batch* b, double dt, int nsteps) {
  NvtxRange nvtx_range("mhd_batch_step");
  int rc = mhd_batch_step_async(b, dt, nsteps);
  if (rc) return rc;
  return batch_check(b);
}

extern "C" int mhd_batch_set_tile(mhd_batch* b, int tx, int ty, int tz) {
  if (!b) return MHD_ERR_INVALID;
  if (tz < 1) return bfail(b, MHD_ERR_INVALID, "tile_z must be >= 1");
  BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  return batch_apply_tile(b, tx, ty, tz);
}

extern "C" int mhd_batch_get_tile(mhd_batch* b, int tile[3], long long* items, int* grid) {
  if (!b || !tile) return MHD_ERR_INVALID;
  tile[0] = b->tx; tile[1] = b->ty; tile[2] = b->tz;
  if (items) *items = b->total_items;
  if (grid) *grid = (int)b->grid;
  return MHD_OK;
}

extern "C" int mhd_batch_set_barrier_timeout(mhd_batch* b, double seconds) {
  if (!b) return MHD_ERR_INVALID;
  if (!(seconds > 0.0)) return bfail(b, MHD_ERR_INVALID, "timeout must be positive");
  b->timeout_s = seconds;
  drop_graph(b);
  return MHD_OK;
}

extern "C" int mhd_batch_inject_missed_arrival(mhd_batch* b, int on) {
  if (!b) return MHD_ERR_INVALID;
  b->skip_arrival = on != 0;
  drop_graph(b);
  return MHD_OK;
}

extern "C" int mhd_batch_box_dt(mhd_batch* b, int box, double* dt_out) {
  if (!b || !dt_out) return MHD_ERR_INVALID;
  if (box < 0 || box >= b->nbox) return bfail(b, MHD_ERR_INVALID, "box index %d out of range", box);
  int rc = batch_ensure_prims(b);
  if (rc) return rc;
  unsigned long long* hp = (unsigned long long*)b->pinned + 32;
  const BoxDesc& d = b->box[box];
  BCUDA_TRY(b, cudaMemcpyAsync(hp, d.words + d.parity, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
  BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  double m;
  memcpy(&m, hp, sizeof m);
  *dt_out = m > 0.0 ? b->cfg[box].cfl / m : 0.0;
  return MHD_OK;
}

extern "C" int mhd_batch_get_stats(mhd_batch* b, mhd_stats* out) {
  if (!b || !out) return MHD_ERR_INVALID;
  unsigned long long* hp = (unsigned long long*)b->pinned;
  BCUDA_TRY(b, cudaMemcpyAsync(hp, b->words, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
  BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
  memset(out, 0, sizeof *out);
  out->status = (int)*(unsigned*)(hp + 3);
  out->rho_floor_hits = (long long)hp[8 + C_RHO_FLOOR];
  out->p_floor_hits = (long long)hp[8 + C_P_FLOOR];
  out->faces_hll = (long long)hp[8 + C_HLL];
  out->faces_hlld = (long long)hp[8 + C_HLLD];
  out->steps = b->steps;
  return MHD_OK;
}

// ---------------------------------------------------------------- autotuner
// Times every instantiated tile shape (and a few z-chunk lengths) on the
// batch itself for `trial_steps` steps, keeps the fastest, and records it in
// a JSON-lines cache keyed by device, precision, Riemann solver and the box
// sizes, so later runs on the same batch skip the trials.

static std::string batch_key(mhd_batch* b) {
  int dev = 0, maj = 0, min = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  unsigned long long h = 1469598103934665603ull;
  long long cells = 0;
  for (int i = 0; i < b->nbox; ++i) {
    const int n[3] = {b->cfg[i].nx, b->cfg[i].ny, b->cfg[i].nz};
    for (int d = 0; d < 3; ++d) h = (h ^ (unsigned long long)(n[d] * 2 + b->cfg[i].bc[d])) * 1099511628211ull;
    cells += (long long)n[0] * n[1] * n[2];
  }
  char buf[256];
  snprintf(buf, sizeof buf, "sm_%d%d|prec%d|riemann%d|nbox%d|cells%lld|dims%016llx", maj, min, b->prec,
           b->cfg[0].riemann, b->nbox, cells, h);
  return buf;
}

static bool cache_lookup(const char* path, const std::string& key, int tile[3], double* ms) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[512];
    int tx, ty, tz;
    double m;
    if (sscanf(line, "{\"key\": \"%511[^\"]\", \"tile\": [%d, %d, %d], \"ms_per_step\": %lf", k, &tx, &ty, &tz, &m) == 5 &&
        key == k) {
      tile[0] = tx; tile[1] = ty; tile[2] = tz;
      *ms = m;
      found = true;  // the last matching line wins
    }
  }
  fclose(f);
  return found;
}

extern "C" int mhd_batch_autotune(mhd_batch* b, int trial_steps, const char* cache_path, int tile_out[3],
                                  double* ms_out) {
  if (!b) return MHD_ERR_INVALID;
  if (trial_steps < 1) return bfail(b, MHD_ERR_INVALID, "trial_steps must be >= 1");
  const std::string key = batch_key(b);
  int best[3] = {b->tx, b->ty, b->tz};
  double best_ms = -1.0;
  if (cache_lookup(cache_path, key, best, &best_ms)) {
    int rc = batch_apply_tile(b, best[0], best[1], best[2]);
    if (rc == MHD_OK) {
      if (tile_out) { tile_out[0] = best[0]; tile_out[1] = best[1]; tile_out[2] = best[2]; }
      if (ms_out) *ms_out = best_ms;
      return MHD_OK;
    }
  }
  // keep the states: trials advance them
  int rc = batch_ensure_prims(b);
  if (rc) return rc;
  std::vector<void*> save(b->nbox, nullptr);
  for (int i = 0; i < b->nbox; ++i) {
    cudaError_t e = cudaMalloc(&save[i], b->ubytes[i]);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(save[i], b->box[i].U[b->box[i].cur], b->ubytes[i], cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) {
      for (void* p : save) cudaFree(p);
      return bfail(b, MHD_ERR_NOMEM, "autotune state copy failed: %s", cudaGetErrorString(e));
    }
  }
  static const int cand_xy[][2] = {{16, 8}, {16, 16}, {32, 8}, {24, 8}, {8, 8}};
  static const int cand_z[] = {16, 32, 64, 128};
  int maxnz = 1;
  for (int i = 0; i < b->nbox; ++i) maxnz = b->cfg[i].nz > maxnz ? b->cfg[i].nz : maxnz;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  best_ms = -1.0;
  for (const auto& xy : cand_xy) {
    for (int zi = 0; zi < 4; ++zi) {
      const int tz = cand_z[zi];
      if (zi > 0 && cand_z[zi - 1] >= maxnz) break;
      if (batch_apply_tile(b, xy[0], xy[1], tz) != MHD_OK) break;   // tile not instantiated
      if (batch_enqueue(b, -1.0, 1) != MHD_OK) continue;
      cudaEventRecord(e0, b->stream);
      if (batch_enqueue(b, -1.0, trial_steps) != MHD_OK) continue;
      cudaEventRecord(e1, b->stream);
      if (batch_check(b) != MHD_OK) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = ms / trial_steps;
      if (best_ms < 0.0 || per < best_ms) {
        best_ms = per;
        best[0] = xy[0]; best[1] = xy[1]; best[2] = tz;
      }
      // restore the states for the next candidate
      for (int i = 0; i < b->nbox; ++i) {
        cudaMemcpyAsync(b->box[i].U[b->box[i].cur], save[i], b->ubytes[i], cudaMemcpyDeviceToDevice, b->stream);
        b->prims_valid[i] = false;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < b->nbox; ++i) {
    cudaMemcpyAsync(b->box[i].U[b->box[i].cur], save[i], b->ubytes[i], cudaMemcpyDeviceToDevice, b->stream);
    b->prims_valid[i] = false;
  }
  cudaStreamSynchronize(b->stream);
  for (void* p : save) cudaFree(p);
  if (best_ms < 0.0) return bfail(b, MHD_ERR_CUDA, "no tile candidate ran");
  rc = batch_apply_tile(b, best[0], best[1], best[2]);
  if (rc) return rc;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "{\"key\": \"%s\", \"tile\": [%d, %d, %d], \"ms_per_step\": %.6f}\n", key.c_str(), best[0], best[1],
              best[2], best_ms);
      fclose(f);
    }
  }
  if (tile_out) { tile_out[0] = best[0]; tile_out[1] = best[1]; tile_out[2] = best[2]; }
  if (ms_out) *ms_out = best_ms;
  return MHD_OK;
}

// Helpers shared with the allocation-free entry point (noalloc.cu).
namespace mhd {
int internal_validate(const mhd_config* c) { return validate(c, nullptr); }
void internal_fill_geo(const mhd_config* c, Geo* g) { fill_geo(c, g); }
long long internal_face_count(const Geo& g, int d) { return face_count(g, d); }
void internal_set_error(const char* msg) { g_create_err = msg; }
}  // namespace mhd

// ---------------------------------------------------------------- learned switch
namespace mhd {
int dump_faces_launch(int prec, const Geo& g, const void* W, const long long* ids, long long n, float* X, float* y,
                      float* score, cudaStream_t st);
}
extern "C" size_t mlp_param_bytes(void);

extern "C" int mhd_dump_faces(mhd_handle* h, const long long* face_ids, long long n, float* features, float* labels,
                              float* scores) {
  if (!h) return MHD_ERR_INVALID;
  if (!face_ids || !features || !labels || n < 0) return fail(h, MHD_ERR_INVALID, "bad arguments");
  for (int d = 0; d < 3; ++d)
    if (h->geo.bc[d] != 0) return fail(h, MHD_ERR_INVALID, "mhd_dump_faces samples periodic boxes only");
  cudaError_t e = ensure_prims(h);
  if (e) return fail(h, MHD_ERR_CUDA, "primitive recovery failed: %s", cudaGetErrorString(e));
  if (n == 0) return MHD_OK;
  int rc = dump_faces_launch(h->cfg.precision, h->geo, h->W[h->cur], face_ids, n, features, labels, scores,
                             h->stream);
  if (rc) return fail(h, rc, "face sampler launch failed");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MHD_OK;
}

extern "C" int mhd_set_switch(mhd_handle* h, const void* block, double tau) {
  if (!h) return MHD_ERR_INVALID;
  if (!block) return fail(h, MHD_ERR_INVALID, "null parameter block");
  if (!(tau > 0.0 && tau < 1.0)) return fail(h, MHD_ERR_INVALID, "tau must lie in (0, 1)");
  if (!h->mlp) CUDA_TRY(h, cudaMalloc(&h->mlp, mlp_param_bytes()));
  CUDA_TRY(h, cudaMemcpyAsync(h->mlp, block, mlp_param_bytes(), cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->mlp_zt = (float)log(tau / (1.0 - tau));
  return MHD_OK;
}

extern "C" int mhd_switch_choices(mhd_handle* h, unsigned char* choices, float* logits) {
  if (!h) return MHD_ERR_INVALID;
  if (h->cfg.riemann != MHD_LEARNED) return fail(h, MHD_ERR_INVALID, "the handle's riemann is not MHD_LEARNED");
  if (!choices) return fail(h, MHD_ERR_INVALID, "null choices pointer");
  if (int rc = need_switch(h)) return rc;
  cudaError_t e = ensure_prims(h);
  if (e) return fail(h, MHD_ERR_CUDA, "primitive recovery failed: %s", cudaGetErrorString(e));
  const Geo& g = h->geo;
  StageArgs a = base_args(h);
  a.dt = 1.0;
  a.dtword = h->words + h->parity;
  a.nextword = h->words + 4;
  a.U = h->U[h->cur];
  a.Win = h->W[h->cur];
  a.K1out = h->K1;                          // scratch: the operator's value is discarded
  a.Wout = nullptr;
  a.choices = choices;
  a.logits = logits;
  e = launch_stage(h->cfg.precision, 1, g.TX, g.TY, (unsigned)(g.ntx * g.nty * g.nchunk), h->smem_bytes,
                   h->stream, g, a);
  if (e) return fail(h, MHD_ERR_CUDA, "stage launch failed: %s", cudaGetErrorString(e));
  return check_status(h);
}
