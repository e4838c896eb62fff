// C ABI of the MHD hot path: handle, device buffers, launches, reductions.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/mhd_gb300.h"
#include "stage.cuh"

using namespace mhd;

struct mhd_handle {
  mhd_config cfg;
  Geo geo;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t elem = 8;          // bytes per state element
  size_t kelem = 8;         // bytes per stage-1 element
  void* U[2] = {nullptr, nullptr};
  void* K1 = nullptr;
  unsigned long long* smax = nullptr;      // step CFL word
  unsigned long long* smax_api = nullptr;  // word for mhd_cfl_dt
  double* dres = nullptr;                  // reduction result
  unsigned int* status = nullptr;
  unsigned long long* counters = nullptr;
  void* pinned = nullptr;                  // host readback buffer (64 B)
  int cur = 0;
  size_t smem_bytes = 0;
  double last_dt = 0.0;
  int steps = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;   // 3 events per recorded step
  size_t ev_used = 0;
  std::string err;
};

static std::string g_create_err;

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

static size_t stage_smem(int prec, int tx, int ty) {
  Smem L;
  L.init(tx, ty);
  return (size_t)L.total * (prec == MHD_FP64 ? sizeof(double) : sizeof(float));
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
  int tx = c->tile_x, ty = c->tile_y, tz = c->tile_z;
  if (tx < 0 || ty < 0 || tz < 0) return fail(h, MHD_ERR_INVALID, "tile sizes must be >= 0");
  if (tx == 0 || ty == 0 || tz == 0) {
    int dx, dy, dz;
    default_tile(c->precision, &dx, &dy, &dz);
    if (!tx) tx = dx;
    if (!ty) ty = dy;
    if (!tz) tz = dz;
  }
  if (tx > 64 || ty > 64 || tz > 4096) return fail(h, MHD_ERR_INVALID, "tile too large");
  if (stage_smem(c->precision, tx, ty) > 227 * 1024)
    return fail(h, MHD_ERR_INVALID, "tile %dx%d needs %zu B of shared memory (> 227 KB)", tx, ty,
                stage_smem(c->precision, tx, ty));
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
  g->gamma = c->gamma; g->rho_floor = c->rho_floor; g->p_floor = c->p_floor; g->cfl = c->cfl;
  g->emf_mean = c->emf == MHD_EMF_MEAN;
  g->riemann = c->riemann == MHD_HLL ? 1 : (c->riemann == MHD_LEARNED ? 2 : 0);
  int tx = c->tile_x, ty = c->tile_y, tz = c->tile_z, dx, dy, dz;
  default_tile(c->precision, &dx, &dy, &dz);
  g->TX = tx ? tx : dx; g->TY = ty ? ty : dy; g->TZ = tz ? tz : dz;
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
  h->smem_bytes = stage_smem(cfg->precision, h->geo.TX, h->geo.TY);
  cudaError_t e = cudaGetDevice(&h->device);
  size_t bytes = (size_t)h->geo.total * h->elem;
  size_t kbytes = (size_t)h->geo.total * h->kelem;
  if (e == cudaSuccess) e = cudaMalloc(&h->U[0], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->U[1], bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->K1, kbytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->smax, 64 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, 256);
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? MHD_ERR_NOMEM : MHD_ERR_CUDA;
    fail(nullptr, code, "device allocation of %zu B failed: %s", 2 * bytes + kbytes, cudaGetErrorString(e));
    cudaGetLastError();
    mhd_destroy(h);
    return code;
  }
  h->smax_api = h->smax + 1;
  h->dres = (double*)(h->smax + 2);
  h->status = (unsigned int*)(h->smax + 3);
  h->counters = h->smax + 8;
  e = cudaMemsetAsync(h->smax, 0, 64 * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->U[0], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->K1, 0, kbytes, h->stream);
  if (e == cudaSuccess) e = stage_set_smem(cfg->precision, h->smem_bytes);
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
  cudaFree(h->U[0]);
  cudaFree(h->U[1]);
  cudaFree(h->K1);
  cudaFree(h->smax);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

extern "C" const char* mhd_last_error(const mhd_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

static int copy_state(mhd_handle* h, bool in, void* const* cell, void* const* face, int on_device) {
  if (!h) return MHD_ERR_INVALID;
  if (!cell || !face) return fail(h, MHD_ERR_INVALID, "null state pointer array");
  for (int v = 0; v < 5; ++v)
    if (!cell[v]) return fail(h, MHD_ERR_INVALID, "null cell array %d", v);
  for (int d = 0; d < 3; ++d)
    if (!face[d]) return fail(h, MHD_ERR_INVALID, "null face array %d", d);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  char* base = (char*)h->U[h->cur];
  for (int v = 0; v < 5; ++v) {
    char* dev = base + (size_t)v * h->geo.ncell * h->elem;
    size_t n = (size_t)h->geo.ncell * h->elem;
    CUDA_TRY(h, in ? cudaMemcpyAsync(dev, cell[v], n, kind, h->stream) : cudaMemcpyAsync(cell[v], dev, n, kind, h->stream));
  }
  for (int d = 0; d < 3; ++d) {
    char* dev = base + (size_t)h->geo.face_off[d] * h->elem;
    size_t n = (size_t)face_count(h->geo, d) * h->elem;
    CUDA_TRY(h, in ? cudaMemcpyAsync(dev, face[d], n, kind, h->stream) : cudaMemcpyAsync(face[d], dev, n, kind, h->stream));
  }
  if (!in || !on_device) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return MHD_OK;
}

extern "C" int mhd_set_state(mhd_handle* h, const void* const cell[5], const void* const face[3], int on_device) {
  return copy_state(h, true, (void* const*)cell, (void* const*)face, on_device);
}

extern "C" int mhd_get_state(mhd_handle* h, void* cell[5], void* face[3], int on_device) {
  return copy_state(h, false, cell, face, on_device);
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

static cudaError_t launch_step(mhd_handle* h, double dt) {
  const Geo& g = h->geo;
  const unsigned nblocks = (unsigned)(g.ntx * g.nty * g.nchunk);
  const int prec = h->cfg.precision;
  StageArgs a;
  memset(&a, 0, sizeof a);
  a.smax = h->smax;
  a.status = h->status;
  a.counters = h->counters;
  a.dt = dt;
  cudaError_t e = cudaSuccess;
  if (!(dt > 0.0)) e = cudaMemsetAsync(h->smax, 0, sizeof(unsigned long long), h->stream);
  if (e) return e;
  a.U = h->U[h->cur];
  a.K1 = nullptr;
  a.OUT = h->K1;
  if (h->profiling && (e = record_event(h))) return e;
  e = launch_stage(prec, 1, nblocks, h->smem_bytes, h->stream, g, a);
  if (e) return e;
  if (h->profiling && (e = record_event(h))) return e;
  a.K1 = h->K1;
  a.OUT = h->U[h->cur ^ 1];
  e = launch_stage(prec, 2, nblocks, h->smem_bytes, h->stream, g, a);
  if (e) return e;
  if (h->profiling && (e = record_event(h))) return e;
  h->cur ^= 1;
  return cudaSuccess;
}

static int enqueue_steps(mhd_handle* h, double dt, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = launch_step(h, dt);
    if (e != cudaSuccess) return fail(h, MHD_ERR_CUDA, "stage launch failed: %s", cudaGetErrorString(e));
    h->steps++;
  }
  return MHD_OK;
}

static int check_status(mhd_handle* h) {
  unsigned long long* hp = (unsigned long long*)h->pinned;
  CUDA_TRY(h, cudaMemcpyAsync(hp, h->smax, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  unsigned st = *(unsigned*)(hp + 3);
  if (st & ST_NONFINITE) return fail(h, MHD_ERR_NONFINITE, "non-finite state value met on the device");
  if (st & ST_TIMEOUT) return fail(h, MHD_ERR_TIMEOUT, "device barrier timed out");
  return MHD_OK;
}

extern "C" int mhd_step_async(mhd_handle* h, double dt, int nsteps) {
  if (!h) return MHD_ERR_INVALID;
  if (nsteps < 0) return fail(h, MHD_ERR_INVALID, "nsteps must be >= 0");
  if (dt != dt) return fail(h, MHD_ERR_INVALID, "dt is NaN");
  int rc = enqueue_steps(h, dt, nsteps);
  if (!rc && nsteps && dt > 0.0) h->last_dt = dt;
  return rc;
}

extern "C" int mhd_set_profiling(mhd_handle* h, int on) {
  if (!h) return MHD_ERR_INVALID;
  h->profiling = on != 0;
  return MHD_OK;
}

extern "C" int mhd_get_profile(mhd_handle* h, double ms[2], long long launches[2]) {
  if (!h) return MHD_ERR_INVALID;
  if (!ms || !launches) return fail(h, MHD_ERR_INVALID, "null output pointer");
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (size_t i = 0; i + 3 <= h->ev_used; i += 3) {
    float a = 0.f, b = 0.f;
    CUDA_TRY(h, cudaEventElapsedTime(&a, h->ev_pool[i], h->ev_pool[i + 1]));
    CUDA_TRY(h, cudaEventElapsedTime(&b, h->ev_pool[i + 1], h->ev_pool[i + 2]));
    ms[0] += a;
    ms[1] += b;
    launches[0]++;
    launches[1]++;
  }
  h->ev_used = 0;
  return MHD_OK;
}

extern "C" int mhd_step(mhd_handle* h, double dt, int nsteps) {
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
      double m;
      unsigned long long bits = ((unsigned long long*)h->pinned)[0];
      memcpy(&m, &bits, sizeof m);
      h->last_dt = m > 0.0 ? h->cfg.cfl / m : 0.0;
    }
  }
  return rc;
}

// ------------------------------------------------------------ reductions
// CFL dt of the current state and max |div B|, both in FP64.

template <typename S>
__device__ double face_at(const Geo& g, const S* U, int d, int i, int j, int k) {
  FaceRef r = face_ref(g, d, i, j, k);
  double f0 = (double)U[r.i0], f1 = (double)U[r.i1];
  return f0 + r.t * (f1 - f0);
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
  CUDA_TRY(h, cudaMemsetAsync(h->smax_api, 0, sizeof(unsigned long long), h->stream));
  long long n = h->geo.ncell;
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  if (h->elem == 8) {
    const double* U = (const double*)h->U[h->cur];
    if (cfl) cfl_kernel<double><<<blocks, 256, 0, h->stream>>>(h->geo, U, h->smax_api);
    else divb_kernel<double><<<blocks, 256, 0, h->stream>>>(h->geo, U, h->smax_api);
  } else {
    const float* U = (const float*)h->U[h->cur];
    if (cfl) cfl_kernel<float><<<blocks, 256, 0, h->stream>>>(h->geo, U, h->smax_api);
    else divb_kernel<float><<<blocks, 256, 0, h->stream>>>(h->geo, U, h->smax_api);
  }
  CUDA_TRY(h, cudaGetLastError());
  unsigned long long* hp = (unsigned long long*)h->pinned;
  CUDA_TRY(h, cudaMemcpyAsync(hp, h->smax_api, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
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
  unsigned long long* hp = (unsigned long long*)h->pinned;
  CUDA_TRY(h, cudaMemcpyAsync(hp, h->smax, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof *out);
  out->status = (int)*(unsigned*)(hp + 3);
  out->rho_floor_hits = (long long)hp[8 + C_RHO_FLOOR];
  out->p_floor_hits = (long long)hp[8 + C_P_FLOOR];
  out->faces_hll = (long long)hp[8 + C_HLL];
  out->faces_hlld = (long long)hp[8 + C_HLLD];
  out->last_dt = h->last_dt;
  out->steps = h->steps;
  return MHD_OK;
}
