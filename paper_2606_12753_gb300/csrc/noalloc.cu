// One RK2 step of one box without any device allocation.
//
// Some callers cannot call cudaMalloc while they run: a service that
// reserves all of its device memory up front and must not allocate later
// (to avoid fragmentation or an out-of-memory error in the middle of a run),
// code that hands memory accounting to its own pool and must not see
// allocations it did not make, or a loop that cannot afford the device-wide
// synchronisation a cudaMalloc/cudaFree can cause.  mhd_step_noalloc serves
// them: it takes the caller's device arrays for the state before and after
// the step and keeps everything else it needs -- a packed copy of both states,
// the stage increment, the primitives of the two stage states and the status
// words -- in one file-scope device array, so it calls no allocating routine.
//
// The array below is reserved in every GPU that loads this library, for as
// long as the library stays loaded: MHD_NOALLOC_SCRATCH_BYTES (8 MiB).  Calls
// share it and it keeps the last call's contents; the status and CFL words
// are cleared at the start of each call.  Two calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race on
// the array and corrupt each other's results: serialise them.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/mhd_gb300.h"
#include "stage.cuh"

namespace mhd {
int internal_validate(const mhd_config* c);
void internal_fill_geo(const mhd_config* c, Geo* g);
long long internal_face_count(const Geo& g, int d);
void internal_set_error(const char* msg);
}  // namespace mhd

using namespace mhd;

static __device__ __align__(256) unsigned char g_noalloc_scratch[MHD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array per device.  In host code the name
// g_noalloc_scratch is only a stand-in, so it is resolved once per device
// (with that device current) and cached.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

static int noalloc_fail(int code, const char* fmt, const char* detail) {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, detail);
  internal_set_error(buf);
  return code;
}

static size_t align256(size_t n) { return (n + 255) / 256 * 256; }

extern "C" int mhd_step_noalloc(const mhd_config* cfg, void* cuda_stream, const void* const cell_in[5],
                                const void* const face_in[3], void* cell_out[5], void* face_out[3], double dt,
                                double* dt_used) {
  if (!cfg || !cell_in || !face_in || !cell_out || !face_out)
    return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s", "null argument");
  for (int v = 0; v < 5; ++v)
    if (!cell_in[v] || !cell_out[v]) return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s", "null cell array");
  for (int d = 0; d < 3; ++d)
    if (!face_in[d] || !face_out[d]) return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s", "null face array");
  if (dt != dt) return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s", "dt is NaN");
  if (cfg->integrator != MHD_RK2 || cfg->recon != MHD_RECON_PRIMITIVE)
    return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s", "runs RK2 with primitive reconstruction only");
  if (cfg->riemann == MHD_LEARNED)
    return noalloc_fail(MHD_ERR_INVALID, "mhd_step_noalloc: %s",
                        "runs HLLD or HLL only (the learned switch needs a network on a handle)");
  int rc = internal_validate(cfg);
  if (rc) return rc;   // message already set
  Geo g;
  internal_fill_geo(cfg, &g);
  const int prec = cfg->precision;
  const size_t elem = prec == MHD_FP32 ? 4 : 8, kelem = prec == MHD_FP64 ? 8 : 4;
  const size_t ubytes = (size_t)g.total * elem, kbytes = (size_t)g.total * kelem;
  const size_t wbytes = (size_t)g.ncell * NW * kelem;
  const size_t need = 2 * align256(ubytes) + align256(kbytes) + 2 * align256(wbytes) + 64 * 8;
  if (need > (size_t)MHD_NOALLOC_SCRATCH_BYTES) {
    char msg[64];
    snprintf(msg, sizeof msg, "%zu B", need);
    return noalloc_fail(MHD_ERR_INVALID,
                        "mhd_step_noalloc: the box needs %s of scratch, more than MHD_NOALLOC_SCRATCH_BYTES", msg);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return noalloc_fail(MHD_ERR_CUDA, "mhd_step_noalloc: %s", "no usable current device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(MHD_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      g_noalloc_ptr[dev] = p;
    }
    base = (unsigned char*)g_noalloc_ptr[dev];
  }
  unsigned char* p = base;
  void* Uin = p;   p += align256(ubytes);
  void* Uout = p;  p += align256(ubytes);
  void* K1 = p;    p += align256(kbytes);
  void* W0 = p;    p += align256(wbytes);
  void* W1 = p;    p += align256(wbytes);
  unsigned long long* words = (unsigned long long*)p;

  cudaError_t e = stage_set_smem(prec, g.TX, g.TY, stage_smem_bytes(prec, g.TX, g.TY));
  if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, 64 * 8, st);
  for (int v = 0; v < 5 && e == cudaSuccess; ++v)
    e = cudaMemcpyAsync((char*)Uin + (size_t)v * g.ncell * elem, cell_in[v], (size_t)g.ncell * elem,
                        cudaMemcpyDeviceToDevice, st);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync((char*)Uin + (size_t)g.face_off[d] * elem, face_in[d],
                        (size_t)internal_face_count(g, d) * elem, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return noalloc_fail(MHD_ERR_CUDA, "mhd_step_noalloc: %s", cudaGetErrorString(e));

  StageArgs a;
  memset(&a, 0, sizeof a);
  a.status = (unsigned int*)(words + 3);
  a.counters = words + 8;
  // primitives and CFL max of the input state
  a.U = Uin;
  a.Wout = W0;
  a.nextword = words + 0;
  unsigned nb = (unsigned)((g.ncell + 255) / 256);
  e = launch_prims(prec, nb, st, g, a);
  // stage 1 and stage 2 of the RK2 step
  const unsigned nblocks = (unsigned)(g.ntx * g.nty * g.nchunk);
  const size_t smem = stage_smem_bytes(prec, g.TX, g.TY);
  if (e == cudaSuccess) {
    a.dt = dt;
    a.dtword = words + 0;
    a.nextword = words + 1;
    a.Win = W0;
    a.K1out = K1;
    a.Wout = W1;
    e = launch_stage(prec, 1, g.TX, g.TY, nblocks, smem, st, g, a);
  }
  if (e == cudaSuccess) {
    a.K1 = K1;
    a.K1out = nullptr;
    a.Win = W1;
    a.Wout = W0;
    a.Uout = Uout;
    e = launch_stage(prec, 2, g.TX, g.TY, nblocks, smem, st, g, a);
  }
  for (int v = 0; v < 5 && e == cudaSuccess; ++v)
    e = cudaMemcpyAsync(cell_out[v], (char*)Uout + (size_t)v * g.ncell * elem, (size_t)g.ncell * elem,
                        cudaMemcpyDeviceToDevice, st);
  for (int d = 0; d < 3 && e == cudaSuccess; ++d)
    e = cudaMemcpyAsync(face_out[d], (char*)Uout + (size_t)g.face_off[d] * elem,
                        (size_t)internal_face_count(g, d) * elem, cudaMemcpyDeviceToDevice, st);
  // status word and the CFL max used by the step, read into host stack memory
  unsigned long long hw[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hw, words, sizeof hw, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(MHD_ERR_CUDA, "mhd_step_noalloc: %s", cudaGetErrorString(e));
  const unsigned status = (unsigned)(hw[3] & 0xffffffffu);
  if (status & ST_NONFINITE)
    return noalloc_fail(MHD_ERR_NONFINITE, "mhd_step_noalloc: %s", "non-finite state value met on the device");
  if (dt_used) {
    if (dt > 0.0) {
      *dt_used = dt;
    } else {
      double m;
      memcpy(&m, &hw[0], sizeof m);
      *dt_used = m > 0.0 ? cfg->cfl / m : 0.0;
    }
  }
  return MHD_OK;
}
