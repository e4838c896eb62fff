// Batched persistent launch: many independent boxes of uneven size advance
// in ONE cooperative kernel.  Work items are (box, tile, z-chunk) of the fused
// stage kernel, listed by the host longest first (a chunk's cost grows with
// its planes plus the three-plane prologue of its march); the CTAs of a
// persistent grid (all co-resident) draw the next item of the list from a
// device counter as they finish one, meet at a device-wide barrier after each
// RK stage, and go on to the next stage / step.  Every box keeps its own CFL
// dt (the max that its stage 2 folded into the box's own word).  The barrier gives up after a
// %globaltimer limit, raises the timeout bit of the status word and every CTA
// returns, so the host sees MHD_ERR_TIMEOUT and the context stays usable.
#pragma once
#include "stage_impl.cuh"

namespace mhd {

struct BoxDesc {
  Geo g;
  void* U[2];
  void* K1;
  void* W[2];                  // W[0]: primitives of the current state, W[1]: of U*
  unsigned long long* words;   // [0], [1]: CFL words, alternating by step parity
  long long item_begin;        // first global work item of this box
  int nitems;
  int cur;                     // U[cur] holds the state at the start of a launch
  int parity;                  // words[parity] holds its CFL max
};

// one entry of the item list: box, and the item's index within the box
struct ItemRef {
  int box;
  int local;
};

struct BatchArgs {
  BoxDesc* boxes;
  int nbox;
  const ItemRef* order;        // the items, longest first
  unsigned long long* work;    // draws from the item list, monotone over one launch (zeroed before it)
  long long total_items;
  int nsteps;
  double dt;                   // > 0: every box takes this dt; <= 0: its own CFL dt
  unsigned* bar_count;         // arrivals, monotone over one launch (zeroed before it)
  unsigned* status;
  unsigned long long* counters;
  unsigned long long timeout_ns;
  int skip_arrival;            // test hook: CTA 0 does not arrive at the first barrier
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-wide barrier number `epoch` (1, 2, ...).  Returns false (in every
// thread of the CTA) when the batch was aborted by a timeout.
__device__ __forceinline__ bool grid_barrier(const BatchArgs& ba, unsigned epoch) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const bool skip = ba.skip_arrival && blockIdx.x == 0 && epoch == 1;
    if (!skip) atomicAdd(ba.bar_count, 1u);
    const unsigned target = epoch * gridDim.x;
    const unsigned long long t0 = global_ns();
    for (;;) {
      const unsigned c = *(volatile unsigned*)ba.bar_count;
      if (c >= target) break;
      if (*(volatile unsigned*)ba.status & ST_TIMEOUT) { ok = 0; break; }
      if (global_ns() - t0 > ba.timeout_ns) {
        atomicOr(ba.status, (unsigned)ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ StageArgs box_stage_args(const BatchArgs& ba, const BoxDesc& bd, int stage, int step) {
  StageArgs a;
  const int cur = (bd.cur + step) & 1;
  const int par = (bd.parity + step) & 1;
  a.U = bd.U[cur];
  a.K1 = stage == 2 ? bd.K1 : nullptr;
  a.K1out = stage == 1 ? bd.K1 : nullptr;
  a.Uout = stage == 2 ? bd.U[cur ^ 1] : nullptr;
  a.Win = stage == 1 ? bd.W[0] : bd.W[1];
  a.Wout = stage == 1 ? bd.W[1] : bd.W[0];
  a.dtword = bd.words + par;
  a.nextword = bd.words + (par ^ 1);
  a.status = ba.status;
  a.counters = ba.counters;
  a.dt = ba.dt;
  return a;
}

// Every CTA draws items until the list of the stage is exhausted: each draw
// takes the next ticket of the launch's counter, and each CTA makes exactly
// one draw past the end per stage, so stage e (0-based within the launch)
// owns tickets [e (T + G), (e + 1)(T + G)) for T items and G CTAs, and no
// draw of stage e + 1 starts before the barrier that ends stage e.
template <int PREC, int TX, int TY>
__global__ void __launch_bounds__(256, PREC == P_FP64 ? 1 : 3) batch_kernel(BatchArgs ba) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long next_item;
  const unsigned long long per_stage = (unsigned long long)ba.total_items + gridDim.x;
  unsigned epoch = 0;
  for (int step = 0; step < ba.nsteps; ++step) {
#pragma unroll 1
    for (int stage = 1; stage <= 2; ++stage) {
      const unsigned long long base = (unsigned long long)epoch * per_stage;
      for (;;) {
        if (threadIdx.x == 0) next_item = (long long)(atomicAdd(ba.work, 1ull) - base);
        __syncthreads();
        const long long it = next_item;   // every thread reads it before run_item's first barrier
        if (it >= ba.total_items) break;
        const ItemRef ref = ba.order[MHD_IDX(it, ba.total_items, ba.status)];
        const BoxDesc& bd = ba.boxes[MHD_IDX(ref.box, ba.nbox, ba.status)];
        const StageArgs a = box_stage_args(ba, bd, stage, step);
        if (stage == 1) StageKernel<PREC, 1, TX, TY>::run_item(bd.g, a, ref.local, smem_raw);
        else StageKernel<PREC, 2, TX, TY>::run_item(bd.g, a, ref.local, smem_raw);
      }
      if (!grid_barrier(ba, ++epoch)) return;
    }
  }
}

// After a launch of nsteps steps every box's state index and CFL parity have
// advanced by nsteps (a graph node, so captured launches can be replayed).
static __global__ void batch_advance(BoxDesc* boxes, int nbox, int nsteps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) {
    boxes[b].cur = (boxes[b].cur + nsteps) & 1;
    boxes[b].parity = (boxes[b].parity + nsteps) & 1;
  }
}

// host-side launchers (one translation unit per precision)
cudaError_t batch_launch(int prec, int tx, int ty, unsigned grid, size_t smem, cudaStream_t st, const BatchArgs& ba);
cudaError_t batch_set_smem(int prec, int tx, int ty, size_t bytes);
int batch_max_blocks_per_sm(int prec, int tx, int ty, size_t smem);

}  // namespace mhd
