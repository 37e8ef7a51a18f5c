// Persistent ensemble kernel: one launch per RK stage steps every box of an
// ensemble (boxes of uneven N) through the stage, pulling work items from a
// device work table.
//
// A work item is (box, pass, tile): one CTA-sized piece of one of the stage's
// passes for one box -- the forcing amplitude, the inverse z and y transforms,
// the X pass, the CFL reset (stage 1), the forward y and z transforms, the
// stage combine and, after stage 4, the deterministic forcing (section 2.2's
// RK4 stage of Eqs. 7-8, as psc_step runs it).  Items are laid out pass by
// pass across all boxes; CTAs take them in that order from one counter, and
// an item waits until every tile of its box's previous pass has completed.
// Since every dependency of an item was taken earlier by a CTA that is
// already running, the waits always end; each is still bounded by time, after
// which the launch is abandoned and the box reports PSC_ETIMEOUT.  The table
// lives in device memory and is rewritten between ensemble steps when boxes
// join or leave, so a captured graph of the four launches stays valid.
//
// The pass bodies are the ones the ordinary kernels run, compiled here with
// virtual block coordinates, without __restrict__ (buffers written by other
// CTAs of the same launch must not be read through the non-coherent path),
// and in their own namespace so that these instantiations stay distinct from
// the ordinary kernels'.
#pragma once
#include <cstdio>
#include <cstring>
#include <vector>

#define PSC_RESTRICT
#define psc psc_persistent
#include "psc_kernels.cuh"
#include "psc_passes.cuh"
#undef psc

namespace {

namespace pp = psc_persistent;

constexpr int kThreads = 128;
// passes of a stage, in order
enum { BP_FAMP = 0, BP_ZINV, BP_YINV, BP_XPASS, BP_CFL, BP_YFWD, BP_ZFWD, BP_COMBINE, BP_HOLD, BP_N };
constexpr int kCombinePerThread = 4;  // compact modes per thread of a combine item
constexpr int kXGroupsPerWarp = 2;    // row groups per warp of an X-pass item

struct Seg {
  long long start;  // index of the segment's first item within the stage
  int box, pass, tiles;
  int per;          // tiles of the pass each item runs
  int dep;          // index into done[] of the pass this one waits for (-1: none)
  int dep_tiles;    // tiles that pass has
  int done_idx;     // index into done[] this segment counts into
};

struct Head {
  int nbox;
  int nseg[4];
  long long nitems[4];
  unsigned long long wait_ns;  // bound of every dependency wait
};

// Device table layout (bytes from the table's start), for max_boxes boxes.
struct TableLayout {
  size_t head, boxes, segs, counters, total;
  size_t seg_cap;      // segments per stage
  size_t counter_bytes;  // per stage: next (8 bytes), abort (4 + 4 pad), done[max_boxes * BP_N]
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

TableLayout table_layout(int max_boxes) {
  TableLayout L;
  L.seg_cap = (size_t)max_boxes * BP_N;
  size_t o = 0;
  L.head = o;
  o = a256(o + sizeof(Head));
  L.boxes = o;
  o = a256(o + sizeof(PscBatchBox) * (size_t)max_boxes);
  L.segs = o;
  o = a256(o + 4 * sizeof(Seg) * L.seg_cap);
  L.counters = o;
  L.counter_bytes = a256(16 + 4 * L.seg_cap);
  o += 4 * L.counter_bytes;
  L.total = a256(o);
  return L;
}

// Strided-pass tile width that gives a CTA of kThreads threads.
template <int N> __host__ __device__ constexpr int width_of() { return kThreads / pp::PlanD<N>::LPL; }

template <int N> int tiles_of(int pass, int stage, const PscBatchBox& b) {
  constexpr int W = width_of<N>();
  constexpr int M = pp::PlanD<N>::M, P = pp::PlanD<N>::P;
  constexpr int gx = (M + W - 1) / W;
  using XC = pp::XCfg<float, N>;
  switch (pass) {
    case BP_FAMP: return 1;
    case BP_ZINV: return gx * P;
    case BP_YINV: return gx * N;
    case BP_XPASS: {
      const long long groups = ((long long)N * N + XC::LPW - 1) / XC::LPW;
      const long long per = (long long)XC::WARPS * kXGroupsPerWarp;
      return (int)((groups + per - 1) / per);
    }
    case BP_CFL: return (stage == 1 && b.cfl_on) ? 1 : 0;
    case BP_YFWD: return gx * N;
    case BP_ZFWD: return gx * P;
    case BP_COMBINE: {
      const long long S = (long long)P * P * M, per = (long long)kThreads * kCombinePerThread;
      return (int)((S + per - 1) / per);
    }
    default: return (stage == 4 && b.forcing == 2) ? 1 : 0;
  }
}

// Tiles one work item runs: several small tiles per item keep the per-item
// cost (taking an item, its dependency check, the completion count) small
// against the work.
inline int tiles_per_item(int pass) {
  switch (pass) {
    case BP_ZINV: case BP_YINV: case BP_YFWD: case BP_ZFWD: return 4;
    case BP_XPASS: return 2;
    case BP_COMBINE: return 4;
    default: return 1;
  }
}

template <int N> size_t smem_of() {
  constexpr int W = width_of<N>();
  const size_t a = pp::StridedSmem<float, N, W>::BYTES, x = pp::XCfg<float, N>::SMEM;
  return a > x ? a : x;
}

#define PSCB_SIZES(X) X(32) X(48) X(64) X(96) X(128) X(192) X(256)

int tiles_dispatch(int N, int pass, int stage, const PscBatchBox& b) {
  switch (N) {
#define PSCB_T(n) case n: return tiles_of<n>(pass, stage, b);
    PSCB_SIZES(PSCB_T)
#undef PSCB_T
    default: return 0;
  }
}

// ---------------------------------------------------------------- device side

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int N, int STAGE>
__device__ __forceinline__ void run_item(const PscBatchBox& b, int pass, int tile, int ntiles, int tid,
                                         unsigned char* smem) {
  using namespace psc_persistent;
  constexpr int W = width_of<N>();
  constexpr int LPL = PlanD<N>::LPL;
  constexpr int M = PlanD<N>::M;
  constexpr int gx = (M + W - 1) / W;
  Ctrl* ctrl = static_cast<Ctrl*>(b.ctrl);
  PassArgs a;
  a.d.N = b.N;
  a.d.K = b.K;
  a.d.M = b.M;
  a.d.P = b.P;
  a.d.sph = 0;
  a.d.S = b.S;
  a.d.zs = b.zs;
  a.d.ys = b.ys;
  a.in = STAGE == 1 ? b.U : b.V;
  a.zb = b.zreg;
  a.yb = b.yreg;
  a.xb = b.zreg;  // the z-inverse streams are dead once the y-inverse pass has run
  a.yf = b.yreg;  // the y-inverse streams are dead once the X pass has run
  a.rb = b.zreg;  // the X-pass output is dead once the y-forward pass has run
  a.tw = b.tw;
  a.partials = nullptr;
  a.ctrl = ctrl;
  a.want_umax = STAGE == 1 && b.cfl_on;
  a.phase = nullptr;
  a.shift = 0;
  a.xrow = 0;
  a.st = nullptr;
  const Tctx strided{tid % W, tid / W, tile % gx, tile / gx, W, LPL, gx, smem};
  switch (pass) {
    case BP_FAMP:
      if (tid == 0) {
        if (STAGE == 1 && b.cfl_on) ctrl->umax_bits = 0ull;
        b_famp<float>(a.d, a.in, ctrl, b.kF2, b.eps_inj, b.forcing, STAGE == 1 ? 1 : 0);
      }
      break;
    case BP_ZINV: b_zinv<float, N, false, W>(a, strided); break;
    case BP_YINV: b_yinv<float, N, YMODE_RHS, W>(a, strided); break;
    case BP_XPASS: b_xpass<float, N, XMODE_RHS>(a, Tctx{tid, 0, tile, 0, kThreads, 1, ntiles, smem}); break;
    case BP_CFL:
      // dt for Eq. 10 from the maximum the X pass reduced, then the integrating
      // factors of that dt (K + 1 <= kThreads entries)
      if (tid == 0) b_cfl(ctrl, b.cfl, b.dx, b.record_every);
      __syncthreads();
      b_iftab<float>(b.K, ctrl, b.nu, b.D, static_cast<float*>(b.eu), static_cast<float*>(b.ep), tid);
      break;
    case BP_YFWD: b_yfwd<float, N, W>(a, strided); break;
    case BP_ZFWD: b_zfwd<float, N, W>(a, strided); break;
    case BP_COMBINE: {
      CombineArgs c;
      c.d = a.d;
      c.rb = b.zreg;
      c.rb2 = nullptr;
      c.vin = a.in;
      c.U = b.U;
      c.V = b.V;
      c.Acc = b.Acc;
      c.out = nullptr;
      c.eu = b.eu;
      c.ep = b.ep;
      c.ctrl = ctrl;
      c.kF2 = b.kF2;
      c.beta = b.beta;
      c.nu = b.nu;
      c.D = b.D;
      c.kF2_floor = b.kF2_floor;
      c.forcing = b.forcing;
      c.integrator = b.integrator;
      c.scalar_on = b.scalar_on;
      const long long base = (long long)tile * kThreads * kCombinePerThread;
#pragma unroll 1
      for (int r = 0; r < kCombinePerThread; ++r) b_combine<float, STAGE>(c, base + (long long)r * kThreads + tid);
      break;
    }
    default:
      if (tid == 0) b_hold<float>(a.d, b.U, ctrl, b.kF2);
      break;
  }
}

// BIG: every persistent size; else the sizes up to 128 (a smaller kernel with
// fewer registers for ensembles of small boxes)
template <int STAGE, bool BIG>
__device__ __forceinline__ void dispatch(const PscBatchBox& b, int pass, int tile, int ntiles, int tid,
                                         unsigned char* smem) {
  switch (b.N) {
#define PSCB_D(n) case n: if (BIG || n <= 128) run_item<n, STAGE>(b, pass, tile, ntiles, tid, smem); break;
    PSCB_SIZES(PSCB_D)
#undef PSCB_D
    default: break;
  }
}

// About two seconds: a wait that lasts longer abandons the launch.
constexpr unsigned long long kWaitNs = 2000000000ull;
// The bound under the stall test (a dependency that is never met, see pscb_upload).
constexpr unsigned long long kStallTestWaitNs = 50000000ull;

#ifndef PSCB_MINB
#define PSCB_MINB 3  // CTAs per SM the register budget is sized for
#endif
template <int STAGE, bool BIG>
__global__ void __launch_bounds__(kThreads, PSCB_MINB)
k_batch_stage(const Head* head, const PscBatchBox* boxes, const Seg* segs, unsigned char* counters) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_seg, s_tile;
  unsigned long long* next = reinterpret_cast<unsigned long long*>(counters);
  int* abort_flag = reinterpret_cast<int*>(counters + 8);
  int* done = reinterpret_cast<int*>(counters + 16);
  const int tid = threadIdx.x;
  const int nseg = head->nseg[STAGE - 1];
  const long long nitems = head->nitems[STAGE - 1];
  const unsigned long long wait_ns = head->wait_ns;
  int seg = 0;  // the segments this CTA's items fall in only move forward
  for (;;) {
    if (tid == 0) {
      int out = -1, tile = 0;
      const long long i = (long long)atomicAdd(next, 1ull);
      if (i < nitems && !*(volatile int*)abort_flag) {
        while (seg + 1 < nseg && segs[seg + 1].start <= i) ++seg;
        const Seg& g = segs[seg];
        bool ok = true;
        if (g.dep >= 0 && ld_acquire(&done[g.dep]) < g.dep_tiles) {
          const unsigned long long t0 = pp::global_ns();
          for (unsigned k = 1;; ++k) {
            if (ld_acquire(&done[g.dep]) >= g.dep_tiles) break;
            if ((k & 63u) == 0) {
              if (*(volatile int*)abort_flag) { ok = false; break; }
              if (pp::global_ns() - t0 > wait_ns) {
                ok = false;
                atomicExch(abort_flag, 1);
                atomicOr(&static_cast<pp::Ctrl*>(boxes[g.box].ctrl)->err, 4);
                break;
              }
            }
          }
        }
        if (ok) {
          out = seg;
          tile = (int)(i - g.start);
        }
      }
      s_seg = out;
      s_tile = tile;
    }
    __syncthreads();
    const int sg = s_seg, item = s_tile;
    if (sg < 0) break;
    // The producers' writes are ordered before thread 0's acquire, and the
    // barrier orders that before every thread's reads.  This unit is built
    // with global loads cached in L2 only (-dlcm=cg), so no SM keeps a stale
    // L1 copy of a buffer another CTA has since rewritten.
    const Seg& g = segs[sg];
    for (int t = item * g.per; t < (item + 1) * g.per && t < g.tiles; ++t) {
      dispatch<STAGE, BIG>(boxes[g.box], g.pass, t, g.tiles, tid, smraw);
      if (g.per > 1) __syncthreads();  // bodies reuse the shared memory
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(&done[g.done_idx], 1);
    }
  }
}

}  // namespace
