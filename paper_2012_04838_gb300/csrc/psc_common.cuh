// Device helpers shared by the kernels: complex arithmetic, the two-step FFT
// plans per grid size, and optional index checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "psc_internal.h"
#include "codelets.cuh"

namespace psc {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

// Complex products with the fused multiply-add written out (one product
// rounded, the other fused), so every kernel that multiplies by a twiddle
// rounds the same way whatever the compiler would contract on its own.
__device__ __forceinline__ float fmul_exact_order(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul_exact_order(double a, double b) { return __dmul_rn(a, b); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(fma(a.x, b.x, -fmul_exact_order(a.y, b.y)), fma(a.x, b.y, fmul_exact_order(a.y, b.x)));
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(fma(a.x, b.x, fmul_exact_order(a.y, b.y)), fma(a.y, b.x, -fmul_exact_order(a.x, b.y)));
}
// i * k * a.  The products are rounded on their own (never fused into a
// following addition), so every kernel variant that forms a derivative this
// way produces the same bits whatever the compiler contracts around it.
__device__ __forceinline__ float2 mul_ik(float2 a, float k) {
  return make_float2(__fmul_rn(-k, a.y), __fmul_rn(k, a.x));
}
__device__ __forceinline__ double2 mul_ik(double2 a, double k) {
  return make_double2(__dmul_rn(-k, a.y), __dmul_rn(k, a.x));
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <class C, typename T> __device__ __forceinline__ C cscale(C a, T s) {
  return mk(a.x * s, a.y * s);
}

// Two-step Cooley-Tukey plan for a line of length N = R1 * R2:
//   step 1: R2 DFTs of size R1 over the stride-R2 subsequences, twiddle
//           exp(s 2 pi i n2 k1 / N), exchange through shared memory;
//   step 2: R1 DFTs of size R2.
// TPL threads cooperate on one line: each runs J1 = R2/TPL step-1 DFTs and
// J2 = R1/TPL step-2 DFTs, so it holds N/TPL values at a time.
template <int N> struct Plan;
#define PSC_PLAN(N_, R1_, R2_, TPL_)                         \
  template <> struct Plan<N_> {                              \
    static constexpr int R1 = R1_, R2 = R2_, TPL = TPL_;     \
  };
PSC_PLAN(8, 4, 2, 2)
PSC_PLAN(12, 4, 3, 1)
PSC_PLAN(16, 4, 4, 4)
PSC_PLAN(24, 6, 4, 2)
PSC_PLAN(32, 8, 4, 4)
PSC_PLAN(48, 12, 4, 4)
PSC_PLAN(64, 8, 8, 8)
PSC_PLAN(96, 12, 8, 4)
PSC_PLAN(128, 16, 8, 8)
PSC_PLAN(192, 24, 8, 8)
PSC_PLAN(256, 16, 16, 16)
PSC_PLAN(512, 32, 16, 16)
PSC_PLAN(520, 20, 26, 2)
PSC_PLAN(1024, 32, 32, 32)
#undef PSC_PLAN

template <int N> struct PlanD : Plan<N> {
  static constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2, TPL = Plan<N>::TPL;
  static constexpr int J1 = R2 / TPL, J2 = R1 / TPL;
  static constexpr int K = (N - 1) / 3, M = K + 1, P = 2 * K + 1;
  // Lines whose lanes would loop more than four times (N = 520 over two lanes)
  // are transformed "wide" by the strided passes: R2 lanes take the first step
  // (one length-R1 DFT each), R1 lanes the second.
  static constexpr bool WIDE = J1 > 4 || J2 > 4;
  static constexpr int LPL = WIDE ? (R1 > R2 ? R1 : R2) : TPL;  // lanes per line
  static_assert(R1 * R2 == N, "plan must factor N");
  static_assert(R1 % TPL == 0 && R2 % TPL == 0, "TPL must divide both radices");
  static_assert(32 % TPL == 0, "a line's threads must sit inside one warp");
};

// Thread and block coordinates of a kernel body: the hardware's in an ordinary
// launch, or virtual ones when the persistent ensemble kernel runs the body as
// one item of its work table (then the body must not rely on gridDim beyond gdx).
struct Tctx {
  int tx, ty, bx, by, bdx, bdy, gdx;
  unsigned char* smem;  // the body's dynamic shared memory
};
__device__ __forceinline__ Tctx hw_ctx(unsigned char* smem) {
  return Tctx{(int)threadIdx.x, (int)threadIdx.y, (int)blockIdx.x, (int)blockIdx.y,
              (int)blockDim.x,  (int)blockDim.y,  (int)gridDim.x,  smem};
}

// Pointer qualifier of pass inputs: __restrict__ in ordinary launches.  The
// persistent ensemble kernel reads buffers that other CTAs of the same launch
// wrote, so it compiles the bodies without it (no non-coherent loads).
#ifndef PSC_RESTRICT
#define PSC_RESTRICT __restrict__
#endif

// f(std::integral_constant<int, I>) for I = B .. E-1, each index a compile-time constant
template <int B, int E, class F> __device__ __forceinline__ void static_for(const F& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Per-thread running sum of one statistics moment.  The FP64 path sums in
// FP64; the FP32 path keeps a compensated FP32 sum (Kahan 1965: the rounding
// error of each addition is carried into the next), whose error stays within
// a few units of FP32 rounding of the sum of magnitudes however many terms it
// takes, at FP32 cost (FP64 arithmetic runs at a small fraction of the FP32
// rate on this part).
template <typename T> struct MomentSum;
template <> struct MomentSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct MomentSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// running maximum that keeps a NaN once one is seen
template <typename T> __device__ __forceinline__ T max_keep_nan(T m, T v) {
  return v > m || v != v ? v : m;
}

// Bulk asynchronous copies (TMA engine) into shared memory, completed on an
// mbarrier.  A wait gives up after a bounded number of polls and reports it.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// make barrier initialisation visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses (and those the last
// barrier made visible to it) before later asynchronous-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase of parity `parity` to complete; false once limit_ns
// (about two seconds by default) have passed (a time bound, whatever each
// poll's own suspend time), or as soon as bit 2 of *abort is seen set
// (another wait already gave up)
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          const int* abort = nullptr,
                                          unsigned long long limit_ns = 2000000000ull) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if ((i & 255u) == 0) {
      if (abort && (*(const volatile int*)abort & 4)) return false;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
}
// one arrival on an mbarrier (release: this thread's earlier accesses first)
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// AND of `pred` over the `count` threads of named barrier `id` (a barrier too)
__device__ __forceinline__ bool bar_and(int id, int count, bool pred) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Optional index checks (build with -DPSC_CHECKED=1): an out-of-range global
// index is not accessed; bit 0 of Ctrl::err is raised instead.
#ifndef PSC_CHECKED
#define PSC_CHECKED 0
#endif
#if PSC_CHECKED
#define PSC_OK_INDEX(idx, n, ctrl) \
  (((idx) >= 0 && (idx) < (n)) ? true : (atomicOr(&(ctrl)->err, 1), false))
#else
#define PSC_OK_INDEX(idx, n, ctrl) true
#endif

}  // namespace psc
