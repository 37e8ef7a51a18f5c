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

template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// i * k * a
template <class C, typename T> __device__ __forceinline__ C mul_ik(C a, T k) {
  return mk(-k * a.y, k * a.x);
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
PSC_PLAN(1024, 32, 32, 32)
#undef PSC_PLAN

template <int N> struct PlanD : Plan<N> {
  static constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2, TPL = Plan<N>::TPL;
  static constexpr int J1 = R2 / TPL, J2 = R1 / TPL;
  static constexpr int K = (N - 1) / 3, M = K + 1, P = 2 * K + 1;
  static_assert(R1 * R2 == N, "plan must factor N");
  static_assert(R1 % TPL == 0 && R2 % TPL == 0, "TPL must divide both radices");
  static_assert(32 % TPL == 0, "a line's threads must sit inside one warp");
};

// f(std::integral_constant<int, I>) for I = B .. E-1, each index a compile-time constant
template <int B, int E, class F> __device__ __forceinline__ void static_for(const F& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Positions j + TH m (j < TH) of a length-N line split into 16 slots of TH:
// 1 if every such position is retained (|k| <= K), 0 if none is, 2 if mixed.
__host__ __device__ constexpr int band_of(int N, int TH, int m) {
  return (TH * m + TH - 1 <= (N - 1) / 3 || TH * m >= N - (N - 1) / 3) ? 1
         : (TH * m > (N - 1) / 3 && TH * m + TH - 1 < N - (N - 1) / 3) ? 0
                                                                      : 2;
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
