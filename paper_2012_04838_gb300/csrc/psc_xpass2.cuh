// X pass for N = 16 * 16 * G (G = 2: N = 512, G = 4: N = 1024).
//
// One row of N points is transformed by TH = 16 G threads holding 16 values
// each.  With n = a + 16 b + 256 c and k = k0 + G k1 + 16 G k2
// (a, b, k1, k2 < 16; c, k0 < G) the DFT factors into
//   X[k] = sum_a w16^(a k2) wN^(a (k0 + G k1)) sum_b w16^(b k1) wN^(16 b k0)
//          sum_c wG^(c k0) x[a + 16 b + 256 c],
// so a transform is: a DFT of size G across G adjacent lanes (shuffles), a
// DFT-16 in registers, one exchange through shared memory, a second DFT-16.
// The inverse runs the same steps in the opposite order, which leaves every
// physical value on the lane and register the forward transform starts from:
// thread (a, r) holds x[a + 16 b + 256 r], b < 16, for every field, so the
// products u x omega and u . grad phi are formed in registers and no field is
// parked in shared memory.  Registers per thread stay near a hundred, which
// keeps 4x more rows in flight per SM than one warp per row of 32 values.
#pragma once

#include "psc_common.cuh"

namespace psc {

template <typename T, int N> struct X2Cfg {
  using C = typename CT<T>::type;
  static constexpr int G = N / 256;
  static constexpr int TH = 16 * G;      // threads per row
  static constexpr int ROWS = 128 / TH;  // rows per 128-thread CTA
  // exchange rows of 16 G values padded to 17 G: the (a, k0 + G k1) accesses
  // of 32 lanes then fall in distinct bank groups
  static constexpr int ROW = 17 * G;
  static constexpr int EXCH = 16 * ROW > N ? 16 * ROW : N;
  static constexpr size_t LINE_BYTES = (EXCH * sizeof(C) + 15) / 16 * 16;
  static constexpr size_t ACC_BYTES = 4 * NQ * sizeof(double);
  // per-role twiddle tables (every row of the CTA uses the same thread roles):
  //   T1[a][tid]  = wN^(a tid)             (inverse step after the first DFT-16)
  //   T3[k1][tid] = wN^(ra (rk0 + G k1))   (forward step before the exchange)
  //   T2[b][k0]   = wN^(16 b k0)           (between the lane DFT and the DFT-16 over b)
  // laid out so the 32 lanes of a warp read consecutive entries (FP32: pairs
  // of consecutive a, k1 or b side by side, see tw_index)
  static constexpr size_t TW_BYTES = (size_t)(2 * 16 * TH + 16 * G) * sizeof(C);
  static constexpr size_t SMEM = LINE_BYTES * ROWS + ACC_BYTES + TW_BYTES;
  static constexpr int K = (N - 1) / 3;
  static_assert(N == 512 || N == 1024, "X2 layout covers N = 512 and 1024");
};

// Positions j + TH m (j < TH) of a length-N line split into 16 slots of TH,
// for the retained half-width K: 1 if every such position is retained, 0 if
// none is, 2 if mixed.
__host__ __device__ constexpr int band_of_k(int N, int TH, int m, int K) {
  return (TH * m + TH - 1 <= K || TH * m >= N - K) ? 1 : (TH * m > K && TH * m + TH - 1 < N - K) ? 0 : 2;
}

// barrier over the TH threads of one row
template <int TH> __device__ __forceinline__ void row_sync(int id) {
  if constexpr (TH == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(TH) : "memory");
  }
}

template <int G> __device__ __forceinline__ int bitrev_lane(int r) {
  if constexpr (G == 4) return ((r & 1) << 1) | (r >> 1);
  else return r;
}

// DFT of size G across the G adjacent lanes of a group, element-wise on v.
// Forward (DIR = -1): lane r holds input c = r and ends with output k0 = bitrev(r).
// Inverse (DIR = +1): lane r holds input k0 = bitrev(r) and ends with c = r.
template <typename T, int G, int DIR>
__device__ __forceinline__ void lane_dft(typename CT<T>::type (&v)[16], int r) {
  using C = typename CT<T>::type;
  // the upper lane of a pair forms o - v, the lower v + o: one fused
  // multiply-add by a per-lane sign, fma(-1, v, o) = o - v and fma(1, v, o) =
  // v + o exactly, instead of both sums and a select
  auto bfly = [&](int mask, bool upper) {
    const T sg = upper ? T(-1) : T(1);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const C o = mk(__shfl_xor_sync(0xffffffffu, v[i].x, mask), __shfl_xor_sync(0xffffffffu, v[i].y, mask));
      v[i] = mk(fma(sg, v[i].x, o.x), fma(sg, v[i].y, o.y));
    }
  };
  auto quarter = [&]() {  // multiply by exp(DIR * 2 pi i / 4) on the lane with both bits set
    if (r == 3) {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = DIR < 0 ? mk(v[i].y, -v[i].x) : mk(-v[i].y, v[i].x);
    }
  };
  if constexpr (G == 2) {
    bfly(1, r & 1);
  } else if constexpr (DIR < 0) {
    bfly(2, r & 2);
    quarter();
    bfly(1, r & 1);
  } else {
    bfly(1, r & 1);
    quarter();
    bfly(2, r & 2);
  }
}

// The first DFT-16 of an inverse transform: slots m whose 16 G positions all
// lie in the zero band for every thread (band_of_k == 0) are known zeros, and
// the pruned codelet DftZ<16, +1, Z0, Z1> skips them (the generator emits it
// for slots 6..9, the band of the 2/3 rule at N = 512 and 1024); a plain
// DFT-16 otherwise.  Adding a known zero is left out, so the sums are the same.
template <int N, int KK> struct x2_first_inverse {
  static constexpr int TH = X2Cfg<float, N>::TH;
  static constexpr int first() {
    for (int m = 0; m < 16; ++m)
      if (band_of_k(N, TH, m, KK) == 0) return m;
    return 16;
  }
  static constexpr int last() {
    for (int m = 15; m >= 0; --m)
      if (band_of_k(N, TH, m, KK) == 0) return m;
    return -1;
  }
  static constexpr bool PRUNED = first() == 6 && last() == 9;
  template <typename T, typename C> static __device__ __forceinline__ void run(C (&v)[16]) {
    if constexpr (PRUNED) DftZ<16, +1, 6, 9>::template run<T, C>(v);
    else Dft<16, +1>::template run<T, C>(v);
  }
};

template <typename C> struct X2Roles {
  int tid;  // thread within the row: inverse input / forward output column j
  int ra;   // a of the (a, r) role
  int rr;   // r of the (a, r) role (lane within the G-group)
  int rk0;  // k0 held by lane rr between the lane DFT and the DFT-16 over b
  int bar;  // named barrier of this row
  const C* t1;  // shared twiddle tables, see X2Cfg
  const C* t2;
  const C* t3;
};

// Twiddle tables hold entries (e, j) (e < 16: a, b or k1; j: the thread's
// column) in pairs of consecutive e for FP32, so one 128-bit shared load
// brings the twiddles of e and e + 1; FP64 entries are 16 bytes already.
template <typename T, int J> __device__ __forceinline__ int tw_index(int e, int j) {
  if constexpr (sizeof(T) == 4) return (((e >> 1) * J + j) << 1) | (e & 1);
  else return e * J + j;
}
// the twiddles of e and e + 1 (e even) for column j
template <typename T, int J>
__device__ __forceinline__ void tw_pair(const typename CT<T>::type* t, int e, int j, typename CT<T>::type& w0,
                                        typename CT<T>::type& w1) {
  if constexpr (sizeof(T) == 4) {
    const float4 p = *reinterpret_cast<const float4*>(t + tw_index<T, J>(e, j));
    w0 = make_float2(p.x, p.y);
    w1 = make_float2(p.z, p.w);
  } else {
    w0 = t[tw_index<T, J>(e, j)];
    w1 = t[tw_index<T, J>(e + 1, j)];
  }
}

// Inverse transform of a Hermitian-packed half spectrum (two real fields):
// Z[p] = X1[p] + i X2[p] (p <= K, imaginary parts dropped at p = 0),
// conj(X1[N-p]) + i conj(X2[N-p]) (p >= N-K), 0 elsewhere.  On return
// z[b] = scale * IDFT(Z) at n = ra + 16 b + 256 rr (SCALE = false: the
// unscaled IDFT; the caller folds 1/N^3 into its products).
template <typename T, int N, bool SCALE = true, int KK = (N - 1) / 3, bool SHIFT = false, class SPEC>
__device__ __forceinline__ void x2inv(const SPEC& spec, typename CT<T>::type (&z)[16],
                                      typename CT<T>::type* ex, const X2Roles<typename CT<T>::type>& q,
                                      T scale, const void* phase = nullptr) {
  using C = typename CT<T>::type;
  using XC = X2Cfg<T, N>;
  constexpr int TH = XC::TH, G = XC::G, ROW = XC::ROW, K = KK;
  C v[16];
  // slots whose positions all lie in the zero band load nothing; slots wholly
  // inside [0, K] or [N-K, N) need no range test
  static_for<0, 16>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    constexpr int band = band_of_k(N, TH, m, K);
    constexpr bool low = TH * m <= K;  // slot starts in [0, K]
    const int p = q.tid + TH * m;
    C x1, x2;
    // the half spectra at k >= 0, times exp(i k pi / N) on the shifted grid
    auto get = [&](int k) {
      spec(k, x1, x2);
      x1 = shift_in<SHIFT, KK>(x1, phase, k);
      x2 = shift_in<SHIFT, KK>(x2, phase, k);
    };
    if constexpr (band == 0) {
      v[m] = mk(T(0), T(0));
    } else if constexpr (band == 1 && low) {
      get(p);
      if (m == 0 && p == 0) { x1.y = T(0); x2.y = T(0); }
      v[m] = mk(x1.x - x2.y, x1.y + x2.x);
    } else if constexpr (band == 1) {
      get(N - p);
      v[m] = mk(x1.x + x2.y, x2.x - x1.y);
    } else {
      if (p <= K) {
        get(p);
        if (m == 0 && p == 0) { x1.y = T(0); x2.y = T(0); }
        v[m] = mk(x1.x - x2.y, x1.y + x2.x);
      } else if (p >= N - K) {
        get(N - p);
        v[m] = mk(x1.x + x2.y, x2.x - x1.y);
      } else {
        v[m] = mk(T(0), T(0));
      }
    }
  });
  x2_first_inverse<N, KK>::template run<T, C>(v);  // over k2 -> a
#pragma unroll
  for (int a = 0; a < 16; a += 2) {
    C w0, w1;
    tw_pair<T, TH>(q.t1, a, q.tid, w0, w1);
    const C u0 = a > 0 ? cmulc(v[a], w0) : v[a];  // wN^(-a j)
    ex[a * ROW + q.tid] = u0;
    ex[(a + 1) * ROW + q.tid] = cmulc(v[a + 1], w1);
  }
  row_sync<TH>(q.bar);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) z[k1] = ex[q.ra * ROW + q.rk0 + G * k1];
  row_sync<TH>(q.bar);
  Dft<16, +1>::template run<T, C>(z);  // over k1 -> b
  if (q.rk0 > 0) {
#pragma unroll
    for (int b = 0; b < 16; b += 2) {  // wN^(-16 b k0)
      C w0, w1;
      tw_pair<T, G>(q.t2, b, q.rk0, w0, w1);
      if (b > 0) z[b] = cmulc(z[b], w0);
      z[b + 1] = cmulc(z[b + 1], w1);
    }
  }
  lane_dft<T, G, +1>(z, q.rr);  // over k0 -> c
  if constexpr (SCALE) {
#pragma unroll
    for (int b = 0; b < 16; ++b) z[b] = cscale(z[b], scale);
  }
}

// Forward transform of two real fields packed as x1 + i x2 at the positions
// x2inv leaves them in; out(kx, X1, X2) receives both half spectra for kx <= K.
template <typename T, int N, int KK = (N - 1) / 3, bool SHIFT = false, class OUT>
__device__ __forceinline__ void x2fwd(typename CT<T>::type (&z)[16], const OUT& out,
                                      typename CT<T>::type* ex, const X2Roles<typename CT<T>::type>& q,
                                      const void* phase = nullptr) {
  using C = typename CT<T>::type;
  using XC = X2Cfg<T, N>;
  constexpr int TH = XC::TH, G = XC::G, ROW = XC::ROW, K = KK;
  lane_dft<T, G, -1>(z, q.rr);  // over c -> k0
  if (q.rk0 > 0) {
#pragma unroll
    for (int b = 0; b < 16; b += 2) {  // wN^(16 b k0)
      C w0, w1;
      tw_pair<T, G>(q.t2, b, q.rk0, w0, w1);
      if (b > 0) z[b] = cmul(z[b], w0);
      z[b + 1] = cmul(z[b + 1], w1);
    }
  }
  Dft<16, -1>::template run<T, C>(z);  // over b -> k1
#pragma unroll
  for (int k1 = 0; k1 < 16; k1 += 2) {
    C w0, w1;
    tw_pair<T, TH>(q.t3, k1, q.tid, w0, w1);  // wN^(a (k0 + G k1))
    const int j = q.rk0 + G * k1;
    C u0 = z[k1];
    if (q.ra > 0 && j > 0) u0 = cmul(u0, w0);
    ex[q.ra * ROW + j] = u0;
    C u1 = z[k1 + 1];
    if (q.ra > 0) u1 = cmul(u1, w1);
    ex[q.ra * ROW + j + G] = u1;
  }
  row_sync<TH>(q.bar);
  C v[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) v[a] = ex[a * ROW + q.tid];
  row_sync<TH>(q.bar);
  Dft<16, -1>::template run<T, C>(v);  // over a -> k2
  // natural order; outputs that can never be retained are not stored (and so
  // not computed)
  static_for<0, 16>([&](auto kc) {
    constexpr int k2 = decltype(kc)::value;
    if constexpr (band_of_k(N, TH, k2, K) != 0) ex[q.tid + TH * k2] = v[k2];
  });
  row_sync<TH>(q.bar);
  for (int kx = q.tid; kx <= K; kx += TH) {
    const C A = ex[kx];
    const C B = ex[kx == 0 ? 0 : N - kx];
    out(kx, shift_out<SHIFT, KK>(mk(T(0.5) * (A.x + B.x), T(0.5) * (A.y - B.y)), phase, kx),
        shift_out<SHIFT, KK>(mk(T(0.5) * (A.y + B.y), T(0.5) * (B.x - A.x)), phase, kx));
  }
  row_sync<TH>(q.bar);
}

// Fill the per-role twiddle tables T1, T3, T2 (see X2Cfg) at `t1` and point
// the roles at them; ends with a CTA barrier.
template <typename T, int N>
__device__ __forceinline__ void x2_twiddles(typename CT<T>::type* t1, const typename CT<T>::type* __restrict__ tw,
                                            X2Roles<typename CT<T>::type>& q) {
  using C = typename CT<T>::type;
  constexpr int TH = X2Cfg<T, N>::TH, G = X2Cfg<T, N>::G;
  C* t3 = t1 + 16 * TH;
  C* t2 = t3 + 16 * TH;
  for (int i = threadIdx.x; i < 16 * TH; i += blockDim.x) {
    const int e = i / TH, tid = i % TH;  // e = a for T1, k1 for T3
    const int ra = tid / G, rk0 = bitrev_lane<G>(tid % G);
    t1[tw_index<T, TH>(e, tid)] = tw[e * tid];
    t3[tw_index<T, TH>(e, tid)] = tw[ra * (rk0 + G * e)];
  }
  for (int i = threadIdx.x; i < 16 * G; i += blockDim.x) t2[tw_index<T, G>(i / G, i % G)] = tw[16 * (i / G) * (i % G)];
  q.t1 = t1;
  q.t2 = t2;
  q.t3 = t3;
  __syncthreads();
}

// Right-hand side of one row (z, y): five inverse transforms of packed field
// pairs, u x omega and u . grad phi in registers, two forward transforms.
// Y(s, kx) reads stream s at kx.  after_a() runs once streams UX..DYUX are no
// longer read, wait_b() before PHI..DZPHI are first read (false aborts the
// row), after_b() once those are no longer read.  Returns false if aborted.
template <typename T, int N, bool PRESSURE = false, int KK = (N - 1) / 3, bool SHIFT = false, class YF, class HA,
          class WB, class HB>
__device__ __forceinline__ bool x2_rhs_row(const YF& Y, const HA& after_a, const WB& wait_b, const HB& after_b,
                                           typename CT<T>::type* __restrict__ xb, long long line, long long ys,
                                           typename CT<T>::type* ex, const X2Roles<typename CT<T>::type>& q,
                                           T scale, bool want_umax, T& um, Ctrl* ctrl,
                                           const void* phase = nullptr) {
  using C = typename CT<T>::type;
  constexpr int M = KK + 1;
  const C zero = mk(T(0), T(0));
  (void)ctrl;
  C z[16];
  // the inverse transforms are left unscaled (N^3 times the fields); each
  // product carries the missing 1/N^6 once
  const T s2 = scale * scale;
  // live per thread at most: u1, u2, u3 and one more field (64 values)
  T u1[16], u2[16], u3[16], W[16];
  // (u1, u2)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UY, kx); }, z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) { u1[b] = z[b].x; u2[b] = z[b].y; }
  // (u3, omega1)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UZ, kx); x2 = Y(Y_WX, kx); }, z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    u3[b] = z[b].x;
    W[b] = z[b].y;  // omega1
    if (want_umax) um = max_keep_nan(um, fabs(u1[b]) + fabs(u2[b]) + fabs(u3[b]));
  }
  // (omega2, omega3): omega2 = d_z u1 - i kx u3, omega3 = i kx u2 - d_y u1
  x2inv<T, N, false, KK, SHIFT>(
      [&](int kx, C& x1, C& x2) {
        x1 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx)));
        x2 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
      },
      z, ex, q, scale, phase);
  after_a();
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const T w1 = W[b], w2 = z[b].x, w3 = z[b].y;
    z[b] = mk((u2[b] * w3 - u3[b] * w2) * s2, (u3[b] * w1 - u1[b] * w3) * s2);  // (NL1, NL2)
    W[b] = u1[b] * w2 - u2[b] * w1;                                              // NL3
  }
  x2fwd<T, N, KK, SHIFT>(z,
              [&](int kx, C X1, C X2) {
                const long long i0 = line * M + kx;
                if (PSC_OK_INDEX(i0 + ys, 4 * ys, ctrl)) { xb[i0] = X1; xb[i0 + ys] = X2; }
              },
              ex, q, phase);
  if constexpr (PRESSURE) {
    // (NL3, |u|^2 / 2): the inputs of the modified pressure
#pragma unroll
    for (int b = 0; b < 16; ++b)
      z[b] = mk(W[b] * s2, T(0.5) * (u1[b] * u1[b] + u2[b] * u2[b] + u3[b] * u3[b]) * s2);
    x2fwd<T, N, KK, SHIFT>(z,
                [&](int kx, C X1, C X2) {
                  const long long i0 = 2 * ys + line * M + kx;
                  if (PSC_OK_INDEX(i0 + ys, 4 * ys, ctrl)) { xb[i0] = X1; xb[i0 + ys] = X2; }
                },
                ex, q, phase);
    return true;
  }
  if (!wait_b()) return false;
  // (dphi/dx1, dphi/dx2); u1 then holds the partial u . grad phi
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_PHI, kx), T(kx)); x2 = Y(Y_DYPHI, kx); },
                     z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) u1[b] = u1[b] * z[b].x + u2[b] * z[b].y;
  // (dphi/dx3, 0)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZPHI, kx); x2 = zero; }, z, ex, q, scale, phase);
  after_b();
#pragma unroll
  for (int b = 0; b < 16; ++b) z[b] = mk(W[b] * s2, (u1[b] + u3[b] * z[b].x) * s2);  // (NL3, u.grad phi)
  x2fwd<T, N, KK, SHIFT>(z,
              [&](int kx, C X1, C X2) {
                const long long i0 = 2 * ys + line * M + kx;
                if (PSC_OK_INDEX(i0 + ys, 4 * ys, ctrl)) { xb[i0] = X1; xb[i0 + ys] = X2; }
              },
              ex, q, phase);
  return true;
}

// The convective form of one row: -(u.grad)u and u.grad phi from u, its nine
// gradients and grad phi (8 inverse transforms of packed pairs, 2 forward).
// With this stream set Y_WX holds d_y u_z and Y_DZUY holds d_z u_y.  The
// hooks as in x2_rhs_row: after_a() once UX, UY, UZ, DZUX, DYUX, DYUY and DZUY
// are no longer read, wait_b() before WX, PHI, DYPHI, DZPHI and DZUZ are first
// read (false aborts the row), after_b() once those are no longer read.
// Returns false if aborted.
template <typename T, int N, int KK = (N - 1) / 3, bool SHIFT = false, class YF, class HA, class WB, class HB>
__device__ __forceinline__ bool x2_conv_row(const YF& Y, const HA& after_a, const WB& wait_b, const HB& after_b,
                                            typename CT<T>::type* __restrict__ xb, long long line,
                                            long long ys, typename CT<T>::type* ex,
                                            const X2Roles<typename CT<T>::type>& q, T scale, bool want_umax, T& um,
                                            Ctrl* ctrl, const void* phase = nullptr) {
  using C = typename CT<T>::type;
  constexpr int M = KK + 1;
  const C zero = mk(T(0), T(0));
  (void)ctrl;
  C z[16];
  const T s2 = scale * scale;  // the transforms are unscaled: each product carries 1/N^6
  T u1[16], u2[16], u3[16], A[16], B[16];
  auto out = [&](int s0) {
    return [&, s0](int kx, C X1, C X2) {
      const long long i0 = s0 * ys + line * M + kx;
      if (PSC_OK_INDEX(i0 + ys, 4 * ys, ctrl)) { xb[i0] = X1; xb[i0 + ys] = X2; }
    };
  };
  // (u1, u2)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UY, kx); }, z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) { u1[b] = z[b].x; u2[b] = z[b].y; }
  // (u3, d1 u1)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UZ, kx); x2 = mul_ik(Y(Y_UX, kx), T(kx)); }, z, ex, q,
                     scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    u3[b] = z[b].x;
    A[b] = u1[b] * z[b].y;
    if (want_umax) um = max_keep_nan(um, fabs(u1[b]) + fabs(u2[b]) + fabs(u3[b]));
  }
  // (d2 u1, d3 u1): A = (u.grad) u1
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYUX, kx); x2 = Y(Y_DZUX, kx); }, z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) A[b] += u2[b] * z[b].x + u3[b] * z[b].y;
  // (d1 u2, d2 u2)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UY, kx), T(kx)); x2 = Y(Y_DYUY, kx); }, z, ex, q,
                     scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) B[b] = u1[b] * z[b].x + u2[b] * z[b].y;
  // (d3 u2, d1 u3): B = (u.grad) u2; A starts (u.grad) u3
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUY, kx); x2 = mul_ik(Y(Y_UZ, kx), T(kx)); }, z, ex, q,
                     scale, phase);
  after_a();
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const T b2 = B[b] + u3[b] * z[b].x, c3 = u1[b] * z[b].y;
    z[b] = mk(-A[b] * s2, -b2 * s2);  // (NL1, NL2)
    A[b] = c3;
  }
  x2fwd<T, N, KK, SHIFT>(z, out(0), ex, q, phase);
  if (!wait_b()) return false;
  // (d2 u3, d3 u3): A = (u.grad) u3
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_WX, kx); x2 = Y(Y_DZUZ, kx); }, z, ex, q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) A[b] += u2[b] * z[b].x + u3[b] * z[b].y;
  // (dphi/dx1, dphi/dx2)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_PHI, kx), T(kx)); x2 = Y(Y_DYPHI, kx); }, z, ex,
                     q, scale, phase);
#pragma unroll
  for (int b = 0; b < 16; ++b) B[b] = u1[b] * z[b].x + u2[b] * z[b].y;
  // (dphi/dx3, 0)
  x2inv<T, N, false, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZPHI, kx); x2 = zero; }, z, ex, q, scale, phase);
  after_b();
#pragma unroll
  for (int b = 0; b < 16; ++b) z[b] = mk(-A[b] * s2, (B[b] + u3[b] * z[b].x) * s2);  // (NL3, u.grad phi)
  x2fwd<T, N, KK, SHIFT>(z, out(2), ex, q, phase);
  return true;
}

template <typename T>
__device__ __forceinline__ double warp_sum_d(T v) {
  double d = (double)v;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  return d;
}

#ifndef PSC_X2_MINB
#define PSC_X2_MINB 4
#endif
template <typename T, int N, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 2 : PSC_X2_MINB) k_xpass2(PassArgs a) {
  using C = typename CT<T>::type;
  using XC = X2Cfg<T, N>;
  constexpr int TH = XC::TH, G = XC::G, ROWS = XC::ROWS, M = KK + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lid = threadIdx.x / TH;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  X2Roles<C> q;
  q.tid = threadIdx.x % TH;
  q.ra = q.tid / G;
  q.rr = q.tid % G;
  q.rk0 = bitrev_lane<G>(q.rr);
  q.bar = 1 + lid;
  C* ex = reinterpret_cast<C*>(smraw + (size_t)lid * XC::LINE_BYTES);
  double* accw = reinterpret_cast<double*>(smraw + XC::LINE_BYTES * ROWS) + wid * NQ;
  const C* __restrict__ yb = static_cast<const C*>(a.yb);
  C* __restrict__ xb = static_cast<C*>(a.xb);
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  x2_twiddles<T, N>(reinterpret_cast<C*>(smraw + XC::LINE_BYTES * ROWS + XC::ACC_BYTES), tw, q);
  // rows and the stream stride come from the arguments (N*N rows for a pass over the box)
  const long long ys = a.d.ys;
  const long long nlines = ys / M;
  const T scale = T(1.0 / ((double)N * N * N));
  const C zero = mk(T(0), T(0));
  // maximum of |u1|+|u2|+|u3| over the thread's points (unscaled fields in the
  // RHS variant, scaled in the statistics variant)
  T um = T(0);
  MomentSum<T> acc[MODE == XMODE_STATS ? NQ : 1];

#pragma unroll 1
  for (long long base = (long long)blockIdx.x * ROWS; base < nlines; base += (long long)gridDim.x * ROWS) {
    const long long line = base + lid;  // the row count (N*N, or a probe's multiple of 64) is a multiple of ROWS
    const C* __restrict__ row = yb + line * M;
    auto Y = [&](int s, int kx) -> C {
      if (!PSC_OK_INDEX(s * ys + line * M + kx, (long long)Y_NSTREAM * ys, a.ctrl)) return zero;
      return row[s * ys + kx];
    };
    C z[16];
    if constexpr (MODE == XMODE_RHS || MODE == XMODE_PRESSURE) {
      x2_rhs_row<T, N, MODE == XMODE_PRESSURE, KK, SHIFT>(Y, [] {}, [] { return true; }, [] {}, xb, line, ys, ex, q,
                                                          scale, a.want_umax != 0, um, a.ctrl, a.phase);
    } else if constexpr (MODE == XMODE_CONVECTIVE) {
      x2_conv_row<T, N, KK, SHIFT>(Y, [] {}, [] { return true; }, [] {}, xb, line, ys, ex, q, scale,
                                   a.want_umax != 0, um, a.ctrl, a.phase);
    } else {
      // statistics (Eqs. 11-13): per pair, partial sums of the thread's 16
      // points, added in FP64 to the thread's accumulators (reduced over the
      // warp once, at the end)
      T s13[16];
      auto put = [&](int slot, T v) { acc[slot].add(v); };
      auto mom3 = [&](int slot, const T (&f)[16]) {
        T m2 = T(0), m3 = T(0), m4 = T(0);
#pragma unroll
        for (int b = 0; b < 16; ++b) { const T v2 = f[b] * f[b]; m2 += v2; m3 += v2 * f[b]; m4 += v2 * v2; }
        put(slot, m2); put(slot + 1, m3); put(slot + 2, m4);
      };
      T f1[16], f2[16];
      auto split = [&]() {
#pragma unroll
        for (int b = 0; b < 16; ++b) { f1[b] = z[b].x; f2[b] = z[b].y; }
      };
      // (u1, u3)
      x2inv<T, N, true, KK>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UZ, kx); }, z, ex, q, scale);
      split();
      {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < 16; ++b) { s += f1[b] * f1[b] + f2[b] * f2[b]; s13[b] = fabs(f1[b]) + fabs(f2[b]); }
        put(0, s);
      }
      // (u2, phi)
      x2inv<T, N, true, KK>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UY, kx); x2 = Y(Y_PHI, kx); }, z, ex, q, scale);
      split();
      {
        T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          s0 += f1[b] * f1[b]; s1 += f2[b] * f1[b]; s2 += f2[b] * f2[b];
          um = max_keep_nan(um, s13[b] + fabs(f1[b]));
        }
        put(0, s0); put(20, s1); put(21, s2);
      }
      // (omega1, omega2)
      x2inv<T, N, true, KK>(
          [&](int kx, C& x1, C& x2) { x1 = Y(Y_WX, kx); x2 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx))); },
          z, ex, q, scale);
      split();
      {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < 16; ++b) s += f1[b] * f1[b] + f2[b] * f2[b];
        put(1, s);
      }
      // (omega3, dphi/dx1)
      x2inv<T, N, true, KK>(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
            x2 = mul_ik(Y(Y_PHI, kx), T(kx));
          },
          z, ex, q, scale);
      split();
      {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < 16; ++b) s += f1[b] * f1[b];
        put(1, s);
        mom3(11, f2);
      }
      // (dphi/dx2, dphi/dx3)
      x2inv<T, N, true, KK>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYPHI, kx); x2 = Y(Y_DZPHI, kx); }, z, ex, q, scale);
      split();
      mom3(14, f1);
      mom3(17, f2);
      // (du1/dx1, du2/dx2)
      x2inv<T, N, true, KK>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UX, kx), T(kx)); x2 = Y(Y_DYUY, kx); }, z, ex,
                  q, scale);
      split();
      mom3(2, f1);
      mom3(5, f2);
      // (du3/dx3, 0)
      x2inv<T, N, true, KK>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUZ, kx); x2 = zero; }, z, ex, q, scale);
      split();
      mom3(8, f1);
    }
  }

  if (MODE == XMODE_STATS || a.want_umax) {
    // the same value as taking the FP64 maximum point by point: conversion and
    // the positive scaling are monotone
    double umax = MODE == XMODE_STATS ? (double)um : (double)um * (double)scale;
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, umax, o);
      umax = other > umax || other != other ? other : umax;
    }
    if (lane == 0) atomicMax(&a.ctrl->umax_bits, (unsigned long long)__double_as_longlong(umax));
  }
  if constexpr (MODE == XMODE_STATS) {
    const long long gw = (long long)blockIdx.x * 4 + wid;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      const double v = warp_sum_d<double>(acc[i].value());
      if (lane == 0) a.partials[gw * NQ + i] = v;
    }
  }
  (void)accw;
}

// ---------------------------------------------------------------------------
// Staged x pass (right-hand side, rotational or convective form; FP32,
// N = 1024).  One CTA per SM holds X2SCfg::ROWS rows in flight; the input
// streams of each row are copied into shared memory by bulk asynchronous
// copies (TMA engine) one row ahead, in two groups completed on two mbarriers:
// group A, the streams of the first inverse transforms, and group B, those of
// the last ones (X2SGroups).  Each group of the next row is issued as soon as
// the current row stops reading it, so global latency overlaps several
// transforms, and the transforms read their inputs from shared memory.
// ---------------------------------------------------------------------------
// Streams a staged row reads, as bit masks over the y-stage streams (a
// stream's shared-memory slot is its index)
template <int MODE> struct X2SGroups;
template <> struct X2SGroups<XMODE_RHS> {
  // UX..DYUX (the first three inverse transforms), PHI..DZPHI (the last two)
  static constexpr unsigned A = (1u << Y_UX) | (1u << Y_UY) | (1u << Y_UZ) | (1u << Y_WX) | (1u << Y_DZUX) |
                                (1u << Y_DYUX);
  static constexpr unsigned B = (1u << Y_PHI) | (1u << Y_DYPHI) | (1u << Y_DZPHI);
  static constexpr int SLOTS = Y_DZPHI + 1;
};
template <> struct X2SGroups<XMODE_CONVECTIVE> {
  // u and the gradients of u1 and u2 (the first five inverse transforms); the
  // gradient of u3 but d_x u3, and phi with its gradient (the last three)
  static constexpr unsigned A = (1u << Y_UX) | (1u << Y_UY) | (1u << Y_UZ) | (1u << Y_DZUX) | (1u << Y_DYUX) |
                                (1u << Y_DYUY) | (1u << Y_DZUY);
  static constexpr unsigned B = (1u << Y_WX) | (1u << Y_PHI) | (1u << Y_DYPHI) | (1u << Y_DZPHI) | (1u << Y_DZUZ);
  static constexpr int SLOTS = Y_DZUY + 1;
};

template <typename T, int N, int KK = (N - 1) / 3, int MODE = XMODE_RHS> struct X2SCfg {
  using C = typename CT<T>::type;
  using XC = X2Cfg<T, N>;
  using G = X2SGroups<MODE>;
#ifndef PSC_X2S_ROWS
#define PSC_X2S_ROWS 6
#endif
  static constexpr int M = KK + 1;
  static constexpr unsigned ROW_BYTES = (unsigned)(M * sizeof(C));
  static constexpr size_t STAGE_BYTES = (size_t)G::SLOTS * ROW_BYTES;
  static constexpr size_t GROUP_BYTES = STAGE_BYTES + XC::LINE_BYTES;
  // rows in flight: PSC_X2S_ROWS, fewer where longer rows (more streams, or the
  // phase-shift sphere's cube) would not fit shared memory
  static constexpr int rows_fit() {
    int r = PSC_X2S_ROWS;
    while (r > 1 && GROUP_BYTES * r + XC::TW_BYTES + 2 * r * 8 > 227 * 1024) --r;
    return r;
  }
  static constexpr int ROWS = rows_fit();
  static constexpr int THREADS = XC::TH * ROWS;
  static constexpr size_t TW_OFF = GROUP_BYTES * ROWS;
  static constexpr size_t BAR_OFF = TW_OFF + XC::TW_BYTES;
  static constexpr size_t SMEM = BAR_OFF + 2 * ROWS * sizeof(unsigned long long);
  static constexpr bool OK = ROW_BYTES % 16 == 0 && SMEM <= 227 * 1024;
  static_assert((G::A & G::B) == 0 && (G::A | G::B) < (1u << G::SLOTS), "stream groups are disjoint slots");
};

template <typename T, int N, int KK = (N - 1) / 3, bool SHIFT = false, int MODE = XMODE_RHS>
__global__ void __launch_bounds__(X2SCfg<T, N, KK, MODE>::THREADS, 1) k_xpass2s(PassArgs a) {
  using C = typename CT<T>::type;
  using XC = X2Cfg<T, N>;
  using SC = X2SCfg<T, N, KK, MODE>;
  using G = typename SC::G;
  static_assert(SC::OK, "staged x pass: rows must be 16-byte multiples and fit shared memory");
  static_assert(MODE == XMODE_RHS || MODE == XMODE_CONVECTIVE, "staged x pass: right-hand side only");
  constexpr int TH = XC::TH, G_ = XC::G, ROWS = SC::ROWS, M = SC::M;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lid = threadIdx.x / TH;
  X2Roles<C> q;
  q.tid = threadIdx.x % TH;
  q.ra = q.tid / G_;
  q.rr = q.tid % G_;
  q.rk0 = bitrev_lane<G_>(q.rr);
  q.bar = 1 + lid;
  unsigned char* grp = smraw + (size_t)lid * SC::GROUP_BYTES;
  C* stg = reinterpret_cast<C*>(grp);
  C* ex = reinterpret_cast<C*>(grp + SC::STAGE_BYTES);
  unsigned long long* barA = reinterpret_cast<unsigned long long*>(smraw + SC::BAR_OFF) + 2 * lid;
  unsigned long long* barB = barA + 1;
  const C* __restrict__ yb = static_cast<const C*>(a.yb);
  C* __restrict__ xb = static_cast<C*>(a.xb);
  if (q.tid == 0) {
    mbar_init(barA, 1);
    mbar_init(barB, 1);
    mbar_init_fence();
  }
  x2_twiddles<T, N>(reinterpret_cast<C*>(smraw + SC::TW_OFF), static_cast<const C*>(a.tw), q);
  const long long ys = a.d.ys;  // N*N*M for a pass over the box
  const long long nlines = ys / M;
  const long long stride = (long long)gridDim.x * ROWS;
  const T scale = T(1.0 / ((double)N * N * N));
  const bool leader = q.tid == 0;
  // bound of the waits; the failure-path test asks one more transaction byte
  // than the copies bring for the first row of CTA 0's first row group, so that
  // row's wait runs out (every copy still lands)
  const unsigned long long lim = a.ctrl->wait_ns ? a.ctrl->wait_ns : 2000000000ull;
  bool stall = a.ctrl->stall_test != 0 && blockIdx.x == 0 && lid == 0;
  // copies of the streams in `mask` of row ln into their staging slots (one thread)
  auto issue = [&](long long ln, unsigned mask, unsigned long long* bar) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, (unsigned)__popc(mask) * SC::ROW_BYTES + (stall ? 16u : 0u));
    stall = false;
#pragma unroll
    for (int st = 0; st < G::SLOTS; ++st) {
      if (!((mask >> st) & 1u)) continue;
      const long long src = st * ys + ln * M;
      if (PSC_OK_INDEX(src + M - 1, (long long)Y_NSTREAM * ys, a.ctrl))
        bulk_copy_g2s(stg + st * M, yb + src, SC::ROW_BYTES, bar);
    }
  };
  T um = T(0);
  unsigned pa = 0, pb = 0;        // parity of the next phase to wait for
  bool ia = false, ib = false;    // a group issued and not yet waited for
  bool ok = true;
  long long line = (long long)blockIdx.x * ROWS + lid;
  if (line < nlines) {
    if (leader) {
      issue(line, G::A, barA);
      issue(line, G::B, barB);
    }
    ia = ib = true;
  }
#pragma unroll 1
  for (; line < nlines; line += stride) {
    const long long next = line + stride;
    // the row's first thread polls; the row barrier shares the outcome and
    // makes the staged streams visible to the row's threads
    ok = bar_and(q.bar, TH, leader ? mbar_wait(barA, pa, &a.ctrl->err, lim) : true);
    if (!ok) break;
    pa ^= 1u;
    ia = false;
    auto Y = [&](int st, int kx) -> C { return stg[st * M + kx]; };
    auto after_a = [&] {
      if (next < nlines) {
        if (leader) issue(next, G::A, barA);
        ia = true;
      }
    };
    auto wait_b = [&] {
      const bool w = bar_and(q.bar, TH, leader ? mbar_wait(barB, pb, &a.ctrl->err, lim) : true);
      if (w) {
        pb ^= 1u;
        ib = false;
      }
      return w;
    };
    auto after_b = [&] {
      if (next < nlines) {
        if (leader) issue(next, G::B, barB);
        ib = true;
      }
    };
    if constexpr (MODE == XMODE_RHS)
      ok = x2_rhs_row<T, N, false, KK, SHIFT>(Y, after_a, wait_b, after_b, xb, line, ys, ex, q, scale,
                                              a.want_umax != 0, um, a.ctrl, a.phase);
    else
      ok = x2_conv_row<T, N, KK, SHIFT>(Y, after_a, wait_b, after_b, xb, line, ys, ex, q, scale,
                                        a.want_umax != 0, um, a.ctrl, a.phase);
    if (!ok) break;
  }
  if (!ok) {
    // a copy did not complete in time: report it, give copies still in flight
    // a bounded time to land in this CTA's shared memory, and stop
    if (leader) {
      atomicOr(&a.ctrl->err, 4);
      if (ia) mbar_wait(barA, pa, nullptr, lim);
      if (ib) mbar_wait(barB, pb, nullptr, lim);
    }
  }
  if (a.want_umax) {
    double umax = (double)um * (double)scale;
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, umax, o);
      umax = other > umax || other != other ? other : umax;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&a.ctrl->umax_bits, (unsigned long long)__double_as_longlong(umax));
  }
}

}  // namespace psc
