// The five FFT passes of one right-hand-side evaluation (section 2.2 and 2.3
// of arXiv:2012.04838: u_hat and i k u_hat are transformed back, the
// nonlinear terms are formed in physical space and transformed forward):
//
//   Z-inverse : compact state -> lines along kz zero-padded to N, inverse DFT;
//               also emits d/dz streams (i kz multiplied before the transform)
//   Y-inverse : lines along ky zero-padded to N, inverse DFT; forms
//               omega_x = d_y u_z - d_z u_y, d_y u_x and d_y phi from i ky
//   X (fused) : per (z, y) row, 9 complex-to-real transforms (packed two per
//               complex DFT), u x omega and u . grad phi, 4 real-to-complex
//               transforms packed in pairs, keep kx <= K.  Physical fields never
//               leave the chip.  The statistics variant accumulates FP64
//               moments of the velocity/scalar gradients instead (Eqs. 11-13).
//   Y-forward : lines along y, forward DFT, keep |ky| <= K
//   Z-forward : lines along z, forward DFT, keep |kz| <= K -> compact RHS
//
// All transforms are the unnormalised DFTs of Eq. 5; the 1/N^3 of the
// inverse is applied once, to the physical fields in the X pass.
#pragma once

#include "psc_common.cuh"

namespace psc {

// ---------------------------------------------------------------------------
// Strided passes: a CTA transforms W adjacent kx columns of one plane; the
// line runs along the strided (outer) axis, so every line element moved is a
// W-wide contiguous run of complex values.
// ---------------------------------------------------------------------------

// Column tile width: FP32 passes are built for W = 8 and 16 (64- and 128-byte
// runs) and the faster is picked per pass and grid size when a simulation is
// created (see psc_capi.cu); FP64 uses W = 8.
template <typename T, int N, int W> struct StridedCfg {
  static constexpr int THREADS = W * PlanD<N>::LPL;
  // FP32: cap registers at 128 per thread so at least 512 threads fit on an SM;
  // FP64 is bound by the FP64 pipe, so it keeps its values in registers instead
  static constexpr int MINB = sizeof(T) == 8 ? 1 : (THREADS >= 512 ? 1 : 512 / THREADS);
};

template <typename T, int N, int W> struct StridedSmem {
  using C = typename CT<T>::type;
  static constexpr int R1 = PlanD<N>::R1, R2 = PlanD<N>::R2;
  // rows of R2*W values; rows start W*sizeof(C) bytes apart modulo 128 so the
  // column-major reads of step 2 spread over all banks
  static constexpr int CPB = 128 / (int)sizeof(C);
  static constexpr int PAD = (W >= CPB) ? 0 : ((((W - R2 * W) % CPB) + CPB) % CPB);
  static constexpr int ROW = R2 * W + PAD;
  static constexpr size_t EXCH_BYTES = (size_t)R1 * ROW * sizeof(C);
  // step-1 twiddles wN^(n2 k1) for this CTA's threads, stored [j][k1][t]
  // (n2 = t + j TPL) so a warp reads consecutive or identical entries
  static constexpr size_t BYTES = EXCH_BYTES + (size_t)N * sizeof(C);
};

// Fill the shared twiddle table of the strided passes (call before the first
// transform; ends with a barrier).
template <typename T, int N, int W>
__device__ __forceinline__ typename CT<T>::type* strided_twiddles(unsigned char* smraw,
                                                                  const typename CT<T>::type* PSC_RESTRICT tw,
                                                                  const Tctx& tcx) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  C* t = reinterpret_cast<C*>(smraw + StridedSmem<T, N, W>::EXCH_BYTES);
  const int nthr = tcx.bdx * tcx.bdy, me = tcx.ty * tcx.bdx + tcx.tx;
  for (int i = me; i < N; i += nthr) {
    if constexpr (PL::WIDE) {
      t[i] = tw[i];  // wide lines index wN^(n2 k1) directly
    } else {
      const int tt = i % PL::TPL, k1 = (i / PL::TPL) % PL::R1, j = i / (PL::TPL * PL::R1);
      t[i] = tw[(tt + j * PL::TPL) * k1];
    }
  }
  __syncthreads();
  return t;
}

// Inputs n1 of the first DFT of an inverse (zero-padded) line that are zero
// for every n2: positions R2 n1 + n2 all lie in the band K < p < N - K.  The
// codelet generator emits DftZ<R1, +1, Z0, Z1> for exactly this range.
template <int N, int KK = (N - 1) / 3> struct ZeroInputs {
  static constexpr int R1 = PlanD<N>::R1, R2 = PlanD<N>::R2, K = KK;
  __host__ __device__ static constexpr bool zero(int n1) { return R2 * n1 > K && R2 * n1 + R2 - 1 < N - K; }
  __host__ __device__ static constexpr int first() {
    for (int n1 = 0; n1 < R1; ++n1)
      if (zero(n1)) return n1;
    return R1;
  }
  __host__ __device__ static constexpr int last() {
    for (int n1 = R1 - 1; n1 >= 0; --n1)
      if (zero(n1)) return n1;
    return -1;
  }
  static constexpr int Z0 = first(), Z1 = last();
  static constexpr bool ANY = Z0 <= Z1;
};

// First DFT of a line: the pruned codelet for an inverse pass, else the full one.
template <typename T, int N, int DIR, int KK = (N - 1) / 3, class C>
__device__ __forceinline__ void first_dft(C (&a)[PlanD<N>::R1]) {
  if constexpr (DIR > 0 && ZeroInputs<N, KK>::ANY)
    DftZ<PlanD<N>::R1, DIR, ZeroInputs<N, KK>::Z0, ZeroInputs<N, KK>::Z1>::template run<T, C>(a);
  else
    Dft<PlanD<N>::R1, DIR>::template run<T, C>(a);
}

// True if no output k1 + R1 k2 (k1 < R1) of a length-N line is a retained
// wavenumber (K < k < N - K): a forward pass need not compute it.
template <int N, int KK = (N - 1) / 3> __host__ __device__ constexpr bool dead_k2(int k2) {
  return PlanD<N>::R1 * k2 > KK && PlanD<N>::R1 * k2 + PlanD<N>::R1 - 1 < N - KK;
}

// One length-N DFT per column, direction DIR (-1 forward, +1 inverse).
// ld(p) returns the element at line position p; st(k, v) stores output k.
// A forward transform only computes the outputs a truncated pass can keep.
template <typename T, int N, int W, int DIR, int KK = (N - 1) / 3, class LD, class ST>
__device__ __forceinline__ void strided_fft(const LD& ld, const ST& st,
                                            typename CT<T>::type* sm,
                                            const typename CT<T>::type* twsm,
                                            int t, int w) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  using SM = StridedSmem<T, N, W>;
  constexpr int R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, J1 = PL::J1, J2 = PL::J2;
  auto step1 = [&](int j) {
    const int n2 = t + j * TPL;
    C a[R1];
    static_for<0, R1>([&](auto nc) {
      constexpr int n1 = decltype(nc)::value;
      if constexpr (DIR > 0 && ZeroInputs<N, KK>::zero(n1)) a[n1] = mk(T(0), T(0));  // not read
      else a[n1] = ld(R2 * n1 + n2);
    });
    first_dft<T, N, DIR, KK>(a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C v = a[k1];
      if (k1 > 0) {
        const C wv = twsm[(j * R1 + k1) * TPL + t];  // wN^(n2 k1)
        v = (DIR < 0) ? cmul(v, wv) : cmulc(v, wv);
      }
      sm[k1 * SM::ROW + n2 * W + w] = v;
    }
  };
  auto step2 = [&](int j) {
    const int k1 = t + j * TPL;
    C b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = sm[k1 * SM::ROW + n2 * W + w];
    Dft<R2, DIR>::template run<T, C>(b);
    static_for<0, R2>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      if constexpr (!(DIR < 0 && dead_k2<N, KK>(k2))) st(k1 + R1 * k2, b[k2]);
    });
  };
  if constexpr (PL::WIDE) {
    // lane t < R2 transforms the R1 points R2 n1 + t; lane t < R1 the R2
    // points of its k1 = t
    if (t < R2) {
      const int n2 = t;
      C a[R1];
      static_for<0, R1>([&](auto nc) {
        constexpr int n1 = decltype(nc)::value;
        if constexpr (DIR > 0 && ZeroInputs<N, KK>::zero(n1)) a[n1] = mk(T(0), T(0));  // not read
        else a[n1] = ld(R2 * n1 + n2);
      });
      first_dft<T, N, DIR, KK>(a);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        C v = a[k1];
        if (k1 > 0) {
          const C wv = twsm[n2 * k1];  // wN^(n2 k1), n2 k1 < N
          v = (DIR < 0) ? cmul(v, wv) : cmulc(v, wv);
        }
        sm[k1 * SM::ROW + n2 * W + w] = v;
      }
    }
    __syncthreads();
    if (t < R1) step2(0);  // k1 = t
    __syncthreads();
  } else {
#pragma unroll
    for (int j = 0; j < J1; ++j) step1(j);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J2; ++j) step2(j);
    __syncthreads();
  }
}

// wavenumber of line position p of a zero-padded / truncated axis; false if
// the position is outside |k| <= K
template <int N, int KK = (N - 1) / 3> __device__ __forceinline__ bool k_of_pos(int p, int& k) {
  constexpr int K = KK;
  if (p <= K) { k = p; return true; }
  if (p >= N - K) { k = p - N; return true; }
  return false;
}

// Multiply by the phase exp(+-i k pi / N) of wavenumber k (table a.phase,
// index k + KK) when SHIFT: the spectra of fields sampled on the grid shifted
// by half a cell (phase-shift dealiasing); identity otherwise.
template <bool SHIFT, int KK, class C>
__device__ __forceinline__ C shift_in(C v, const void* phase, int k) {
  if constexpr (SHIFT) return cmul(v, static_cast<const C*>(phase)[k + KK]);
  else return v;
}
template <bool SHIFT, int KK, class C>
__device__ __forceinline__ C shift_out(C v, const void* phase, int k) {
  if constexpr (SHIFT) return cmulc(v, static_cast<const C*>(phase)[k + KK]);
  else return v;
}

// Each kernel runs its transforms through one copy of the transform code (a
// runtime loop over its stream table), so the instruction footprint stays that
// of a single two-step FFT however many streams the pass carries.
template <typename T, int N, bool STATS, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__device__ __forceinline__ void b_zinv(const PassArgs& a, const Tctx& tcx) {
  using C = typename CT<T>::type;
  constexpr int K = KK, M = KK + 1, P = 2 * KK + 1;
  unsigned char* smraw = tcx.smem;
  C* sm = reinterpret_cast<C*>(smraw);
  const int w = tcx.tx, t = tcx.ty;
  const int ix = tcx.bx * W + w;
  const int iy = tcx.by;
  const bool act = ix < M;
  const C* PSC_RESTRICT in = static_cast<const C*>(a.in);
  C* PSC_RESTRICT zb = static_cast<C*>(a.zb);
  const C* tw = strided_twiddles<T, N, W>(smraw, static_cast<const C*>(a.tw), tcx);
  const long long S = (long long)P * P * M, zs = (long long)N * P * M;
  const C zero = mk(T(0), T(0));
  // (input field, multiply by i kz, output stream)
  constexpr int nt = STATS ? 8 : 7;
#pragma unroll 1
  for (int tr = 0; tr < nt; ++tr) {
    int f, s;
    bool deriv;
    switch (tr) {
      case 0: f = 0; deriv = false; s = Z_UX; break;
      case 1: f = 1; deriv = false; s = Z_UY; break;
      case 2: f = 2; deriv = false; s = Z_UZ; break;
      case 3: f = 1; deriv = true; s = Z_DZUY; break;
      case 4: f = 0; deriv = true; s = Z_DZUX; break;
      case 5: f = 3; deriv = false; s = Z_PHI; break;
      case 6: f = 3; deriv = true; s = Z_DZPHI; break;
      default: f = 2; deriv = true; s = Z_DZUZ; break;
    }
    const C* PSC_RESTRICT src = in + f * S + (long long)iy * M + ix;
    strided_fft<T, N, W, +1, KK>(
        [&](int p) -> C {
          int kz;
          if (!act || !k_of_pos<N, KK>(p, kz)) return zero;
          const long long off = (long long)(kz + K) * P * M;
          if (!PSC_OK_INDEX(f * S + off + (long long)iy * M + ix, 4 * S, a.ctrl)) return zero;
          const C v = shift_in<SHIFT, KK>(src[off], a.phase, kz);
          return deriv ? mul_ik(v, T(kz)) : v;
        },
        [&](int z, C v) {
          if (!act) return;
          const long long idx = s * zs + ((long long)z * P + iy) * M + ix;
          if (PSC_OK_INDEX(idx, (long long)Z_NSTREAM * zs, a.ctrl)) zb[idx] = v;
        },
        sm, tw, t, w);
  }
}

template <typename T, int N, bool STATS, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(StridedCfg<T, N, W>::THREADS, StridedCfg<T, N, W>::MINB)
k_zinv(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  b_zinv<T, N, STATS, W, KK, SHIFT>(a, hw_ctx(smraw));
}

template <typename T, int N, int YM, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__device__ __forceinline__ void b_yinv(const PassArgs& a, const Tctx& tcx) {
  using C = typename CT<T>::type;
  constexpr int K = KK, M = KK + 1, P = 2 * KK + 1;
  unsigned char* smraw = tcx.smem;
  C* sm = reinterpret_cast<C*>(smraw);
  const int w = tcx.tx, t = tcx.ty;
  const int ix = tcx.bx * W + w;
  const int z = tcx.by;
  const bool act = ix < M;
  const C* PSC_RESTRICT zb = static_cast<const C*>(a.zb);
  C* PSC_RESTRICT yb = static_cast<C*>(a.yb);
  const C* tw = strided_twiddles<T, N, W>(smraw, static_cast<const C*>(a.tw), tcx);
  const long long zs = (long long)N * P * M, ys = (long long)N * N * M;
  const C zero = mk(T(0), T(0));
  // (kind, s1, s2, out): kind 0 = s1, 1 = i ky s1, 2 = i ky s1 - s2
  constexpr int nt = YM == YMODE_CONVECTIVE ? 12 : YM == YMODE_STATS ? 11 : 9;
#pragma unroll 1
  for (int tr = 0; tr < nt; ++tr) {
    int kind, s1, s2 = 0, so;
    switch (tr) {
      case 0: kind = 0; s1 = Z_UX; so = Y_UX; break;
      case 1: kind = 0; s1 = Z_UY; so = Y_UY; break;
      case 2: kind = 0; s1 = Z_UZ; so = Y_UZ; break;
      case 3:  // omega_x = d_y u_z - d_z u_y (convective form: d_y u_z alone)
        kind = YM == YMODE_CONVECTIVE ? 1 : 2; s1 = Z_UZ; s2 = Z_DZUY; so = Y_WX; break;
      case 4: kind = 0; s1 = Z_DZUX; so = Y_DZUX; break;
      case 5: kind = 1; s1 = Z_UX; so = Y_DYUX; break;
      case 6: kind = 0; s1 = Z_PHI; so = Y_PHI; break;
      case 7: kind = 1; s1 = Z_PHI; so = Y_DYPHI; break;
      case 8: kind = 0; s1 = Z_DZPHI; so = Y_DZPHI; break;
      case 9: kind = 1; s1 = Z_UY; so = Y_DYUY; break;
      case 10: kind = 0; s1 = Z_DZUZ; so = Y_DZUZ; break;
      default: kind = 0; s1 = Z_DZUY; so = Y_DZUY; break;
    }
    const long long rowz = (long long)z * P * M + ix;
    strided_fft<T, N, W, +1, KK>(
        [&](int p) -> C {
          int ky;
          if (!act || !k_of_pos<N, KK>(p, ky)) return zero;
          const long long o = rowz + (long long)(ky + K) * M;
          if (!PSC_OK_INDEX(s1 * zs + o, (long long)Z_NSTREAM * zs, a.ctrl)) return zero;
          const C v1 = shift_in<SHIFT, KK>(zb[s1 * zs + o], a.phase, ky);
          if (kind == 0) return v1;
          const C d = mul_ik(v1, T(ky));
          if (kind == 1) return d;
          if (!PSC_OK_INDEX(s2 * zs + o, (long long)Z_NSTREAM * zs, a.ctrl)) return zero;
          return csub(d, shift_in<SHIFT, KK>(zb[s2 * zs + o], a.phase, ky));
        },
        [&](int y, C v) {
          if (!act) return;
          const long long idx = so * ys + ((long long)z * N + y) * M + ix;
          if (PSC_OK_INDEX(idx, (long long)Y_NSTREAM * ys, a.ctrl)) yb[idx] = v;
        },
        sm, tw, t, w);
  }
}

template <typename T, int N, int YM, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(StridedCfg<T, N, W>::THREADS, StridedCfg<T, N, W>::MINB)
k_yinv(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  b_yinv<T, N, YM, W, KK, SHIFT>(a, hw_ctx(smraw));
}

template <typename T, int N, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__device__ __forceinline__ void b_yfwd(const PassArgs& a, const Tctx& tcx) {
  using C = typename CT<T>::type;
  constexpr int K = KK, M = KK + 1, P = 2 * KK + 1;
  unsigned char* smraw = tcx.smem;
  C* sm = reinterpret_cast<C*>(smraw);
  const int w = tcx.tx, t = tcx.ty;
  const int ix = tcx.bx * W + w;
  const int z = tcx.by;
  const bool act = ix < M;
  const C* PSC_RESTRICT xb = static_cast<const C*>(a.xb);
  C* PSC_RESTRICT yf = static_cast<C*>(a.yf);
  const C* tw = strided_twiddles<T, N, W>(smraw, static_cast<const C*>(a.tw), tcx);
  const long long zs = (long long)N * P * M, ys = (long long)N * N * M;
  const C zero = mk(T(0), T(0));
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    strided_fft<T, N, W, -1, KK>(
        [&](int y) -> C {
          if (!act) return zero;
          const long long idx = s * ys + ((long long)z * N + y) * M + ix;
          if (!PSC_OK_INDEX(idx, 4 * ys, a.ctrl)) return zero;
          return xb[idx];
        },
        [&](int k, C v) {
          int ky;
          if (!act || !k_of_pos<N, KK>(k, ky)) return;
          const long long idx = s * zs + ((long long)z * P + (ky + K)) * M + ix;
          if (PSC_OK_INDEX(idx, 4 * zs, a.ctrl)) yf[idx] = shift_out<SHIFT, KK>(v, a.phase, ky);
        },
        sm, tw, t, w);
  }
}

template <typename T, int N, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(StridedCfg<T, N, W>::THREADS, StridedCfg<T, N, W>::MINB)
k_yfwd(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  b_yfwd<T, N, W, KK, SHIFT>(a, hw_ctx(smraw));
}

template <typename T, int N, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__device__ __forceinline__ void b_zfwd(const PassArgs& a, const Tctx& tcx) {
  using C = typename CT<T>::type;
  constexpr int K = KK, M = KK + 1, P = 2 * KK + 1;
  unsigned char* smraw = tcx.smem;
  C* sm = reinterpret_cast<C*>(smraw);
  const int w = tcx.tx, t = tcx.ty;
  const int ix = tcx.bx * W + w;
  const int iy = tcx.by;
  const bool act = ix < M;
  const C* PSC_RESTRICT yf = static_cast<const C*>(a.yf);
  C* PSC_RESTRICT rb = static_cast<C*>(a.rb);
  const C* tw = strided_twiddles<T, N, W>(smraw, static_cast<const C*>(a.tw), tcx);
  const long long S = (long long)P * P * M, zs = (long long)N * P * M;
  const C zero = mk(T(0), T(0));
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    strided_fft<T, N, W, -1, KK>(
        [&](int z) -> C {
          if (!act) return zero;
          const long long idx = s * zs + ((long long)z * P + iy) * M + ix;
          if (!PSC_OK_INDEX(idx, 4 * zs, a.ctrl)) return zero;
          return yf[idx];
        },
        [&](int k, C v) {
          int kz;
          if (!act || !k_of_pos<N, KK>(k, kz)) return;
          const long long idx = s * S + ((long long)(kz + K) * P + iy) * M + ix;
          if (PSC_OK_INDEX(idx, 4 * S, a.ctrl)) rb[idx] = shift_out<SHIFT, KK>(v, a.phase, kz);
        },
        sm, tw, t, w);
  }
}

template <typename T, int N, int W, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(StridedCfg<T, N, W>::THREADS, StridedCfg<T, N, W>::MINB)
k_zfwd(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  b_zfwd<T, N, W, KK, SHIFT>(a, hw_ctx(smraw));
}

// ---------------------------------------------------------------------------
// X pass: one warp transforms 32/TPL adjacent rows (z, y); TPL lanes per row.
// ---------------------------------------------------------------------------

template <typename T, int N> struct XCfg {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  static constexpr int TPL = PL::TPL, LPW = 32 / TPL;
  static constexpr int WARPS = 4;
  static constexpr int PER = N / TPL;         // values per thread per field
  static constexpr bool STASH = PER >= 20;    // velocity parked in shared memory
  static constexpr int ROWI = PL::R2 + 1;     // inverse exchange rows (odd stride)
  static constexpr int ROWF = PL::R1 + 1;     // forward exchange rows
  static constexpr int EX0 = PL::R1 * ROWI > PL::R2 * ROWF ? PL::R1 * ROWI : PL::R2 * ROWF;
  static constexpr int EXCH = EX0 > N ? EX0 : N;
  static constexpr int STASH_REALS = STASH ? 3 * N : 0;
  static constexpr size_t LINE_BYTES =
      ((EXCH * sizeof(C) + STASH_REALS * sizeof(T)) + 15) / 16 * 16;
  // twiddles of the inverse (wN^(n2 k1), n2 = t + j TPL < R2, k1 < R1) and of the
  // transposed forward plan (n2 < R1, k1 < R2), each stored [j][k1][t] so the
  // lanes of a row read consecutive entries
  static constexpr size_t TW_BYTES = (size_t)2 * N * sizeof(C);
  static constexpr size_t SMEM = LINE_BYTES * LPW * WARPS + TW_BYTES;
};

// Inverse DFT of one row from its half spectrum, two real fields at once:
// Z[p] = X1[p] + i X2[p] (p <= K; imaginary parts dropped at p = 0),
// conj(X1[N-p]) + i conj(X2[N-p]) (p >= N-K), 0 elsewhere.  On return
// z[j][k2] holds scale * IDFT(Z) at position (t + j TPL) + R1 k2, whose real
// and imaginary parts are the two real fields.
template <typename T, int N, int KK = (N - 1) / 3, bool SHIFT = false, class SPEC>
__device__ __forceinline__ void xinv(const SPEC& spec,
                                     typename CT<T>::type (&z)[PlanD<N>::J2][PlanD<N>::R2],
                                     typename CT<T>::type* ex,
                                     const typename CT<T>::type* tw, int t, T scale,
                                     const void* phase = nullptr) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  using XC = XCfg<T, N>;
  constexpr int R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, K = KK;
#pragma unroll
  for (int j = 0; j < PL::J1; ++j) {
    const int n2 = t + j * TPL;
    C a[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int p = R2 * n1 + n2;
      C x1, x2;
      if (p <= K) {
        spec(p, x1, x2);
        x1 = shift_in<SHIFT, KK>(x1, phase, p);
        x2 = shift_in<SHIFT, KK>(x2, phase, p);
        if (p == 0) { x1.y = T(0); x2.y = T(0); }
        a[n1] = mk(x1.x - x2.y, x1.y + x2.x);
      } else if (p >= N - K) {
        spec(N - p, x1, x2);
        x1 = shift_in<SHIFT, KK>(x1, phase, N - p);
        x2 = shift_in<SHIFT, KK>(x2, phase, N - p);
        a[n1] = mk(x1.x + x2.y, x2.x - x1.y);
      } else {
        a[n1] = mk(T(0), T(0));
      }
    }
    Dft<R1, +1>::template run<T, C>(a);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C v = a[k1];
      if (k1 > 0) v = cmulc(v, tw[(j * R1 + k1) * TPL + t]);  // wN^(-n2 k1)
      ex[k1 * XC::ROWI + n2] = v;
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < PL::J2; ++j) {
    const int k1 = t + j * TPL;
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) z[j][n2] = ex[k1 * XC::ROWI + n2];
    Dft<R2, +1>::template run<T, C>(z[j]);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) z[j][k2] = cscale(z[j][k2], scale);
  }
  __syncwarp();
}

// Forward DFT of a row holding two real fields packed as x1 + i x2 at the
// positions xinv leaves them in; out(kx, X1, X2) receives both half spectra
// for kx <= K: X1 = (Z[k] + conj Z[N-k])/2, X2 = (Z[k] - conj Z[N-k])/(2i).
template <typename T, int N, int KK = (N - 1) / 3, bool SHIFT = false, class OUT>
__device__ __forceinline__ void xfwd(typename CT<T>::type (&x)[PlanD<N>::J2][PlanD<N>::R2],
                                     const OUT& out, typename CT<T>::type* ex,
                                     const typename CT<T>::type* tw, int t, const void* phase = nullptr) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  using XC = XCfg<T, N>;
  constexpr int R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, K = KK;
  // transposed plan: n = R1 n1' + n2' with n2' = t + j TPL < R1, n1' < R2
#pragma unroll
  for (int j = 0; j < PL::J2; ++j) {
    const int n2 = t + j * TPL;
    Dft<R2, -1>::template run<T, C>(x[j]);
#pragma unroll
    for (int k1 = 0; k1 < R2; ++k1) {
      C v = x[j][k1];
      if (k1 > 0) v = cmul(v, tw[N + (j * R2 + k1) * TPL + t]);  // wN^(n2 k1)
      ex[k1 * XC::ROWF + n2] = v;
    }
  }
  __syncwarp();
  C b[PL::J1][R1];
#pragma unroll
  for (int j = 0; j < PL::J1; ++j) {
    const int k1 = t + j * TPL;
#pragma unroll
    for (int n2 = 0; n2 < R1; ++n2) b[j][n2] = ex[k1 * XC::ROWF + n2];
    Dft<R1, -1>::template run<T, C>(b[j]);
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < PL::J1; ++j) {
    const int k1 = t + j * TPL;
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) ex[k1 + R2 * k2] = b[j][k2];
  }
  __syncwarp();
  for (int kx = t; kx <= K; kx += TPL) {
    const C A = ex[kx];
    const C B = ex[kx == 0 ? 0 : N - kx];
    out(kx, shift_out<SHIFT, KK>(mk(T(0.5) * (A.x + B.x), T(0.5) * (A.y - B.y)), phase, kx),
        shift_out<SHIFT, KK>(mk(T(0.5) * (A.y + B.y), T(0.5) * (B.x - A.x)), phase, kx));
  }
  __syncwarp();
}

__device__ __forceinline__ void umax_update(Ctrl* c, double v) {
  atomicMax(&c->umax_bits, (unsigned long long)__double_as_longlong(v));
}

template <typename T, int N, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__device__ __forceinline__ void b_xpass(const PassArgs& a, const Tctx& tcx) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  using XC = XCfg<T, N>;
  constexpr int R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, J2 = PL::J2, M = KK + 1;
  constexpr int LPW = XC::LPW;
  unsigned char* smraw = tcx.smem;
  const int lane = tcx.tx & 31, wid = tcx.tx >> 5;
  const int t = lane % TPL, g = lane / TPL;
  unsigned char* myline = smraw + (size_t)(wid * LPW + g) * XC::LINE_BYTES;
  C* ex = reinterpret_cast<C*>(myline);
  T* stash = reinterpret_cast<T*>(myline + XC::EXCH * sizeof(C));
  const C* PSC_RESTRICT yb = static_cast<const C*>(a.yb);
  C* PSC_RESTRICT xb = static_cast<C*>(a.xb);
  C* tw = reinterpret_cast<C*>(smraw + XC::LINE_BYTES * LPW * XC::WARPS);
  {
    const C* PSC_RESTRICT twg = static_cast<const C*>(a.tw);
    for (int i = tcx.tx; i < N; i += tcx.bdx) {
      const int tt = i % TPL;
      const int k1i = (i / TPL) % R1, ji = i / (TPL * R1);  // inverse: k1 < R1, j < J1
      tw[i] = twg[(tt + ji * TPL) * k1i];
      const int k1f = (i / TPL) % R2, jf = i / (TPL * R2);  // forward: k1 < R2, j < J2
      tw[N + i] = twg[(tt + jf * TPL) * k1f];
    }
    __syncthreads();
  }
  const long long ys = (long long)N * N * M;
  const long long nlines = (long long)N * N;
  const T scale = T(1.0 / ((double)N * N * N));
  const C zero = mk(T(0), T(0));
  T um = T(0);  // maximum of |u1|+|u2|+|u3| over the thread's points
  MomentSum<T> acc[MODE == XMODE_STATS ? NQ : 1];

#pragma unroll 1
  for (long long grp = (long long)tcx.bx * XC::WARPS + wid; grp * LPW < nlines;
       grp += (long long)tcx.gdx * XC::WARPS) {
    const long long line = grp * LPW + g;
    const bool valid = line < nlines;
    auto Y = [&](int s, int kx) -> C {
      if (!valid) return zero;
      const long long idx = s * ys + line * M + kx;
      if (!PSC_OK_INDEX(idx, (long long)Y_NSTREAM * ys, a.ctrl)) return zero;
      return yb[idx];
    };
    auto pos = [&](int j, int k2) { return (t + j * TPL) + R1 * k2; };
    C z[J2][R2];

    if constexpr (MODE == XMODE_RHS || MODE == XMODE_PRESSURE) {
      T ux[J2][R2], uy[J2][R2], uz[J2][R2];
      T nlx[J2][R2], nly[J2][R2], nlz[J2][R2], sv[J2][R2];
      auto getu = [&](int c, int j, int k2) -> T {
        if constexpr (XC::STASH) return stash[c * N + pos(j, k2)];
        else return c == 0 ? ux[j][k2] : (c == 1 ? uy[j][k2] : uz[j][k2]);
      };
      // (u1, u2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UY, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          if constexpr (XC::STASH) {
            stash[0 * N + pos(j, k2)] = z[j][k2].x;
            stash[1 * N + pos(j, k2)] = z[j][k2].y;
          } else {
            ux[j][k2] = z[j][k2].x;
            uy[j][k2] = z[j][k2].y;
          }
        }
      // (u3, omega_1)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UZ, kx); x2 = Y(Y_WX, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const T u3 = z[j][k2].x, w1 = z[j][k2].y;
          if constexpr (XC::STASH) stash[2 * N + pos(j, k2)] = u3;
          else uz[j][k2] = u3;
          nly[j][k2] = u3 * w1;
          nlz[j][k2] = -getu(1, j, k2) * w1;
          if (a.want_umax) um = max_keep_nan(um, fabs(getu(0, j, k2)) + fabs(getu(1, j, k2)) + fabs(u3));
        }
      // (omega_2, omega_3):  omega_2 = d_z u_1 - i kx u_3,  omega_3 = i kx u_2 - d_y u_1
      xinv<T, N, KK, SHIFT>(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx)));
            x2 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
          },
          z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const T w2 = z[j][k2].x, w3 = z[j][k2].y;
          const T u1 = getu(0, j, k2), u2 = getu(1, j, k2), u3 = getu(2, j, k2);
          nlx[j][k2] = u2 * w3 - u3 * w2;
          nly[j][k2] -= u1 * w3;
          nlz[j][k2] += u1 * w2;
        }
      // forward (NL1, NL2)
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) z[j][k2] = mk(nlx[j][k2], nly[j][k2]);
      xfwd<T, N, KK, SHIFT>(z,
                 [&](int kx, C X1, C X2) {
                   if (!valid) return;
                   const long long i0 = line * M + kx;
                   if (PSC_OK_INDEX(i0 + ys, 4 * ys, a.ctrl)) {
                     xb[i0] = X1;
                     xb[ys + i0] = X2;
                   }
                 },
                 ex, tw, t, a.phase);
      if constexpr (MODE == XMODE_PRESSURE) {
        // (NL3, |u|^2 / 2): the inputs of the modified pressure
#pragma unroll
        for (int j = 0; j < J2; ++j)
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const T u1 = getu(0, j, k2), u2 = getu(1, j, k2), u3 = getu(2, j, k2);
            z[j][k2] = mk(nlz[j][k2], T(0.5) * (u1 * u1 + u2 * u2 + u3 * u3));
          }
        xfwd<T, N, KK, SHIFT>(z,
                   [&](int kx, C X1, C X2) {
                     if (!valid) return;
                     const long long i0 = line * M + kx;
                     if (PSC_OK_INDEX(i0 + 3 * ys, 4 * ys, a.ctrl)) {
                       xb[2 * ys + i0] = X1;
                       xb[3 * ys + i0] = X2;
                     }
                   },
                   ex, tw, t, a.phase);
        continue;
      }
      // (dphi/dx1, dphi/dx2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_PHI, kx), T(kx)); x2 = Y(Y_DYPHI, kx); },
                 z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          sv[j][k2] = getu(0, j, k2) * z[j][k2].x + getu(1, j, k2) * z[j][k2].y;
      // (dphi/dx3, 0)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZPHI, kx); x2 = zero; }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          sv[j][k2] += getu(2, j, k2) * z[j][k2].x;
          z[j][k2] = mk(nlz[j][k2], sv[j][k2]);
        }
      // forward (NL3, u.grad phi)
      xfwd<T, N, KK, SHIFT>(z,
                 [&](int kx, C X1, C X2) {
                   if (!valid) return;
                   const long long i0 = line * M + kx;
                   if (PSC_OK_INDEX(i0 + 3 * ys, 4 * ys, a.ctrl)) {
                     xb[2 * ys + i0] = X1;
                     xb[3 * ys + i0] = X2;
                   }
                 },
                 ex, tw, t, a.phase);
    } else if constexpr (MODE == XMODE_CONVECTIVE) {
      // -(u.grad)u and u.grad phi from u, its nine gradients and grad phi; with
      // this stream set Y_WX holds d_y u_z and Y_DZUY holds d_z u_y
      T ux[J2][R2], uy[J2][R2], uz[J2][R2], aa[J2][R2], bb[J2][R2];
      auto getu = [&](int c, int j, int k2) -> T {
        if constexpr (XC::STASH) return stash[c * N + pos(j, k2)];
        else return c == 0 ? ux[j][k2] : (c == 1 ? uy[j][k2] : uz[j][k2]);
      };
      auto putu = [&](int c, int j, int k2, T v) {
        if constexpr (XC::STASH) {
          stash[c * N + pos(j, k2)] = v;
        } else {
          if (c == 0) ux[j][k2] = v;
          else if (c == 1) uy[j][k2] = v;
          else uz[j][k2] = v;
        }
      };
      auto store = [&](int s0) {
        return [&, s0](int kx, C X1, C X2) {
          if (!valid) return;
          const long long i0 = line * M + kx;
          if (PSC_OK_INDEX(i0 + (s0 + 1) * ys, 4 * ys, a.ctrl)) {
            xb[s0 * ys + i0] = X1;
            xb[(s0 + 1) * ys + i0] = X2;
          }
        };
      };
      // (u1, u2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UY, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) { putu(0, j, k2, z[j][k2].x); putu(1, j, k2, z[j][k2].y); }
      // (u3, d1 u1)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UZ, kx); x2 = mul_ik(Y(Y_UX, kx), T(kx)); }, z, ex, tw, t,
                 scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          putu(2, j, k2, z[j][k2].x);
          aa[j][k2] = getu(0, j, k2) * z[j][k2].y;
          if (a.want_umax) um = max_keep_nan(um, fabs(getu(0, j, k2)) + fabs(getu(1, j, k2)) + fabs(z[j][k2].x));
        }
      // (d2 u1, d3 u1): aa = (u.grad) u1
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYUX, kx); x2 = Y(Y_DZUX, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) aa[j][k2] += getu(1, j, k2) * z[j][k2].x + getu(2, j, k2) * z[j][k2].y;
      // (d1 u2, d2 u2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UY, kx), T(kx)); x2 = Y(Y_DYUY, kx); }, z, ex, tw, t,
                 scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) bb[j][k2] = getu(0, j, k2) * z[j][k2].x + getu(1, j, k2) * z[j][k2].y;
      // (d3 u2, d1 u3): bb = (u.grad) u2; aa starts (u.grad) u3
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUY, kx); x2 = mul_ik(Y(Y_UZ, kx), T(kx)); }, z, ex, tw, t,
                 scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const T b2 = bb[j][k2] + getu(2, j, k2) * z[j][k2].x, c3 = getu(0, j, k2) * z[j][k2].y;
          z[j][k2] = mk(-aa[j][k2], -b2);  // (NL1, NL2)
          aa[j][k2] = c3;
        }
      xfwd<T, N, KK, SHIFT>(z, store(0), ex, tw, t, a.phase);
      // (d2 u3, d3 u3): aa = (u.grad) u3
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_WX, kx); x2 = Y(Y_DZUZ, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) aa[j][k2] += getu(1, j, k2) * z[j][k2].x + getu(2, j, k2) * z[j][k2].y;
      // (dphi/dx1, dphi/dx2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_PHI, kx), T(kx)); x2 = Y(Y_DYPHI, kx); }, z, ex, tw, t,
                 scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) bb[j][k2] = getu(0, j, k2) * z[j][k2].x + getu(1, j, k2) * z[j][k2].y;
      // (dphi/dx3, 0)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZPHI, kx); x2 = zero; }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          z[j][k2] = mk(-aa[j][k2], bb[j][k2] + getu(2, j, k2) * z[j][k2].x);  // (NL3, u.grad phi)
      xfwd<T, N, KK, SHIFT>(z, store(2), ex, tw, t, a.phase);
    } else {
      // statistics: moments of the diagonal velocity gradients and the scalar
      // gradient (Eqs. 11-12), |omega|^2, u.u, phi u2, phi^2 (Eq. 13)
      T s13[J2][R2];
      auto mom = [&](int q, T v) { (void)q; return v; };
      (void)mom;
      auto acc234 = [&](int q, int j, int k2, T v) {
        const T v2 = v * v;
        acc[q].add(v2);
        acc[q + 1].add(v2 * v);
        acc[q + 2].add(v2 * v2);
        (void)j; (void)k2;
      };
      // (u1, u3)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UZ, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const T u1 = z[j][k2].x, u3 = z[j][k2].y;
          acc[0].add(u1 * u1 + u3 * u3);
          s13[j][k2] = fabs(u1) + fabs(u3);
        }
      // (u2, phi)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_UY, kx); x2 = Y(Y_PHI, kx); }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const T u2 = z[j][k2].x, ph = z[j][k2].y;
          acc[0].add(u2 * u2);
          acc[20].add(ph * u2);
          acc[21].add(ph * ph);
          um = max_keep_nan(um, s13[j][k2] + fabs(u2));
        }
      // (omega_1, omega_2)
      xinv<T, N, KK, SHIFT>(
          [&](int kx, C& x1, C& x2) {
            x1 = Y(Y_WX, kx);
            x2 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx)));
          },
          z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          acc[1].add(z[j][k2].x * z[j][k2].x + z[j][k2].y * z[j][k2].y);
      // (omega_3, dphi/dx1)
      xinv<T, N, KK, SHIFT>(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
            x2 = mul_ik(Y(Y_PHI, kx), T(kx));
          },
          z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          acc[1].add(z[j][k2].x * z[j][k2].x);
          acc234(11, j, k2, z[j][k2].y);
        }
      // (dphi/dx2, dphi/dx3)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYPHI, kx); x2 = Y(Y_DZPHI, kx); }, z, ex, tw, t,
                 scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          acc234(14, j, k2, z[j][k2].x);
          acc234(17, j, k2, z[j][k2].y);
        }
      // (du1/dx1, du2/dx2)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UX, kx), T(kx)); x2 = Y(Y_DYUY, kx); }, z,
                 ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          acc234(2, j, k2, z[j][k2].x);
          acc234(5, j, k2, z[j][k2].y);
        }
      // (du3/dx3, 0)
      xinv<T, N, KK, SHIFT>([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUZ, kx); x2 = zero; }, z, ex, tw, t, scale, a.phase);
#pragma unroll
      for (int j = 0; j < J2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) acc234(8, j, k2, z[j][k2].x);
    }
  }

  if (MODE == XMODE_STATS || a.want_umax) {
    double umax = (double)um;  // the fields here are scaled
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, umax, o);
      umax = other > umax || other != other ? other : umax;
    }
    if (lane == 0) umax_update(a.ctrl, umax);
  }
  if constexpr (MODE == XMODE_STATS) {
    const long long gw = (long long)tcx.bx * XC::WARPS + wid;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double v = acc[q].value();
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) a.partials[gw * NQ + q] = v;
    }
  }
}

template <typename T, int N, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(32 * XCfg<T, N>::WARPS)
k_xpass(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  b_xpass<T, N, MODE, KK, SHIFT>(a, hw_ctx(smraw));
}

}  // namespace psc

#include "psc_xpass2.cuh"
#include "psc_staged.cuh"
#include "psc_xrow.cuh"

namespace psc {

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

template <typename T, int N> struct Passes {
  static constexpr int TPL = PlanD<N>::TPL;
  static constexpr int M = PlanD<N>::M, P = PlanD<N>::P;
  // tile widths of the two variants (v = 0, 1)
  static constexpr int WV0 = 8, WV1 = sizeof(T) == 4 ? 16 : 8;

  // rows of N = 512 and 1024 use the 16-values-per-thread layout of psc_xpass2.cuh
#ifndef PSC_X2_MIN_N
#define PSC_X2_MIN_N 512
#endif
  static constexpr bool X2 = (N == 512 || N == 1024) && N >= PSC_X2_MIN_N;
  // rows whose plan gives each lane more than 64 values (N = 520: 2 lanes)
  // take the shared-memory row X pass; it also runs on request (PassArgs::xrow)
  // at the sizes with the register X pass, for testing
  static constexpr bool XROW = !X2 && N / TPL > 64;
  static constexpr bool XROW_OK = !X2;
  using XRC = XRowCfg<T, N>;
  static int xrow_grid() {
    const long long g = ((long long)N * N + XRC::WR - 1) / XRC::WR;
    const long long cap = 152 * 64;
    return (int)(g < cap ? g : cap);
  }
  // X-pass CTAs (row X pass) or warps (register X passes) that write statistics partials
  static int xwarps() {
    if constexpr (XROW) return xrow_grid();
    else return xgrid() * (X2 ? 4 : XCfg<T, N>::WARPS);
  }
  // grid: one CTA per statistics partials slot (xwarps()) except where the
  // row X pass is the only one
  template <int MODE, int KK, bool SH> static void xrow_launch(const PassArgs& a) {
    constexpr int WR = XRC::WR;
    using XS = XRowSmem<T, N, WR>;
    const int grid = XROW ? xrow_grid() : xwarps();
    prep(k_xrow<T, N, WR, MODE, KK, SH>, XS::SMEM);
    k_xrow<T, N, WR, MODE, KK, SH><<<grid, XS::THREADS, XS::SMEM, a.st>>>(a);
  }
  template <int MODE, int KK, bool SH> static void xrow_k(const PassArgs& a) {
    if constexpr (XROW_OK) xrow_launch<MODE, KK, SH>(a);
    else (void)a;
  }

  static int xgrid() {
    if constexpr (X2) {
      const long long g = (long long)N * N / X2Cfg<T, N>::ROWS;
      const long long cap = 152 * 16;
      return (int)(g < cap ? g : cap);
    } else {
      const long long groups = ((long long)N * N + XCfg<T, N>::LPW - 1) / XCfg<T, N>::LPW;
      long long g = (groups + XCfg<T, N>::WARPS - 1) / XCfg<T, N>::WARPS;
      const long long cap = 152 * 8;
      return (int)(g < cap ? g : cap);
    }
  }

  template <class KER> static void prep(KER k, size_t smem) {
    if (smem > 48 * 1024) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    }
  }

  template <int W> static void zinv_w(const PassArgs& a, bool stats) {
    constexpr size_t sm = StridedSmem<T, N, W>::BYTES;
    dim3 grid((M + W - 1) / W, P), block(W, PlanD<N>::LPL);
    if (stats) { prep(k_zinv<T, N, true, W>, sm); k_zinv<T, N, true, W><<<grid, block, sm, a.st>>>(a); }
    else { prep(k_zinv<T, N, false, W>, sm); k_zinv<T, N, false, W><<<grid, block, sm, a.st>>>(a); }
  }
  template <int W, int YM> static void yinv_m(const PassArgs& a) {
    constexpr size_t sm = StridedSmem<T, N, W>::BYTES;
    dim3 grid((M + W - 1) / W, N), block(W, PlanD<N>::LPL);
    prep(k_yinv<T, N, YM, W>, sm);
    k_yinv<T, N, YM, W><<<grid, block, sm, a.st>>>(a);
  }
  template <int W> static void yinv_w(const PassArgs& a, int ym) {
    if (ym == YMODE_STATS) yinv_m<W, YMODE_STATS>(a);
    else if (ym == YMODE_CONVECTIVE) yinv_m<W, YMODE_CONVECTIVE>(a);
    else yinv_m<W, YMODE_RHS>(a);
  }
  template <int W> static void yfwd_w(const PassArgs& a) {
    constexpr size_t sm = StridedSmem<T, N, W>::BYTES;
    dim3 grid((M + W - 1) / W, N), block(W, PlanD<N>::LPL);
    prep(k_yfwd<T, N, W>, sm);
    k_yfwd<T, N, W><<<grid, block, sm, a.st>>>(a);
  }
  template <int W> static void zfwd_w(const PassArgs& a) {
    constexpr size_t sm = StridedSmem<T, N, W>::BYTES;
    dim3 grid((M + W - 1) / W, P), block(W, PlanD<N>::LPL);
    prep(k_zfwd<T, N, W>, sm);
    k_zfwd<T, N, W><<<grid, block, sm, a.st>>>(a);
  }
  // variants 2 and 3: input tiles staged by TMA, 4 and 8 columns (FP32, M even)
#ifndef PSC_STAGED
#define PSC_STAGED 1
#endif
  // the plan and precision allow staged variants (the row length is the caller's)
  static constexpr bool STAGED_OK = PSC_STAGED && sizeof(T) == 4 && N >= 64 && TPL >= 4;
  static constexpr bool STAGED = STAGED_OK && M % 2 == 0;
  // variant 4: staged, 16 columns, for the inverse passes where it fits one CTA
  static constexpr bool STAGED16 = STAGED && StagedTile<T, N, 16, true>::SMEM <= 227 * 1024;
  static constexpr int NV = STAGED16 ? 5 : STAGED ? 4 : (WV0 != WV1 ? 2 : 1);
  static constexpr unsigned MASK_INV = (1u << NV) - 1u;
  static constexpr unsigned MASK_FWD = STAGED16 ? 0xFu : (1u << NV) - 1u;
  template <int W, int PASS, int MODE> static bool launch_s(const PassArgs& a) {
    if constexpr (STAGED) {
      using TL = StagedTile<T, N, W, PASS == SP_ZINV || PASS == SP_YINV>;
      CUtensorMap m;
      bool ok;
      int rows;
      if constexpr (PASS == SP_ZINV) {
        ok = make_row_map(&m, a.in, 3, M, P, 4LL * P, (long long)P * M, W, TL::BOXR);
        rows = P;
      } else if constexpr (PASS == SP_YINV) {
        ok = make_row_map(&m, a.zb, 2, M, (long long)Z_NSTREAM * N * P, 0, 0, W, TL::BOXR);
        rows = N;
      } else if constexpr (PASS == SP_YFWD) {
        ok = make_row_map(&m, a.xb, 2, M, 4LL * N * N, 0, 0, W, TL::BOXR);
        rows = N;
      } else {
        ok = make_row_map(&m, a.yf, 3, M, P, 4LL * N, (long long)P * M, W, TL::BOXR);
        rows = P;
      }
      if (!ok) return false;
      prep(k_strided_s<T, N, W, PASS, MODE>, TL::SMEM);
      k_strided_s<T, N, W, PASS, MODE><<<dim3((M + W - 1) / W, rows), dim3(W, TPL), TL::SMEM, a.st>>>(a, m);
      return true;
    } else {
      (void)a;
      return false;
    }
  }
  template <int PASS, int W> static bool staged_w(const PassArgs& a, int mode) {
    if constexpr (PASS == SP_YINV) {
      if (mode == YMODE_STATS) return launch_s<W, PASS, YMODE_STATS>(a);
      if (mode == YMODE_CONVECTIVE) return launch_s<W, PASS, YMODE_CONVECTIVE>(a);
      return launch_s<W, PASS, YMODE_RHS>(a);
    } else if constexpr (PASS == SP_ZINV) {
      return mode ? launch_s<W, PASS, 1>(a) : launch_s<W, PASS, 0>(a);
    } else {
      (void)mode;
      return launch_s<W, PASS, 0>(a);
    }
  }
  // mode: z-inverse 0/1 (right-hand side / 8 streams), y-inverse YMODE_*
  template <int PASS> static bool staged(const PassArgs& a, int mode, int v) {
    if (v == 2) return staged_w<PASS, 4>(a, mode);
    if constexpr (STAGED16 && (PASS == SP_ZINV || PASS == SP_YINV)) {
      if (v == 4) return staged_w<PASS, 16>(a, mode);
    }
    return staged_w<PASS, 8>(a, mode);
  }
  // a staged variant falls back to variant 0 if its tensor map cannot be made
  static void zinv(const PassArgs& a, bool stats, int v) {
    if (v >= 2 && staged<SP_ZINV>(a, stats ? 1 : 0, v)) return;
    v == 1 ? zinv_w<WV1>(a, stats) : zinv_w<WV0>(a, stats);
  }
  static void yinv(const PassArgs& a, int ym, int v) {
    if (v >= 2 && staged<SP_YINV>(a, ym, v)) return;
    v == 1 ? yinv_w<WV1>(a, ym) : yinv_w<WV0>(a, ym);
  }
  static void yfwd(const PassArgs& a, int v) {
    if (v >= 2 && staged<SP_YFWD>(a, 0, v)) return;
    v == 1 ? yfwd_w<WV1>(a) : yfwd_w<WV0>(a);
  }
  static void zfwd(const PassArgs& a, int v) {
    if (v >= 2 && staged<SP_ZFWD>(a, 0, v)) return;
    v == 1 ? zfwd_w<WV1>(a) : zfwd_w<WV0>(a);
  }
  // the right-hand side at N = 1024 (FP32) stages its rows through shared memory
#ifndef PSC_X2S
#define PSC_X2S 1
#endif
  static constexpr bool X2S = PSC_X2S && X2 && N == 1024 && sizeof(T) == 4;
  static int sm_count() {
    static int n[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (n[dev] == 0) {
      int c = 0;
      cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
      n[dev] = c > 0 ? c : 152;
    }
    return n[dev];
  }
  template <int MODE> static void xpass_plain(const PassArgs& a) {
    if constexpr (XROW) {
      (void)a;
    } else if constexpr (X2) {
      const size_t sm2 = X2Cfg<T, N>::SMEM;
      prep(k_xpass2<T, N, MODE>, sm2);
      k_xpass2<T, N, MODE><<<xgrid(), 128, sm2, a.st>>>(a);
    } else {
      const size_t sm = XCfg<T, N>::SMEM;
      prep(k_xpass<T, N, MODE>, sm);
      k_xpass<T, N, MODE><<<xgrid(), dim3(32 * XCfg<T, N>::WARPS), sm, a.st>>>(a);
    }
  }
  // the staged x pass of the right-hand side (rotational or convective form)
  template <int MODE> static void xpass_staged(const PassArgs& a) {
    constexpr int KD = (N - 1) / 3;
    using SC = X2SCfg<T, N, KD, MODE>;
    const long long rows = (long long)N * N / SC::ROWS;
    const int grid = (int)(rows < sm_count() ? rows : sm_count());
    prep(k_xpass2s<T, N, KD, false, MODE>, SC::SMEM);
    k_xpass2s<T, N, KD, false, MODE><<<grid, SC::THREADS, SC::SMEM, a.st>>>(a);
  }
  static void xpass_reg(const PassArgs& a, int mode) {
    if (mode == XMODE_PRESSURE) return xpass_plain<XMODE_PRESSURE>(a);
    if constexpr (X2S) {
      if (mode == XMODE_RHS) return xpass_staged<XMODE_RHS>(a);
      if (mode == XMODE_CONVECTIVE) return xpass_staged<XMODE_CONVECTIVE>(a);
    }
    if (mode == XMODE_CONVECTIVE) return xpass_plain<XMODE_CONVECTIVE>(a);
    if constexpr (XROW) {
      (void)a;
      (void)mode;
    } else if constexpr (X2) {
      const size_t sm2 = X2Cfg<T, N>::SMEM;
      if (mode == XMODE_STATS) {
        prep(k_xpass2<T, N, XMODE_STATS>, sm2);
        k_xpass2<T, N, XMODE_STATS><<<xgrid(), 128, sm2, a.st>>>(a);
      } else {
        prep(k_xpass2<T, N, XMODE_RHS>, sm2);
        k_xpass2<T, N, XMODE_RHS><<<xgrid(), 128, sm2, a.st>>>(a);
      }
    } else {
      const size_t sm = XCfg<T, N>::SMEM;
      dim3 block(32 * XCfg<T, N>::WARPS);
      if (mode == XMODE_STATS) {
        prep(k_xpass<T, N, XMODE_STATS>, sm);
        k_xpass<T, N, XMODE_STATS><<<xgrid(), block, sm, a.st>>>(a);
      } else {
        prep(k_xpass<T, N, XMODE_RHS>, sm);
        k_xpass<T, N, XMODE_RHS><<<xgrid(), block, sm, a.st>>>(a);
      }
    }
  }
  // The row X pass serves the right-hand side, the pressure inputs and the
  // statistics; the convective form needs the register X passes (it is
  // refused at the grid sizes that only have the row X pass).
  static void xpass(const PassArgs& a, int mode) {
    if constexpr (XROW_OK) {
      if (XROW || a.xrow) {
        constexpr int K = PlanD<N>::K;
        if (mode == XMODE_STATS) return xrow_k<XMODE_STATS, K, false>(a);
        if (mode == XMODE_PRESSURE) return xrow_k<XMODE_PRESSURE, K, false>(a);
        if (mode == XMODE_RHS) return xrow_k<XMODE_RHS, K, false>(a);
      }
    }
    if constexpr (!XROW) xpass_reg(a, mode);
  }
  static const PassTable* table() {
    static const PassTable tb = {&zinv, &yinv, &xpass, &yfwd, &zfwd,
                                 xwarps(), NV,
                                 {WV0, WV1, 4, 8, 16}, {0, 0, 1, 1, 1},
                                 {MASK_INV, MASK_INV, MASK_FWD, MASK_FWD}, XROW ? 1 : 0};
    return &tb;
  }
};

// Passes of phase-shift dealiasing (section 2.3): the generic strided passes
// and X pass over the cube |k_i| <= KS that holds the sphere 9|k|^2 < 2 N^2,
// evaluated on the grid (a.shift = 0) or on the grid shifted by half a cell in
// every direction (a.shift = 1: inputs times exp(i k pi/N) per axis, outputs
// times its conjugate).
template <typename T, int N> struct PassesPS {
  static constexpr int KS = sphere_storage_halfwidth(N);
  static constexpr int TPL = PlanD<N>::TPL;
  static constexpr int M = KS + 1, P = 2 * KS + 1;
  static constexpr int WV0 = 8, WV1 = sizeof(T) == 4 ? 16 : 8;
  static constexpr int NV = WV0 != WV1 ? 2 : 1;
  static_assert(P <= N, "the sphere's cube must fit the grid");
  using B = Passes<T, N>;

  template <class KER> static void go(KER k, dim3 grid, dim3 block, size_t sm, const PassArgs& a) {
    B::prep(k, sm);
    k<<<grid, block, sm, a.st>>>(a);
  }
  template <int W, bool STATS, bool SH> static void zinv_k(const PassArgs& a) {
    go(k_zinv<T, N, STATS, W, KS, SH>, dim3((M + W - 1) / W, P), dim3(W, PlanD<N>::LPL), StridedSmem<T, N, W>::BYTES, a);
  }
  template <int W, int YM, bool SH> static void yinv_k(const PassArgs& a) {
    go(k_yinv<T, N, YM, W, KS, SH>, dim3((M + W - 1) / W, N), dim3(W, PlanD<N>::LPL), StridedSmem<T, N, W>::BYTES, a);
  }
  template <int W, bool SH> static void yfwd_k(const PassArgs& a) {
    go(k_yfwd<T, N, W, KS, SH>, dim3((M + W - 1) / W, N), dim3(W, PlanD<N>::LPL), StridedSmem<T, N, W>::BYTES, a);
  }
  template <int W, bool SH> static void zfwd_k(const PassArgs& a) {
    go(k_zfwd<T, N, W, KS, SH>, dim3((M + W - 1) / W, P), dim3(W, PlanD<N>::LPL), StridedSmem<T, N, W>::BYTES, a);
  }
  // X pass over the sphere's cube: the 16-values-per-thread register pass at
  // 512 and 1024, the row X pass at 520 (no convective form there), the
  // generic register pass below
  static constexpr bool ROWS = B::XROW;
  template <int MODE, bool SH> static void xpass_k(const PassArgs& a) {
    if constexpr (MODE != XMODE_CONVECTIVE && (ROWS || B::XROW_OK)) {
      if (ROWS || a.xrow) return B::template xrow_launch<MODE, KS, SH>(a);
    }
    if constexpr (B::X2) {
      if constexpr (B::X2S && MODE == XMODE_RHS) {
        // the right-hand side at N = 1024 stages its rows through shared memory
        using SC = X2SCfg<T, N, KS>;
        const long long rows = (long long)N * N / SC::ROWS;
        const int grid = (int)(rows < B::sm_count() ? rows : B::sm_count());
        go(k_xpass2s<T, N, KS, SH>, dim3(grid), dim3(SC::THREADS), SC::SMEM, a);
        return;
      }
      go(k_xpass2<T, N, MODE, KS, SH>, dim3(B::xgrid()), dim3(128), X2Cfg<T, N>::SMEM, a);
    } else if constexpr (!ROWS) {
      go(k_xpass<T, N, MODE, KS, SH>, dim3(B::xgrid()), dim3(32 * XCfg<T, N>::WARPS), XCfg<T, N>::SMEM, a);
    }
  }
  // the 8-stream z-inverse serves the statistics (unshifted) and the
  // convective form (both grids); the statistics y-inverse and X pass run on
  // the grid itself only
  template <int W> static void zinv_w(const PassArgs& a, bool stats) {
    if (stats) a.shift ? zinv_k<W, true, true>(a) : zinv_k<W, true, false>(a);
    else a.shift ? zinv_k<W, false, true>(a) : zinv_k<W, false, false>(a);
  }
  template <int W> static void yinv_w(const PassArgs& a, int ym) {
    if (ym == YMODE_STATS) yinv_k<W, YMODE_STATS, false>(a);
    else if (ym == YMODE_CONVECTIVE) a.shift ? yinv_k<W, YMODE_CONVECTIVE, true>(a) : yinv_k<W, YMODE_CONVECTIVE, false>(a);
    else a.shift ? yinv_k<W, YMODE_RHS, true>(a) : yinv_k<W, YMODE_RHS, false>(a);
  }
  // variants 2-4: input tiles staged by TMA (4, 8 and, for the inverse passes,
  // 16 columns), where the stored cube's kx rows are 16-byte multiples
  static constexpr bool STAGED = B::STAGED_OK && M % 2 == 0;
  static constexpr bool STAGED16 = STAGED && StagedTile<T, N, 16, true, KS>::SMEM <= 227 * 1024;
  static constexpr int NVS = STAGED16 ? 5 : STAGED ? 4 : NV;
  static constexpr unsigned MASK_INV = (1u << NVS) - 1u;
  static constexpr unsigned MASK_FWD = STAGED16 ? 0xFu : (1u << NVS) - 1u;
  template <int W, int PASS, int MODE, bool SH> static bool launch_s(const PassArgs& a) {
    if constexpr (STAGED) {
      using TL = StagedTile<T, N, W, PASS == SP_ZINV || PASS == SP_YINV, KS>;
      CUtensorMap m;
      bool ok;
      int rows;
      if constexpr (PASS == SP_ZINV) {
        ok = make_row_map(&m, a.in, 3, M, P, 4LL * P, (long long)P * M, W, TL::BOXR);
        rows = P;
      } else if constexpr (PASS == SP_YINV) {
        ok = make_row_map(&m, a.zb, 2, M, (long long)Z_NSTREAM * N * P, 0, 0, W, TL::BOXR);
        rows = N;
      } else if constexpr (PASS == SP_YFWD) {
        ok = make_row_map(&m, a.xb, 2, M, 4LL * N * N, 0, 0, W, TL::BOXR);
        rows = N;
      } else {
        ok = make_row_map(&m, a.yf, 3, M, P, 4LL * N, (long long)P * M, W, TL::BOXR);
        rows = P;
      }
      if (!ok) return false;
      B::prep(k_strided_s<T, N, W, PASS, MODE, KS, SH>, TL::SMEM);
      k_strided_s<T, N, W, PASS, MODE, KS, SH><<<dim3((M + W - 1) / W, rows), dim3(W, TPL), TL::SMEM, a.st>>>(a, m);
      return true;
    } else {
      (void)a;
      return false;
    }
  }
  template <int PASS, int W, int MODE> static bool staged_sh(const PassArgs& a) {
    return a.shift ? launch_s<W, PASS, MODE, true>(a) : launch_s<W, PASS, MODE, false>(a);
  }
  // mode: z-inverse 0/1 (right-hand side / 8 streams), y-inverse YMODE_*; the
  // statistics stream sets run on the grid itself only
  template <int PASS, int W> static bool staged_w(const PassArgs& a, int mode) {
    if constexpr (PASS == SP_YINV) {
      if (mode == YMODE_STATS) return launch_s<W, PASS, YMODE_STATS, false>(a);
      if (mode == YMODE_CONVECTIVE) return staged_sh<PASS, W, YMODE_CONVECTIVE>(a);
      return staged_sh<PASS, W, YMODE_RHS>(a);
    } else if constexpr (PASS == SP_ZINV) {
      return mode ? staged_sh<PASS, W, 1>(a) : staged_sh<PASS, W, 0>(a);
    } else {
      (void)mode;
      return staged_sh<PASS, W, 0>(a);
    }
  }
  template <int PASS> static bool staged(const PassArgs& a, int mode, int v) {
    if (v == 2) return staged_w<PASS, 4>(a, mode);
    if constexpr (STAGED16 && (PASS == SP_ZINV || PASS == SP_YINV)) {
      if (v == 4) return staged_w<PASS, 16>(a, mode);
    }
    return staged_w<PASS, 8>(a, mode);
  }
  // a staged variant falls back to variant 0 if its tensor map cannot be made
  static void zinv(const PassArgs& a, bool stats, int v) {
    if (v >= 2 && staged<SP_ZINV>(a, stats ? 1 : 0, v)) return;
    v == 1 ? zinv_w<WV1>(a, stats) : zinv_w<WV0>(a, stats);
  }
  static void yinv(const PassArgs& a, int ym, int v) {
    if (v >= 2 && staged<SP_YINV>(a, ym, v)) return;
    v == 1 ? yinv_w<WV1>(a, ym) : yinv_w<WV0>(a, ym);
  }
  static void yfwd(const PassArgs& a, int v) {
    if (v >= 2 && staged<SP_YFWD>(a, 0, v)) return;
    if (v == 1) a.shift ? yfwd_k<WV1, true>(a) : yfwd_k<WV1, false>(a);
    else a.shift ? yfwd_k<WV0, true>(a) : yfwd_k<WV0, false>(a);
  }
  static void zfwd(const PassArgs& a, int v) {
    if (v >= 2 && staged<SP_ZFWD>(a, 0, v)) return;
    if (v == 1) a.shift ? zfwd_k<WV1, true>(a) : zfwd_k<WV1, false>(a);
    else a.shift ? zfwd_k<WV0, true>(a) : zfwd_k<WV0, false>(a);
  }
  static void xpass(const PassArgs& a, int mode) {
    if (mode == XMODE_STATS) return xpass_k<XMODE_STATS, false>(a);
    if (mode == XMODE_PRESSURE) return a.shift ? xpass_k<XMODE_PRESSURE, true>(a) : xpass_k<XMODE_PRESSURE, false>(a);
    if (mode == XMODE_CONVECTIVE)
      return a.shift ? xpass_k<XMODE_CONVECTIVE, true>(a) : xpass_k<XMODE_CONVECTIVE, false>(a);
    a.shift ? xpass_k<XMODE_RHS, true>(a) : xpass_k<XMODE_RHS, false>(a);
  }
  static const PassTable* table() {
    static const PassTable tb = {&zinv, &yinv, &xpass, &yfwd, &zfwd,
                                 B::xwarps(), NVS,
                                 {WV0, WV1, 4, 8, 16}, {0, 0, 1, 1, 1},
                                 {MASK_INV, MASK_INV, MASK_FWD, MASK_FWD}, ROWS ? 1 : 0};
    return &tb;
  }
};

}  // namespace psc
