// X pass through shared-memory rows: the fused x transforms and products of
// the right-hand side (u x omega, u . grad phi), the pressure inputs and the
// statistics moments, for grids whose two-step plan gives a line too few lanes
// to hold a row's values in registers (N = 520 = 20 x 26 over two lanes).
//
// One warp takes one row (z, y).  A row DFT is the two-step split N = R1 R2
// done across the warp: lanes n2 < R2 each transform the R1 points
// R2 n1 + n2 (with the twiddle wN^(n2 k1)), the results cross through a
// per-warp exchange in shared memory, and lanes k1 < R1 each transform R2
// points into outputs k1 + R1 k2.  An inverse reads the packed half spectra
// of two real fields from the y-inverse streams and leaves the two physical
// fields, scaled by 1/N^3, in per-row buffers in shared memory; products are
// formed in the store callbacks, point by point; a forward transform reads a
// packed pair of buffers and writes both half spectra kx <= K.  Six buffers of
// N reals per row suffice for the right-hand side (u1, u2, u3 and the three
// components of the nonlinear term while it is assembled).
// Included by psc_passes.cuh after the transforms it builds on.
#pragma once

namespace psc {

template <typename T, int N, int WR> struct XRowSmem {
  static constexpr int NB = 6;                     // row buffers of N reals
  static constexpr int THREADS = 32 * WR;          // one warp per row
  static constexpr int R1 = PlanD<N>::R1, R2 = PlanD<N>::R2;
  static constexpr int RS = R2 + 1;                // exchange row stride (odd)
  static constexpr size_t TW_BYTES = (size_t)N * sizeof(typename CT<T>::type);
  static constexpr size_t EX_BYTES = ((size_t)R1 * RS * sizeof(typename CT<T>::type) + 15) / 16 * 16;
  static constexpr size_t ROW_BYTES = EX_BYTES + ((size_t)NB * N * sizeof(T) + 15) / 16 * 16;
  static constexpr size_t RED_BYTES = (size_t)NQ * THREADS * sizeof(double);
  static constexpr size_t BODY = (size_t)WR * ROW_BYTES;
  static constexpr size_t SMEM = TW_BYTES + (BODY > RED_BYTES ? BODY : RED_BYTES);
  static_assert(R1 <= 32 && R2 <= 32, "a row DFT step must fit one warp");
};

// Rows (warps) per CTA: 4 in FP32, 2 in FP64 (about 67 KB of shared memory
// per CTA at N = 520, three CTAs per SM).
template <typename T, int N> struct XRowCfg {
  static constexpr int WR = sizeof(T) == 4 ? 4 : 2;
  using S = XRowSmem<T, N, WR>;
  static_assert(S::SMEM <= 220 * 1024, "row buffers do not fit in shared memory");
};

// One length-N DFT of a row by one warp, direction DIR; ld(p) gives position
// p, st(k, v) takes output k (a forward transform skips the outputs a
// truncated pass drops).  Ends with __syncwarp.
template <typename T, int N, int DIR, int KK, class LD, class ST>
__device__ __forceinline__ void warp_row_fft(const LD& ld, const ST& st, typename CT<T>::type* ex,
                                             const typename CT<T>::type* tw, int lane) {
  using C = typename CT<T>::type;
  constexpr int R1 = PlanD<N>::R1, R2 = PlanD<N>::R2, RS = R2 + 1;
  if (lane < R2) {
    const int n2 = lane;
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
        const C wv = tw[n2 * k1];  // wN^(n2 k1), n2 k1 < N
        v = (DIR < 0) ? cmul(v, wv) : cmulc(v, wv);
      }
      ex[k1 * RS + n2] = v;
    }
  }
  __syncwarp();
  if (lane < R1) {
    const int k1 = lane;
    C b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = ex[k1 * RS + n2];
    Dft<R2, DIR>::template run<T, C>(b);
    static_for<0, R2>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      if constexpr (!(DIR < 0 && dead_k2<N, KK>(k2))) st(k1 + R1 * k2, b[k2]);
    });
  }
  __syncwarp();
}

template <typename T, int N, int WR, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(XRowSmem<T, N, WR>::THREADS, 3) k_xrow(PassArgs a) {
  using C = typename CT<T>::type;
  using XS = XRowSmem<T, N, WR>;
  constexpr int K = KK, M = KK + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  C* tw = reinterpret_cast<C*>(smraw);
  {
    const C* __restrict__ twg = static_cast<const C*>(a.tw);
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
  }
  unsigned char* myrow = smraw + XS::TW_BYTES + (size_t)wid * XS::ROW_BYTES;
  C* ex = reinterpret_cast<C*>(myrow);
  T* buf = reinterpret_cast<T*>(myrow + XS::EX_BYTES);
  const C* __restrict__ yb = static_cast<const C*>(a.yb);
  C* __restrict__ xb = static_cast<C*>(a.xb);
  const long long ys = (long long)N * N * M;
  const long long nrows = (long long)N * N;
  const T scale = T(1.0 / ((double)N * N * N));
  const C zero = mk(T(0), T(0));
  // buffer f of this warp's row, position pos
  auto B = [&](int f, int pos) -> T& { return buf[f * N + pos]; };
  T um = T(0);
  MomentSum<T> acc[MODE == XMODE_STATS ? NQ : 1];

  // rows are independent: a warp loops over its rows without block barriers
#pragma unroll 1
  for (long long row = (long long)blockIdx.x * WR + wid; row < nrows; row += (long long)gridDim.x * WR) {
    auto Y = [&](int s, int kx) -> C {
      const long long idx = s * ys + row * M + kx;
      if (!PSC_OK_INDEX(idx, (long long)Y_NSTREAM * ys, a.ctrl)) return zero;
      return yb[idx];
    };
    // Inverse DFT of the packed pair Z[p] = X1[p] + i X2[p] (p <= K; imaginary
    // parts dropped at p = 0), conj(X1[N-p]) + i conj(X2[N-p]) (p >= N-K), 0
    // elsewhere; spec(k, x1, x2) gives X1, X2 at k >= 0 and put(pos, v1, v2)
    // receives the two real fields at position pos.
    auto inv = [&](const auto& spec, const auto& put) {
      warp_row_fft<T, N, +1, KK>(
          [&](int p) -> C {
            C x1, x2;
            if (p <= K) {
              spec(p, x1, x2);
              x1 = shift_in<SHIFT, KK>(x1, a.phase, p);
              x2 = shift_in<SHIFT, KK>(x2, a.phase, p);
              if (p == 0) { x1.y = T(0); x2.y = T(0); }
              return mk(x1.x - x2.y, x1.y + x2.x);
            }
            if (p >= N - K) {
              spec(N - p, x1, x2);
              x1 = shift_in<SHIFT, KK>(x1, a.phase, N - p);
              x2 = shift_in<SHIFT, KK>(x2, a.phase, N - p);
              return mk(x1.x + x2.y, x2.x - x1.y);
            }
            return zero;
          },
          [&](int pos, C v) { put(pos, v.x * scale, v.y * scale); }, ex, tw, lane);
    };
    // Forward DFT of the packed pair get(pos) = x1 + i x2; the transform is
    // staged in buffers b1 (real) and b2 (imaginary), which get may read only
    // in the first step, and the half spectra X1 = (Z[k] + conj Z[N-k])/2,
    // X2 = (Z[k] - conj Z[N-k])/(2i), k <= K, go to streams s0 and s0 + 1.
    auto fwd = [&](const auto& get, int b1, int b2, int s0) {
      warp_row_fft<T, N, -1, KK>(
          get, [&](int k, C v) { B(b1, k) = v.x; B(b2, k) = v.y; }, ex, tw, lane);
      for (int kx = lane; kx <= K; kx += 32) {
        const int kn = kx == 0 ? 0 : N - kx;
        const C A = mk(B(b1, kx), B(b2, kx)), Bn = mk(B(b1, kn), B(b2, kn));
        const C X1 = shift_out<SHIFT, KK>(mk(T(0.5) * (A.x + Bn.x), T(0.5) * (A.y - Bn.y)), a.phase, kx);
        const C X2 = shift_out<SHIFT, KK>(mk(T(0.5) * (A.y + Bn.y), T(0.5) * (Bn.x - A.x)), a.phase, kx);
        const long long i0 = row * M + kx;
        if (PSC_OK_INDEX(i0 + (s0 + 1) * ys, 4 * ys, a.ctrl)) {
          xb[s0 * ys + i0] = X1;
          xb[(s0 + 1) * ys + i0] = X2;
        }
      }
      // the staging buffers are next written after the __syncwarp inside the
      // following transform, which every lane reaches after this loop
    };
    if constexpr (MODE == XMODE_RHS || MODE == XMODE_PRESSURE) {
      // buffers: 0..2 = u1, u2, u3; 3..5 = NL1, NL2, NL3 = (u x omega)_i
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UY, kx); },
          [&](int pos, T u1, T u2) { B(0, pos) = u1; B(1, pos) = u2; });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_UZ, kx); x2 = Y(Y_WX, kx); },
          [&](int pos, T u3, T w1) {
            const T u1 = B(0, pos), u2 = B(1, pos);
            B(2, pos) = u3;
            B(4, pos) = u3 * w1;
            B(5, pos) = -u2 * w1;
            if (a.want_umax) um = max_keep_nan(um, fabs(u1) + fabs(u2) + fabs(u3));
          });
      // omega_2 = d_z u_1 - i kx u_3,  omega_3 = i kx u_2 - d_y u_1
      inv(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx)));
            x2 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
          },
          [&](int pos, T w2, T w3) {
            const T u1 = B(0, pos), u2 = B(1, pos), u3 = B(2, pos);
            B(3, pos) = u2 * w3 - u3 * w2;
            B(4, pos) -= u1 * w3;
            B(5, pos) += u1 * w2;
          });
      fwd([&](int pos) -> C { return mk(B(3, pos), B(4, pos)); }, 3, 4, 0);
      if constexpr (MODE == XMODE_PRESSURE) {
        // (NL3, |u|^2 / 2): the inputs of the modified pressure
        fwd(
            [&](int pos) -> C {
              const T u1 = B(0, pos), u2 = B(1, pos), u3 = B(2, pos);
              return mk(B(5, pos), T(0.5) * (u1 * u1 + u2 * u2 + u3 * u3));
            },
            5, 3, 2);
        continue;
      }
      // u . grad phi into buffer 3 (free again)
      inv([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_PHI, kx), T(kx)); x2 = Y(Y_DYPHI, kx); },
          [&](int pos, T g1, T g2) { B(3, pos) = B(0, pos) * g1 + B(1, pos) * g2; });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZPHI, kx); x2 = zero; },
          [&](int pos, T g3, T) { B(3, pos) += B(2, pos) * g3; });
      fwd([&](int pos) -> C { return mk(B(5, pos), B(3, pos)); }, 5, 3, 2);
    } else if constexpr (MODE == XMODE_STATS) {
      // moments of the diagonal velocity gradients and the scalar gradient
      // (Eqs. 11-12), |omega|^2, u.u, phi u2, phi^2 (Eq. 13)
      auto acc234 = [&](int q, T v) {
        const T v2 = v * v;
        acc[q].add(v2);
        acc[q + 1].add(v2 * v);
        acc[q + 2].add(v2 * v2);
      };
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_UX, kx); x2 = Y(Y_UZ, kx); },
          [&](int pos, T u1, T u3) {
            B(0, pos) = fabs(u1) + fabs(u3);
            acc[0].add(u1 * u1 + u3 * u3);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_UY, kx); x2 = Y(Y_PHI, kx); },
          [&](int pos, T u2, T ph) {
            acc[0].add(u2 * u2);
            acc[20].add(ph * u2);
            acc[21].add(ph * ph);
            um = max_keep_nan(um, B(0, pos) + fabs(u2));
          });
      inv(
          [&](int kx, C& x1, C& x2) {
            x1 = Y(Y_WX, kx);
            x2 = csub(Y(Y_DZUX, kx), mul_ik(Y(Y_UZ, kx), T(kx)));
          },
          [&](int, T w1, T w2) {
            acc[1].add(w1 * w1 + w2 * w2);
          });
      inv(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
            x2 = mul_ik(Y(Y_PHI, kx), T(kx));
          },
          [&](int, T w3, T g1) {
            acc[1].add(w3 * w3);
            acc234(11, g1);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYPHI, kx); x2 = Y(Y_DZPHI, kx); },
          [&](int, T g2, T g3) {
            acc234(14, g2);
            acc234(17, g3);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UX, kx), T(kx)); x2 = Y(Y_DYUY, kx); },
          [&](int, T d11, T d22) {
            acc234(2, d11);
            acc234(5, d22);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUZ, kx); x2 = zero; },
          [&](int, T d33, T) {
            acc234(8, d33);
          });
    }
  }

  // CTA reductions in a fixed order (FP64), through the row buffers
  const int me = threadIdx.x;
  constexpr int NT = XS::THREADS;
  double* red = reinterpret_cast<double*>(smraw + XS::TW_BYTES);
  if (MODE == XMODE_STATS || a.want_umax) {
    __syncthreads();
    red[me] = (double)um;  // the fields here are scaled
    __syncthreads();
    if (me == 0) {
      double m = 0.0;
      for (int i = 0; i < NT; ++i) {
        const double o = red[i];
        m = o > m || o != o ? o : m;
      }
      umax_update(a.ctrl, m);
    }
  }
  if constexpr (MODE == XMODE_STATS) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q * NT + me] = acc[q].value();
    __syncthreads();
    for (int q = me; q < NQ; q += NT) {
      double s = 0.0;
      for (int i = 0; i < NT; ++i) s += red[q * NT + i];
      a.partials[(long long)blockIdx.x * NQ + q] = s;
    }
  }
}

}  // namespace psc
