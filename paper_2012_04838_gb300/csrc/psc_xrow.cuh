// X pass through shared-memory rows: the fused x transforms and products of
// the right-hand side (u x omega, u . grad phi), the pressure inputs and the
// statistics moments, for grids whose two-step plan gives a row too few lanes
// to hold its values in registers (N = 520 = 20 x 26 splits over 2 lanes).
//
// A CTA takes W rows (z, y) with TPL threads each.  Every transform runs
// through strided_fft along the row (the "column" index of the strided passes
// is the row here): an inverse reads the packed half spectra of two real
// fields from the y-inverse streams and leaves the two physical fields, scaled
// by 1/N^3, in per-row buffers in shared memory; products are formed in the
// store callbacks, point by point; a forward transform reads a packed pair of
// buffers and writes both half spectra kx <= K.  Six buffers of N reals per
// row suffice for the right-hand side (u1, u2, u3 and the three components of
// the nonlinear term while it is assembled).
// Included by psc_passes.cuh after the strided transforms it builds on.
#pragma once

namespace psc {

template <typename T, int N, int W> struct XRowSmem {
  static constexpr int NB = 6;  // row buffers of N reals
  static constexpr int THREADS = W * PlanD<N>::TPL;
  static constexpr size_t BUF_OFF = (StridedSmem<T, N, W>::BYTES + 15) / 16 * 16;
  static constexpr size_t BUF_BYTES = (size_t)NB * N * W * sizeof(T);
  static constexpr size_t RED_BYTES = (size_t)NQ * THREADS * sizeof(double);
  static constexpr size_t SMEM = BUF_OFF + (BUF_BYTES > RED_BYTES ? BUF_BYTES : RED_BYTES);
};

// Rows per CTA: the widest of 16, 8, 4 (FP64: 8, 4) whose shared memory fits.
template <typename T, int N> struct XRowCfg {
  static constexpr size_t LIMIT = 220 * 1024;
  static constexpr int W = (sizeof(T) == 4 && XRowSmem<T, N, 16>::SMEM <= LIMIT) ? 16
                           : (XRowSmem<T, N, 8>::SMEM <= LIMIT)                    ? 8
                                                                                   : 4;
  using S = XRowSmem<T, N, W>;
  static_assert(S::SMEM <= LIMIT, "row buffers do not fit in shared memory");
};

template <typename T, int N, int W, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(XRowSmem<T, N, W>::THREADS) k_xrow(PassArgs a) {
  using C = typename CT<T>::type;
  using XS = XRowSmem<T, N, W>;
  constexpr int K = KK, M = KK + 1, TPL = PlanD<N>::TPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  T* buf = reinterpret_cast<T*>(smraw + XS::BUF_OFF);
  const int w = threadIdx.x, t = threadIdx.y;
  const C* tw = strided_twiddles<T, N, W>(smraw, static_cast<const C*>(a.tw));
  const C* __restrict__ yb = static_cast<const C*>(a.yb);
  C* __restrict__ xb = static_cast<C*>(a.xb);
  const long long ys = (long long)N * N * M;
  const long long nrows = (long long)N * N;
  const T scale = T(1.0 / ((double)N * N * N));
  const C zero = mk(T(0), T(0));
  // buffer f of this thread's row, position pos
  auto B = [&](int f, int pos) -> T& { return buf[((size_t)f * N + pos) * W + w]; };
  T um = T(0);
  MomentSum<T> acc[MODE == XMODE_STATS ? NQ : 1];

#pragma unroll 1
  for (long long r0 = (long long)blockIdx.x * W; r0 < nrows; r0 += (long long)gridDim.x * W) {
    const long long row = r0 + w;
    const bool valid = row < nrows;
    auto Y = [&](int s, int kx) -> C {
      if (!valid) return zero;
      const long long idx = s * ys + row * M + kx;
      if (!PSC_OK_INDEX(idx, (long long)Y_NSTREAM * ys, a.ctrl)) return zero;
      return yb[idx];
    };
    // Inverse DFT of the packed pair Z[p] = X1[p] + i X2[p] (p <= K; imaginary
    // parts dropped at p = 0), conj(X1[N-p]) + i conj(X2[N-p]) (p >= N-K), 0
    // elsewhere; spec(k, x1, x2) gives X1, X2 at k >= 0 and put(pos, v1, v2)
    // receives the two real fields at position pos.
    auto inv = [&](const auto& spec, const auto& put) {
      strided_fft<T, N, W, +1, KK>(
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
          [&](int pos, C v) { put(pos, v.x * scale, v.y * scale); }, sm, tw, t, w);
    };
    // Forward DFT of the packed pair get(pos) = x1 + i x2; the transform is
    // staged in buffers b1 (real) and b2 (imaginary), which get may read only
    // in the first step, and the half spectra X1 = (Z[k] + conj Z[N-k])/2,
    // X2 = (Z[k] - conj Z[N-k])/(2i), k <= K, go to streams s0 and s0 + 1.
    auto fwd = [&](const auto& get, int b1, int b2, int s0) {
      strided_fft<T, N, W, -1, KK>(
          get, [&](int k, C v) { B(b1, k) = v.x; B(b2, k) = v.y; }, sm, tw, t, w);
      for (int kx = t; kx <= K; kx += TPL) {
        const int kn = kx == 0 ? 0 : N - kx;
        const C A = mk(B(b1, kx), B(b2, kx)), Bn = mk(B(b1, kn), B(b2, kn));
        const C X1 = shift_out<SHIFT, KK>(mk(T(0.5) * (A.x + Bn.x), T(0.5) * (A.y - Bn.y)), a.phase, kx);
        const C X2 = shift_out<SHIFT, KK>(mk(T(0.5) * (A.y + Bn.y), T(0.5) * (Bn.x - A.x)), a.phase, kx);
        if (!valid) continue;
        const long long i0 = row * M + kx;
        if (PSC_OK_INDEX(i0 + (s0 + 1) * ys, 4 * ys, a.ctrl)) {
          xb[s0 * ys + i0] = X1;
          xb[(s0 + 1) * ys + i0] = X2;
        }
      }
      // the staging buffers are next written after the barrier inside the
      // following transform, which every thread reaches after this loop
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
            if (a.want_umax && valid) um = max_keep_nan(um, fabs(u1) + fabs(u2) + fabs(u3));
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
            if (valid) acc[0].add(u1 * u1 + u3 * u3);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_UY, kx); x2 = Y(Y_PHI, kx); },
          [&](int pos, T u2, T ph) {
            if (!valid) return;
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
            if (valid) acc[1].add(w1 * w1 + w2 * w2);
          });
      inv(
          [&](int kx, C& x1, C& x2) {
            x1 = csub(mul_ik(Y(Y_UY, kx), T(kx)), Y(Y_DYUX, kx));
            x2 = mul_ik(Y(Y_PHI, kx), T(kx));
          },
          [&](int, T w3, T g1) {
            if (!valid) return;
            acc[1].add(w3 * w3);
            acc234(11, g1);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_DYPHI, kx); x2 = Y(Y_DZPHI, kx); },
          [&](int, T g2, T g3) {
            if (!valid) return;
            acc234(14, g2);
            acc234(17, g3);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = mul_ik(Y(Y_UX, kx), T(kx)); x2 = Y(Y_DYUY, kx); },
          [&](int, T d11, T d22) {
            if (!valid) return;
            acc234(2, d11);
            acc234(5, d22);
          });
      inv([&](int kx, C& x1, C& x2) { x1 = Y(Y_DZUZ, kx); x2 = zero; },
          [&](int, T d33, T) {
            if (valid) acc234(8, d33);
          });
    }
  }

  // CTA reductions in a fixed order (FP64), through the row buffers
  const int me = t * W + w;
  constexpr int NT = XS::THREADS;
  double* red = reinterpret_cast<double*>(smraw + XS::BUF_OFF);
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
