// Pointwise spectral kernels: the stage combine (projection, forcing, scalar
// source, Lawson IF-RK4 update), forcing amplitude, integrating-factor tables,
// CFL time step, the FP64 statistics reductions and the initial condition.
// Kernels that are not templates are static: several units compile this header.
#pragma once

#include "psc_common.cuh"

namespace psc {

struct CombineArgs {
  Dims d;
  const void* rb;     // unprojected (NL1, NL2, NL3, u.grad phi) in compact layout
  const void* rb2;    // phase-shift dealiasing: the same on the unshifted grid (else null)
  const void* vin;    // stage input state
  void* U;            // state u_n (updated in place at stage 4)
  void* V;            // next stage input
  void* Acc;          // RK accumulator
  void* out;          // RHS output (stage 0 only)
  const void* eu;     // exp(-nu k^2 dt/2), k = 0..K
  const void* ep;     // exp(-D k^2 dt/2)
  Ctrl* ctrl;
  double kF2, beta, nu, D;
  int kF2_floor;  // floor(kF2): the band test in integers
  int forcing, integrator, scalar_on;
};

// Per-mode wavevector of compact index i = ((kz+K) P + (ky+K)) M + kx.
__device__ __forceinline__ void mode_of(const Dims& d, long long i, int& kx, int& ky, int& kz) {
  kx = (int)(i % d.M);
  const long long r = i / d.M;
  ky = (int)(r % d.P) - d.K;
  kz = (int)(r / d.P) - d.K;
}

// A mode of the cube outside the sphere 9|k|^2 < 2 N^2 when that is the retained set.
__device__ __forceinline__ bool outside_sphere(const Dims& d, long long k2) {
  return d.sph && 9 * k2 >= 2LL * d.N * d.N;
}

// STAGE 0: write the right-hand side N(v) to `out`.
// STAGE 1..4: Lawson IF-RK4 with E1 = exp(L dt/2), E2 = E1^2 (L = -nu|k|^2, -D|k|^2):
//   1: V = E1 (U + dt/2 r),   Acc = E2 (U + dt/6 r)
//   2: V = E1 U + dt/2 r,     Acc += dt/3 E1 r
//   3: V = E2 U + dt E1 r,    Acc += dt/3 E1 r
//   4: U = Acc + dt/6 r
// For plain RK4 (section 2.2) E1 = E2 = 1 and r carries the linear terms.
template <typename T, int STAGE>
__device__ __forceinline__ void b_combine(const CombineArgs& c, const long long i) {
  using C = typename CT<T>::type;
  const Dims& d = c.d;
  const long long S = d.S;
  if (STAGE == 4 && i == 0) {
    c.ctrl->t += c.ctrl->dt;
    c.ctrl->step += 1;
  }
  if (i >= S) return;
  int kx, ky, kz;
  mode_of(d, i, kx, ky, kz);
  const int k2 = kx * kx + ky * ky + kz * kz;
  const C* PSC_RESTRICT rb = static_cast<const C*>(c.rb);
  const C* PSC_RESTRICT vin = static_cast<const C*>(c.vin);
  C r0 = rb[i], r1 = rb[S + i], r2 = rb[2 * S + i];
  C r3 = rb[3 * S + i];
  if (c.rb2) {
    // phase-shift dealiasing: the mean of the products of the two grids
    const C* PSC_RESTRICT rc = static_cast<const C*>(c.rb2);
    const C q0 = rc[i], q1 = rc[S + i], q2 = rc[2 * S + i], q3 = rc[3 * S + i];
    r0 = mk(T(0.5) * (q0.x + r0.x), T(0.5) * (q0.y + r0.y));
    r1 = mk(T(0.5) * (q1.x + r1.x), T(0.5) * (q1.y + r1.y));
    r2 = mk(T(0.5) * (q2.x + r2.x), T(0.5) * (q2.y + r2.y));
    r3 = mk(T(0.5) * (q3.x + r3.x), T(0.5) * (q3.y + r3.y));
  }
  // Leray projection (Eq. 7): r - k (k.r)/|k|^2; the k = 0 mode carries no velocity
  if (k2 > 0) {
    const T ik2 = T(1) / T(k2);
    const C dot = mk((kx * r0.x + ky * r1.x + kz * r2.x) * ik2, (kx * r0.y + ky * r1.y + kz * r2.y) * ik2);
    r0 = mk(r0.x - kx * dot.x, r0.y - kx * dot.y);
    r1 = mk(r1.x - ky * dot.x, r1.y - ky * dot.y);
    r2 = mk(r2.x - kz * dot.x, r2.y - kz * dot.y);
  } else {
    r0 = r1 = r2 = mk(T(0), T(0));
  }
  // the stage input is needed in full only on the forcing band and for the
  // explicit linear terms of plain RK4; elsewhere only u2 (scalar source)
  const bool band = c.forcing == 1 && k2 > 0 && k2 <= c.kF2_floor;  // in-stage (constant power) only
  const bool all = band || c.integrator == 1;
  const C zero = mk(T(0), T(0));
  const C v1 = vin[S + i];
  const C v0 = all ? vin[i] : zero, v2 = all ? vin[2 * S + i] : zero, v3 = all ? vin[3 * S + i] : zero;
  // constant-power forcing A u on 0 < |k|^2 <= kF^2
  if (band) {
    const T A = (T)c.ctrl->A;
    r0 = mk(r0.x + A * v0.x, r0.y + A * v0.y);
    r1 = mk(r1.x + A * v1.x, r1.y + A * v1.y);
    r2 = mk(r2.x + A * v2.x, r2.y + A * v2.y);
  }
  // scalar: -(u.grad phi) - beta u2 (Eq. 8)
  C rp = mk(T(0), T(0));
  if (c.scalar_on) {
    const T b = (T)c.beta;
    rp = mk(-r3.x - b * v1.x, -r3.y - b * v1.y);
  }
  if (outside_sphere(d, k2)) {
    // not retained: no tendency (the state is zero there)
    r0 = r1 = r2 = rp = zero;
  }
  T E1u = T(1), E1p = T(1);
  if (c.integrator == 1) {
    const T lu = (T)(-c.nu * k2), lp = c.scalar_on ? (T)(-c.D * k2) : T(0);
    r0 = mk(r0.x + lu * v0.x, r0.y + lu * v0.y);
    r1 = mk(r1.x + lu * v1.x, r1.y + lu * v1.y);
    r2 = mk(r2.x + lu * v2.x, r2.y + lu * v2.y);
    rp = mk(rp.x + lp * v3.x, rp.y + lp * v3.y);
  } else {
    const T* eu = static_cast<const T*>(c.eu);
    const T* ep = static_cast<const T*>(c.ep);
    const int ax = kx, ay = ky < 0 ? -ky : ky, az = kz < 0 ? -kz : kz;
    E1u = eu[ax] * eu[ay] * eu[az];
    E1p = ep[ax] * ep[ay] * ep[az];
  }
  if (STAGE == 0) {
    C* out = static_cast<C*>(c.out);
    out[i] = r0;
    out[S + i] = r1;
    out[2 * S + i] = r2;
    out[3 * S + i] = rp;
    return;
  }
  C* PSC_RESTRICT U = static_cast<C*>(c.U);
  C* PSC_RESTRICT V = static_cast<C*>(c.V);
  C* PSC_RESTRICT Acc = static_cast<C*>(c.Acc);
  const T h = (T)c.ctrl->dt;
  const C r[4] = {r0, r1, r2, rp};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const long long j = f * S + i;
    const T E1 = f < 3 ? E1u : E1p;
    const T E2 = E1 * E1;
    const C rf = r[f];
    if (STAGE == 1) {
      const C u = U[j];
      V[j] = mk(E1 * (u.x + T(0.5) * h * rf.x), E1 * (u.y + T(0.5) * h * rf.y));
      Acc[j] = mk(E2 * (u.x + h / T(6) * rf.x), E2 * (u.y + h / T(6) * rf.y));
    } else if (STAGE == 2) {
      const C u = U[j], a = Acc[j];
      V[j] = mk(E1 * u.x + T(0.5) * h * rf.x, E1 * u.y + T(0.5) * h * rf.y);
      Acc[j] = mk(a.x + h / T(3) * E1 * rf.x, a.y + h / T(3) * E1 * rf.y);
    } else if (STAGE == 3) {
      const C u = U[j], a = Acc[j];
      V[j] = mk(E2 * u.x + h * E1 * rf.x, E2 * u.y + h * E1 * rf.y);
      Acc[j] = mk(a.x + h / T(3) * E1 * rf.x, a.y + h / T(3) * E1 * rf.y);
    } else {
      const C a = Acc[j];
      U[j] = mk(a.x + h / T(6) * rf.x, a.y + h / T(6) * rf.y);
    }
  }
}
template <typename T, int STAGE>
__global__ void __launch_bounds__(256) k_combine(CombineArgs c) {
  b_combine<T, STAGE>(c, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Modified pressure (section 2.2, Eq. 6) from the transformed pressure inputs
// r = (u x omega, |u|^2/2) on the retained set: with u.grad u = -u x omega +
// grad(|u|^2/2), p_hat = i k.(u.grad u)_hat/|k|^2 = -i k.(u x omega)_hat/|k|^2
// - (|u|^2/2)_hat; p_hat = 0 at k = 0.
template <typename T>
__global__ void __launch_bounds__(256) k_pressure(Dims d, const void* rb_, void* out_) {
  using C = typename CT<T>::type;
  const long long S = d.S;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S) return;
  int kx, ky, kz;
  mode_of(d, i, kx, ky, kz);
  const int k2 = kx * kx + ky * ky + kz * kz;
  const C* r = static_cast<const C*>(rb_);
  C* out = static_cast<C*>(out_);
  if (k2 == 0) {
    out[i] = mk(T(0), T(0));
    return;
  }
  const C a = r[i], b = r[S + i], c = r[2 * S + i], q = r[3 * S + i];
  const T ik2 = T(1) / T(k2);
  const C kdot = mk(kx * a.x + ky * b.x + kz * c.x, kx * a.y + ky * b.y + kz * c.y);
  // -i (k.NL) / |k|^2 - q
  out[i] = mk(kdot.y * ik2 - q.x, -kdot.x * ik2 - q.y);
}

// Band energy E_f = sum_{0<|k|^2<=kF^2} w |u_k|^2 / (2 N^6) of the state `in`
// in a fixed order (one thread), and A = eps_inj / (2 E_f) (0 if E_f = 0).
template <typename T>
__device__ __forceinline__ void b_famp(Dims d, const void* in_, Ctrl* ctrl, double kF2, double eps_inj, int forcing,
                                       int step_start) {
  using C = typename CT<T>::type;
  const C* in = static_cast<const C*>(in_);
  int kb = 0;
  while ((double)(kb + 1) * (kb + 1) <= kF2) ++kb;
  if (kb > d.K) kb = d.K;
  double s = 0.0;
  for (int kz = -kb; kz <= kb; ++kz)
    for (int ky = -kb; ky <= kb; ++ky)
      for (int kx = 0; kx <= kb; ++kx) {
        const int k2 = kx * kx + ky * ky + kz * kz;
        if (k2 == 0 || (double)k2 > kF2) continue;
        const long long i = ((long long)(kz + d.K) * d.P + (ky + d.K)) * d.M + kx;
        const double w = kx == 0 ? 1.0 : 2.0;
        for (int f = 0; f < 3; ++f) {
          const C v = in[f * d.S + i];
          s += w * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
        }
      }
  const double n3 = (double)d.N * d.N * d.N;
  const double ef = s / (2.0 * n3 * n3);
  ctrl->Ef = ef;
  if (step_start) ctrl->Ef_start = ef;
  // the deterministic forcing keeps the rate of its last rescaling in A
  if (forcing != 2) ctrl->A = (forcing == 1 && ef > 1e-300) ? eps_inj / (2.0 * ef) : 0.0;
}
template <typename T>
__global__ void k_famp(Dims d, const void* in_, Ctrl* ctrl, double kF2, double eps_inj, int forcing,
                       int step_start) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  b_famp<T>(d, in_, ctrl, kF2, eps_inj, forcing, step_start);
}

// The paper's deterministic forcing (section 2.3), after the last stage of a
// step: the band 0 < |k|^2 <= kF^2 of the new state is multiplied by
// f = sqrt(Ef0 / E_f) so that it keeps the energy Ef0 it had at the start of
// the first step (Ef0 < 0: the target is taken from this step's start).  A
// records the equivalent rate ln(f) / dt.  One thread, fixed order.
template <typename T>
__device__ __forceinline__ void b_hold(Dims d, void* u_, Ctrl* ctrl, double kF2) {
  using C = typename CT<T>::type;
  C* u = static_cast<C*>(u_);
  int kb = 0;
  while ((double)(kb + 1) * (kb + 1) <= kF2) ++kb;
  if (kb > d.K) kb = d.K;
  auto for_band = [&](auto&& fn) {
    for (int kz = -kb; kz <= kb; ++kz)
      for (int ky = -kb; ky <= kb; ++ky)
        for (int kx = 0; kx <= kb; ++kx) {
          const int k2 = kx * kx + ky * ky + kz * kz;
          if (k2 == 0 || (double)k2 > kF2) continue;
          fn(((long long)(kz + d.K) * d.P + (ky + d.K)) * d.M + kx, kx == 0 ? 1.0 : 2.0);
        }
  };
  double s = 0.0;
  for_band([&](long long i, double w) {
    for (int f = 0; f < 3; ++f) {
      const C v = u[f * d.S + i];
      s += w * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
    }
  });
  const double n3 = (double)d.N * d.N * d.N;
  const double ef = s / (2.0 * n3 * n3);
  double ef0 = ctrl->Ef0;
  if (ef0 < 0.0) {
    ef0 = ctrl->Ef_start;
    ctrl->Ef0 = ef0;
  }
  const double f = ef > 1e-300 ? sqrt(ef0 / ef) : 1.0;
  for_band([&](long long i, double) {
    for (int c = 0; c < 3; ++c) u[c * d.S + i] = cscale(u[c * d.S + i], (T)f);
  });
  ctrl->A = log(f) / ctrl->dt;
  ctrl->Ef = ef * f * f;
}
template <typename T>
__global__ void k_hold(Dims d, void* u_, Ctrl* ctrl, double kF2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  b_hold<T>(d, u_, ctrl, kF2);
}

// Integrating factors per axis: e(k) = exp(-nu k^2 dt / 2) (and with D), so
// that exp(-nu |k|^2 dt/2) = e(|kx|) e(|ky|) e(|kz|).  FP64 exp, stored as T.
template <typename T>
__device__ __forceinline__ void b_iftab(int K, const Ctrl* ctrl, double nu, double D, T* eu, T* ep, int k) {
  if (k > K) return;
  const double dt = ctrl->dt;
  eu[k] = (T)exp(-nu * (double)k * k * dt * 0.5);
  ep[k] = (T)exp(-D * (double)k * k * dt * 0.5);
}
template <typename T>
__global__ void k_iftab(int K, const Ctrl* ctrl, double nu, double D, T* eu, T* ep) {
  b_iftab<T>(K, ctrl, nu, D, eu, ep, blockIdx.x * blockDim.x + threadIdx.x);
}

#ifndef PSC_SHELLS_ONLY
// dt = cfl dx / max(|u1|+|u2|+|u3|)  (Eq. 10) on every record_every-th step
// (the step count lives on the device, so the launch sequence of a step never
// changes and can be captured in a CUDA graph); a non-finite maximum raises the
// instability flag and leaves dt unchanged.
__device__ __forceinline__ void b_cfl(Ctrl* c, double cfl, double dx, int record_every) {
  if (c->step % record_every != 0) return;
  const double m = __longlong_as_double((long long)c->umax_bits);
  if (!(m <= 1.7976931348623157e308)) { c->err |= 2; return; }
  if (m > 0.0) c->dt = cfl * dx / m;
}
static __global__ void k_cfl(Ctrl* c, double cfl, double dx, int record_every) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  b_cfl(c, cfl, dx, record_every);
}

#endif  // PSC_SHELLS_ONLY

// Fixed-order block sum of one double (every thread passes its value; the
// result is valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
  return s;
}

// floor(sqrt(a)) for 0 <= a < 2^46: an FP32 estimate corrected in integers
// (exact; the FP64 square root is slow on this part)
__device__ __forceinline__ long long isqrt_floor(long long a) {
  if (a <= 0) return 0;
  long long s = (long long)sqrtf((float)a);
  while (s * s > a) --s;
  while ((s + 1) * (s + 1) <= a) ++s;
  return s;
}

// Shell n = floor(|k| + 1/2), i.e. n^2 - n < |k|^2 <= n^2 + n.  One CTA per
// shell sums w |u|^2, w |phi|^2, |k|^2 w |u|^2, |k|^2 w |phi|^2 and
// w Re(conj(phi) u2) over the shell's stored modes (w = 1 at kx = 0, else 2).
// Each thread accumulates in the state's precision (compensated sums in FP32,
// since FP64 arithmetic is slow on this part), then the CTA adds the threads'
// sums in FP64 in a fixed order.  out[q * nshell + n] holds the raw sums.
template <typename T>
__global__ void __launch_bounds__(256) k_shells(Dims d, const void* u_, const void* phi_, int nshell,
                                               double* out) {
  using C = typename CT<T>::type;
  __shared__ double sm[32];
  const C* u = static_cast<const C*>(u_);
  const C* phi = static_cast<const C*>(phi_);
  const int n = blockIdx.x;
  const long long lo = n == 0 ? -1 : (long long)n * n - n;  // exclusive
  const long long hi = n == 0 ? 0 : (long long)n * n + n;   // inclusive
  const int kb = (n + 1) < d.K ? (n + 1) : d.K;
  const int side = 2 * kb + 1;
  MomentSum<T> acc[NSQ];
  // amplitudes are summed as u_hat / N^3 (order-one numbers, far from the FP32
  // range limits); the raw sums are restored in FP64 at the end
  const double n3 = (double)d.N * d.N * d.N;
  const T sc = (T)(1.0 / n3);
  for (int q = threadIdx.x; q < side * side; q += blockDim.x) {
    const int kz = q / side - kb, ky = q % side - kb;
    const long long r2 = (long long)kz * kz + (long long)ky * ky;
    if (r2 > hi) continue;
    const long long x0 = (lo - r2 < 0) ? 0 : isqrt_floor(lo - r2) + 1;
    long long x1 = isqrt_floor(hi - r2);
    if (x1 > d.K) x1 = d.K;
    const long long base = ((long long)(kz + d.K) * d.P + (ky + d.K)) * d.M;
    for (long long kx = x0; kx <= x1; ++kx) {
      const long long i = base + kx;
      const T w = kx == 0 ? T(1) : T(2);
      const T k2 = (T)(r2 + kx * kx);  // exact: |k|^2 < 2^24
      const C a = cscale(u[i], sc), b = cscale(u[d.S + i], sc), c = cscale(u[2 * d.S + i], sc);
      const T eu = w * (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y + c.x * c.x + c.y * c.y);
      acc[0].add(eu);
      acc[2].add(k2 * eu);
      if (phi) {
        const C p = cscale(phi[i], sc);
        const T ep = w * (p.x * p.x + p.y * p.y);
        acc[1].add(ep);
        acc[3].add(k2 * ep);
        acc[4].add(w * (p.x * b.x + p.y * b.y));
      }
    }
  }
  for (int q = 0; q < NSQ; ++q) {
    const double s = block_sum(acc[q].value(), sm);
    if (threadIdx.x == 0) out[q * nshell + n] = s * n3 * n3;
    __syncthreads();
  }
}

#ifndef PSC_SHELLS_ONLY
// Sum the X-pass partials over warps in a fixed order.
static __global__ void k_reduce_moments(const double* partials, int nw, Ctrl* ctrl) {
  const int q = threadIdx.x;
  if (q >= NQ) return;
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += partials[(long long)w * NQ + q];
  ctrl->moments[q] = s;
}

// ---------------------------------------------------------------------------
// Initial condition (section 2.3; Rogallo-type random solenoidal field)
// ---------------------------------------------------------------------------

// Element i of the SplitMix64 stream seeded with `seed` (Steele, Lea and
// Flood 2014): mix(seed + (i+1) gamma).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform_at(unsigned long long seed, unsigned long long i) {
  return ((double)(splitmix64_at(seed, i) >> 11) + 1.0) * 0x1.0p-53;
}

// Raw draw: for the canonical wavevector c of each mode (kx > 0, or kx = 0 and
// (ky, kz) > 0 lexicographically; otherwise c = -k), one Box-Muller complex
// Gaussian per component from stream elements 8 key(c) + 2j, + 2j + 1,
// projected normal to c; non-canonical modes take the conjugate.
static __global__ void k_ic_draw(Dims d, unsigned long long seed, double2* z) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.S) return;
  int kx, ky, kz;
  mode_of(d, i, kx, ky, kz);
  const bool canon = kx > 0 || (kx == 0 && (ky > 0 || (ky == 0 && kz > 0)));
  const int cx = canon ? kx : -kx, cy = canon ? ky : -ky, cz = canon ? kz : -kz;
  const long long k2 = (long long)kx * kx + (long long)ky * ky + (long long)kz * kz;
  double re[3], im[3];
  const unsigned long long key = ((unsigned long long)(cx + 2048) << 24) |
                                 ((unsigned long long)(cy + 2048) << 12) |
                                 (unsigned long long)(cz + 2048);
  for (int c = 0; c < 3; ++c) {
    const double u1 = uniform_at(seed, key * 8ull + 2ull * c);
    const double u2 = uniform_at(seed, key * 8ull + 2ull * c + 1ull);
    const double r = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    re[c] = r * co;
    im[c] = r * s;
  }
  if (k2 == 0 || outside_sphere(d, k2)) {
    for (int c = 0; c < 3; ++c) z[c * d.S + i] = make_double2(0.0, 0.0);
    return;
  }
  const double kc[3] = {(double)cx, (double)cy, (double)cz};
  const double kdr = (kc[0] * re[0] + kc[1] * re[1] + kc[2] * re[2]) / (double)k2;
  const double kdi = (kc[0] * im[0] + kc[1] * im[1] + kc[2] * im[2]) / (double)k2;
  for (int c = 0; c < 3; ++c) {
    const double a = re[c] - kc[c] * kdr, b = im[c] - kc[c] * kdi;
    z[c * d.S + i] = make_double2(a, canon ? b : -b);
  }
}

// Per-shell factors sqrt(E_target(n) / E_raw(n)); E_target follows the chosen
// shape (0: n^4 exp(-2 (n/4)^2), 2: Eq. 9 with kF), normalised to K0 over the
// shells that hold modes.  Eraw holds the raw sums w|z|^2 (any common scale).
static __global__ void k_ic_factors(int nshell, const double* Eraw, double norm, double K0, int shape,
                             double kF, double* fac) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  auto target = [&](int n) -> double {
    if (n == 0) return 0.0;
    const double x = (double)n;
    if (shape == 2) return x <= kF ? (x / kF) * (x / kF) : pow(x / kF, -5.0 / 3.0);
    return x * x * x * x * exp(-2.0 * (x / 4.0) * (x / 4.0));
  };
  double tot = 0.0;
  for (int n = 0; n < nshell; ++n)
    if (Eraw[n] > 0.0) tot += target(n);
  for (int n = 0; n < nshell; ++n) {
    const double raw = Eraw[n] * norm;
    fac[n] = (raw > 0.0 && tot > 0.0 && K0 > 0.0) ? sqrt(K0 * target(n) / tot / raw) : 0.0;
  }
}

// U = fac[shell] z (+ Taylor-Green u = (sin x cos y cos z, -cos x sin y cos z, 0),
// whose coefficients at kx = 1, |ky| = |kz| = 1 are -i N^3/8 and i ky N^3/8);
// phi = 0.
template <typename T>
__global__ void k_ic_finish(Dims d, const double2* z, const double* fac, int taylor_green, void* U_) {
  using C = typename CT<T>::type;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.S) return;
  int kx, ky, kz;
  mode_of(d, i, kx, ky, kz);
  const long long k2 = (long long)kx * kx + (long long)ky * ky + (long long)kz * kz;
  long long n = isqrt_floor(k2);
  if (k2 > n * n + n) ++n;
  const double f = outside_sphere(d, k2) ? 0.0 : fac[n];
  double v[3][2];
  for (int c = 0; c < 3; ++c) {
    const double2 q = z[c * d.S + i];
    v[c][0] = f * q.x;
    v[c][1] = f * q.y;
  }
  if (taylor_green && kx == 1 && (ky == 1 || ky == -1) && (kz == 1 || kz == -1)) {
    const double n3 = (double)d.N * d.N * d.N;
    v[0][1] += -n3 / 8.0;
    v[1][1] += (double)ky * n3 / 8.0;
  }
  C* U = static_cast<C*>(U_);
  for (int c = 0; c < 3; ++c) U[c * d.S + i] = mk((T)v[c][0], (T)v[c][1]);
  U[3 * d.S + i] = mk(T(0), T(0));
}

#endif  // PSC_SHELLS_ONLY

}  // namespace psc
