// Staged strided passes: the same transforms as k_zinv / k_yinv / k_yfwd /
// k_zfwd, with each CTA's input tile (the W-wide kx runs of every position of
// its lines) brought into shared memory by TMA tensor copies
// (cp.async.bulk.tensor) on an mbarrier.  The tile of the next transform is
// requested as soon as the current one has been read into registers, so its
// global latency overlaps the current transform's compute and stores.
//
// Built for FP32 where a kx row is a multiple of 16 bytes (M even), which the
// tensor-map strides require; elsewhere the unstaged kernels run.
#pragma once

#include <cuda.h>

#include "psc_common.cuh"

namespace psc {

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// Staging tile of a pass: ROWS line positions (the P retained wavenumbers of an
// inverse pass, the N points of a forward pass) of W complex values each,
// fetched as NBOX boxes of BOXR rows (a box has at most 256 rows).
template <typename T, int N, int W, bool INV, int KK = (N - 1) / 3> struct StagedTile {
  using C = typename CT<T>::type;
  static constexpr int ROWS = INV ? 2 * KK + 1 : N;
  static constexpr int NBOX = (ROWS + 255) / 256;
  // rows per box: enough for NBOX boxes to cover ROWS, rounded up so that every
  // box starts 128-byte aligned (a multiple of 128 / (W * sizeof(C)) rows, and even)
  static constexpr int RALIGN = 128 / (W * (int)sizeof(C)) > 2 ? 128 / (W * (int)sizeof(C)) : 2;
  static constexpr int BOXR = ((ROWS + NBOX - 1) / NBOX + RALIGN - 1) / RALIGN * RALIGN;
  static constexpr unsigned BOX_BYTES = (unsigned)(BOXR * W * sizeof(C));
  static constexpr unsigned BYTES = NBOX * BOX_BYTES;
  // The exchange buffer, then the staging tile, then (TW_SMEM) the step-1
  // twiddle table.  The table is kept in shared memory when it costs no CTA
  // per SM; otherwise the twiddles are read through L1
  static constexpr size_t EXCH = StridedSmem<T, N, W>::EXCH_BYTES;
  static constexpr size_t TWB = (size_t)N * sizeof(C);
  static constexpr size_t STG_OFF = (EXCH + 127) / 128 * 128;
  static constexpr size_t BASE = STG_OFF + BYTES + sizeof(unsigned long long);
  static constexpr int fit(size_t b) { return (int)((228 * 1024) / (b + 1024)); }
  // (inverse passes only: measured faster there, slower for the forward ones)
  static constexpr bool TW_SMEM =
      INV && BASE + TWB <= 227 * 1024 && (fit(BASE + TWB) >= fit(BASE) || fit(BASE + TWB) >= 4);
  static constexpr size_t TW_OFF = STG_OFF + BYTES;  // 128-byte aligned
  static constexpr size_t BAR_OFF = TW_OFF + (TW_SMEM ? TWB : 0);
  static constexpr size_t SMEM = BAR_OFF + sizeof(unsigned long long);
  // CTAs per SM that fit its 228 KB of shared memory (1 KB reserved per CTA)
  static constexpr int FIT = fit(SMEM);
  // no more CTAs than leave every thread 128 registers
  static constexpr int RFIT = 512 / (W * PlanD<N>::TPL) < 1 ? 1 : 512 / (W * PlanD<N>::TPL);
  static constexpr int MINB = FIT < 1 ? 1 : (FIT < RFIT ? FIT : RFIT);
  static_assert(BOX_BYTES % 128 == 0, "boxes start 128-byte aligned");
  static_assert(W * sizeof(C) % 16 == 0, "a box row is a multiple of 16 bytes");
};

// One length-N DFT per column from step-1 inputs already in registers:
// in[j][n1] is line position R2 n1 + t + j TPL.  Same steps as strided_fft,
// with the step-1 twiddles wN^(n2 k1) from the shared table of
// strided_twiddles (TW_SMEM) or from the global table tw.  It does not end
// with a barrier: the caller's next CTA barrier must come before the exchange
// buffer is written again.
template <typename T, int N, int W, int DIR, bool TW_SMEM, int KK, class ST>
__device__ __forceinline__ void strided_fft_regs(typename CT<T>::type (&in)[PlanD<N>::J1][PlanD<N>::R1],
                                                 const ST& st, typename CT<T>::type* sm,
                                                 const typename CT<T>::type* __restrict__ tw, int t, int w) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  using SM = StridedSmem<T, N, W>;
  constexpr int R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, J1 = PL::J1, J2 = PL::J2;
#pragma unroll
  for (int j = 0; j < J1; ++j) {
    const int n2 = t + j * TPL;
    first_dft<T, N, DIR, KK>(in[j]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C v = in[j][k1];
      if (k1 > 0) {
        // wN^(n2 k1), n2 k1 < N
        const C wv = TW_SMEM ? tw[(j * R1 + k1) * TPL + t] : __ldg(&tw[n2 * k1]);
        v = (DIR < 0) ? cmul(v, wv) : cmulc(v, wv);
      }
      sm[k1 * SM::ROW + n2 * W + w] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J2; ++j) {
    const int k1 = t + j * TPL;
    C b[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) b[n2] = sm[k1 * SM::ROW + n2 * W + w];
    Dft<R2, DIR>::template run<T, C>(b);
    static_for<0, R2>([&](auto kc) {
      constexpr int k2 = decltype(kc)::value;
      if constexpr (!(DIR < 0 && dead_k2<N, KK>(k2))) st(k1 + R1 * k2, b[k2]);
    });
  }
}

// Transform tr of a pass: source field / stream, how its line is formed, and
// the output stream.  kind 0: the source; 1: i k times the source; 2: i k
// times the source minus stream s2 (omega_x = d_y u_z - d_z u_y).
// MODE: z-inverse 0 (7 streams) or 1 (8, for the statistics and the convective
// form); y-inverse YMODE_RHS (9), YMODE_STATS (11) or YMODE_CONVECTIVE (12).
// Transforms of one source run one after another: the second reads the tile
// still staged instead of copying it again (reuses()).
template <int PASS, int MODE> struct StagedPlan {
  static constexpr int NT = PASS == SP_ZINV   ? (MODE ? 8 : 7)
                            : PASS == SP_YINV ? (MODE == YMODE_CONVECTIVE ? 12 : MODE == YMODE_STATS ? 11 : 9)
                                              : 4;
  __device__ __forceinline__ static void get(int tr, int& src, int& kind, int& s2, int& out) {
    s2 = 0;
    if constexpr (PASS == SP_ZINV) {
      // u_x, d_z u_x, u_y, d_z u_y, u_z, [d_z u_z], phi, d_z phi
      int t = tr;
      if (MODE) {
        if (t == 5) { src = 2; kind = 1; out = Z_DZUZ; return; }
        if (t > 5) --t;
      }
      switch (t) {
        case 0: src = 0; kind = 0; out = Z_UX; break;
        case 1: src = 0; kind = 1; out = Z_DZUX; break;
        case 2: src = 1; kind = 0; out = Z_UY; break;
        case 3: src = 1; kind = 1; out = Z_DZUY; break;
        case 4: src = 2; kind = 0; out = Z_UZ; break;
        case 5: src = 3; kind = 0; out = Z_PHI; break;
        default: src = 3; kind = 1; out = Z_DZPHI; break;
      }
    } else if constexpr (PASS == SP_YINV) {
      // u_x, d_y u_x, u_y, [d_y u_y], u_z, omega_x, d_z u_x, phi, d_y phi,
      // d_z phi, [d_z u_z, [d_z u_y]]
      int t = tr;
      if (MODE != YMODE_RHS) {
        if (t == 3) { src = Z_UY; kind = 1; out = Y_DYUY; return; }
        if (t > 3) --t;
      }
      switch (t) {
        case 0: src = Z_UX; kind = 0; out = Y_UX; break;
        case 1: src = Z_UX; kind = 1; out = Y_DYUX; break;
        case 2: src = Z_UY; kind = 0; out = Y_UY; break;
        case 3: src = Z_UZ; kind = 0; out = Y_UZ; break;
        case 4:  // omega_x = d_y u_z - d_z u_y (convective form: d_y u_z alone)
          src = Z_UZ; kind = MODE == YMODE_CONVECTIVE ? 1 : 2; s2 = Z_DZUY; out = Y_WX; break;
        case 5: src = Z_DZUX; kind = 0; out = Y_DZUX; break;
        case 6: src = Z_PHI; kind = 0; out = Y_PHI; break;
        case 7: src = Z_PHI; kind = 1; out = Y_DYPHI; break;
        case 8: src = Z_DZPHI; kind = 0; out = Y_DZPHI; break;
        case 9: src = Z_DZUZ; kind = 0; out = Y_DZUZ; break;
        default: src = Z_DZUY; kind = 0; out = Y_DZUY; break;
      }
    } else {
      src = tr;
      kind = 0;
      out = tr;
    }
  }
  // transform tr reads the same tile as transform tr - 1
  __device__ __forceinline__ static bool reuses(int tr) {
    if (tr == 0) return false;
    int s0, s1, k, x, o;
    get(tr - 1, s0, k, x, o);
    get(tr, s1, k, x, o);
    return s0 == s1;
  }
};

// grid (ceil(M/W), P or N), block (W, TPL).  blockIdx.y is the fixed ky (z
// passes) or z (y passes) of the CTA's lines.  `tm` describes the pass input:
//   z-inverse: compact fields, 3D {2M floats, P (ky), 4P (field, kz)}
//   y-inverse: z-stage streams, 2D {2M, Z_NSTREAM N P}
//   y-forward: x-pass output,   2D {2M, 4 N N}
//   z-forward: y-forward output, 3D {2M, P (ky), 4N (stream, z)}
// KK: the retained half-width (the 2/3 rule's, or the cube that stores the
// phase-shift sphere); SHIFT: the inputs are multiplied by exp(i k pi / N) and
// the outputs by its conjugate (the grid shifted by half a cell).
template <typename T, int N, int W, int PASS, int MODE, int KK = (N - 1) / 3, bool SHIFT = false>
__global__ void __launch_bounds__(W * PlanD<N>::TPL,
                                  StagedTile<T, N, W, PASS == SP_ZINV || PASS == SP_YINV, KK>::MINB)
k_strided_s(PassArgs a, const __grid_constant__ CUtensorMap tm) {
  using C = typename CT<T>::type;
  using PL = PlanD<N>;
  constexpr bool INV = PASS == SP_ZINV || PASS == SP_YINV;
  using TL = StagedTile<T, N, W, INV, KK>;
  using SPL = StagedPlan<PASS, MODE>;
  constexpr int K = KK, M = KK + 1, P = 2 * KK + 1, R1 = PL::R1, R2 = PL::R2, TPL = PL::TPL, J1 = PL::J1;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  C* stg = reinterpret_cast<C*>(smraw + TL::STG_OFF);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + TL::BAR_OFF);
  const int w = threadIdx.x, t = threadIdx.y;
  const bool leader = w == 0 && t == 0;
  const int x0 = blockIdx.x * W, ix = x0 + w, row = blockIdx.y;
  const bool act = ix < M;
  // a TMA destination must be 128-byte aligned: check rather than assume
  if (smem_addr(stg) & 127u) {
    if (leader) atomicOr(&a.ctrl->err, 4);
    return;
  }
  if (leader) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  const C* tw;
  if constexpr (TL::TW_SMEM) {
    // the shared table of strided_twiddles, laid out [j][k1][t]
    C* t1 = reinterpret_cast<C*>(smraw + TL::TW_OFF);
    const C* __restrict__ g = static_cast<const C*>(a.tw);
    const int nthr = blockDim.x * blockDim.y, me = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = me; i < N; i += nthr) {
      const int tt = i % TPL, k1 = (i / TPL) % R1, j = i / (TPL * R1);
      t1[i] = g[(tt + j * TPL) * k1];
    }
    tw = t1;
  } else {
    tw = static_cast<const C*>(a.tw);
  }
  __syncthreads();  // barrier initialised and twiddles in place before use
  const long long S = (long long)P * P * M, zs = (long long)N * P * M, ys = (long long)N * N * M;
  auto issue = [&](int tr) {
    int src, kind, s2, out;
    SPL::get(tr, src, kind, s2, out);
    fence_proxy_async_smem();
    mbar_expect_tx(bar, TL::BYTES);
#pragma unroll
    for (int b = 0; b < TL::NBOX; ++b) {
      C* dst = stg + (size_t)b * TL::BOXR * W;
      if constexpr (PASS == SP_ZINV) tma_load_3d(dst, &tm, 2 * x0, row, src * P + b * TL::BOXR, bar);
      else if constexpr (PASS == SP_YINV) tma_load_2d(dst, &tm, 2 * x0, (src * N + row) * P + b * TL::BOXR, bar);
      else if constexpr (PASS == SP_YFWD) tma_load_2d(dst, &tm, 2 * x0, (src * N + row) * N + b * TL::BOXR, bar);
      else tma_load_3d(dst, &tm, 2 * x0, row, src * N + b * TL::BOXR, bar);
    }
  };
  if (leader) issue(0);
  const C zero = mk(T(0), T(0));
  const C* __restrict__ zb = static_cast<const C*>(a.zb);
  unsigned parity = 0;
#pragma unroll 1
  for (int tr = 0; tr < SPL::NT; ++tr) {
    int src, kind, s2, out;
    SPL::get(tr, src, kind, s2, out);
    if (!SPL::reuses(tr)) {
      // every thread polls the barrier, and the CTA barrier shares the
      // outcome (a transform that reuses the staged tile has nothing to wait for)
      const bool landed = mbar_wait(bar, parity, &a.ctrl->err);
      if (!__syncthreads_and(landed)) {
        // the tile did not arrive in time: report, give it a bounded time to
        // land in this CTA's shared memory, and stop
        if (leader) {
          atomicOr(&a.ctrl->err, 4);
          mbar_wait(bar, parity);
        }
        return;
      }
      parity ^= 1u;
    }
    C in[J1][R1];
#pragma unroll
    for (int j = 0; j < J1; ++j)
      static_for<0, R1>([&](auto nc) {
        constexpr int n1 = decltype(nc)::value;
        const int p = R2 * n1 + t + j * TPL;
        if constexpr (INV && ZeroInputs<N, KK>::zero(n1)) {
          in[j][n1] = zero;  // in the zero band for every column: not read
        } else if constexpr (INV) {
          int k;
          if (!act || !k_of_pos<N, KK>(p, k)) {
            in[j][n1] = zero;
          } else {
            const C v = shift_in<SHIFT, KK>(stg[(k + K) * W + w], a.phase, k);
            if (kind == 0) {
              in[j][n1] = v;
            } else {
              const C d = mul_ik(v, T(k));
              if (kind == 1) {
                in[j][n1] = d;
              } else {
                // second source of omega_x, read directly (y-inverse only)
                const long long o = s2 * zs + ((long long)row * P + (k + K)) * M + ix;
                in[j][n1] = PSC_OK_INDEX(o, (long long)Z_NSTREAM * zs, a.ctrl)
                                ? csub(d, shift_in<SHIFT, KK>(zb[o], a.phase, k))
                                : zero;
              }
            }
          }
        } else {
          in[j][n1] = stg[p * W + w];
        }
      });
    // the staging tile is free (unless the next transform reads it again), and
    // the last transform's exchange reads come before this one's writes
    __syncthreads();
    if (leader && tr + 1 < SPL::NT && !SPL::reuses(tr + 1)) issue(tr + 1);
    if constexpr (PASS == SP_ZINV) {
      C* __restrict__ zo = static_cast<C*>(a.zb);
      strided_fft_regs<T, N, W, +1, TL::TW_SMEM, KK>(
          in,
          [&](int z, C v) {
            if (!act) return;
            const long long idx = out * zs + ((long long)z * P + row) * M + ix;
            if (PSC_OK_INDEX(idx, (long long)Z_NSTREAM * zs, a.ctrl)) zo[idx] = v;
          },
          sm, tw, t, w);
    } else if constexpr (PASS == SP_YINV) {
      C* __restrict__ yo = static_cast<C*>(a.yb);
      strided_fft_regs<T, N, W, +1, TL::TW_SMEM, KK>(
          in,
          [&](int y, C v) {
            if (!act) return;
            const long long idx = out * ys + ((long long)row * N + y) * M + ix;
            if (PSC_OK_INDEX(idx, (long long)Y_NSTREAM * ys, a.ctrl)) yo[idx] = v;
          },
          sm, tw, t, w);
    } else if constexpr (PASS == SP_YFWD) {
      C* __restrict__ yo = static_cast<C*>(a.yf);
      strided_fft_regs<T, N, W, -1, TL::TW_SMEM, KK>(
          in,
          [&](int k, C v) {
            int ky;
            if (!act || !k_of_pos<N, KK>(k, ky)) return;
            const long long idx = out * zs + ((long long)row * P + (ky + K)) * M + ix;
            if (PSC_OK_INDEX(idx, 4 * zs, a.ctrl)) yo[idx] = shift_out<SHIFT, KK>(v, a.phase, ky);
          },
          sm, tw, t, w);
    } else {
      C* __restrict__ ro = static_cast<C*>(a.rb);
      strided_fft_regs<T, N, W, -1, TL::TW_SMEM, KK>(
          in,
          [&](int k, C v) {
            int kz;
            if (!act || !k_of_pos<N, KK>(k, kz)) return;
            const long long idx = out * S + ((long long)(kz + K) * P + row) * M + ix;
            if (PSC_OK_INDEX(idx, 4 * S, a.ctrl)) ro[idx] = shift_out<SHIFT, KK>(v, a.phase, kz);
          },
          sm, tw, t, w);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps of the pass inputs (cuTensorMapEncodeTiled, reached
// through the runtime's driver entry point so no driver library is linked).
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// FP32 view of rows of M complex values: dims {2M, d1[, d2]}, row stride M
// complex, plane stride P M complex (rank 3); boxes of {2W, 1, boxr} (rank 3)
// or {2W, boxr} (rank 2).  False if the map cannot be made.
inline bool make_row_map(CUtensorMap* m, const void* base, int rank, int M, long long d1, long long d2,
                         long long plane, int W, int boxr) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn || ((uintptr_t)base & 15) != 0 || (M * 8) % 16 != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)(2 * M), (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)M * 8, (cuuint64_t)plane * 8};
  cuuint32_t box[3], es[3] = {1, 1, 1};
  box[0] = (cuuint32_t)(2 * W);
  if (rank == 3) {
    box[1] = 1;
    box[2] = (cuuint32_t)boxr;
  } else {
    box[1] = (cuuint32_t)boxr;
  }
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace psc
