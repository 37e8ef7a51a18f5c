// Internal declarations shared by the host API and the per-(precision, N)
// kernel instantiations.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace psc {

// Number of FP64 physical-space moments the statistics pass accumulates.
//  0 sum u.u            1 sum |omega|^2
//  2..4  (du1/dx1)^2,3,4   5..7 (du2/dx2)^2,3,4   8..10 (du3/dx3)^2,3,4
// 11..13 (dphi/dx1)^2,3,4 14..16 (dphi/dx2)^2,3,4 17..19 (dphi/dx3)^2,3,4
// 20 sum phi u2        21 sum phi^2
constexpr int NQ = 24;

// Per-shell quantities of the spectral statistics: E, E_phi, sum k^2 E,
// sum k^2 E_phi, sum w Re(conj(phi) u2)/N^6.
constexpr int NSQ = 5;

struct Dims {
  int N, K, M, P;
  int sph;       // 1: retained set is the sphere 9|k|^2 < 2 N^2 inside the cube |k_i| <= K
  long long S;   // compact elements per field: P*P*M
  long long zs;  // one stream of the z-transformed stage: N*P*M
  long long ys;  // one stream of the y-transformed stage: N*N*M
};

// Largest integer k with k < sqrt(2) N / 3, i.e. 9 k^2 < 2 N^2: the half-width
// of the cube that holds the sphere kept by phase-shift dealiasing (section 2.3).
__host__ __device__ constexpr int sphere_halfwidth(int N) {
  int k = 0;
  while (9 * (k + 1) * (k + 1) < 2 * N * N) ++k;
  return k;
}

// Half-width of the cube that stores the sphere: the sphere's own half-width,
// or one more where that makes a kx row an even number of complex values (a
// 16-byte multiple in FP32, which the tensor maps of the TMA-staged passes
// need) and the cube still fits the grid.  The added planes lie outside the
// sphere and stay zero.
__host__ __device__ constexpr int sphere_storage_halfwidth(int N) {
  return (sphere_halfwidth(N) % 2 == 0 && 2 * (sphere_halfwidth(N) + 1) + 1 <= N) ? sphere_halfwidth(N) + 1
                                                                                    : sphere_halfwidth(N);
}

// Retained half-width K: the 2/3 rule (N-1)/3, or the cube that stores the sphere.
inline Dims make_dims(int N, int sph = 0) {
  Dims d;
  d.N = N;
  d.sph = sph ? 1 : 0;
  d.K = sph ? sphere_storage_halfwidth(N) : (N - 1) / 3;
  d.M = d.K + 1;
  d.P = 2 * d.K + 1;
  d.S = (long long)d.P * d.P * d.M;
  d.zs = (long long)N * d.P * d.M;
  d.ys = (long long)N * N * d.M;
  return d;
}

// Shells n = 0 .. floor(|k|_max + 1/2), n = floor(|k| + 1/2), of the retained
// set: up to the cube's corner |k| = sqrt(3) K under the 2/3 rule; below
// sqrt(2) N / 3 for the sphere (at most its half-width + 1 there, so that + 2
// shells).
inline int shell_count(const Dims& d) {
  if (d.sph) return sphere_halfwidth(d.N) + 2;
  // largest n with n^2 - n < 3 K^2 (the shell of the corner), in integers
  const long long k2 = 3LL * d.K * d.K;
  long long n = 0;
  while ((n + 1) * (n + 1) - (n + 1) < k2) ++n;
  return (int)n + 1;
}

// Device-resident control block: scalars every pass reads or writes.
struct Ctrl {
  double t, dt;
  double A, Ef;                   // forcing amplitude, band energy of the last forced state
  unsigned long long umax_bits;   // max |u1|+|u2|+|u3| as the bits of a non-negative double
  int err;                        // bit 0: index check failed; bit 1: non-finite velocity
  int pad;
  double moments[NQ];
  long long step;                 // RK4 steps taken (advanced by the last stage of each step)
  double Ef0;                     // band energy held by the deterministic forcing (< 0: not yet set)
  double Ef_start;                // band energy of the state at the start of the current step
  unsigned long long wait_ns;     // bound of the TMA waits (0: two seconds)
  int stall_test;                 // 1: the X pass's first staged row of CTA 0 never completes (test)
  int pad2;
};

// Streams of the intermediate buffers (indices into zb / yb).
enum { Z_UX, Z_UY, Z_UZ, Z_DZUY, Z_DZUX, Z_PHI, Z_DZPHI, Z_DZUZ, Z_NSTREAM };
// (with the convective form the Y_WX stream holds d_y u_z, and Y_DZUY is added)
enum { Y_UX, Y_UY, Y_UZ, Y_WX, Y_DZUX, Y_DYUX, Y_PHI, Y_DYPHI, Y_DZPHI, Y_DYUY, Y_DZUZ, Y_DZUY, Y_NSTREAM };
constexpr int Y_NSTREAM_ROT = Y_DZUY;  // streams the rotational form and the statistics use

struct PassArgs {
  Dims d;
  const void* in;   // stage input, compact 4 fields
  void* zb;         // z-inverse output  [Z_NSTREAM][N][P][M]
  void* yb;         // y-inverse output  [Y_NSTREAM][N][N][M]
  void* xb;         // x-pass output     [4][N][N][M]   (aliases zb)
  void* yf;         // y-forward output  [4][N][P][M]   (aliases yb)
  void* rb;         // z-forward output  [4][P][P][M]   compact, unprojected
  const void* tw;   // exp(-2 pi i j/N), j < N
  double* partials; // X-pass statistics partials [xwarps][NQ]
  Ctrl* ctrl;
  int want_umax;    // X pass also reduces max |u1|+|u2|+|u3|
  const void* phase; // exp(i k pi / N), k = -K..K (phase-shift dealiasing)
  int shift;        // 1: evaluate on the grid shifted by half a cell
  int xrow;         // 1: the shared-memory row X pass where the register one exists
  cudaStream_t st;
};

// X-pass modes: the right-hand side (u x omega, u . grad phi); the statistics
// moments; the pressure inputs (u x omega and |u|^2/2 in place of the scalar term)
enum { XMODE_RHS = 0, XMODE_STATS = 1, XMODE_PRESSURE = 2, XMODE_CONVECTIVE = 3 };
// y-inverse stream sets: the right-hand side (9), the statistics (11), the
// convective form (12)
enum { YMODE_RHS = 0, YMODE_STATS = 1, YMODE_CONVECTIVE = 2 };

// Strided passes come in tile-width variants v (index into widths[]).
enum { SP_ZINV = 0, SP_YINV = 1, SP_YFWD = 2, SP_ZFWD = 3, SP_N = 4 };

struct PassTable {
  void (*zinv)(const PassArgs&, bool stats, int v);
  void (*yinv)(const PassArgs&, int ymode, int v);
  void (*xpass)(const PassArgs&, int mode);
  void (*yfwd)(const PassArgs&, int v);
  void (*zfwd)(const PassArgs&, int v);
  int xwarps;       // warps launched by the X pass (rows of `partials`)
  int nvariants;    // variants of the strided passes (at most 5)
  int widths[5];    // their column tile widths
  int staged[5];    // 1: input tiles staged through shared memory by TMA
  unsigned vmask[SP_N];  // variants built for each pass (bit v)
  int row_only;  // 1: the X pass exists only as the row X pass (no convective form)
};

const PassTable* table_f32(int N);
const PassTable* table_f64(int N);

}  // namespace psc

// ---------------------------------------------------------------------------
// Persistent ensemble kernel (psc_batch.cu): the plain-data description of one
// box of its device work table and the host entry points of that file.  The
// kernel's bodies are compiled in their own namespace there, so only plain
// types cross between the two files.
// ---------------------------------------------------------------------------
struct PscBatchBox {
  int N, K, M, P;                 // grid and retained half-width (2/3 rule)
  long long S, zs, ys;            // element counts of the compact, z and y stages
  void *U, *V, *Acc, *zreg, *yreg;
  void *eu, *ep;                  // integrating-factor tables
  const void* tw;                 // twiddles exp(-2 pi i j / N)
  void* ctrl;                     // the simulation's control block
  double kF2, eps_inj, beta, nu, D, cfl, dx;
  int kF2_floor, forcing, integrator, scalar_on, record_every, cfl_on;
};

// Grid sizes the persistent kernel runs (FP32-mixed, 2/3 rule, rotational form).
bool pscb_size_supported(int N);
// Dynamic shared memory the kernel needs for boxes of up to max_N points.
size_t pscb_smem_bytes(int max_N);
// Device bytes of a work table for up to max_boxes boxes.
size_t pscb_table_bytes(int max_boxes);
// Build the work table of these boxes on the host and copy it to `table`
// (device) on `st`; `staging` is a host buffer of pscb_table_bytes() bytes
// that must stay valid until the copy has completed.  stall_test: the first
// dependency wait of stage 1 can never be met and is bounded at 50 ms instead
// of two seconds (a test of the failure path).
cudaError_t pscb_upload(void* table, void* staging, int max_boxes, const PscBatchBox* boxes, int n,
                        cudaStream_t st, bool stall_test);
// One ensemble RK4 step: clear the counters, then one persistent launch per stage.
cudaError_t pscb_step(void* table, int max_boxes, int max_N, int grid, size_t smem, cudaStream_t st);
// CTAs of the persistent kernel for boxes up to max_N that fit on the device
// at once with `smem` bytes of dynamic shared memory each.
int pscb_grid(int max_N, size_t smem);

