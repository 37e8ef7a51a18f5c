/*
 * psc.h -- C ABI of the GB300 pseudo-spectral solver for forced homogeneous
 * isotropic turbulence with a passive scalar (arXiv:2012.04838, section 2).
 *
 * The library advances, on one GPU, the Fourier-Galerkin system of the paper:
 *   d u_k/dt   = P_k (u x omega)_k - nu |k|^2 u_k + A u_k 1[0<|k|^2<=kF^2]   (Eqs. 6-7)
 *   d phi_k/dt = -(u . grad phi)_k - beta u2_k - D |k|^2 phi_k, D = nu/Sc    (Eq. 8)
 * on the periodic box [0, 2 pi]^3 with N^3 points (Eq. 4) and the DFT
 * convention of Eq. 5 (forward unnormalised, inverse scaled by 1/N^3).
 *
 * Conventions shared by every entry point
 *   - Status: every call returns psc_status; nothing is thrown across the ABI.
 *     psc_last_error() gives a message for the last failing call.
 *   - Memory: the caller owns all device memory.  psc_workspace_size() says how
 *     many bytes of device memory one simulation needs; the caller allocates
 *     them (for example with PyTorch) and passes the pointer to psc_create().
 *     The library itself allocates no device memory.
 *   - Streams: all device work of a simulation is enqueued on the CUDA stream
 *     given to psc_create() (NULL = legacy default stream).  Calls that return
 *     data to host memory synchronise that stream; the others are asynchronous.
 *   - Threads: one simulation must not be used from two host threads at once;
 *     distinct simulations are independent.
 *   - Spectral layout ("compact state"): with K = floor((N-1)/3) (2/3 rule;
 *     with PSC_DEALIAS_PHASE_SHIFT the largest k with 9 k^2 < 2 N^2, or one
 *     more where that makes K + 1 even and 2K + 1 <= N: the planes it adds lie
 *     outside the sphere and are zero),
 *     P = 2K+1 and M = K+1, the state is four fields (u1, u2, u3, phi), each
 *     a [P][P][M] array of complex numbers (interleaved real, imaginary) with
 *     element [kz+K][ky+K][kx] holding the unnormalised Fourier coefficient
 *     of wavevector (kx, ky, kz), |kx|,|ky|,|kz| <= K, kx >= 0.  The kx = 0
 *     plane is conjugate-symmetric (real fields); the k = 0 entry is zero.
 *     Complex numbers are float pairs (PSC_FP32_MIXED) or double pairs (PSC_FP64).
 */
#ifndef PSC_H
#define PSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSC_OK = 0,
  PSC_EINVAL = 1,          /* invalid argument or parameter                      */
  PSC_ENOMEM_BUDGET = 2,   /* workspace smaller than psc_workspace_size()         */
  PSC_ECUDA = 3,           /* a CUDA runtime call failed (see psc_last_error)     */
  PSC_EUNSTABLE = 4,       /* non-finite velocity seen by the CFL monitor (Eq. 10)*/
  PSC_ETIMEOUT = 5,        /* a bounded device wait gave up (reported at the next
                              statistics call)                                     */
  PSC_EUNSUPPORTED_N = 6   /* N outside the supported set of grid sizes           */
} psc_status;

typedef enum { PSC_FP64 = 0, PSC_FP32_MIXED = 1 } psc_precision;
typedef enum { PSC_IC_SPECTRUM_K4 = 0, PSC_IC_TAYLOR_GREEN_NOISE = 1, PSC_IC_PAPER_EQ9 = 2 } psc_ic;
/* Forcing of the band 0 < |k| <= kF (section 2.3).  CONST_POWER adds A u with
 * A = eps_inj / (2 E_f) at every RK stage.  HOLD_ENERGY is the paper's
 * deterministic scheme, applied after the last stage: the band is rescaled so
 * that it keeps the energy it had at the first step after psc_init_field or
 * psc_set_state (eps_inj unused); records report the equivalent rate
 * A = ln(factor) / dt. */
typedef enum { PSC_FORCE_NONE = 0, PSC_FORCE_CONST_POWER = 1, PSC_FORCE_HOLD_ENERGY = 2 } psc_forcing;

/* Form of the nonlinear term (section 2.3).  ROTATIONAL: P(u x omega), 9
 * physical fields per right-hand side.  CONVECTIVE: -P((u.grad)u) as the paper
 * writes it, with u and the 9 velocity gradients formed in physical space (12
 * fields; a larger workspace).  The two agree to round-off on the retained set.
 * CONVECTIVE is not built for N = 520 (PSC_EUNSUPPORTED_N). */
typedef enum { PSC_NL_ROTATIONAL = 0, PSC_NL_CONVECTIVE = 1 } psc_nonlinear;
typedef enum { PSC_INTEG_IFRK4 = 0, PSC_INTEG_RK4 = 1 } psc_integrator;
/* Dealiasing of the products (section 2.3).  TWO_THIRDS: the retained set is the
 * cube |k_i| <= K = (N-1)/3, whose quadratic products are alias-free on one grid.
 * PHASE_SHIFT: the paper's sphere |k| < sqrt(2) N / 3, stored in the cube of
 * half-width K of the layout above (modes of that cube outside the sphere are
 * zero); every product is formed on the grid and on the grid shifted
 * by half a cell in each direction, and the two transforms are averaged, which
 * cancels the aliases that the sphere alone leaves (Patterson and Orszag 1971).
 * Twice the transforms of the right-hand side; psc_pressure is not offered with
 * it (PSC_EINVAL). */
typedef enum { PSC_DEALIAS_TWO_THIRDS = 0, PSC_DEALIAS_PHASE_SHIFT = 1 } psc_dealias;

/* Problem statement (Table 2 of the paper; Sc and beta from section 2.3).
 * Fields are plain values; zero-initialise and set what you need. */
typedef struct {
  int32_t N;            /* grid points per side; box side 2 pi (section 3.1)          */
  int32_t precision;    /* psc_precision                                              */
  double nu;            /* kinematic viscosity (Eq. 1)                                */
  double Sc;            /* Schmidt number, D = nu/Sc (section 2.3)                    */
  double beta;          /* uniform mean scalar gradient along x2 (Eq. 3)              */
  int32_t forcing;      /* psc_forcing                                                */
  int32_t integrator;   /* psc_integrator: Lawson IF-RK4 or plain RK4 (section 2.2)   */
  double kF;            /* forcing sphere 0 < |k| <= kF (section 2.3)                 */
  double eps_inj;       /* injected power for PSC_FORCE_CONST_POWER                   */
  double dt;            /* time step; used as is when cfl <= 0                        */
  double cfl;           /* > 0: dt reset to reach this CFL (Eq. 10) at step 0 and at
                           every record_every-th step, held in between                */
  uint64_t seed;        /* initial-condition seed                                     */
  int32_t ic;           /* psc_ic                                                     */
  int32_t record_every; /* steps between CFL resets (>= 1)                            */
  double ic_energy;     /* target K of the random IC (u_rms = 1 gives 1.5)            */
  double ic_noise_frac; /* Taylor-Green IC: noise energy as a fraction of 1/8         */
  int32_t scalar_on;    /* 0: phi is held at zero                                     */
  int32_t nonlinear_form; /* psc_nonlinear                                            */
  int32_t dealias;        /* psc_dealias                                              */
  int32_t reserved;       /* must be zero                                             */
} psc_params;

/* One statistics record of the current state (section 2.3): Table 1,
 * Eqs. 11-12 (velocity- and scalar-gradient skewness and flatness) and the
 * terms of Eq. 13.  eps and chi come from the spectrum; eps_phys = nu <|omega|^2>
 * and chi_phys = 2 D <|grad phi|^2> are grid averages (equal up to rounding).
 * Precision: every sum is finished in FP64 in a fixed order.  With
 * PSC_FP32_MIXED each thread first accumulates its share in compensated FP32
 * (the shell sums behind E(n), K, eps, chi, phi_var, phi_prod, E_forced; the
 * grid moments behind K_phys, eps_phys, chi_phys, phi_prod_phys, skew, flat,
 * skew_phi, flat_phi), which keeps these fields within 2e-5 relative of the
 * FP64 values (skewness and flatness within 1e-4 absolute; tested). */
typedef struct {
  double t, dt;
  double K, K_phys, eps, eps_phys, eta, Re_lambda, Te, urms, lambda, l0;
  double cfl, umax, kmax_eta, kmax_eta_sqrt2;
  double skew[3], flat[3];
  double phi_var, phi_prod, phi_prod_phys, chi, chi_phys;
  double skew_phi[3], flat_phi[3];
  double A, E_forced, P_inj;
  int64_t step;
} psc_stats;

typedef struct psc_sim psc_sim;

/* Bytes of device workspace needed for these parameters.  Fails with
 * PSC_EUNSUPPORTED_N for an unsupported N and PSC_EINVAL for bad parameters. */
psc_status psc_workspace_size(const psc_params* p, size_t* bytes);

/* Grid sizes this build supports (ascending); returns how many, writes at most cap. */
int32_t psc_supported_sizes(int32_t* out, int32_t cap);

/* Create a simulation on the current CUDA device.  dev_ws: caller-owned device
 * memory of ws_bytes >= psc_workspace_size() bytes, 256-byte aligned, kept alive
 * until psc_destroy().  stream: a cudaStream_t (NULL = default stream).
 * The state is zero until psc_init_field() or psc_set_state(). */
psc_status psc_create(const psc_params* p, void* dev_ws, size_t ws_bytes, void* stream,
                      psc_sim** out);

/* Initial condition (section 2.3): the random solenoidal field with the chosen
 * shell spectrum, or the Taylor-Green vortex plus that noise; phi = 0.
 * Deterministic in (seed, N, ic).  Resets t and the step counter.  Synchronises. */
psc_status psc_init_field(psc_sim* s);

/* Advance nsteps RK4 steps (section 2.2), asynchronously on the stream. */
psc_status psc_step(psc_sim* s, int32_t nsteps);

/* Statistics of the current state.  Ek and Ephi (host, may be NULL) receive up
 * to nshell_cap shell values E(n), E_phi(n), n = floor(|k|+1/2); *nshell (may
 * be NULL) receives the number of shells.  out (host, may be NULL) receives the
 * record.  Synchronises; returns PSC_EUNSTABLE if a non-finite velocity was seen. */
psc_status psc_spectra_and_stats(psc_sim* s, double* Ek, double* Ephi, int32_t nshell_cap,
                                 int32_t* nshell, psc_stats* out);

/* Bytes of the compact state (4 fields). */
psc_status psc_state_bytes(const psc_sim* s, size_t* bytes);

/* Copy the compact state to / from host or device memory (any pointer CUDA can
 * address).  set_state also accepts an initial state from the caller.  Both
 * synchronise the stream.  Pinned (or registered) host buffers with 16-byte
 * alignment are copied by the SMs through the host mapping, other buffers by
 * cudaMemcpyAsync; the bits are the same either way.  `bytes` must equal
 * psc_state_bytes() (else PSC_EINVAL). */
psc_status psc_get_state(psc_sim* s, void* dst, size_t bytes);
psc_status psc_set_state(psc_sim* s, const void* src, size_t bytes);

/* One evaluation of the right-hand side without the linear terms,
 * N(u, phi) = (P(u x omega)_k + A u_k 1_F, -(u.grad phi)_k - beta u2_k),
 * for a compact state at device pointer `in`, written in compact layout to the
 * device pointer `out` (both psc_state_bytes() long, not overlapping the
 * workspace).  With the plain RK4 integrator the linear terms are included.
 * Asynchronous on the stream. */
psc_status psc_rhs(psc_sim* s, const void* in, void* out);

/* The modified pressure of the current state (section 2.2, Eq. 6):
 * p_k = i k.(u.grad u)_k / |k|^2 on the retained set, p_0 = 0, written to the
 * device pointer `out` as one compact field ((2K+1)^2 (K+1) complex values in
 * the state's precision, layout [kz+K][ky+K][kx]; `bytes` must be that size;
 * `out` must not overlap the workspace).  Computed as -i k.(u x omega)_k/|k|^2
 * - (|u|^2/2)_k.  Asynchronous on the stream. */
psc_status psc_pressure(psc_sim* s, void* out, size_t bytes);

/* Time, step counter and current dt (host values; synchronises). */
psc_status psc_time(psc_sim* s, double* t, int64_t* step, double* dt);

/* Ensembles (boxes of any mix of N and precision stepped together).
 *
 * psc_batch_create() captures one RK4 step of every member into a single CUDA
 * graph, each member on its own stream as a parallel branch forked from and
 * joined back into `stream`; psc_batch_step() replays that graph, so an
 * ensemble step costs one graph launch and small boxes run concurrently.
 * Each member advances exactly as psc_step() would advance it (the step counter
 * and the CFL decision live on the device).  Members need non-NULL streams;
 * members that share a stream become consecutive steps of one branch (correct,
 * but not concurrent).  `stream` must be non-NULL.  Members stay usable on their own,
 * but their own calls and batch steps must not overlap in time: synchronise
 * `stream` before touching a member directly, and the members' streams before
 * the next batch step.  Profiling is suspended while the graph is captured. */
typedef struct psc_batch psc_batch;
psc_status psc_batch_create(psc_sim* const* sims, int32_t n, void* stream, psc_batch** out);
psc_status psc_batch_step(psc_batch* b, int32_t nsteps); /* asynchronous on `stream` */
psc_status psc_batch_destroy(psc_batch* b);

/* Persistent ensembles: one launch per RK stage over a device work table.
 *
 * The paper runs an ensemble as separate serial runs (Table 2); this batched
 * form is an addition for many small boxes.  psc_batch_create_persistent()
 * captures, into one CUDA graph, a reset of the table's counters and four
 * launches of a persistent kernel, one per RK4 stage; each launch steps every
 * member through that stage (forcing amplitude, the five transform passes,
 * the CFL reset of Eq. 10 at stage 1, the stage combine, and after stage 4 the
 * deterministic forcing), its CTAs taking (box, pass, tile) items from the
 * work table in pass order.  An item waits until every tile of its box's
 * previous pass has completed; such a wait is bounded (about two seconds),
 * after which the step is abandoned and the member reports PSC_ETIMEOUT at its
 * next statistics call.  Each member advances bit for bit as psc_step() would
 * advance it alone.
 *
 * Members: FP32-mixed, 2/3 rule, rotational form, N in {32, 48, 64, 96, 128,
 * 192, 256} and N <= max_N (max_N sets the kernel's shared memory, so keep it
 * as small as the ensemble allows); otherwise PSC_EINVAL / PSC_EUNSUPPORTED_N.
 * dev_table: caller-owned device memory of psc_batch_table_bytes(max_boxes)
 * bytes, 256-byte aligned, kept until psc_batch_destroy().  stream: non-NULL;
 * every batch step and table update runs on it (members' own streams are not
 * used by the batch).
 *
 * psc_batch_set_members() replaces the member list (up to max_boxes, 0 allowed)
 * by rewriting the table on `stream`, ordered after the steps already
 * enqueued; the captured graph stays valid, so boxes join and leave between
 * steps without a new capture.  Members must not be used on their own while a
 * batch step may be running (synchronise `stream` first), and a member must be
 * taken out of the table (psc_batch_set_members without it) before it is
 * destroyed: the table holds its device addresses.  psc_batch_step() and
 * psc_batch_destroy() serve both kinds of batch. */
#define PSC_BATCH_MAX_BOXES 4096
typedef enum { PSC_BATCH_GRAPH = 0, PSC_BATCH_PERSISTENT = 1 } psc_batch_mode;
psc_status psc_batch_table_bytes(int32_t max_boxes, size_t* bytes);
psc_status psc_batch_create_persistent(psc_sim* const* sims, int32_t n, int32_t max_boxes, int32_t max_N,
                                       void* dev_table, size_t table_bytes, void* stream, psc_batch** out);
psc_status psc_batch_set_members(psc_batch* b, psc_sim* const* sims, int32_t n);
/* The batch's kind (psc_batch_mode), its persistent grid (CTAs; 0 for a graph
 * batch) and the kernel launches its steps have made (persistent batches). */
psc_status psc_batch_info(const psc_batch* b, int32_t* mode, int32_t* grid, int64_t* launches);

/* Kernel classes for profiling. */
typedef enum {
  PSC_K_FORCING = 0,  /* band energy and forcing amplitude                   */
  PSC_K_ZINV = 1,     /* inverse transform along z (+ d/dz streams)          */
  PSC_K_YINV = 2,     /* inverse transform along y (+ omega_x, d/dy streams) */
  PSC_K_XPASS = 3,    /* fused x transforms and nonlinear products           */
  PSC_K_YFWD = 4,     /* forward transform along y, truncation               */
  PSC_K_ZFWD = 5,     /* forward transform along z, truncation               */
  PSC_K_COMBINE = 6,  /* projection, forcing, scalar source, RK stage update */
  PSC_K_OTHER = 7,    /* CFL, IF tables, statistics passes and reductions, IC */
  PSC_K_NKIND = 8
} psc_kernel_kind;

/* Profiling: while enabled, every kernel launch of this simulation is
 * bracketed by CUDA events on its stream.  psc_profile_read() synchronises,
 * writes the summed device milliseconds and launch counts per kernel kind
 * (arrays of nkind <= PSC_K_NKIND entries, either may be NULL) and clears them. */
psc_status psc_profile_enable(psc_sim* s, int32_t on);
psc_status psc_profile_read(psc_sim* s, double* ms, int64_t* launches, int32_t nkind);

/* Column tile widths chosen for the four strided passes (z-inverse, y-inverse,
 * y-forward, z-forward; w receives 4 values).  psc_create() times the compiled
 * widths of each FP32 pass on the simulation's workspace and keeps the fastest
 * (cached per grid size for the process; PSC_TUNE=0 in the environment keeps
 * fixed defaults instead). */
psc_status psc_tile_widths(const psc_sim* s, int32_t* w);

/* Whether each of the four strided passes (same order as psc_tile_widths)
 * runs its TMA-staged kernel: 1 if the pass brings its input tiles into shared
 * memory with bulk tensor copies ahead of each transform, 0 if its threads
 * load from global memory directly.  Chosen by the same autotuning. */
psc_status psc_tile_staged(const psc_sim* s, int32_t* staged);

/* Total kernels this simulation has launched since creation (always counted). */
psc_status psc_launch_count(const psc_sim* s, int64_t* n);

psc_status psc_destroy(psc_sim* s);

/* Shell spectra without device allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory or provide a workspace (code replayed inside a
 * pre-sized CUDA graph pipeline, plugins whose host application owns the
 * device allocator, tools that only hold a pointer to a state).  It computes
 * the same E(n) and E_phi(n), n = floor(|k| + 1/2), as psc_spectra_and_stats()
 * of a simulation with the same N, precision and dealias.
 *
 * state: device pointer to a compact state of grid size N in `precision`
 * and in the layout `dealias` selects (layout above).  Ek, Ephi: device
 * pointers to at least nshell_cap doubles; the first nshell entries are
 * written, nshell = the count psc_spectra_and_stats() reports (2/3 rule:
 * floor(sqrt(3) K + 1/2) + 1, 592 at N = 1024; phase shifts: K + 2).
 * stream: a cudaStream_t (NULL = default stream); the call is asynchronous on
 * it.  PSC_EINVAL, before anything is launched, for: a null pointer; N
 * outside 8..65536, a bad precision or dealias; nshell_cap < nshell; a state,
 * Ek or Ephi that is not device (or managed) memory of the current device.
 *
 * The per-shell partial sums go to one fixed device array of
 * PSC_NOALLOC_MAX_SHELLS x 5 doubles inside the library, which every GPU that
 * loads the library holds until the process exits.  Grids needing more shells
 * than that (2/3 rule: N >= 1774; phase shifts: N >= 2171) are rejected with
 * PSC_EINVAL.  The call allocates no memory.  The first call on each device
 * looks up that array's device address (once per device, with the device
 * current); make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's sums, so calls that
 * overlap on the GPU (different streams, or different host threads) race with
 * each other: serialise them. */
#define PSC_NOALLOC_MAX_SHELLS 1024
psc_status psc_shell_spectra_noalloc(const void* state, int32_t N, int32_t precision, int32_t dealias,
                                     double* Ek, double* Ephi, int32_t nshell_cap, void* stream);

/* Profiling aid (no counterpart in the paper): the right-hand-side X pass
 * that psc_step() runs for grid size N and precision (2/3 rule), launched
 * nlaunch times over `rows` rows of a deterministic synthetic input instead of
 * the N*N rows of a box, so that hardware-counter captures of it fit in a few
 * GB of device memory.  rows: a positive multiple of 64, at most N*N.  buf:
 * caller-owned device memory of psc_xpass_probe_bytes() bytes, 256-byte
 * aligned, holding a control block, twiddles, the nine input streams
 * [stream][row][kx] and the four output streams; the call fills all but the
 * outputs.  Asynchronous on `stream`.  N = 520 (row X pass only) is refused
 * with PSC_EUNSUPPORTED_N. */
psc_status psc_xpass_probe_bytes(int32_t N, int32_t precision, int64_t rows, size_t* bytes);
psc_status psc_xpass_probe(int32_t N, int32_t precision, int64_t rows, void* buf, size_t bytes, void* stream,
                           int32_t nlaunch);

/* Measurement aid (no counterpart in the paper): `blocks` CTAs of 256 threads
 * whose threads each run 128 * iters fused multiply-adds (8 independent chains
 * of 16 * iters) in FP32 (PSC_FP32_MIXED) or FP64, storing one value per
 * thread to the device buffer `out` (blocks * 256 elements).  That is
 * 2 * 128 * iters * 256 * blocks floating-point operations; timed by the
 * caller, it gives the device's FMA peak that the FP32 and FP64 paths are
 * compared against.  Asynchronous on `stream`. */
psc_status psc_fma_probe(int32_t precision, int32_t iters, int32_t blocks, void* out, void* stream);

/* Message for the last failing call on this thread (never NULL). */
const char* psc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PSC_H */
