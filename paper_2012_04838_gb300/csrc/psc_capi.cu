// Host side of the C ABI (include/psc.h): parameter checks, workspace
// layout, stage orchestration and assembly of the statistics record.
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "psc.h"
#include "psc_kernels.cuh"

// ---------------------------------------------------------------- dispatch

// Grid sizes with compiled pass kernels (one object file per size and precision).
#define PSC_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(512) X(520) X(1024)
#define PSC_DECL(n)                                     \
  const psc::PassTable* psc_pass_table_float_##n();     \
  const psc::PassTable* psc_pass_table_double_##n();    \
  const psc::PassTable* psc_pass_table_ps_float_##n();  \
  const psc::PassTable* psc_pass_table_ps_double_##n();
PSC_SIZES(PSC_DECL)
#undef PSC_DECL

namespace psc {

const PassTable* table_f32(int N) {
  switch (N) {
#define PSC_CASE(n) case n: return psc_pass_table_float_##n();
    PSC_SIZES(PSC_CASE)
#undef PSC_CASE
    default: return nullptr;
  }
}
const PassTable* table_f64(int N) {
  switch (N) {
#define PSC_CASE(n) case n: return psc_pass_table_double_##n();
    PSC_SIZES(PSC_CASE)
#undef PSC_CASE
    default: return nullptr;
  }
}
// phase-shift dealiasing (null where not built)
const PassTable* table_ps(int N, bool fp64) {
  switch (N) {
#define PSC_CASE(n) case n: return fp64 ? psc_pass_table_ps_double_##n() : psc_pass_table_ps_float_##n();
    PSC_SIZES(PSC_CASE)
#undef PSC_CASE
    default: return nullptr;
  }
}

static const int kSizes[] = {
#define PSC_LIST(n) n,
    PSC_SIZES(PSC_LIST)
#undef PSC_LIST
};

static bool size_supported(int N) {
  for (int n : kSizes)
    if (n == N) return true;
  return false;
}

// ---------------------------------------------------------------- errors

static thread_local std::string g_err;

static psc_status fail(psc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

void set_error(const std::string& msg) { g_err = msg; }
static psc_status cuda_fail(cudaError_t e, const char* where) {
  return fail(PSC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define PSC_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)
#define PSC_LAUNCHED(where)                             \
  do {                                                  \
    cudaError_t e_ = cudaGetLastError();                \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// ---------------------------------------------------------------- layout

static int num_shells(const Dims& d) { return shell_count(d); }

struct Layout {
  size_t ctrl, U, V, Acc, zreg, yreg, tw, eu, ep, partials, shells, fac, R0, phase, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout make_layout(const Dims& d, int fp64, int xwarps, int convective) {
  const size_t cs = fp64 ? 16 : 8, rs = fp64 ? 8 : 4;
  const size_t S = (size_t)d.S, zs = (size_t)d.zs, ys = (size_t)d.ys;
  size_t zreg = Z_NSTREAM * zs;
  if (4 * ys > zreg) zreg = 4 * ys;
  if (4 * S > zreg) zreg = 4 * S;
  size_t yreg = (size_t)(convective ? Y_NSTREAM : Y_NSTREAM_ROT) * ys * cs;
  if (4 * zs * cs > yreg) yreg = 4 * zs * cs;
  if (3 * S * 16 > yreg) yreg = 3 * S * 16;  // FP64 scratch of the initial condition
  const int nsh = num_shells(d);
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  L.ctrl = take(sizeof(Ctrl));
  L.U = take(4 * S * cs);
  L.V = take(4 * S * cs);
  L.Acc = take(4 * S * cs);
  L.zreg = take(zreg * cs);
  L.yreg = take(yreg);
  L.tw = take(d.N * cs);
  L.eu = take((d.K + 1) * rs);
  L.ep = take((d.K + 1) * rs);
  L.partials = take((size_t)xwarps * NQ * 8);
  L.shells = take((size_t)NSQ * nsh * 8);
  L.fac = take((size_t)nsh * 8);
  // phase-shift dealiasing: the products of the unshifted grid, and the phases
  L.R0 = take(d.sph ? 4 * S * cs : 0);
  L.phase = take(d.sph ? (size_t)d.P * cs : 0);
  L.total = o;
  return L;
}

// exp(-2 pi i j / N) to FP64 accuracy: reduce to a quarter turn exactly, then
// rotate by whole quarter turns.
static void twiddle(long j, long N, double* c, double* s) {
  j %= N;
  const long q = (4 * j) / N;
  const long rem = 4 * j - q * N;  // angle = q pi/2 + (pi/2) rem/N
  const double th = (M_PI / 2.0) * ((double)rem / (double)N);
  double c0 = std::cos(th), s0 = std::sin(th);
  for (long r = 0; r < q; ++r) {  // multiply by i
    const double t = c0;
    c0 = -s0;
    s0 = t;
  }
  *c = c0;
  *s = -s0;  // forward sign
}

}  // namespace psc

using namespace psc;

struct psc_sim {
  psc_params p;
  Dims d;
  int fp64;
  const PassTable* tb;
  cudaStream_t st;
  unsigned char* ws;
  Layout L;
  Ctrl* ctrl;
  int64_t step;
  int nshell;
  int wv[SP_N];  // tile-width variant of each strided pass (autotuned at creation)
  int xrow = 0;  // PSC_XPASS_ROWS=1 at creation: the row X pass where the register one exists
  int stall_test = 0;  // PSC_XPASS_STALL_TEST=1 at creation: failure-path test of the TMA waits
  // launch accounting and optional per-launch event timing
  int64_t launches = 0;
  bool profiling = false;
  struct Timed { int kind; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> pool;
};

namespace {

cudaEvent_t take_event(psc_sim* s) {
  if (!s->pool.empty()) {
    cudaEvent_t e = s->pool.back();
    s->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// NVTX range names of the kernel kinds (psc_kernel_kind)
const char* const kKindName[PSC_K_NKIND] = {"psc forcing", "psc z-inverse", "psc y-inverse", "psc x pass",
                                            "psc y-forward", "psc z-forward", "psc combine", "psc other"};

// An NVTX range on the calling thread for the life of the object (nothing
// happens unless an NVTX tool is attached to the process)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Run `launch` (which enqueues kernels on s->st) as `n` launches of `kind`,
// inside an NVTX range named for the kind.
template <class F> void launch(psc_sim* s, int kind, int n, F&& f) {
  NvtxRange r(kKindName[kind]);
  s->launches += n;
  if (!s->profiling) {
    f();
    return;
  }
  psc_sim::Timed t{kind, take_event(s), take_event(s)};
  cudaEventRecord(t.a, s->st);
  f();
  cudaEventRecord(t.b, s->st);
  s->timed.push_back(t);
}

}  // namespace

static const PassTable* pick_table(const psc_params* p);

static psc_status check_params(const psc_params* p) {
  if (!p) return fail(PSC_EINVAL, "null params");
  if (!size_supported(p->N)) return fail(PSC_EUNSUPPORTED_N, "unsupported grid size N=" + std::to_string(p->N));
  if (p->precision != PSC_FP64 && p->precision != PSC_FP32_MIXED) return fail(PSC_EINVAL, "bad precision");
  if (!(p->nu >= 0.0) || !(p->Sc > 0.0)) return fail(PSC_EINVAL, "nu must be >= 0 and Sc > 0");
  if (p->cfl <= 0.0 && !(p->dt > 0.0)) return fail(PSC_EINVAL, "dt must be > 0 when cfl <= 0");
  if (p->record_every < 1) return fail(PSC_EINVAL, "record_every must be >= 1");
  if (p->forcing != PSC_FORCE_NONE && p->forcing != PSC_FORCE_CONST_POWER && p->forcing != PSC_FORCE_HOLD_ENERGY)
    return fail(PSC_EINVAL, "bad forcing");
  if (p->nonlinear_form != PSC_NL_ROTATIONAL && p->nonlinear_form != PSC_NL_CONVECTIVE)
    return fail(PSC_EINVAL, "bad nonlinear_form");
  if (p->integrator != PSC_INTEG_IFRK4 && p->integrator != PSC_INTEG_RK4) return fail(PSC_EINVAL, "bad integrator");
  if (p->dealias != PSC_DEALIAS_TWO_THIRDS && p->dealias != PSC_DEALIAS_PHASE_SHIFT)
    return fail(PSC_EINVAL, "bad dealias");
  if (p->reserved != 0) return fail(PSC_EINVAL, "reserved must be zero");
  if (p->nonlinear_form == PSC_NL_CONVECTIVE && pick_table(p)->row_only)
    return fail(PSC_EUNSUPPORTED_N, std::string("the convective form is not built for N=") + std::to_string(p->N) +
                                        (p->dealias == PSC_DEALIAS_PHASE_SHIFT ? " with phase-shift dealiasing" : ""));
  if (p->ic < 0 || p->ic > 2) return fail(PSC_EINVAL, "bad ic");
  if (!(p->kF >= 0.0) || !(p->eps_inj >= 0.0)) return fail(PSC_EINVAL, "kF and eps_inj must be >= 0");
  if (!(p->ic_energy >= 0.0) || !(p->ic_noise_frac >= 0.0)) return fail(PSC_EINVAL, "IC energies must be >= 0");
  return PSC_OK;
}

static const PassTable* pick_table(const psc_params* p) {
  if (p->dealias == PSC_DEALIAS_PHASE_SHIFT) return table_ps(p->N, p->precision == PSC_FP64);
  return p->precision == PSC_FP64 ? table_f64(p->N) : table_f32(p->N);
}

static Dims dims_of(const psc_params* p) { return make_dims(p->N, p->dealias == PSC_DEALIAS_PHASE_SHIFT); }

namespace {
template <typename T> void launch_iftab(psc_sim* s);
psc_status autotune(psc_sim* s);
}

extern "C" {

const char* psc_last_error(void) { return g_err.c_str(); }

int32_t psc_supported_sizes(int32_t* out, int32_t cap) {
  const int n = (int)(sizeof(kSizes) / sizeof(kSizes[0]));
  for (int i = 0; i < n && i < cap; ++i) out[i] = kSizes[i];
  return n;
}

psc_status psc_workspace_size(const psc_params* p, size_t* bytes) {
  psc_status s = check_params(p);
  if (s != PSC_OK) return s;
  if (!bytes) return fail(PSC_EINVAL, "null bytes");
  const PassTable* tb = pick_table(p);
  *bytes = make_layout(dims_of(p), p->precision == PSC_FP64, tb->xwarps,
                       p->nonlinear_form == PSC_NL_CONVECTIVE).total;
  return PSC_OK;
}

psc_status psc_create(const psc_params* p, void* dev_ws, size_t ws_bytes, void* stream, psc_sim** out) {
  psc_status s = check_params(p);
  if (s != PSC_OK) return s;
  if (!out || !dev_ws) return fail(PSC_EINVAL, "null workspace or output handle");
  if (((uintptr_t)dev_ws & 255) != 0) return fail(PSC_EINVAL, "workspace must be 256-byte aligned");
  const PassTable* tb = pick_table(p);
  Layout L = make_layout(dims_of(p), p->precision == PSC_FP64, tb->xwarps,
                         p->nonlinear_form == PSC_NL_CONVECTIVE);
  if (ws_bytes < L.total)
    return fail(PSC_ENOMEM_BUDGET, "workspace of " + std::to_string(ws_bytes) + " bytes < required " +
                                       std::to_string(L.total));
  psc_sim* sim = new (std::nothrow) psc_sim();
  if (!sim) return fail(PSC_EINVAL, "host allocation failed");
  sim->p = *p;
  sim->d = dims_of(p);
  sim->fp64 = p->precision == PSC_FP64;
  sim->tb = tb;
  sim->st = (cudaStream_t)stream;
  sim->ws = (unsigned char*)dev_ws;
  sim->L = L;
  sim->ctrl = (Ctrl*)(sim->ws + L.ctrl);
  sim->step = 0;
  sim->nshell = num_shells(sim->d);
  {
    // test knob: the shared-memory row X pass at sizes that also have the register one
    const char* xr = std::getenv("PSC_XPASS_ROWS");
    sim->xrow = (xr && xr[0] == '1') ? 1 : 0;
    // test knob: the X pass's first staged row never completes and its waits are
    // bounded at 1 ms, so the failure path (PSC_ETIMEOUT) runs without a fault
    const char* st = std::getenv("PSC_XPASS_STALL_TEST");
    sim->stall_test = (st && st[0] == '1') ? 1 : 0;
  }
  // twiddles, control block, zero state
  const int N = p->N;
  std::vector<double> twd(2 * (size_t)N);
  for (int j = 0; j < N; ++j) twiddle(j, N, &twd[2 * j], &twd[2 * j + 1]);
  std::vector<float> twf(2 * (size_t)N);
  for (size_t i = 0; i < twd.size(); ++i) twf[i] = (float)twd[i];
  Ctrl c0;
  std::memset(&c0, 0, sizeof(c0));
  c0.dt = p->dt;
  c0.Ef0 = -1.0;
  c0.stall_test = sim->stall_test;
  c0.wait_ns = sim->stall_test ? 1000000ull : 0ull;
  cudaError_t e;
  if (sim->fp64) e = cudaMemcpyAsync(sim->ws + L.tw, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice, sim->st);
  else e = cudaMemcpyAsync(sim->ws + L.tw, twf.data(), twf.size() * 4, cudaMemcpyHostToDevice, sim->st);
  // phase factors exp(i k pi / N) = conj(exp(-2 pi i k / 2N)), k = -K..K
  std::vector<double> phd(2 * (size_t)sim->d.P);
  std::vector<float> phf(phd.size());
  for (int k = -sim->d.K; k <= sim->d.K; ++k) {
    double c, sn;
    twiddle(k < 0 ? 2L * N + k : (long)k, 2L * N, &c, &sn);
    phd[2 * (k + sim->d.K)] = c;
    phd[2 * (k + sim->d.K) + 1] = -sn;
  }
  for (size_t i = 0; i < phd.size(); ++i) phf[i] = (float)phd[i];
  if (e == cudaSuccess && sim->d.sph) {
    if (sim->fp64) e = cudaMemcpyAsync(sim->ws + L.phase, phd.data(), phd.size() * 8, cudaMemcpyHostToDevice, sim->st);
    else e = cudaMemcpyAsync(sim->ws + L.phase, phf.data(), phf.size() * 4, cudaMemcpyHostToDevice, sim->st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(sim->ctrl, &c0, sizeof(c0), cudaMemcpyHostToDevice, sim->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sim->ws + L.U, 0, L.V - L.U, sim->st);
  if (e == cudaSuccess) {
    // integrating factors for the initial dt, so a state set by psc_set_state can be stepped
    if (sim->fp64) launch_iftab<double>(sim);
    else launch_iftab<float>(sim);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(sim->st);
  if (e != cudaSuccess) {
    delete sim;
    return cuda_fail(e, "psc_create");
  }
  psc_status ts = autotune(sim);
  if (ts != PSC_OK) {
    delete sim;
    return ts;
  }
  *out = sim;
  return PSC_OK;
}

psc_status psc_destroy(psc_sim* s) {
  if (!s) return PSC_OK;
  for (auto& t : s->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : s->pool) cudaEventDestroy(e);
  delete s;
  return PSC_OK;
}

psc_status psc_profile_enable(psc_sim* s, int32_t on) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  s->profiling = on != 0;
  return PSC_OK;
}

psc_status psc_profile_read(psc_sim* s, double* ms, int64_t* launches, int32_t nkind) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  if (nkind < 0 || nkind > PSC_K_NKIND) return fail(PSC_EINVAL, "bad nkind");
  PSC_CUDA(cudaStreamSynchronize(s->st));
  std::vector<double> t(PSC_K_NKIND, 0.0);
  std::vector<int64_t> n(PSC_K_NKIND, 0);
  for (auto& e : s->timed) {
    float x = 0.f;
    PSC_CUDA(cudaEventElapsedTime(&x, e.a, e.b));
    t[e.kind] += x;
    n[e.kind] += 1;
    s->pool.push_back(e.a);
    s->pool.push_back(e.b);
  }
  s->timed.clear();
  for (int k = 0; k < nkind; ++k) {
    if (ms) ms[k] = t[k];
    if (launches) launches[k] = n[k];
  }
  return PSC_OK;
}

psc_status psc_tile_widths(const psc_sim* s, int32_t* w) {
  if (!s || !w) return fail(PSC_EINVAL, "null argument");
  for (int p = 0; p < SP_N; ++p) w[p] = s->tb->widths[s->wv[p]];
  return PSC_OK;
}

psc_status psc_tile_staged(const psc_sim* s, int32_t* staged) {
  if (!s || !staged) return fail(PSC_EINVAL, "null argument");
  for (int p = 0; p < SP_N; ++p) staged[p] = s->tb->staged[s->wv[p]];
  return PSC_OK;
}

psc_status psc_launch_count(const psc_sim* s, int64_t* n) {
  if (!s || !n) return fail(PSC_EINVAL, "null argument");
  *n = s->launches;
  return PSC_OK;
}

psc_status psc_state_bytes(const psc_sim* s, size_t* bytes) {
  if (!s || !bytes) return fail(PSC_EINVAL, "null argument");
  *bytes = 4 * (size_t)s->d.S * (s->fp64 ? 16 : 8);
  return PSC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- internals

namespace {

// Plain 16-byte copy by the SMs.
__global__ void k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// The device address of host memory the GPU can access directly (pinned or
// registered), else null.
void* device_view(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // unregistered pointer on an older runtime: clear the error
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// State copy between the workspace and a caller buffer on the simulation's
// stream.  With pinned host memory on the other side the SMs copy through the
// host mapping: on GB300 with a Grace host, the copy engines were measured to
// move a 1024^3 state to pinned memory at a tenth of the host link's rate right
// after the solver had run, while SM stores and loads kept the link's rate.
// Anything else goes through cudaMemcpyAsync.
cudaError_t copy_state(psc_sim* s, void* dst, const void* src, size_t nb) {
  const bool to_host = src == s->ws + s->L.U;
  void* hv = device_view(to_host ? dst : src);
  void* d = to_host ? hv : dst;
  const void* sp = to_host ? src : (const void*)hv;
  if (hv && ((uintptr_t)d & 15) == 0 && ((uintptr_t)sp & 15) == 0 && nb % 16 == 0) {
    s->launches += 1;
    k_copy16<<<152 * 16, 256, 0, s->st>>>((const uint4*)sp, (uint4*)d, nb / 16);
    return cudaGetLastError();
  }
  return cudaMemcpyAsync(dst, src, nb, cudaMemcpyDefault, s->st);
}

PassArgs pass_args(psc_sim* s, const void* in) {
  PassArgs a;
  a.d = s->d;
  a.in = in;
  a.zb = s->ws + s->L.zreg;
  a.yb = s->ws + s->L.yreg;
  a.xb = s->ws + s->L.zreg;  // the z-inverse streams are dead once the y-inverse pass has run
  a.yf = s->ws + s->L.yreg;  // the y-inverse streams are dead once the X pass has run
  a.rb = s->ws + s->L.zreg;  // the X-pass output is dead once the y-forward pass has run
  a.tw = s->ws + s->L.tw;
  a.partials = (double*)(s->ws + s->L.partials);
  a.ctrl = s->ctrl;
  a.want_umax = 0;
  a.phase = s->ws + s->L.phase;
  a.shift = 0;
  a.xrow = s->xrow;
  a.st = s->st;
  return a;
}

template <typename T>
void launch_famp(psc_sim* s, const void* in, bool step_start = false) {
  launch(s, PSC_K_FORCING, 1, [&] {
    k_famp<T><<<1, 32, 0, s->st>>>(s->d, in, s->ctrl, s->p.kF * s->p.kF, s->p.eps_inj, s->p.forcing,
                                   step_start ? 1 : 0);
  });
}

template <typename T>
void launch_iftab(psc_sim* s) {
  const int n = s->d.K + 1;
  launch(s, PSC_K_OTHER, 1, [&] {
    k_iftab<T><<<(n + 127) / 128, 128, 0, s->st>>>(s->d.K, s->ctrl, s->p.nu, s->p.nu / s->p.Sc,
                                                     (T*)(s->ws + s->L.eu), (T*)(s->ws + s->L.ep));
  });
}

CombineArgs combine_args(psc_sim* s, const void* vin) {
  CombineArgs c;
  c.d = s->d;
  c.rb = s->ws + s->L.zreg;
  c.rb2 = s->d.sph ? (const void*)(s->ws + s->L.R0) : nullptr;
  c.vin = vin;
  c.U = s->ws + s->L.U;
  c.V = s->ws + s->L.V;
  c.Acc = s->ws + s->L.Acc;
  c.out = nullptr;
  c.eu = s->ws + s->L.eu;
  c.ep = s->ws + s->L.ep;
  c.ctrl = s->ctrl;
  c.kF2 = s->p.kF * s->p.kF;
  c.kF2_floor = c.kF2 >= 2.0e9 ? 2000000000 : (int)std::floor(c.kF2);
  c.beta = s->p.beta;
  c.nu = s->p.nu;
  c.D = s->p.nu / s->p.Sc;
  c.forcing = s->p.forcing;
  c.integrator = s->p.integrator;
  c.scalar_on = s->p.scalar_on;
  return c;
}

template <typename T>
void launch_combine(psc_sim* s, int stage, const CombineArgs& c) {
  const long long S = s->d.S;
  const int blocks = (int)((S + 255) / 256);
  launch(s, PSC_K_COMBINE, 1, [&] {
    switch (stage) {
      case 0: k_combine<T, 0><<<blocks, 256, 0, s->st>>>(c); break;
      case 1: k_combine<T, 1><<<blocks, 256, 0, s->st>>>(c); break;
      case 2: k_combine<T, 2><<<blocks, 256, 0, s->st>>>(c); break;
      case 3: k_combine<T, 3><<<blocks, 256, 0, s->st>>>(c); break;
      default: k_combine<T, 4><<<blocks, 256, 0, s->st>>>(c); break;
    }
  });
}

// The five FFT passes of one RHS evaluation of `in`, leaving the unprojected
// compact (NL, u.grad phi) in the z region.  With phase-shift dealiasing the
// products are formed twice, on the grid (into the R0 region) and on the grid
// shifted by half a cell (into the z region); the combine averages them.
template <typename T>
void rhs_passes(psc_sim* s, const void* in, bool umax, bool step_start = false) {
  if (umax) cudaMemsetAsync(&s->ctrl->umax_bits, 0, sizeof(unsigned long long), s->st);
  launch_famp<T>(s, in, step_start);
  // the convective form takes the 8 z-stage streams of the statistics pass and
  // d_y u_z, d_z u_y separately at the y stage
  const bool conv = s->p.nonlinear_form == PSC_NL_CONVECTIVE;
  const int nshift = s->d.sph ? 2 : 1;
  for (int sh = 0; sh < nshift; ++sh) {
    PassArgs a = pass_args(s, in);
    a.shift = sh;
    a.want_umax = umax && sh == 0 ? 1 : 0;
    if (nshift == 2 && sh == 0) a.rb = s->ws + s->L.R0;
    launch(s, PSC_K_ZINV, 1, [&] { s->tb->zinv(a, conv, s->wv[SP_ZINV]); });
    launch(s, PSC_K_YINV, 1, [&] { s->tb->yinv(a, conv ? YMODE_CONVECTIVE : YMODE_RHS, s->wv[SP_YINV]); });
    launch(s, PSC_K_XPASS, 1, [&] { s->tb->xpass(a, conv ? XMODE_CONVECTIVE : XMODE_RHS); });
    if (a.want_umax && s->p.cfl > 0.0) {
      launch(s, PSC_K_OTHER, 1, [&] {
        k_cfl<<<1, 32, 0, s->st>>>(s->ctrl, s->p.cfl, 2.0 * M_PI / s->p.N, s->p.record_every);
      });
      launch_iftab<T>(s);
    }
    launch(s, PSC_K_YFWD, 1, [&] { s->tb->yfwd(a, s->wv[SP_YFWD]); });
    launch(s, PSC_K_ZFWD, 1, [&] { s->tb->zfwd(a, s->wv[SP_ZFWD]); });
  }
}

template <typename T>
psc_status do_step(psc_sim* s, int nsteps) {
  unsigned char* U = s->ws + s->L.U;
  unsigned char* V = s->ws + s->L.V;
  for (int n = 0; n < nsteps; ++n) {
    // with a CFL target every step measures max |u| at stage 1 and the device
    // decides whether this is a reset step, so all steps enqueue the same work
    const bool reset_dt = s->p.cfl > 0.0;
    for (int stage = 1; stage <= 4; ++stage) {
      const void* vin = stage == 1 ? (const void*)U : (const void*)V;
      rhs_passes<T>(s, vin, stage == 1 && reset_dt, stage == 1);
      launch_combine<T>(s, stage, combine_args(s, vin));
    }
    if (s->p.forcing == PSC_FORCE_HOLD_ENERGY) {
      launch(s, PSC_K_FORCING, 1, [&] {
        k_hold<T><<<1, 32, 0, s->st>>>(s->d, U, s->ctrl, s->p.kF * s->p.kF);
      });
    }
    PSC_LAUNCHED("psc_step");
    ++s->step;
  }
  return PSC_OK;
}

template <typename T>
psc_status do_rhs(psc_sim* s, const void* in, void* out) {
  rhs_passes<T>(s, in, false);
  CombineArgs c = combine_args(s, in);
  c.out = out;
  launch_combine<T>(s, 0, c);
  PSC_LAUNCHED("psc_rhs");
  return PSC_OK;
}

template <typename T>
psc_status do_pressure(psc_sim* s, void* out) {
  const void* U = s->ws + s->L.U;
  PassArgs a = pass_args(s, U);
  launch(s, PSC_K_ZINV, 1, [&] { s->tb->zinv(a, false, s->wv[SP_ZINV]); });
  launch(s, PSC_K_YINV, 1, [&] { s->tb->yinv(a, YMODE_RHS, s->wv[SP_YINV]); });
  launch(s, PSC_K_XPASS, 1, [&] { s->tb->xpass(a, XMODE_PRESSURE); });
  launch(s, PSC_K_YFWD, 1, [&] { s->tb->yfwd(a, s->wv[SP_YFWD]); });
  launch(s, PSC_K_ZFWD, 1, [&] { s->tb->zfwd(a, s->wv[SP_ZFWD]); });
  const int blocks = (int)((s->d.S + 255) / 256);
  launch(s, PSC_K_OTHER, 1, [&] { k_pressure<T><<<blocks, 256, 0, s->st>>>(s->d, a.rb, out); });
  PSC_LAUNCHED("psc_pressure");
  return PSC_OK;
}

template <typename T>
psc_status do_init(psc_sim* s) {
  const Dims& d = s->d;
  double2* z = (double2*)(s->ws + s->L.yreg);
  double* shells = (double*)(s->ws + s->L.shells);
  double* fac = (double*)(s->ws + s->L.fac);
  const int blocks = (int)((d.S + 255) / 256);
  const bool tg = s->p.ic == PSC_IC_TAYLOR_GREEN_NOISE;
  const double K0 = tg ? s->p.ic_noise_frac * 0.125 : s->p.ic_energy;
  const int shape = s->p.ic == PSC_IC_PAPER_EQ9 ? 2 : 0;
  const double n3 = (double)d.N * d.N * d.N;
  launch(s, PSC_K_OTHER, 4, [&] {
    k_ic_draw<<<blocks, 256, 0, s->st>>>(d, (unsigned long long)s->p.seed, z);
    k_shells<double><<<s->nshell, 256, 0, s->st>>>(d, z, nullptr, s->nshell, shells);
    k_ic_factors<<<1, 32, 0, s->st>>>(s->nshell, shells, 1.0 / (2.0 * n3 * n3), K0, shape, s->p.kF, fac);
    k_ic_finish<T><<<blocks, 256, 0, s->st>>>(d, z, fac, tg ? 1 : 0, s->ws + s->L.U);
  });
  Ctrl c0;
  std::memset(&c0, 0, sizeof(c0));
  c0.dt = s->p.dt;
  c0.Ef0 = -1.0;
  c0.stall_test = s->stall_test;
  c0.wait_ns = s->stall_test ? 1000000ull : 0ull;
  PSC_CUDA(cudaMemcpyAsync(s->ctrl, &c0, sizeof(c0), cudaMemcpyHostToDevice, s->st));
  launch_iftab<T>(s);
  PSC_LAUNCHED("psc_init_field");
  PSC_CUDA(cudaStreamSynchronize(s->st));
  s->step = 0;
  return PSC_OK;
}

template <typename T>
psc_status do_stats(psc_sim* s, double* Ek, double* Ephi, int cap, int* nshell, psc_stats* out) {
  const Dims& d = s->d;
  const void* U = s->ws + s->L.U;
  PassArgs a = pass_args(s, U);
  PSC_CUDA(cudaMemsetAsync(&s->ctrl->umax_bits, 0, sizeof(unsigned long long), s->st));
  launch_famp<T>(s, U);
  launch(s, PSC_K_OTHER, 3, [&] {
    s->tb->zinv(a, true, s->wv[SP_ZINV]);
    s->tb->yinv(a, YMODE_STATS, s->wv[SP_YINV]);
    s->tb->xpass(a, XMODE_STATS);
  });
  double* shells = (double*)(s->ws + s->L.shells);
  launch(s, PSC_K_OTHER, 2, [&] {
    k_reduce_moments<<<1, 32, 0, s->st>>>(a.partials, s->tb->xwarps, s->ctrl);
    k_shells<T><<<s->nshell, 256, 0, s->st>>>(d, U, (const unsigned char*)U + 3 * d.S * (s->fp64 ? 16 : 8),
                                               s->nshell, shells);
  });
  PSC_LAUNCHED("psc_spectra_and_stats");
  Ctrl c;
  std::vector<double> sh((size_t)NSQ * s->nshell);
  PSC_CUDA(cudaMemcpyAsync(&c, s->ctrl, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  PSC_CUDA(cudaMemcpyAsync(sh.data(), shells, sh.size() * 8, cudaMemcpyDeviceToHost, s->st));
  PSC_CUDA(cudaStreamSynchronize(s->st));
  if (c.err & 1) return fail(PSC_ECUDA, "device index check failed");
  const int ns = s->nshell;
  const double n3 = (double)d.N * d.N * d.N, n6 = n3 * n3;
  const double nu = s->p.nu, D = s->p.nu / s->p.Sc, beta = s->p.beta;
  double Ks = 0, dK = 0, Vp = 0, dV = 0, pr = 0;
  for (int n = 0; n < ns; ++n) {
    const double E = sh[0 * ns + n] / (2 * n6), Ep = sh[1 * ns + n] / (2 * n6);
    if (Ek && n < cap) Ek[n] = E;
    if (Ephi && n < cap) Ephi[n] = Ep;
    Ks += E;
    Vp += Ep;
    dK += sh[2 * ns + n] / (2 * n6);
    dV += sh[3 * ns + n] / (2 * n6);
    pr += sh[4 * ns + n] / n6;
  }
  if (nshell) *nshell = ns;
  double umax;
  std::memcpy(&umax, &c.umax_bits, sizeof(umax));
  if (out) {
    psc_stats& r = *out;
    std::memset(&r, 0, sizeof(r));
    const double* m = c.moments;
    r.t = c.t;
    r.dt = c.dt;
    // at a CFL reset step the record carries the dt that step will use (Eq. 10)
    if (s->p.cfl > 0.0 && (s->step % s->p.record_every) == 0 && umax > 0.0 &&
        umax <= 1.7976931348623157e308)
      r.dt = s->p.cfl * (2.0 * M_PI / d.N) / umax;
    r.step = s->step;
    r.K = Ks;
    r.K_phys = 0.5 * m[0] / n3;
    r.eps = 2.0 * nu * dK;
    r.eps_phys = nu * m[1] / n3;
    r.urms = std::sqrt(2.0 * Ks / 3.0);
    const double eps = r.eps;
    r.eta = eps > 0 ? std::pow(nu * nu * nu / eps, 0.25) : INFINITY;
    r.lambda = eps > 0 ? r.urms * std::sqrt(15.0 * nu / eps) : INFINITY;
    r.Re_lambda = eps > 0 && nu > 0 ? r.lambda * r.urms / nu : INFINITY;
    r.l0 = eps > 0 ? r.urms * r.urms * r.urms / eps : INFINITY;
    r.Te = r.urms > 0 ? r.l0 / r.urms : INFINITY;
    r.umax = umax;
    r.cfl = r.dt / (2.0 * M_PI / d.N) * umax;
    r.kmax_eta = (d.N / 3.0) * r.eta;
    r.kmax_eta_sqrt2 = (std::sqrt(2.0) * d.N / 3.0) * r.eta;
    for (int i = 0; i < 3; ++i) {
      const double m2 = m[2 + 3 * i] / n3, m3 = m[3 + 3 * i] / n3, m4 = m[4 + 3 * i] / n3;
      r.skew[i] = m2 > 0 ? m3 / std::pow(m2, 1.5) : 0.0;
      r.flat[i] = m2 > 0 ? m4 / (m2 * m2) : 0.0;
      const double p2 = m[11 + 3 * i] / n3, p3 = m[12 + 3 * i] / n3, p4 = m[13 + 3 * i] / n3;
      r.skew_phi[i] = p2 > 0 ? p3 / std::pow(p2, 1.5) : 0.0;
      r.flat_phi[i] = p2 > 0 ? p4 / (p2 * p2) : 0.0;
    }
    r.phi_var = m[21] / n3;
    r.phi_prod = -2.0 * beta * pr;
    r.phi_prod_phys = -2.0 * beta * m[20] / n3;
    r.chi = 2.0 * D * 2.0 * dV;
    r.chi_phys = 2.0 * D * (m[11] + m[14] + m[17]) / n3;
    r.A = c.A;
    r.E_forced = c.Ef;
    r.P_inj = 2.0 * c.A * c.Ef;
  }
  (void)Vp;
  // a wait that gave up left the state incomplete: report it before what followed from it
  if (c.err & 4)
    return fail(PSC_ETIMEOUT, "a bounded device wait gave up (an asynchronous copy into shared memory, or a "
                              "dependency of the persistent ensemble kernel, did not complete in time)");
  if ((c.err & 2) || !(umax <= 1.7976931348623157e308))
    return fail(PSC_EUNSTABLE, "non-finite velocity in the CFL monitor");
  return PSC_OK;
}

// Autotuner of the strided passes.  Every compiled variant of each pass (tile
// widths, and for FP32 grids with an even M the TMA-staged kernels) is timed
// on this simulation's own workspace (one warm-up and three timed launches
// each, CUDA events on its stream) and the fastest is kept.
// Choices are cached per (grid size, precision) for the life of the process,
// so ensembles and servers tune once per N.  PSC_TUNE=0 in the environment
// skips the timing and uses 128-byte runs (16 columns) for the z passes and for
// N < 512, 64-byte runs for the y passes at N >= 512.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::array<int, SP_N>> g_tune_cache;

psc_status autotune(psc_sim* s) {
  const int N = s->d.N;
  for (int p = 0; p < SP_N; ++p) s->wv[p] = 0;
  if (s->tb->nvariants < 2) return PSC_OK;
  const bool ypass_narrow = N >= 512;
  s->wv[SP_ZINV] = 1;
  s->wv[SP_ZFWD] = 1;
  s->wv[SP_YINV] = ypass_narrow ? 0 : 1;
  s->wv[SP_YFWD] = ypass_narrow ? 0 : 1;
  // PSC_STRIDED_VARIANT=v runs variant v of every strided pass; four digits
  // give the z-inverse, y-inverse, y-forward and z-forward variants (tests)
  const char* force = std::getenv("PSC_STRIDED_VARIANT");
  if (force && force[0] >= '0' && force[0] <= '9') {
    const size_t len = std::strlen(force);
    for (int p = 0; p < SP_N; ++p) {
      const char c = len == (size_t)SP_N ? force[p] : force[0];
      const int v = c - '0';
      if (len != 1 && len != (size_t)SP_N) return fail(PSC_EINVAL, "PSC_STRIDED_VARIANT: one or four digits");
      if (v < 0 || v >= s->tb->nvariants || !((s->tb->vmask[p] >> v) & 1u))
        return fail(PSC_EINVAL, "PSC_STRIDED_VARIANT: variant not built for this grid and pass");
      s->wv[p] = v;
    }
    return PSC_OK;
  }
  const char* env = std::getenv("PSC_TUNE");
  if (env && env[0] == '0') return PSC_OK;
  const std::pair<int, int> key(N, s->fp64 + 2 * s->d.sph);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int p = 0; p < SP_N; ++p) s->wv[p] = it->second[p];
      return PSC_OK;
    }
  }
  PassArgs a = pass_args(s, s->ws + s->L.U);
  cudaEvent_t e0, e1;
  PSC_CUDA(cudaEventCreate(&e0));
  PSC_CUDA(cudaEventCreate(&e1));
  auto run = [&](int p, int v) {
    switch (p) {
      case SP_ZINV: s->tb->zinv(a, false, v); break;
      case SP_YINV: s->tb->yinv(a, YMODE_RHS, v); break;
      case SP_YFWD: s->tb->yfwd(a, v); break;
      default: s->tb->zfwd(a, v); break;
    }
  };
  std::array<int, SP_N> best;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < SP_N && e == cudaSuccess; ++p) {
    float tbest = 0.f;
    best[p] = s->wv[p];
    for (int v = 0; v < s->tb->nvariants && e == cudaSuccess; ++v) {
      if (!((s->tb->vmask[p] >> v) & 1u)) continue;
      run(p, v);
      cudaEventRecord(e0, s->st);
      for (int r = 0; r < 3; ++r) run(p, v);
      cudaEventRecord(e1, s->st);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (v == 0 || ms < tbest)) {
        tbest = ms;
        best[p] = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "psc_create: tile autotuning");
  for (int p = 0; p < SP_N; ++p) s->wv[p] = best[p];
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return PSC_OK;
}

}  // namespace

extern "C" {

psc_status psc_init_field(psc_sim* s) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  return s->fp64 ? do_init<double>(s) : do_init<float>(s);
}

psc_status psc_step(psc_sim* s, int32_t nsteps) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  if (nsteps < 0) return fail(PSC_EINVAL, "nsteps must be >= 0");
  NvtxRange r("psc_step");
  return s->fp64 ? do_step<double>(s, nsteps) : do_step<float>(s, nsteps);
}

psc_status psc_rhs(psc_sim* s, const void* in, void* out) {
  if (!s || !in || !out) return fail(PSC_EINVAL, "null argument");
  return s->fp64 ? do_rhs<double>(s, in, out) : do_rhs<float>(s, in, out);
}

psc_status psc_pressure(psc_sim* s, void* out, size_t bytes) {
  if (!s || !out) return fail(PSC_EINVAL, "null argument");
  if (bytes != (size_t)s->d.S * (s->fp64 ? 16 : 8)) return fail(PSC_EINVAL, "pressure buffer size mismatch");
  if (s->d.sph) return fail(PSC_EINVAL, "the pressure is formed with the 2/3 rule only");
  return s->fp64 ? do_pressure<double>(s, out) : do_pressure<float>(s, out);
}

psc_status psc_spectra_and_stats(psc_sim* s, double* Ek, double* Ephi, int32_t cap, int32_t* nshell,
                                 psc_stats* out) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  if (cap < 0) return fail(PSC_EINVAL, "negative capacity");
  NvtxRange r("psc_spectra_and_stats");
  return s->fp64 ? do_stats<double>(s, Ek, Ephi, cap, nshell, out)
                 : do_stats<float>(s, Ek, Ephi, cap, nshell, out);
}

psc_status psc_get_state(psc_sim* s, void* dst, size_t bytes) {
  size_t nb;
  if (!s || !dst) return fail(PSC_EINVAL, "null argument");
  psc_state_bytes(s, &nb);
  if (bytes != nb) return fail(PSC_EINVAL, "state size mismatch");
  PSC_CUDA(copy_state(s, dst, s->ws + s->L.U, nb));
  PSC_CUDA(cudaStreamSynchronize(s->st));
  return PSC_OK;
}

psc_status psc_set_state(psc_sim* s, const void* src, size_t bytes) {
  size_t nb;
  if (!s || !src) return fail(PSC_EINVAL, "null argument");
  psc_state_bytes(s, &nb);
  if (bytes != nb) return fail(PSC_EINVAL, "state size mismatch");
  PSC_CUDA(copy_state(s, s->ws + s->L.U, src, nb));
  // the deterministic forcing holds the band energy of the state it starts from
  const double unset[2] = {0.0, -1.0};  // A, Ef0
  PSC_CUDA(cudaMemcpyAsync(&s->ctrl->A, &unset[0], sizeof(double), cudaMemcpyHostToDevice, s->st));
  PSC_CUDA(cudaMemcpyAsync(&s->ctrl->Ef0, &unset[1], sizeof(double), cudaMemcpyHostToDevice, s->st));
  PSC_CUDA(cudaStreamSynchronize(s->st));
  return PSC_OK;
}

psc_status psc_time(psc_sim* s, double* t, int64_t* step, double* dt) {
  if (!s) return fail(PSC_EINVAL, "null sim");
  Ctrl c;
  PSC_CUDA(cudaMemcpyAsync(&c, s->ctrl, sizeof(c), cudaMemcpyDeviceToHost, s->st));
  PSC_CUDA(cudaStreamSynchronize(s->st));
  if (t) *t = c.t;
  if (dt) *dt = c.dt;
  if (step) *step = s->step;
  return PSC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- ALU probe

namespace {

// Eight independent fused multiply-add chains per thread (enough to hide the
// pipe latency); the result is stored so nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T* out) {
  T a[8];
  const T b = (T)0.999999, c = (T)1e-7;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (T)(threadIdx.x + j);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" psc_status psc_fma_probe(int32_t precision, int32_t iters, int32_t blocks, void* out, void* stream) {
  if ((precision != PSC_FP64 && precision != PSC_FP32_MIXED) || iters < 1 || blocks < 1 || !out)
    return fail(PSC_EINVAL, "psc_fma_probe: bad arguments");
  const cudaStream_t st = (cudaStream_t)stream;
  if (precision == PSC_FP64) k_fma_probe<double><<<blocks, 256, 0, st>>>(iters, (double*)out);
  else k_fma_probe<float><<<blocks, 256, 0, st>>>(iters, (float*)out);
  PSC_LAUNCHED("psc_fma_probe");
  return PSC_OK;
}

// ---------------------------------------------------------------- X-pass probe

namespace {

// Deterministic input pattern of the probe: values in [-1, 1) scaled to the
// magnitude of unnormalised coefficients, from a 64-bit mix of the index.
template <typename T>
__global__ void k_probe_fill(T* p, long long n, T amp) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 29;
    p[i] = amp * (T)((double)(z >> 11) * 0x1.0p-52 - 1.0);
  }
}

struct ProbeLayout {
  size_t ctrl, tw, yb, xb, total;
};

ProbeLayout probe_layout(const Dims& d, int fp64, long long rows) {
  const size_t cs = fp64 ? 16 : 8;
  ProbeLayout L;
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o = align256(o + b); return r; };
  L.ctrl = take(sizeof(Ctrl));
  L.tw = take((size_t)d.N * cs);
  L.yb = take((size_t)Y_NSTREAM_ROT * rows * d.M * cs);
  L.xb = take((size_t)4 * rows * d.M * cs);
  L.total = o;
  return L;
}

psc_status probe_check(int32_t N, int32_t precision, int64_t rows) {
  if (!size_supported(N) || N == 520) return fail(PSC_EUNSUPPORTED_N, "probe: unsupported N");
  if (precision != PSC_FP64 && precision != PSC_FP32_MIXED) return fail(PSC_EINVAL, "probe: bad precision");
  if (rows <= 0 || rows % 64 != 0 || rows > (int64_t)N * N)
    return fail(PSC_EINVAL, "probe: rows must be a positive multiple of 64, at most N*N");
  return PSC_OK;
}

}  // namespace

extern "C" {

psc_status psc_xpass_probe_bytes(int32_t N, int32_t precision, int64_t rows, size_t* bytes) {
  psc_status st = probe_check(N, precision, rows);
  if (st != PSC_OK) return st;
  if (!bytes) return fail(PSC_EINVAL, "null bytes");
  *bytes = probe_layout(make_dims(N), precision == PSC_FP64, rows).total;
  return PSC_OK;
}

psc_status psc_xpass_probe(int32_t N, int32_t precision, int64_t rows, void* buf, size_t bytes, void* stream,
                           int32_t nlaunch) {
  psc_status st = probe_check(N, precision, rows);
  if (st != PSC_OK) return st;
  const int fp64 = precision == PSC_FP64;
  Dims d = make_dims(N);
  const ProbeLayout L = probe_layout(d, fp64, rows);
  if (!buf || ((uintptr_t)buf & 255) != 0 || bytes < L.total || nlaunch < 0)
    return fail(PSC_EINVAL, "probe: buffer must be 256-byte aligned and psc_xpass_probe_bytes() long; nlaunch >= 0");
  const cudaStream_t cs = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)buf;
  std::vector<double> twd(2 * (size_t)N);
  for (int j = 0; j < N; ++j) twiddle(j, N, &twd[2 * j], &twd[2 * j + 1]);
  std::vector<float> twf(twd.begin(), twd.end());
  Ctrl c0;
  std::memset(&c0, 0, sizeof(c0));
  PSC_CUDA(cudaMemcpyAsync(b + L.ctrl, &c0, sizeof(c0), cudaMemcpyHostToDevice, cs));
  if (fp64) PSC_CUDA(cudaMemcpyAsync(b + L.tw, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice, cs));
  else PSC_CUDA(cudaMemcpyAsync(b + L.tw, twf.data(), twf.size() * 4, cudaMemcpyHostToDevice, cs));
  const long long nre = 2LL * Y_NSTREAM_ROT * rows * d.M;
  const double amp = 0.05 * (double)N * N * N;
  if (fp64) k_probe_fill<double><<<152 * 8, 256, 0, cs>>>((double*)(b + L.yb), nre, amp);
  else k_probe_fill<float><<<152 * 8, 256, 0, cs>>>((float*)(b + L.yb), nre, (float)amp);
  PSC_LAUNCHED("psc_xpass_probe: fill");
  d.ys = (long long)rows * d.M;  // the X pass reads rows and stream strides from here
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.d = d;
  a.yb = b + L.yb;
  a.xb = b + L.xb;
  a.tw = b + L.tw;
  a.ctrl = (Ctrl*)(b + L.ctrl);
  a.st = cs;
  const PassTable* tb = fp64 ? table_f64(N) : table_f32(N);
  for (int i = 0; i < nlaunch; ++i) tb->xpass(a, XMODE_RHS);
  PSC_LAUNCHED("psc_xpass_probe");
  return PSC_OK;
}

}  // extern "C"

struct psc_batch {
  std::vector<psc_sim*> sims;
  std::vector<int64_t> launches_per_step;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;
  // persistent mode: the device work table and the launch shape baked into the graph
  int mode = PSC_BATCH_GRAPH;
  int max_boxes = 0, max_N = 0, grid = 0;
  size_t smem = 0;
  void* table = nullptr;
  std::vector<unsigned char> staging;
  int64_t launches = 0;  // kernels and memsets the batch's own graph ran
  bool stall_test = false;  // PSC_BATCH_STALL_TEST=1 at creation (failure-path test)
};

static void batch_free(psc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->events) cudaEventDestroy(e);
  delete b;
}

extern "C" {

psc_status psc_batch_create(psc_sim* const* sims, int32_t n, void* stream, psc_batch** out) {
  if (!sims || n < 1 || !out) return fail(PSC_EINVAL, "psc_batch_create: need n >= 1 members and an output handle");
  if (!stream) return fail(PSC_EINVAL, "psc_batch_create: the batch stream must be non-NULL");
  for (int i = 0; i < n; ++i) {
    if (!sims[i] || !sims[i]->st) return fail(PSC_EINVAL, "psc_batch_create: members need non-NULL streams");
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return fail(PSC_EINVAL, "psc_batch_create: members must be distinct");
  }
  psc_batch* b = new (std::nothrow) psc_batch();
  if (!b) return fail(PSC_EINVAL, "host allocation failed");
  b->st = (cudaStream_t)stream;
  b->sims.assign(sims, sims + n);
  // fork/join events (one fork, one join per member)
  b->events.resize(n + 1, nullptr);
  for (auto& e : b->events) {
    cudaError_t ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) { batch_free(b); return cuda_fail(ce, "psc_batch_create"); }
  }
  std::vector<bool> prof(n);
  std::vector<int64_t> step0(n), launch0(n);
  for (int i = 0; i < n; ++i) {
    prof[i] = sims[i]->profiling;
    sims[i]->profiling = false;
    step0[i] = sims[i]->step;
    launch0[i] = sims[i]->launches;
  }
  cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed);
  psc_status st = PSC_OK;
  if (e == cudaSuccess) e = cudaEventRecord(b->events[0], b->st);
  for (int i = 0; i < n && e == cudaSuccess && st == PSC_OK; ++i) {
    psc_sim* m = sims[i];
    if (m->st != b->st) e = cudaStreamWaitEvent(m->st, b->events[0], 0);
    if (e != cudaSuccess) break;
    st = m->fp64 ? do_step<double>(m, 1) : do_step<float>(m, 1);
    if (st == PSC_OK && m->st != b->st) {
      e = cudaEventRecord(b->events[i + 1], m->st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->events[i + 1], 0);
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  for (int i = 0; i < n; ++i) {
    sims[i]->profiling = prof[i];
    b->launches_per_step.push_back(sims[i]->launches - launch0[i]);
    sims[i]->step = step0[i];
    sims[i]->launches = launch0[i];
  }
  if (st != PSC_OK) { if (g) cudaGraphDestroy(g); batch_free(b); return st; }
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) { b->graph = g; e = cudaGraphInstantiate(&b->exec, g, 0); }
  else if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) { batch_free(b); return cuda_fail(e, "psc_batch_create: graph capture"); }
  *out = b;
  return PSC_OK;
}

psc_status psc_batch_step(psc_batch* b, int32_t nsteps) {
  if (!b) return fail(PSC_EINVAL, "null batch");
  if (nsteps < 0) return fail(PSC_EINVAL, "nsteps must be >= 0");
  NvtxRange r(b->mode == PSC_BATCH_PERSISTENT ? "psc_batch_step persistent" : "psc_batch_step graph");
  for (int k = 0; k < nsteps; ++k) PSC_CUDA(cudaGraphLaunch(b->exec, b->st));
  for (size_t i = 0; i < b->sims.size(); ++i) {
    b->sims[i]->step += nsteps;
    if (b->mode == PSC_BATCH_GRAPH) b->sims[i]->launches += nsteps * b->launches_per_step[i];
  }
  if (b->mode == PSC_BATCH_PERSISTENT) b->launches += 4LL * nsteps;
  return PSC_OK;
}

// ---------------------------------------------------------------- persistent ensembles

static psc_status persistent_member_ok(const psc_sim* m, int max_N) {
  if (!m) return fail(PSC_EINVAL, "psc_batch: null member");
  if (m->fp64 || m->d.sph || m->p.nonlinear_form != PSC_NL_ROTATIONAL)
    return fail(PSC_EINVAL, "persistent batch: members must be FP32-mixed, 2/3 rule, rotational form");
  if (!pscb_size_supported(m->d.N) || m->d.N > max_N)
    return fail(PSC_EUNSUPPORTED_N, "persistent batch: N=" + std::to_string(m->d.N) +
                                        " not among the persistent sizes up to max_N=" + std::to_string(max_N));
  return PSC_OK;
}

static PscBatchBox box_of(psc_sim* s) {
  PscBatchBox b;
  std::memset(&b, 0, sizeof(b));
  b.N = s->d.N;
  b.K = s->d.K;
  b.M = s->d.M;
  b.P = s->d.P;
  b.S = s->d.S;
  b.zs = s->d.zs;
  b.ys = s->d.ys;
  b.U = s->ws + s->L.U;
  b.V = s->ws + s->L.V;
  b.Acc = s->ws + s->L.Acc;
  b.zreg = s->ws + s->L.zreg;
  b.yreg = s->ws + s->L.yreg;
  b.eu = s->ws + s->L.eu;
  b.ep = s->ws + s->L.ep;
  b.tw = s->ws + s->L.tw;
  b.ctrl = s->ctrl;
  const CombineArgs c = combine_args(s, nullptr);
  b.kF2 = c.kF2;
  b.kF2_floor = c.kF2_floor;
  b.eps_inj = s->p.eps_inj;
  b.beta = c.beta;
  b.nu = c.nu;
  b.D = c.D;
  b.cfl = s->p.cfl;
  b.dx = 2.0 * M_PI / s->p.N;
  b.forcing = s->p.forcing;
  b.integrator = s->p.integrator;
  b.scalar_on = s->p.scalar_on;
  b.record_every = s->p.record_every;
  b.cfl_on = s->p.cfl > 0.0 ? 1 : 0;
  return b;
}

static psc_status persistent_upload(psc_batch* b, psc_sim* const* sims, int n) {
  std::vector<PscBatchBox> boxes;
  for (int i = 0; i < n; ++i) {
    psc_status st = persistent_member_ok(sims[i], b->max_N);
    if (st != PSC_OK) return st;
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return fail(PSC_EINVAL, "psc_batch: members must be distinct");
    boxes.push_back(box_of(sims[i]));
  }
  PSC_CUDA(pscb_upload(b->table, b->staging.data(), b->max_boxes, boxes.data(), n, b->st, b->stall_test));
  b->sims.assign(sims, sims + n);
  b->launches_per_step.assign(n, 0);
  return PSC_OK;
}

extern "C" {

psc_status psc_batch_table_bytes(int32_t max_boxes, size_t* bytes) {
  if (max_boxes < 1 || max_boxes > PSC_BATCH_MAX_BOXES || !bytes)
    return fail(PSC_EINVAL, "psc_batch_table_bytes: max_boxes in 1..PSC_BATCH_MAX_BOXES and non-null bytes");
  *bytes = pscb_table_bytes(max_boxes);
  return PSC_OK;
}

psc_status psc_batch_create_persistent(psc_sim* const* sims, int32_t n, int32_t max_boxes, int32_t max_N,
                                       void* dev_table, size_t table_bytes, void* stream, psc_batch** out) {
  if (!sims || n < 0 || !out || !stream || !dev_table)
    return fail(PSC_EINVAL, "psc_batch_create_persistent: null argument or negative n");
  if (max_boxes < 1 || max_boxes > PSC_BATCH_MAX_BOXES || n > max_boxes)
    return fail(PSC_EINVAL, "psc_batch_create_persistent: need n <= max_boxes <= PSC_BATCH_MAX_BOXES");
  if (!pscb_size_supported(max_N)) return fail(PSC_EUNSUPPORTED_N, "psc_batch_create_persistent: bad max_N");
  if (((uintptr_t)dev_table & 255) != 0 || table_bytes < pscb_table_bytes(max_boxes))
    return fail(PSC_EINVAL, "psc_batch_create_persistent: table must be 256-byte aligned and "
                            "psc_batch_table_bytes() long");
  psc_batch* b = new (std::nothrow) psc_batch();
  if (!b) return fail(PSC_EINVAL, "host allocation failed");
  b->mode = PSC_BATCH_PERSISTENT;
  b->st = (cudaStream_t)stream;
  b->max_boxes = max_boxes;
  b->max_N = max_N;
  b->table = dev_table;
  b->staging.resize(pscb_table_bytes(max_boxes));
  b->smem = pscb_smem_bytes(max_N);
  b->grid = pscb_grid(max_N, b->smem);
  {
    // test knob: one dependency of stage 1 is never met, so its bounded wait
    // runs out and the members report PSC_ETIMEOUT (the failure path)
    const char* e = std::getenv("PSC_BATCH_STALL_TEST");
    b->stall_test = e && e[0] == '1';
  }
  psc_status st = persistent_upload(b, sims, n);
  if (st != PSC_OK) { batch_free(b); return st; }
  // one ensemble step: a counter reset and one persistent launch per RK stage
  cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t e1 = pscb_step(b->table, b->max_boxes, b->max_N, b->grid, b->smem, b->st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->st, &g);
    if (e == cudaSuccess) e = e1;
    if (e == cudaSuccess) { b->graph = g; e = cudaGraphInstantiate(&b->exec, g, 0); }
    else if (g) cudaGraphDestroy(g);
  }
  if (e != cudaSuccess) { batch_free(b); return cuda_fail(e, "psc_batch_create_persistent: graph capture"); }
  *out = b;
  return PSC_OK;
}

psc_status psc_batch_set_members(psc_batch* b, psc_sim* const* sims, int32_t n) {
  if (!b || (n > 0 && !sims) || n < 0) return fail(PSC_EINVAL, "psc_batch_set_members: null batch or members");
  if (b->mode != PSC_BATCH_PERSISTENT) return fail(PSC_EINVAL, "psc_batch_set_members: persistent batches only");
  if (n > b->max_boxes) return fail(PSC_EINVAL, "psc_batch_set_members: more members than max_boxes");
  return persistent_upload(b, sims, n);
}

psc_status psc_batch_info(const psc_batch* b, int32_t* mode, int32_t* grid, int64_t* launches) {
  if (!b) return fail(PSC_EINVAL, "null batch");
  if (mode) *mode = b->mode;
  if (grid) *grid = b->mode == PSC_BATCH_PERSISTENT ? b->grid : 0;
  if (launches) *launches = b->launches;
  return PSC_OK;
}

}  // extern "C"

psc_status psc_batch_destroy(psc_batch* b) {
  if (b) batch_free(b);
  return PSC_OK;
}

}  // extern "C"
