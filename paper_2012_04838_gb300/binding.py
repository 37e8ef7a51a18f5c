"""Thin ctypes binding of ``include/psc.h``.

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``libpsc.so``.  PyTorch supplies the device workspace and the stream.  If
the library has not been built the import of a simulation fails loudly; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
import os

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- C structs


class CParams(ct.Structure):
    _fields_ = [
        ("N", ct.c_int32), ("precision", ct.c_int32),
        ("nu", ct.c_double), ("Sc", ct.c_double), ("beta", ct.c_double),
        ("forcing", ct.c_int32), ("integrator", ct.c_int32),
        ("kF", ct.c_double), ("eps_inj", ct.c_double), ("dt", ct.c_double), ("cfl", ct.c_double),
        ("seed", ct.c_uint64), ("ic", ct.c_int32), ("record_every", ct.c_int32),
        ("ic_energy", ct.c_double), ("ic_noise_frac", ct.c_double),
        ("scalar_on", ct.c_int32), ("nonlinear_form", ct.c_int32),
        ("dealias", ct.c_int32), ("reserved", ct.c_int32),
    ]


class CStats(ct.Structure):
    _fields_ = [(n, ct.c_double) for n in (
        "t", "dt", "K", "K_phys", "eps", "eps_phys", "eta", "Re_lambda", "Te", "urms", "lambda_",
        "l0", "cfl", "umax", "kmax_eta", "kmax_eta_sqrt2")] + [
        ("skew", ct.c_double * 3), ("flat", ct.c_double * 3)] + [
        (n, ct.c_double) for n in ("phi_var", "phi_prod", "phi_prod_phys", "chi", "chi_phys")] + [
        ("skew_phi", ct.c_double * 3), ("flat_phi", ct.c_double * 3)] + [
        (n, ct.c_double) for n in ("A", "E_forced", "P_inj")] + [("step", ct.c_int64)]

    def to_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out["lam" if name == "lambda_" else name] = list(v) if not isinstance(v, (int, float)) else v
        return out


PSC_OK, PSC_EINVAL, PSC_ENOMEM_BUDGET, PSC_ECUDA, PSC_EUNSTABLE, PSC_ETIMEOUT, PSC_EUNSUPPORTED_N = range(7)
FP64, FP32_MIXED = 0, 1
IC_SPECTRUM_K4, IC_TAYLOR_GREEN_NOISE, IC_PAPER_EQ9 = 0, 1, 2
FORCE_NONE, FORCE_CONST_POWER, FORCE_HOLD_ENERGY = 0, 1, 2
NL_ROTATIONAL, NL_CONVECTIVE = 0, 1
DEALIAS_TWO_THIRDS, DEALIAS_PHASE_SHIFT = 0, 1
INTEG_IFRK4, INTEG_RK4 = 0, 1

# every entry point of include/psc.h: (name, restype, argtypes)
_VP, _SZ = ct.c_void_p, ct.c_size_t
EXPORTS = [
    ("psc_workspace_size", ct.c_int, [ct.POINTER(CParams), ct.POINTER(_SZ)]),
    ("psc_supported_sizes", ct.c_int32, [ct.POINTER(ct.c_int32), ct.c_int32]),
    ("psc_create", ct.c_int, [ct.POINTER(CParams), _VP, _SZ, _VP, ct.POINTER(_VP)]),
    ("psc_init_field", ct.c_int, [_VP]),
    ("psc_step", ct.c_int, [_VP, ct.c_int32]),
    ("psc_spectra_and_stats", ct.c_int, [_VP, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                         ct.c_int32, ct.POINTER(ct.c_int32), ct.POINTER(CStats)]),
    ("psc_state_bytes", ct.c_int, [_VP, ct.POINTER(_SZ)]),
    ("psc_get_state", ct.c_int, [_VP, _VP, _SZ]),
    ("psc_set_state", ct.c_int, [_VP, _VP, _SZ]),
    ("psc_rhs", ct.c_int, [_VP, _VP, _VP]),
    ("psc_time", ct.c_int, [_VP, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_double)]),
    ("psc_batch_create", ct.c_int, [ct.POINTER(_VP), ct.c_int32, _VP, ct.POINTER(_VP)]),
    ("psc_batch_step", ct.c_int, [_VP, ct.c_int32]),
    ("psc_batch_destroy", ct.c_int, [_VP]),
    ("psc_batch_table_bytes", ct.c_int, [ct.c_int32, ct.POINTER(_SZ)]),
    ("psc_batch_create_persistent", ct.c_int, [ct.POINTER(_VP), ct.c_int32, ct.c_int32, ct.c_int32, _VP, _SZ,
                                               _VP, ct.POINTER(_VP)]),
    ("psc_batch_set_members", ct.c_int, [_VP, ct.POINTER(_VP), ct.c_int32]),
    ("psc_batch_info", ct.c_int, [_VP, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int64)]),
    ("psc_profile_enable", ct.c_int, [_VP, ct.c_int32]),
    ("psc_profile_read", ct.c_int, [_VP, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int32]),
    ("psc_launch_count", ct.c_int, [_VP, ct.POINTER(ct.c_int64)]),
    ("psc_tile_widths", ct.c_int, [_VP, ct.POINTER(ct.c_int32)]),
    ("psc_tile_staged", ct.c_int, [_VP, ct.POINTER(ct.c_int32)]),
    ("psc_pressure", ct.c_int, [_VP, _VP, ct.c_size_t]),
    ("psc_destroy", ct.c_int, [_VP]),
    ("psc_shell_spectra_noalloc", ct.c_int, [_VP, ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_double),
                                             ct.POINTER(ct.c_double), ct.c_int32, _VP]),
    ("psc_xpass_probe_bytes", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int64, ct.POINTER(_SZ)]),
    ("psc_xpass_probe", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int64, _VP, _SZ, _VP, ct.c_int32]),
    ("psc_fma_probe", ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, _VP, _VP]),
    ("psc_last_error", ct.c_char_p, []),
]

_LIB = {}


def lib_path(checked: bool | None = None) -> str:
    if os.environ.get("PSC_LIB"):
        return os.environ["PSC_LIB"]
    if checked is None:
        checked = os.environ.get("PSC_CHECKED", "0") == "1"
    return _build.lib_path(checked)


def load(checked: bool | None = None) -> ct.CDLL:
    """Load libpsc (raises if it has not been built)."""
    path = lib_path(checked)
    if path in _LIB:
        return _LIB[path]
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ct.CDLL(path)
    for name, res, args in EXPORTS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB[path] = lib
    return lib


class PscError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"psc status {status}: {msg}")
        self.status = status


def _check(lib, status: int) -> None:
    if status != PSC_OK:
        raise PscError(status, lib.psc_last_error().decode())


# ---------------------------------------------------------------- Python API


@dataclasses.dataclass
class Params:
    """Mirror of ``psc_params`` (defaults: the 32^3 Taylor-Green case)."""
    N: int = 32
    precision: int = FP64
    nu: float = 0.02
    Sc: float = 1.0
    beta: float = 1.0
    forcing: int = FORCE_CONST_POWER
    integrator: int = INTEG_IFRK4
    kF: float = 2.0
    eps_inj: float = 0.1
    dt: float = 0.005
    cfl: float = 0.0
    seed: int = 1
    ic: int = IC_TAYLOR_GREEN_NOISE
    record_every: int = 10
    ic_energy: float = 1.5
    ic_noise_frac: float = 0.01
    scalar_on: int = 1
    nonlinear_form: int = 0  # NL_ROTATIONAL
    dealias: int = 0  # DEALIAS_TWO_THIRDS

    def c(self) -> CParams:
        return CParams(**{f.name: getattr(self, f.name) for f in dataclasses.fields(self)})


def workspace_size(p: Params) -> int:
    lib = load()
    n = ct.c_size_t()
    cp = p.c()
    _check(lib, lib.psc_workspace_size(ct.byref(cp), ct.byref(n)))
    return n.value


def supported_sizes() -> list[int]:
    lib = load()
    buf = (ct.c_int32 * 64)()
    n = lib.psc_supported_sizes(buf, 64)
    return list(buf[:n])


def sphere_halfwidth(N: int) -> int:
    """The largest k with 9 k^2 < 2 N^2 (the sphere of phase-shift dealiasing)."""
    k = 0
    while 9 * (k + 1) ** 2 < 2 * N * N:
        k += 1
    return k


def retained_halfwidth(N: int, dealias: int = DEALIAS_TWO_THIRDS) -> int:
    """K of the compact layout: (N-1)//3 (2/3 rule), or the half-width of the
    cube that stores the sphere of phase-shift dealiasing: the sphere's own, or
    one more where that makes K + 1 even and the cube still fits the grid (the
    added planes lie outside the sphere and stay zero)."""
    if dealias == DEALIAS_PHASE_SHIFT:
        k = sphere_halfwidth(N)
        return k + 1 if k % 2 == 0 and 2 * (k + 1) + 1 <= N else k
    return (N - 1) // 3


def compact_shape(N: int, dealias: int = DEALIAS_TWO_THIRDS):
    K = retained_halfwidth(N, dealias)
    return (4, 2 * K + 1, 2 * K + 1, K + 1)


class Simulation:
    """One simulation on one GPU: workspace and stream come from PyTorch."""

    def __init__(self, p: Params, device=None, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.p = p
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = workspace_size(p)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ct.c_void_p()
        cp = p.c()
        with torch.cuda.device(self.device):
            _check(self.lib, self.lib.psc_create(ct.byref(cp), ct.c_void_p(self._ws_ptr), nbytes,
                                                 ct.c_void_p(self.stream.cuda_stream), ct.byref(self._h)))
        self.cdtype = torch.complex128 if p.precision == FP64 else torch.complex64
        self.shape = compact_shape(p.N, p.dealias)

    # -- lifecycle
    def close(self) -> None:
        if self._h:
            self.lib.psc_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points
    def init_field(self) -> None:
        _check(self.lib, self.lib.psc_init_field(self._h))

    def step(self, n: int = 1) -> None:
        _check(self.lib, self.lib.psc_step(self._h, n))

    def stats(self):
        """(record dict, E(n), E_phi(n)) of the current state."""
        cap = 4096
        E = (ct.c_double * cap)()
        Ep = (ct.c_double * cap)()
        ns = ct.c_int32()
        st = CStats()
        _check(self.lib, self.lib.psc_spectra_and_stats(self._h, E, Ep, cap, ct.byref(ns), ct.byref(st)))
        n = ns.value
        return st.to_dict(), np.array(E[:n]), np.array(Ep[:n])

    def state_bytes(self) -> int:
        n = ct.c_size_t()
        _check(self.lib, self.lib.psc_state_bytes(self._h, ct.byref(n)))
        return n.value

    def get_state(self, device=None):
        """Compact state as a (4, P, P, M) complex tensor (on the GPU by default)."""
        t = self.torch.empty(self.shape, dtype=self.cdtype,
                             device=self.device if device is None else device)
        _check(self.lib, self.lib.psc_get_state(self._h, ct.c_void_p(t.data_ptr()), self.state_bytes()))
        return t

    def set_state(self, t) -> None:
        t = t.to(self.cdtype).contiguous()
        if tuple(t.shape) != self.shape:
            raise ValueError(f"state shape {tuple(t.shape)} != {self.shape}")
        _check(self.lib, self.lib.psc_set_state(self._h, ct.c_void_p(t.data_ptr()), self.state_bytes()))

    def rhs(self, state):
        """N(u, phi) of a compact state (device tensor), as a new device tensor."""
        x = state.to(device=self.device, dtype=self.cdtype).contiguous()
        out = self.torch.empty_like(x)
        _check(self.lib, self.lib.psc_rhs(self._h, ct.c_void_p(x.data_ptr()), ct.c_void_p(out.data_ptr())))
        self.stream.synchronize()
        return out

    def pressure(self):
        """Modified pressure p_hat of the current state (Eq. 6), one compact
        field as a new device tensor [2K+1][2K+1][K+1]."""
        K = retained_halfwidth(self.p.N, self.p.dealias)
        out = self.torch.empty((2 * K + 1, 2 * K + 1, K + 1), dtype=self.cdtype, device=self.device)
        _check(self.lib, self.lib.psc_pressure(self._h, ct.c_void_p(out.data_ptr()),
                                               out.numel() * out.element_size()))
        self.stream.synchronize()
        return out

    KERNEL_KINDS = ("forcing", "zinv", "yinv", "xpass", "yfwd", "zfwd", "combine", "other")

    def profile(self, on: bool = True) -> None:
        _check(self.lib, self.lib.psc_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{kind: (device ms, launches)} since the last read (synchronises)."""
        n = len(self.KERNEL_KINDS)
        ms = (ct.c_double * n)()
        cnt = (ct.c_int64 * n)()
        _check(self.lib, self.lib.psc_profile_read(self._h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNEL_KINDS)}

    def tile_widths(self) -> dict:
        w = (ct.c_int32 * 4)()
        _check(self.lib, self.lib.psc_tile_widths(self._h, w))
        return dict(zip(("zinv", "yinv", "yfwd", "zfwd"), list(w)))

    def tile_staged(self) -> dict:
        """{pass: True if it stages input tiles through shared memory by TMA}."""
        w = (ct.c_int32 * 4)()
        _check(self.lib, self.lib.psc_tile_staged(self._h, w))
        return dict(zip(("zinv", "yinv", "yfwd", "zfwd"), [bool(v) for v in w]))

    def launch_count(self) -> int:
        n = ct.c_int64()
        _check(self.lib, self.lib.psc_launch_count(self._h, ct.byref(n)))
        return n.value

    def time(self):
        t, dt = ct.c_double(), ct.c_double()
        n = ct.c_int64()
        _check(self.lib, self.lib.psc_time(self._h, ct.byref(t), ct.byref(n), ct.byref(dt)))
        return t.value, n.value, dt.value


PERSISTENT_SIZES = (32, 48, 64, 96, 128, 192, 256)
BATCH_GRAPH, BATCH_PERSISTENT = 0, 1


class PersistentBatch:
    """Members stepped by one persistent launch per RK stage over a device work
    table (psc_batch_create_persistent); members can be replaced between steps
    (set_members) without a new graph capture.  Members: FP32-mixed, 2/3 rule,
    rotational form, N in PERSISTENT_SIZES and N <= max_N."""

    def __init__(self, sims, max_boxes: int, max_N: int, device=None, stream=None):
        import torch
        self.lib = load()
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        n = ct.c_size_t()
        _check(self.lib, self.lib.psc_batch_table_bytes(max_boxes, ct.byref(n)))
        self.nbytes = n.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.sims = list(sims)
        arr = (ct.c_void_p * max(1, len(self.sims)))(*[s._h.value for s in self.sims])
        self._h = ct.c_void_p()
        for s in self.sims:
            s.stream.synchronize()
        with torch.cuda.device(self.device):
            _check(self.lib, self.lib.psc_batch_create_persistent(arr, len(self.sims), max_boxes, max_N,
                                                                  ct.c_void_p(self.ptr), self.nbytes,
                                                                  ct.c_void_p(self.stream.cuda_stream),
                                                                  ct.byref(self._h)))

    def set_members(self, sims) -> None:
        self.sims = list(sims)
        arr = (ct.c_void_p * max(1, len(self.sims)))(*[s._h.value for s in self.sims])
        _check(self.lib, self.lib.psc_batch_set_members(self._h, arr, len(self.sims)))

    def step(self, n: int = 1) -> None:
        _check(self.lib, self.lib.psc_batch_step(self._h, n))

    def synchronize(self) -> None:
        self.stream.synchronize()

    def info(self) -> dict:
        mode, grid, launches = ct.c_int32(), ct.c_int32(), ct.c_int64()
        _check(self.lib, self.lib.psc_batch_info(self._h, ct.byref(mode), ct.byref(grid), ct.byref(launches)))
        return {"mode": mode.value, "grid": grid.value, "launches": launches.value}

    def close(self) -> None:
        if self._h:
            self.lib.psc_batch_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Members stepped together through one captured CUDA graph per step.

    Members on different streams (``Simulation(..., stream=torch.cuda.Stream())``)
    run as concurrent branches; members sharing a stream run one after another.
    The batch replays on ``stream`` (a fresh stream by default).  Synchronise the
    batch stream before touching a member directly."""

    def __init__(self, sims, stream=None):
        import torch
        self.lib = load()
        self.sims = list(sims)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.sims[0].device)
        arr = (ct.c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        self._h = ct.c_void_p()
        for s in self.sims:
            s.stream.synchronize()
        with torch.cuda.device(self.sims[0].device):
            _check(self.lib, self.lib.psc_batch_create(arr, len(self.sims),
                                                       ct.c_void_p(self.stream.cuda_stream),
                                                       ct.byref(self._h)))

    def step(self, n: int = 1) -> None:
        _check(self.lib, self.lib.psc_batch_step(self._h, n))

    def synchronize(self) -> None:
        self.stream.synchronize()

    def close(self) -> None:
        if self._h:
            self.lib.psc_batch_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class XPassProbe:
    """The right-hand-side X pass of an N-grid over `rows` rows of synthetic
    input (psc_xpass_probe): a small-footprint stand-in for profiling."""

    def __init__(self, N: int, precision: int, rows: int, device=None, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.N, self.precision, self.rows = N, precision, rows
        self.device = torch.device(device if device is not None else "cuda")
        n = ct.c_size_t()
        _check(self.lib, self.lib.psc_xpass_probe_bytes(N, precision, rows, ct.byref(n)))
        self.nbytes = n.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)

    def run(self, nlaunch: int = 1) -> None:
        _check(self.lib, self.lib.psc_xpass_probe(self.N, self.precision, self.rows, ct.c_void_p(self.ptr),
                                                  self.nbytes, ct.c_void_p(self.stream.cuda_stream), nlaunch))


def fma_peak_tflops(precision: int, device=None, iters: int = 2000, repeats: int = 3) -> float:
    """FMA throughput of the device in TFLOP/s (psc_fma_probe, best of
    `repeats` launches of 8 CTAs per SM, CUDA events)."""
    import torch
    lib = load()
    dev = torch.device(device if device is not None else "cuda")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * sms
    out = torch.empty(blocks * 256, dtype=torch.float64 if precision == FP64 else torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    _check(lib, lib.psc_fma_probe(precision, 10, blocks, ct.c_void_p(out.data_ptr()), ct.c_void_p(st.cuda_stream)))
    best = None
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib, lib.psc_fma_probe(precision, iters, blocks, ct.c_void_p(out.data_ptr()),
                                      ct.c_void_p(st.cuda_stream)))
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    flops = 2.0 * 128 * iters * 256 * blocks  # 128 iters FMAs per thread
    return flops / (best / 1000.0) / 1e12
