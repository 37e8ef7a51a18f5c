"""The allocation-free shell-spectrum entry point.

For callers that cannot allocate device memory (pre-sized graph pipelines,
plugins whose host owns the allocator): psc_shell_spectra_noalloc() keeps its
partial sums in a fixed array inside the library.  Its spectra must equal those
of psc_spectra_and_stats() on the same state, call after call, because every
call reuses (and must fully rewrite) that array.  This file is collected last."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from oracle import psc_oracle as O

B = pytest.importorskip("paper_2012_04838_gb300.binding")

TOL = {B.FP64: 1e-12, B.FP32_MIXED: 1e-6}
DEALIAS = [B.DEALIAS_TWO_THIRDS, B.DEALIAS_PHASE_SHIFT]


@pytest.fixture(scope="module")
def lib():
    from paper_2012_04838_gb300 import build
    if not os.path.exists(B.lib_path()):
        build.build()
    return B.load()


def _dptr(p):
    return ct.cast(ct.c_void_p(p), ct.POINTER(ct.c_double))


def _shells_needed(lib, N, dealias):
    """The shell count the entry point derives for (N, dealias), read from its
    refusal of zero-capacity outputs (decided on the host, before any CUDA call);
    None if it refuses the grid as too large for its scratch."""
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(256), N, B.FP32_MIXED, dealias, _dptr(256), _dptr(256), 0,
                                       None)
    assert st == B.PSC_EINVAL
    msg = lib.psc_last_error().decode()
    if "fixed scratch" in msg:
        return None
    m = re.search(r"hold 0 shells, (\d+) needed", msg)
    assert m, msg
    return int(m.group(1))


@pytest.mark.parametrize("dealias", DEALIAS, ids=["two_thirds", "phase_shift"])
def test_noalloc_shell_count_is_the_simulations(lib, dealias):
    # the count of psc_spectra_and_stats (the oracle's num_shells is pinned to the
    # shell definition n = floor(|k| + 1/2) and the retained sets)
    for N in (8, 16, 48, 96, 256, 512, 520, 1024):
        assert _shells_needed(lib, N, dealias) == O.num_shells(N, dealias), N
    # the scratch limit of PSC_NOALLOC_MAX_SHELLS = 1024 shells
    last_ok, first_no = (1773, 1774) if dealias == B.DEALIAS_TWO_THIRDS else (2170, 2171)
    assert _shells_needed(lib, last_ok, dealias) == O.num_shells(last_ok, dealias) <= 1024
    assert O.num_shells(first_no, dealias) > 1024
    assert _shells_needed(lib, first_no, dealias) is None


def test_noalloc_rejects_bad_arguments_on_the_host(lib):
    p = _dptr(256)
    for args in [(ct.c_void_p(256), 4, B.FP64, 0), (ct.c_void_p(256), 64, 7, 0), (ct.c_void_p(256), 64, B.FP64, 2),
                 (None, 64, B.FP64, 0)]:
        st = lib.psc_shell_spectra_noalloc(args[0], args[1], args[2], args[3], p, p, 4096, None)
        assert st == B.PSC_EINVAL


def _noalloc(lib, torch, state, N, prec, dealias, cap, stream):
    Ek = torch.full((cap,), float("nan"), dtype=torch.float64, device=state.device)
    Ep = torch.full((cap,), float("nan"), dtype=torch.float64, device=state.device)
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(state.data_ptr()), N, prec, dealias, _dptr(Ek.data_ptr()),
                                       _dptr(Ep.data_ptr()), cap, ct.c_void_p(stream.cuda_stream))
    assert st == B.PSC_OK, lib.psc_last_error().decode()
    stream.synchronize()
    return Ek.cpu().numpy(), Ep.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("dealias", DEALIAS, ids=["two_thirds", "phase_shift"])
@pytest.mark.parametrize("prec", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_noalloc_spectra_match_spectra_and_stats_on_consecutive_calls(lib, prec, dealias):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 48
    sim = B.Simulation(B.Params(N=N, precision=prec, ic=B.IC_SPECTRUM_K4, seed=21, nu=0.02, dt=0.004,
                                dealias=dealias), device="cuda:0")
    sim.init_field()
    cap = 64
    for call in range(2):
        sim.step(3)  # a different state (with a developed scalar) for each call
        _, E, Ep = sim.stats()
        state = sim.get_state()
        gE, gEp = _noalloc(lib, torch, state, N, prec, dealias, cap, sim.stream)
        n = len(E)
        assert n == O.num_shells(N, dealias)
        assert np.allclose(gE[:n], E, rtol=TOL[prec], atol=TOL[prec] * E.max()), call
        assert np.allclose(gEp[:n], Ep, rtol=TOL[prec], atol=TOL[prec] * Ep.max()), call
        assert np.isnan(gE[n:]).all()  # nothing written past the last shell
    sim.close()


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dummy = torch.zeros(8, dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(2048, dtype=torch.float64, device="cuda:0")
    p = _dptr(out.data_ptr())
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(dummy.data_ptr()), 2048, B.FP32_MIXED, 0, p, p, 2048, None)
    assert st == B.PSC_EINVAL
    assert b"shells" in lib.psc_last_error()
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(dummy.data_ptr()), 64, B.FP32_MIXED, 0, p, p, 10, None)
    assert st == B.PSC_EINVAL


@pytest.mark.gpu
def test_noalloc_rejects_host_memory_before_launching(lib):
    # a host buffer (pageable or pinned) is refused as an argument error; the
    # checks run before any kernel, so nothing on the device reads it
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 16
    state = torch.zeros(B.compact_shape(N), dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(64, dtype=torch.float64, device="cuda:0")
    host = np.zeros(4 * 64, dtype=np.float64)
    pinned = torch.zeros(64, dtype=torch.float64).pin_memory()
    hstate = torch.zeros(B.compact_shape(N), dtype=torch.complex64).pin_memory()
    cases = [
        (state.data_ptr(), host.ctypes.data, out.data_ptr()),
        (state.data_ptr(), out.data_ptr(), pinned.data_ptr()),
        (hstate.data_ptr(), out.data_ptr(), out.data_ptr()),
    ]
    for s_, e_, p_ in cases:
        st = lib.psc_shell_spectra_noalloc(ct.c_void_p(s_), N, B.FP32_MIXED, 0, _dptr(e_), _dptr(p_), 64, None)
        assert st == B.PSC_EINVAL, lib.psc_last_error().decode()
        assert b"device memory" in lib.psc_last_error()
    torch.cuda.synchronize()
