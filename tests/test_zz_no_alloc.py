"""The allocation-free shell-spectrum entry point.

For callers that cannot allocate device memory (pre-sized graph pipelines,
plugins whose host owns the allocator): psc_shell_spectra_noalloc() keeps its
partial sums in a fixed array inside the library.  Its spectra must equal those
of psc_spectra_and_stats() on the same state, call after call, because every
call reuses (and must fully rewrite) that array.  This file is collected last."""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
B = pytest.importorskip("paper_2012_04838_gb300.binding")

TOL = {B.FP64: 1e-12, B.FP32_MIXED: 1e-6}


def _noalloc(lib, state, N, prec, cap, stream):
    Ek = torch.full((cap,), float("nan"), dtype=torch.float64, device=state.device)
    Ep = torch.full((cap,), float("nan"), dtype=torch.float64, device=state.device)
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(state.data_ptr()), N, prec,
                                       ct.cast(ct.c_void_p(Ek.data_ptr()), ct.POINTER(ct.c_double)),
                                       ct.cast(ct.c_void_p(Ep.data_ptr()), ct.POINTER(ct.c_double)),
                                       cap, ct.c_void_p(stream.cuda_stream))
    assert st == B.PSC_OK, lib.psc_last_error().decode()
    stream.synchronize()
    return Ek.cpu().numpy(), Ep.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [B.FP64, B.FP32_MIXED], ids=["fp64", "fp32"])
def test_noalloc_spectra_match_spectra_and_stats_on_consecutive_calls(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load()
    N = 48
    sim = B.Simulation(B.Params(N=N, precision=prec, ic=B.IC_SPECTRUM_K4, seed=21, nu=0.02, dt=0.004),
                       device="cuda:0")
    sim.init_field()
    cap = 64
    for call in range(2):
        sim.step(3)  # a different state (with a developed scalar) for each call
        _, E, Ep = sim.stats()
        state = sim.get_state()
        gE, gEp = _noalloc(lib, state, N, prec, cap, sim.stream)
        n = len(E)
        assert np.allclose(gE[:n], E, rtol=TOL[prec], atol=TOL[prec] * E.max()), call
        assert np.allclose(gEp[:n], Ep, rtol=TOL[prec], atol=TOL[prec] * Ep.max()), call
        assert np.isnan(gE[n:]).all()  # nothing written past the last shell
    sim.close()


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load()
    dummy = torch.zeros(8, dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(2048, dtype=torch.float64, device="cuda:0")
    p = ct.cast(ct.c_void_p(out.data_ptr()), ct.POINTER(ct.c_double))
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(dummy.data_ptr()), 2048, B.FP32_MIXED, p, p, 2048, None)
    assert st == B.PSC_EINVAL
    assert b"shells" in lib.psc_last_error()
    st = lib.psc_shell_spectra_noalloc(ct.c_void_p(dummy.data_ptr()), 64, B.FP32_MIXED, p, p, 10, None)
    assert st == B.PSC_EINVAL
