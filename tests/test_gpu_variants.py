"""Every compiled variant of the strided passes gives the same numbers.

The strided passes come in tile-width variants and, for FP32 grids whose kx
rows are a multiple of 16 bytes (M even), in variants that stage their input
tiles through shared memory with TMA tensor copies.  All variants run the same
arithmetic per column, so the right-hand side and the statistics records must
agree bit for bit; variant 0 is also checked against the oracle.  The variant
is forced with PSC_STRIDED_VARIANT when the simulation is created."""
import numpy as np
import pytest

from tests.psc_inputs import random_compact_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2012_04838_gb300.binding")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    return torch.device("cuda:0")


def variant_codes(N, prec):
    """PSC_STRIDED_VARIANT codes (z-inverse, y-inverse, y-forward, z-forward)
    covering every variant built for the grid: 0/1 unstaged 8/16 columns,
    2/3 staged 4/8 columns, 4 staged 16 columns (inverse passes only)."""
    if prec == B.FP64:
        return ["0000"]
    M = (N - 1) // 3 + 1
    if N >= 64 and M % 2 == 0:
        return ["0000", "1111", "2222", "3333", "4433"]
    return ["0000", "1111"]


def run_variant(dev, monkeypatch, p, x, v):
    monkeypatch.setenv("PSC_STRIDED_VARIANT", v)
    sim = B.Simulation(p, device=dev)
    try:
        staged = sim.tile_staged()
        r = sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy()
        sim.set_state(torch.from_numpy(x).to(dev))
        rec, E, Ep = sim.stats()
    finally:
        sim.close()
    return staged, r, rec, E, Ep


@pytest.mark.parametrize("N", [64, 96, 128, 192, 256])
def test_variants_agree_bit_for_bit(dev, monkeypatch, N):
    p = B.Params(N=N, precision=B.FP32_MIXED, nu=0.013, Sc=0.7, beta=1.1, eps_inj=0.1, kF=2.0, dt=1e-3)
    x = random_compact_state(N, 300 + N, kpeak=6.0).astype(np.complex64)
    codes = variant_codes(N, B.FP32_MIXED)
    nv = len(codes)
    out = [run_variant(dev, monkeypatch, p, x, c) for c in codes]
    for v in range(nv):
        assert all(out[v][0].values()) == (v >= 2), (v, out[v][0])
    for v in range(1, nv):
        np.testing.assert_array_equal(out[v][1], out[0][1])
        np.testing.assert_array_equal(out[v][3], out[0][3])
        np.testing.assert_array_equal(out[v][4], out[0][4])
        for k in ("K", "eps", "eps_phys", "chi", "chi_phys", "skew", "flat", "phi_var"):
            assert out[v][2][k] == out[0][2][k], (v, k)
    for bad in ("5", "4444", "12"):  # not built / not for the forward passes / malformed
        monkeypatch.setenv("PSC_STRIDED_VARIANT", bad)
        with pytest.raises(B.PscError):
            B.Simulation(p, device=dev)


def test_variants_agree_bit_for_bit_1024(dev, monkeypatch):
    """The full-size grid: the right-hand side of one state under each variant
    (one simulation at a time, 62 GB each)."""
    N = 1024
    p = B.Params(N=N, precision=B.FP32_MIXED, nu=3.341e-4, Sc=1.0, beta=1.0, eps_inj=0.1, kF=2.0, dt=1e-3)
    M, P = 342, 683
    g = torch.Generator(device=dev).manual_seed(11)
    x = torch.view_as_complex(torch.randn((4, P, P, M, 2), generator=g, device=dev, dtype=torch.float32)) * 1e3
    x[:, :, :, 0] = 0  # keep the kx = 0 plane trivially Hermitian
    ref = None
    for v in variant_codes(N, B.FP32_MIXED):
        monkeypatch.setenv("PSC_STRIDED_VARIANT", v)
        sim = B.Simulation(p, device=dev)
        try:
            r = sim.rhs(x)
            if ref is None:
                ref = r
            else:
                assert torch.equal(r, ref), v
                del r
        finally:
            sim.close()
        torch.cuda.empty_cache()
