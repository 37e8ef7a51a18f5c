"""Long forced runs, FP32-mixed against FP64 on the GPU (whose FP64 path matches
the oracle to 1e-13 per step): the trajectories decorrelate, so the comparison
is statistical.  Time-averaged E(k) must agree within 2% per shell for
k <= k_max/2 (k_max = N/3) and the time-averaged dissipation within 1%."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")
S = pytest.importorskip("paper_2012_04838_gb300.serve")


def _run(prec, N, steps, every):
    p = B.Params(N=N, precision=prec, nu=S.nu_for_resolution(N, 1.5), Sc=1.0, beta=1.0, kF=2.0, eps_inj=0.1, cfl=0.5, ic=B.IC_SPECTRUM_K4, seed=2,
                 ic_energy=1.5, record_every=every)
    sim = B.Simulation(p, device="cuda:0")
    sim.init_field()
    recs, spectra = [], []
    for n in range(0, steps + 1, every):
        if n:
            sim.step(every)
        rec, E, _ = sim.stats()
        recs.append(rec)
        spectra.append(E)
    sim.close()
    return recs, np.array(spectra)


def test_long_run_statistics_fp32_vs_fp64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, steps, every = 128, 2000, 10
    r32, E32 = _run(B.FP32_MIXED, N, steps, every)
    r64, E64 = _run(B.FP64, N, steps, every)
    half = len(r32) // 2
    e32 = np.mean([r["eps"] for r in r32[half:]])
    e64 = np.mean([r["eps"] for r in r64[half:]])
    assert abs(e32 - e64) <= 0.01 * e64, (e32, e64)
    m32, m64 = E32[half:].mean(axis=0), E64[half:].mean(axis=0)
    kmax_half = int((N / 3) / 2)
    rel = np.abs(m32[1:kmax_half + 1] - m64[1:kmax_half + 1]) / m64[1:kmax_half + 1]
    assert rel.max() <= 0.02, rel


def _golden_longrun_64():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "longrun_64_oracle.txt")
    vals = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        vals[tuple(parts[:-1])] = float(parts[-1])
    return vals


@pytest.mark.parametrize("prec", [B.FP32_MIXED, B.FP64], ids=["fp32", "fp64"])
def test_long_run_statistics_match_the_oracle_64(prec):
    """64^3, 2000 forced steps against the FP64 oracle's own run of the same
    configuration (time averages stored by tests/golden/make_longrun_64.py):
    E(k) within 2% per shell for k <= k_max/2 and eps within 1%, over all 201
    records and over the second half."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, steps, every = 64, 2000, 10
    ref = _golden_longrun_64()
    recs, E = _run(prec, N, steps, every)
    assert len(recs) == 201
    kmax_half = int((N / 3) / 2)
    for tag, rs, Es in (("all", recs, E), ("half", recs[len(recs) // 2:], E[len(recs) // 2:])):
        eps = np.mean([r["eps"] for r in rs])
        assert abs(eps - ref[(tag, "eps")]) <= 0.01 * ref[(tag, "eps")], (tag, eps, ref[(tag, "eps")])
        m = Es.mean(axis=0)
        want = np.array([ref[(tag, f"E{n}")] for n in range(1, kmax_half + 1)])
        rel = np.abs(m[1:kmax_half + 1] - want) / want
        assert rel.max() <= 0.02, (tag, rel)
