"""The plain cuFFT-style comparator of bench.py (whole-grid torch.fft transforms
and torch elementwise kernels) computes the same right-hand side as the
oracle, so the time it reports is the time of the same work.  Runs on CPU."""
import numpy as np
import pytest

from oracle import psc_oracle as O
from tests.psc_inputs import compact_to_full, full_to_compact, random_compact_state

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N", [16, 24])
def test_plain_comparator_equals_the_oracle_rhs(N):
    import bench
    x = random_compact_state(N, 31)
    got = bench.plain_rhs_torch(torch.from_numpy(x), N).numpy()
    g = O.Grid(N)
    f = compact_to_full(x, N)
    ru, rp = O.rhs_nonlinear(f[:3], f[3], g, O.Params(N=N, beta=1.0, kF=2.0, eps_inj=0.1))
    want = full_to_compact(np.array(list(ru) + [rp]), N)
    got_c = full_to_compact(got, N)
    assert np.linalg.norm(got_c - want) / np.linalg.norm(want) < 1e-12
    # nothing outside the retained cube
    full = np.zeros_like(got)
    full[...] = got
    K = (N - 1) // 3
    idx = np.arange(-K, K + 1) % N
    full[:, idx[:, None], idx[None, :], :K + 1] = 0
    assert np.abs(full).max() < 1e-12 * np.abs(want).max()


def test_stationary_window_means_of_the_paper_example():
    """bench.stationary_means averages the last 40% of a run, counted in
    large-eddy turnover times, and takes the scalar-gradient moments along
    the mean gradient (component 2)."""
    import bench
    series = []
    for i in range(11):  # t/T_e = 0, 1, ..., 10
        series.append({"t_over_Te": float(i), "Re_lambda": 100.0 + 10 * i,
                       "skew": [-0.5, -0.6, -0.7], "flat": [6.0, 7.0, 8.0],
                       "skew_phi": [0.0, 1.0 + 0.1 * i, 0.0], "flat_phi": [9.0, 20.0, 9.0],
                       "prod_over_chi": None if i == 0 else 1.0, "kmax_eta_sqrt2": 1.5})
    m = bench.stationary_means(series)
    assert m["window_t_over_Te"] == [6.0, 10.0] and m["records"] == 5
    assert abs(m["Re_lambda"] - 180.0) < 1e-12          # mean of 160 ... 200
    assert abs(m["skew_du"] + 0.6) < 1e-12 and abs(m["flat_du"] - 7.0) < 1e-12
    assert abs(m["skew_dphi_2"] - 1.8) < 1e-12 and m["flat_dphi_2"] == 20.0
    assert m["prod_over_chi"] == 1.0
    assert bench.stationary_means(series[:1]) is None
