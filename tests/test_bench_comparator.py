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
