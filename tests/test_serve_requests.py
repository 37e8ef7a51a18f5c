"""Seeded request streams of the serving benchmark (host logic only)."""
import numpy as np

from paper_2012_04838_gb300 import serve as S


def test_poisson_requests_are_seeded_and_in_range():
    a = S.poisson_requests(200, rate=4.0, seed=5)
    b = S.poisson_requests(200, rate=4.0, seed=5)
    assert [(r.arrival, r.N, r.steps, r.nu, r.Sc, r.seed) for r in a] == \
           [(r.arrival, r.N, r.steps, r.nu, r.Sc, r.seed) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert 0.18 < gaps.mean() < 0.32  # mean inter-arrival 1/4 s
    assert {r.N for r in a} <= {64, 96, 128, 192, 256}
    assert all(100 <= r.steps <= 2000 for r in a)
    assert {r.Sc for r in a} <= {0.7, 1.0, 2.0}


def test_viscosity_hits_the_requested_resolution():
    for N in (64, 256, 1024):
        for ke in (1.0, 1.5, 2.0):
            nu = S.nu_for_resolution(N, ke)
            eta = (nu ** 3 / 0.1) ** 0.25
            assert abs(N / 3.0 * eta - ke) < 1e-12
    # the 256^3 and 1024^3 workloads: nu from k_max eta = 1.5
    assert abs(S.nu_for_resolution(1024, 1.5) - 3.341e-4) < 1e-7
    assert abs(S.nu_for_resolution(256, 1.5) - 2.121e-3) < 1e-6
