"""Pins for the FP64 oracle: each test checks the oracle against something the
paper or the mathematics fixes independently of the oracle's own code
(brute-force sums, closed forms, conservation laws, published test vectors)."""
import math
import os

import numpy as np
import pytest

from oracle import psc_oracle as O
from tests.psc_inputs import (compact_to_full, full_to_compact, random_compact_state, separable_compact_state,
                              separable_factors)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_velocity(N, seed, solenoidal=True):
    g = O.Grid(N)
    c = random_compact_state(N, seed, nfields=4)
    f = compact_to_full(c, N)
    uh = f[:3]
    if solenoidal:
        uh = np.array(O.project(list(uh), g))
    return g, uh, f[3]


# ---------------------------------------------------------------- DFT (Eq. 5)

def _brute_dft(a):
    N = a.shape[0]
    n = np.arange(N)
    W = np.exp(-2j * np.pi * np.outer(n, n) / N)
    out = np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
    for kz in range(N):
        for ky in range(N):
            for kx in range(N // 2 + 1):
                s = 0.0
                for z in range(N):
                    s += W[kz, z] * np.sum(a[z] * np.outer(W[ky], W[kx]))
                out[kz, ky, kx] = s
    return out


@pytest.mark.parametrize("N", [8, 10, 12, 26])
def test_fwd_matches_bruteforce_dft(N):
    a = np.random.default_rng(N).standard_normal((N, N, N))
    ref = _brute_dft(a)
    assert np.allclose(O.fwd(a), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("N", [8, 10, 12])
def test_inverse_is_normalised_bruteforce_sum(N):
    g = O.Grid(N)
    _, uh, _ = _rand_velocity(N, 3, solenoidal=False)
    ah = uh[0]
    x = O.inv(ah, N)
    # phi(x) = N^-3 sum over the full k set; expand the half spectrum by symmetry
    full = np.zeros((N, N, N), dtype=np.complex128)
    full[:, :, : N // 2 + 1] = ah
    for kx in range(1, N - N // 2):
        full[:, :, N - kx] = np.conj(ah[(-np.arange(N)) % N][:, (-np.arange(N)) % N, kx])
    n = np.arange(N)
    E = np.exp(2j * np.pi * np.outer(n, n) / N)
    ref = np.einsum("az,by,cx,abc->zyx", E, E, E, full).real / N ** 3
    assert np.allclose(x, ref, atol=1e-12 * np.abs(ref).max())


def test_parseval():
    N = 16
    a = np.random.default_rng(5).standard_normal((N, N, N))
    g = O.Grid(N)
    ah = O.fwd(a)
    lhs = np.sum(a * a)
    rhs = np.sum(g.w[..., : N // 2 + 1] * np.where(g.kx == N // 2, 0.5, 1.0) * np.abs(ah) ** 2) / N ** 3
    assert abs(lhs - rhs) < 1e-12 * lhs


def test_spectral_derivative_is_exact_for_trig_polynomial():
    N = 16
    g = O.Grid(N)
    a = np.sin(3 * g.x) * np.cos(2 * g.y) * np.sin(g.z)
    a = np.broadcast_to(a, (N, N, N))
    gx, gy, gz = [O.inv(c, N) for c in O.grad_hat(O.fwd(a), g)]
    assert np.allclose(gx, 3 * np.cos(3 * g.x) * np.cos(2 * g.y) * np.sin(g.z), atol=1e-13)
    assert np.allclose(gy, -2 * np.sin(3 * g.x) * np.sin(2 * g.y) * np.sin(g.z), atol=1e-13)
    assert np.allclose(gz, np.sin(3 * g.x) * np.cos(2 * g.y) * np.cos(g.z), atol=1e-13)


def test_truncation_keeps_two_thirds_cube():
    for N in (12, 16, 32, 96):
        g = O.Grid(N)
        K = g.K
        assert 3 * K < N <= 3 * K + 3
        assert int(g.mask.sum()) == (2 * K + 1) ** 2 * (K + 1)


def test_product_of_retained_modes_is_alias_free_on_R():
    # 3K < N: a product of two band-limited fields is exact on the retained set.
    N = 24
    g = O.Grid(N)
    _, uh, ph = _rand_velocity(N, 9, solenoidal=False)
    a, b = O.inv(uh[0], N), O.inv(ph, N)
    prod = O.truncate(O.fwd(a * b), g)
    # zero-padded product on a 2N grid has no aliasing on |k| <= 2K
    M = 2 * N
    gm = O.Grid(M)
    idx = np.arange(-g.K, g.K + 1)
    def pad(x):
        out = np.zeros(gm.shape_hat, dtype=complex)
        out[np.ix_(idx % M, idx % M, np.arange(g.K + 1))] = x[np.ix_(idx % N, idx % N, np.arange(g.K + 1))]
        return out * (M / N) ** 3
    big = O.fwd(O.inv(pad(uh[0]), M) * O.inv(pad(ph), M)) * (N / M) ** 3
    ref = big[np.ix_(idx % M, idx % M, np.arange(g.K + 1))]
    got = prod[np.ix_(idx % N, idx % N, np.arange(g.K + 1))]
    assert np.allclose(got, ref, atol=1e-9 * np.abs(ref).max())


# ---------------------------------------------------------------- projection (Eq. 7)

def test_projection_is_divergence_free_and_idempotent():
    g, uh, _ = _rand_velocity(24, 1, solenoidal=False)
    pu = O.project(list(uh), g)
    div = sum(kc * c for kc, c in zip(g.kvec, pu))
    assert np.abs(div).max() <= 1e-13 * np.abs(uh).max() * g.K
    ppu = O.project(pu, g)
    assert max(np.abs(a - b).max() for a, b in zip(pu, ppu)) < 1e-12 * np.abs(uh).max()


def test_rotational_equals_convective_form():
    g, uh, _ = _rand_velocity(24, 2)
    a = O.nonlinear_rotational(uh, g)
    b = O.nonlinear_convective(uh, g)
    scale = max(np.abs(x).max() for x in a)
    assert max(np.abs(x - y).max() for x, y in zip(a, b)) < 1e-11 * scale


@pytest.mark.parametrize("N", [8, 16])
def test_taylor_green_pressure_closed_form(N):
    # u = (sin x cos y cos z, -cos x sin y cos z, 0) has the pressure
    # p = (cos 2x + cos 2y)(cos 2z + 2)/16 up to a constant (from -lap p =
    # d_i u_j d_j u_i); all its modes have |k_i| <= 2 <= K, so it is exact on R
    g = O.Grid(N)
    x, y, z = g.x, g.y, g.z
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    uh = np.array([O.fwd(np.broadcast_to(u, (N,) * 3)), O.fwd(np.broadcast_to(v, (N,) * 3)),
                   O.fwd(np.zeros((N,) * 3))])
    p = O.inv(O.pressure_hat(uh, g), N)
    exact = (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2) / 16.0
    exact = np.broadcast_to(exact - exact.mean(), (N,) * 3)
    assert np.abs(p - exact).max() < 1e-14


def test_pressure_balances_the_projection():
    # the projection removes exactly the pressure gradient:
    # -(u.grad u)_hat - i k p_hat is solenoidal and equals P[-(u.grad u)_hat]
    g, uh, _ = _rand_velocity(16, 3)
    p = O.pressure_hat(uh, g)
    conv = O.nonlinear_convective(uh, g)  # -P[(u.grad u)_hat]
    u = O.velocity(uh, g)
    raw = []
    for i in range(3):
        gi = [O.inv(c, g.N) for c in O.grad_hat(uh[i], g)]
        raw.append(-O.truncate(O.fwd(u[0] * gi[0] + u[1] * gi[1] + u[2] * gi[2]), g))
    rebuilt = [raw[c] - 1j * g.kvec[c] * p for c in range(3)]
    scale = max(np.abs(c).max() for c in conv)
    assert max(np.abs(a - b).max() for a, b in zip(rebuilt, conv)) < 1e-12 * scale


def test_convective_and_rotational_runs_agree():
    # the two forms differ by a gradient that the projection removes, so whole
    # forced runs with scalar agree to round-off
    p = O.Params(N=24, nu=0.02, dt=0.005, ic=O.IC_TAYLOR_GREEN_NOISE, seed=3)
    c = O.Params(**{**p.__dict__, "nonlinear_form": O.NL_CONVECTIVE})
    u1, p1, _, _, _ = O.run(p, 10, with_records=False)
    u2, p2, _, _, _ = O.run(c, 10, with_records=False)
    assert np.abs(u1 - u2).max() < 1e-12 * np.abs(u1).max()
    assert np.abs(p1 - p2).max() < 1e-12 * np.abs(p1).max()


def test_nonlinear_terms_conserve_energy_and_variance():
    # sum_k Re(u* . N(u)) = 0 and sum_k Re(phi* . (u.grad phi)) = 0 on the
    # Galerkin-truncated system (3K < N makes the grid sums exact).
    p = O.Params(N=24, forcing=O.FORCE_NONE, beta=0.0)
    g, uh, ph = _rand_velocity(24, 4)
    ph = O.truncate(ph, g)
    ru, rp = O.rhs_nonlinear(uh, ph, g, p)
    e = sum(np.sum(g.w * np.real(np.conj(uh[c]) * ru[c])) for c in range(3))
    s = np.sum(g.w * np.real(np.conj(ph) * rp))
    escale = sum(np.sum(g.w * np.abs(uh[c]) * np.abs(ru[c])) for c in range(3))
    sscale = np.sum(g.w * np.abs(ph) * np.abs(rp))
    assert abs(e) < 1e-12 * escale
    assert abs(s) < 1e-12 * sscale


# ---------------------------------------------------------------- time stepping

def _shear(g, kk, amp=1.0):
    ux = amp * np.sin(kk * g.y) * np.ones((g.N, 1, g.N))
    z = np.zeros((g.N, g.N, g.N))
    return np.array([O.fwd(np.broadcast_to(ux, (g.N,) * 3)), O.fwd(z), O.fwd(z)])


@pytest.mark.parametrize("integ", [O.INTEG_IFRK4, O.INTEG_RK4])
def test_single_mode_shear_decays_exactly(integ):
    # u = (sin k y, 0, 0): u x omega = grad(sin^2(ky)/2) is removed by P, so
    # u(t) = exp(-nu k^2 t) u0; IF-RK4 reproduces it to round-off, plain RK4
    # reproduces its stability polynomial R(z) = 1+z+z^2/2+z^3/6+z^4/24 exactly.
    N, kk, nu, dt, n = 16, 3, 0.05, 0.01, 25
    p = O.Params(N=N, nu=nu, forcing=O.FORCE_NONE, beta=0.0, integrator=integ)
    g = O.Grid(N)
    uh = _shear(g, kk)
    u0 = uh.copy()
    ph = np.zeros(g.shape_hat, dtype=complex)
    for _ in range(n):
        uh, ph = O.step(uh, ph, g, p, dt)
    z = -nu * kk * kk * dt
    fac = math.exp(z * n) if integ == O.INTEG_IFRK4 else (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) ** n
    assert np.abs(uh - fac * u0).max() < 1e-12 * np.abs(u0).max()
    assert np.abs(ph).max() == 0.0


@pytest.mark.parametrize("integ", [O.INTEG_IFRK4, O.INTEG_RK4])
def test_hold_forcing_keeps_a_decaying_band_mode_exactly(integ):
    # u = (sin y, 0, 0) lies in the forced sphere (|k| = 1 <= kF = 2) and only
    # decays viscously (its u x omega is removed by P), by exp(-nu dt) per step
    # under IF-RK4 and by R(-nu dt) under RK4.  Holding the band energy
    # multiplies it back by exactly the inverse, so the state never changes and
    # the equivalent forcing rate is A = nu (IF-RK4) or -ln R(-nu dt)/dt (RK4):
    # the injected power 2 A E_f then equals the dissipation 2 nu |k|^2 E_f.
    N, nu, dt, n = 16, 0.05, 0.01, 12
    p = O.Params(N=N, nu=nu, forcing=O.FORCE_HOLD_ENERGY, kF=2.0, beta=0.0, integrator=integ,
                 dt=dt, record_every=4)
    g = O.Grid(N)
    uh = _shear(g, 1, amp=0.7)
    ph = np.zeros(g.shape_hat, dtype=complex)
    u1, ph1, recs, _, _ = O.run(p, n, uh=uh.copy(), ph=ph)
    assert np.abs(u1 - uh).max() < 1e-13 * np.abs(uh).max()
    z = -nu * dt
    rate = nu if integ == O.INTEG_IFRK4 else -math.log(1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) / dt
    assert recs[0]["A"] == 0.0  # before the first step
    for r in recs[1:]:
        assert abs(r["A"] - rate) < 1e-10 * rate
        assert abs(r["P_inj"] - 2.0 * nu * r["E_forced"]) < 1e-6 * r["P_inj"] * (integ == O.INTEG_RK4) + 1e-10 * r["P_inj"]


def test_hold_forcing_rescales_only_the_band():
    # one step of a turbulent state: the band energy returns to its starting
    # value, and every mode outside the band is exactly the unforced step's
    N = 24
    g = O.Grid(N)
    p = O.Params(N=N, nu=0.02, forcing=O.FORCE_HOLD_ENERGY, kF=2.0, ic=O.IC_SPECTRUM_K4, seed=7, dt=0.004)
    uh, ph = O.init_field(g, p)
    ef0 = O.forced_energy(uh, g, p.kF)
    free = O.Params(**{**p.__dict__, "forcing": O.FORCE_NONE})
    uf, pf = O.step(uh, ph, g, free, p.dt)
    u1, ph1, _, _, _ = O.run(p, 1, uh=uh.copy(), ph=ph.copy(), with_records=False)
    assert abs(O.forced_energy(u1, g, p.kF) - ef0) < 1e-13 * ef0
    b = O.band(g, p.kF)
    assert np.array_equal(np.where(b, 0, u1), np.where(b, 0, uf))
    assert np.array_equal(ph1, pf)
    # and the band itself is the unforced band times one real factor
    f = math.sqrt(ef0 / O.forced_energy(uf, g, p.kF))
    assert np.abs(np.where(b, u1 - f * uf, 0)).max() < 1e-14 * np.abs(uf).max()


@pytest.mark.parametrize("Sc", [1.0, 0.1])
def test_mean_gradient_scalar_closed_form(Sc):
    # u = (0, a sin kx, 0), phi0 = 0: u.grad phi = 0 and u x omega is a gradient,
    # so phi = b(t) sin kx with b = -beta a (e^{-nu k^2 t} - e^{-D k^2 t}) / ((D - nu) k^2)
    # (-beta a t e^{-nu k^2 t} when D = nu).  At Sc = 1 the integrating-factor
    # frame makes the forcing constant and IF-RK4 is exact; otherwise 4th order.
    N, kk, a, nu, beta = 16, 4, 0.7, 0.03, 1.3
    g = O.Grid(N)
    p = O.Params(N=N, nu=nu, Sc=Sc, beta=beta, forcing=O.FORCE_NONE)
    D = nu / Sc
    uy = a * np.sin(kk * g.x) * np.ones((N, N, 1))
    z = np.zeros((N, N, N))
    uh0 = np.array([O.fwd(z), O.fwd(np.broadcast_to(uy, (N,) * 3)), O.fwd(z)])
    T = 0.4

    def b_exact(t):
        if Sc == 1.0:
            return -beta * a * t * math.exp(-nu * kk * kk * t)
        return -beta * a * (math.exp(-nu * kk * kk * t) - math.exp(-D * kk * kk * t)) / ((D - nu) * kk * kk)

    errs = []
    for n in (10, 20):
        dt = T / n
        uh, ph = uh0.copy(), np.zeros(g.shape_hat, dtype=complex)
        for _ in range(n):
            uh, ph = O.step(uh, ph, g, p, dt)
        phi = O.inv(ph, N)
        ref = b_exact(T) * np.sin(kk * g.x) * np.ones((N, N, 1))
        errs.append(np.abs(phi - ref).max())
    if Sc == 1.0:
        assert errs[1] < 1e-13
    else:
        assert errs[0] < 1e-4
        assert 12.0 < errs[0] / errs[1] < 20.0


def test_inviscid_conservation_converges_at_fourth_order():
    N = 16
    p = O.Params(N=N, nu=0.0, Sc=1.0, beta=0.0, forcing=O.FORCE_NONE)
    g, uh0, ph0 = _rand_velocity(N, 7)
    ph0 = O.truncate(ph0, g)
    E0 = O.spectra(uh0, ph0, g)
    K0, V0 = E0[0].sum(), E0[1].sum()
    T = 0.2
    drifts = []
    for n in (8, 16):
        uh, ph = uh0.copy(), ph0.copy()
        for _ in range(n):
            uh, ph = O.step(uh, ph, g, p, T / n)
        E = O.spectra(uh, ph, g)
        drifts.append((abs(E[0].sum() - K0) / K0, abs(E[1].sum() - V0) / V0))
    assert drifts[0][0] < 1e-4 and drifts[0][1] < 1e-4
    assert drifts[1][0] < drifts[0][0] / 10 and drifts[1][1] < drifts[0][1] / 10


def test_taylor_green_early_time_derivatives():
    # Pure Taylor-Green: K(0) = 1/8; every mode has |k|^2 = 3, so dK/dt(0) = -6 nu K0;
    # the t = 0 transfer lands on |k|^2 in {4, 8} (disjoint from the TG modes) and
    # d^2K/dt^2(0) = 36 nu^2 K0.
    N, nu = 16, 0.05
    p = O.Params(N=N, nu=nu, forcing=O.FORCE_NONE, beta=0.0, ic=O.IC_TAYLOR_GREEN_NOISE,
                 ic_noise_frac=0.0)
    g = O.Grid(N)
    uh0, ph0 = O.init_field(g, p)
    K0 = O.spectra(uh0, ph0, g)[0].sum()
    assert abs(K0 - 0.125) < 1e-15
    h = 2e-3
    Ks = {}
    for s in (-1, 1):
        uh, ph = O.step(uh0, ph0, g, p, s * h)
        Ks[s] = O.spectra(uh, ph, g)[0].sum()
    d1 = (Ks[1] - Ks[-1]) / (2 * h)
    d2 = (Ks[1] - 2 * K0 + Ks[-1]) / h ** 2
    assert abs(d1 - (-6 * nu * K0)) < 1e-6 * abs(6 * nu * K0)
    assert abs(d2 - 36 * nu * nu * K0) < 1e-3 * 36 * nu * nu * K0
    ru, _ = O.rhs_nonlinear(uh0, ph0, g, p)
    nl_k2 = set(np.unique(np.broadcast_to(g.k2, g.shape_hat)[np.abs(sum(np.abs(r) for r in ru)) > 1e-9]))
    assert nl_k2 <= {4, 8}


def test_taylor_green_coefficients_match_trig_expansion():
    # sin x cos y cos z = sum over signs of sx/(8i) e^{i(sx x + sy y + sz z)}
    N = 16
    g = O.Grid(N)
    uh = O.ic_taylor_green(g)
    for sy in (-1, 1):
        for sz in (-1, 1):
            assert abs(uh[0][sz % N, sy % N, 1] - N ** 3 / 8 / 1j) < 1e-10
            assert abs(uh[1][sz % N, sy % N, 1] - (-sy) * N ** 3 / 8 / 1j) < 1e-10
    assert np.abs(uh[2]).max() < 1e-10


def test_ifrk4_fourth_order_on_forced_nonlinear_system():
    N = 16
    p = O.Params(N=N, nu=0.02, Sc=0.7, beta=1.0, eps_inj=0.1, ic=O.IC_SPECTRUM_K4, seed=3)
    g = O.Grid(N)
    uh0, ph0 = O.init_field(g, p)
    T = 0.1

    def run(n):
        uh, ph = uh0.copy(), ph0.copy()
        for _ in range(n):
            uh, ph = O.step(uh, ph, g, p, T / n)
        return uh, ph
    ref = run(64)
    e = []
    for n in (4, 8):
        uh, ph = run(n)
        e.append(np.abs(uh - ref[0]).max() + np.abs(ph - ref[1]).max())
    assert 11.0 < e[0] / e[1] < 21.0


# ---------------------------------------------------------------- statistics

def test_dissipation_and_budget_identities():
    N = 24
    p = O.Params(N=N, nu=0.02, Sc=0.7, beta=1.3, eps_inj=0.1, kF=2.0)
    g, uh, ph = _rand_velocity(N, 11)
    ph = O.truncate(ph, g)
    s = O.stats(uh, ph, g, p)
    assert abs(s["eps_phys"] - s["eps"]) < 1e-12 * s["eps"]
    assert abs(p.nu * s["enstrophy"] - s["eps"]) < 1e-12 * s["eps"]
    assert abs(s["chi_phys"] - s["chi"]) < 1e-12 * s["chi"]
    assert abs(s["phi_prod_phys"] - s["phi_prod"]) < 1e-11 * abs(s["phi_prod"])
    assert abs(s["E"].sum() - s["K"]) < 1e-14 * s["K"]
    assert abs(s["K_phys"] - s["K"]) < 1e-12 * s["K"]
    assert abs(2 * s["Ephi"].sum() - s["phi_var"]) < 1e-12 * s["phi_var"]
    assert abs(s["P_inj"] - p.eps_inj) < 1e-14
    # semi-discrete budgets: dK/dt = P_inj - eps and Eq. 13
    ru, rp = O.rhs_nonlinear(uh, ph, g, p)
    Lu, Lp = O.linear_rates(g, p)
    n6 = float(N) ** 6
    dK = sum(np.sum(g.w * np.real(np.conj(uh[c]) * (ru[c] + Lu * uh[c]))) for c in range(3)) / n6
    assert abs(dK - (s["P_inj"] - s["eps"])) < 1e-12 * s["eps"]
    dV = 2 * np.sum(g.w * np.real(np.conj(ph) * (rp + Lp * ph))) / n6
    assert abs(dV - (s["phi_prod"] - s["chi"])) < 1e-11 * s["chi"]


def test_budgets_close_over_a_record_interval():
    # integrated over a record interval the energy and scalar-variance budgets
    # close up to the time-integration error (Eq. 13 and its energy analogue)
    p = O.Params(N=16, nu=0.02, Sc=1.0, beta=1.0, eps_inj=0.1, ic=O.IC_SPECTRUM_K4, seed=4,
                 dt=0.0025)
    g = O.Grid(16)
    uh, ph = O.init_field(g, p)
    for _ in range(20):  # let the scalar develop
        uh, ph = O.step(uh, ph, g, p, p.dt)
    ss = [O.stats(uh, ph, g, p)]
    for _ in range(8):
        uh, ph = O.step(uh, ph, g, p, p.dt)
        ss.append(O.stats(uh, ph, g, p))
    t = np.arange(len(ss)) * p.dt
    simpson = lambda f: p.dt / 3 * (f[0] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum() + f[-1])
    dK = ss[-1]["K"] - ss[0]["K"]
    srcK = simpson(np.array([s["P_inj"] - s["eps"] for s in ss]))
    dV = ss[-1]["phi_var"] - ss[0]["phi_var"]
    srcV = simpson(np.array([s["phi_prod"] - s["chi"] for s in ss]))
    eps = ss[0]["eps"]
    assert abs(dK - srcK) < 1e-3 * eps * t[-1]
    assert abs(dV - srcV) < 1e-3 * abs(ss[0]["chi"]) * t[-1] + 1e-12


def test_shell_index_matches_integer_definition():
    # n = floor(|k| + 1/2)  <=>  n^2 - n < |k|^2 <= n^2 + n  (exact integers)
    k2 = np.arange(0, 3 * 341 ** 2 + 1)
    n = np.floor(np.sqrt(k2.astype(np.float64)) + 0.5).astype(np.int64)
    ok = (k2 == 0) & (n == 0) | ((n * n - n < k2) & (k2 <= n * n + n))
    assert ok.all()


def test_cfl_dt_hits_target():
    g, uh, _ = _rand_velocity(16, 12)
    dt = O.cfl_dt(uh, g, 0.5)
    assert abs(O.cfl_number(uh, g, dt) - 0.5) < 1e-15


@pytest.mark.parametrize("N", [8, 10, 16, 24])
def test_cfl_maximum_is_of_the_component_sum(N):
    # Eq. 10 takes max(|u1| + |u2| + |u3|).  For u = a (sin z, sin x, sin y) the
    # three terms depend on different coordinates, so the maximum of their sum over
    # the grid is the sum of their maxima, 3 a max_j |sin(2 pi j / N)|: 3a where
    # the grid holds pi/2 (N divisible by 4).  The largest |u| (sqrt(3) a there)
    # and the largest component (a) differ from it.
    a = 1.7
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    uh = np.array([O.fwd(a * np.sin(Z)), O.fwd(a * np.sin(X)), O.fwd(a * np.sin(Y))])
    g = O.Grid(N)
    want = 3 * a * np.abs(np.sin(x)).max()
    if N % 4 == 0:
        assert abs(want - 3 * a) < 1e-15
    assert abs(O.max_abs_sum(uh, g) - want) < 1e-13
    dx = 2 * np.pi / N
    assert abs(O.cfl_number(uh, g, 0.01) - 0.01 / dx * want) < 1e-13
    assert abs(O.cfl_dt(uh, g, 0.5) - 0.5 * dx / want) < 1e-15


def test_skewness_and_flatness_closed_form():
    # Eqs. 11-12 on fields whose gradients have exact grid moments.  With
    # u1 = sin x + a sin 2x, u2 = sin y + b sin 2y, u3 = sin z + c sin 2z and
    # phi = sum of (sin + d sin 2.) over the three axes, each d(.)/dx_i is
    # f = cos t + e cos 2t (e = 2a, ...), whose grid means are exact for N > 8:
    #   <f^2> = (1 + e^2)/2,   <f^3> = 3e/4,   <f^4> = 3/8 + 3e^2/2 + 3e^4/8.
    N = 32
    x = 2 * np.pi * np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    coef_u = (0.3, -0.7, 0.45)
    coef_p = (-0.2, 0.6, 1.1)
    axes = (X, Y, Z)
    uh = np.array([O.fwd(np.sin(axes[i]) + coef_u[i] * np.sin(2 * axes[i])) for i in range(3)])
    ph = O.fwd(sum(np.sin(axes[i]) + coef_p[i] * np.sin(2 * axes[i]) for i in range(3)))
    g = O.Grid(N)
    s = O.stats(uh, ph, g, O.Params(N=N))

    def closed(c):
        e = 2 * c
        m2, m3, m4 = (1 + e * e) / 2, 3 * e / 4, 3 / 8 + 1.5 * e * e + 3 * e ** 4 / 8
        return m3 / m2 ** 1.5, m4 / m2 ** 2

    for i in range(3):
        sk, fl = closed(coef_u[i])
        assert abs(s["skew"][i] - sk) < 1e-12 and abs(s["flat"][i] - fl) < 1e-12
        sk, fl = closed(coef_p[i])
        assert abs(s["skew_phi"][i] - sk) < 1e-12 and abs(s["flat_phi"][i] - fl) < 1e-12
    # the sign follows the third moment: a negative coefficient gives a negative skewness
    assert s["skew"][1] < 0 < s["skew"][0]


# ---------------------------------------------------------------- initial condition

def test_splitmix64_published_vector():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    for i, v in rows:
        assert O.splitmix64(0, int(i)) == int(v, 16)
    arr = O.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in arr] == [int(v, 16) for _, v in rows]


def test_random_ic_is_real_solenoidal_and_on_target_spectrum():
    N = 32
    p = O.Params(N=N, ic=O.IC_SPECTRUM_K4, ic_energy=1.5, seed=2)
    g = O.Grid(N)
    uh, ph = O.init_field(g, p)
    # real field: the half spectrum round-trips through the inverse transform
    for c in range(3):
        assert np.abs(O.fwd(O.inv(uh[c], N)) - uh[c]).max() < 1e-9 * np.abs(uh[c]).max()
    div = sum(kc * c for kc, c in zip(g.kvec, uh))
    assert np.abs(div).max() < 1e-12 * np.abs(uh).max()
    E, _ = O.spectra(uh, ph, g)
    tgt = O.target_shell_energy(len(E), O.IC_SPECTRUM_K4, 1.0, p.kF)
    tgt = 1.5 * tgt / tgt.sum()
    assert abs(E.sum() - 1.5) < 1e-13
    assert np.allclose(E, tgt, rtol=1e-12, atol=1e-18)
    assert np.abs(ph).max() == 0.0


def test_random_ic_is_gaussian():
    # the paper's IC has Gaussian velocity and velocity-gradient components
    N = 64
    p = O.Params(N=N, ic=O.IC_SPECTRUM_K4, seed=5)
    g = O.Grid(N)
    uh, ph = O.init_field(g, p)
    s = O.stats(uh, ph, g, p)
    for c in range(3):
        u = O.inv(uh[c], N)
        _, sk, fl = O._moments(u)
        assert abs(sk) < 0.1 and abs(fl - 3) < 0.3
        assert abs(s["skew"][c]) < 0.1 and abs(s["flat"][c] - 3) < 0.3


def test_ic_grid_independent_low_modes():
    # the draw depends only on (k, seed): shells fully inside both boxes agree
    p = O.Params(ic=O.IC_SPECTRUM_K4, seed=7)
    g1, g2 = O.Grid(24), O.Grid(48)
    p.N = 24
    u1, _ = O.init_field(g1, p)
    p.N = 48
    u2, _ = O.init_field(g2, p)
    # shell 3 is inside both cubes; compare one mode up to the N^3 scaling and
    # the per-shell factor (which differs only through shells cut by the cube)
    m1 = u1[:, 2, 1, 1] / 24 ** 3
    m2 = u2[:, 2, 1, 1] / 48 ** 3
    r = m1 / m2
    assert np.allclose(r, r[0], rtol=1e-12)


def test_scalar_advection_sign_and_mean_gradient_source():
    # u = (sin y, 0, 0), phi = sin x: dphi/dt = -u.grad phi - beta u2 = -sin y cos x
    # (u2 = 0); with u = (0, sin x, 0) instead the source is -beta sin x.
    N = 16
    g = O.Grid(N)
    p = O.Params(N=N, forcing=O.FORCE_NONE, beta=0.8)
    one = np.ones((N, N, N))
    z = np.zeros((N, N, N))
    uh = np.array([O.fwd(np.sin(g.y) * one), O.fwd(z), O.fwd(z)])
    ph = O.fwd(np.sin(g.x) * one)
    _, rp = O.rhs_nonlinear(uh, ph, g, p)
    assert np.allclose(O.inv(rp, N), -np.sin(g.y) * np.cos(g.x) * one, atol=1e-13)
    uh = np.array([O.fwd(z), O.fwd(np.sin(g.x) * one), O.fwd(z)])
    _, rp = O.rhs_nonlinear(uh, O.fwd(z), g, p)
    assert np.allclose(O.inv(rp, N), -0.8 * np.sin(g.x) * one, atol=1e-13)


def test_table1_derived_scales_are_consistent():
    # Table 1 relations: Re_lambda = K sqrt(20/(3 nu eps)), l0/eta = Re_lambda^{3/2}/15^{3/4}
    N = 16
    p = O.Params(N=N, nu=0.01)
    g, uh, ph = _rand_velocity(N, 13)
    s = O.stats(uh, ph, g, p)
    assert abs(s["Re_lambda"] - s["K"] * math.sqrt(20.0 / (3.0 * p.nu * s["eps"]))) < 1e-12 * s["Re_lambda"]
    assert abs(s["l0"] / s["eta"] - s["Re_lambda"] ** 1.5 / 15 ** 0.75) < 1e-10 * s["l0"] / s["eta"]
    assert abs(s["Te"] - s["l0"] / s["urms"]) < 1e-14 * s["Te"]


def test_sparse_triad_rhs_matches_fft_rhs():
    # two independent formulations of the same Galerkin right-hand side
    N = 24
    K = (N - 1) // 3
    p = O.Params(N=N, nu=0.02, beta=0.9, eps_inj=0.1, kF=2.0)
    rng = np.random.default_rng(3)
    modes = {}
    picks = [(1, 0, 1), (0, 2, -1), (2, 1, 0), (K, -K, 3), (3, K, -K), (1, -1, -1), (0, 1, 1)]
    for k in picks:
        v = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        modes[k] = v * N ** 3 * 0.1
        if k[0] == 0:
            modes[(0, -k[1], -k[2])] = np.conj(modes[k])
    full = np.zeros((4,) + O.Grid(N).shape_hat, dtype=np.complex128)
    for (kx, ky, kz), v in modes.items():
        full[:, kz % N, ky % N, kx] = v
    g = O.Grid(N)
    ru, rp = O.rhs_nonlinear(full[:3], full[3], g, p)
    ref = np.array(list(ru) + [rp])
    got = O.rhs_sparse_triads(modes, N, p)
    scale = np.abs(ref).max()
    seen = np.zeros(ref.shape[1:], dtype=bool)
    for (kx, ky, kz), v in got.items():
        assert np.abs(ref[:, kz % N, ky % N, kx] - v).max() < 1e-11 * scale
        seen[kz % N, ky % N, kx] = True
    # every mode the FFT path fills is one the triad sum found
    assert np.abs(np.where(seen[None], 0, ref)).max() < 1e-11 * scale


def test_sparse_triad_rhs_matches_fft_rhs_on_the_sphere():
    # the triad sum restricted to the sphere 9|k|^2 < 2N^2 against the phase-shift
    # FFT path: modes near the sphere's edge, whose single-grid products alias
    N = 24
    K = O.sphere_halfwidth(N)
    p = O.Params(N=N, nu=0.02, beta=0.9, eps_inj=0.1, kF=2.0, dealias=O.DEALIAS_PHASE_SHIFT)
    rng = np.random.default_rng(5)
    modes = {}
    picks = [(1, 0, 1), (0, 2, -1), (K, 0, 2), (2, K - 1, -3), (6, -6, 5), (0, K, 1), (1, -1, -1)]
    for k in picks:
        assert 9 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2) < 2 * N * N
        v = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        modes[k] = v * N ** 3 * 0.1
        if k[0] == 0:
            modes[(0, -k[1], -k[2])] = np.conj(modes[k])
    g = O.Grid(N, O.DEALIAS_PHASE_SHIFT)
    full = np.zeros((4,) + g.shape_hat, dtype=np.complex128)
    for (kx, ky, kz), v in modes.items():
        full[:, kz % N, ky % N, kx] = v
    ru, rp = O.rhs_nonlinear(full[:3], full[3], g, p)
    ref = np.array(list(ru) + [rp])
    got = O.rhs_sparse_triads(modes, N, p)
    scale = np.abs(ref).max()
    seen = np.zeros(ref.shape[1:], dtype=bool)
    for (kx, ky, kz), v in got.items():
        assert np.abs(ref[:, kz % N, ky % N, kx] - v).max() < 1e-11 * scale
        seen[kz % N, ky % N, kx] = True
    assert np.abs(np.where(seen[None], 0, ref)).max() < 1e-11 * scale
    # some output lies outside the 2/3 cube, where only the sphere keeps it
    K3 = (N - 1) // 3
    assert any(max(abs(c) for c in k) > K3 for k in got)


# ---------------------------------------------------------------- phase-shift dealiasing

def _sphere_field(g, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((g.N,) * 3)
    return O.truncate(O.fwd(a), g)


def _exact_product_on_grid(ah, bh, g):
    """a*b computed on a 2N grid (no aliasing for modes below N/2), returned as
    the N-grid transform restricted to the retained set."""
    N, N2 = g.N, 2 * g.N
    kf2 = np.fft.fftfreq(N2, 1.0 / N2).round().astype(np.int64)
    big = [np.zeros((N2, N2, N2 // 2 + 1), dtype=complex) for _ in range(2)]
    kz, ky, kx = np.nonzero(np.broadcast_to(g.mask, g.shape_hat))
    wz = np.broadcast_to(g.kz, g.shape_hat)[kz, ky, kx]
    wy = np.broadcast_to(g.ky, g.shape_hat)[kz, ky, kx]
    for dst, src in zip(big, (ah, bh)):
        dst[wz % N2, wy % N2, kx] = src[kz, ky, kx] * 8.0
    p = O.fwd(O.inv(big[0], N2) * O.inv(big[1], N2))
    out = np.zeros(g.shape_hat, dtype=complex)
    out[kz, ky, kx] = p[wz % N2, wy % N2, kx] / 8.0
    return out


@pytest.mark.parametrize("N", [16, 20, 24])
def test_phase_shift_dealiasing_removes_every_alias(N):
    # Patterson-Orszag: averaging the product formed on the grid and on the grid
    # shifted by half a cell cancels the aliases wrapped an odd number of times;
    # truncating to |k| < sqrt(2) N / 3 removes the rest, so the product of two
    # fields on the sphere equals the exact (2N-grid) product on the sphere
    g = O.Grid(N, O.DEALIAS_PHASE_SHIFT)
    a, b = _sphere_field(g, 1), _sphere_field(g, 2)
    got = O.dealiased_products([a, b], lambda x, y: [x * y], g)[0]
    exact = _exact_product_on_grid(a, b, g)
    scale = np.abs(exact).max()
    assert np.abs(got - exact).max() < 1e-12 * scale
    # one grid alone is not alias-free for this retained set
    single = O.truncate(O.fwd(O.inv(a, N) * O.inv(b, N)), g)
    assert np.abs(single - exact).max() > 1e-3 * scale
    assert O.sphere_halfwidth(N) == max(k for k in range(N) if 9 * k * k < 2 * N * N)


def test_phase_shift_galerkin_system_conserves_energy_and_forms_agree():
    N = 16
    g = O.Grid(N, O.DEALIAS_PHASE_SHIFT)
    rng = np.random.default_rng(5)
    uh = O.project([O.truncate(O.fwd(rng.standard_normal((N,) * 3)), g) for _ in range(3)], g)
    uh = np.array(uh)
    rot = O.nonlinear_rotational(uh, g)
    conv = O.nonlinear_convective(uh, g)
    scale = max(np.abs(c).max() for c in rot)
    assert max(np.abs(a - b).max() for a, b in zip(rot, conv)) < 1e-11 * scale
    e = sum(np.sum(g.w * np.real(np.conj(uh[c]) * rot[c])) for c in range(3))
    escale = sum(np.sum(g.w * np.abs(uh[c]) * np.abs(rot[c])) for c in range(3))
    assert abs(e) < 1e-12 * escale


# ---------------------------------------------------------------- separable states

@pytest.mark.parametrize("N,forcing,scalar_on", [(24, O.FORCE_CONST_POWER, 1), (32, O.FORCE_NONE, 1),
                                                 (36, O.FORCE_CONST_POWER, 0)])
def test_separable_rhs_equals_the_fft_rhs(N, forcing, scalar_on):
    # the factorised triad sums of SeparableRHS against the FFT right-hand side
    # of the same (materialised) state, element by element on the retained set
    f = separable_factors(N, 40 + N, rank=2)
    c = separable_compact_state(f, N)
    full = compact_to_full(c, N)
    p = O.Params(N=N, forcing=forcing, scalar_on=scalar_on, eps_inj=0.1, kF=2.0, beta=0.7)
    g = O.Grid(N)
    ru, rp = O.rhs_nonlinear(full[:3], full[3], g, p)
    want = full_to_compact(np.array(list(ru) + [rp]), N)
    sep = O.SeparableRHS(f[:3], f[3], N, p)
    K = (N - 1) // 3
    got = np.array([sep.plane(kz) for kz in range(-K, K + 1)]).transpose(1, 0, 2, 3)
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() < 1e-12 * scale
