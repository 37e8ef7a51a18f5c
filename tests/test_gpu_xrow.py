"""The shared-memory row X pass (the X pass of 520^3, whose plan splits a row
over two lanes) against the FP64 oracle at sizes the oracle transforms in
seconds.  PSC_XPASS_ROWS=1 at creation makes a simulation take the row X pass
where the register X pass also exists; tolerances are those of the other
parity tests (one right-hand side 1e-13 FP64 / 2e-6 FP32-mixed, 20 steps
1e-11 / 1e-4)."""
import numpy as np
import pytest

from oracle import psc_oracle as O
from tests.psc_inputs import compact_to_full, full_to_compact, random_compact_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")

TOL_RHS = {B.FP64: 1e-13, B.FP32_MIXED: 2e-6}
TOL_TRAJ = {B.FP64: 1e-11, B.FP32_MIXED: 1e-4}
PREC = [B.FP64, B.FP32_MIXED]
PNAME = {B.FP64: "fp64", B.FP32_MIXED: "fp32"}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def oparams(p):
    return O.Params(N=p.N, nu=p.nu, Sc=p.Sc, beta=p.beta, forcing=p.forcing, kF=p.kF,
                    eps_inj=p.eps_inj, dt=p.dt, cfl=p.cfl, seed=p.seed, ic=p.ic,
                    ic_energy=p.ic_energy, ic_noise_frac=p.ic_noise_frac,
                    integrator=p.integrator, scalar_on=p.scalar_on, record_every=p.record_every,
                    nonlinear_form=p.nonlinear_form, dealias=p.dealias)


def as_input(x, prec):
    if prec == B.FP32_MIXED:
        return x.astype(np.complex64).astype(np.complex128)
    return x


@pytest.fixture
def rows(monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    monkeypatch.setenv("PSC_XPASS_ROWS", "1")
    return torch.device("cuda:0")


def gpu_rhs(dev, p, x):
    sim = B.Simulation(p, device=dev)
    try:
        return sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    finally:
        sim.close()


def oracle_rhs(x, p):
    g = O.Grid(p.N, p.dealias)
    f = compact_to_full(x, p.N)
    ru, rp = O.rhs_nonlinear(f[:3], f[3], g, oparams(p))
    return full_to_compact(np.array(list(ru) + [rp]), p.N, B.retained_halfwidth(p.N, p.dealias))


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [8, 12, 16, 24, 48, 96, 192])
def test_row_xpass_rhs_matches_oracle(rows, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.013, Sc=0.7, beta=1.1, eps_inj=0.1, kF=2.0)
    x = as_input(random_compact_state(N, 500 + N, kpeak=4.0 if N < 128 else 8.0), prec)
    got = gpu_rhs(rows, p, x)
    ref = oracle_rhs(x, p)
    assert rel(got, ref) < TOL_RHS[prec]
    for f in range(4):
        assert rel(got[f], ref[f]) < 10 * TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 48])
def test_row_xpass_phase_shift_rhs_matches_oracle(rows, N, prec):
    PS = B.DEALIAS_PHASE_SHIFT
    p = B.Params(N=N, precision=prec, nu=0.01, beta=0.9, dealias=PS)
    K = B.retained_halfwidth(N, PS)
    x = as_input(random_compact_state(N, 70 + N, K=K, sphere=True), prec)
    assert rel(gpu_rhs(rows, p, x), oracle_rhs(x, p)) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [24, 32])
def test_row_xpass_stats_match_oracle(rows, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.02, Sc=0.7, beta=1.0, dt=0.005, ic=B.IC_SPECTRUM_K4, seed=4)
    sim = B.Simulation(p, device=rows)
    sim.init_field()
    sim.step(10)
    rec, E, Ep = sim.stats()
    st = sim.get_state().cpu().numpy().astype(np.complex128)
    sim.close()
    f = compact_to_full(st, N)
    ref = O.stats(f[:3], f[3], O.Grid(N), oparams(p), rec["t"], rec["dt"])
    tol = 1e-11 if prec == B.FP64 else 2e-5
    for k in ("K", "K_phys", "eps", "eps_phys", "umax", "phi_var", "phi_prod_phys", "chi_phys"):
        assert abs(rec[k] - ref[k]) <= tol * abs(ref[k]) + 1e-300, (k, rec[k], ref[k])
    atol = 1e-10 if prec == B.FP64 else 1e-4
    for k in ("skew", "flat", "skew_phi", "flat_phi"):
        assert np.allclose(rec[k], ref[k], rtol=atol, atol=atol), (k, rec[k], ref[k])


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 48])
def test_row_xpass_pressure_matches_oracle(rows, N, prec):
    p = B.Params(N=N, precision=prec)
    sim = B.Simulation(p, device=rows)
    x = as_input(random_compact_state(N, 31 + N), prec)
    sim.set_state(torch.from_numpy(x).to(rows))
    got = sim.pressure().cpu().numpy().astype(np.complex128)
    sim.close()
    f = compact_to_full(x, N)
    ref = full_to_compact(O.pressure_hat(f[:3], O.Grid(N))[None], N)[0]
    assert rel(got, ref) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_row_xpass_20_steps_with_cfl_match_oracle(rows, prec):
    N = 32
    p = B.Params(N=N, precision=prec, nu=0.01, cfl=0.5, record_every=5, ic=B.IC_TAYLOR_GREEN_NOISE, seed=1)
    sim = B.Simulation(p, device=rows)
    sim.init_field()
    sim.step(20)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    _, _, gdt = sim.time()
    sim.close()
    uh, ph, _, _, dt = O.run(oparams(p), 20, with_records=False)
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(got, ref) < TOL_TRAJ[prec]
    assert abs(gdt - dt) < (1e-13 if prec == B.FP64 else 1e-6) * dt
