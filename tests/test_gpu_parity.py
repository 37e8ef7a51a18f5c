"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances (relative L2 unless stated): one right-hand side 1e-13 in FP64 and
2e-6 in FP32-mixed; 20-step trajectories 1e-11 and 1e-4.  Sizes span one and
several FFT tiles, radix-3 lengths and ragged kx tiles (M not a multiple of the
column tile)."""
import math

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


def oparams(p: "B.Params") -> O.Params:
    return O.Params(N=p.N, nu=p.nu, Sc=p.Sc, beta=p.beta, forcing=p.forcing, kF=p.kF,
                    eps_inj=p.eps_inj, dt=p.dt, cfl=p.cfl, seed=p.seed, ic=p.ic,
                    ic_energy=p.ic_energy, ic_noise_frac=p.ic_noise_frac,
                    integrator=p.integrator, scalar_on=p.scalar_on, record_every=p.record_every,
                    nonlinear_form=p.nonlinear_form)


def oracle_rhs(x, p):
    N = p.N
    op = oparams(p)
    g = O.Grid(N)
    f = compact_to_full(x, N)
    ru, rp = O.rhs_nonlinear(f[:3], f[3], g, op)
    if p.integrator == B.INTEG_RK4:
        Lu, Lp = O.linear_rates(g, op)
        ru = [ru[c] + Lu * f[c] for c in range(3)]
        rp = rp + Lp * f[3]
    return full_to_compact(np.array(list(ru) + [rp]), N)


def as_input(x, prec):
    """The state the GPU sees (rounded to FP32 in mixed mode) as complex128."""
    if prec == B.FP32_MIXED:
        return x.astype(np.complex64).astype(np.complex128)
    return x


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    return torch.device("cuda:0")


# ---------------------------------------------------------------- right-hand side

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96])
def test_rhs_matches_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.013, Sc=0.7, beta=1.1, eps_inj=0.1, kF=2.0)
    sim = B.Simulation(p, device=dev)
    x = as_input(random_compact_state(N, 100 + N), prec)
    got = sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    ref = oracle_rhs(x, p)
    assert rel(got, ref) < TOL_RHS[prec]
    # each field separately, so no field hides behind a larger one
    for f in range(4):
        assert rel(got[f], ref[f]) < 10 * TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [128, 192, 256])
def test_rhs_matches_oracle_large(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.002, beta=1.0)
    sim = B.Simulation(p, device=dev)
    x = as_input(random_compact_state(N, 7 + N, kpeak=8.0), prec)
    got = sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    ref = oracle_rhs(x, p)
    assert rel(got, ref) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_rhs_plain_rk4_includes_linear_terms(dev, prec):
    N = 24
    p = B.Params(N=N, precision=prec, integrator=B.INTEG_RK4, nu=0.05, Sc=2.0)
    sim = B.Simulation(p, device=dev)
    x = as_input(random_compact_state(N, 5), prec)
    got = sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    assert rel(got, oracle_rhs(x, p)) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_rhs_edge_cases(dev, prec):
    N = 16
    p = B.Params(N=N, precision=prec)
    sim = B.Simulation(p, device=dev)
    # zero state: zero right-hand side (forcing amplitude 0 when the band is empty)
    z = np.zeros(B.compact_shape(N), dtype=np.complex128)
    got = sim.rhs(torch.from_numpy(z).to(dev)).cpu().numpy()
    assert np.abs(got).max() == 0.0
    # only modes outside the forcing band, no scalar: pure nonlinear term
    x = as_input(random_compact_state(N, 9), prec)
    K = (N - 1) // 3
    x[:, K - 2:K + 3, K - 2:K + 3, :3] = 0.0
    p2 = B.Params(N=N, precision=prec, forcing=B.FORCE_NONE, scalar_on=0)
    sim2 = B.Simulation(p2, device=dev)
    got = sim2.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    ref = oracle_rhs(x, p2)
    assert rel(got, ref) < TOL_RHS[prec]
    assert np.abs(got[3]).max() == 0.0


# ---------------------------------------------------------------- initial condition

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N,ic", [(16, B.IC_SPECTRUM_K4), (32, B.IC_TAYLOR_GREEN_NOISE),
                                  (48, B.IC_PAPER_EQ9), (64, B.IC_SPECTRUM_K4)])
def test_initial_condition_matches_oracle(dev, N, ic, prec):
    p = B.Params(N=N, precision=prec, ic=ic, seed=11 + N, ic_energy=1.5, ic_noise_frac=0.01)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    g = O.Grid(N)
    uh, ph = O.init_field(g, oparams(p))
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(got, ref) < (1e-13 if prec == B.FP64 else 1e-6)
    assert np.abs(got[3]).max() == 0.0


# ---------------------------------------------------------------- trajectories

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N,integ", [(32, B.INTEG_IFRK4), (24, B.INTEG_RK4), (48, B.INTEG_IFRK4)])
def test_20_step_trajectory_matches_oracle(dev, N, integ, prec):
    # the 32^3 Taylor-Green case: nu = 0.02, Sc = 1, beta = 1, eps_inj = 0.1 on |k| <= 2
    p = B.Params(N=N, precision=prec, integrator=integ, nu=0.02, dt=0.005,
                 ic=B.IC_TAYLOR_GREEN_NOISE, seed=1)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    sim.step(20)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    op = oparams(p)
    uh, ph, _, t, _ = O.run(op, 20, with_records=False)
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(got[:3], ref[:3]) < TOL_TRAJ[prec]
    assert rel(got[3], ref[3]) < TOL_TRAJ[prec]
    tt, nstep, _ = sim.time()
    assert nstep == 20 and abs(tt - t) < 1e-12


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_config_c1_full_run_matches_oracle(dev, prec):
    """The small configuration end to end: 32^3 Taylor-Green plus 1% k^4 noise,
    nu = 0.02, Sc = 1, beta = 1, constant power 0.1 on |k|^2 <= 4, dt = 0.005,
    200 steps, a record every 10 steps (21 records with spectra)."""
    N = 32
    p = B.Params(N=N, precision=prec, nu=0.02, Sc=1.0, beta=1.0, eps_inj=0.1, kF=2.0, dt=0.005,
                 ic=B.IC_TAYLOR_GREEN_NOISE, seed=1, record_every=10)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    got = []
    for n in range(0, 201, 10):
        if n:
            sim.step(10)
        got.append(sim.stats())
    uh, ph, recs, t, _ = O.run(oparams(p), 200, with_records=True)
    assert len(recs) == len(got) == 21
    tol = 1e-10 if prec == B.FP64 else 2e-4
    keys = ("K", "eps", "eps_phys", "chi", "chi_phys", "phi_var", "phi_prod", "A", "E_forced")
    # scalar quantities start from exactly zero (phi = 0 at t = 0): an absolute
    # floor relative to each quantity's largest value over the run
    scale = {k: max(abs(r[k]) for r in recs) for k in keys}
    for (rec, E, Ep), ref in zip(got, recs):
        assert rec["step"] == ref["step"]
        assert abs(rec["t"] - ref["t"]) <= 1e-12 * max(1.0, ref["t"])
        for k in keys:
            assert abs(rec[k] - ref[k]) <= tol * abs(ref[k]) + 1e-12 * scale[k], (ref["step"], k, rec[k], ref[k])
        assert np.allclose(E, ref["E"], rtol=tol, atol=tol * ref["E"].max())
        if ref["Ephi"].max() > 0:
            assert np.allclose(Ep, ref["Ephi"], rtol=tol, atol=tol * ref["Ephi"].max())
        sk = 1e-8 if prec == B.FP64 else 2e-3
        assert np.allclose(rec["skew"], ref["skew"], rtol=sk, atol=sk), (ref["step"], rec["skew"], ref["skew"])
        assert np.allclose(rec["flat"], ref["flat"], rtol=sk, atol=sk), (ref["step"], rec["flat"], ref["flat"])
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    final = sim.get_state().cpu().numpy().astype(np.complex128)
    assert rel(final, ref) < (1e-10 if prec == B.FP64 else 1e-3)


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("integ", [B.INTEG_IFRK4, B.INTEG_RK4])
def test_hold_energy_forcing_matches_oracle(dev, prec, integ):
    """The paper's deterministic forcing: the band 0 < |k| <= 2 is rescaled
    after every step to the energy it had at the first step."""
    N = 32
    p = B.Params(N=N, precision=prec, integrator=integ, nu=0.02, dt=0.005, forcing=B.FORCE_HOLD_ENERGY,
                 kF=2.0, ic=B.IC_TAYLOR_GREEN_NOISE, seed=1, record_every=10)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    got = []
    for n in (0, 10, 20):
        if n:
            sim.step(10)
        got.append(sim.stats()[0])
    final = sim.get_state().cpu().numpy().astype(np.complex128)
    uh, ph, recs, _, _ = O.run(oparams(p), 20, with_records=True)
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(final, ref) < TOL_TRAJ[prec]
    tol = 1e-10 if prec == B.FP64 else 1e-4
    # A = ln(f)/dt with f - 1 ~ A dt: a relative error e of the band energy
    # moves A by about e/(2 dt), so FP32-mixed gets an absolute allowance
    atol_A = 0.0 if prec == B.FP64 else 1e-6 / p.dt
    for rec, r in zip(got, recs):
        assert abs(rec["E_forced"] - r["E_forced"]) <= tol * r["E_forced"]
        assert abs(rec["A"] - r["A"]) <= tol * abs(r["A"]) + atol_A, (rec["step"], rec["A"], r["A"])
    assert got[0]["A"] == 0.0 and got[2]["A"] != 0.0
    # the band energy is held at its starting value
    assert abs(got[2]["E_forced"] - got[0]["E_forced"]) <= (1e-12 if prec == B.FP64 else 1e-6) * got[0]["E_forced"]
    # a state set from outside becomes the new target
    x = as_input(random_compact_state(N, 77, kpeak=3.0), prec)
    sim.set_state(torch.from_numpy(x).to(dev))
    sim.step(5)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    f = compact_to_full(x, N)
    uh, ph, _, _, _ = O.run(oparams(p), 5, uh=f[:3], ph=f[3], with_records=False)
    assert rel(got, full_to_compact(np.concatenate([uh, ph[None]]), N)) < TOL_TRAJ[prec]
    sim.close()


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_cfl_controlled_run_matches_oracle(dev, prec):
    N = 32
    p = B.Params(N=N, precision=prec, nu=0.01, cfl=0.5, record_every=5, ic=B.IC_SPECTRUM_K4,
                 seed=2, ic_energy=1.5)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    sim.step(12)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    uh, ph, _, t, dt = O.run(oparams(p), 12, with_records=False)
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(got, ref) < TOL_TRAJ[prec]
    tt, _, gdt = sim.time()
    assert abs(gdt - dt) < (1e-13 if prec == B.FP64 else 1e-6) * dt
    assert abs(tt - t) < (1e-12 if prec == B.FP64 else 1e-6) * t


# ---------------------------------------------------------------- statistics

SCALARS = ["K", "K_phys", "eps", "eps_phys", "eta", "Re_lambda", "urms", "l0", "Te", "umax",
           "phi_var", "phi_prod", "phi_prod_phys", "chi", "chi_phys", "A", "E_forced", "P_inj"]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [24, 32])
def test_stats_match_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.02, Sc=0.7, beta=1.0, dt=0.005, ic=B.IC_SPECTRUM_K4, seed=4)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    sim.step(10)  # develop a scalar field
    rec, E, Ep = sim.stats()
    st = sim.get_state().cpu().numpy().astype(np.complex128)
    f = compact_to_full(st, N)
    op = oparams(p)
    ref = O.stats(f[:3], f[3], O.Grid(N), op, rec["t"], rec["dt"])
    tol = 1e-11 if prec == B.FP64 else 2e-5
    assert np.allclose(E, ref["E"], rtol=tol, atol=tol * ref["E"].max())
    assert np.allclose(Ep, ref["Ephi"], rtol=tol, atol=tol * ref["Ephi"].max())
    for k in SCALARS:
        assert abs(rec[k] - ref[k]) <= tol * abs(ref[k]) + 1e-300, (k, rec[k], ref[k])
    atol = 1e-10 if prec == B.FP64 else 1e-4
    for k in ("skew", "flat", "skew_phi", "flat_phi"):
        assert np.allclose(rec[k], ref[k], rtol=atol, atol=atol), (k, rec[k], ref[k])
    assert rec["step"] == 10


# ---------------------------------------------------------------- state round trip

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_state_roundtrip_and_restart_are_bit_exact(dev, prec):
    N = 32
    p = B.Params(N=N, precision=prec, ic=B.IC_SPECTRUM_K4, seed=3, dt=0.004)
    a = B.Simulation(p, device=dev)
    a.init_field()
    a.step(5)
    mid = a.get_state(device="cpu")
    a.step(5)
    end_a = a.get_state().cpu()
    b = B.Simulation(p, device=dev)
    b.set_state(mid)
    assert torch.equal(b.get_state(device="cpu"), mid)
    # dt and t are part of the run, not of the state: restart from step 5 with the same dt
    b.step(5)
    assert torch.equal(b.get_state().cpu(), end_a)


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_state_copies_through_pinned_host_memory_are_bit_exact(dev, prec):
    """get_state/set_state with pinned host buffers (copied by the SMs through
    the host mapping), pageable host buffers and device buffers give the same
    bits, also right after steps and for a buffer offset by 16 bytes."""
    N = 48
    p = B.Params(N=N, precision=prec, ic=B.IC_SPECTRUM_K4, seed=8, dt=0.004)
    a = B.Simulation(p, device=dev)
    a.init_field()
    a.step(3)
    ref = a.get_state()
    pinned = torch.empty(ref.shape, dtype=ref.dtype, pin_memory=True)
    nb = a.state_bytes()
    assert a.lib.psc_get_state(a._h, pinned.data_ptr(), nb) == 0
    assert torch.equal(pinned, ref.cpu())
    assert torch.equal(a.get_state(device="cpu"), ref.cpu())
    # an offset view of a larger pinned block (16-byte aligned, not 256)
    block = torch.empty(ref.numel() + 2, dtype=ref.dtype, pin_memory=True)
    view = block[2 // (ref.element_size() // 8):][:ref.numel()].view(ref.shape)
    assert a.lib.psc_get_state(a._h, view.data_ptr(), nb) == 0
    assert torch.equal(view, ref.cpu())
    # set_state from pinned memory, then steps, against set_state from the device
    b = B.Simulation(p, device=dev)
    assert b.lib.psc_set_state(b._h, pinned.data_ptr(), nb) == 0
    b.step(2)
    c = B.Simulation(p, device=dev)
    c.set_state(ref)
    c.step(2)
    assert torch.equal(b.get_state(), c.get_state())
    for s in (a, b, c):
        s.close()


def test_unsupported_and_short_workspace(dev):
    with pytest.raises(B.PscError):
        B.Simulation(B.Params(N=100), device=dev)


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_nonfinite_state_is_reported_unstable(dev, prec):
    # failure injected on the host: a non-finite mode in an otherwise valid state
    N = 16
    x = random_compact_state(N, 3)
    K = (N - 1) // 3
    x[1, K + 2, K - 1, 3] = np.nan
    p = B.Params(N=N, precision=prec, cfl=0.5)
    sim = B.Simulation(p, device=dev)
    sim.set_state(torch.from_numpy(x))
    with pytest.raises(B.PscError) as e:
        sim.stats()
    assert e.value.status == B.PSC_EUNSTABLE
    # a CFL-controlled step from it raises the device flag; the context stays usable
    sim.step(1)
    with pytest.raises(B.PscError) as e:
        sim.stats()
    assert e.value.status == B.PSC_EUNSTABLE
    ok = B.Simulation(B.Params(N=N, precision=prec), device=dev)
    ok.init_field()
    ok.step(1)
    rec, _, _ = ok.stats()
    assert np.isfinite(rec["K"])


# ---------------------------------------------------------------- pressure

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 32, 48, 96])
def test_pressure_matches_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec)
    sim = B.Simulation(p, device=dev)
    x = as_input(random_compact_state(N, 500 + N), prec)
    sim.set_state(torch.from_numpy(x).to(dev))
    got = sim.pressure().cpu().numpy().astype(np.complex128)
    f = compact_to_full(x, N)
    ref = full_to_compact(O.pressure_hat(f[:3], O.Grid(N))[None], N)[0]
    assert rel(got, ref) < TOL_RHS[prec]
    sim.close()


def _embed(small, n1, n2):
    """A compact state of an n1 grid as the same physical field on an n2 grid
    (unnormalised coefficients scale with N^3)."""
    k1, k2 = (n1 - 1) // 3, (n2 - 1) // 3
    big = np.zeros((small.shape[0], 2 * k2 + 1, 2 * k2 + 1, k2 + 1), dtype=small.dtype)
    big[:, k2 - k1:k2 + k1 + 1, k2 - k1:k2 + k1 + 1, :k1 + 1] = small * (n2 / n1) ** 3
    return big


@pytest.mark.parametrize("N,prec", [(512, B.FP32_MIXED), (512, B.FP64), (520, B.FP32_MIXED), (520, B.FP64),
                                    (1024, B.FP32_MIXED)],
                         ids=["512-fp32", "512-fp64", "520-fp32", "520-fp64", "1024-fp32"])
def test_pressure_of_taylor_green_at_full_size(dev, N, prec):
    """The Taylor-Green field has the closed-form pressure
    (cos 2x + cos 2y)(cos 2z + 2)/16 (pinned in the oracle at 16^3); the same
    field on the large grid must give the same coefficients, and nothing else."""
    n1 = 16
    g = O.Grid(n1)
    u = np.broadcast_to(np.sin(g.x) * np.cos(g.y) * np.cos(g.z), (n1,) * 3)
    v = np.broadcast_to(-np.cos(g.x) * np.sin(g.y) * np.cos(g.z), (n1,) * 3)
    uh = np.array([O.fwd(u), O.fwd(v), O.fwd(np.zeros((n1,) * 3))])
    small = full_to_compact(np.concatenate([uh, np.zeros((1,) + uh.shape[1:], complex)]), n1)
    ref_small = full_to_compact(O.pressure_hat(uh, g)[None], n1)
    p = B.Params(N=N, precision=prec)
    sim = B.Simulation(p, device=dev)
    big = _embed(small, n1, N)
    sim.set_state(torch.from_numpy(big.astype(np.complex64) if prec == B.FP32_MIXED else big).to(dev))
    got = sim.pressure().cpu().numpy().astype(np.complex128)
    ref = _embed(ref_small, n1, N)[0]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < (1e-6 if prec == B.FP32_MIXED else 1e-12) * scale
    sim.close()
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- convective form

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 24, 48, 96, 192, 256])
def test_convective_rhs_matches_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.013, Sc=0.7, beta=1.1, eps_inj=0.1, kF=2.0,
                 nonlinear_form=B.NL_CONVECTIVE)
    sim = B.Simulation(p, device=dev)
    x = as_input(random_compact_state(N, 700 + N, kpeak=4.0 if N < 128 else 8.0), prec)
    got = sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    ref = oracle_rhs(x, p)
    assert rel(got, ref) < TOL_RHS[prec]
    for f in range(4):
        assert rel(got[f], ref[f]) < 10 * TOL_RHS[prec]
    # and the rotational form on the same input agrees to the same tolerance
    rot = B.Simulation(B.Params(**{**p.__dict__, "nonlinear_form": B.NL_ROTATIONAL}), device=dev)
    other = rot.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    assert rel(got, other) < 2 * TOL_RHS[prec]
    sim.close()
    rot.close()


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_convective_trajectory_matches_oracle(dev, prec):
    N = 32
    p = B.Params(N=N, precision=prec, nu=0.02, dt=0.005, ic=B.IC_TAYLOR_GREEN_NOISE, seed=1,
                 nonlinear_form=B.NL_CONVECTIVE, cfl=0.5, record_every=5)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    sim.step(20)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    uh, ph, _, _, _ = O.run(oparams(p), 20, with_records=False)
    ref = full_to_compact(np.concatenate([uh, ph[None]]), N)
    assert rel(got, ref) < TOL_TRAJ[prec]
    sim.close()
