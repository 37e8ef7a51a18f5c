"""Phase-shift dealiasing (section 2.3) on the GPU vs the FP64 oracle, through
the C ABI.

The retained set is the sphere 9|k|^2 < 2 N^2, stored in the cube of half-width
K = the largest k with 9 k^2 < 2 N^2; every product is formed on the grid and
on the grid shifted by half a cell and the two transforms are averaged.
Tolerances are those of the 2/3-rule path: one right-hand side 1e-13 (FP64) and
2e-6 (FP32-mixed) relative L2, 20-step trajectories 1e-11 and 1e-4."""
import numpy as np
import pytest

from oracle import psc_oracle as O
from tests.psc_inputs import compact_to_full, full_to_compact, random_compact_state
from tests.sparse_states import check_sparse_rhs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2012_04838_gb300.binding")

PS = B.DEALIAS_PHASE_SHIFT
TOL_RHS = {B.FP64: 1e-13, B.FP32_MIXED: 2e-6}
TOL_TRAJ = {B.FP64: 1e-11, B.FP32_MIXED: 1e-4}
PREC = [B.FP64, B.FP32_MIXED]
PNAME = {B.FP64: "fp64", B.FP32_MIXED: "fp32"}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def Ks(N):
    return B.retained_halfwidth(N, PS)


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


def oracle_rhs(x, p):
    g = O.Grid(p.N, O.DEALIAS_PHASE_SHIFT)
    f = compact_to_full(x, p.N)
    ru, rp = O.rhs_nonlinear(f[:3], f[3], g, oparams(p))
    return full_to_compact(np.array(list(ru) + [rp]), p.N, Ks(p.N))


def state_of(uh, ph, N):
    return full_to_compact(np.concatenate([uh, ph[None]]), N, Ks(N))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load()
    return torch.device("cuda:0")


def gpu_rhs(dev, p, x):
    sim = B.Simulation(p, device=dev)
    try:
        return sim.rhs(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    finally:
        sim.close()


# ---------------------------------------------------------------- layout

def test_layout_is_the_spheres_cube(dev):
    for N in (8, 16, 32, 64, 256):
        K, ks = Ks(N), O.sphere_halfwidth(N)
        assert 9 * ks * ks < 2 * N * N <= 9 * (ks + 1) * (ks + 1)
        # the sphere's own half-width, or one more so that a kx row holds an
        # even number of values (the planes added lie outside the sphere)
        assert K == ks or (K == ks + 1 and ks % 2 == 0 and 2 * K + 1 <= N)
        assert (K + 1) % 2 == 0 or 2 * K + 3 > N
        p = B.Params(N=N, precision=B.FP32_MIXED, dealias=PS)
        sim = B.Simulation(p, device=dev)
        assert sim.get_state().shape == (4, 2 * K + 1, 2 * K + 1, K + 1)
        sim.close()


# ---------------------------------------------------------------- right-hand side

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96])
def test_phase_shift_rhs_matches_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.013, Sc=0.7, beta=1.1, eps_inj=0.1, kF=2.0, dealias=PS)
    x = as_input(random_compact_state(N, 300 + N, K=Ks(N), sphere=True), prec)
    got = gpu_rhs(dev, p, x)
    ref = oracle_rhs(x, p)
    assert rel(got, ref) < TOL_RHS[prec]
    for f in range(4):
        assert rel(got[f], ref[f]) < 10 * TOL_RHS[prec]
    # nothing outside the sphere
    K = Ks(N)
    k = np.arange(-K, K + 1)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + np.arange(K + 1)[None, None, :] ** 2
    assert np.abs(got[:, 9 * k2 >= 2 * N * N]).max(initial=0.0) == 0.0


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [128, 192, 256])
def test_phase_shift_rhs_matches_oracle_large(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.002, beta=1.0, dealias=PS)
    x = as_input(random_compact_state(N, 17 + N, kpeak=8.0, K=Ks(N), sphere=True), prec)
    assert rel(gpu_rhs(dev, p, x), oracle_rhs(x, p)) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 48, 128])
def test_phase_shift_convective_rhs_matches_oracle(dev, N, prec):
    p = B.Params(N=N, precision=prec, nu=0.01, beta=0.9, dealias=PS, nonlinear_form=B.NL_CONVECTIVE)
    x = as_input(random_compact_state(N, 41 + N, K=Ks(N), sphere=True), prec)
    assert rel(gpu_rhs(dev, p, x), oracle_rhs(x, p)) < TOL_RHS[prec]


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N", [16, 32, 48])
def test_phase_shift_agrees_with_the_two_thirds_rule_where_both_are_exact(dev, N, prec):
    """A state on the 2/3 cube inside the sphere: both rules give the exact
    product on the modes they both keep (an alias that wraps in one direction
    cancels in the shifted average; one that wraps in two or three lands
    outside both sets), so the two GPU paths agree there."""
    K3, K = (N - 1) // 3, Ks(N)
    x3 = as_input(random_compact_state(N, 900 + N, K=K3, sphere=True), prec)
    x = np.zeros((4, 2 * K + 1, 2 * K + 1, K + 1), dtype=np.complex128)
    x[:, K - K3:K + K3 + 1, K - K3:K + K3 + 1, :K3 + 1] = x3
    kw = dict(N=N, precision=prec, nu=0.01, beta=1.0)
    got = gpu_rhs(dev, B.Params(dealias=PS, **kw), x)
    got3 = gpu_rhs(dev, B.Params(**kw), x3)
    k = np.arange(-K3, K3 + 1)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + np.arange(K3 + 1)[None, None, :] ** 2
    both = 9 * k2 < 2 * N * N
    inner = got[:, K - K3:K + K3 + 1, K - K3:K + K3 + 1, :K3 + 1]
    assert rel(inner[:, both], got3[:, both]) < 10 * TOL_RHS[prec]
    # and the phase-shift result itself is the oracle's
    assert rel(got, oracle_rhs(x, B.Params(dealias=PS, **kw))) < TOL_RHS[prec]


# ---------------------------------------------------------------- initial condition

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N,ic", [(16, B.IC_SPECTRUM_K4), (32, B.IC_TAYLOR_GREEN_NOISE), (64, B.IC_PAPER_EQ9)])
def test_phase_shift_initial_condition_matches_oracle(dev, N, ic, prec):
    p = B.Params(N=N, precision=prec, ic=ic, seed=5 + N, ic_energy=1.5, ic_noise_frac=0.01, dealias=PS)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    sim.close()
    g = O.Grid(N, O.DEALIAS_PHASE_SHIFT)
    uh, ph = O.init_field(g, oparams(p))
    assert rel(got, state_of(uh, ph, N)) < (1e-13 if prec == B.FP64 else 1e-6)


# ---------------------------------------------------------------- trajectories and records

@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
@pytest.mark.parametrize("N,integ,form", [(32, B.INTEG_IFRK4, B.NL_ROTATIONAL), (24, B.INTEG_RK4, B.NL_ROTATIONAL),
                                          (32, B.INTEG_IFRK4, B.NL_CONVECTIVE)])
def test_phase_shift_20_steps_match_oracle(dev, N, integ, form, prec):
    p = B.Params(N=N, precision=prec, integrator=integ, nu=0.02, dt=0.005, ic=B.IC_TAYLOR_GREEN_NOISE,
                 seed=1, dealias=PS, nonlinear_form=form)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    sim.step(20)
    got = sim.get_state().cpu().numpy().astype(np.complex128)
    tt, nstep, _ = sim.time()
    sim.close()
    uh, ph, _, t, _ = O.run(oparams(p), 20, with_records=False)
    ref = state_of(uh, ph, N)
    assert rel(got[:3], ref[:3]) < TOL_TRAJ[prec]
    assert rel(got[3], ref[3]) < TOL_TRAJ[prec]
    assert nstep == 20 and abs(tt - t) < 1e-12


@pytest.mark.parametrize("prec", PREC, ids=PNAME.get)
def test_phase_shift_records_match_oracle(dev, prec):
    """A CFL-controlled forced run with records: Table 1 quantities, the
    gradient moments and the shell spectra (shells 0 .. K+1 of the sphere)."""
    N = 32
    p = B.Params(N=N, precision=prec, nu=0.01, Sc=0.7, cfl=0.5, record_every=5, ic=B.IC_SPECTRUM_K4,
                 seed=2, ic_energy=1.5, dealias=PS)
    sim = B.Simulation(p, device=dev)
    sim.init_field()
    got = []
    for n in range(0, 16, 5):
        if n:
            sim.step(5)
        got.append(sim.stats())
    sim.close()
    uh, _, recs, _, _ = O.run(oparams(p), 15, with_records=True)
    assert len(recs) == len(got) == 4
    assert len(got[0][1]) == O.num_shells(N, O.DEALIAS_PHASE_SHIFT) == O.sphere_halfwidth(N) + 2
    tol = 1e-10 if prec == B.FP64 else 2e-4
    keys = ("K", "K_phys", "eps", "eps_phys", "chi", "chi_phys", "phi_var", "umax", "dt", "A", "E_forced")
    scale = {k: max(abs(r[k]) for r in recs) for k in keys}
    # the oracle's end-of-run record keeps the last step's dt; the C ABI's
    # record at a reset step gives the dt that step will use (Eq. 10 at the
    # final state)
    recs[-1]["dt"] = O.cfl_dt(uh, O.Grid(N, O.DEALIAS_PHASE_SHIFT), p.cfl)
    for (rec, E, Ep), ref in zip(got, recs):
        assert rec["step"] == ref["step"]
        for k in keys:
            assert abs(rec[k] - ref[k]) <= tol * abs(ref[k]) + 1e-12 * scale[k], (ref["step"], k, rec[k], ref[k])
        assert np.allclose(E, ref["E"], rtol=tol, atol=tol * ref["E"].max())
        if ref["Ephi"].max() > 0:
            assert np.allclose(Ep, ref["Ephi"], rtol=tol, atol=tol * ref["Ephi"].max())
        sk = 1e-8 if prec == B.FP64 else 2e-3
        assert np.allclose(rec["skew"], ref["skew"], rtol=sk, atol=sk)
        assert np.allclose(rec["flat"], ref["flat"], rtol=sk, atol=sk)


# ---------------------------------------------------------------- refusals

def test_phase_shift_refusals(dev):
    with pytest.raises(B.PscError) as e:
        B.Simulation(B.Params(N=520, precision=B.FP32_MIXED, dealias=PS, nonlinear_form=B.NL_CONVECTIVE),
                     device=dev)
    assert e.value.status == B.PSC_EUNSUPPORTED_N
    with pytest.raises(B.PscError) as e:
        B.Simulation(B.Params(N=32, dealias=2), device=dev)
    assert e.value.status == B.PSC_EINVAL
    sim = B.Simulation(B.Params(N=32, dealias=PS), device=dev)
    sim.init_field()
    with pytest.raises(B.PscError) as e:
        sim.pressure()
    assert e.value.status == B.PSC_EINVAL
    sim.close()


# ---------------------------------------------------------------- full size

@pytest.mark.parametrize("N,prec,form", [(512, B.FP32_MIXED, B.NL_ROTATIONAL), (512, B.FP64, B.NL_ROTATIONAL),
                                         (512, B.FP32_MIXED, B.NL_CONVECTIVE), (1024, B.FP32_MIXED, B.NL_ROTATIONAL)],
                         ids=["512-fp32", "512-fp64", "512-fp32-convective", "1024-fp32"])
def test_phase_shift_full_size_rhs_on_sparse_state_matches_triad_sums(dev, N, prec, form):
    """512^3 and 1024^3 (the 16-values-per-thread X pass over the sphere's
    cube): a sparse state at the sphere's edge against the oracle's triad sums
    on the sphere (the convective form equals them after projection)."""
    p = B.Params(N=N, precision=prec, nu=8e-4, beta=1.0, eps_inj=0.1, kF=2.0, dealias=PS, nonlinear_form=form)
    free, _ = torch.cuda.mem_get_info()
    if free < B.workspace_size(p) + 16e9:
        pytest.skip("not enough device memory")
    sim = B.Simulation(p, device=dev)
    try:
        check_sparse_rhs(torch, B, sim, 11 + N)
    finally:
        sim.close()
        torch.cuda.empty_cache()
