"""Full-size checks at 1024^3 FP32-mixed, in the launch configuration the
benchmark times.  The oracle cannot transform a 1024^3 field, so the checks use
(a) a sparse state whose right-hand side the oracle sums triad by triad, and
(b) properties of the initial condition that hold at any size."""
import numpy as np
import pytest

from oracle import psc_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")

N = 1024
K = (N - 1) // 3


@pytest.fixture(scope="module")
def sim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    p = B.Params(N=N, precision=B.FP32_MIXED, nu=3.341e-4, Sc=1.0, beta=1.0, eps_inj=0.1, kF=2.0,
                 cfl=0.5, ic=B.IC_SPECTRUM_K4, seed=3, ic_energy=1.5, record_every=10)
    if free < B.workspace_size(p) + 16e9:
        pytest.skip("not enough device memory for the 1024^3 case")
    s = B.Simulation(p, device="cuda:0")
    yield s
    s.close()


def _sparse_modes(seed, Nn=N):
    Kn = (Nn - 1) // 3
    rng = np.random.default_rng(seed)
    ks = [(1, 0, 1), (0, 2, -1), (2, 1, 0), (1, -1, 2), (3, 2, -2), (5, -4, 1), (Kn, -Kn, 7),
          (Kn - 3, Kn, -Kn), (Kn * 3 // 5, -Kn * 4 // 9, Kn // 4), (0, 1, 1), (Kn // 3, Kn, 0), (2, 0, 0)]
    modes = {}
    for k in ks:
        v = (rng.standard_normal(4) + 1j * rng.standard_normal(4)) * float(Nn) ** 3 * 0.05
        modes[k] = v
        if k[0] == 0:
            modes[(0, -k[1], -k[2])] = np.conj(v)
    return modes


def _sparse_check(s, Nn, prec, seed):
    Kn = (Nn - 1) // 3
    modes = _sparse_modes(seed, Nn)
    dev = torch.device("cuda:0")
    cdt = torch.complex64 if prec == B.FP32_MIXED else torch.complex128
    x = torch.zeros(B.compact_shape(Nn), dtype=cdt, device=dev)
    rounded = {}
    for (kx, ky, kz), v in modes.items():
        vv = v.astype(np.complex64) if prec == B.FP32_MIXED else v
        rounded[(kx, ky, kz)] = vv.astype(np.complex128)
        x[:, kz + Kn, ky + Kn, kx] = torch.from_numpy(vv).to(dev)
    out = s.rhs(x)
    ref = O.rhs_sparse_triads(rounded, Nn, O.Params(N=Nn, nu=s.p.nu, Sc=s.p.Sc, beta=s.p.beta,
                                                    eps_inj=s.p.eps_inj, kF=s.p.kF))
    scale = max(np.abs(v).max() for v in ref.values())
    mask = torch.zeros(B.compact_shape(Nn)[1:], dtype=torch.bool, device=dev)
    got, want = [], []
    for (kx, ky, kz), v in ref.items():
        got.append(out[:, kz + Kn, ky + Kn, kx].cpu().numpy().astype(np.complex128))
        want.append(v)
        mask[kz + Kn, ky + Kn, kx] = True
    got, want = np.array(got), np.array(want)
    tol = 2e-6 if prec == B.FP32_MIXED else 1e-13
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
    assert np.abs(got - want).max() < tol * scale
    # every other mode holds only round-off spread by the transforms: no single
    # element's error may exceed tol times the norm of the exact output (an
    # element's error is at most the L2 error of the whole output; the L2 sum
    # over the ~10^9 zero modes of a sparse state is the dense tests' concern)
    out[:, mask] = 0
    rest = float(out.abs().max())
    assert rest < tol * np.linalg.norm(want), (rest / np.linalg.norm(want), rest / scale)


def test_fullsize_rhs_on_sparse_state_matches_triad_sums(sim):
    _sparse_check(sim, N, B.FP32_MIXED, 1)


@pytest.mark.parametrize("form", [B.NL_ROTATIONAL, B.NL_CONVECTIVE], ids=["rotational", "convective"])
@pytest.mark.parametrize("prec", [B.FP32_MIXED, B.FP64], ids=["fp32", "fp64"])
def test_512_rhs_on_sparse_state_matches_triad_sums(prec, form):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = B.Params(N=512, precision=prec, nu=8.419e-4, beta=1.0, eps_inj=0.1, kF=2.0, nonlinear_form=form)
    s = B.Simulation(p, device="cuda:0")
    try:
        _sparse_check(s, 512, prec, 2)
    finally:
        s.close()


def test_fullsize_convective_rhs_on_sparse_state_matches_triad_sums():
    """The convective form (u, nine gradients, 12 y-stage streams) at 1024^3:
    after projection it equals the rotational triad sums."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = B.Params(N=N, precision=B.FP32_MIXED, nu=3.341e-4, beta=1.0, eps_inj=0.1, kF=2.0,
                 nonlinear_form=B.NL_CONVECTIVE)
    free, _ = torch.cuda.mem_get_info()
    if free < B.workspace_size(p) + 16e9:
        pytest.skip("not enough device memory for the 1024^3 case")
    s = B.Simulation(p, device="cuda:0")
    try:
        _sparse_check(s, N, B.FP32_MIXED, 4)
    finally:
        s.close()
        torch.cuda.empty_cache()


def test_fullsize_initial_condition_properties(sim):
    sim.init_field()
    rec, E, Ep = sim.stats()
    assert abs(rec["K"] - 1.5) < 1e-6 * 1.5
    assert abs(E.sum() - rec["K"]) < 1e-9
    assert abs(rec["K_phys"] - rec["K"]) < 1e-5 * rec["K"]
    assert abs(rec["eps_phys"] - rec["eps"]) < 1e-5 * rec["eps"]
    tgt = O.target_shell_energy(len(E), O.IC_SPECTRUM_K4, 1.0, 2.0)
    tgt = tgt * 1.5 / tgt.sum()
    big = tgt > 1e-8 * tgt.max()
    assert np.allclose(E[big], tgt[big], rtol=1e-5)
    assert np.abs(Ep).max() == 0.0
    # Gaussian velocity-gradient statistics of the random-phase IC (section 3.1)
    for i in range(3):
        assert abs(rec["skew"][i]) < 0.1 and abs(rec["flat"][i] - 3.0) < 0.3
    st = sim.get_state()
    dev = st.device
    kx = torch.arange(0, K + 1, device=dev, dtype=torch.float32).view(1, 1, -1)
    ky = torch.arange(-K, K + 1, device=dev, dtype=torch.float32).view(1, -1, 1)
    kz = ky.view(-1, 1, 1)
    div = kx * st[0] + ky * st[1] + kz * st[2]
    mag = torch.sqrt(kx * kx + ky * ky + kz * kz) * (st[0].abs() + st[1].abs() + st[2].abs())
    assert float(div.abs().max()) <= 1e-5 * float(mag.max())
    # sampled modes: same direction as the oracle's raw draw, a positive factor apart
    for k in [(1, 2, 3), (0, 4, -1), (7, -3, 2), (17, 0, -9)]:
        raw = _oracle_raw_draw(3, *k)
        g = st[:3, k[2] + K, k[1] + K, k[0]].cpu().numpy().astype(np.complex128)
        r = g / raw
        assert np.allclose(r.imag, 0, atol=1e-5 * abs(r[0])) and r.real.min() > 0
        assert np.allclose(r.real, r.real[0], rtol=1e-5)
    del st


def _oracle_raw_draw(seed, kx, ky, kz):
    """The oracle's projected raw draw of one canonical mode (its IC recipe)."""
    key = np.array([O.mode_key(kx, ky, kz)], dtype=np.uint64)
    z = []
    for c in range(3):
        u1 = O.uniform01(seed, key * np.uint64(8) + np.uint64(2 * c))
        u2 = O.uniform01(seed, key * np.uint64(8) + np.uint64(2 * c + 1))
        r = np.sqrt(-2.0 * np.log(u1))
        z.append((r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2))[0])
    z = np.array(z)
    k = np.array([kx, ky, kz], dtype=np.float64)
    return z - k * (k @ z) / (k @ k)


def test_fullsize_steps_conserve_budget(sim):
    # two forced steps from the IC: energy budget dK/dt = P_inj - eps closes to
    # the time-integration error (semi-discrete identity at any N)
    sim.init_field()
    r0, _, _ = sim.stats()
    sim.step(2)
    r1, _, _ = sim.stats()
    dt = r1["t"] - r0["t"]
    assert dt > 0 and r1["step"] == 2
    dK = r1["K"] - r0["K"]
    src = 0.5 * ((r0["P_inj"] - r0["eps"]) + (r1["P_inj"] - r1["eps"])) * dt
    assert abs(dK - src) < 0.05 * abs(r0["eps"]) * dt + 1e-6
    assert abs(r0["cfl"] - 0.5) < 1e-5


def test_xpass_tma_wait_runs_out_and_reports_timeout(monkeypatch):
    """The failure path of the X pass's bounded TMA waits, without a GPU fault:
    with PSC_XPASS_STALL_TEST=1 at creation, CTA 0 asks its first staged row's
    mbarrier for 16 transaction bytes more than its copies bring (every copy
    still lands), so that wait runs out after 1 ms; the row group stops, the
    simulation reports PSC_ETIMEOUT at its next statistics call, and a fresh
    simulation afterwards steps and reports normally."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = B.Params(N=N, precision=B.FP32_MIXED, nu=3.341e-4, Sc=1.0, beta=1.0, eps_inj=0.1, kF=2.0,
                 dt=2e-4, ic=B.IC_SPECTRUM_K4, seed=5, ic_energy=1.5)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < B.workspace_size(p) + 16e9:
        pytest.skip("not enough device memory for the 1024^3 case")
    monkeypatch.setenv("PSC_XPASS_STALL_TEST", "1")
    s = B.Simulation(p, device="cuda:0")
    monkeypatch.delenv("PSC_XPASS_STALL_TEST")
    s.init_field()
    s.step(1)
    with pytest.raises(B.PscError) as e:
        s.stats()
    assert e.value.status == B.PSC_ETIMEOUT
    s.close()
    del s
    torch.cuda.empty_cache()
    s = B.Simulation(p, device="cuda:0")
    s.init_field()
    s.step(1)
    rec, _, _ = s.stats()
    assert rec["step"] == 1 and rec["K"] > 0
    s.close()
    torch.cuda.empty_cache()
