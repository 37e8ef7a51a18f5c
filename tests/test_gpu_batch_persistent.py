"""Ensembles stepped by the persistent kernel (one launch per RK stage over a
device work table): every member must advance as it does when stepped on its
own with psc_step, whatever the mix of sizes, forcing, integrator and CFL
control, and members may join and leave between steps.

The persistent kernel runs the same pass bodies as the ordinary kernels,
compiled into one kernel; at some grid sizes (32, 48, 128) the compiler
rounds a few operations differently there, so states agree to FP32 rounding
(measured: 3e-8 of the largest coefficient after one step, 8e-8 after nine)
and are bit-identical at the others (64, 96, 192, 256)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")

CFGS = [
    dict(N=32, ic=B.IC_SPECTRUM_K4, seed=21, nu=0.03, cfl=0.5, record_every=5),
    dict(N=48, ic=B.IC_TAYLOR_GREEN_NOISE, seed=22, nu=0.02, dt=0.004, Sc=0.7),
    dict(N=64, ic=B.IC_SPECTRUM_K4, seed=23, nu=0.01, cfl=0.4, record_every=3, Sc=2.0),
    dict(N=96, ic=B.IC_SPECTRUM_K4, seed=24, nu=0.008, dt=0.002, forcing=B.FORCE_HOLD_ENERGY),
    dict(N=64, ic=B.IC_SPECTRUM_K4, seed=25, nu=0.01, dt=0.003, integrator=B.INTEG_RK4, scalar_on=0),
    dict(N=128, ic=B.IC_PAPER_EQ9, seed=26, nu=0.005, cfl=0.5, record_every=4, forcing=B.FORCE_NONE),
]
BIG = [dict(N=192, ic=B.IC_SPECTRUM_K4, seed=27, nu=0.004, cfl=0.5, record_every=5),
       dict(N=256, ic=B.IC_SPECTRUM_K4, seed=28, nu=0.003, dt=0.001, Sc=0.7)]


def _sim(c, dev):
    s = B.Simulation(B.Params(precision=B.FP32_MIXED, **c), device=dev)
    s.init_field()
    return s


BITWISE = (64, 96, 192, 256)


def _same(a, m):
    x, y = a.get_state(), m.get_state()
    if a.p.N in BITWISE:
        assert torch.equal(x, y), a.p.N
    else:
        assert float((x - y).abs().max()) <= 1e-6 * float(x.abs().max()), a.p.N
    (ta, na, da), (tm, nm, dm) = a.time(), m.time()
    assert na == nm and abs(ta - tm) <= 1e-6 * abs(ta) and abs(da - dm) <= 1e-6 * abs(da)


@pytest.fixture()
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_persistent_batch_matches_individual_steps(dev):
    alone = [_sim(c, dev) for c in CFGS]
    mixed = [_sim(c, dev) for c in CFGS]
    for s in alone:
        s.step(9)
    b = B.PersistentBatch(mixed, max_boxes=16, max_N=128, device=dev)
    assert b.info()["mode"] == B.BATCH_PERSISTENT and b.info()["grid"] >= 152
    b.step(4)
    b.step(5)
    b.synchronize()
    assert b.info()["launches"] == 4 * 9
    for a, m in zip(alone, mixed):
        _same(a, m)
        assert m.time()[1] == 9
    # members stay usable on their own, and records agree
    for a, m in zip(alone, mixed):
        a.step(2)
        m.step(2)
        _same(a, m)
        ra, ea, pa = a.stats()
        rm, em, pm = m.stats()
        assert abs(ra["K"] - rm["K"]) <= 1e-6 * ra["K"] and abs(ra["eps"] - rm["eps"]) <= 1e-6 * ra["eps"]
        if a.p.N in BITWISE:
            assert ra == rm and (ea == em).all() and (pa == pm).all()
    b.close()


def test_persistent_batch_members_join_and_leave_without_recapture(dev):
    alone = {i: _sim(c, dev) for i, c in enumerate(CFGS[:4])}
    mixed = {i: _sim(c, dev) for i, c in enumerate(CFGS[:4])}
    b = B.PersistentBatch([mixed[0], mixed[1]], max_boxes=4, max_N=128, device=dev)
    b.step(3)
    for i in (0, 1):
        alone[i].step(3)
    b.set_members([mixed[1], mixed[2], mixed[3]])  # 0 leaves, 2 and 3 join
    b.step(4)
    for i in (1, 2, 3):
        alone[i].step(4)
    b.set_members([])  # an empty table steps nothing
    b.step(2)
    b.set_members([mixed[0], mixed[3]])
    b.step(2)
    for i in (0, 3):
        alone[i].step(2)
    b.synchronize()
    for i in range(4):
        _same(alone[i], mixed[i])
    with pytest.raises(B.PscError):
        b.set_members([mixed[0]] * 5)  # more than max_boxes
    b.close()


def test_persistent_batch_large_boxes(dev):
    alone = [_sim(c, dev) for c in BIG + CFGS[:2]]
    mixed = [_sim(c, dev) for c in BIG + CFGS[:2]]
    for s in alone:
        s.step(3)
    b = B.PersistentBatch(mixed, max_boxes=8, max_N=256, device=dev)
    b.step(3)
    b.synchronize()
    for a, m in zip(alone, mixed):
        _same(a, m)
    b.close()


def test_persistent_batch_refuses_members_it_cannot_run(dev):
    ok = _sim(CFGS[0], dev)
    for bad in (B.Params(N=32, precision=B.FP64), B.Params(N=32, precision=B.FP32_MIXED, dealias=B.DEALIAS_PHASE_SHIFT),
                B.Params(N=32, precision=B.FP32_MIXED, nonlinear_form=B.NL_CONVECTIVE),
                B.Params(N=16, precision=B.FP32_MIXED)):
        s = B.Simulation(bad, device=dev)
        with pytest.raises(B.PscError):
            B.PersistentBatch([ok, s], max_boxes=4, max_N=128, device=dev)
        s.close()
    big = _sim(BIG[0], dev)
    with pytest.raises(B.PscError):  # N above max_N
        B.PersistentBatch([big], max_boxes=4, max_N=128, device=dev)


def test_persistent_batch_wait_runs_out_and_reports_timeout(dev, monkeypatch):
    """The failure path of the kernel's bounded waits, without a GPU fault: with
    PSC_BATCH_STALL_TEST=1 one dependency of stage 1 is never met (a counter
    nothing completes), its wait runs out after 50 ms, the launch is abandoned,
    and the member reports PSC_ETIMEOUT at its next statistics call.  The
    context stays usable: a fresh batch afterwards steps correctly."""
    monkeypatch.setenv("PSC_BATCH_STALL_TEST", "1")
    s = _sim(CFGS[2], dev)
    b = B.PersistentBatch([s], max_boxes=2, max_N=128, device=dev)
    monkeypatch.delenv("PSC_BATCH_STALL_TEST")
    b.step(1)
    b.synchronize()
    with pytest.raises(B.PscError) as e:
        s.stats()
    assert e.value.status == B.PSC_ETIMEOUT
    b.close()
    s.close()
    a, m = _sim(CFGS[2], dev), _sim(CFGS[2], dev)
    a.step(2)
    b2 = B.PersistentBatch([m], max_boxes=2, max_N=128, device=dev)
    b2.step(2)
    b2.synchronize()
    _same(a, m)
    m.stats()  # no error
    b2.close()
