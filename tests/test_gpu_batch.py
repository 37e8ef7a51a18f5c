"""Ensemble stepping through one captured CUDA graph: every member must advance
exactly (bit for bit) as it does when stepped on its own."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")


def _members(dev):
    cfgs = [dict(N=16, precision=B.FP64, ic=B.IC_SPECTRUM_K4, seed=11, nu=0.02, dt=0.004),
            dict(N=24, precision=B.FP32_MIXED, ic=B.IC_SPECTRUM_K4, seed=12, nu=0.03, cfl=0.5, record_every=5),
            dict(N=32, precision=B.FP32_MIXED, ic=B.IC_TAYLOR_GREEN_NOISE, seed=13, nu=0.02, dt=0.005, Sc=0.7),
            dict(N=48, precision=B.FP64, ic=B.IC_SPECTRUM_K4, seed=14, nu=0.01, cfl=0.4, record_every=3),
            dict(N=64, precision=B.FP32_MIXED, ic=B.IC_SPECTRUM_K4, seed=15, nu=0.01, dt=0.002, Sc=2.0)]
    sims = []
    for c in cfgs:
        s = B.Simulation(B.Params(**c), device=dev, stream=torch.cuda.Stream(dev))
        s.init_field()
        sims.append(s)
    return sims


def test_batch_steps_match_individual_steps_bitwise():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    alone = _members(dev)
    mixed = _members(dev)
    for s in alone:
        s.step(13)
    b = B.Batch(mixed)
    b.step(6)
    b.step(7)
    b.synchronize()
    for a, m in zip(alone, mixed):
        assert torch.equal(a.get_state(), m.get_state())
        ta, na, da = a.time()
        tm, nm, dm = m.time()
        assert (ta, na, da) == (tm, nm, dm) and nm == 13
    # members remain usable on their own after batch steps
    for a, m in zip(alone, mixed):
        a.step(2)
        m.step(2)
        assert torch.equal(a.get_state(), m.get_state())
    b.close()


def test_batch_members_sharing_a_stream_and_duplicates():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    st = torch.cuda.Stream(dev)
    p = B.Params(N=16, ic=B.IC_SPECTRUM_K4, seed=3)
    s1 = B.Simulation(p, device=dev, stream=st)
    s2 = B.Simulation(B.Params(N=24, ic=B.IC_SPECTRUM_K4, seed=4), device=dev, stream=st)
    ref = B.Simulation(p, device=dev)
    for s in (s1, s2, ref):
        s.init_field()
    b = B.Batch([s1, s2])  # same stream: one branch, still exact
    b.step(4)
    b.synchronize()
    ref.step(4)
    assert torch.equal(s1.get_state(), ref.get_state())
    b.close()
    with pytest.raises(B.PscError):
        B.Batch([s1, s1])
