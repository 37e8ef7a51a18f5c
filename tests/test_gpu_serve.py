"""Serving loop: runs admitted while others are on the GPU must produce the same
result in the mix as alone (the kernels are deterministic, so bit for bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2012_04838_gb300.binding")
S = pytest.importorskip("paper_2012_04838_gb300.serve")


def test_served_results_equal_alone_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [S.Request(0, 0.00, 32, 37, 0.02, 1.0, 7),
            S.Request(1, 0.00, 24, 23, 0.03, 0.7, 8, precision=B.FP64),
            S.Request(2, 0.05, 48, 41, 0.01, 2.0, 9),
            S.Request(3, 0.10, 16, 12, 0.05, 1.0, 10, precision=B.FP64, cfl=0.0),
            S.Request(4, 0.15, 32, 30, 0.02, 1.0, 11)]
    seen = []
    res, summ = S.Server(budget_bytes=2e9, chunk=10).run(reqs, on_record=lambda rid, r: seen.append(rid))
    assert summ["requests"] == len(reqs) and len(res) == len(reqs)
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] > 0
    assert set(seen) == {r.rid for r in reqs}
    for r, out in zip(reqs, res):
        p = S.make_params(r)
        alone = B.Simulation(p, device="cuda:0")
        alone.init_field()
        alone.step(r.steps)
        rec, E, Ep = alone.stats()
        last = out.records[-1]
        assert last["step"] == r.steps == rec["step"]
        for k in ("K", "eps", "phi_var", "chi", "t", "dt"):
            assert last[k] == rec[k], (r.rid, k)
        assert np.array_equal(last["E"], E) and np.array_equal(last["Ephi"], Ep)
        alone.close()


def test_admission_respects_the_budget():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [S.Request(i, 0.0, 32, 10, 0.02, 1.0, 20 + i) for i in range(6)]
    one = B.workspace_size(S.make_params(reqs[0]))
    res, summ = S.Server(budget_bytes=2.5 * one, chunk=5).run(reqs)
    assert summ["peak_active"] <= 2 and summ["peak_bytes"] <= 2.5 * one
    assert len(res) == 6


def test_served_results_equal_alone_runs_persistent_mode():
    """The persistent-kernel server (work table rewritten as runs join and
    leave): runs at 64^3 and 96^3, where that kernel is bit-identical to
    psc_step, end with the same records as alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [S.Request(0, 0.00, 64, 23, 0.02, 1.0, 7),
            S.Request(1, 0.00, 96, 17, 0.01, 0.7, 8),
            S.Request(2, 0.02, 64, 31, 0.015, 2.0, 9),
            S.Request(3, 0.05, 96, 12, 0.02, 1.0, 10, cfl=0.0),
            S.Request(4, 0.08, 64, 9, 0.02, 1.0, 11)]
    res, summ = S.Server(budget_bytes=8e9, chunk=5, mode="persistent").run(reqs)
    assert summ["mode"] == "persistent" and summ["graph_builds"] == 0 and summ["table_updates"] >= 2
    assert summ["requests"] == len(reqs)
    for r, out in zip(reqs, res):
        alone = B.Simulation(S.make_params(r), device="cuda:0")
        alone.init_field()
        alone.step(r.steps)
        rec, E, Ep = alone.stats()
        last = out.records[-1]
        assert last["step"] == r.steps == rec["step"]
        for k in ("K", "eps", "phi_var", "chi", "t", "dt"):
            assert last[k] == rec[k], (r.rid, k)
        assert np.array_equal(last["E"], E) and np.array_equal(last["Ephi"], Ep)
        alone.close()
