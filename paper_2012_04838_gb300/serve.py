"""Continuous-batching simulation server on one GPU.

Requests (grid size N, steps, viscosity, Schmidt number, seed) arrive over time.
The server admits them in arrival order while their workspaces fit an HBM
budget, keeps every admitted run's spectral state resident, steps all active
runs together, streams each run's statistics records, and retires runs as
they finish, freeing their memory for waiting requests.

Two ways of stepping the active set: "graph" (the default) captures every
member's kernels into one CUDA graph per RK4 step, rebuilt when the set
changes; "persistent" steps it with one persistent launch per RK stage over a
device work table that is rewritten when runs join or leave, so nothing is
recaptured (FP32-mixed runs at the persistent sizes; on GB300 it has run at
about half the graph path's rate, its pass bodies being latency-bound at the
occupancy one kernel for every pass allows).  While a chunk of steps runs on
the GPU the host admits and initialises newly arrived runs.

Everything numeric happens in libpsc's kernels; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float        # seconds after the server starts
    N: int
    steps: int
    nu: float
    Sc: float
    seed: int
    precision: int = B.FP32_MIXED
    cfl: float = 0.5
    record_every: int = 10


@dataclasses.dataclass
class Result:
    rid: int
    N: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    records: list

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def nu_for_resolution(N: int, kmax_eta: float, eps: float = 0.1) -> float:
    """Viscosity giving k_max eta = kmax_eta with k_max = N/3 and eta = (nu^3/eps)^(1/4)."""
    eta = kmax_eta / (N / 3.0)
    return (eta ** 4 * eps) ** (1.0 / 3.0)


def poisson_requests(n: int, rate: float = 4.0, seed: int = 5, sizes=(64, 96, 128, 192, 256),
                     steps=(100, 2000), kmax_eta=(1.0, 2.0), Scs=(0.7, 1.0, 2.0)) -> list:
    """A seeded stream of requests with exponential inter-arrival times."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(sizes))
        out.append(Request(rid=i, arrival=t, N=N, steps=int(rng.integers(steps[0], steps[1] + 1)),
                           nu=nu_for_resolution(N, float(rng.uniform(*kmax_eta))),
                           Sc=float(rng.choice(Scs)), seed=int(rng.integers(1, 2 ** 31))))
    return out


def make_params(r: Request) -> B.Params:
    return B.Params(N=r.N, precision=r.precision, nu=r.nu, Sc=r.Sc, beta=1.0, kF=2.0, eps_inj=0.1,
                    cfl=r.cfl, seed=r.seed, ic=B.IC_SPECTRUM_K4, ic_energy=1.5,
                    record_every=r.record_every)


class Server:
    """Admit, batch, step and retire runs on one device.

    budget_bytes: HBM the runs' workspaces may occupy together.
    chunk: steps between scheduling decisions (and statistics records).
    records: "chunk" takes a record of every active run after every chunk (the
    stream of records a server returns); "final" only of each run when it ends."""

    def __init__(self, budget_bytes: float = 150e9, chunk: int = 50, device="cuda:0",
                 clock=time.perf_counter, sleep=time.sleep, records: str = "chunk", mode: str = "graph",
                 max_boxes: int = 1024, max_N: int | None = None):
        if records not in ("chunk", "final"):
            raise ValueError("records must be 'chunk' or 'final'")
        if mode not in ("graph", "persistent"):
            raise ValueError("mode must be 'graph' or 'persistent'")
        self.records = records
        self.mode = mode
        self.max_boxes = max_boxes
        self.max_N = max_N
        import torch
        self.torch = torch
        self.budget = budget_bytes
        self.chunk = chunk
        self.device = torch.device(device)
        self.clock = clock
        self.sleep = sleep
        self.stream = torch.cuda.Stream(self.device)

    def _persistent_ok(self, requests) -> bool:
        return all(r.precision == B.FP32_MIXED and r.N in B.PERSISTENT_SIZES for r in requests)

    def run(self, requests, on_record=None):
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        mode = self.mode
        if mode == "persistent" and not self._persistent_ok(pending):
            raise ValueError("persistent mode needs FP32-mixed runs at persistent sizes")
        active = []       # dicts: req, sim, left, records, admitted
        results = []
        used = 0
        batch = None
        dirty = True
        stats = dict(mode=mode, graph_builds=0, graph_build_s=0.0, table_updates=0, chunks=0,
                     grid_point_stages=0.0, peak_active=0, peak_bytes=0, records=0, step_s=0.0,
                     admit_s=0.0, record_s=0.0)
        if mode == "persistent":
            max_N = self.max_N or max(r.N for r in pending)
            max_N = min(n for n in B.PERSISTENT_SIZES if n >= max_N)
            batch = B.PersistentBatch([], max_boxes=self.max_boxes, max_N=max_N, device=self.device,
                                      stream=self.stream)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = self.clock()

        def admit(now):
            nonlocal used, dirty
            ta = self.clock()
            while pending and pending[0].arrival <= now:
                r = pending[0]
                p = make_params(r)
                need = B.workspace_size(p)
                if used + need > self.budget:
                    if not active:
                        raise RuntimeError(f"request {r.rid} needs {need} bytes, more than the budget")
                    break
                pending.pop(0)
                sim = B.Simulation(p, device=self.device, stream=torch.cuda.Stream(self.device))
                sim.init_field()
                active.append(dict(req=r, sim=sim, left=r.steps, records=[], admitted=now, bytes=need,
                                   joined=False))
                used += need
                dirty = True
            stats["admit_s"] += self.clock() - ta

        while pending or active:
            admit(self.clock() - t0)
            stats["peak_active"] = max(stats["peak_active"], len(active))
            stats["peak_bytes"] = max(stats["peak_bytes"], used)
            if not active:
                now = self.clock() - t0
                self.sleep(max(0.0, min(0.05, pending[0].arrival - now)))
                continue
            members = [a for a in active if a["left"] > 0]
            if dirty:
                tb = self.clock()
                if mode == "persistent":
                    batch.set_members([a["sim"] for a in members])
                    stats["table_updates"] += 1
                else:
                    if batch is not None:
                        batch.close()
                    batch = B.Batch([a["sim"] for a in members], stream=self.stream)
                    stats["graph_builds"] += 1
                stats["graph_build_s"] += self.clock() - tb
                for a in members:
                    a["joined"] = True
                dirty = False
            n = min(self.chunk, min(a["left"] for a in members))
            ev0.record(self.stream)
            batch.step(n)
            ev1.record(self.stream)
            # while the chunk runs: admit and initialise runs that have arrived
            # (they join at the next chunk)
            admit(self.clock() - t0)
            batch.synchronize()
            stats["step_s"] += ev0.elapsed_time(ev1) / 1000.0
            stats["chunks"] += 1
            finished = []
            tr = self.clock()
            for a in members:
                a["left"] -= n
                stats["grid_point_stages"] += 4.0 * n * a["req"].N ** 3
                if self.records == "chunk" or a["left"] == 0:
                    rec, E, Ep = a["sim"].stats()
                    rec["E"], rec["Ephi"] = E, Ep
                    a["records"].append(rec)
                    stats["records"] += 1
                    if on_record is not None:
                        on_record(a["req"].rid, rec)
                if a["left"] == 0:
                    finished.append(a)
            stats["record_s"] += self.clock() - tr
            if finished:
                done_t = self.clock() - t0
                # the batch refers to the members' memory: drop them from it first
                remaining = [a for a in active if a not in finished]
                if mode == "persistent":
                    batch.set_members([a["sim"] for a in remaining if a["joined"]])
                    stats["table_updates"] += 1
                elif batch is not None:
                    batch.close()
                    batch = None
                for a in finished:
                    results.append(Result(a["req"].rid, a["req"].N, a["req"].steps, a["req"].arrival,
                                          a["admitted"], done_t, a["records"]))
                    active.remove(a)
                    used -= a["bytes"]
                    a["sim"].close()
                    del a["sim"]
                dirty = True
                if pending:  # hand freed memory back for the next admissions
                    torch.cuda.empty_cache()
        if batch is not None:
            batch.close()
        wall = self.clock() - t0
        lat = np.array([r.latency for r in results])
        idle = max(0.0, wall - stats["step_s"] - stats["record_s"] - stats["admit_s"] - stats["graph_build_s"])
        summary = dict(requests=len(results), wall_s=wall,
                       p50_latency_s=float(np.percentile(lat, 50)) if len(lat) else math.nan,
                       p99_latency_s=float(np.percentile(lat, 99)) if len(lat) else math.nan,
                       grid_point_stages_per_s=stats["grid_point_stages"] / wall if wall > 0 else math.nan,
                       sims_per_hour=3600.0 * len(results) / wall if wall > 0 else math.nan,
                       step_busy_fraction=stats["step_s"] / wall if wall > 0 else math.nan,
                       other_s=idle, **stats)
        return sorted(results, key=lambda r: r.rid), summary
