"""Scheduler logic of the serving loop with a host-only fake backend."""

import threading
import time

import numpy as np

import workloads as W
from paper_1104_0623_gb300.serve import Request, Server, mesh_key, summarize


class FakeBackend:
    def __init__(self, budget):
        self.budget = budget
        self.live = {}
        self.peak = 0
        self.closed = 0
        self.running = 0
        self.max_running = 0
        self.mu = threading.Lock()

    def new_stream(self):
        return None

    def make_plan(self, mesh, energies=None):
        return ("plan", mesh_key(mesh), mesh.nx * mesh.ny)

    def plan_bytes(self, plan):
        return 10.0 * plan[2]

    def solve(self, plan, energies, stream):
        with self.mu:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.live[plan[1]] = self.plan_bytes(plan)
            self.peak = max(self.peak, sum(self.live.values()))
        time.sleep(0.002 * len(energies))
        n = plan[2]
        G = np.outer(energies, np.arange(1, n + 1))
        with self.mu:
            self.running -= 1
        return G, 1j * G

    def free_bytes(self):
        return self.budget

    def close_plan(self, plan):
        with self.mu:
            self.live.pop(plan[1], None)
            self.closed += 1


def make_requests():
    meshes = [W.Mesh(4, 5, 5, seed=1), W.Mesh(6, 5, 5, seed=2), W.Mesh(8, 5, 5, seed=3)]
    reqs = []
    for k in range(9):
        m = meshes[k % 3]
        E = W.energy_grid(0.1, 3.0 + k, 5 + 3 * k)
        reqs.append(Request(k, 0.004 * k, m, E))
    return reqs


def test_results_latencies_and_admission():
    be = FakeBackend(budget=1000.0)
    srv = Server(be, slots=3, chunk=4, mem_budget=650.0)   # at most 2 of the 3 plans fit at once
    res = srv.run(make_requests())
    for r, req in zip(res, make_requests()):
        n = req.mesh.nx * req.mesh.ny
        assert np.array_equal(r.diagG, np.outer(req.energies, np.arange(1, n + 1)))
        assert r.done_s >= r.admit_s >= r.arrival_s - 1e-9
    assert srv.max_active <= 3
    assert be.max_running >= 2          # work of different requests overlapped
    assert be.peak <= 650.0             # never more plans resident than the budget
    assert be.closed >= 1               # an idle plan was evicted to admit another mesh
    s = summarize(res)
    assert s["requests"] == 9 and s["p99_s"] >= s["p50_s"] > 0
    srv.close()


class SlowPlanBackend(FakeBackend):
    """Plans take 0.2 s to build (as with autotuning); solves are timestamped."""

    def __init__(self, budget):
        super().__init__(budget)
        self.solves = []      # (start time, mesh key)
        self.builds = []      # (start, end, mesh key)

    def make_plan(self, mesh, energies=None):
        t = time.perf_counter()
        time.sleep(0.2)
        self.builds.append((t, time.perf_counter(), mesh_key(mesh)))
        return super().make_plan(mesh, energies)

    def solve(self, plan, energies, stream):
        with self.mu:
            self.solves.append((time.perf_counter(), plan[1]))
        return super().solve(plan, energies, stream)


def test_plans_are_built_without_stalling_running_requests():
    be = SlowPlanBackend(budget=1e9)
    srv = Server(be, slots=2, chunk=1)
    a = Request(0, 0.0, W.Mesh(4, 5, 5, seed=1), W.energy_grid(0.1, 3.0, 200))
    b = Request(1, 0.05, W.Mesh(6, 5, 5, seed=2), W.energy_grid(0.1, 3.0, 4))
    res = srv.run([a, b])
    srv.close()
    for r, req in zip(res, (a, b)):
        n = req.mesh.nx * req.mesh.ny
        assert np.array_equal(r.diagG, np.outer(req.energies, np.arange(1, n + 1)))
    # while the second mesh's plan was being built, the first request's
    # chunks kept running
    t0, t1, kb = next(x for x in be.builds if x[2] == mesh_key(b.mesh))
    during = [t for t, k in be.solves if k == mesh_key(a.mesh) and t0 < t < t1]
    assert len(during) >= 5
    assert len(be.builds) == 2   # each plan built once



def test_a_server_runs_a_second_stream_with_its_plans_cached():
    be = FakeBackend(budget=1e9)
    built = []
    make = be.make_plan
    be.make_plan = lambda mesh, energies=None: built.append(mesh_key(mesh)) or make(mesh, energies)
    srv = Server(be, slots=2, chunk=4)
    first = srv.run(make_requests())
    n_plans = len(built)
    second = srv.run(make_requests())
    assert n_plans == 3 and len(built) == 3   # the second stream reuses every plan
    for a, b in zip(first, second):
        assert np.array_equal(a.diagG, b.diagG)
    srv.close()
