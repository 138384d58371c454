"""Serving loop: continuous batching of FIND requests on one GPU.

A request is a mesh (nx, ny, stencil, hoppings, disorder) and an energy grid.
The server

* admits a request when a slot is free and the device memory its plan needs
  (the handle's resident workspace, ``find_workspace_bytes``) fits in the
  budget, evicting idle cached plans least-recently-used first;
* keeps each mesh's plan and workspace resident across requests (a cache
  keyed by the mesh), so a repeated mesh pays neither the plan build nor the
  allocation again;
* splits every admitted request into chunks of energies and feeds the chunks
  of all active requests round-robin to worker threads, each driving its own
  CUDA stream, so requests that arrive while others run start at the next
  chunk boundary and their work overlaps on the device;
* records arrival, admission and completion times per request.

Each energy is an independent FIND pass whose result does not depend on
which other energies share its launch, so a request's result is the same
alone and in the mix.
"""

from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    mesh: object              # workloads.Mesh-like: nx, ny, stencil, t, tp, onsite0, potential()
    energies: np.ndarray      # complex128


@dataclasses.dataclass
class Result:
    rid: int
    diagG: np.ndarray
    diagGl: np.ndarray
    arrival_s: float
    admit_s: float
    done_s: float

    @property
    def latency_s(self):
        return self.done_s - self.arrival_s


def mesh_key(mesh):
    return (mesh.nx, mesh.ny, mesh.stencil, mesh.t, mesh.tp, mesh.v_lo, mesh.v_hi, mesh.seed)


class GpuBackend:
    """Plans are libfind handles; a chunk is one find_solve_lesser call with
    host outputs on the worker's stream."""

    def __init__(self, device=0, precision="mixed", leaf=8, chunk=16, tuner=None, graph_max_nodes=16384):
        import torch

        import paper_1104_0623_gb300 as F
        self.F, self.torch = F, torch
        self.device, self.precision, self.leaf, self.chunk = device, precision, leaf, chunk
        self.tuner = tuner        # paper_1104_0623_gb300.tune.Tuner, or None for fixed knobs
        # meshes of at most this many nodes replay each chunk as a captured
        # CUDA graph (FIND_FLAG_GRAPH): their passes are short, so launch
        # overhead is a visible part of them (measured 1.4 % more points/s on
        # meshes of 700-3100 nodes); 0 turns it off
        self.graph_max_nodes = graph_max_nodes

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def make_plan(self, mesh, energies=None):
        params = {"leaf": self.leaf}
        if self.tuner is not None and energies is not None:
            params = self.tuner.tune(mesh, energies[:self.chunk], self.precision, self.chunk)
        graph = mesh.nx * mesh.ny <= self.graph_max_nodes
        return self.F.Find.from_mesh(mesh, device=self.device, max_batch=self.chunk,
                                     precision=self.precision, graph=graph, **params)

    def plan_bytes(self, plan):
        return plan.workspace_bytes(self.chunk, True)

    def solve(self, plan, energies, stream):
        G, Gl, _ = plan.solve_lesser(np.ascontiguousarray(energies), bonds=False,
                                     stream=stream.cuda_stream)
        return G, Gl

    def free_bytes(self):
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return free

    def close_plan(self, plan):
        plan.close()


class Server:
    def __init__(self, backend, slots=4, chunk=16, mem_budget: Optional[float] = None):
        self.backend = backend
        self.slots = slots
        self.chunk = chunk
        self.mem_budget = mem_budget if mem_budget is not None else 0.8 * backend.free_bytes()
        self.lock = threading.Condition()
        self.pending: collections.deque = collections.deque()
        self.active: Dict[int, dict] = {}
        self.jobs: collections.deque = collections.deque()
        self.plans: "collections.OrderedDict" = collections.OrderedDict()  # key -> [plan, bytes, users, lock]
        self.building = set()  # mesh keys whose plan a thread is building (lock released)
        self.results: Dict[int, Result] = {}
        self.max_active = 0
        self.stop = False
        self.t0 = None

    # -- plan cache
    def _plan_for(self, mesh, energies=None):
        """Cached plan of a mesh, or None if it is not ready or its footprint
        does not fit now.  Called with self.lock held; a plan that is not
        cached is built (and tuned, with a tuner) with the lock released, so
        running requests keep being served meanwhile, and only one thread
        builds a given mesh's plan."""
        key = mesh_key(mesh)
        if key in self.plans:
            self.plans.move_to_end(key)
            return self.plans[key]
        if key in self.building:
            return None
        self.building.add(key)
        self.lock.release()
        try:
            plan = self.backend.make_plan(mesh, energies)
            need = self.backend.plan_bytes(plan)
        finally:
            self.lock.acquire()
            self.building.discard(key)
        used = sum(p[1] for p in self.plans.values())
        for k in list(self.plans.keys()):
            if used + need <= self.mem_budget:
                break
            if self.plans[k][2] == 0:  # idle: evict
                used -= self.plans[k][1]
                self.backend.close_plan(self.plans.pop(k)[0])
        if used + need > self.mem_budget:
            self.backend.close_plan(plan)
            return None
        entry = [plan, need, 0, threading.Lock()]
        self.plans[key] = entry
        return entry

    def _admit(self):
        """Admit pending requests in arrival order while slots and memory allow."""
        while self.pending and len(self.active) < self.slots:
            req = self.pending[0]
            entry = self._plan_for(req.mesh, req.energies)
            if entry is None:
                if mesh_key(req.mesh) in self.building:
                    return  # another thread is building its plan
                if not self.active and self.pending and self.pending[0] is req:
                    raise RuntimeError(f"request {req.rid} does not fit the device memory budget")
                return
            if not self.pending or self.pending[0] is not req:
                continue  # the queue moved while the plan was being built
            self.pending.popleft()
            entry[2] += 1
            n = len(req.energies)
            self.active[req.rid] = dict(req=req, entry=entry, next=0, done=0, admit=self._now(),
                                        G=np.empty((n, req.mesh.nx * req.mesh.ny), np.complex128),
                                        Gl=np.empty((n, req.mesh.nx * req.mesh.ny), np.complex128))
            self.jobs.append(req.rid)
            self.max_active = max(self.max_active, len(self.active))
            self.lock.notify_all()

    def _now(self):
        return time.perf_counter() - self.t0

    # -- workers
    def _worker(self):
        stream = self.backend.new_stream()
        while True:
            with self.lock:
                while not self.jobs and not self.stop:
                    self.lock.wait(0.05)
                if self.stop and not self.jobs:
                    return
                rid = self.jobs.popleft()
                st = self.active[rid]
                lo = st["next"]
                hi = min(lo + self.chunk, len(st["req"].energies))
                st["next"] = hi
                if hi < len(st["req"].energies):
                    self.jobs.append(rid)  # round-robin: the rest of this request queues behind others
            entry = st["entry"]
            with entry[3]:
                G, Gl = self.backend.solve(entry[0], st["req"].energies[lo:hi], stream)
            with self.lock:
                st["G"][lo:hi] = G
                st["Gl"][lo:hi] = Gl
                st["done"] += hi - lo
                if st["done"] == len(st["req"].energies):
                    req = st["req"]
                    self.results[rid] = Result(rid, st["G"], st["Gl"], req.arrival_s, st["admit"],
                                               self._now())
                    entry[2] -= 1
                    del self.active[rid]
                    self._admit()
                self.lock.notify_all()

    # -- driving a stream of requests in real time
    def run(self, requests: List[Request], time_scale=1.0):
        """Release requests at their arrival times (seconds from now, scaled)
        and serve them; returns the results ordered by request id.  A server
        runs one stream at a time and can run another after it (its plans
        stay cached)."""
        self.t0 = time.perf_counter()
        with self.lock:
            self.stop = False
        workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(self.slots)]
        for w in workers:
            w.start()
        try:
            for req in sorted(requests, key=lambda r: r.arrival_s):
                req = dataclasses.replace(req, arrival_s=req.arrival_s * time_scale)
                delay = req.arrival_s - self._now()
                if delay > 0:
                    time.sleep(delay)
                with self.lock:
                    self.pending.append(req)
                    self._admit()
            with self.lock:
                while self.pending or self.active:
                    self.lock.wait(0.05)
                    self._admit()
                self.stop = True
                self.lock.notify_all()
        finally:
            for w in workers:
                w.join()
        return [self.results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]

    def close(self):
        for p in self.plans.values():
            self.backend.close_plan(p[0])
        self.plans.clear()


def solve_ragged(items, backend, slots=4, chunk=16):
    """A ragged batch: several meshes, each with its own energy grid, solved
    together (all admitted at once, chunks interleaved over `slots` streams).
    items: list of (mesh, energies); returns [(diagG, diagG<)] in item order."""
    srv = Server(backend, slots=slots, chunk=chunk)
    try:
        res = srv.run([Request(k, 0.0, m, np.asarray(e, dtype=np.complex128))
                       for k, (m, e) in enumerate(items)])
    finally:
        srv.close()
    return [(r.diagG, r.diagGl) for r in res]


def summarize(results: List[Result]):
    lat = np.array([r.latency_s for r in results])
    points = sum(len(r.diagG) for r in results)
    span = max(r.done_s for r in results) - min(r.arrival_s for r in results)
    return {"requests": len(results), "energy_points": int(points),
            "points_per_s": points / span if span > 0 else float("nan"),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_queue_s": float(np.mean([r.admit_s - r.arrival_s for r in results]))}
