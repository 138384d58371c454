"""Schedule autotuner: per mesh shape, precision and device, choose the knobs
of a FIND plan by timing candidates on the device.

Knobs (none changes what is computed beyond rounding order; the tree shape
changes which Schur complements are formed, and Theorem 1 of the paper makes
the results independent of it):

* ``leaf``            leaf cluster size (flops grow with it; the number of
                      small, launch-bound problems shrinks);
* ``energy_group``    energies per concurrent stream group within a pass;
* ``gemm_small_max``  output size up to which a GEMM runs on 32x32 tiles
                      rather than 64x64 (tile shape per product; 0 = by
                      padding area, 4096 = all on 32x32);
* ``invert_smem``     bordered leaf systems up to this size are inverted in
                      shared memory.

Search: coordinate descent from the defaults (leaf, then tiles, then group,
then the leaf inversion), each candidate built as a plan and timed on a
sample of the request's energies (one untimed call, then the best of
``repeats`` timed calls, CUDA-synchronised).  Results are cached in a JSON
file keyed by (nx, ny, stencil, precision, batch, device name), so a shape is
tuned once per machine.
"""

from __future__ import annotations

import json
import os
import threading
import time

import numpy as np

DEFAULTS = {"leaf": 8, "energy_group": 8, "gemm_small_max": 0, "invert_smem": 0}
SPACE = [("leaf", (6, 8, 10, 12)),
         ("gemm_small_max", (32, 64, 4096)),  # 0 (default): by padding; 4096: all 32x32
         ("energy_group", (4, 8, 16, 32)),
         ("invert_smem", (0, 112))]


def default_cache_path():
    return os.environ.get("FIND_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "find_gb300", "tune.json"))


class Tuner:
    def __init__(self, device=0, cache_path=None, repeats=2, sample=None, budget_s=120.0):
        self.device = int(device)
        self.cache_path = cache_path or default_cache_path()
        self.repeats = int(repeats)
        self.sample = sample            # energies timed per candidate (None: the batch)
        self.budget_s = float(budget_s)  # stop searching after this much wall time
        self.lock = threading.Lock()
        self.cache = {}
        if os.path.exists(self.cache_path):
            try:
                with open(self.cache_path) as fh:
                    self.cache = json.load(fh)
            except (OSError, ValueError):
                self.cache = {}
        self.log = []

    # -- keys and persistence
    def _device_name(self):
        import torch
        return torch.cuda.get_device_name(self.device)

    def key(self, mesh, precision, batch):
        return f"{mesh.nx}x{mesh.ny}:{mesh.stencil}:{precision}:{batch}:{self._device_name()}"

    def _save(self):
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(self.cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    # -- measurement
    def _time(self, mesh, energies, precision, batch, params, V=None):
        import torch

        import paper_1104_0623_gb300 as F
        f = F.Find.from_mesh(mesh, V=V, device=self.device, max_batch=batch, precision=precision,
                             **params)
        try:
            E = torch.tensor(np.ascontiguousarray(energies), dtype=torch.complex128,
                             device=f"cuda:{self.device}")
            f.solve_lesser(E, bonds=False)
            torch.cuda.synchronize(self.device)
            best = float("inf")
            for _ in range(self.repeats):
                t = time.perf_counter()
                f.solve_lesser(E, bonds=False)
                torch.cuda.synchronize(self.device)
                best = min(best, time.perf_counter() - t)
        finally:
            f.close()
        return best

    def tune(self, mesh, energies, precision="mixed_ff", batch=None, V=None, force=False):
        """Best knobs for this mesh shape; measured once, then cached."""
        energies = np.asarray(energies, dtype=np.complex128)
        batch = int(batch or len(energies))
        key = self.key(mesh, precision, batch)
        with self.lock:
            if not force and key in self.cache:
                return dict(self.cache[key]["params"])
        n = min(len(energies), self.sample or batch)
        sample = energies[np.linspace(0, len(energies) - 1, n).astype(int)]
        t0 = time.perf_counter()
        best = dict(DEFAULTS)
        best_t = self._time(mesh, sample, precision, batch, best, V)
        tried = {tuple(sorted(best.items())): best_t}
        for name, values in SPACE:
            for v in values:
                if time.perf_counter() - t0 > self.budget_s:
                    break
                cand = dict(best, **{name: v})
                sig = tuple(sorted(cand.items()))
                if sig in tried:
                    continue
                tried[sig] = self._time(mesh, sample, precision, batch, cand, V)
                if tried[sig] < best_t:
                    best, best_t = cand, tried[sig]
        entry = {"params": best, "seconds_per_energy": best_t / n,
                 "default_seconds_per_energy": tried[tuple(sorted(DEFAULTS.items()))] / n,
                 "candidates": len(tried), "tuning_s": time.perf_counter() - t0}
        self.log.append((key, entry))
        with self.lock:
            self.cache[key] = entry
            self._save()
        return dict(best)


def tuned_find(mesh, energies, precision="mixed_ff", batch=None, tuner=None, V=None, device=0):
    """A Find handle built with the tuner's knobs for this mesh shape."""
    import paper_1104_0623_gb300 as F
    tuner = tuner or Tuner(device=device)
    params = tuner.tune(mesh, energies, precision, batch, V=V)
    return F.Find.from_mesh(mesh, V=V, device=device, precision=precision,
                            max_batch=int(batch or len(energies)), **params)
