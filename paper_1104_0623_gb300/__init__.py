"""GB300 FIND: selected inversion of A = E I - H - Sigma on 2D meshes.

The compute runs in libfind_gb300.so (hand-written sm_103a CUDA behind the C
ABI of include/find.h).  This module only marshals arguments: it allocates
outputs with PyTorch (device memory) or numpy (host memory) and passes raw
pointers and the current CUDA stream.  There is no CPU fallback: if the
library is missing, importing the binding raises.

    f = Find(nx=40, ny=40, V=v)            # plan only, no GPU touched
    dG = f.solve_diag(E)                   # E: complex128 torch (cuda) or numpy
    dG, dGl, J = f.solve_lesser(E, fL=1.0, fR=0.0)
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (FIND_FP64, FIND_MIXED, FIND_MIXED_FF, FindError, find_create, find_destroy, find_last_error,  # noqa: F401
                   find_plan_info, find_profile, find_profile_read, find_rgf_solve_lesser,
                   find_solve_diag, find_solve_lesser, find_workspace_bytes)

__all__ = ["Find", "FindError", "find_create", "find_destroy", "find_last_error", "find_plan_info",
           "find_profile", "find_profile_read", "find_rgf_solve_lesser", "find_solve_diag",
           "find_solve_lesser", "find_workspace_bytes"]


def _ptr(x, dtype_name):
    """Raw data pointer of a contiguous torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.dtype.name != dtype_name:
            raise TypeError(f"expected a C-contiguous {dtype_name} array")
        return x.ctypes.data
    import torch
    want = {"complex128": torch.complex128, "float64": torch.float64}[dtype_name]
    if not isinstance(x, torch.Tensor) or x.dtype != want or not x.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype_name} tensor")
    return x.data_ptr()


class Find:
    """One mesh: plan built at construction, device workspace kept resident."""

    def __init__(self, nx, ny, stencil=5, t=1.0, tp=0.0, V=None, onsite0=None, leaf=8,
                 device=0, max_batch=0, precision="fp64", fp64_top_levels=2, energy_group=0,
                 invert_smem=0, sigma_c64_depth=0, full_u=False, gemm_small_max=0, sym_u=False,
                 graph=False, tensor_cores=True, tc_slices=0, tc_slices_mixed=0, tc_min=0,
                 ldl=None):
        _abi.load()
        self.nx, self.ny, self.stencil = int(nx), int(ny), int(stencil)
        self.n = self.nx * self.ny
        self.t, self.tp = float(t), float(tp)
        if onsite0 is None:
            onsite0 = 4.0 * t + (4.0 * tp if stencil == 9 else 0.0)
        self._V = None if V is None else np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
        if self._V is not None and self._V.size != self.n:
            raise ValueError("V must have nx*ny entries")
        self.device = int(device)
        prec = {"fp64": FIND_FP64, "mixed": FIND_MIXED, "mixed_ff": FIND_MIXED_FF}[precision]
        self.precision = precision
        d = _abi.find_desc(self.nx, self.ny, self.stencil, self.t, self.tp,
                           None if self._V is None else self._V.ctypes.data, float(onsite0),
                           int(leaf), prec, self.device, int(max_batch), int(fp64_top_levels),
                           int(energy_group), int(invert_smem), int(sigma_c64_depth),
                           (_abi.FIND_FLAG_FULL_U if full_u else 0) | (_abi.FIND_FLAG_SYM_U if sym_u else 0)
                           | (_abi.FIND_FLAG_GRAPH if graph else 0)
                           | (0 if tensor_cores else _abi.FIND_FLAG_NO_TC)
                           | {None: 0, True: _abi.FIND_FLAG_LDL, False: _abi.FIND_FLAG_LU}[ldl],
                           int(gemm_small_max), int(tc_slices), int(tc_slices_mixed), int(tc_min))
        self.handle = find_create(d)
        self.stats = find_plan_info(self.handle)
        self.n_bonds = self.stats.n_bonds

    @classmethod
    def from_mesh(cls, mesh, V=None, **kw):
        return cls(mesh.nx, mesh.ny, mesh.stencil, mesh.t, mesh.tp,
                   mesh.potential() if V is None else V, mesh.onsite0, **kw)

    def close(self):
        if getattr(self, "handle", None):
            find_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers
    def _stream(self, stream, nE=1):
        if stream is not None:
            return stream
        if nE == 0:  # the library returns before any device work
            return None
        import torch
        return torch.cuda.current_stream(self.device).cuda_stream

    def _out(self, like, shape, dtype):
        """Outputs live where the energies live: numpy, pinned host torch, or cuda."""
        if isinstance(like, np.ndarray):
            return np.empty(shape, dtype=dtype)
        import torch
        tdt = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        if like.device.type == "cpu":
            return torch.empty(shape, dtype=tdt, pin_memory=True)
        return torch.empty(shape, dtype=tdt, device=f"cuda:{self.device}")

    def solve_diag(self, E, sigmaL=None, sigmaR=None, stream=None, out=None):
        """diag(G) for every energy in E -> (nE, nx*ny) complex128."""
        nE = int(E.shape[0])
        out = self._out(E, (nE, self.n), np.complex128) if out is None else out
        find_solve_diag(self.handle, _ptr(E, "complex128"), nE, _ptr(sigmaL, "complex128"),
                        _ptr(sigmaR, "complex128"), _ptr(out, "complex128"), self._stream(stream, nE))
        return out

    def solve_lesser(self, E, fL=1.0, fR=0.0, sigmaL=None, sigmaR=None, sigma_lesser_diag=None,
                     bonds=True, stream=None, out=None):
        """diag(G), diag(G<) and (optionally) bond currents for every energy."""
        nE = int(E.shape[0])
        if out is None:
            dG = self._out(E, (nE, self.n), np.complex128)
            dGl = self._out(E, (nE, self.n), np.complex128)
            J = self._out(E, (nE, self.n_bonds), np.float64) if bonds else None
        else:
            dG, dGl, J = out
        per_e = 0
        if sigma_lesser_diag is not None:
            per_e = 1 if sigma_lesser_diag.ndim == 2 else 0
        find_solve_lesser(self.handle, _ptr(E, "complex128"), nE, _ptr(sigmaL, "complex128"),
                          _ptr(sigmaR, "complex128"), fL, fR, _ptr(sigma_lesser_diag, "complex128"),
                          per_e, _ptr(dG, "complex128"), _ptr(dGl, "complex128"),
                          _ptr(J, "float64"), self._stream(stream, nE))
        return dG, dGl, J

    def solve_rgf(self, E, fL=1.0, fR=0.0, stream=None, out=None):
        """diag(G), diag(G<) by the recursive Green's function baseline (FP64)."""
        nE = int(E.shape[0])
        if out is None:
            dG = self._out(E, (nE, self.n), np.complex128)
            dGl = self._out(E, (nE, self.n), np.complex128)
        else:
            dG, dGl = out
        find_rgf_solve_lesser(self.handle, _ptr(E, "complex128"), nE, fL, fR, _ptr(dG, "complex128"),
                              _ptr(dGl, "complex128"), self._stream(stream, nE))
        return dG, dGl

    def profile(self, enable=True):
        find_profile(self.handle, enable)

    def profile_read(self):
        return find_profile_read(self.handle)

    def workspace_bytes(self, batch, lesser=True):
        return find_workspace_bytes(self.handle, batch, lesser)


_ = ctypes  # the binding is ctypes-only
