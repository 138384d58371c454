"""ctypes binding of include/find.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are
passed as integers (a torch tensor's ``data_ptr()`` or a numpy array's
``ctypes.data``); complex arrays are interleaved (re, im) doubles.  The
library must have been built (``paper_1104_0623_gb300.build.build()``); a
missing library raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfind_gb300.so")

FIND_OK, FIND_EINVAL, FIND_ENOMEM, FIND_ESINGULAR, FIND_ETIMEOUT, FIND_ECUDA = range(6)
FIND_FP64 = 0
FIND_MIXED = 1
FIND_MIXED_FF = 2
FIND_FLAG_FULL_U = 1
FIND_FLAG_SYM_U = 2
FIND_FLAG_GRAPH = 4
FIND_FLAG_NO_TC = 8
FIND_FLAG_LU = 16
FIND_FLAG_LDL = 32

STATUS_NAMES = {0: "FIND_OK", 1: "FIND_EINVAL", 2: "FIND_ENOMEM", 3: "FIND_ESINGULAR",
                4: "FIND_ETIMEOUT", 5: "FIND_ECUDA"}

EXPORTED = ["find_create", "find_plan_info", "find_workspace_bytes", "find_solve_diag",
            "find_solve_diag_static", "find_solve_lesser", "find_profile", "find_profile_read",
            "find_destroy", "find_last_error", "find_peak_probe", "find_rgf_solve_lesser"]


class find_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("stencil", ctypes.c_int),
                ("t", ctypes.c_double), ("tp", ctypes.c_double),
                ("onsite_V", ctypes.c_void_p), ("onsite0", ctypes.c_double),
                ("leaf", ctypes.c_int), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("fp64_top_levels", ctypes.c_int),
                ("energy_group", ctypes.c_int), ("invert_smem", ctypes.c_int),
                ("sigma_c64_depth", ctypes.c_int), ("flags", ctypes.c_int),
                ("gemm_small_max", ctypes.c_int), ("tc_slices", ctypes.c_int),
                ("tc_slices_mixed", ctypes.c_int), ("tc_min", ctypes.c_int)]


class find_plan_stats(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int), ("n_leaves", ctypes.c_int),
                ("n_up_levels", ctypes.c_int), ("n_down_levels", ctypes.c_int),
                ("max_s", ctypes.c_int), ("max_b", ctypes.c_int), ("max_kn", ctypes.c_int),
                ("n_bonds", ctypes.c_int), ("flops_diag", ctypes.c_double),
                ("flops_lesser", ctypes.c_double), ("ur_bytes", ctypes.c_double),
                ("scratch_bytes", ctypes.c_double)]


class find_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def load():
    """Load libfind_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1104_0623_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.find_create.argtypes = [ctypes.POINTER(find_desc), ctypes.POINTER(vp)]
    lib.find_plan_info.argtypes = [vp, ctypes.POINTER(find_plan_stats)]
    lib.find_workspace_bytes.argtypes = [vp, ip, ip, ctypes.POINTER(dp)]
    lib.find_solve_diag.argtypes = [vp, vp, ip, vp, vp, vp, vp]
    lib.find_solve_diag_static.argtypes = [vp, vp, ip, vp, vp, vp, vp]
    lib.find_solve_lesser.argtypes = [vp, vp, ip, vp, vp, dp, dp, vp, ip, vp, vp, vp, vp]
    lib.find_profile.argtypes = [vp, ip]
    lib.find_profile_read.argtypes = [vp, ctypes.POINTER(find_kernel_stat), ip, ctypes.POINTER(ip)]
    lib.find_destroy.argtypes = [vp]
    lib.find_peak_probe.argtypes = [ip, dp, ip, ctypes.POINTER(dp)]
    lib.find_rgf_solve_lesser.argtypes = [vp, vp, ip, dp, dp, vp, vp, vp]
    lib.find_last_error.argtypes = [vp]
    lib.find_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "find_last_error":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class FindError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc, handle=None):
    if rc != FIND_OK:
        msg = load().find_last_error(handle).decode(errors="replace")
        raise FindError(rc, msg)


def find_create(desc: find_desc) -> int:
    h = ctypes.c_void_p()
    _check(load().find_create(ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def find_plan_info(handle: int) -> find_plan_stats:
    s = find_plan_stats()
    _check(load().find_plan_info(handle, ctypes.byref(s)), handle)
    return s


def find_workspace_bytes(handle: int, batch: int, lesser: bool) -> float:
    b = ctypes.c_double()
    _check(load().find_workspace_bytes(handle, batch, int(lesser), ctypes.byref(b)), handle)
    return b.value


def find_solve_diag(handle, E, nE, sigmaL, sigmaR, diagG, stream):
    _check(load().find_solve_diag(handle, E, nE, sigmaL, sigmaR, diagG, stream), handle)


def find_solve_diag_static(handle, E, nE, sigmaL, sigmaR, diagG, stream):
    """find_solve_diag with every device buffer in the library's fixed 64 MiB
    array: for callers that cannot allocate device memory (see find.h)."""
    _check(load().find_solve_diag_static(handle, E, nE, sigmaL, sigmaR, diagG, stream), handle)


def find_solve_lesser(handle, E, nE, sigmaL, sigmaR, fL, fR, sigma_lesser_diag, diag_per_energy,
                      diagG, diagGl, bond_current, stream):
    _check(load().find_solve_lesser(handle, E, nE, sigmaL, sigmaR, float(fL), float(fR),
                                    sigma_lesser_diag, int(diag_per_energy), diagG, diagGl,
                                    bond_current, stream), handle)


def find_rgf_solve_lesser(handle, E, nE, fL, fR, diagG, diagGl, stream):
    """diag G and diag G< by the recursive Green's function baseline (see find.h)."""
    _check(load().find_rgf_solve_lesser(handle, E, nE, float(fL), float(fR), diagG, diagGl, stream),
           handle)


def find_profile(handle: int, enable: bool) -> None:
    _check(load().find_profile(handle, int(enable)), handle)


def find_profile_read(handle: int):
    """Per-kernel-class dicts: name, launches, ms, flops, bytes."""
    arr = (find_kernel_stat * 32)()
    cnt = ctypes.c_int()
    _check(load().find_profile_read(handle, arr, 32, ctypes.byref(cnt)), handle)
    return [dict(name=arr[k].name.decode(), launches=arr[k].launches, ms=arr[k].ms,
                 flops=arr[k].flops, bytes=arr[k].bytes) for k in range(min(cnt.value, 32))]


def find_destroy(handle: int) -> None:
    _check(load().find_destroy(handle))


def find_peak_probe(kind: int, seconds: float, device: int = 0) -> float:
    """TFLOP/s of one arithmetic unit: 0 FFMA, 1 DFMA, 2 DMMA (see find.h)."""
    t = ctypes.c_double()
    _check(load().find_peak_probe(int(kind), float(seconds), int(device), ctypes.byref(t)))
    return t.value


def find_last_error(handle=None) -> str:
    return load().find_last_error(handle).decode(errors="replace")
