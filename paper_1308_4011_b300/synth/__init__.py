"""Seeded synthetic-system generator (Python binding of ``synth.c``).

The paper evaluates on 13 Java systems (Table I) that are not available here;
these seeded systems stand in for them.  This module only generates inputs:
it holds none of the metric or move arithmetic, and both the CUDA library and
the CPU oracle consume what it produces.

A system is a set of int32 ids in CSR form (the paper's ``cls``/``dpnd``
arrays of Sec. IV.C): ``method_class[m]``, ``attr_class[a]``, the sorted
attribute accesses of each method (``acc_rowptr``/``acc_idx``) and its sorted
callees (``call_rowptr``/``call_idx``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libmmsynth.so")


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libmmsynth.so`` next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("n_classes", ctypes.c_int32), ("n_methods", ctypes.c_int32),
        ("n_attrs", ctypes.c_int32), ("max_class", ctypes.c_int32),
        ("zipf_s", ctypes.c_double), ("lambda_acc", ctypes.c_double),
        ("lambda_call", ctypes.c_double), ("p_loc", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class _Sys(ctypes.Structure):
    _fields_ = [
        ("n_classes", ctypes.c_int32), ("n_methods", ctypes.c_int32),
        ("n_attrs", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("n_acc", ctypes.c_int64), ("n_call", ctypes.c_int64),
        ("method_class", ctypes.POINTER(ctypes.c_int32)),
        ("attr_class", ctypes.POINTER(ctypes.c_int32)),
        ("acc_rowptr", ctypes.POINTER(ctypes.c_int64)),
        ("call_rowptr", ctypes.POINTER(ctypes.c_int64)),
        ("acc_idx", ctypes.POINTER(ctypes.c_int32)),
        ("call_idx", ctypes.POINTER(ctypes.c_int32)),
        ("class_size", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.synth_generate.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.POINTER(_Sys))]
        _lib.synth_generate.restype = ctypes.c_int
        _lib.synth_free.argtypes = [ctypes.POINTER(_Sys)]
        _lib.synth_free.restype = None
        _lib.synth_candidates.argtypes = [ctypes.POINTER(_Sys), ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_void_p]
        _lib.synth_candidates.restype = ctypes.c_int
        _lib.synth_logu_classes.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        _lib.synth_logu_classes.restype = ctypes.c_int32
        _lib.synth_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib.synth_u64.restype = ctypes.c_uint64
    return _lib


@dataclass
class System:
    """A system in CSR form; every array is a contiguous numpy array."""
    n_classes: int
    n_methods: int
    n_attrs: int
    method_class: np.ndarray      # int32 [n_methods]
    attr_class: np.ndarray        # int32 [n_attrs]
    acc_rowptr: np.ndarray        # int64 [n_methods+1]
    acc_idx: np.ndarray           # int32 [n_acc], each row strictly increasing
    call_rowptr: np.ndarray       # int64 [n_methods+1]
    call_idx: np.ndarray          # int32 [n_call], each row strictly increasing, no self
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n_acc(self) -> int:
        return int(self.acc_rowptr[-1])

    @property
    def n_call(self) -> int:
        return int(self.call_rowptr[-1])

    def acc(self, x: int) -> np.ndarray:
        return self.acc_idx[self.acc_rowptr[x]:self.acc_rowptr[x + 1]]

    def calls(self, x: int) -> np.ndarray:
        return self.call_idx[self.call_rowptr[x]:self.call_rowptr[x + 1]]


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def generate(n_classes: int, n_methods: int, n_attrs: int, *, max_class: int, seed: int,
             zipf_s: float = 1.2, lambda_acc: float = 3.0, lambda_call: float = 4.0,
             p_loc: float = 0.70, name: str = "") -> System:
    """Generate one seeded system (see the module docstring of ``synth.c``)."""
    lib = _load()
    p = _Params(n_classes, n_methods, n_attrs, max_class, zipf_s, lambda_acc, lambda_call, p_loc, seed)
    out = ctypes.POINTER(_Sys)()
    rc = lib.synth_generate(ctypes.byref(p), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"synth_generate failed (code {rc}) for {n_classes}/{n_methods}/{n_attrs} max={max_class}")
    try:
        s = out.contents
        sysm = System(
            n_classes=s.n_classes, n_methods=s.n_methods, n_attrs=s.n_attrs,
            method_class=_arr(s.method_class, s.n_methods, np.int32),
            attr_class=_arr(s.attr_class, s.n_attrs, np.int32),
            acc_rowptr=_arr(s.acc_rowptr, s.n_methods + 1, np.int64),
            acc_idx=_arr(s.acc_idx, s.n_acc, np.int32),
            call_rowptr=_arr(s.call_rowptr, s.n_methods + 1, np.int64),
            call_idx=_arr(s.call_idx, s.n_call, np.int32),
            name=name,
            params=dict(n_classes=n_classes, n_methods=n_methods, n_attrs=n_attrs, max_class=max_class,
                        seed=seed, zipf_s=zipf_s, lambda_acc=lambda_acc, lambda_call=lambda_call, p_loc=p_loc),
        )
    finally:
        lib.synth_free(out)
    return sysm


def candidates(system: System, n_extra: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Restricted destinations per method: classes it calls into or whose
    attributes it accesses (the R2/R3 destination sets of Sec. III.A), plus
    ``n_extra`` uniformly drawn other classes.  Returns (rowptr int64, dst int32),
    each row sorted, ``cls(m)`` never included."""
    lib = _load()
    s = _Sys(system.n_classes, system.n_methods, system.n_attrs, 0, system.n_acc, system.n_call,
             system.method_class.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             system.attr_class.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             system.acc_rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
             system.call_rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
             system.acc_idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             system.call_idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
             None)
    rowptr = np.zeros(system.n_methods + 1, dtype=np.int64)
    rc = lib.synth_candidates(ctypes.byref(s), n_extra, seed, rowptr.ctypes.data, None)
    if rc:
        raise MemoryError("synth_candidates")
    dst = np.zeros(max(int(rowptr[-1]), 1), dtype=np.int32)
    rc = lib.synth_candidates(ctypes.byref(s), n_extra, seed, rowptr.ctypes.data, dst.ctypes.data)
    if rc:
        raise MemoryError("synth_candidates")
    return rowptr, dst[: int(rowptr[-1])]


def u64(seed: int, stream: int, index: int) -> int:
    """The generator's raw counter draw (for edit streams and sampling)."""
    return int(_load().synth_u64(seed, stream, index))


def logu_classes(seed: int, lo: int = 100, hi: int = 20000) -> int:
    return int(_load().synth_logu_classes(seed, lo, hi))


# Named workloads.  Sizes, class-size caps and degree/locality parameters of
# the five workloads used throughout the tests and the benchmark.
TINY = dict(n_classes=200, n_methods=2000, n_attrs=1000, max_class=80, seed=0,
            zipf_s=1.2, lambda_acc=3.0, lambda_call=4.0, p_loc=0.70)
MEDIUM = dict(n_classes=5000, n_methods=60000, n_attrs=30000, max_class=400, seed=1,
              zipf_s=1.2, lambda_acc=4.0, lambda_call=6.0, p_loc=0.75)
LARGE = dict(n_classes=50000, n_methods=500000, n_attrs=250000, max_class=2000, seed=2,
             zipf_s=1.2, lambda_acc=4.0, lambda_call=6.0, p_loc=0.75)
LARGE_EXTRA_CANDIDATES = 64


def batched_params(seed: int) -> dict:
    """One system of the batched/served mixes: class count log-uniform in
    100..20,000, 12 methods and 6 attributes per class, tiny-system shape."""
    c = logu_classes(seed)
    return dict(n_classes=c, n_methods=12 * c, n_attrs=6 * c, max_class=80, seed=seed,
                zipf_s=1.2, lambda_acc=3.0, lambda_call=4.0, p_loc=0.70)


def named(name: str) -> System:
    table = {"tiny": TINY, "medium": MEDIUM, "large": LARGE}
    return generate(**table[name], name=name)
