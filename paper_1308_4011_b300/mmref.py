"""Python binding of the mmref C ABI (``include/mmref.h``): argument
marshalling only.  Every step of the path runs in the CUDA library
``libmmref.so``; there is no CPU fallback -- importing this module without the
built library raises.

Device memory and streams come from PyTorch: device inputs/outputs are CUDA
tensors (passed by ``data_ptr()``), the stream is
``torch.cuda.current_stream().cuda_stream`` unless one is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmmref.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"mmref: {LIB_PATH} is missing; build it with `python -m paper_1308_4011_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ENOTFOUND, MM_EEXIST, MM_ETIMEOUT, MM_EBUDGET = range(8)
PTR_HOST, PTR_DEVICE = 0, 1
LCOM_CK, LCOM_HS, CBO = 1, 2, 4
# default criteria: LCOM only (both forms), improve source and target (Table I's mode)
DEFAULT_MASK = LCOM_CK | LCOM_HS
DEFAULT_MIN_IMPROVED = 2

EXPORTED = ("mm_load_system", "mm_set_stream", "mm_compute_metrics", "mm_evaluate_moves", "mm_suggest_moves",
            "mm_system_info_get", "mm_free_system", "mm_last_error", "mm_status_string", "mm_abi_version",
            "mm_launch_count", "mm_suggest_moves_noalloc", "mm_batch_create", "mm_batch_set_tile",
            "mm_batch_autotune", "mm_batch_run", "mm_batch_suggestions", "mm_batch_free", "mm_apply_edit",
            "mm_export_system", "mm_server_create", "mm_server_add_system", "mm_server_run", "mm_server_stats_get",
            "mm_server_snapshot", "mm_server_free", "mm_selftest_bounded_wait", "mm_last_eval_ms",
            "mm_export_metrics", "mm_similarity", "mm_suggest_r1", "mm_apply_sequence",
            "mm_suggest_r3", "mm_selftest_stall_scans", "mm_metric_variants", "mm_rank_classes",
            "mm_batch_config_get", "mm_stage_candidates")

CLASS_METRICS_DTYPE = np.dtype([("n_methods", "<i4"), ("n_attrs", "<i4"), ("P", "<i8"), ("Q", "<i8"),
                                ("S", "<i8"), ("lcom_ck", "<i8"), ("hs_num", "<i8"), ("hs_den", "<i8"),
                                ("cbo", "<i4"), ("reserved", "<i4")])
METHOD_METRICS_DTYPE = np.dtype([("fan_in", "<i4"), ("fan_out", "<i4"), ("own", "<i4"), ("q", "<i4")])
MOVE_EVAL_DTYPE = np.dtype([("s", "<i4"), ("t", "<u2"), ("dcbo_src", "<i2"), ("dcbo_dst", "<i2"),
                            ("n_improved", "<u2"), ("n_worsened", "<u2"), ("flags", "<u2")])
MOVE_DTYPE = np.dtype([("m", "<i4"), ("d", "<i4"), ("n_improved", "<i4"), ("d_lcom_ck_sum", "<i4"),
                       ("d_cbo_sum", "<i4"), ("reserved", "<i4")])
assert CLASS_METRICS_DTYPE.itemsize == 64 and MOVE_EVAL_DTYPE.itemsize == 16 and MOVE_DTYPE.itemsize == 24


class _Desc(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("n_methods", ctypes.c_int32), ("n_attrs", ctypes.c_int32),
                ("ptr_kind", ctypes.c_int32), ("n_acc", ctypes.c_int64), ("n_call", ctypes.c_int64),
                ("method_class", ctypes.c_void_p), ("attr_class", ctypes.c_void_p),
                ("acc_rowptr", ctypes.c_void_p), ("acc_idx", ctypes.c_void_p),
                ("call_rowptr", ctypes.c_void_p), ("call_idx", ctypes.c_void_p),
                ("cbo_attrs", ctypes.c_int32), ("flags", ctypes.c_int32)]


LOAD_PACKED_COUPLING, LOAD_BITSET_COUPLING = 1, 2
class _Crit(ctypes.Structure):
    _fields_ = [("metric_mask", ctypes.c_uint32), ("min_improved", ctypes.c_int32)]


class _Cands(ctypes.Structure):
    _fields_ = [("rowptr", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("n_cand", ctypes.c_int64),
                ("ptr_kind", ctypes.c_int32), ("flags", ctypes.c_int32)]


class _SimInfo(ctypes.Structure):
    _fields_ = [("n_values", ctypes.c_int64), ("n_cooccurrences", ctypes.c_int64), ("n_high", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("average", ctypes.c_double), ("max_union", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("n_methods", ctypes.c_int32), ("n_attrs", ctypes.c_int32),
                ("cbo_attrs", ctypes.c_int32), ("n_acc", ctypes.c_int64), ("n_call", ctypes.c_int64),
                ("n_class_edges", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


_vp = ctypes.c_void_p
_lib.mm_load_system.argtypes = [ctypes.POINTER(_Desc), _vp, ctypes.POINTER(_vp)]
_lib.mm_set_stream.argtypes = [_vp, _vp]
_lib.mm_compute_metrics.argtypes = [_vp, _vp, _vp, ctypes.c_int32]
_lib.mm_export_metrics.argtypes = [_vp, _vp, _vp, ctypes.c_int32]
_lib.mm_similarity.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_SimInfo)]
_lib.mm_similarity.restype = ctypes.c_int
_lib.mm_suggest_r1.argtypes = [_vp, ctypes.POINTER(_Crit), ctypes.c_int32, _vp, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_SimInfo)]
_lib.mm_suggest_r1.restype = ctypes.c_int
_lib.mm_export_metrics.restype = ctypes.c_int
_lib.mm_evaluate_moves.argtypes = [_vp, ctypes.POINTER(_Crit), ctypes.POINTER(_Cands), _vp, _vp, ctypes.c_int32]
_lib.mm_suggest_moves.argtypes = [_vp, ctypes.POINTER(_Crit), ctypes.POINTER(_Cands), ctypes.c_int32, _vp,
                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
_lib.mm_system_info_get.argtypes = [_vp, ctypes.POINTER(_Info)]
_lib.mm_last_eval_ms.argtypes = [_vp, ctypes.POINTER(ctypes.c_float)]
_lib.mm_last_eval_ms.restype = ctypes.c_int
_lib.mm_suggest_moves_noalloc.argtypes = [_vp, ctypes.POINTER(_Crit), ctypes.POINTER(_Cands), ctypes.c_int32, _vp,
                                          ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
_lib.mm_suggest_moves_noalloc.restype = ctypes.c_int
_lib.mm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_Crit), ctypes.c_int64, _vp,
                                 ctypes.POINTER(_vp)]
_lib.mm_batch_set_tile.argtypes = [_vp, ctypes.c_int32]
_lib.mm_batch_autotune.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
_lib.mm_batch_run.argtypes = [_vp, _vp, _vp]
_lib.mm_batch_suggestions.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int64)]
_lib.mm_stage_candidates.argtypes = [_vp, ctypes.POINTER(_Cands)]
_lib.mm_stage_candidates.restype = ctypes.c_int
_lib.mm_batch_config_get.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
_lib.mm_batch_config_get.restype = ctypes.c_int
_lib.mm_batch_free.argtypes = [_vp]
_lib.mm_batch_free.restype = None
for _n in ("mm_batch_create", "mm_batch_set_tile", "mm_batch_autotune", "mm_batch_run", "mm_batch_suggestions"):
    getattr(_lib, _n).restype = ctypes.c_int
class _Edit(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("m", ctypes.c_int32), ("target", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib.mm_apply_edit.argtypes = [_vp, ctypes.POINTER(_Edit)]
_lib.mm_apply_edit.restype = ctypes.c_int
_lib.mm_export_system.argtypes = [_vp] + [_vp] * 6
_lib.mm_apply_sequence.argtypes = [_vp, ctypes.POINTER(_Crit), ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_int64)]
_lib.mm_apply_sequence.restype = ctypes.c_int
R3_DTYPE = np.dtype([("m", "<i4"), ("d", "<i4"), ("fan_in", "<i4"), ("fan_out", "<i4"), ("dcbo_src", "<i4"),
                     ("dcbo_dst", "<i4")])
_lib.mm_suggest_r3.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
_lib.mm_suggest_r3.restype = ctypes.c_int
APPLIED_DTYPE = np.dtype([("round", "<i4"), ("m", "<i4"), ("from", "<i4"), ("to", "<i4")])
_lib.mm_export_system.restype = ctypes.c_int
_lib.mm_selftest_stall_scans.argtypes = [_vp, ctypes.c_int32]
_lib.mm_selftest_stall_scans.restype = ctypes.c_int
VARIANTS_DTYPE = np.dtype([("P_all", "<i8"), ("Q_all", "<i8"), ("lcom_ck_all", "<i8"), ("lcom_pq", "<i8"),
                           ("lcom_pq_all", "<i8"), ("cbo_out", "<i4"), ("cbo_in", "<i4"), ("cbo_bi", "<i4"),
                           ("reserved", "<i4")])
assert VARIANTS_DTYPE.itemsize == 56
RANK_LCOM_CK, RANK_LCOM_PQ, RANK_LCOM_CK_ALL, RANK_LCOM_PQ_ALL, RANK_CBO, RANK_CBO_IN, RANK_CBO_BI = range(1, 8)
_lib.mm_metric_variants.argtypes = [_vp, _vp, _vp, ctypes.c_int32]
_lib.mm_metric_variants.restype = ctypes.c_int
_lib.mm_rank_classes.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int32]
_lib.mm_rank_classes.restype = ctypes.c_int
EDIT_ADD_ACCESS, EDIT_REMOVE_ACCESS, EDIT_ADD_CALL, EDIT_REMOVE_CALL, EDIT_MOVE = 1, 2, 3, 4, 5
NOALLOC_MAX_METHODS = 1048576
NOALLOC_MAX_KEPT = 65536
_lib.mm_free_system.argtypes = [_vp]
_lib.mm_free_system.restype = None
_lib.mm_last_error.restype = ctypes.c_char_p
_lib.mm_status_string.argtypes = [ctypes.c_int]
_lib.mm_status_string.restype = ctypes.c_char_p
_lib.mm_abi_version.restype = ctypes.c_int32
_lib.mm_launch_count.restype = ctypes.c_int64
for _n in ("mm_load_system", "mm_set_stream", "mm_compute_metrics", "mm_evaluate_moves", "mm_suggest_moves",
           "mm_system_info_get"):
    getattr(_lib, _n).restype = ctypes.c_int


class MMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.mm_status_string(status).decode()}: {msg}")
        self.status = status


def _check(st: int):
    if st != MM_OK:
        raise MMError(st, _lib.mm_last_error().decode())


def abi_version() -> int:
    return int(_lib.mm_abi_version())


def selftest_bounded_wait() -> int:
    """mm_selftest_bounded_wait: the status the host reads after a device-side
    wait that cannot be satisfied ran out (MM_ETIMEOUT when it works)."""
    return int(_lib.mm_selftest_bounded_wait())

def selftest_stall_scans(sys: "System", n: int):
    """mm_selftest_stall_scans: the next n multi-tile scans of calls on sys run
    out of their bounded wait (results stay exact; the next synchronising call
    reports MM_ETIMEOUT)."""
    _check(_lib.mm_selftest_stall_scans(sys.handle, int(n)))


def launch_count() -> int:
    """Kernels launched by libmmref.so in this process so far."""
    return int(_lib.mm_launch_count())


def _ptr(a):
    """Address of a numpy array or torch tensor (None for None / empty)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() if a.numel() else None
    return a.ctypes.data if a.size else None


def _stream_handle(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _kind(x) -> int:
    if hasattr(x, "is_cuda"):
        return PTR_DEVICE if x.is_cuda else PTR_HOST
    return PTR_HOST


class System:
    """A loaded system (owns device memory until ``free()``)."""

    def __init__(self, handle, n_classes, n_methods, n_attrs, keepalive):
        self._h = ctypes.c_void_p(handle)
        self.n_classes, self.n_methods, self.n_attrs = n_classes, n_methods, n_attrs
        self._keep = keepalive

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.mm_free_system(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        inf = _Info()
        _check(_lib.mm_system_info_get(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _Info._fields_}

    def last_eval_ms(self) -> float:
        """mm_last_eval_ms: GPU time of the last evaluation kernel on this handle."""
        v = ctypes.c_float()
        _check(_lib.mm_last_eval_ms(self._h, ctypes.byref(v)))
        return float(v.value)

    def set_stream(self, stream):
        _check(_lib.mm_set_stream(self._h, _stream_handle(stream)))

    @property
    def n_candidates_full(self) -> int:
        return self.n_methods * (self.n_classes - 1)


def load_system(n_classes, method_class, attr_class, acc_rowptr, acc_idx, call_rowptr, call_idx, *,
                cbo_attrs: bool = True, stream=None, flags: int = 0) -> System:
    """mm_load_system.  Arrays are either all numpy (host) or all CUDA tensors;
    flags: 0 or LOAD_PACKED_COUPLING / LOAD_BITSET_COUPLING."""
    arrs = (method_class, attr_class, acc_rowptr, acc_idx, call_rowptr, call_idx)
    kinds = {_kind(a) for a in arrs}
    if len(kinds) != 1:
        raise ValueError("load_system: all arrays must be host (numpy) or all device (CUDA tensors)")
    kind = kinds.pop()
    if kind == PTR_HOST:
        arrs = tuple(np.ascontiguousarray(a, dtype=dt) for a, dt in
                     zip(arrs, (np.int32, np.int32, np.int64, np.int32, np.int64, np.int32)))
    n_methods = int(arrs[0].shape[0])
    d = _Desc(int(n_classes), n_methods, int(arrs[1].shape[0]), kind, int(arrs[3].shape[0]), int(arrs[5].shape[0]),
              _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]), _ptr(arrs[4]), _ptr(arrs[5]),
              1 if cbo_attrs else 0, int(flags))
    h = ctypes.c_void_p()
    _check(_lib.mm_load_system(ctypes.byref(d), _stream_handle(stream), ctypes.byref(h)))
    return System(h.value, int(n_classes), n_methods, int(arrs[1].shape[0]), arrs)


def load_synth(system, *, cbo_attrs: bool = True, device: bool = False, stream=None, flags: int = 0) -> System:
    """Load a ``synth.System``; with device=True the arrays are first moved to
    CUDA tensors (the inputs-resident-in-HBM form)."""
    arrs = (system.method_class, system.attr_class, system.acc_rowptr, system.acc_idx, system.call_rowptr,
            system.call_idx)
    if device:
        import torch
        arrs = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)
    return load_system(system.n_classes, *arrs, cbo_attrs=cbo_attrs, stream=stream, flags=flags)


def compute_metrics(sys: System, out_class=None, out_method=None):
    """mm_compute_metrics.  out_* are optional buffers: numpy arrays of
    CLASS_METRICS_DTYPE / METHOD_METRICS_DTYPE, or CUDA uint8 tensors of
    64*n_classes / 16*n_methods bytes.  Pass the string "host" to get new
    numpy arrays back."""
    if isinstance(out_class, str):
        out_class = np.zeros(sys.n_classes, dtype=CLASS_METRICS_DTYPE)
    if isinstance(out_method, str):
        out_method = np.zeros(sys.n_methods, dtype=METHOD_METRICS_DTYPE)
    outs = [o for o in (out_class, out_method) if o is not None]
    kind = _kind(outs[0]) if outs else PTR_HOST
    if any(_kind(o) != kind for o in outs):
        raise ValueError("compute_metrics: outputs must be both host or both device")
    _check(_lib.mm_compute_metrics(sys.handle, _ptr(out_class), _ptr(out_method), kind))
    return out_class, out_method


def export_metrics(sys: System, out_class="host", out_method="host"):
    """mm_export_metrics: the system's current metrics, not recomputed (same
    buffers as compute_metrics)."""
    if isinstance(out_class, str):
        out_class = np.zeros(sys.n_classes, dtype=CLASS_METRICS_DTYPE)
    if isinstance(out_method, str):
        out_method = np.zeros(sys.n_methods, dtype=METHOD_METRICS_DTYPE)
    outs = [o for o in (out_class, out_method) if o is not None]
    kind = _kind(outs[0]) if outs else PTR_HOST
    _check(_lib.mm_export_metrics(sys.handle, _ptr(out_class), _ptr(out_method), kind))
    return out_class, out_method


def _sim_info(inf) -> dict:
    return {f: getattr(inf, f) for f, _ in _SimInfo._fields_ if f != "reserved"}


def similarity_info(sys: System) -> dict:
    """mm_similarity with no outputs: computes the similarity values of the
    current state on the device and returns only the info dict."""
    inf = _SimInfo()
    _check(_lib.mm_similarity(sys.handle, None, None, None, None, 0, PTR_HOST, ctypes.byref(inf)))
    return _sim_info(inf)


def similarity(sys: System, cap=None):
    """mm_similarity: every similarity value (x < y, i, u) as host arrays (up
    to cap of them; all by default), and the info dict."""
    inf = _SimInfo()
    _check(_lib.mm_similarity(sys.handle, None, None, None, None, 0, PTR_HOST, ctypes.byref(inf)))
    n = inf.n_values if cap is None else min(int(cap), inf.n_values)
    out = [np.zeros(max(n, 1), dtype=np.int32) for _ in range(4)]
    _check(_lib.mm_similarity(sys.handle, *[a.ctypes.data for a in out], n, PTR_HOST, ctypes.byref(inf)))
    return tuple(a[:n] for a in out), _sim_info(inf)


def suggest_r1(sys: System, k: int, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED, out=None):
    """mm_suggest_r1: (top-k moves, n_kept, n_methods_with_kept, info dict)."""
    crit = _Crit(mask, min_improved)
    if out is None:
        out = np.zeros(max(k, 0), dtype=MOVE_DTYPE)
    nk, nm = ctypes.c_int64(), ctypes.c_int64()
    inf = _SimInfo()
    _check(_lib.mm_suggest_r1(sys.handle, ctypes.byref(crit), int(k), _ptr(out), _kind(out), ctypes.byref(nk),
                              ctypes.byref(nm), ctypes.byref(inf)))
    n = min(int(k), int(nk.value))
    return (out[:n] if _kind(out) == PTR_HOST else out), int(nk.value), int(nm.value), _sim_info(inf)


CANDS_UNCHANGED = 1


def _cands(cand_rowptr, cand_dst, flags=0):
    if cand_rowptr is None:
        return None, None
    kind = _kind(cand_rowptr)
    if kind == PTR_HOST:
        cand_rowptr = np.ascontiguousarray(cand_rowptr, dtype=np.int64)
        cand_dst = np.ascontiguousarray(cand_dst, dtype=np.int32)
    n = int(cand_dst.shape[0])
    c = _Cands(_ptr(cand_rowptr), _ptr(cand_dst), n, kind, int(flags))
    return c, (cand_rowptr, cand_dst)


def stage_candidates(sys: System, cand_rowptr, cand_dst):
    """mm_stage_candidates: start copying host lists (numpy; pinned memory for
    an asynchronous copy) to the device and checking them; a later call with
    the same arrays and lists_unchanged=True uses them.  The arrays must stay
    alive and unchanged until then."""
    cd, keep = _cands(cand_rowptr, cand_dst)
    if cd is None or cd.ptr_kind != PTR_HOST:
        raise ValueError("stage_candidates: host (numpy) lists")
    sys._staged = keep  # the arrays stay referenced while the copy may run
    _check(_lib.mm_stage_candidates(sys.handle, ctypes.byref(cd)))


def evaluate_moves(sys: System, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED,
                   cand_rowptr=None, cand_dst=None, records=None, digest=None, lists_unchanged: bool = False):
    """mm_evaluate_moves.  records: a numpy array of MOVE_EVAL_DTYPE or a CUDA
    uint8 tensor of 16*n_cand bytes (or None).  digest: a 1-element numpy
    uint64 array or CUDA int64 tensor (or None).  Both in the same memory.
    lists_unchanged: the same device lists as the last call that took lists
    (MM_CANDS_UNCHANGED)."""
    crit = _Crit(mask, min_improved)
    cd, keep = _cands(cand_rowptr, cand_dst, CANDS_UNCHANGED if lists_unchanged else 0)
    outs = [o for o in (records, digest) if o is not None]
    kind = _kind(outs[0]) if outs else PTR_DEVICE
    if any(_kind(o) != kind for o in outs):
        raise ValueError("evaluate_moves: records and digest must be in the same memory")
    _check(_lib.mm_evaluate_moves(sys.handle, ctypes.byref(crit), ctypes.byref(cd) if cd else None,
                                  _ptr(records), _ptr(digest), kind))
    del keep
    return records, digest


def suggest_moves(sys: System, k: int, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED,
                  cand_rowptr=None, cand_dst=None, out=None, lists_unchanged: bool = False):
    """mm_suggest_moves.  Returns (top-k moves as a MOVE_DTYPE numpy array, or
    the given out buffer), n_kept, n_methods_with_kept.  lists_unchanged: the
    same device lists as the last call that took lists (MM_CANDS_UNCHANGED)."""
    crit = _Crit(mask, min_improved)
    cd, keep = _cands(cand_rowptr, cand_dst, CANDS_UNCHANGED if lists_unchanged else 0)
    if out is None:
        out = np.zeros(max(k, 0), dtype=MOVE_DTYPE)
    nk, nm = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.mm_suggest_moves(sys.handle, ctypes.byref(crit), ctypes.byref(cd) if cd else None, int(k),
                                 _ptr(out), _kind(out), ctypes.byref(nk), ctypes.byref(nm)))
    del keep
    n = min(int(k), int(nk.value))
    return (out[:n] if _kind(out) == PTR_HOST else out), int(nk.value), int(nm.value)


def suggest_moves_noalloc(sys: System, k: int, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED,
                          cand_rowptr=None, cand_dst=None, out=None):
    """mm_suggest_moves_noalloc: same result as suggest_moves, computed in the
    library's fixed static device array without allocating device memory (for
    callers that cannot allocate).  Candidate lists must be CUDA tensors."""
    crit = _Crit(mask, min_improved)
    cd, keep = _cands(cand_rowptr, cand_dst)
    if out is None:
        out = np.zeros(max(k, 0), dtype=MOVE_DTYPE)
    nk, nm = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.mm_suggest_moves_noalloc(sys.handle, ctypes.byref(crit), ctypes.byref(cd) if cd else None, int(k),
                                         _ptr(out), _kind(out), ctypes.byref(nk), ctypes.byref(nm)))
    del keep
    n = min(int(k), int(nk.value))
    return (out[:n] if _kind(out) == PTR_HOST else out), int(nk.value), int(nm.value)


class Batch:
    """Many systems evaluated by one persistent launch under a CUDA graph
    (mm_batch_*).  The systems must stay alive while the batch exists."""

    def __init__(self, systems, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED,
                 kept_cap: int = 4096, stream=None):
        self.systems = list(systems)
        arr = (_vp * len(self.systems))(*[s.handle.value for s in self.systems])
        crit = _Crit(mask, min_improved)
        h = _vp()
        _check(_lib.mm_batch_create(arr, len(self.systems), ctypes.byref(crit), int(kept_cap),
                                    _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.n = len(self.systems)

    def set_tile(self, methods_per_tile: int):
        _check(_lib.mm_batch_set_tile(self._h, int(methods_per_tile)))

    def autotune(self) -> int:
        c = ctypes.c_int32()
        _check(_lib.mm_batch_autotune(self._h, ctypes.byref(c)))
        return int(c.value)

    def config(self) -> tuple[int, int]:
        """mm_batch_config_get: (methods per tile, persistent blocks)."""
        t, g = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.mm_batch_config_get(self._h, ctypes.byref(t), ctypes.byref(g)))
        return int(t.value), int(g.value)

    def run(self, digest: bool = True):
        """One replay of the batch graph; returns (digests or None, kept counts)."""
        dig = np.zeros(self.n, dtype=np.uint64) if digest else None
        nk = np.zeros(self.n, dtype=np.int64)
        _check(_lib.mm_batch_run(self._h, dig.ctypes.data if digest else None, nk.ctypes.data))
        return dig, nk

    def suggestions(self, i: int, k: int):
        out = np.zeros(max(k, 1), dtype=MOVE_DTYPE)
        nk = ctypes.c_int64()
        _check(_lib.mm_batch_suggestions(self._h, int(i), int(k), out.ctypes.data, PTR_HOST, ctypes.byref(nk)))
        return out[: min(k, nk.value)], int(nk.value)

    def free(self):
        if self._h:
            _lib.mm_batch_free(self._h)
            self._h = _vp(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def apply_edit(sys: System, kind: int, m: int, target: int):
    """mm_apply_edit: one edit (EDIT_* kind, method m, attribute / callee / class)."""
    e = _Edit(int(kind), int(m), int(target), 0)
    _check(_lib.mm_apply_edit(sys.handle, ctypes.byref(e)))


def apply_sequence(sys: System, rounds: int, mask: int = DEFAULT_MASK, min_improved: int = DEFAULT_MIN_IMPROVED,
                   per_round: int = 0, cap: int | None = None):
    """mm_apply_sequence: rounds of non-conflicting kept moves applied to the
    system; returns the applied moves (APPLIED_DTYPE array, in order)."""
    cap = sys.n_methods * max(rounds, 1) if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=APPLIED_DTYPE)
    n = ctypes.c_int64()
    _check(_lib.mm_apply_sequence(sys.handle, ctypes.byref(_Crit(mask, min_improved)), int(rounds), int(per_round),
                                  out.ctypes.data, cap, ctypes.byref(n)))
    return out[: min(cap, n.value)]


def suggest_r3(sys: System, k: int):
    """mm_suggest_r3: (top-k R3 moves as an R3_DTYPE array, n_kept,
    n_candidates, n_high_classes)."""
    out = np.zeros(max(k, 1), dtype=R3_DTYPE)
    nk, nc, nh = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(_lib.mm_suggest_r3(sys.handle, int(k), out.ctypes.data, ctypes.byref(nk), ctypes.byref(nc),
                              ctypes.byref(nh)))
    return out[: min(k, nk.value)], int(nk.value), int(nc.value), int(nh.value)


def metric_variants(sys: System, out="host", out_q_all="host"):
    """mm_metric_variants: the LCOM and CBO variants per class (VARIANTS_DTYPE)
    and q_all per method.  Buffers as compute_metrics ("host" = new numpy
    arrays; CUDA uint8 tensors of 56*n_classes / 4*n_methods bytes)."""
    if isinstance(out, str):
        out = np.zeros(sys.n_classes, dtype=VARIANTS_DTYPE)
    if isinstance(out_q_all, str):
        out_q_all = np.zeros(sys.n_methods, dtype=np.int32)
    outs = [o for o in (out, out_q_all) if o is not None]
    kind = _kind(outs[0]) if outs else PTR_HOST
    if any(_kind(o) != kind for o in outs):
        raise ValueError("metric_variants: outputs must be both host or both device")
    _check(_lib.mm_metric_variants(sys.handle, _ptr(out), _ptr(out_q_all), kind))
    return out, out_q_all


def rank_classes(sys: System, metric: int, k: int):
    """mm_rank_classes: the first k classes by a metric (RANK_*), largest
    first, ties by ascending id; returns (ids, values) as numpy arrays."""
    n = max(0, min(int(k), sys.n_classes))
    ids = np.zeros(max(n, 1), dtype=np.int32)
    vals = np.zeros(max(n, 1), dtype=np.int64)
    _check(_lib.mm_rank_classes(sys.handle, int(metric), int(k), ids.ctypes.data, vals.ctypes.data, PTR_HOST))
    return ids[:n], vals[:n]


def export_system(sys: System):
    """mm_export_system: the system's current arrays as numpy arrays
    (method_class, attr_class, acc_rowptr, acc_idx, call_rowptr, call_idx)."""
    inf = sys.info()
    M, A = sys.n_methods, sys.n_attrs
    out = (np.zeros(M, np.int32), np.zeros(A, np.int32), np.zeros(M + 1, np.int64), np.zeros(inf["n_acc"], np.int32),
           np.zeros(M + 1, np.int64), np.zeros(inf["n_call"], np.int32))
    _check(_lib.mm_export_system(sys.handle, *[_ptr(a) for a in out]))
    return out


# ---------------------------------------------------------------- serving

class _ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("crit", _Crit)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("served", ctypes.c_int64), ("failed", ctypes.c_int64), ("loads", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("resident_bytes", ctypes.c_int64), ("n_snapshots", ctypes.c_int64),
                ("wall_s", ctypes.c_double)]


class _SnapInfo(ctypes.Structure):
    _fields_ = [("request", ctypes.c_int64), ("system", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("n_methods", ctypes.c_int32), ("n_attrs", ctypes.c_int32), ("n_acc", ctypes.c_int64),
                ("n_call", ctypes.c_int64)]


REQUEST_DTYPE = np.dtype([("system", "<i4"), ("kind", "<i4"), ("m", "<i4"), ("reserved", "<i4"),
                          ("selector", "<u8"), ("arrival_s", "<f8")])
RESPONSE_DTYPE = np.dtype([("status", "<i4"), ("slot", "<i4"), ("kind", "<i4"), ("m", "<i4"), ("target", "<i4"),
                           ("reserved", "<i4"), ("arrival_s", "<f8"), ("start_s", "<f8"), ("done_s", "<f8"),
                           ("n_kept", "<i8"), ("n_methods_with_kept", "<i8")])
assert REQUEST_DTYPE.itemsize == 32 and RESPONSE_DTYPE.itemsize == 64

_lib.mm_server_create.argtypes = [ctypes.POINTER(_ServerConfig), ctypes.POINTER(_vp)]
_lib.mm_server_add_system.argtypes = [_vp, ctypes.POINTER(_Desc), ctypes.POINTER(ctypes.c_int32)]
_lib.mm_server_run.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_int64]
_lib.mm_server_stats_get.argtypes = [_vp, ctypes.POINTER(_ServerStats)]
_lib.mm_server_snapshot.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(_SnapInfo)] + [_vp] * 6
_lib.mm_server_free.argtypes = [_vp]
_lib.mm_server_free.restype = None
for _n in ("mm_server_create", "mm_server_add_system", "mm_server_run", "mm_server_stats_get", "mm_server_snapshot"):
    getattr(_lib, _n).restype = ctypes.c_int


class Server:
    """mm_server_*: resident evolving systems answering edit requests."""

    def __init__(self, budget_bytes: int, n_slots: int = 4, topk: int = 10, mask: int = DEFAULT_MASK,
                 min_improved: int = DEFAULT_MIN_IMPROVED):
        cfg = _ServerConfig(int(budget_bytes), int(n_slots), int(topk), _Crit(mask, min_improved))
        h = _vp()
        _check(_lib.mm_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.topk = int(topk)

    def add_system(self, system, cbo_attrs: bool = True) -> int:
        arrs = [np.ascontiguousarray(a, dtype=dt) for a, dt in
                zip((system.method_class, system.attr_class, system.acc_rowptr, system.acc_idx,
                     system.call_rowptr, system.call_idx),
                    (np.int32, np.int32, np.int64, np.int32, np.int64, np.int32))]
        d = _Desc(system.n_classes, system.n_methods, system.n_attrs, PTR_HOST, arrs[3].size, arrs[5].size,
                  *[_ptr(a) for a in arrs], 1 if cbo_attrs else 0, 0)
        i = ctypes.c_int32()
        _check(_lib.mm_server_add_system(self._h, ctypes.byref(d), ctypes.byref(i)))
        return int(i.value)

    def run(self, requests: np.ndarray, snapshot_every: int = 0):
        req = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
        n = len(req)
        resp = np.zeros(n, dtype=RESPONSE_DTYPE)
        top = np.zeros(max(n * self.topk, 1), dtype=MOVE_DTYPE)
        _check(_lib.mm_server_run(self._h, req.ctypes.data if n else None, n, resp.ctypes.data if n else None,
                                  top.ctypes.data if self.topk else None, int(snapshot_every)))
        return resp, top[: n * self.topk].reshape(n, self.topk)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_lib.mm_server_stats_get(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def snapshot(self, k: int):
        """(request index, system id, the system's arrays after that request)."""
        inf = _SnapInfo()
        _check(_lib.mm_server_snapshot(self._h, int(k), ctypes.byref(inf), *([None] * 6)))
        M, A = inf.n_methods, inf.n_attrs
        out = (np.zeros(M, np.int32), np.zeros(A, np.int32), np.zeros(M + 1, np.int64),
               np.zeros(max(inf.n_acc, 1), np.int32), np.zeros(M + 1, np.int64), np.zeros(max(inf.n_call, 1), np.int32))
        _check(_lib.mm_server_snapshot(self._h, int(k), ctypes.byref(inf), *[a.ctypes.data for a in out]))
        return int(inf.request), int(inf.system), inf.n_classes, (out[0], out[1], out[2], out[3][: inf.n_acc],
                                                                  out[4], out[5][: inf.n_call])

    def free(self):
        if self._h:
            _lib.mm_server_free(self._h)
            self._h = _vp(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_requests(systems_methods, n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """A seeded open-loop request stream: Poisson arrivals at rate_per_s, a
    uniform system, one of the five edit kinds with probability 1/5 each, a
    uniform method of that system, a 64-bit selector."""
    rng = np.random.default_rng(seed)
    req = np.zeros(n, dtype=REQUEST_DTYPE)
    req["system"] = rng.integers(0, len(systems_methods), size=n)
    req["kind"] = rng.integers(1, 6, size=n)
    ms = np.asarray(systems_methods, dtype=np.int64)
    req["m"] = (rng.random(n) * ms[req["system"]]).astype(np.int64)
    req["selector"] = rng.integers(0, 2 ** 63 - 1, size=n, dtype=np.int64).astype(np.uint64)
    req["arrival_s"] = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n)) if rate_per_s > 0 else 0.0
    return req
