"""Thin ctypes binding of libbldtt.so (C ABI in include/bldtt.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are torch CUDA float64 tensors (PyTorch provides
device memory and streams); host arrays are numpy float64 arrays.  If the
library is missing or cannot be loaded this module raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbldtt.so")

COULOMB, YUKAWA, OSCILLATORY, REG_COULOMB, TEST_POLY = 0, 1, 2, 3, 99
VARIANT_FULL, VARIANT_CC_PP_ONLY = 0, 1
FP64, FP32_BULK = 0, 1
PASS_SIMT, PASS_TENSOR = 0, 1
PP, PC, CP, CC = 0, 1, 2, 3

EXPORTED = (
    "bldtt_setup", "bldtt_setup_ex", "bldtt_setup_batch", "bldtt_set_charges",
    "bldtt_compute_graph", "bldtt_autotune", "bldtt_compute", "bldtt_check_error", "bldtt_stats",
    "bldtt_destroy", "bldtt_status_string", "bldtt_last_error", "bldtt_tree_size",
    "bldtt_export_tree", "bldtt_export_lists", "bldtt_export_proxy_charges",
    "bldtt_export_proxy_potentials", "bldtt_direct_sum", "bldtt_solve_host",
    "bldtt_bounding_box_noalloc", "bldtt_selector_param_count", "bldtt_setup_learned",
    "bldtt_list_classes", "bldtt_mlp_forward", "bldtt_mlp_gradients", "bldtt_mlp_adam",
    "bldtt_pair_features", "bldtt_pair_errors", "bldtt_wait_probe", "bldtt_compute_shard",
    "bldtt_partition_leaves", "bldtt_autotune_table", "bldtt_set_pass_engine",
    "bldtt_pass_engine_used",
)


class BLDTTError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(what)


class SelectorStruct(ctypes.Structure):
    _fields_ = [("num_degrees", ctypes.c_int), ("degrees", ctypes.c_int * 8),
                ("weights", ctypes.POINTER(ctypes.c_float)),
                ("feature_lo", ctypes.c_float * 6), ("feature_hi", ctypes.c_float * 6),
                ("log10_budget", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("kappa", ctypes.c_double), ("n", ctypes.c_int),
                ("theta", ctypes.c_double), ("N0", ctypes.c_int), ("M0", ctypes.c_int),
                ("precision", ctypes.c_int), ("variant", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("num_targets", ctypes.c_int64), ("num_sources", ctypes.c_int64),
        ("num_target_clusters", ctypes.c_int32), ("num_source_clusters", ctypes.c_int32),
        ("num_target_leaves", ctypes.c_int32), ("num_source_leaves", ctypes.c_int32),
        ("target_levels", ctypes.c_int32), ("source_levels", ctypes.c_int32),
        ("list_entries", ctypes.c_int64 * 4), ("interactions", ctypes.c_double * 4),
        ("executed_evaluations", ctypes.c_double), ("work_items", ctypes.c_int64),
        ("interact_grid", ctypes.c_int32), ("interact_threads", ctypes.c_int32),
        ("ms_tree", ctypes.c_float), ("ms_lists", ctypes.c_float),
        ("ms_upward", ctypes.c_float), ("ms_interact", ctypes.c_float),
        ("ms_downward", ctypes.c_float), ("ms_compute", ctypes.c_float),
        ("launches_setup", ctypes.c_int64), ("launches_compute", ctypes.c_int64),
        ("computed_evaluations", ctypes.c_double),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbldtt.so (raises if it is missing: build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    P_i32 = ctypes.POINTER(ctypes.c_int32)
    P_i64 = ctypes.POINTER(ctypes.c_int64)
    P_dbl = ctypes.POINTER(ctypes.c_double)
    sig = {
        "bldtt_setup": (i32, [ctypes.POINTER(vp), vp, i64, vp, i64, vp, i32, dbl, i32, dbl, i32,
                               i32, i32, vp]),
        "bldtt_setup_ex": (i32, [ctypes.POINTER(vp), vp, i64, vp, i64, vp, ctypes.POINTER(Params), vp]),
        "bldtt_setup_batch": (i32, [ctypes.POINTER(vp), i32, vp, P_i64, vp, P_i64, vp,
                                    ctypes.POINTER(ctypes.c_int), P_dbl, ctypes.POINTER(Params), vp]),
        "bldtt_compute_graph": (i32, [vp, vp, vp]),
        "bldtt_autotune": (i32, [vp, vp, vp, ctypes.POINTER(ctypes.c_int)]),
        "bldtt_set_charges": (i32, [vp, vp, vp]),
        "bldtt_compute": (i32, [vp, vp, vp]),
        "bldtt_check_error": (i32, [vp]),
        "bldtt_stats": (i32, [vp, ctypes.POINTER(Stats)]),
        "bldtt_destroy": (None, [vp]),
        "bldtt_status_string": (ctypes.c_char_p, [i32]),
        "bldtt_last_error": (ctypes.c_char_p, []),
        "bldtt_tree_size": (i32, [vp, i32, P_i32, P_i32]),
        "bldtt_export_tree": (i32, [vp, i32, P_i32, P_i32, P_i32, P_dbl, P_dbl, P_i32, P_i32]),
        "bldtt_export_lists": (i32, [vp, i32, P_i32, P_i32, P_i64]),
        "bldtt_export_proxy_charges": (i32, [vp, P_dbl]),
        "bldtt_export_proxy_potentials": (i32, [vp, P_dbl]),
        "bldtt_direct_sum": (i32, [vp, i64, vp, i64, vp, i32, dbl, vp, vp]),
        "bldtt_solve_host": (i32, [P_dbl, i64, P_dbl, i64, P_dbl, i32, dbl, i32, dbl, i32, i32,
                                   i32, P_dbl, ctypes.POINTER(Stats)]),
        "bldtt_bounding_box_noalloc": (i32, [vp, i64, vp, vp, vp]),
        "bldtt_selector_param_count": (i64, [i32]),
        "bldtt_setup_learned": (i32, [ctypes.POINTER(vp), vp, i64, vp, i64, vp, ctypes.POINTER(Params),
                                      ctypes.POINTER(SelectorStruct), vp]),
        "bldtt_list_classes": (i32, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
        "bldtt_mlp_forward": (i32, [vp, i32, vp, i64, vp, vp]),
        "bldtt_mlp_gradients": (i32, [vp, i32, vp, vp, vp, i64, vp, vp, vp]),
        "bldtt_mlp_adam": (i32, [vp, vp, vp, vp, i64, i32, ctypes.c_float, vp]),
        "bldtt_pair_features": (i32, [vp, i64, vp, vp, vp]),
        "bldtt_pair_errors": (i32, [vp, i64, vp, i32, i32, ctypes.POINTER(ctypes.c_int), vp, vp]),
        "bldtt_wait_probe": (i32, [i64, vp]),
        "bldtt_compute_shard": (i32, [vp, i32, i32, vp, vp]),
        "bldtt_partition_leaves": (i32, [P_dbl, ctypes.c_int32, ctypes.c_int32, P_i32]),
        "bldtt_set_pass_engine": (i32, [vp, i32, i32]),
        "bldtt_pass_engine_used": (i32, [vp, i32]),
        "bldtt_autotune_table": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_float)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        lib = load_library()
        name = lib.bldtt_status_string(status).decode()
        detail = lib.bldtt_last_error().decode()
        raise BLDTTError(status, f"{name}: {detail}")


def _dptr(t, n_expected=None):
    """Device pointer of a contiguous CUDA float64 tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if n_expected is not None and t.numel() != n_expected:
        raise ValueError(f"expected {n_expected} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _np_ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Plan:
    """A set-up BLDTT problem (bldtt_setup); compute() runs the compute phase."""

    def __init__(self, targets, sources, charges, kernel=COULOMB, kappa=0.0, n=8, theta=0.7,
                 N0=2000, M0=2000, precision=FP32_BULK, stream=None, variant=VARIANT_FULL):
        lib = load_library()
        if targets.dim() != 2 or targets.shape[0] != 3 or sources.dim() != 2 or sources.shape[0] != 3:
            raise ValueError("targets and sources must have shape (3, count)")
        self.M = int(targets.shape[1])
        self.N = int(sources.shape[1])
        self.n = int(n)
        self.P = self.n + 1
        self.np = self.P ** 3
        self._h = ctypes.c_void_p()
        if variant == VARIANT_FULL:
            _check(lib.bldtt_setup(ctypes.byref(self._h), _dptr(targets), self.M, _dptr(sources),
                                   self.N, _dptr(charges, self.N), int(kernel), float(kappa),
                                   self.n, float(theta), int(N0), int(M0), int(precision),
                                   _stream_ptr(stream)))
        else:
            prm = Params(int(kernel), float(kappa), self.n, float(theta), int(N0), int(M0),
                         int(precision), int(variant))
            _check(lib.bldtt_setup_ex(ctypes.byref(self._h), _dptr(targets), self.M,
                                      _dptr(sources), self.N, _dptr(charges, self.N),
                                      ctypes.byref(prm), _stream_ptr(stream)))

    def _handle(self):
        if not self._h:
            raise RuntimeError("plan already destroyed")
        return self._h

    @classmethod
    def learned(cls, targets, sources, charges, selector, kernel=COULOMB, kappa=0.0, theta=0.7,
                N0=2000, M0=2000, precision=FP32_BULK, variant=VARIANT_FULL, stream=None):
        """A plan whose traversal asks the learned selector (bldtt_setup_learned).
        selector: a Selector (degrees, float32 master weights or None, feature
        box, log10 budget)."""
        lib = load_library()
        self = cls.__new__(cls)
        self.M = int(targets.shape[1])
        self.N = int(sources.shape[1])
        self.n = int(selector.degrees[-1])
        self.P = self.n + 1
        self.np = self.P ** 3
        self._h = ctypes.c_void_p()
        prm = Params(int(kernel), float(kappa), self.n, float(theta), int(N0), int(M0),
                     int(precision), int(variant))
        st, keep = selector.as_struct()
        _check(lib.bldtt_setup_learned(ctypes.byref(self._h), _dptr(targets), self.M, _dptr(sources),
                                       self.N, _dptr(charges, self.N), ctypes.byref(prm),
                                       ctypes.byref(st), _stream_ptr(stream)))
        del keep
        return self

    @classmethod
    def batch(cls, targets, target_offsets, sources, source_offsets, charges, kernels, kappas,
              n=6, theta=0.7, N0=500, M0=500, precision=FP32_BULK, variant=VARIANT_FULL,
              stream=None):
        """A plan over independent problems (bldtt_setup_batch).  targets/sources
        are CUDA float64 (3, total) concatenations; offsets, kernels and kappas
        are per-problem host sequences."""
        lib = load_library()
        self = cls.__new__(cls)
        self.M = int(targets.shape[1])
        self.N = int(sources.shape[1])
        self.n = int(n)
        self.P = self.n + 1
        self.np = self.P ** 3
        self._h = ctypes.c_void_p()
        nprob = len(kernels)
        to = np.ascontiguousarray(target_offsets, dtype=np.int64)
        so = np.ascontiguousarray(source_offsets, dtype=np.int64)
        ks = np.ascontiguousarray(kernels, dtype=np.int32)
        kp = np.ascontiguousarray(kappas, dtype=np.float64)
        prm = Params(0, 0.0, self.n, float(theta), int(N0), int(M0), int(precision), int(variant))
        _check(lib.bldtt_setup_batch(ctypes.byref(self._h), nprob, _dptr(targets),
                                     _np_ptr(to, ctypes.c_int64), _dptr(sources),
                                     _np_ptr(so, ctypes.c_int64), _dptr(charges, self.N),
                                     ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     _np_ptr(kp, ctypes.c_double), ctypes.byref(prm),
                                     _stream_ptr(stream)))
        return self

    def compute_graph(self, phi, stream):
        """Compute through a captured CUDA graph (stream: a created torch stream)."""
        _check(load_library().bldtt_compute_graph(self._handle(), _dptr(phi, self.M),
                                                   _stream_ptr(stream)))
        return phi

    def autotune(self, phi=None, stream=None) -> int:
        import torch
        if phi is None:
            phi = torch.empty(self.M, dtype=torch.float64, device="cuda")
        chosen = ctypes.c_int(-1)
        _check(load_library().bldtt_autotune(self._handle(), _dptr(phi, self.M), _stream_ptr(stream),
                                             ctypes.byref(chosen)))
        return chosen.value

    def set_pass_engine(self, upward: int, downward: int):
        """Leaf contractions of the upward and downward passes on SIMT
        (PASS_SIMT) or on the tensor cores (PASS_TENSOR)."""
        _check(load_library().bldtt_set_pass_engine(self._handle(), int(upward), int(downward)))

    def pass_engine_used(self, which: int) -> int:
        """Engine of the upward (0) or downward (1) leaf contraction."""
        return int(load_library().bldtt_pass_engine_used(self._handle(), int(which)))

    def autotune_table(self):
        """The last autotune's searched table: (launch, kernel, layout, ms) rows."""
        lib = load_library()
        rows = ctypes.c_int(0)
        _check(lib.bldtt_autotune_table(self._handle(), 0, ctypes.byref(rows), None, None, None, None))
        n = rows.value
        ints = [(ctypes.c_int * max(n, 1))() for _ in range(3)]
        ms = (ctypes.c_float * max(n, 1))()
        _check(lib.bldtt_autotune_table(self._handle(), n, ctypes.byref(rows), *ints, ms))
        return [(ints[0][i], ints[1][i], ints[2][i], ms[i]) for i in range(n)]

    def compute(self, phi=None, stream=None):
        import torch
        if phi is None:
            phi = torch.empty(self.M, dtype=torch.float64, device="cuda")
        _check(load_library().bldtt_compute(self._handle(), _dptr(phi, self.M), _stream_ptr(stream)))
        return phi

    def compute_shard(self, shard: int, nshards: int, phi, stream=None):
        """The compute phase of one shard of the target leaves
        (bldtt_compute_shard): writes phi at that shard's targets only."""
        _check(load_library().bldtt_compute_shard(self._handle(), int(shard), int(nshards),
                                                  _dptr(phi, self.M), _stream_ptr(stream)))
        return phi

    def set_charges(self, charges, stream=None):
        _check(load_library().bldtt_set_charges(self._handle(), _dptr(charges, self.N),
                                                 _stream_ptr(stream)))

    def check_error(self):
        _check(load_library().bldtt_check_error(self._handle()))

    def stats(self) -> dict:
        st = Stats()
        _check(load_library().bldtt_stats(self._handle(), ctypes.byref(st)))
        return st.as_dict()

    def export_tree(self, which: int) -> dict:
        lib = load_library()
        nc, nl = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.bldtt_tree_size(self._handle(), which, ctypes.byref(nc), ctypes.byref(nl)))
        C = nc.value
        npart = self.M if which == 0 else self.N
        perm = np.empty(npart, dtype=np.int32)
        begin = np.empty(C, dtype=np.int32)
        end = np.empty(C, dtype=np.int32)
        parent = np.empty(C, dtype=np.int32)
        level = np.empty(C, dtype=np.int32)
        lo = np.empty(3 * C, dtype=np.float64)
        hi = np.empty(3 * C, dtype=np.float64)
        _check(lib.bldtt_export_tree(self._handle(), which, _np_ptr(perm, ctypes.c_int32),
                                     _np_ptr(begin, ctypes.c_int32), _np_ptr(end, ctypes.c_int32),
                                     _np_ptr(lo, ctypes.c_double), _np_ptr(hi, ctypes.c_double),
                                     _np_ptr(parent, ctypes.c_int32), _np_ptr(level, ctypes.c_int32)))
        return dict(perm=perm, begin=begin, end=end, lo=lo.reshape(3, C), hi=hi.reshape(3, C),
                    parent=parent, level=level, levels=nl.value)

    def list_classes(self):
        """(number of list classes, degrees of the plan)."""
        nc, nd = ctypes.c_int(), ctypes.c_int()
        deg = (ctypes.c_int * 8)()
        _check(load_library().bldtt_list_classes(self._handle(), ctypes.byref(nc), deg,
                                                 ctypes.byref(nd)))
        return nc.value, [deg[i] for i in range(nd.value)]

    def export_lists(self, classes=None):
        """(target, source) int32 array pairs per list class: PP, PC, CP, CC for a
        plan of one degree; 0 = PP, 1 + 3 i + (PC, CP, CC) at degree i otherwise."""
        lib = load_library()
        out = []
        nclass = self.list_classes()[0] if classes is None else classes
        for typ in range(nclass):
            cnt = ctypes.c_int64(0)
            st = lib.bldtt_export_lists(self._handle(), typ, None, None, ctypes.byref(cnt))
            if st != 0 and cnt.value == 0:
                _check(st)
            t = np.empty(cnt.value, dtype=np.int32)
            s = np.empty(cnt.value, dtype=np.int32)
            _check(lib.bldtt_export_lists(self._handle(), typ, _np_ptr(t, ctypes.c_int32),
                                          _np_ptr(s, ctypes.c_int32), ctypes.byref(cnt)))
            out.append((t, s))
        return out

    def proxy_charges(self):
        lib = load_library()
        nc = ctypes.c_int32()
        _check(lib.bldtt_tree_size(self._handle(), 1, ctypes.byref(nc), None))
        q = np.empty(nc.value * self.np, dtype=np.float64)
        _check(lib.bldtt_export_proxy_charges(self._handle(), _np_ptr(q, ctypes.c_double)))
        return q.reshape(nc.value, self.P, self.P, self.P)

    def proxy_potentials(self):
        lib = load_library()
        nc = ctypes.c_int32()
        _check(lib.bldtt_tree_size(self._handle(), 0, ctypes.byref(nc), None))
        p = np.empty(nc.value * self.np, dtype=np.float64)
        _check(lib.bldtt_export_proxy_potentials(self._handle(), _np_ptr(p, ctypes.c_double)))
        return p.reshape(nc.value, self.P, self.P, self.P)

    def close(self):
        if self._h:
            load_library().bldtt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Selector:
    """Learned pair selector of bldtt_setup_learned: degrees, float32 master
    weights (packed as bldtt_selector_param_count describes) or None for the
    MAC everywhere, the feature box and the per-pair log10 budget."""

    def __init__(self, degrees, weights=None, lo=None, hi=None, log10_budget=-6.0):
        self.degrees = [int(d) for d in degrees]
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        self.lo = np.full(6, -np.inf, np.float32) if lo is None else np.asarray(lo, np.float32)
        self.hi = np.full(6, np.inf, np.float32) if hi is None else np.asarray(hi, np.float32)
        self.log10_budget = float(log10_budget)
        if self.weights is not None and self.weights.size != param_count(len(self.degrees)):
            raise ValueError("selector weights have the wrong length")

    def as_struct(self):
        st = SelectorStruct()
        st.num_degrees = len(self.degrees)
        for i, d in enumerate(self.degrees):
            st.degrees[i] = d
        keep = None
        if self.weights is not None:
            keep = self.weights
            st.weights = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        for i in range(6):
            st.feature_lo[i] = float(max(self.lo[i], -3.0e38))
            st.feature_hi[i] = float(min(self.hi[i], 3.0e38))
        st.log10_budget = self.log10_budget
        return st, keep


def param_count(num_degrees: int) -> int:
    return int(load_library().bldtt_selector_param_count(int(num_degrees)))


def _fptr(t, n_expected=None, dtype_name="float32"):
    import torch
    dt = {"float32": torch.float32, "float64": torch.float64, "int32": torch.int32}[dtype_name]
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {dtype_name} tensor")
    if n_expected is not None and t.numel() != n_expected:
        raise ValueError(f"expected {n_expected} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(params, num_out, x, y=None, stream=None):
    """Selector network outputs for x (CUDA float32 [batch, 6])."""
    import torch
    B = int(x.shape[0])
    if y is None:
        y = torch.empty(B, num_out, dtype=torch.float32, device="cuda")
    _check(load_library().bldtt_mlp_forward(_fptr(params), int(num_out), _fptr(x, B * 6), B,
                                            _fptr(y, B * num_out), _stream_ptr(stream)))
    return y


def mlp_gradients(params, num_out, x, target, mask, grads=None, loss=None, stream=None):
    """Loss and gradient of the masked squared error (bldtt_mlp_gradients)."""
    import torch
    B = int(x.shape[0])
    if grads is None:
        grads = torch.empty_like(params)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(load_library().bldtt_mlp_gradients(_fptr(params), int(num_out), _fptr(x, B * 6),
                                              _fptr(target, B * num_out), _fptr(mask, B * num_out), B,
                                              _fptr(grads, params.numel()), _fptr(loss, 1),
                                              _stream_ptr(stream)))
    return grads, loss


def mlp_adam(params, m, v, grads, step, lr, stream=None):
    n = params.numel()
    _check(load_library().bldtt_mlp_adam(_fptr(params, n), _fptr(m, n), _fptr(v, n), _fptr(grads, n),
                                         n, int(step), float(lr), _stream_ptr(stream)))


def pair_features(plan, pairs, stream=None):
    """FP64 selector features of (target, source) cluster pairs (CUDA int32 [n, 2])."""
    import torch
    n = int(pairs.shape[0])
    out = torch.empty(n, 6, dtype=torch.float64, device="cuda")
    _check(load_library().bldtt_pair_features(plan._handle(), n, _fptr(pairs, 2 * n, "int32"),
                                              _fptr(out, 6 * n, "float64"), _stream_ptr(stream)))
    return out


def pair_errors(plan, pairs, degrees, samples=64, stream=None):
    """FP64 relative errors [n, len(degrees), 3] of PC, CP, CC per pair and degree."""
    import torch
    n = int(pairs.shape[0])
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    out = torch.empty(n, len(deg), 3, dtype=torch.float64, device="cuda")
    _check(load_library().bldtt_pair_errors(plan._handle(), n, _fptr(pairs, 2 * n, "int32"),
                                            int(samples), len(deg),
                                            deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                            _fptr(out, out.numel(), "float64"), _stream_ptr(stream)))
    return out


def partition_leaves(leaf_cost, nshards: int):
    """Contiguous ranges of leaves of nearly equal cost (bldtt_partition_leaves,
    host only): returns the nshards + 1 range boundaries."""
    cost = np.ascontiguousarray(leaf_cost, dtype=np.float64)
    out = np.zeros(int(nshards) + 1, dtype=np.int32)
    _check(load_library().bldtt_partition_leaves(_np_ptr(cost, ctypes.c_double), cost.size,
                                                 int(nshards), _np_ptr(out, ctypes.c_int32)))
    return out


def wait_probe(limit_ns: int, stream=None) -> int:
    """Run the bounded-wait probe (bldtt_wait_probe) and return its status
    without raising: BLDTT_ETIMEOUT (4) is the expected outcome."""
    return int(load_library().bldtt_wait_probe(int(limit_ns), _stream_ptr(stream)))


def direct_sum(targets, sources, charges, kernel=COULOMB, kappa=0.0, phi=None, stream=None):
    """FP64 direct sum on the device (bldtt_direct_sum)."""
    import torch
    M, N = int(targets.shape[1]), int(sources.shape[1])
    if phi is None:
        phi = torch.empty(M, dtype=torch.float64, device="cuda")
    _check(load_library().bldtt_direct_sum(_dptr(targets), M, _dptr(sources), N,
                                           _dptr(charges, N), int(kernel), float(kappa),
                                           _dptr(phi, M), _stream_ptr(stream)))
    return phi


def solve_host(targets, sources, charges, kernel=COULOMB, kappa=0.0, n=8, theta=0.7, N0=2000,
               M0=2000, precision=FP32_BULK):
    """One-shot solve from host numpy arrays (bldtt_solve_host); returns (phi, stats)."""
    t = np.ascontiguousarray(targets, dtype=np.float64)
    s = t if sources is targets else np.ascontiguousarray(sources, dtype=np.float64)
    q = np.ascontiguousarray(charges, dtype=np.float64)
    M, N = t.shape[1], s.shape[1]
    phi = np.empty(M, dtype=np.float64)
    st = Stats()
    _check(load_library().bldtt_solve_host(_np_ptr(t, ctypes.c_double), M,
                                           _np_ptr(s, ctypes.c_double), N,
                                           _np_ptr(q, ctypes.c_double), int(kernel), float(kappa),
                                           int(n), float(theta), int(N0), int(M0), int(precision),
                                           _np_ptr(phi, ctypes.c_double), ctypes.byref(st)))
    return phi, st.as_dict()


def bounding_box_noalloc(points, box=None, nonfinite=None, stream=None):
    """Root-cluster bounding box without device allocation by the library
    (bldtt_bounding_box_noalloc).  points: CUDA float64 (3, n); returns the
    6-element device box and the device int flag (1 if a value was not finite)."""
    import torch
    n = int(points.shape[1])
    if box is None:
        box = torch.empty(6, dtype=torch.float64, device=points.device)
    if nonfinite is None:
        nonfinite = torch.empty(1, dtype=torch.int32, device=points.device)
    _check(load_library().bldtt_bounding_box_noalloc(_dptr(points), n, _dptr(box, 6),
                                                     ctypes.c_void_p(nonfinite.data_ptr()),
                                                     _stream_ptr(stream)))
    return box, nonfinite


def status_string(status: int) -> str:
    return load_library().bldtt_status_string(status).decode()


def setup_status(targets_ptr, M, sources_ptr, N, charges_ptr, kernel, kappa, n, theta, N0, M0,
                 precision):
    """Raw bldtt_setup status for the given (possibly invalid) arguments; used
    to test argument validation, which happens before any device work."""
    lib = load_library()
    h = ctypes.c_void_p()
    st = lib.bldtt_setup(ctypes.byref(h), targets_ptr, M, sources_ptr, N, charges_ptr, kernel,
                         float(kappa), n, float(theta), N0, M0, precision, None)
    if h:
        lib.bldtt_destroy(h)
    return st
