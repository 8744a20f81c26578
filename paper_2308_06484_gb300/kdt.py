"""Python binding of libkdt.so (argument marshalling only).

Every step of the method runs in the CUDA library behind the C ABI declared in
include/kdt.h; this module only converts arrays to pointers and codes to
exceptions.  There is no fallback: if the library cannot be loaded, importing
anything that needs it raises.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); they must be
int32 and C-contiguous.  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KDT_OK = 0
ERRORS = {
    -1: "KDT_ERR_ARG", -2: "KDT_ERR_RANGE", -3: "KDT_ERR_DUPLICATE", -4: "KDT_ERR_DEGENERATE",
    -5: "KDT_ERR_CAPACITY", -6: "KDT_ERR_RETRY_EXHAUSTED", -7: "KDT_ERR_CUDA",
    -8: "KDT_ERR_INTERNAL", -9: "KDT_ERR_STATE", -10: "KDT_ERR_TOO_LARGE",
}


class KDTError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__("%s: %s (%d)" % (where, ERRORS.get(code, "?"), code))
        self.code = code
        self.name = ERRORS.get(code, "?")


class Config(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("domain_bits", ctypes.c_int32),
                ("retry_cap", ctypes.c_int32), ("fallback", ctypes.c_int32),
                ("rebuild_ratio", ctypes.c_float), ("filter", ctypes.c_int32),
                ("verify", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("build_warps", ctypes.c_int32),
                ("kinetic_warps", ctypes.c_int32), ("debug", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("points_per_partition", ctypes.c_int32),
                ("warps_per_partition", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("quadtree", ctypes.c_int32),
                ("rebuild_displacement", ctypes.c_float), ("plan", ctypes.c_int32),
                ("batch_build", ctypes.c_int32), ("kinetic_blocks_per_sm", ctypes.c_int32),
                ("partition_order", ctypes.c_int32)]


_STAT_FIELDS = ["steps", "moves", "rebuilds", "fallbacks", "kernel_launches", "flips", "retries",
                "walk_steps", "exact_incircle", "sos_ties", "deferred", "violations", "fixup_flips",
                "deleted_degree_sum", "stack_drops", "edge_splits", "ghost_splits", "deletes",
                "inserts", "flip_tests"]


_STAT_FIELDS2 = ["staged_to_global", "cycles_move", "cycles_move_max", "cycles_gather", "cycles_claim",
                 "cycles_local", "cycles_writeback"]

_STAT_FIELDS3 = ["cycles_ear", "cycles_lawson", "cycles_certify", "proposal_moves", "proposal_hits",
                 "trace_rows", "tail_moves", "cycles_tail", "big_moves", "cycles_big", "drain_moves",
                 "span_tickets_ns", "span_drain_ns", "span_kernel_ns", "span_huge_ns", "span_drained_ns",
                 "cycles_drained_max", "redeferred", "far_rebuilds", "big_in_place", "cycles_big_in_place",
                 "cycles_big_delete", "cycles_big_insert", "cycles_unyielding_max", "cycles_global_insert",
                 "cycles_global_insert_max", "tensor_timeouts"]


class Stats(ctypes.Structure):
    _fields_ = ([(f, ctypes.c_int64) for f in _STAT_FIELDS]
                + [("kinetic_kernel_ms", ctypes.c_double), ("kinetic_kernel_timed", ctypes.c_int64),
                   ("last_fallback_reason", ctypes.c_int64), ("last_fallback_point", ctypes.c_int64)]
                + [(f, ctypes.c_int64) for f in _STAT_FIELDS2]
                + [("step_graph_ms", ctypes.c_double), ("tuned_points_per_partition", ctypes.c_int64),
                   ("tuned_warps_per_partition", ctypes.c_int64)]
                + [(f, ctypes.c_int64) for f in _STAT_FIELDS3]
                )


class DInfo(ctypes.Structure):
    _fields_ = [("min2", ctypes.c_int64), ("d2", ctypes.c_int64), ("spread", ctypes.c_double),
                ("max_degree", ctypes.c_int64), ("cells", ctypes.c_int64)]


_lib = None

# every symbol include/kdt.h declares (checked by the loader test)
SYMBOLS = ["kdt_default_config", "kdt_create", "kdt_destroy", "kdt_build", "kdt_step",
           "kdt_rebuild", "kdt_export_triangles", "kdt_export_points", "kdt_verify",
           "kdt_num_points", "kdt_get_stats", "kdt_reset_stats", "kdt_error_string",
           "kdt_version", "kdt_stats_size", "kdt_config_size", "kdt_eval_predicates", "kdt_export_store",
           "kdt_export_triangles_noalloc", "kdt_build_batch", "kdt_step_batch",
           "kdt_export_triangles_inst", "kdt_num_instances", "kdt_set_trace", "kdt_trace_count",
           "kdt_set_proposal", "kdt_mlp_forward", "kdt_mlp_forward_tc", "kdt_mlp_loss_grad",
           "kdt_mlp_loss_grad_tc", "kdt_mlp_adam", "kdt_d_values",
           "kdt_num_cells"]

MLP_IN, MLP_OUT, MLP_SLOTS, MLP_PARAMS = 32, 18, 17, 7442


def lib_path():
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libkdt.so (compiling it first when sources are newer and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libkdt.so is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.kdt_default_config.argtypes = [ctypes.POINTER(Config)]
    L.kdt_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Config), i32, vp]
    L.kdt_destroy.argtypes = [vp]
    L.kdt_build.argtypes = [vp, vp, i64]
    L.kdt_step.argtypes = [vp, vp, i64]
    L.kdt_rebuild.argtypes = [vp]
    L.kdt_export_triangles.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.kdt_export_points.argtypes = [vp, vp, i64]
    L.kdt_verify.argtypes = [vp, ctypes.POINTER(i64)]
    L.kdt_num_points.argtypes = [vp]
    L.kdt_num_points.restype = i64
    L.kdt_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.kdt_reset_stats.argtypes = [vp]
    L.kdt_error_string.argtypes = [i32]
    L.kdt_error_string.restype = ctypes.c_char_p
    L.kdt_version.restype = i32
    L.kdt_stats_size.restype = i64
    L.kdt_config_size.restype = i64
    L.kdt_eval_predicates.argtypes = [vp, vp, i64, vp, i32, vp]
    L.kdt_export_store.argtypes = [vp, vp, vp, vp, i64]
    L.kdt_export_triangles_noalloc.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.kdt_build_batch.argtypes = [vp, vp, vp, ctypes.c_int32]
    L.kdt_step_batch.argtypes = [vp, vp, vp, ctypes.c_int32]
    L.kdt_export_triangles_inst.argtypes = [vp, ctypes.c_int32, vp, i64, ctypes.POINTER(i64)]
    L.kdt_num_instances.argtypes = [vp]
    L.kdt_num_instances.restype = ctypes.c_int32
    f32 = ctypes.c_float
    L.kdt_set_trace.argtypes = [vp, vp, vp, i64]
    L.kdt_trace_count.argtypes = [vp, ctypes.POINTER(i64)]
    L.kdt_set_proposal.argtypes = [vp, vp]
    L.kdt_mlp_forward.argtypes = [vp, vp, vp, i64, vp]
    L.kdt_mlp_forward_tc.argtypes = [vp, vp, vp, i64, vp]
    L.kdt_mlp_loss_grad.argtypes = [vp, vp, vp, vp, vp, i64, f32, vp, vp]
    L.kdt_mlp_loss_grad_tc.argtypes = [vp, vp, vp, vp, vp, i64, f32, vp, vp]
    L.kdt_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, vp]
    L.kdt_d_values.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.POINTER(DInfo)]
    L.kdt_num_cells.argtypes = [vp]
    L.kdt_num_cells.restype = i64
    for s in SYMBOLS:
        getattr(L, s)
    _lib = L
    return L


def _ptr(a, nd_last=None):
    """(pointer, n_rows) of an int32 C-contiguous numpy array or torch tensor."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.int32 or not a.is_contiguous():
            raise ValueError("expected a contiguous int32 tensor")
        return ctypes.c_void_p(a.data_ptr()), a.shape[0] if a.dim() else 0
    if not isinstance(a, np.ndarray) or a.dtype != np.int32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous int32 numpy array")
    return ctypes.c_void_p(a.ctypes.data), a.shape[0] if a.ndim else 0


def _dptr(t, dtype_name, n_last=None):
    """Device pointer of a contiguous CUDA torch tensor of the given dtype (None -> NULL)."""
    if t is None:
        return None
    import torch
    want = getattr(torch, dtype_name)
    if not hasattr(t, "data_ptr") or t.dtype != want or not t.is_contiguous() or not t.is_cuda:
        raise ValueError("expected a contiguous CUDA %s tensor" % dtype_name)
    if n_last is not None and (t.dim() < 1 or t.shape[-1] != n_last):
        raise ValueError("expected last dimension %d" % n_last)
    return ctypes.c_void_p(t.data_ptr())


def _check(rc, where):
    if rc != KDT_OK:
        raise KDTError(rc, where)


def default_config(**kw) -> Config:
    c = Config()
    load().kdt_default_config(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Triangulation:
    """One kinetic Delaunay triangulation on one GPU (a kdt handle)."""

    def __init__(self, config: Config | None = None, device: int = 0, stream=None, **kw):
        self.L = load()
        if config is None:
            config = default_config(**kw)
        self.config = config
        h = ctypes.c_void_p()
        _check(self.L.kdt_create(ctypes.byref(h), ctypes.byref(config), device,
                                 _stream_handle(stream)), "kdt_create")
        self.h = h

    # lifecycle
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.kdt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # the method
    def build(self, xy):
        p, n = _ptr(xy)
        self._n_hint = n
        _check(self.L.kdt_build(self.h, p, n), "kdt_build")

    def step(self, moves):
        p, m = _ptr(moves)
        _check(self.L.kdt_step(self.h, p, m), "kdt_step")

    def build_batch(self, xys):
        """Build one triangulation per point set in `xys` (list of (n_i, 2) int32 arrays)."""
        sizes = [int(np.asarray(x).shape[0]) for x in xys]
        offs = np.zeros(len(sizes) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(sizes)
        allxy = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int32).reshape(-1, 2) for x in xys]))
        self._n_hint = int(offs[-1])
        self._offs = offs
        _check(self.L.kdt_build_batch(self.h, ctypes.c_void_p(allxy.ctypes.data),
                                      ctypes.c_void_p(offs.ctypes.data), len(sizes)), "kdt_build_batch")

    def step_batch(self, moves, move_offsets):
        """One step of every instance: moves (m, 3) int32 with instance-local ids
        (numpy or torch, host or CUDA) and int64 CSR offsets (n_inst + 1)."""
        p, _ = _ptr(moves)
        mo = np.ascontiguousarray(np.asarray(move_offsets, dtype=np.int64))
        _check(self.L.kdt_step_batch(self.h, p, ctypes.c_void_p(mo.ctypes.data), mo.shape[0] - 1),
               "kdt_step_batch")

    def export_triangles_inst(self, inst):
        nt = ctypes.c_int64(0)
        rc = self.L.kdt_export_triangles_inst(self.h, inst, None, 0, ctypes.byref(nt))
        if rc not in (KDT_OK, -5):
            _check(rc, "kdt_export_triangles_inst")
        out = np.empty((nt.value, 3), dtype=np.int32)
        _check(self.L.kdt_export_triangles_inst(self.h, inst, ctypes.c_void_p(out.ctypes.data), nt.value,
                                                ctypes.byref(nt)), "kdt_export_triangles_inst")
        return out

    @property
    def n_instances(self):
        return int(self.L.kdt_num_instances(self.h))

    def rebuild(self):
        _check(self.L.kdt_rebuild(self.h), "kdt_rebuild")

    @property
    def n(self):
        return int(self.L.kdt_num_points(self.h))

    def export_triangles(self, out=None):
        """Canonical sorted (T, 3) triangle list; into `out` (numpy / torch) if given."""
        nt = ctypes.c_int64(0)
        if out is None:
            rc = self.L.kdt_export_triangles(self.h, None, 0, ctypes.byref(nt))
            if rc not in (KDT_OK, -5):
                _check(rc, "kdt_export_triangles")
            out = np.empty((nt.value, 3), dtype=np.int32)
        p, cap = _ptr(out)
        _check(self.L.kdt_export_triangles(self.h, p, cap, ctypes.byref(nt)), "kdt_export_triangles")
        return out[: nt.value]

    def export_triangles_noalloc(self, out):
        """Canonical list into the CUDA int32 tensor `out` (rows x 3) without any
        device allocation by the library; returns the row count."""
        nt = ctypes.c_int64(0)
        p, cap = _ptr(out)
        _check(self.L.kdt_export_triangles_noalloc(self.h, p, cap, ctypes.byref(nt)),
               "kdt_export_triangles_noalloc")
        return int(nt.value)

    def export_points(self):
        out = np.empty((self.n, 2), dtype=np.int32)
        p, cap = _ptr(out)
        _check(self.L.kdt_export_points(self.h, p, cap), "kdt_export_points")
        return out

    def d_values(self, N: int, dist2=None, cell_min2=None) -> dict:
        """d-calculation (kdt_d_values): the N-th nearest-neighbour squared distance of
        every point into dist2 and the per-partition minima into cell_min2 (int64 numpy
        arrays or CUDA tensors, or None); returns min2, d2, spread, max_degree, cells."""
        def ptr64(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                import torch
                if a.dtype != torch.int64 or not a.is_contiguous():
                    raise ValueError("expected a contiguous int64 tensor")
                return ctypes.c_void_p(a.data_ptr())
            if not isinstance(a, np.ndarray) or a.dtype != np.int64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("expected a C-contiguous int64 numpy array")
            return a.ctypes.data_as(ctypes.c_void_p)
        if dist2 is not None and dist2.shape[0] < self.L.kdt_num_points(self.h):
            raise ValueError("dist2 needs one entry per point")
        if cell_min2 is not None and cell_min2.shape[0] < self.L.kdt_num_cells(self.h):
            raise ValueError("cell_min2 needs one entry per partition")
        info = DInfo()
        _check(self.L.kdt_d_values(self.h, int(N), ptr64(dist2), ptr64(cell_min2), ctypes.byref(info)),
               "kdt_d_values")
        return {f: getattr(info, f) for f, _ in DInfo._fields_}

    def num_cells(self) -> int:
        return int(self.L.kdt_num_cells(self.h))

    def verify(self) -> int:
        bad = ctypes.c_int64(0)
        _check(self.L.kdt_verify(self.h, ctypes.byref(bad)), "kdt_verify")
        return int(bad.value)

    def export_store(self):
        """(tv, tn, pt_tri) raw arrays of the triangle store (diagnostics)."""
        n = self.L.kdt_num_points(self.h)
        if n == 0:
            n = self._n_hint
        cap = 2 * n - 2
        tv = np.empty((cap, 4), dtype=np.int32)
        tn = np.empty((cap, 4), dtype=np.int32)
        pt = np.empty(n, dtype=np.int32)
        _check(self.L.kdt_export_store(self.h, ctypes.c_void_p(tv.ctypes.data), ctypes.c_void_p(tn.ctypes.data),
                                       ctypes.c_void_p(pt.ctypes.data), cap), "kdt_export_store")
        return tv, tn, pt

    def stats(self) -> dict:
        s = Stats()
        _check(self.L.kdt_get_stats(self.h, ctypes.byref(s)), "kdt_get_stats")
        d = {f: int(getattr(s, f)) for f in _STAT_FIELDS}
        d["kinetic_kernel_ms"] = float(s.kinetic_kernel_ms)
        d["kinetic_kernel_timed"] = int(s.kinetic_kernel_timed)
        d["last_fallback_reason"] = int(s.last_fallback_reason)
        d["last_fallback_point"] = int(s.last_fallback_point)
        for f in _STAT_FIELDS2:
            d[f] = int(getattr(s, f))
        d["step_graph_ms"] = float(s.step_graph_ms)
        d["tuned_points_per_partition"] = int(s.tuned_points_per_partition)
        d["tuned_warps_per_partition"] = int(s.tuned_warps_per_partition)
        for f in _STAT_FIELDS3:
            d[f] = int(getattr(s, f))
        return d

    def reset_stats(self):
        _check(self.L.kdt_reset_stats(self.h), "kdt_reset_stats")

    # learned locate proposal (library extension)
    def set_trace(self, features=None, labels=None):
        """Record training rows into CUDA tensors features (cap, 32) float32 and labels
        (cap, 2) int32; no arguments stop recording."""
        if features is None:
            _check(self.L.kdt_set_trace(self.h, None, None, 0), "kdt_set_trace")
            return
        cap = features.shape[0]
        if labels.shape != (cap, 2):
            raise ValueError("labels must be (cap, 2)")
        _check(self.L.kdt_set_trace(self.h, _dptr(features, "float32", MLP_IN), _dptr(labels, "int32", 2), cap),
               "kdt_set_trace")

    def trace_count(self) -> int:
        n = ctypes.c_int64(0)
        _check(self.L.kdt_trace_count(self.h, ctypes.byref(n)), "kdt_trace_count")
        return int(n.value)

    def set_proposal(self, params_bf16=None):
        """Use the network with these BF16 parameters (CUDA int16 tensor or numpy uint16
        array of 7442 bit patterns) as the locate proposal; None turns it off."""
        if params_bf16 is None:
            _check(self.L.kdt_set_proposal(self.h, None), "kdt_set_proposal")
            return
        if isinstance(params_bf16, np.ndarray):
            a = np.ascontiguousarray(params_bf16, dtype=np.uint16)
            if a.size != MLP_PARAMS:
                raise ValueError("expected %d parameters" % MLP_PARAMS)
            _check(self.L.kdt_set_proposal(self.h, ctypes.c_void_p(a.ctypes.data)), "kdt_set_proposal")
            return
        if params_bf16.numel() != MLP_PARAMS:
            raise ValueError("expected %d parameters" % MLP_PARAMS)
        _check(self.L.kdt_set_proposal(self.h, _dptr(params_bf16, "int16")), "kdt_set_proposal")

    def mlp_forward(self, params_bf16, x, out):
        _check(self.L.kdt_mlp_forward(self.h, _dptr(params_bf16, "int16"), _dptr(x, "float32", MLP_IN),
                                      x.shape[0], _dptr(out, "float32", MLP_OUT)), "kdt_mlp_forward")

    def mlp_forward_tc(self, params_bf16, x, out):
        _check(self.L.kdt_mlp_forward_tc(self.h, _dptr(params_bf16, "int16"), _dptr(x, "float32", MLP_IN),
                                         x.shape[0], _dptr(out, "float32", MLP_OUT)), "kdt_mlp_forward_tc")

    def mlp_loss_grad(self, params_bf16, x, labels, grad, loss=None, index=None, rows=None, lam=0.25,
                      tensor_cores=False):
        """kdt_mlp_loss_grad, or kdt_mlp_loss_grad_tc with tensor_cores."""
        rows = (index.shape[0] if index is not None else x.shape[0]) if rows is None else rows
        fn, name = ((self.L.kdt_mlp_loss_grad_tc, "kdt_mlp_loss_grad_tc") if tensor_cores
                    else (self.L.kdt_mlp_loss_grad, "kdt_mlp_loss_grad"))
        _check(fn(self.h, _dptr(params_bf16, "int16"), _dptr(x, "float32", MLP_IN), _dptr(labels, "int32", 2),
                  _dptr(index, "int64"), rows, lam, _dptr(grad, "float32"), _dptr(loss, "float32")), name)

    def mlp_adam(self, master, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, params_bf16=None):
        _check(self.L.kdt_mlp_adam(self.h, _dptr(master, "float32"), _dptr(grad, "float32"), _dptr(m, "float32"),
                                   _dptr(v, "float32"), t, lr, beta1, beta2, eps, _dptr(params_bf16, "int16")),
               "kdt_mlp_adam")


def eval_predicates(xy_dev, quads_dev, out_dev, use_filter: bool = True, stream=None):
    """Device predicates on (a,b,c,d) rows: orient, exact incircle, filter verdict, SoS."""
    L = load()
    px, _ = _ptr(xy_dev)
    pq, m = _ptr(quads_dev)
    po, _ = _ptr(out_dev)
    _check(L.kdt_eval_predicates(px, pq, m, po, int(use_filter), _stream_handle(stream)),
           "kdt_eval_predicates")
