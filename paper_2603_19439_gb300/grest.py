"""Thin ctypes binding of libgrest (include/grest.h): argument marshalling only.

Every step of the G-REST update runs in the library's CUDA kernels; this
module only converts NumPy arrays / torch tensors to pointers and back.  It
never computes anything itself and has no CPU fallback: if the shared library
is missing or cannot be loaded, constructing a tracker raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrest.so")

OP_ADJ, OP_LAP, OP_NLAP = 0, 1, 2
SUB_GREST2, SUB_GREST3, SUB_RSVD, SUB_AUTO = 0, 1, 2, 3
FP64, MIXED, MIXED_FAST = 0, 1, 2
PROJ_EXACT, PROJ_LOWRANK = 0, 1
WB_RESID, WB_DELTA = 0, 1
FLAG_CHECK = 1
FLAG_PROFILE = 2
FLAG_TWO_STREAMS = 4
PROF_CLASSES = ("spmm", "gram", "gemm", "small", "graph")
PROF_KINDS = ("spmm_f32", "spmm_f64", "gram_tc", "gram_narrow", "gram_cuda", "gemm_tc", "gemm_cuda", "double_float",
              "small", "graph")
PROF_KIND_KERNELS = ("k_spmm_rows<float> + k_spmm_long<float>", "k_spmm_rows<double> + k_spmm_long<double>",
                     "k_gram_tc", "k_gram_narrow", "k_gram_part / k_gram_pair_upper", "k_gemm_tc", "k_gemm_nn",
                     "k_spmm_df / k_gram_df / k_lift_df", "small dense group", "graph update group")

STATUS = {0: "ok", 1: "invalid argument", 2: "invalid update batch", 3: "device out of memory",
          4: "capacity exceeded", 5: "numerical breakdown", 6: "CUDA error", 7: "device wait timed out",
          8: "unsupported option"}


class GrestError(RuntimeError):
    def __init__(self, code, where):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(int(code), 'unknown')} ({int(code)})")


class Config(C.Structure):
    _fields_ = [("op", C.c_int32), ("k", C.c_int32), ("subspace", C.c_int32), ("L", C.c_int32), ("P", C.c_int32),
                ("precision", C.c_int32), ("projection", C.c_int32), ("w_block", C.c_int32), ("flags", C.c_uint32),
                ("seed", C.c_uint64), ("drop_tol", C.c_double), ("node_capacity", C.c_int64),
                ("nnz_capacity", C.c_int64), ("max_batch_edges", C.c_int64)]


class Update(C.Structure):
    _fields_ = [("n_new_nodes", C.c_int64), ("n_ins", C.c_int64), ("ins_u", C.c_void_p), ("ins_v", C.c_void_p),
                ("ins_w", C.c_void_p), ("n_del", C.c_int64), ("del_u", C.c_void_p), ("del_v", C.c_void_p),
                ("n_del_nodes", C.c_int64), ("del_nodes", C.c_void_p), ("on_device", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_nodes", C.c_int64), ("nnz", C.c_int64), ("m", C.c_int32), ("k_u", C.c_int32),
                ("rank_q", C.c_int32), ("rank_y", C.c_int32), ("mode", C.c_int32), ("pad0", C.c_int32),
                ("pivot_kept_min", C.c_double), ("pivot_dropped_max", C.c_double), ("boundary_gap", C.c_double),
                ("orth_err", C.c_double), ("max_residual", C.c_double), ("galerkin", C.c_double),
                ("ms_total", C.c_float), ("ms_graph", C.c_float), ("ms_spmm", C.c_float), ("ms_basis", C.c_float),
                ("ms_project", C.c_float), ("ms_eig", C.c_float), ("ms_lift", C.c_float), ("ms_refine", C.c_float),
                ("prof_ms", C.c_double * 5), ("prof_work", C.c_double * 5), ("prof_launches", C.c_int64 * 5),
                ("kernel_launches", C.c_int64), ("prof_bytes", C.c_double * 5),
                ("prof_kind_ms", C.c_double * 10), ("prof_kind_work", C.c_double * 10),
                ("prof_kind_bytes", C.c_double * 10), ("prof_kind_launches", C.c_int64 * 10)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            if f == "pad0":
                continue
            v = getattr(self, f)
            out[f] = list(v) if f.startswith("prof_") else v
        return out


EXPORTS = ["grest_config_default", "grest_init", "grest_apply_update", "grest_sync", "grest_get_embedding",
           "grest_set_embedding", "grest_get_embedding_async", "grest_wait_embedding", "grest_get_ritz_values", "grest_get_stats", "grest_apply_operator", "grest_gram",
           "grest_gram_f32", "grest_gemm_f32", "grest_gram_noalloc", "grest_centrality", "grest_batch_create",
           "grest_batch_apply_updates", "grest_batch_destroy", "grest_get_device_bytes", "grest_server_create",
           "grest_server_add_graph", "grest_server_submit", "grest_server_wait", "grest_server_poll", "grest_server_remove_graph",
           "grest_server_get_embedding", "grest_server_resident", "grest_server_destroy", "grest_checkpoint",
           "grest_restore", "grest_checkpoint_embedding", "grest_server_set_eviction", "grest_server_counters",
           "grest_group_create", "grest_group_apply_updates", "grest_group_get_embedding", "grest_group_get_ritz_values",
           "grest_group_info", "grest_group_destroy", "grest_check_bounded_wait", "grest_check_fast_recip",
           "grest_destroy", "grest_status_str"]

_lib = None


def load_library(path=None):
    """Load libgrest.so (raises OSError when it is absent or unloadable)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"libgrest.so not built: {p} (run __graft_entry__.build())")
    lib = C.CDLL(p)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.grest_config_default.argtypes = [C.POINTER(Config), i32]
    lib.grest_init.argtypes = [C.POINTER(Config), i64, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
    lib.grest_apply_update.argtypes = [vp, C.POINTER(Update), C.POINTER(Stats)]
    lib.grest_sync.argtypes = [vp]
    lib.grest_get_embedding.argtypes = [vp, vp, vp, vp, C.POINTER(i64), i32]
    lib.grest_set_embedding.argtypes = [vp, vp, vp, i32]
    lib.grest_get_embedding_async.argtypes = [vp, vp, vp, C.POINTER(i64)]
    lib.grest_wait_embedding.argtypes = [vp]
    lib.grest_get_ritz_values.argtypes = [vp, vp, C.POINTER(i32)]
    lib.grest_get_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.grest_apply_operator.argtypes = [vp, vp, i64, vp, i64, i32]
    lib.grest_gram.argtypes = [vp, vp, i64, i32, vp, i64, i32, i64, vp, i64]
    lib.grest_gram_f32.argtypes = [vp, vp, i64, i32, vp, i64, i32, i64, vp, i64]
    lib.grest_gemm_f32.argtypes = [vp, i64, i32, i32, C.c_double, vp, i64, vp, i64, C.c_double, vp, i64, vp, i64]
    lib.grest_centrality.argtypes = [vp, i32, vp, vp, vp, i32]
    lib.grest_gram_noalloc.argtypes = [vp, i64, i32, vp, i64, i32, i64, vp, i64, vp]
    lib.grest_batch_create.argtypes = [i32, C.POINTER(vp), i32, C.POINTER(vp)]
    lib.grest_batch_apply_updates.argtypes = [vp, C.POINTER(Update), C.POINTER(i32), C.POINTER(Stats)]
    lib.grest_batch_destroy.argtypes = [vp]
    lib.grest_batch_destroy.restype = None
    lib.grest_get_device_bytes.argtypes = [vp, C.POINTER(i64)]
    lib.grest_server_create.argtypes = [i32, i64, C.POINTER(vp)]
    lib.grest_server_add_graph.argtypes = [vp, C.POINTER(Config), i64, vp, vp, vp, vp, vp, C.POINTER(i32)]
    lib.grest_server_submit.argtypes = [vp, i32, C.POINTER(Update), C.POINTER(i64)]
    lib.grest_server_wait.argtypes = [vp, i64, C.POINTER(i32), C.POINTER(Stats), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
    lib.grest_server_poll.argtypes = [vp, i64, C.POINTER(i32)]
    lib.grest_server_remove_graph.argtypes = [vp, i32]
    lib.grest_server_get_embedding.argtypes = [vp, i32, vp, vp, vp, C.POINTER(i64)]
    lib.grest_server_resident.argtypes = [vp, C.POINTER(i64), C.POINTER(i32)]
    lib.grest_server_destroy.argtypes = [vp]
    lib.grest_server_destroy.restype = None
    lib.grest_checkpoint.argtypes = [vp, vp, C.POINTER(i64)]
    lib.grest_restore.argtypes = [vp, i64, vp, C.POINTER(vp)]
    lib.grest_checkpoint_embedding.argtypes = [vp, i64, vp, vp, vp, C.POINTER(i64), C.POINTER(i32)]
    lib.grest_server_set_eviction.argtypes = [vp, i32]
    lib.grest_server_counters.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.grest_group_create.argtypes = [i32, C.POINTER(vp), C.POINTER(i64), C.c_double, C.POINTER(vp)]
    lib.grest_group_apply_updates.argtypes = [vp, C.POINTER(Update), C.POINTER(i32), C.POINTER(Stats)]
    lib.grest_group_get_embedding.argtypes = [vp, i32, vp, vp, C.POINTER(i64)]
    lib.grest_group_get_ritz_values.argtypes = [vp, i32, vp, C.POINTER(i32)]
    lib.grest_group_info.argtypes = [vp] + [C.POINTER(i32)] * 6
    lib.grest_check_bounded_wait.argtypes = [vp]
    lib.grest_check_fast_recip.argtypes = [vp, i64, vp, vp]
    lib.grest_group_destroy.argtypes = [vp]
    lib.grest_group_destroy.restype = None
    lib.grest_destroy.argtypes = [vp]
    lib.grest_destroy.restype = None
    lib.grest_status_str.argtypes = [i32]
    lib.grest_status_str.restype = C.c_char_p
    for f in EXPORTS[:-2]:
        if f not in ("grest_destroy", "grest_batch_destroy", "grest_server_destroy", "grest_group_destroy"):
            getattr(lib, f).restype = i32
    if path is None:
        _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def default_config(k, **kw):
    lib = load_library()
    cfg = Config()
    lib.grest_config_default(C.byref(cfg), int(k))
    for key, val in kw.items():
        if not hasattr(cfg, key):
            raise KeyError(key)
        setattr(cfg, key, val)
    return cfg


def check_gram_args(X, Y, C, in_dtype, where, out_dtype="float64", require_cuda=True):
    """Raise GrestError(invalid argument) unless X (n x a) and Y (n x b) are
    2-D torch tensors of in_dtype and C (at least a x b) one of out_dtype, all
    with unit inner stride, X and Y with equal row counts, all on a CUDA
    device.  The kernels read n rows of X and Y and write a x b entries of C
    through raw pointers, so a short Y or a small C would be an out-of-bounds
    access on the device."""
    for t, dt in ((X, in_dtype), (Y, in_dtype), (C, out_dtype)):
        if not hasattr(t, "data_ptr") or t.dim() != 2 or str(t.dtype) != "torch." + dt:
            raise GrestError(1, where)
        if t.stride(1) != 1 or t.stride(0) < t.shape[1]:
            raise GrestError(1, where)
    if X.shape[0] != Y.shape[0] or X.shape[0] < 1 or X.shape[1] < 1 or Y.shape[1] < 1:
        raise GrestError(1, where)
    if C.shape[0] < X.shape[1] or C.shape[1] < Y.shape[1]:
        raise GrestError(1, where)
    if require_cuda and not (X.is_cuda and Y.is_cuda and C.is_cuda):
        raise GrestError(1, where)


def gram_noalloc(X, Y, C, stream=None):
    """C = X^T Y through grest_gram_noalloc (no device allocation inside the
    library); X, Y, C are torch CUDA float64 tensors, row-major.  Enqueued on
    `stream` (a cudaStream_t handle), by default torch's current stream of
    the current device, so that it is ordered after the writes to X and Y;
    the caller synchronizes."""
    check_gram_args(X, Y, C, "float64", "grest_gram_noalloc")
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.grest_gram_noalloc(X.data_ptr(), X.stride(0), X.shape[1], Y.data_ptr(), Y.stride(0), Y.shape[1],
                                X.shape[0], C.data_ptr(), C.stride(0), stream)
    if st != 0:
        raise GrestError(st, "grest_gram_noalloc")


def checkpoint_embedding(blob):
    """(U, theta, live) read out of grest_checkpoint bytes on the host."""
    lib = load_library()
    buf = np.frombuffer(blob, np.uint8)
    n, k = C.c_int64(), C.c_int32()
    st = lib.grest_checkpoint_embedding(_ptr(buf), buf.size, None, None, None, C.byref(n), C.byref(k))
    if st != 0:
        raise GrestError(st, "grest_checkpoint_embedding")
    U, th, live = np.empty((n.value, k.value)), np.empty(k.value), np.empty(n.value, np.uint8)
    st = lib.grest_checkpoint_embedding(_ptr(buf), buf.size, _ptr(U), _ptr(th), _ptr(live), C.byref(n), None)
    if st != 0:
        raise GrestError(st, "grest_checkpoint_embedding")
    return U, th, live.astype(bool)


def _batch_arrays(batch, on_device):
    if on_device:
        return [batch.ins_u, batch.ins_v, batch.ins_w, batch.del_u, batch.del_v, batch.del_nodes]
    return [_host(batch.ins_u, np.int32), _host(batch.ins_v, np.int32), _host(batch.ins_w, np.float64),
            _host(batch.del_u, np.int32), _host(batch.del_v, np.int32), _host(batch.del_nodes, np.int32)]


def _update_struct(batch, arrs, on_device):
    iu, iv, iw, du, dv, dn = arrs
    return Update(n_new_nodes=int(batch.n_new), n_ins=int(len(iu)), ins_u=_ptr(iu), ins_v=_ptr(iv), ins_w=_ptr(iw),
                  n_del=int(len(du)), del_u=_ptr(du), del_v=_ptr(dv),
                  n_del_nodes=int(len(dn)) if dn is not None else 0, del_nodes=_ptr(dn),
                  on_device=1 if on_device else 0)


class Batch:
    """Many Trackers updated together (grest_batch_apply_updates): one update
    each per call, n_threads native host threads, each tracker on its own
    stream.  The batch owns none of the trackers."""

    def __init__(self, trackers, n_threads=8):
        self.lib = load_library()
        self.trackers = list(trackers)
        arr = (C.c_void_p * len(self.trackers))(*[t.h.value for t in self.trackers])
        h = C.c_void_p()
        st = self.lib.grest_batch_create(len(self.trackers), arr, int(n_threads), C.byref(h))
        if st != 0:
            raise GrestError(st, "grest_batch_create")
        self.h = h

    def update(self, batches, on_device=False):
        """Apply batches[i] to tracker i.  Returns the per-tracker status codes
        (0 = ok) and step diagnostics; raises when any tracker failed."""
        n = len(self.trackers)
        if len(batches) != n:
            raise ValueError("one update per tracker")
        keep = [_batch_arrays(b, on_device) for b in batches]
        ups = (Update * n)(*[_update_struct(b, a, on_device) for b, a in zip(batches, keep)])
        status = (C.c_int32 * n)()
        stats = (Stats * n)()
        st = self.lib.grest_batch_apply_updates(self.h, ups, status, stats)
        codes = [int(x) for x in status]
        if st != 0:
            raise GrestError(st, "grest_batch_apply_updates")
        return codes, [s.as_dict() for s in stats]

    def close(self):
        if getattr(self, "h", None):
            self.lib.grest_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many small graphs updated together by grouped launches (grest_group_*):
    one launch per stage for all graphs, the update captured as a CUDA graph,
    launch shapes autotuned.  Built from checkpoints (bytes) of trackers."""

    def __init__(self, checkpoints, capacity_factor=1.25):
        self.lib = load_library()
        self._blobs = [np.frombuffer(b, np.uint8) for b in checkpoints]
        n = len(self._blobs)
        ptrs = (C.c_void_p * n)(*[b.ctypes.data for b in self._blobs])
        sizes = (C.c_int64 * n)(*[b.size for b in self._blobs])
        h = C.c_void_p()
        st = self.lib.grest_group_create(n, ptrs, sizes, float(capacity_factor), C.byref(h))
        self._blobs = None
        if st != 0:
            raise GrestError(st, "grest_group_create")
        self.h = h
        self.n = n
        self.k = int(np.frombuffer(checkpoints[0][12:16], np.int32)[0])

    def update(self, batches):
        """Apply batches[i] (host arrays) to graph i.  Returns (per-graph status
        codes, per-graph step diagnostics); raises only on a call error."""
        if len(batches) != self.n:
            raise ValueError("one update per graph")
        keep = [_batch_arrays(b, False) for b in batches]
        ups = (Update * self.n)(*[_update_struct(b, a, False) for b, a in zip(batches, keep)])
        status = (C.c_int32 * self.n)()
        stats = (Stats * self.n)()
        st = self.lib.grest_group_apply_updates(self.h, ups, status, stats)
        codes = [int(x) for x in status]
        if st != 0 and all(c == 0 for c in codes):
            raise GrestError(st, "grest_group_apply_updates")
        return codes, [s.as_dict() for s in stats]

    def embedding(self, i):
        n = C.c_int64()
        st = self.lib.grest_group_get_embedding(self.h, int(i), None, None, C.byref(n))
        if st != 0:
            raise GrestError(st, "grest_group_get_embedding")
        U, th = np.empty((n.value, self.k)), np.empty(self.k)
        st = self.lib.grest_group_get_embedding(self.h, int(i), _ptr(U), _ptr(th), C.byref(n))
        if st != 0:
            raise GrestError(st, "grest_group_get_embedding")
        return U, th

    def ritz_values(self, i):
        m = C.c_int32()
        self.lib.grest_group_get_ritz_values(self.h, int(i), None, C.byref(m))
        out = np.empty(m.value)
        self.lib.grest_group_get_ritz_values(self.h, int(i), _ptr(out), C.byref(m))
        return out

    def info(self):
        v = [C.c_int32() for _ in range(6)]
        st = self.lib.grest_group_info(self.h, *[C.byref(x) for x in v])
        if st != 0:
            raise GrestError(st, "grest_group_info")
        keys = ("captured", "launches_per_update", "tuned", "spmm_blocks", "spmm_rows_per_warp", "gemm_blocks")
        return {k: x.value for k, x in zip(keys, v)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.grest_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over many resident graphs (grest_server_*): native worker
    threads, one context and stream per admitted graph, admission by a device
    memory budget, requests of a graph in submission order."""

    def __init__(self, n_workers=8, hbm_budget=1 << 50):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.grest_server_create(int(n_workers), int(hbm_budget), C.byref(h))
        if st != 0:
            raise GrestError(st, "grest_server_create")
        self.h = h
        self.k = {}

    def add_graph(self, n, rowptr, col, val, k, U0=None, theta0=None, **cfg_fields):
        cfg = default_config(k, **cfg_fields)
        keep = [_host(rowptr, np.int64), _host(col, np.int32), _host(val, np.float64), _host(U0, np.float64),
                _host(theta0, np.float64)]
        gid = C.c_int32()
        st = self.lib.grest_server_add_graph(self.h, C.byref(cfg), int(n), *[_ptr(a) for a in keep], C.byref(gid))
        if st != 0:
            raise GrestError(st, "grest_server_add_graph")
        self.k[gid.value] = int(k)
        return gid.value

    def submit(self, gid, batch):
        """Queue one update (host arrays, copied); returns a ticket."""
        arrs = _batch_arrays(batch, False)
        u = _update_struct(batch, arrs, False)
        t = C.c_int64()
        st = self.lib.grest_server_submit(self.h, int(gid), C.byref(u), C.byref(t))
        if st != 0:
            raise GrestError(st, "grest_server_submit")
        return t.value

    def wait(self, ticket):
        """(status code, step diagnostics, ms waited, ms run) of a ticket."""
        res, s, w, r = C.c_int32(), Stats(), C.c_double(), C.c_double()
        st = self.lib.grest_server_wait(self.h, int(ticket), C.byref(res), C.byref(s), C.byref(w), C.byref(r))
        if st != 0:
            raise GrestError(st, "grest_server_wait")
        return res.value, s.as_dict(), w.value, r.value

    def done(self, ticket):
        d = C.c_int32()
        st = self.lib.grest_server_poll(self.h, int(ticket), C.byref(d))
        if st != 0:
            raise GrestError(st, "grest_server_poll")
        return bool(d.value)

    def remove_graph(self, gid):
        st = self.lib.grest_server_remove_graph(self.h, int(gid))
        if st != 0:
            raise GrestError(st, "grest_server_remove_graph")

    def embedding(self, gid):
        n = C.c_int64()
        st = self.lib.grest_server_get_embedding(self.h, int(gid), None, None, None, C.byref(n))
        if st != 0:
            raise GrestError(st, "grest_server_get_embedding")
        k = self.k[gid]
        U, th, live = np.empty((n.value, k)), np.empty(k), np.empty(n.value, np.uint8)
        st = self.lib.grest_server_get_embedding(self.h, int(gid), _ptr(U), _ptr(th), _ptr(live), C.byref(n))
        if st != 0:
            raise GrestError(st, "grest_server_get_embedding")
        return U, th, live.astype(bool)

    def resident(self):
        b, n = C.c_int64(), C.c_int32()
        self.lib.grest_server_resident(self.h, C.byref(b), C.byref(n))
        return b.value, n.value

    def set_eviction(self, on=True):
        """Checkpoint idle resident graphs to host memory when a waiting graph
        does not fit the budget (restored at their next admission)."""
        st = self.lib.grest_server_set_eviction(self.h, 1 if on else 0)
        if st != 0:
            raise GrestError(st, "grest_server_set_eviction")

    def counters(self):
        """(admissions, evictions, restores) so far."""
        a, e, r = C.c_int64(), C.c_int64(), C.c_int64()
        st = self.lib.grest_server_counters(self.h, C.byref(a), C.byref(e), C.byref(r))
        if st != 0:
            raise GrestError(st, "grest_server_counters")
        return a.value, e.value, r.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.grest_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tracker:
    """One evolving graph and its K tracked eigenpairs on the GPU."""

    def __init__(self, n, rowptr, col, val, U0, theta0, k, stream=None, **cfg_fields):
        self.lib = load_library()
        self.k = int(k)
        self.cfg = default_config(k, **cfg_fields)
        self._keep = [_host(rowptr, np.int64), _host(col, np.int32), _host(val, np.float64),
                      _host(U0, np.float64), _host(theta0, np.float64)]
        rp, cl, vl, u0, t0 = self._keep
        h = C.c_void_p()
        st = self.lib.grest_init(C.byref(self.cfg), int(n), _ptr(rp), _ptr(cl), _ptr(vl), _ptr(u0), _ptr(t0),
                                 stream, C.byref(h))
        if st != 0:
            raise GrestError(st, "grest_init")
        self.h = h
        self._keep = None
        self.n = int(n)  # node ids after the last update

    def update(self, batch, on_device=False):
        """Apply one batch (workloads.Batch with host arrays, or torch CUDA tensors
        when on_device=True).  Returns the step diagnostics as a dict."""
        if on_device:
            arrs = [batch.ins_u, batch.ins_v, batch.ins_w, batch.del_u, batch.del_v, batch.del_nodes]
        else:
            arrs = [_host(batch.ins_u, np.int32), _host(batch.ins_v, np.int32), _host(batch.ins_w, np.float64),
                    _host(batch.del_u, np.int32), _host(batch.del_v, np.int32), _host(batch.del_nodes, np.int32)]
        u = _update_struct(batch, arrs, on_device)
        s = Stats()
        st = self.lib.grest_apply_update(self.h, C.byref(u), C.byref(s))
        if st != 0:
            raise GrestError(st, "grest_apply_update")
        self.n = int(s.n_nodes)
        return s.as_dict()

    def embedding(self):
        n = C.c_int64()
        st = self.lib.grest_get_embedding(self.h, None, None, None, C.byref(n), 0)
        if st != 0:
            raise GrestError(st, "grest_get_embedding")
        U = np.empty((n.value, self.k))
        th = np.empty(self.k)
        live = np.empty(n.value, np.uint8)
        st = self.lib.grest_get_embedding(self.h, _ptr(U), _ptr(th), _ptr(live), C.byref(n), 0)
        if st != 0:
            raise GrestError(st, "grest_get_embedding")
        return U, th, live.astype(bool)

    def embedding_async(self, U_buf, theta_buf):
        """Start copying (X_K, Lambda_K) into caller buffers (numpy arrays or
        tensors: U_buf rows >= n, k columns, contiguous float64; pinned host
        memory for the copy to overlap the next update).  Returns n; the
        buffers are complete after wait_embedding()."""
        if U_buf is not None and (U_buf.shape[0] < self.n or U_buf.shape[1] != self.k):
            raise ValueError("U_buf needs at least %d rows and %d columns" % (self.n, self.k))
        if theta_buf is not None and theta_buf.shape[0] < self.k:
            raise ValueError("theta_buf needs %d values" % self.k)
        n = C.c_int64()
        st = self.lib.grest_get_embedding_async(self.h, _ptr(U_buf), _ptr(theta_buf), C.byref(n))
        if st != 0:
            raise GrestError(st, "grest_get_embedding_async")
        return n.value

    def wait_embedding(self):
        st = self.lib.grest_wait_embedding(self.h)
        if st != 0:
            raise GrestError(st, "grest_wait_embedding")

    def embedding_device(self, U_dev, theta_dev):
        """Copy (X_K, Lambda_K) into device tensors (n x k and k, float64)."""
        n = C.c_int64()
        st = self.lib.grest_get_embedding(self.h, _ptr(U_dev), _ptr(theta_dev), None, C.byref(n), 1)
        if st != 0:
            raise GrestError(st, "grest_get_embedding")
        return n.value

    def set_embedding(self, U, theta):
        """Replace (X_K, Lambda_K): numpy arrays, or torch CUDA float64 tensors."""
        dev = hasattr(U, "data_ptr")
        if not dev:
            U = _host(U, np.float64)
            theta = _host(theta, np.float64)
        st = self.lib.grest_set_embedding(self.h, _ptr(U), _ptr(theta), 1 if dev else 0)
        if st != 0:
            raise GrestError(st, "grest_set_embedding")

    def ritz_values(self):
        m = C.c_int32()
        self.lib.grest_get_ritz_values(self.h, None, C.byref(m))
        out = np.empty(m.value)
        self.lib.grest_get_ritz_values(self.h, _ptr(out), C.byref(m))
        return out

    def stats(self):
        s = Stats()
        self.lib.grest_get_stats(self.h, C.byref(s))
        return s.as_dict()

    def apply_operator(self, X, Y):
        """Y = M X with X, Y torch CUDA float64 tensors (n x w, row-major)."""
        st = self.lib.grest_apply_operator(self.h, X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0), X.shape[1])
        if st != 0:
            raise GrestError(st, "grest_apply_operator")

    def gram(self, X, Y, C):
        """C = X^T Y for torch CUDA float64 tensors (row-major)."""
        check_gram_args(X, Y, C, "float64", "grest_gram")
        st = self.lib.grest_gram(self.h, X.data_ptr(), X.stride(0), X.shape[1], Y.data_ptr(), Y.stride(0), Y.shape[1],
                                 X.shape[0], C.data_ptr(), C.stride(0))
        if st != 0:
            raise GrestError(st, "grest_gram")

    def gram_f32(self, X, Y, C):
        """C (float64) = X^T Y for torch CUDA float32 tensors (row-major)."""
        check_gram_args(X, Y, C, "float32", "grest_gram_f32")
        st = self.lib.grest_gram_f32(self.h, X.data_ptr(), X.stride(0), X.shape[1], Y.data_ptr(), Y.stride(0),
                                     Y.shape[1], X.shape[0], C.data_ptr(), C.stride(0))
        if st != 0:
            raise GrestError(st, "grest_gram_f32")

    def gemm_f32(self, X, B, Out, alpha=1.0, beta=0.0, Cin=None):
        """Out = beta Cin + alpha X B for torch CUDA float32 X, Cin, Out and
        float64 B (row-major); Cin may be Out itself."""
        cin, ldc = (Cin.data_ptr(), Cin.stride(0)) if Cin is not None else (None, 0)
        st = self.lib.grest_gemm_f32(self.h, X.shape[0], X.shape[1], B.shape[1], alpha, X.data_ptr(), X.stride(0),
                                     B.data_ptr(), B.stride(0), beta, cin, ldc, Out.data_ptr(), Out.stride(0))
        if st != 0:
            raise GrestError(st, "grest_gemm_f32")

    def centrality(self, J=0, values=True):
        """Sec. 5 subgraph centrality exp(-theta_max) X_K exp(Lambda_K) X_K^T 1
        (host arrays): returns (c or None, top-J ids, top-J values)."""
        cn = C.c_int64()
        st = self.lib.grest_get_embedding(self.h, None, None, None, C.byref(cn), 0)
        if st != 0:
            raise GrestError(st, "grest_get_embedding")
        c = np.empty(cn.value) if values else None
        ids = np.empty(max(int(J), 0), np.int32)
        vals = np.empty(max(int(J), 0))
        st = self.lib.grest_centrality(self.h, int(J), _ptr(c), _ptr(ids) if J > 0 else None,
                                       _ptr(vals) if J > 0 else None, 0)
        if st != 0:
            raise GrestError(st, "grest_centrality")
        return c, ids, vals

    def centrality_device(self, J, cent=None, ids=None, vals=None):
        """The same into torch CUDA tensors (cent float64 n, ids int32 J, vals float64 J; each may be None)."""
        st = self.lib.grest_centrality(self.h, int(J), _ptr(cent), _ptr(ids), _ptr(vals), 1)
        if st != 0:
            raise GrestError(st, "grest_centrality")

    def checkpoint(self):
        """The context's state as bytes (grest_checkpoint)."""
        nb = C.c_int64()
        st = self.lib.grest_checkpoint(self.h, None, C.byref(nb))
        if st != 0:
            raise GrestError(st, "grest_checkpoint")
        buf = np.empty(nb.value, np.uint8)
        st = self.lib.grest_checkpoint(self.h, _ptr(buf), C.byref(nb))
        if st != 0:
            raise GrestError(st, "grest_checkpoint")
        return buf[:nb.value].tobytes()

    @classmethod
    def restore(cls, blob, stream=None):
        """A new Tracker from grest_checkpoint bytes (grest_restore)."""
        lib = load_library()
        buf = np.frombuffer(blob, np.uint8)
        n, k = C.c_int64(), C.c_int32()
        st = lib.grest_checkpoint_embedding(_ptr(buf), buf.size, None, None, None, C.byref(n), C.byref(k))
        if st != 0:
            raise GrestError(st, "grest_checkpoint_embedding")
        h = C.c_void_p()
        st = lib.grest_restore(_ptr(buf), buf.size, stream, C.byref(h))
        if st != 0:
            raise GrestError(st, "grest_restore")
        self = cls.__new__(cls)
        self.lib, self.k, self.cfg, self.h, self._keep = lib, k.value, None, h, None
        self.n = n.value
        return self

    def device_bytes(self):
        b = C.c_int64()
        st = self.lib.grest_get_device_bytes(self.h, C.byref(b))
        if st != 0:
            raise GrestError(st, "grest_get_device_bytes")
        return b.value

    def sync(self):
        st = self.lib.grest_sync(self.h)
        if st != 0:
            raise GrestError(st, "grest_sync")

    def close(self):
        if getattr(self, "h", None):
            self.lib.grest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
