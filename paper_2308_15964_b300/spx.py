"""Thin ctypes binding of libspx.so (include/spx.h): argument marshalling only.

Every step of the hot path (DAG derivation, scheduling, tile ops) runs in the
library's CUDA kernels.  If the library is missing this module raises at
import time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libspx.so")

READ, WRITE, COMMUTATIVE_WRITE, ATOMIC_WRITE, MAYBE_WRITE = 0, 1, 2, 3, 4
(OP_POTRF, OP_TRSM, OP_SYRK, OP_GEMM_NT_SUB, OP_GEMM_NN_ADD, OP_TRSM_L_FWD, OP_GEMM_FWD,
 OP_TRSM_LT_BWD, OP_GEMM_BWD, OP_NOP, OP_SPIN, OP_COPY, OP_AXPY, OP_TRMM, OP_TRTRI,
 OP_TRSM_INV, OP_NBODY_SELF, OP_NBODY_PAIR, OP_POTRF_PANEL, OP_SPLIT, OP_SPLIT_T) = range(21)
OP_NAMES = ("POTRF", "TRSM", "SYRK", "GEMM_NT_SUB", "GEMM_NN_ADD", "TRSM_L_FWD", "GEMM_FWD",
            "TRSM_LT_BWD", "GEMM_BWD", "NOP", "SPIN", "COPY", "AXPY", "TRMM", "TRTRI", "TRSM_INV",
            "NBODY_SELF", "NBODY_PAIR", "POTRF_PANEL", "SPLIT", "SPLIT_T")
F64, TF32, BF16, F64_OZAKI = 0, 1, 2, 3
DT_F64, DT_F32, DT_BF16 = 0, 1, 2
EXEC_PERSISTENT, EXEC_PER_TASK, EXEC_STREAMS = 0, 1, 2

OK, NOT_SPD = 0, 1
ERR_INVALID_ARG, ERR_BAD_HANDLE, ERR_STATE, ERR_OOM, ERR_QUEUE_FULL, ERR_TIMEOUT, ERR_CUDA, \
    ERR_BAD_OP, ERR_NO_DEVICE = -1, -2, -3, -4, -5, -6, -7, -8, -9


class SpxError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("num_ctas", ctypes.c_int), ("executor", ctypes.c_int), ("trace", ctypes.c_int),
                ("no_split", ctypes.c_int), ("watchdog_ns", ctypes.c_ulonglong),
                ("queue_capacity", ctypes.c_longlong), ("cuda_graph", ctypes.c_int),
                ("priorities", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2308_15964_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    LL, ULL = ctypes.c_longlong, ctypes.c_ulonglong
    sig = {
        "spx_config_default": (None, [P]),
        "spx_graph_create": (I, [P, P]),
        "spx_tile_register": (I, [P, P, I, I, I, I, P, I, P]),
        "spx_task_insert": (I, [P, I, P, P, I, I, I, P]),
        "spx_task_set_arg": (I, [P, U, LL]),
        "spx_task_set_scalar": (I, [P, U, ctypes.c_double]),
        "spx_axpy_insert": (I, [P, P, P, LL, LL, ctypes.c_double, P]),
        "spx_nbody_insert": (I, [P, I, P, P, I, P]),
        "spx_graph_derive": (I, [P, P]),
        "spx_graph_execute": (I, [P, P]),
        "spx_batch_execute": (I, [P, I, P]),
        "spx_graph_wait": (I, [P, ULL, P]),
        "spx_graph_sizes": (I, [P, P, P, P, P]),
        "spx_graph_edges": (I, [P, P, P, P]),
        "spx_graph_tickets": (I, [P, P, P]),
        "spx_graph_trace": (I, [P, P]),
        "spx_graph_stats": (I, [P, P, I]),
        "spx_graph_assign_priorities": (I, [P]),
        "spx_graph_task_ops": (I, [P, P, P]),
        "spx_graph_write_dot": (I, [P, ctypes.c_char_p]),
        "spx_graph_reset": (I, [P]),
        "spx_graph_clear": (I, [P]),
        "spx_graph_destroy": (None, [P]),
        "spx_strerror": (ctypes.c_char_p, [I]),
        "spx_graph_timing": (I, [P, P, P]),
        "spx_cholesky_insert": (I, [P, P, I, I, I, P, I, I, I, I, P]),
        "spx_gemm_insert": (I, [P, P, P, P, I, I, I, I, P]),
        "spx_gemm_insert_ozaki": (I, [P, P, P, P, I, I, I, I, P, LL, P]),
        "spx_cholesky_host_ozaki": (I, [P, P, P, I, I, I, P, I, P, LL, P, I, P, P]),
        "spx_graph_tasks_done": (I, [P, P, I, P]),
        "spx_stream_copy_h2d": (I, [P, P, ctypes.c_size_t, P, ctypes.c_size_t, ctypes.c_size_t,
                                    ctypes.c_size_t]),
        "spx_cholesky_insert_batch": (I, [P, I, P, P, P, P, P, P, P, I, I, P]),
        "spx_tc_gemm_nt": (I, [P, I, I, I, P, I, P, I, I, I, P, P]),
        "spx_lowp_register": (I, [P, P, I, I, I, I, P]),
        "spx_ozaki_slot_bytes": (LL, [I]),
        "spx_stream_begin": (I, [P, P, I, I, LL, LL]),
        "spx_stream_flush": (I, [P]),
        "spx_stream_end": (I, [P]),
        "spx_graph_host_preds": (I, [P, P, P, LL, P]),
        "spx_ozaki_register": (I, [P, P, I, I, P]),
        "spx_cholesky_insert_ozaki": (I, [P, P, I, I, I, P, LL, P, I, I, P, I, I, I, P]),
        "spx_cholesky_insert_mixed": (I, [P, P, I, I, I, P, I, P, I, I, I, I, P]),
        "spx_cholesky_insert_mixed_inv": (I, [P, P, I, I, I, P, I, P, I, P, I, I, I, I, P]),
        "spx_solve_insert": (I, [P, P, I, I, I, P, I, I, P]),
        "spx_trtri_insert": (I, [P, P, I, I, I, P, I, P]),
        "spx_overhead_insert": (I, [P, I, I, I, I, LL, P]),
        "spx_refine_inv_insert": (I, [P, P, I, I, P, I, I, P, I, P, P, P, P, I, I, I, P]),
        "spx_solve_inv_insert": (I, [P, P, I, I, I, P, I, P, P, I, I, P]),
        "spx_solve_inv_f32_insert": (I, [P, P, I, I, I, P, I, P, P, P, P, I, I, P]),
        "spx_residual_f64": (I, [P, I, I, P, I, P, I, P, I, I, P, P]),
        "spx_residual_eta_f64": (I, [P, I, I, P, I, P, I, P, I, I, P, P, P, I, P]),
        "spx_gmres_ir_workspace": (LL, [I, I, I]),
        "spx_gmres_ir": (I, [P, I, I, P, P, I, P, P, P, LL, P, P, P]),
        "spx_norm_inf_f64": (I, [P, I, I, P, P]),
        "spx_axpy_f64": (I, [P, P, LL, ctypes.c_double, P]),
        "spx_server_config_default": (None, [P]),
        "spx_server_create": (I, [P, P]),
        "spx_server_submit": (I, [P, P, P]),
        "spx_server_poll": (I, [P, ULL, P, P]),
        "spx_server_stop": (I, [P]),
        "spx_server_stats": (I, [P, P, I]),
        "spx_server_destroy": (None, [P]),
        "spx_refine_insert": (I, [P, P, I, I, P, I, I, P, P, P, I, I, I, P]),
        "spx_copy2d": (I, [P, ctypes.c_size_t, P, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t, P]),
        "spx_graph_derive_noalloc": (I, [P, P, P, P, I, I, LL, P, P, LL, P, P, P]),
        "spx_abi_version": (I, []),
        "spx_probe": (I, [I, I, P, P]),
        "spx_device_sm_count": (I, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def strerror(code: int) -> str:
    return lib.spx_strerror(code).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise SpxError(rc, what)
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return ctypes.c_void_p(int(stream))


class Graph:
    """An STF task graph (spx_graph_t)."""

    def __init__(self, num_ctas=0, executor=EXEC_PERSISTENT, trace=False, no_split=False,
                 watchdog_ns=0, queue_capacity=0, cuda_graph=False, priorities=0):
        cfg = Config()
        lib.spx_config_default(ctypes.byref(cfg))
        cfg.num_ctas = num_ctas
        cfg.executor = executor
        cfg.trace = 1 if trace else 0
        cfg.no_split = 1 if no_split else 0
        if watchdog_ns:
            cfg.watchdog_ns = watchdog_ns
        cfg.queue_capacity = queue_capacity
        cfg.cuda_graph = 1 if cuda_graph else 0
        cfg.priorities = int(priorities)
        h = ctypes.c_void_p()
        _check(lib.spx_graph_create(ctypes.byref(h), ctypes.byref(cfg)), "spx_graph_create")
        self._h = h
        self._keep = []          # tensors whose memory the graph refers to

    # -- building ---------------------------------------------------------
    def register(self, ptr: int, rows: int, cols: int, ld: int, dtype=DT_F64, lowp_ptr=0,
                 lowp_ld=0) -> int:
        out = ctypes.c_uint()
        _check(lib.spx_tile_register(self._h, ctypes.c_void_p(ptr), rows, cols, ld, dtype,
                                     ctypes.c_void_p(lowp_ptr or None), lowp_ld, ctypes.byref(out)),
               "spx_tile_register")
        return out.value

    def register_tensor(self, t, dtype=DT_F64) -> int:
        """Register a 2-D row-major view (stride(1) == 1) of a CUDA tensor."""
        assert t.dim() == 2 and t.stride(1) == 1
        return self.register(t.data_ptr(), t.shape[0], t.shape[1], t.stride(0), dtype)

    def register_ozaki(self, ptr: int, nslots: int, b: int) -> int:
        """spx_ozaki_register: a store of nslots split slots of pitch b."""
        out = ctypes.c_uint()
        _check(lib.spx_ozaki_register(self._h, ctypes.c_void_p(ptr), nslots, b, ctypes.byref(out)),
               "spx_ozaki_register")
        return out.value

    def insert(self, op: int, handles, modes, priority=0, prec=F64) -> int:
        h = np.ascontiguousarray(handles, dtype=np.uint32)
        m = np.ascontiguousarray(modes, dtype=np.int32)
        out = ctypes.c_uint()
        _check(lib.spx_task_insert(self._h, op, _ptr(h), _ptr(m), len(h), priority, prec,
                                   ctypes.byref(out)), "spx_task_insert")
        return out.value

    def set_arg(self, task: int, arg: int):
        _check(lib.spx_task_set_arg(self._h, task, arg), "spx_task_set_arg")

    # -- streaming --------------------------------------------------------
    def stream_begin(self, max_tasks, max_tiles, max_records, max_preds, stream=None):
        """spx_stream_begin: run the tasks inserted so far and keep running;
        insert more, then stream_flush / stream_end."""
        _check(lib.spx_stream_begin(self._h, _stream_ptr(stream), max_tasks, max_tiles,
                                    max_records, max_preds), "spx_stream_begin")

    def stream_flush(self):
        _check(lib.spx_stream_flush(self._h), "spx_stream_flush")

    def stream_end(self):
        _check(lib.spx_stream_end(self._h), "spx_stream_end")

    def host_preds(self):
        """(pred_ptr, pred): the host-side derivation's predecessor lists."""
        n = self.sizes()[0]
        ptr = np.zeros(n + 1, np.uint32)
        total = ctypes.c_longlong()
        lib.spx_graph_host_preds(self._h, _ptr(ptr), None, 0, ctypes.byref(total))
        pred = np.zeros(max(1, total.value), np.uint32)
        _check(lib.spx_graph_host_preds(self._h, _ptr(ptr), _ptr(pred), total.value,
                                        ctypes.byref(total)), "spx_graph_host_preds")
        return ptr, pred[:total.value]

    # -- running ----------------------------------------------------------
    def derive(self, stream=None):
        _check(lib.spx_graph_derive(self._h, _stream_ptr(stream)), "spx_graph_derive")

    def execute(self, stream=None):
        _check(lib.spx_graph_execute(self._h, _stream_ptr(stream)), "spx_graph_execute")

    def wait(self, timeout_ns: int = 0):
        """Returns (status, info); status is OK, NOT_SPD or a negative error code."""
        info = ctypes.c_int()
        rc = lib.spx_graph_wait(self._h, timeout_ns, ctypes.byref(info))
        return rc, info.value

    def run(self, stream=None, timeout_ns: int = 0):
        self.execute(stream)
        return self.wait(timeout_ns)

    def reset(self):
        _check(lib.spx_graph_reset(self._h), "spx_graph_reset")

    def clear(self):
        _check(lib.spx_graph_clear(self._h), "spx_graph_clear")
        self._keep.clear()

    # -- inspection -------------------------------------------------------
    def sizes(self):
        v = [ctypes.c_longlong() for _ in range(4)]
        _check(lib.spx_graph_sizes(self._h, *[ctypes.byref(x) for x in v]), "spx_graph_sizes")
        return tuple(x.value for x in v)  # ntasks, nedges, naccesses, ntiles

    def edges(self):
        n, e, _, _ = self.sizes()
        row_ptr = np.zeros(n + 1, np.uint32)
        col = np.zeros(max(e, 1), np.uint32)
        indeg = np.zeros(max(n, 1), np.uint32)
        _check(lib.spx_graph_edges(self._h, _ptr(row_ptr), _ptr(col), _ptr(indeg)), "spx_graph_edges")
        return row_ptr, col[:e].copy(), indeg[:n].copy()

    def tickets(self):
        n = self.sizes()[0]
        s = np.zeros(n, np.uint32)
        e = np.zeros(n, np.uint32)
        _check(lib.spx_graph_tickets(self._h, _ptr(s), _ptr(e)), "spx_graph_tickets")
        return s, e

    def tasks_done(self, tasks):
        """spx_graph_tasks_done: 1 for each task that has finished, else 0."""
        t = np.ascontiguousarray(tasks, dtype=np.uint32)
        d = np.zeros(len(t), dtype=np.int32)
        _check(lib.spx_graph_tasks_done(self._h, _ptr(t), len(t), _ptr(d)), "spx_graph_tasks_done")
        return d

    def trace(self):
        n = self.sizes()[0]
        r = np.zeros((n, 4), np.uint64)
        _check(lib.spx_graph_trace(self._h, _ptr(r)), "spx_graph_trace")
        return r

    def assign_priorities(self):
        _check(lib.spx_graph_assign_priorities(self._h), "spx_graph_assign_priorities")

    def task_ops(self):
        """(op, priority class) of every task, in insertion order."""
        n = self.sizes()[0]
        ops = np.zeros(max(n, 1), np.int32)
        pr = np.zeros(max(n, 1), np.int32)
        _check(lib.spx_graph_task_ops(self._h, _ptr(ops), _ptr(pr)), "spx_graph_task_ops")
        return ops[:n], pr[:n]

    def stats(self):
        v = np.zeros(9 + len(OP_NAMES), np.int64)
        _check(lib.spx_graph_stats(self._h, _ptr(v), len(v)), "spx_graph_stats")
        keys = ["parts", "queue_hiwater", "empty_pops", "ctas", "busy_cycles", "total_cycles",
                "queue_capacity", "pushed_high", "pushed_normal"]
        out = dict(zip(keys, (int(x) for x in v[:9])))
        out["op_cycles"] = {nm: int(c) for nm, c in zip(OP_NAMES, v[9:]) if c}
        return out

    def timing(self):
        """(prep_ms, run_ms) of the last execution (device events)."""
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(lib.spx_graph_timing(self._h, ctypes.byref(a), ctypes.byref(b)), "spx_graph_timing")
        return a.value, b.value

    def write_dot(self, path: str):
        _check(lib.spx_graph_write_dot(self._h, path.encode()), "spx_graph_write_dot")

    def close(self):
        if self._h:
            lib.spx_graph_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_execute(graphs, stream=None):
    """Run built graphs in one persistent launch (spx_batch_execute); then
    wait on each graph for its own status."""
    arr = (ctypes.c_void_p * len(graphs))(*[g._h.value for g in graphs])
    _check(lib.spx_batch_execute(arr, len(graphs), _stream_ptr(stream)), "spx_batch_execute")


class GmresConfig(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("tol", ctypes.c_double)]


class GmresResult(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer", ctypes.c_int), ("inner", ctypes.c_int),
                ("pad_", ctypes.c_int), ("eta", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_tasks", ctypes.c_longlong), ("max_tiles", ctypes.c_longlong),
                ("max_records", ctypes.c_longlong), ("max_edges", ctypes.c_longlong),
                ("max_maps", ctypes.c_longlong), ("queue_capacity", ctypes.c_longlong),
                ("num_ctas", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("watchdog_ns", ctypes.c_ulonglong), ("idle_ns", ctypes.c_ulonglong)]


class Server:
    """Continuous-batching server (spx_server_t): one resident persistent
    kernel; graphs submitted while it runs are admitted and interleaved."""

    def __init__(self, **kw):
        cfg = ServerConfig()
        lib.spx_server_config_default(ctypes.byref(cfg))
        for k, v in kw.items():
            setattr(cfg, k, int(v))
        h = ctypes.c_void_p()
        _check(lib.spx_server_create(ctypes.byref(h), ctypes.byref(cfg)), "spx_server_create")
        self._h = h
        self._keep = {}

    def submit(self, g: "Graph"):
        """Request id, or None when the server has no room now (retry later)."""
        rid = ctypes.c_ulonglong()
        rc = lib.spx_server_submit(self._h, g._h, ctypes.byref(rid))
        if rc == ERR_OOM:
            return None
        _check(rc, "spx_server_submit")
        self._keep[rid.value] = list(g._keep)
        return rid.value

    def poll(self, rid: int):
        """None while running, else (status, info)."""
        st, info = ctypes.c_int(), ctypes.c_int()
        rc = _check(lib.spx_server_poll(self._h, rid, ctypes.byref(st), ctypes.byref(info)),
                    "spx_server_poll")
        if rc == 0:
            return None
        self._keep.pop(rid, None)
        return st.value, info.value

    def stop(self) -> int:
        return lib.spx_server_stop(self._h)

    def assign_priorities(self):
        _check(lib.spx_graph_assign_priorities(self._h), "spx_graph_assign_priorities")

    def task_ops(self):
        """(op, priority class) of every task, in insertion order."""
        n = self.sizes()[0]
        ops = np.zeros(max(n, 1), np.int32)
        pr = np.zeros(max(n, 1), np.int32)
        _check(lib.spx_graph_task_ops(self._h, _ptr(ops), _ptr(pr)), "spx_graph_task_ops")
        return ops[:n], pr[:n]

    def stats(self):
        v = np.zeros(6, np.int64)
        _check(lib.spx_server_stats(self._h, _ptr(v), 6), "spx_server_stats")
        return dict(zip(["parts", "tasks", "requests", "live", "busy_cycles", "total_cycles"],
                        (int(x) for x in v)))

    def close(self):
        if self._h:
            lib.spx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe(which: int, iters: int):
    rate, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.spx_probe(which, iters, ctypes.byref(rate), ctypes.byref(ms)), "spx_probe")
    return rate.value, ms.value
