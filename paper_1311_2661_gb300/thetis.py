"""Thin ctypes binding of libthetis.so (include/thetis.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA); all arrays of one call must live in the same place.  Streams
may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or ``None``
(the handle then owns a private stream).

The functions carry the C names (``thetis_build_vc``, ``thetis_solve``, ...).
If the library has not been built, importing this module raises: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthetis.so")

THETIS_OK, THETIS_E_INVALID, THETIS_E_NOMEM, THETIS_E_BUDGET, THETIS_E_CUDA = 0, 1, 2, 3, 4
THETIS_E_TIMEOUT, THETIS_E_REPAIR, THETIS_PENDING, THETIS_NOT_CONVERGED = 5, 6, 7, 8
MEM_HOST, MEM_DEVICE = 0, 1
ROW_EQ, ROW_GE, ROW_LE = 0, 1, 2
ROUND_VC, ROUND_IS, ROUND_MC, ROUND_SC, ROUND_SC_RAND, ROUND_MAP = 0, 1, 2, 3, 4, 5
MODE_COLORED, MODE_ASYNC = 0, 1

STATUS_NAMES = {0: "OK", 1: "E_INVALID", 2: "E_NOMEM", 3: "E_BUDGET", 4: "E_CUDA", 5: "E_TIMEOUT",
                6: "E_REPAIR", 7: "PENDING", 8: "NOT_CONVERGED"}


class ThetisError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"thetis {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ProblemDesc(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("csc_ptr", C.c_void_p), ("csc_row", C.c_void_p),
                ("csc_val", C.c_void_p), ("b", C.c_void_p), ("c", C.c_void_p), ("lo", C.c_void_p),
                ("hi", C.c_void_p), ("row_kind", C.c_void_p), ("block_k", C.c_int32),
                ("n_blocks", C.c_int64), ("block_first", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("beta", C.c_double), ("epochs", C.c_int32), ("tol", C.c_double),
                ("refresh_every", C.c_int32), ("step_rule", C.c_int32), ("mode", C.c_int32),
                ("ubar", C.c_void_p), ("xbar", C.c_void_p), ("x0", C.c_void_p), ("mem", C.c_int32),
                ("engine", C.c_int32), ("async_ctas", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("epochs_run", C.c_int32), ("converged", C.c_int32), ("ncolors", C.c_int32),
                ("rho", C.c_double), ("obj", C.c_double), ("infeas", C.c_double), ("fbeta", C.c_double),
                ("updates", C.c_int64), ("solve_ms", C.c_double), ("epoch_ms", C.c_double),
                ("launches_per_epoch", C.c_int32)]


class RoundInfo(C.Structure):
    _fields_ = [("obj", C.c_double), ("repair", C.c_double), ("best_rep", C.c_int32),
                ("near", C.c_int64), ("valid", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1311_2661_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    P, i64, i32, u64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
    st = C.c_int
    sigs = {
        "thetis_last_error": (C.c_char_p, []),
        "thetis_launch_count": (u64, []),
        "thetis_create": (st, [P, i32, u64, P, P]),
        "thetis_build_vc": (st, [i64, i64, P, P, P, i32, u64, P, P]),
        "thetis_build_is": (st, [i64, i64, P, P, P, i32, u64, P, P]),
        "thetis_build_mc": (st, [i64, i64, P, P, P, i32, P, i32, u64, P, P]),
        "thetis_build_sc": (st, [i64, i64, P, P, P, i32, u64, P, P]),
        "thetis_build_map": (st, [i64, i64, i32, P, P, P, P, i32, u64, P, P]),
        "thetis_get_sizes": (st, [P, P, P, P, P, P, P]),
        "thetis_solve": (st, [P, P, P]),
        "thetis_round": (st, [P, i32, u64, i32, P, i32, P]),
        "thetis_get_x": (st, [P, P, i32]),
        "thetis_get_slack": (st, [P, P, i32]),
        "thetis_get_colors": (st, [P, P, P]),
        "thetis_sync": (st, [P]),
        "thetis_destroy": (st, [P]),
        "thetis_round_is_static": (st, [i64, i64, P, P, P, P, u64, i32, P, P, P]),
        "thetis_check_labels": (st, [P, i32, P, i32, P, P]),
        "thetis_set_wait_limit": (st, [P, C.c_double, i32]),
        "thetis_batch_latency": (st, [P, P]),
        "thetis_batch_placement": (st, [P, P, P]),
        "thetis_set_batch_shape": (st, [P, i32, i32]),
        "thetis_solve_round_batch": (st, [P, P, u64, i32, P, i32, P, P, P, P]),
        "thetis_server_set_queue_limit": (st, [P, i64, P]),
        "thetis_build_batch": (st, [i32, P, P, P, P, P, P, i32, u64, P, P]),
        "thetis_autotune": (st, [P, P, i32, P, P]),
        "thetis_set_launch_shape": (st, [P, i32, i32]),
        "thetis_server_create": (st, [C.c_size_t, i32, i32, P]),
        "thetis_submit": (st, [P, P, P]),
        "thetis_poll": (st, [P, u64, P, P, P]),
        "thetis_server_stats": (st, [P, P, P, P, P]),
        "thetis_server_destroy": (st, [P]),
        "thetis_round_batch": (st, [P, u64, i32, P, i32, P, P, P]),
        "thetis_batch_info": (st, [P, P, P]),
        "thetis_solve_al": (st, [P, P, i32, C.c_double, P, P, P, P]),
        "thetis_get_duals": (st, [P, P, i32]),
        "thetis_cache_info": (st, [P, P]),
        "thetis_trim_cache": (st, [u64]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def thetis_last_error() -> str:
    m = _lib.thetis_last_error()
    return m.decode() if m else ""


def thetis_launch_count() -> int:
    return int(_lib.thetis_launch_count())


def thetis_cache_info():
    """(reserved, in-use) bytes of the library's device memory pool."""
    r, u = C.c_uint64(), C.c_uint64()
    _check(_lib.thetis_cache_info(C.byref(r), C.byref(u)))
    return int(r.value), int(u.value)


def thetis_trim_cache(keep_bytes=0):
    """Give the pool's unused reserve back until at most keep_bytes stay reserved."""
    _check(_lib.thetis_trim_cache(int(keep_bytes)))


def _check(st, allow=(THETIS_OK,)):
    if st not in allow:
        raise ThetisError(st, thetis_last_error())
    return st


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Args:
    """Collects array pointers for one call and checks they share one memory space."""

    def __init__(self):
        self.keep = []
        self.mem = None

    def __call__(self, a, dtype):
        if a is None:
            return None
        if _is_torch(a):
            import torch

            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.float32: torch.float32,
                   np.uint8: torch.uint8}[dtype]
            t = a.to(tdt).contiguous()
            mem = MEM_DEVICE if t.is_cuda else MEM_HOST
            self.keep.append(t)
            ptr = t.data_ptr()
        else:
            arr = np.ascontiguousarray(a, dtype=dtype)
            self.keep.append(arr)
            mem = MEM_HOST
            ptr = arr.ctypes.data
        if self.mem is None:
            self.mem = mem
        elif self.mem != mem:
            raise ValueError("all arrays of one call must live in the same memory space")
        return ptr

    @property
    def memspace(self):
        return MEM_HOST if self.mem is None else self.mem


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Handle:
    """Owns a thetis_handle; destroyed with the object."""

    def __init__(self, ptr, n_vertices=None, kind=None):
        self._h = ptr
        self.n_vertices = n_vertices
        self.kind = kind
        self.sizes = thetis_get_sizes(self)

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            _lib.thetis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience methods
    def solve(self, **kw):
        return thetis_solve(self, **kw)

    def solve_al(self, **kw):
        return thetis_solve_al(self, **kw)

    def duals(self):
        return thetis_get_duals(self)

    @property
    def round_kind(self):
        return {"vc": ROUND_VC, "is": ROUND_IS, "mc": ROUND_MC, "sc": ROUND_SC, "map": ROUND_MAP}[self.kind]

    def round(self, kind=None, **kw):
        return thetis_round(self, self.round_kind if kind is None else kind, **kw)

    def check_labels(self, labels, kind=None):
        return thetis_check_labels(self, labels, kind)

    def get_x(self, out=None):
        return thetis_get_x(self, out)

    def get_slack(self, out=None):
        return thetis_get_slack(self, out)

    def colors(self):
        return thetis_get_colors(self)


def thetis_get_sizes(h: Handle):
    vals = [C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()]
    _check(_lib.thetis_get_sizes(h.ptr, *[C.byref(v) for v in vals]))
    return dict(rows=vals[0].value, struct_cols=vals[1].value, slack_cols=vals[2].value,
                free_coords=vals[3].value, nnz=vals[4].value, ncolors=vals[5].value)


def _build(fn, kind, n, eu, ev, weights, seed, stream, k=None, terminals=None):
    A = _Args()
    m = int(eu.shape[0])
    peu, pev = A(eu, np.int32), A(ev, np.int32)
    pw = A(weights, np.float32)
    out = C.c_void_p()
    if kind == "mc":
        pt = A(terminals, np.int32)
        st = fn(n, m, peu, pev, pw, int(k), pt, A.memspace, seed, _stream_ptr(stream), C.byref(out))
    else:
        st = fn(n, m, peu, pev, pw, A.memspace, seed, _stream_ptr(stream), C.byref(out))
    _check(st)
    return Handle(out.value, n_vertices=n, kind=kind)


def thetis_build_vc(n, eu, ev, w, seed=0, stream=None) -> Handle:
    return _build(_lib.thetis_build_vc, "vc", int(n), eu, ev, w, seed, stream)


def thetis_build_is(n, eu, ev, w, seed=0, stream=None) -> Handle:
    return _build(_lib.thetis_build_is, "is", int(n), eu, ev, w, seed, stream)


def thetis_build_mc(n, eu, ev, ce, k, terminals, seed=0, stream=None) -> Handle:
    return _build(_lib.thetis_build_mc, "mc", int(n), eu, ev, ce, seed, stream, k=k, terminals=terminals)


def thetis_build_sc(n_elements, set_ptr, set_elems, cost, seed=0, stream=None) -> Handle:
    """Set cover (sets = columns, elements = rows); labels of a rounding mark sets."""
    A = _Args()
    pp = A(set_ptr, np.int64)
    pe = A(set_elems, np.int32)
    pc = A(cost, np.float32)
    n_sets = int(set_ptr.shape[0]) - 1
    out = C.c_void_p()
    _check(_lib.thetis_build_sc(int(n_elements), n_sets, pp, pe, pc, A.memspace, seed, _stream_ptr(stream),
                                C.byref(out)))
    return Handle(out.value, n_vertices=n_sets, kind="sc")


def thetis_build_map(n, k, eu, ev, theta_node, theta_edge, seed=0, stream=None) -> Handle:
    """Pairwise MAP as the local-polytope LP; labels of a rounding are variable labels."""
    A = _Args()
    m = int(eu.shape[0])
    peu, pev = A(eu, np.int32), A(ev, np.int32)
    ptn, pte = A(theta_node, np.float32), A(theta_edge, np.float32)
    out = C.c_void_p()
    _check(_lib.thetis_build_map(int(n), m, int(k), peu, pev, ptn, pte, A.memspace, seed, _stream_ptr(stream),
                                 C.byref(out)))
    return Handle(out.value, n_vertices=int(n), kind="map")


def thetis_create(m, n, csc_ptr, csc_row, b, c, lo, hi, row_kind, csc_val=None, block_k=1, block_first=None,
                  seed=0, stream=None) -> Handle:
    A = _Args()
    d = ProblemDesc()
    d.m, d.n = int(m), int(n)
    d.csc_ptr = A(csc_ptr, np.int64)
    d.csc_row = A(csc_row, np.int32)
    d.csc_val = A(csc_val, np.float32)
    d.b, d.c = A(b, np.float32), A(c, np.float32)
    d.lo, d.hi = A(lo, np.float32), A(hi, np.float32)
    d.row_kind = A(row_kind, np.uint8)
    d.block_k = int(block_k)
    d.n_blocks = 0 if block_first is None else int(len(block_first))
    d.block_first = A(block_first, np.int64)
    out = C.c_void_p()
    _check(_lib.thetis_create(C.byref(d), A.memspace, seed, _stream_ptr(stream), C.byref(out)))
    return Handle(out.value, kind="general")


def thetis_solve(h: Handle, beta=1e2, epochs=50, tol=0.0, refresh_every=10, step_rule=0, mode=MODE_COLORED,
                 ubar=None, xbar=None, x0=None, engine=0, async_ctas=0):
    A = _Args()
    p = Params()
    p.beta, p.epochs, p.tol = float(beta), int(epochs), float(tol)
    p.refresh_every, p.step_rule, p.mode = int(refresh_every), int(step_rule), int(mode)
    p.ubar, p.xbar, p.x0 = A(ubar, np.float32), A(xbar, np.float32), A(x0, np.float32)
    p.mem = A.memspace
    p.engine = int(engine)
    p.async_ctas = int(async_ctas)
    info = SolveInfo()
    st = _check(_lib.thetis_solve(h.ptr, C.byref(p), C.byref(info)), allow=(THETIS_OK, THETIS_NOT_CONVERGED))
    return dict(status=st, epochs_run=info.epochs_run, converged=bool(info.converged), ncolors=info.ncolors,
                rho=info.rho, obj=info.obj, infeas=info.infeas, fbeta=info.fbeta, updates=info.updates,
                solve_ms=info.solve_ms, epoch_ms=info.epoch_ms, launches_per_epoch=info.launches_per_epoch)


def thetis_solve_al(h: Handle, beta=1e2, epochs=50, tol=0.0, refresh_every=10, outer=5, beta_growth=1.0,
                    step_rule=0, mode=MODE_COLORED, ubar=None, xbar=None, x0=None, engine=0):
    """Augmented-Lagrangian outer loop; returns (info of the last inner solve,
    dict of per-outer arrays infeas / obj / rho)."""
    A = _Args()
    p = Params()
    p.beta, p.epochs, p.tol = float(beta), int(epochs), float(tol)
    p.refresh_every, p.step_rule, p.mode = int(refresh_every), int(step_rule), int(mode)
    p.ubar, p.xbar, p.x0 = A(ubar, np.float32), A(xbar, np.float32), A(x0, np.float32)
    p.mem = A.memspace
    p.engine = int(engine)
    info = SolveInfo()
    hist = {k: np.zeros(int(outer), np.float64) for k in ("infeas", "obj", "rho")}
    st = _check(_lib.thetis_solve_al(h.ptr, C.byref(p), int(outer), float(beta_growth), C.byref(info),
                                     hist["infeas"].ctypes.data, hist["obj"].ctypes.data, hist["rho"].ctypes.data),
                allow=(THETIS_OK, THETIS_NOT_CONVERGED))
    return dict(status=st, epochs_run=info.epochs_run, converged=bool(info.converged), ncolors=info.ncolors,
                rho=info.rho, obj=info.obj, infeas=info.infeas, fbeta=info.fbeta, updates=info.updates,
                solve_ms=info.solve_ms, epoch_ms=info.epoch_ms,
                launches_per_epoch=info.launches_per_epoch), hist


def thetis_get_duals(h: Handle, out=None):
    """The multiplier estimate ubar (original row order)."""
    m = thetis_get_sizes(h)["rows"]
    o = np.zeros(m, np.float32) if out is None else out
    ptr, mem = _out_ptr(o)
    _check(_lib.thetis_get_duals(h.ptr, ptr, mem))
    return o


def thetis_round(h: Handle, kind, seed=0, reps=10, out=None):
    """Returns (labels, info).  ``out`` may be a CUDA uint8 tensor (labels stay on the device)."""
    info = RoundInfo()
    if out is None:
        lab = np.zeros(h.n_vertices, np.uint8)
        ptr, mem = lab.ctypes.data, MEM_HOST
    else:
        lab = out
        if _is_torch(out):
            ptr, mem = out.data_ptr(), (MEM_DEVICE if out.is_cuda else MEM_HOST)
        else:
            ptr, mem = out.ctypes.data, MEM_HOST
    st = _lib.thetis_round(h.ptr, int(kind), int(seed), int(reps), ptr, mem, C.byref(info))
    if st == THETIS_E_REPAIR:
        return None, dict(status=st, repair=info.repair, valid=False)
    _check(st)
    return lab, dict(status=st, obj=info.obj, repair=info.repair, best_rep=info.best_rep, near=info.near,
                     valid=bool(info.valid))


def _out_ptr(out):
    if _is_torch(out):
        return out.data_ptr(), (MEM_DEVICE if out.is_cuda else MEM_HOST)
    return out.ctypes.data, MEM_HOST


def thetis_autotune(h: Handle, beta=1e2, step_rule=0, trial_epochs=3):
    """Pick and apply the sweep's launch shape; returns (small_group, ctas_per_sm)."""
    p = Params()
    p.beta, p.step_rule, p.refresh_every = float(beta), int(step_rule), 10
    g, k = C.c_int32(), C.c_int32()
    _check(_lib.thetis_autotune(h.ptr, C.byref(p), int(trial_epochs), C.byref(g), C.byref(k)))
    return g.value, k.value


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int64), ("m", C.c_int64), ("eu", C.c_void_p), ("ev", C.c_void_p),
                ("w", C.c_void_p), ("ce", C.c_void_p), ("k", C.c_int32), ("terminals", C.c_void_p),
                ("beta", C.c_double), ("epochs", C.c_int32), ("tol", C.c_double), ("refresh_every", C.c_int32),
                ("seed", C.c_uint64), ("reps", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("obj", C.c_double), ("valid", C.c_int32), ("epochs_run", C.c_int32),
                ("rho", C.c_double), ("queue_ms", C.c_double), ("service_ms", C.c_double),
                ("latency_ms", C.c_double), ("batch_size", C.c_int32), ("message", C.c_char * 160)]


class Server:
    """thetis_server: continuous-batching request server (host arrays only)."""

    def __init__(self, budget_bytes=120 << 30, workers=4, max_batch=64):
        h = C.c_void_p()
        _check(_lib.thetis_server_create(int(budget_bytes), int(workers), int(max_batch), C.byref(h)))
        self._h = h.value
        self._sizes = {}

    def submit(self, kind, g, beta=1e2, epochs=1000, tol=1e-3, refresh_every=10, seed=0, reps=10):
        """kind in {"vc", "is", "mc"}; g a synth.Graph.  Returns the request id."""
        q = Request()
        q.kind = {"vc": ROUND_VC, "is": ROUND_IS, "mc": ROUND_MC}[kind]
        q.n, q.m = int(g.n), int(g.m)
        keep = [np.ascontiguousarray(g.eu, np.int32), np.ascontiguousarray(g.ev, np.int32)]
        q.eu, q.ev = keep[0].ctypes.data, keep[1].ctypes.data
        if kind == "mc":
            ce = np.ascontiguousarray(g.ce, np.float32)
            t = np.ascontiguousarray(g.terminals, np.int32)
            keep += [ce, t]
            q.ce, q.terminals, q.k = ce.ctypes.data, t.ctypes.data, int(len(t))
        else:
            w = np.ascontiguousarray(g.w, np.float32)
            keep.append(w)
            q.w = w.ctypes.data
        q.beta, q.epochs, q.tol, q.refresh_every = float(beta), int(epochs), float(tol), int(refresh_every)
        q.seed, q.reps = int(seed), int(reps)
        rid = C.c_uint64()
        _check(_lib.thetis_submit(self._h, C.byref(q), C.byref(rid)))
        self._sizes[rid.value] = (int(g.n), int(g.n) * (q.k if kind == "mc" else 1))
        return rid.value

    def set_queue_limit(self, max_queued):
        """Refuse submits while max_queued requests wait (0: no limit); returns
        the number refused so far."""
        ref = C.c_int64()
        _check(_lib.thetis_server_set_queue_limit(self._h, int(max_queued), C.byref(ref)))
        return int(ref.value)

    def poll(self, rid):
        """None while pending; else (labels, x, result dict)."""
        n, nx = self._sizes[rid]
        lab = np.empty(n, np.uint8)
        x = np.empty(nx, np.float32)
        res = Result()
        st = _lib.thetis_poll(self._h, C.c_uint64(rid), lab.ctypes.data, x.ctypes.data, C.byref(res))
        if st == THETIS_PENDING:
            return None
        _check(st)
        del self._sizes[rid]
        info = {f: getattr(res, f) for f, _ in Result._fields_}
        info["message"] = res.message.decode(errors="replace")
        return lab, x, info

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        _check(_lib.thetis_server_stats(self._h, *[C.byref(a) for a in v]))
        return dict(submitted=v[0].value, completed=v[1].value, queued=v[2].value, in_flight_bytes=v[3].value)

    def close(self):
        if self._h:
            _lib.thetis_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def thetis_server_create(budget_bytes=120 << 30, workers=4, max_batch=64):
    return Server(budget_bytes, workers, max_batch)


def thetis_submit(server: Server, kind, g, **kw):
    return server.submit(kind, g, **kw)


def thetis_poll(server: Server, rid):
    return server.poll(rid)


def thetis_server_stats(server: Server):
    return server.stats()


def thetis_server_set_queue_limit(server: Server, max_queued):
    return server.set_queue_limit(max_queued)


def thetis_server_destroy(server: Server):
    server.close()


def thetis_set_launch_shape(h: Handle, small_group, ctas_per_sm=0):
    _check(_lib.thetis_set_launch_shape(h.ptr, int(small_group), int(ctas_per_sm)))


def thetis_build_batch(kinds, vertex_offset, edge_offset, eu, ev, w, seed=0, stream=None) -> Handle:
    """A batch of independent VC / IS LPs as one handle.  kinds[t] is ROUND_VC or
    ROUND_IS; eu / ev hold instance-local endpoints, concatenated; offsets have
    count + 1 entries."""
    A = _Args()
    count = int(len(kinds))
    pk = A(kinds, np.uint8)
    pn, pe = A(vertex_offset, np.int64), A(edge_offset, np.int64)
    peu, pev, pw = A(eu, np.int32), A(ev, np.int32), A(w, np.float32)
    out = C.c_void_p()
    _check(_lib.thetis_build_batch(count, pk, pn, pe, peu, pev, pw, A.memspace, seed, _stream_ptr(stream),
                                   C.byref(out)))
    nv = int(vertex_offset[-1])
    h = Handle(out.value, n_vertices=nv, kind="batch")
    h.count = count
    return h


def thetis_build_batch_graphs(items, seed=0, stream=None, device=False) -> Handle:
    """Convenience: items = [(kind, synth.Graph), ...] with kind "vc" or "is"."""
    kinds = np.array([ROUND_VC if k == "vc" else ROUND_IS for k, _ in items], np.uint8)
    noff = np.concatenate([[0], np.cumsum([g.n for _, g in items])]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum([g.m for _, g in items])]).astype(np.int64)
    eu = np.concatenate([g.eu for _, g in items]).astype(np.int32)
    ev = np.concatenate([g.ev for _, g in items]).astype(np.int32)
    w = np.concatenate([g.w for _, g in items]).astype(np.float32)
    if device:
        import torch

        dv = lambda a: torch.from_numpy(a).cuda()
        return thetis_build_batch(dv(kinds), dv(noff), dv(eoff), dv(eu), dv(ev), dv(w), seed=seed, stream=stream)
    return thetis_build_batch(kinds, noff, eoff, eu, ev, w, seed=seed, stream=stream)


def thetis_solve_round_batch(h: Handle, seed=0, reps=10, out=None, beta=1e2, epochs=50, tol=0.0, refresh_every=10,
                             step_rule=0, engine=0):
    """Solve a batch and round every instance (in the instance kernel as each
    stops).  Returns (info, labels, obj[count], status[count], best_rep[count])."""
    A = _Args()
    p = Params()
    p.beta, p.epochs, p.tol = float(beta), int(epochs), float(tol)
    p.refresh_every, p.step_rule, p.mode = int(refresh_every), int(step_rule), MODE_COLORED
    p.mem = MEM_HOST
    p.engine = int(engine)
    count = h.count
    obj = np.zeros(count, np.float64)
    status = np.zeros(count, np.int32)
    best = np.zeros(count, np.int32)
    lab = np.zeros(h.n_vertices, np.uint8) if out is None else out
    ptr, mem = _out_ptr(lab)
    info = SolveInfo()
    st = _check(_lib.thetis_solve_round_batch(h.ptr, C.byref(p), int(seed), int(reps), ptr, mem, obj.ctypes.data,
                                              status.ctypes.data, best.ctypes.data, C.byref(info)),
                allow=(THETIS_OK, THETIS_NOT_CONVERGED))
    inf = dict(status=st, epochs_run=info.epochs_run, converged=bool(info.converged), ncolors=info.ncolors,
               rho=info.rho, obj=info.obj, infeas=info.infeas, fbeta=info.fbeta, updates=info.updates,
               solve_ms=info.solve_ms, epoch_ms=info.epoch_ms, launches_per_epoch=info.launches_per_epoch)
    return inf, lab, obj, status, best


def thetis_round_batch(h: Handle, seed=0, reps=10, out=None):
    """Returns (labels, obj[count], status[count], best_rep[count])."""
    count = h.count
    obj = np.zeros(count, np.float64)
    status = np.zeros(count, np.int32)
    best = np.zeros(count, np.int32)
    lab = np.zeros(h.n_vertices, np.uint8) if out is None else out
    ptr, mem = _out_ptr(lab)
    _check(_lib.thetis_round_batch(h.ptr, int(seed), int(reps), ptr, mem, obj.ctypes.data, status.ctypes.data,
                                   best.ctypes.data))
    return lab, obj, status, best


def thetis_batch_info(h: Handle):
    """Per-instance (epochs, rho) of the last solve of a batch handle."""
    ep = np.zeros(h.count, np.int32)
    rho = np.zeros(h.count, np.float64)
    _check(_lib.thetis_batch_info(h.ptr, ep.ctypes.data, rho.ctypes.data))
    return ep, rho


def thetis_set_wait_limit(h: Handle, limit_ms=2000.0, missing_ctas=0):
    """Time limit of the persistent sweep's bounded waits; missing_ctas > 0 makes
    them wait for CTAs that never arrive (tests the THETIS_E_TIMEOUT path)."""
    _check(_lib.thetis_set_wait_limit(h.ptr, float(limit_ms), int(missing_ctas)))


def thetis_check_labels(h: Handle, labels, kind=None):
    """Exact validity and objective of a caller's integral solution: returns
    (valid, obj).  kind defaults to the handle's own rounding kind."""
    A = _Args()
    ptr = A(labels, np.uint8)
    valid, obj = C.c_int32(), C.c_double()
    k = h.round_kind if kind is None else kind
    _check(_lib.thetis_check_labels(h.ptr, int(k), ptr, A.memspace, C.byref(valid), C.byref(obj)))
    return bool(valid.value), float(obj.value)


def thetis_set_batch_shape(h: Handle, lanes_per_column=1, clusters=0):
    """Launch shape of the instance-resident batch engine (see include/thetis.h)."""
    _check(_lib.thetis_set_batch_shape(h.ptr, int(lanes_per_column), int(clusters)))


def thetis_batch_latency(h: Handle):
    """Per instance: ms from the start of the last solve until its result was final."""
    out = np.zeros(h.count, np.float64)
    _check(_lib.thetis_batch_latency(h.ptr, out.ctypes.data))
    return out


def thetis_batch_placement(h: Handle):
    """Per instance: (ms from the start of the last solve until its CTA /
    cluster began, CTAs of that CTA / cluster); zeros after a union sweep."""
    start = np.zeros(h.count, np.float64)
    ctas = np.zeros(h.count, np.int32)
    _check(_lib.thetis_batch_placement(h.ptr, start.ctypes.data, ctas.ctypes.data))
    return start, ctas


def thetis_round_is_static(n, eu, ev, w, x, labels_out, seed=0, reps=10, stream=None):
    """Independent-set rounding with no device allocation (scratch is a fixed
    64 MiB static device array).  eu, ev (int32), w, x (float32) and labels_out
    (uint8) must already be contiguous CUDA tensors of those types: nothing is
    converted or copied here, so the call allocates nothing and the labels land
    in labels_out itself.  Returns the info dict.  Requires n * reps <=
    33,488,624."""
    import torch

    want = ((eu, torch.int32, "eu"), (ev, torch.int32, "ev"), (w, torch.float32, "w"),
            (x, torch.float32, "x"), (labels_out, torch.uint8, "labels_out"))
    for t, dt, name in want:
        if not (_is_torch(t) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"thetis_round_is_static: {name} must be a contiguous CUDA tensor of {dt}")
    n = int(n)
    if eu.shape != ev.shape or eu.dim() != 1:
        raise ValueError("thetis_round_is_static: eu and ev must be 1-D of the same length")
    for t, name in ((w, "w"), (x, "x"), (labels_out, "labels_out")):
        if t.numel() < n:
            raise ValueError(f"thetis_round_is_static: {name} holds fewer than n = {n} elements")
    info = RoundInfo()
    st = _lib.thetis_round_is_static(n, int(eu.shape[0]), eu.data_ptr(), ev.data_ptr(), w.data_ptr(),
                                     x.data_ptr(), int(seed), int(reps), labels_out.data_ptr(),
                                     C.byref(info), _stream_ptr(stream))
    _check(st)
    return dict(status=st, obj=info.obj, repair=info.repair, best_rep=info.best_rep, near=info.near,
                valid=bool(info.valid))


def thetis_get_x(h: Handle, out=None):
    """Structural part of the iterate, original column order (FP32)."""
    if out is None:
        out = np.zeros(h.sizes["struct_cols"], np.float32)
    ptr, mem = _out_ptr(out)
    _check(_lib.thetis_get_x(h.ptr, ptr, mem))
    return out


def thetis_get_slack(h: Handle, out=None):
    """Slack part of the iterate, one value per GE/LE row in row order."""
    if out is None:
        out = np.zeros(h.sizes["slack_cols"], np.float32)
    ptr, mem = _out_ptr(out)
    _check(_lib.thetis_get_slack(h.ptr, ptr, mem))
    return out


def thetis_get_colors(h: Handle):
    nu = C.c_int64()
    _check(_lib.thetis_get_colors(h.ptr, None, C.byref(nu)))
    out = np.zeros(nu.value, np.int32)
    _check(_lib.thetis_get_colors(h.ptr, out.ctypes.data, C.byref(nu)))
    return out


def thetis_sync(h: Handle):
    _check(_lib.thetis_sync(h.ptr))


def thetis_destroy(h: Handle):
    h.close()
