"""FP64 serial oracle of the SCD + LP-rounding method (arXiv 1311.2661).

TEST INFRASTRUCTURE ONLY: this package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg,
and by nothing else.  The CUDA library never loads it and shares no code with
it.  The arithmetic lives in ``thetis_oracle.c`` (plain C, FP64, serial); this
module only compiles it with gcc and marshals numpy arrays through ctypes.

Parity status of each function (the pins are in tests/test_oracle_*.py):
  build_vc / build_is / build_mc   pinned (LP optimum vs scipy HiGHS, closed forms)
  color                            pinned (networkx greedy_color, validity)
  project_simplex                  pinned (bisection + brute-force KKT)
  solve                            pinned (single-edge closed form, active-set
                                   enumeration of x(beta), Thm. 1 bounds,
                                   monotone f_beta, LCP)
  checks                           pinned (through solve pins and closed forms)
  solve_al                         pinned (convergence to LP optima and strong
                                   duality on closed-form / HiGHS instances,
                                   infeasibility far below the fixed-beta penalty)
  round_vc / round_is / round_mc   pinned (validity, 2x bound, exact selection
                                   probabilities, CKR expectation for k=2)
  map_lp, round_map                pinned (LP tight = Viterbi on chains,
                                   brute force on one edge / small cycles,
                                   relaxation bound, AL + rounding = MAP)
  set_cover, round_sc(_rand)       pinned (equal to the VC rounding when every
                                   element lies in two sets, f-approximation
                                   against LP* / brute-force IP*, pick
                                   frequencies, validity)
  rng                              pinned (published splitmix64 outputs)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "thetis_oracle.c")
_LIB = os.path.join(_HERE, "libthetis_oracle.so")
_lock = threading.Lock()
_lib = None

ROW_EQ, ROW_GE, ROW_LE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no arch-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Info(C.Structure):
    _fields_ = [("epochs_run", C.c_int32), ("ncolors", C.c_int32), ("converged", C.c_int32),
                ("rho", C.c_double), ("obj", C.c_double), ("infeas", C.c_double),
                ("fbeta", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("beta", C.c_double), ("epochs", C.c_int32), ("tol", C.c_double),
                ("refresh_every", C.c_int32), ("step_rule", C.c_int32), ("seed", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, u64, dbl = C.c_int64, C.c_int32, C.c_uint64, C.c_double
        sig = {
            "or_splitmix64_at": (u64, [u64, u64]),
            "or_rng_u64": (u64, [u64, u64, u64, u64]),
            "or_rng_uniform": (dbl, [u64, u64, u64, u64]),
            "or_free": (None, [P]),
            "or_num_rows": (i64, [P]), "or_num_cols": (i64, [P]), "or_num_struct": (i64, [P]),
            "or_num_units": (i64, [P]), "or_nnz": (i64, [P]), "or_num_free_coords": (i64, [P]),
            "or_create": (P, [i64, i64, P, P, P, P, P, P, P, P, i32, i64, P]),
            "or_build_vc": (P, [i64, i64, P, P, P]),
            "or_build_is": (P, [i64, i64, P, P, P]),
            "or_build_mc": (P, [i64, i64, P, P, P, i32, P]),
            "or_export": (None, [P, P, P, P, P, P, P, P]),
            "or_export_units": (None, [P, P, P, P]),
            "or_priority_order": (None, [P, u64, P]),
            "or_color": (i32, [P, u64, P]),
            "or_project_simplex": (None, [i32, P, P]),
            "or_residual": (None, [P, P, P]),
            "or_checks": (None, [P, P, dbl, P, P, P]),
            "or_initial_x": (None, [P, P]),
            "or_solve": (C.c_int, [P, P, P, i32, P, P, P, P, P, P]),
            "or_epoch_fbeta_steps": (None, [P, dbl, i32, P, i32, P, P]),
            "or_round_vc": (C.c_int, [P, P, P, P, P, P, dbl]),
            "or_round_is_rep": (None, [P, P, u64, i32, P]),
            "or_round_is": (C.c_int, [P, P, u64, i32, P, P, P, P]),
            "or_round_mc_rep": (None, [P, P, u64, i32, P]),
            "or_round_mc": (C.c_int, [P, P, u64, i32, P, P, P]),
            "or_mc_cut_cost": (dbl, [P, P]),
            "or_valid": (C.c_int, [P, P]),
            "or_sc_frequency": (C.c_int32, [P]),
            "or_round_sc": (C.c_int, [P, P, P, P, P, P, C.c_double]),
            "or_round_sc_rand_rep": (None, [P, P, u64, i32, P]),
            "or_round_sc_rand": (C.c_int, [P, P, u64, i32, P, P, P, P]),
            "or_valid_sc": (C.c_int, [P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def splitmix64_at(seed: int, i: int) -> int:
    return int(_load().or_splitmix64_at(seed, i))


def rng_u64(seed, rep, stream, idx) -> int:
    return int(_load().or_rng_u64(seed, rep, stream, idx))


def rng_uniform(seed, rep, stream, idx) -> float:
    return float(_load().or_rng_uniform(seed, rep, stream, idx))


def project_simplex(y) -> np.ndarray:
    y = np.ascontiguousarray(y, np.float64)
    x = np.empty_like(y)
    _load().or_project_simplex(y.shape[0], _p(y), _p(x))
    return x


class OracleLP:
    """A standard-form LP held by the oracle (columns: structural, then one
    slack per inequality row)."""

    def __init__(self, handle, keep=()):
        if not handle:
            raise RuntimeError("oracle build failed")
        self._h = handle
        self._keep = keep
        L = _load()
        self.M = int(L.or_num_rows(handle))
        self.N = int(L.or_num_cols(handle))
        self.Ns = int(L.or_num_struct(handle))
        self.U = int(L.or_num_units(handle))
        self.nnz = int(L.or_nnz(handle))
        self.free_coords = int(L.or_num_free_coords(handle))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_free(h)
            self._h = None

    # -- construction -------------------------------------------------------
    @classmethod
    def vc(cls, n, eu, ev, w):
        eu = np.ascontiguousarray(eu, np.int32); ev = np.ascontiguousarray(ev, np.int32)
        w = np.ascontiguousarray(w, np.float64)
        return cls(_load().or_build_vc(n, eu.shape[0], _p(eu), _p(ev), _p(w)))

    @classmethod
    def is_(cls, n, eu, ev, w):
        eu = np.ascontiguousarray(eu, np.int32); ev = np.ascontiguousarray(ev, np.int32)
        w = np.ascontiguousarray(w, np.float64)
        return cls(_load().or_build_is(n, eu.shape[0], _p(eu), _p(ev), _p(w)))

    @classmethod
    def mc(cls, n, eu, ev, ce, k, terminals):
        eu = np.ascontiguousarray(eu, np.int32); ev = np.ascontiguousarray(ev, np.int32)
        ce = np.ascontiguousarray(ce, np.float64)
        t = np.ascontiguousarray(terminals, np.int32)
        return cls(_load().or_build_mc(n, eu.shape[0], _p(eu), _p(ev), _p(ce), int(k), _p(t)))

    @classmethod
    def general(cls, M, colptr, rowidx, val, b, c, lo, hi, row_kind, block_k=1, block_first=None):
        colptr = np.ascontiguousarray(colptr, np.int64)
        rowidx = np.ascontiguousarray(rowidx, np.int32)
        val = None if val is None else np.ascontiguousarray(val, np.float64)
        b = np.ascontiguousarray(b, np.float64); c = np.ascontiguousarray(c, np.float64)
        lo = np.ascontiguousarray(lo, np.float64); hi = np.ascontiguousarray(hi, np.float64)
        rk = np.ascontiguousarray(row_kind, np.int32)
        bf = None if block_first is None else np.ascontiguousarray(block_first, np.int64)
        nb = 0 if bf is None else bf.shape[0]
        h = _load().or_create(M, colptr.shape[0] - 1, _p(colptr), _p(rowidx), _p(val), _p(b), _p(c),
                              _p(lo), _p(hi), _p(rk), int(block_k), nb, _p(bf))
        return cls(h)

    # -- inspection ---------------------------------------------------------
    def export(self):
        cp = np.empty(self.N + 1, np.int64); ri = np.empty(self.nnz, np.int64)
        av = np.empty(self.nnz, np.float64); b = np.empty(self.M, np.float64)
        c = np.empty(self.N, np.float64); lo = np.empty(self.N, np.float64)
        hi = np.empty(self.N, np.float64)
        _load().or_export(self._h, _p(cp), _p(ri), _p(av), _p(b), _p(c), _p(lo), _p(hi))
        return dict(colptr=cp, rowidx=ri, val=av, b=b, c=c, lo=lo, hi=hi)

    def units(self):
        us = np.empty(self.U, np.int64); ul = np.empty(self.U, np.int32); sx = np.empty(self.U, np.int32)
        _load().or_export_units(self._h, _p(us), _p(ul), _p(sx))
        return us, ul, sx

    def dense_A(self):
        e = self.export()
        A = np.zeros((self.M, self.N))
        for j in range(self.N):
            for q in range(e["colptr"][j], e["colptr"][j + 1]):
                A[e["rowidx"][q], j] += e["val"][q]
        return A

    # -- method -------------------------------------------------------------
    def priority_order(self, seed):
        o = np.empty(self.U, np.int64)
        _load().or_priority_order(self._h, seed, _p(o))
        return o

    def color(self, seed):
        col = np.empty(self.U, np.int32)
        nc = _load().or_color(self._h, seed, _p(col))
        return col, int(nc)

    def initial_x(self):
        x = np.empty(self.N, np.float64)
        _load().or_initial_x(self._h, _p(x))
        return x

    def residual(self, x):
        x = np.ascontiguousarray(x, np.float64)
        r = np.empty(self.M, np.float64)
        _load().or_residual(self._h, _p(x), _p(r))
        return r

    def checks(self, x, beta, ubar=None, xbar=None):
        x = np.ascontiguousarray(x, np.float64)
        ub = None if ubar is None else np.ascontiguousarray(ubar, np.float64)
        xb = None if xbar is None else np.ascontiguousarray(xbar, np.float64)
        info = _Info()
        _load().or_checks(self._h, _p(x), float(beta), _p(ub), _p(xb), C.byref(info))
        return dict(rho=info.rho, obj=info.obj, infeas=info.infeas, fbeta=info.fbeta)

    def solve(self, beta=1e2, epochs=50, tol=0.0, refresh_every=10, step_rule=0, seed=0,
              color=None, ubar=None, xbar=None, x0=None):
        if color is None:
            color, nc = self.color(seed)
        else:
            color = np.ascontiguousarray(color, np.int32)
            nc = int(color.max()) + 1 if color.size else 0
        x = self.initial_x() if x0 is None else np.array(x0, np.float64, copy=True)
        ub = None if ubar is None else np.ascontiguousarray(ubar, np.float64)
        xb = None if xbar is None else np.ascontiguousarray(xbar, np.float64)
        prm = _Params(float(beta), int(epochs), float(tol), int(refresh_every), int(step_rule), int(seed))
        info = _Info()
        maxt = epochs // max(refresh_every, 1) + 2
        trace = np.zeros((maxt, 4), np.float64)
        nt = C.c_int32(0)
        _load().or_solve(self._h, C.byref(prm), _p(color), nc, _p(ub), _p(xb), _p(x), C.byref(info),
                         _p(trace), C.byref(nt))
        return x, dict(epochs_run=info.epochs_run, ncolors=info.ncolors, converged=bool(info.converged),
                       rho=info.rho, obj=info.obj, infeas=info.infeas, fbeta=info.fbeta,
                       trace=trace[: nt.value].copy())

    def solve_al(self, beta=1e2, epochs=50, tol=0.0, refresh_every=10, outer=5, beta_growth=1.0, step_rule=0,
                 seed=0, color=None, ubar=None, xbar=None, x0=None):
        """Augmented-Lagrangian outer loop of Sec. 3.4 (a proximal method of
        multipliers): solve eq. QP at (ubar, xbar, beta) from the previous
        iterate, then ubar <- ubar - beta (A x - b), xbar <- x and
        beta <- beta * beta_growth.  Returns (x, ubar after the last update,
        per-outer list of the inner solve's info with its beta)."""
        ub = np.zeros(self.M) if ubar is None else np.array(ubar, np.float64, copy=True)
        xb = np.zeros(self.N) if xbar is None else np.array(xbar, np.float64, copy=True)
        x = x0
        hist = []
        for _ in range(outer):
            x, info = self.solve(beta=beta, epochs=epochs, tol=tol, refresh_every=refresh_every,
                                 step_rule=step_rule, seed=seed, color=color, ubar=ub, xbar=xb, x0=x)
            info["beta"] = beta
            hist.append(info)
            ub = ub - beta * self.residual(x)
            xb = x.copy()
            beta *= beta_growth
        return x, ub, hist

    def fbeta_steps(self, x, beta, color, step_rule=0):
        x = np.array(x, np.float64, copy=True)
        color = np.ascontiguousarray(color, np.int32)
        f = np.empty(self.U, np.float64)
        _load().or_epoch_fbeta_steps(self._h, float(beta), int(step_rule), _p(color),
                                     int(color.max()) + 1, _p(x), _p(f))
        return f, x

    # -- rounding (x = the structural part, original column order) ----------
    def round_vc(self, x, band=1e-4):
        x = np.ascontiguousarray(x, np.float64)
        n = self._n_vertices()
        lab = np.zeros(n, np.uint8)
        eps = C.c_double(); obj = C.c_double(); near = C.c_int64()
        st = _load().or_round_vc(self._h, _p(x), _p(lab), C.byref(eps), C.byref(obj), C.byref(near), band)
        return dict(status=st, labels=lab, eps=eps.value, obj=obj.value, near=near.value)

    def round_is_rep(self, xt, seed, rep):
        xt = np.ascontiguousarray(xt, np.float64)
        keep = np.zeros(xt.shape[0], np.uint8)
        _load().or_round_is_rep(self._h, _p(xt), int(seed), int(rep), _p(keep))
        return keep

    def round_is(self, x, seed, reps=10):
        x = np.ascontiguousarray(x, np.float64)
        n = self._n_vertices()
        lab = np.zeros(n, np.uint8)
        alpha = C.c_double(); obj = C.c_double(); br = C.c_int32()
        st = _load().or_round_is(self._h, _p(x), int(seed), int(reps), _p(lab), C.byref(alpha),
                                 C.byref(obj), C.byref(br))
        return dict(status=st, labels=lab, alpha=alpha.value, obj=obj.value, best_rep=br.value)

    def round_mc_rep(self, x, seed, rep):
        x = np.ascontiguousarray(x, np.float64)
        lab = np.zeros(self._n_vertices(), np.uint8)
        _load().or_round_mc_rep(self._h, _p(x), int(seed), int(rep), _p(lab))
        return lab

    def round_mc(self, x, seed, reps=10):
        x = np.ascontiguousarray(x, np.float64)
        lab = np.zeros(self._n_vertices(), np.uint8)
        obj = C.c_double(); br = C.c_int32()
        st = _load().or_round_mc(self._h, _p(x), int(seed), int(reps), _p(lab), C.byref(obj), C.byref(br))
        return dict(status=st, labels=lab, obj=obj.value, best_rep=br.value)

    def mc_cut_cost(self, labels):
        labels = np.ascontiguousarray(labels, np.uint8)
        return float(_load().or_mc_cut_cost(self._h, _p(labels)))

    # -- set cover (App. B.1); x = the set columns, original order ------------
    @classmethod
    def set_cover(cls, n_elements, set_ptr, set_elems, cost):
        """Covering LP of a set system: min c'x, sum_{s holds a} x_s >= 1 for
        every element a, 0 <= x <= 1 (rows = elements, columns = sets)."""
        set_ptr = np.ascontiguousarray(set_ptr, np.int64)
        k = set_ptr.shape[0] - 1
        lp = cls.general(int(n_elements), set_ptr, set_elems, None, np.ones(n_elements), np.asarray(cost, np.float64),
                         np.zeros(k), np.ones(k), np.full(n_elements, ROW_GE, np.int32))
        lp.n_sets = k
        return lp

    def sc_frequency(self):
        return int(_load().or_sc_frequency(self._h))

    def round_sc(self, x, band=1e-4):
        x = np.ascontiguousarray(x, np.float64)
        lab = np.zeros(self.n_sets, np.uint8)
        eps = C.c_double(); obj = C.c_double(); near = C.c_int64()
        st = _load().or_round_sc(self._h, _p(x), _p(lab), C.byref(eps), C.byref(obj), C.byref(near), band)
        return dict(status=st, labels=lab, eps=eps.value, obj=obj.value, near=near.value)

    def round_sc_rand_rep(self, xt, seed, rep):
        xt = np.ascontiguousarray(xt, np.float64)
        take = np.zeros(self.n_sets, np.uint8)
        _load().or_round_sc_rand_rep(self._h, _p(xt), int(seed), int(rep), _p(take))
        return take

    def round_sc_rand(self, x, seed, reps=10):
        x = np.ascontiguousarray(x, np.float64)
        lab = np.zeros(self.n_sets, np.uint8)
        eps = C.c_double(); obj = C.c_double(); br = C.c_int32()
        st = _load().or_round_sc_rand(self._h, _p(x), int(seed), int(reps), _p(lab), C.byref(eps), C.byref(obj),
                                      C.byref(br))
        return dict(status=st, labels=lab, eps=eps.value, obj=obj.value, best_rep=br.value)

    def valid_sc(self, labels):
        labels = np.ascontiguousarray(labels, np.uint8)
        return bool(_load().or_valid_sc(self._h, _p(labels)))

    # -- pairwise MAP (Sec. 4.1, the local-polytope LP with node rounding) ---
    @classmethod
    def map_lp(cls, n, k, eu, ev, theta_node, theta_edge):
        """Local-polytope LP of pairwise MAP, as a minimisation: node marginals
        mu_i(a) (column i*k + a, one simplex block per variable) and edge
        marginals mu_e(a, b) (column n*k + e*k*k + a*k + b, in [0, 1]); for
        every edge e = (u, v) and label a the rows
          sum_b mu_e(a, b) - mu_u(a) = 0     (row 2*e*k + a)
          sum_a mu_e(a, b) - mu_v(b) = 0     (row 2*e*k + k + b);
        costs -theta (the score is maximised)."""
        eu = np.asarray(eu, np.int64); ev = np.asarray(ev, np.int64)
        E = eu.shape[0]
        th_n = np.asarray(theta_node, np.float64).reshape(n, k)
        th_e = np.asarray(theta_edge, np.float64).reshape(E, k, k)
        Ns, M = n * k + E * k * k, 2 * E * k
        a = np.arange(k)
        # node entries: incidence t = (vertex, edge, side), every label a
        vert = np.concatenate([eu, ev]); edge = np.concatenate([np.arange(E), np.arange(E)])
        side = np.concatenate([np.zeros(E, np.int64), np.ones(E, np.int64)])
        ncol = (vert[:, None] * k + a[None, :]).ravel()
        nrow = (2 * edge[:, None] * k + side[:, None] * k + a[None, :]).ravel()
        # edge entries: column (e, a, b) in rows 2ek + a and 2ek + k + b
        e3 = np.arange(E)[:, None, None]
        ecol = (n * k + e3 * k * k + a[None, :, None] * k + a[None, None, :]).ravel()
        erow_u = (2 * e3 * k + a[None, :, None] + 0 * a[None, None, :]).ravel()
        erow_v = (2 * e3 * k + k + a[None, None, :] + 0 * a[None, :, None]).ravel()
        col = np.concatenate([ncol, ecol, ecol])
        row = np.concatenate([nrow, erow_u, erow_v])
        val = np.concatenate([-np.ones(ncol.shape[0]), np.ones(2 * ecol.shape[0])])
        order = np.argsort(col, kind="stable")
        colptr = np.zeros(Ns + 1, np.int64)
        np.cumsum(np.bincount(col, minlength=Ns), out=colptr[1:])
        rowidx = row[order].astype(np.int32)
        val = val[order]
        c = np.concatenate([-th_n.ravel(), -th_e.ravel()])
        lp = cls.general(M, colptr, rowidx, val, np.zeros(M), c, np.zeros(Ns), np.ones(Ns),
                         np.zeros(M, np.int32), block_k=k, block_first=np.arange(n, dtype=np.int64) * k)
        lp.map_meta = (n, k, eu, ev, th_n, th_e)
        return lp

    def round_map(self, x):
        """Node rounding: every variable takes the label of its largest node
        marginal (ties: lowest label).  Returns labels and the LP objective of
        the integral point (minus the score)."""
        n, k, eu, ev, th_n, th_e = self.map_meta
        mu = np.asarray(x[: n * k], np.float64).reshape(n, k)
        lab = np.argmax(mu, axis=1).astype(np.uint8)
        return dict(labels=lab, obj=self.map_energy(lab))

    def map_energy(self, lab):
        n, k, eu, ev, th_n, th_e = self.map_meta
        lab = np.asarray(lab, np.int64)
        return -(th_n[np.arange(n), lab].sum() + th_e[np.arange(len(eu)), lab[eu], lab[ev]].sum())

    def valid(self, labels):
        labels = np.ascontiguousarray(labels, np.uint8)
        return bool(_load().or_valid(self._h, _p(labels)))

    def _n_vertices(self):
        n = getattr(self, "n_vertices", None)
        if n is None:
            raise RuntimeError("rounding needs a graph-built LP (set n_vertices)")
        return n


def build_problem(kind: str, g, k: int | None = None) -> OracleLP:
    """Oracle standard form for a synth.Graph: kind in {"vc", "is", "mc"}."""
    if kind == "vc":
        lp = OracleLP.vc(g.n, g.eu, g.ev, g.w.astype(np.float64))
    elif kind == "is":
        lp = OracleLP.is_(g.n, g.eu, g.ev, g.w.astype(np.float64))
    elif kind == "mc":
        kk = int(k if k is not None else len(g.terminals))
        lp = OracleLP.mc(g.n, g.eu, g.ev, g.ce.astype(np.float64), kk, g.terminals)
    else:
        raise ValueError(kind)
    lp.n_vertices = g.n
    lp.kind = kind
    return lp
