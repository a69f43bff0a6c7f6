"""FP64 CPU oracle of the PNCG solver (Shen et al., SIGGRAPH 2024) -- TEST INFRASTRUCTURE ONLY.

The arithmetic lives in ``pncg_oracle.c`` (plain C, double precision, serial, summed in index order); this module
compiles it with gcc and wraps it with ctypes.  Only the test-suite, the smoke check and the CPU-baseline leg of
the benchmark may import this package.  It shares no code with the CUDA library, and the library never calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pncg_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "invalid argument", 2: "inverted tet", 3: "penetration", 4: "non-finite", 5: "out of memory"}
PT, EE = 0, 1


class OracleError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"oracle status {status} ({ERRORS.get(status, '?')}): {msg}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction) into oracle/_liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


# energy densities (Sec. 3.1): the paper's Neo-Hookean, stable Neo-Hookean, fixed corotated, as-rigid-as-possible
NH, SNH, FCR, ARAP = 0, 1, 2, 3


class _Params(C.Structure):
    _fields_ = [("nv", C.c_int32), ("nt", C.c_int32), ("rest_x", C.c_void_p), ("tets", C.c_void_p),
                ("youngs_per_tet", C.c_void_p), ("youngs", C.c_double), ("poisson", C.c_double),
                ("density", C.c_double), ("h", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double),
                ("gravity", C.c_double * 3), ("has_plane", C.c_int32), ("plane_n", C.c_double * 3),
                ("plane_o", C.c_double), ("fixed", C.c_void_p), ("beta_rule", C.c_int32), ("pnorm", C.c_int32),
                ("excl_factor", C.c_double), ("model", C.c_int32)]


class _Scalars(C.Structure):
    _fields_ = [("k", C.c_int32), ("dE0", C.c_double), ("beta", C.c_double), ("gp", C.c_double),
                ("pHp", C.c_double), ("pmax", C.c_double), ("alpha_bar", C.c_double), ("alpha_up", C.c_double),
                ("alpha", C.c_double), ("dE", C.c_double), ("restarted", C.c_int32), ("capped", C.c_int32),
                ("n_active", C.c_int32), ("n_plane", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P, I32, D = C.c_void_p, C.c_int32, C.c_double
        sig = {
            "or_last_error": (C.c_char_p, []),
            "or_model_new": (P, [P]),
            "or_model_free": (None, [P]),
            "or_model_sizes": (None, [P, P]),
            "or_model_arrays": (None, [P, P, P, P]),
            "or_surface": (None, [P, P, P, P]),
            "or_barrier_fn": (None, [D, D, P]),
            "or_pair_geometry": (D, [I32, P, P, P]),
            "or_energy": (C.c_int, [P, P, P, P, P]),
            "or_grad_diag": (C.c_int, [P, P, P, P, P, P]),
            "or_grad_diag_scale": (C.c_int, [P, P, P, P, P]),
            "or_pHp": (C.c_int, [P, P, P, P]),
            "or_active_pairs": (C.c_int, [P, P, I32, D, I32, P, P, P, I32, P]),
            "or_ncg_direction": (C.c_int, [I32, P, P, P, P, P, I32, I32, P, P, P]),
            "or_pmax": (D, [I32, P, I32]),
            "or_ncg_alpha": (None, [D, D, D, D, P]),
            "or_iteration": (C.c_int, [P, P, P, P, P, P, P]),
            "or_iteration_split": (C.c_int, [P, I32, P, P, P, P, P, P, P, P]),
            "or_iteration_groups": (C.c_int, [P, I32, P, P, P, P, P, P, P, P]),
            "or_contact_vertices": (C.c_int, [P, P, P]),
            "or_step": (C.c_int, [P, P, P, P, I32, D, P, P]),
            "or_predict": (None, [P, P, P, P, P]),
            "or_intersections": (I32, [P, P]),
            "or_hvp": (C.c_int, [P, P, P, P]),
            "or_adjoint_step": (C.c_int, [P, P, P, P, P, P, P, D, I32, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(st):
    if st != 0:
        raise OracleError(st, _load().or_last_error().decode())


def barrier_fn(d: float, dhat: float):
    """(b, b', b'') of the IPC log barrier at distance d."""
    out = np.zeros(3)
    _load().or_barrier_fn(float(d), float(dhat), _ptr(out))
    return tuple(out)


def pair_geometry(ptype: int, x4):
    """Distance, c[4] and t[3] of a point-triangle (0) or edge-edge (1) primitive pair, x4 = [4,3]."""
    x = _f64(x4, (4, 3))
    c = np.zeros(4)
    t = np.zeros(3)
    d = _load().or_pair_geometry(int(ptype), _ptr(x), _ptr(c), _ptr(t))
    return d, c, t


def ncg_direction(g1, P1, g0, P0, p, k: int, rule: int = 0):
    """PNCG direction: returns (p_new, beta, g^T p_new, restarted).  Arrays are flat, same length."""
    g1, P1, g0, P0 = (_f64(a).ravel() for a in (g1, P1, g0, P0))
    pn = _f64(p).ravel().copy()
    beta, gp, rs = C.c_double(), C.c_double(), C.c_int32()
    _check(_load().or_ncg_direction(len(g1), _ptr(g1), _ptr(P1), _ptr(g0), _ptr(P0), _ptr(pn), int(k), int(rule),
                                    C.byref(beta), C.byref(gp), C.byref(rs)))
    return pn, beta.value, gp.value, bool(rs.value)


def pmax(p, pnorm: int = 0) -> float:
    p = _f64(p).reshape(-1, 3)
    return _load().or_pmax(p.shape[0], _ptr(p), int(pnorm))


def ncg_alpha(gp: float, pHp: float, pmax_: float, dhat: float):
    """(alpha, alpha_bar, alpha_upper, dE, capped) of the single-pass step rule."""
    out = np.zeros(5)
    _load().or_ncg_alpha(float(gp), float(pHp), float(pmax_), float(dhat), _ptr(out))
    return out[0], out[1], out[2], out[3], bool(out[4])


class Oracle:
    """The oracle's model of one scene (rest data, surface, exclusion set) and its operations."""

    def __init__(self, rest_x, tets, *, youngs, poisson, density, dt, dhat, kappa, gravity=(0, 0, 0), plane=None,
                 fixed=None, youngs_per_tet=None, beta_rule=0, pnorm=0, excl_factor=1.5, model=0):
        lib = _load()
        self._X = _f64(rest_x).reshape(-1, 3)
        self._T = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        self._E = None if youngs_per_tet is None else _f64(youngs_per_tet).ravel()
        self._F = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8).ravel()
        pr = _Params()
        pr.nv, pr.nt = self._X.shape[0], self._T.shape[0]
        pr.rest_x, pr.tets = _ptr(self._X), _ptr(self._T)
        pr.youngs_per_tet = _ptr(self._E)
        pr.youngs, pr.poisson, pr.density = youngs, poisson, density
        pr.h, pr.dhat, pr.kappa = dt, dhat, kappa
        pr.gravity[:] = list(gravity)
        if plane is not None:
            pr.has_plane = 1
            pr.plane_n[:] = list(plane[0])
            pr.plane_o = float(plane[1])
        pr.fixed = _ptr(self._F)
        pr.beta_rule, pr.pnorm, pr.excl_factor, pr.model = beta_rule, pnorm, excl_factor, model
        self._m = lib.or_model_new(C.byref(pr))
        if not self._m:
            raise OracleError(1, lib.or_last_error().decode())
        self.nv, self.nt = pr.nv, pr.nt
        self.dhat, self.dt = dhat, dt
        self.fixed = self._F

    @classmethod
    def from_scene(cls, sc, **kw):
        return cls(sc.rest_x, sc.tets, youngs=sc.youngs, poisson=sc.poisson, density=sc.density, dt=sc.dt,
                   dhat=sc.dhat, kappa=sc.kappa, gravity=sc.gravity, plane=sc.plane, fixed=sc.fixed,
                   youngs_per_tet=sc.youngs_per_tet, **kw)

    def __del__(self):
        m = getattr(self, "_m", None)
        if m:
            _load().or_model_free(m)
            self._m = None

    def sizes(self):
        out = np.zeros(6, dtype=np.int32)
        _load().or_model_sizes(self._m, _ptr(out))
        return dict(zip(["nv", "nt", "nf", "ne", "ns", "nexcl"], out.tolist()))

    def mass(self):
        m = np.zeros(self.nv)
        _load().or_model_arrays(self._m, _ptr(m), None, None)
        return m

    def volumes(self):
        v = np.zeros(self.nt)
        _load().or_model_arrays(self._m, None, _ptr(v), None)
        return v

    def surface(self):
        s = self.sizes()
        tri = np.zeros((s["nf"], 3), np.int32)
        edge = np.zeros((s["ne"], 2), np.int32)
        sv = np.zeros(s["ns"], np.int32)
        _load().or_surface(self._m, _ptr(tri), _ptr(edge), _ptr(sv))
        return tri, edge, sv

    def energy(self, x, xtilde):
        x, xt = _f64(x), _f64(xtilde)
        E = C.c_double()
        parts = np.zeros(4)
        _check(_load().or_energy(self._m, _ptr(x), _ptr(xt), C.byref(E), _ptr(parts)))
        return E.value, parts

    def grad_diag(self, x, xtilde):
        x, xt = _f64(x), _f64(xtilde)
        g = np.zeros((self.nv, 3))
        d = np.zeros((self.nv, 3))
        na = C.c_int32()
        _check(_load().or_grad_diag(self._m, _ptr(x), _ptr(xt), _ptr(g), _ptr(d), C.byref(na)))
        return g, d, na.value

    def grad_diag_scale(self, x, xtilde):
        """Per-entry sums of the magnitudes of the contributions to g and diag(H) at x: the scale a rounding error of
        each term is relative to (inertia, each tet's force, each barrier force; m, each elastic and barrier term of
        the diagonal)."""
        x, xt = _f64(x), _f64(xtilde)
        gs = np.zeros((self.nv, 3))
        ds = np.zeros((self.nv, 3))
        _check(_load().or_grad_diag_scale(self._m, _ptr(x), _ptr(xt), _ptr(gs), _ptr(ds)))
        return gs, ds

    def pHp(self, x, p):
        x, p = _f64(x), _f64(p)
        out = C.c_double()
        _check(_load().or_pHp(self._m, _ptr(x), _ptr(p), C.byref(out)))
        return out.value

    def active_pairs(self, x, brute=False, threshold=0.0, use_excl=True, max_pairs=None):
        x = _f64(x)
        cnt = C.c_int32()
        if max_pairs is None:
            _check(_load().or_active_pairs(self._m, _ptr(x), int(brute), float(threshold), int(use_excl), None, None,
                                           None, 0, C.byref(cnt)))
            max_pairs = cnt.value
        idx = np.zeros((max(max_pairs, 1), 5), np.int32)
        d = np.zeros(max(max_pairs, 1))
        c = np.zeros((max(max_pairs, 1), 4))
        _check(_load().or_active_pairs(self._m, _ptr(x), int(brute), float(threshold), int(use_excl), _ptr(idx),
                                       _ptr(d), _ptr(c), max_pairs, C.byref(cnt)))
        n = min(cnt.value, max_pairs)
        return idx[:n], d[:n], c[:n]

    def predict(self, x, v, targets=None):
        x, v = _f64(x), _f64(v)
        tg = None if targets is None else _f64(targets)
        out = np.zeros((self.nv, 3))
        _load().or_predict(self._m, _ptr(x), _ptr(v), _ptr(tg), _ptr(out))
        return out

    def iteration(self, x, xtilde, g, P, p, k, dE0=0.0):
        """One PNCG iteration in place on x, g, P, p (float64 [nv,3] C-contiguous arrays); returns the scalars."""
        for a in (x, g, P, p):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        xt = _f64(xtilde)
        s = _Scalars()
        s.k, s.dE0 = int(k), float(dE0)
        _check(_load().or_iteration(self._m, _ptr(x), _ptr(xt), _ptr(g), _ptr(P), _ptr(p), C.byref(s)))
        return {f: getattr(s, f) for f, _ in _Scalars._fields_}

    def iteration_split(self, x, xtilde, g, P, p, off, state, moving=None):
        """One PNCG iteration with per-object splitting (Sec. 5.2) in place on x, g, P, p.  off: object boundaries
        [nobj + 1] (object o = vertices off[o] .. off[o+1]-1); state: a list of nobj dicts carrying each object's
        "k" and "dE0" between calls (start with [{}] * nobj, or None entries); moving: nobj flags (None = all move).
        Returns the per-object scalars (and updates state)."""
        for a in (x, g, P, p):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        off = np.ascontiguousarray(off, dtype=np.int32)
        nobj = len(off) - 1
        ss = (_Scalars * nobj)()
        for o in range(nobj):
            st = state[o] or {}
            ss[o].k, ss[o].dE0 = int(st.get("k", 0)), float(st.get("dE0", 0.0))
        mv = None if moving is None else np.ascontiguousarray(moving, dtype=np.int32)
        _check(_load().or_iteration_split(self._m, nobj, _ptr(off), _ptr(mv), _ptr(x), _ptr(_f64(xtilde)), _ptr(g),
                                          _ptr(P), _ptr(p), ss))
        out = [{f: getattr(ss[o], f) for f, _ in _Scalars._fields_} for o in range(nobj)]
        for o in range(nobj):
            state[o] = {"k": out[o]["k"], "dE0": out[o]["dE0"]}
        return out

    def iteration_groups(self, x, xtilde, g, P, p, group, state, moving=None):
        """One PNCG iteration with splitting over arbitrary vertex groups (Sec. 5.2): group[i] in 0..G-1 for each
        vertex; state and moving as in iteration_split.  Returns the per-group scalars."""
        for a in (x, g, P, p):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        grp = np.ascontiguousarray(group, dtype=np.int32)
        ng = int(grp.max()) + 1
        ss = (_Scalars * ng)()
        for q in range(ng):
            st = state[q] or {}
            ss[q].k, ss[q].dE0 = int(st.get("k", 0)), float(st.get("dE0", 0.0))
        mv = None if moving is None else np.ascontiguousarray(moving, dtype=np.int32)
        _check(_load().or_iteration_groups(self._m, ng, _ptr(grp), _ptr(mv), _ptr(x), _ptr(_f64(xtilde)), _ptr(g),
                                           _ptr(P), _ptr(p), ss))
        out = [{f: getattr(ss[q], f) for f, _ in _Scalars._fields_} for q in range(ng)]
        for q in range(ng):
            state[q] = {"k": out[q]["k"], "dE0": out[q]["dE0"]}
        return out

    def contact_vertices(self, x):
        """1 for the vertices of the active pairs and those within dhat of the plane at x, else 0."""
        mark = np.zeros(self.nv, np.int32)
        _check(_load().or_contact_vertices(self._m, _ptr(_f64(x)), _ptr(mark)))
        return mark

    def step_parts(self, x, v, obj, targets=None, iters=50, eps=0.0):
        """One time step with every object split into its collision and non-collision parts (Sec. 5.2), in place on
        x and v: after the prediction and the kinematic targets, the vertices in contact at x_0 form each object's
        collision part; the parts then iterate as the groups of iteration_groups (eps rule per part).  obj: the
        object of each vertex.  Returns (iterations done, group labels)."""
        xt = self.predict(x, v, targets)
        x0 = x.copy()
        if targets is not None and self.fixed is not None:
            x[self.fixed.astype(bool)] = _f64(targets).reshape(-1, 3)
        raw = 2 * np.asarray(obj, dtype=np.int64) + self.contact_vertices(x)
        _, group = np.unique(raw, return_inverse=True)
        group = group.astype(np.int32)
        ng = int(group.max()) + 1
        g, P, p = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
        state, moving = [None] * ng, np.ones(ng, dtype=np.int32)
        k = 0
        while k < iters and moving.any():
            sc = self.iteration_groups(x, xt, g, P, p, group, state, moving)
            k += 1
            if eps > 0.0:
                for q in range(ng):
                    if moving[q] and sc[q]["dE"] < eps * sc[q]["dE0"]:
                        moving[q] = 0
        v[:] = (x - x0) / self.dt
        return k, group

    def step_split(self, x, v, off, targets=None, iters=50, eps=0.0):
        """One time step with per-object splitting, in place on x and v: the prediction and kinematic targets of
        `step`, then iterations of `iteration_split`; under the eps rule (Sec. 4.4) an object stops moving once its
        Delta E < eps Delta E_0 and the step ends when every object has stopped.  Returns the iterations done."""
        xt = self.predict(x, v, targets)
        x0 = x.copy()
        if targets is not None and self.fixed is not None:
            x[self.fixed.astype(bool)] = _f64(targets).reshape(-1, 3)
        g, P, p = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
        nobj = len(off) - 1
        state, moving = [None] * nobj, np.ones(nobj, dtype=np.int32)
        k = 0
        while k < iters and moving.any():
            sc = self.iteration_split(x, xt, g, P, p, off, state, moving)
            k += 1
            if eps > 0.0:
                for o in range(nobj):
                    if moving[o] and sc[o]["dE"] < eps * sc[o]["dE0"]:
                        moving[o] = 0
        v[:] = (x - x0) / self.dt
        return k

    def step(self, x, v, targets=None, iters=50, eps=0.0):
        """One time step in place on x and v; returns (iterations done, trace [iters, 8])."""
        assert x.dtype == np.float64 and x.flags.c_contiguous and v.dtype == np.float64 and v.flags.c_contiguous
        tg = None if targets is None else _f64(targets)
        trace = np.zeros((iters, 8))
        done = C.c_int32()
        _check(_load().or_step(self._m, _ptr(x), _ptr(v), _ptr(tg), int(iters), float(eps), _ptr(trace),
                               C.byref(done)))
        return done.value, trace[:done.value]

    def hvp(self, x, v):
        """H(x) v (frozen closest points; kinematic rows and columns dropped)."""
        out = np.zeros((self.nv, 3))
        _check(_load().or_hvp(self._m, _ptr(_f64(x)), _ptr(_f64(v)), _ptr(out)))
        return out

    def adjoint_step(self, x1, ax1, av1, dE=None, tol=1e-10, max_iters=5000):
        """The reverse of one time step at its end state x1: (ax0, av0, iters, residual), adding dL/dE_e to dE
        (float64 [n_tets], updated in place) when given."""
        ax0 = np.zeros((self.nv, 3))
        av0 = np.zeros((self.nv, 3))
        if dE is not None:
            assert dE.dtype == np.float64 and dE.flags.c_contiguous and dE.size == self.nt
        it = C.c_int32()
        res = C.c_double()
        _check(_load().or_adjoint_step(self._m, _ptr(_f64(x1)), _ptr(_f64(ax1)), _ptr(_f64(av1)), _ptr(ax0),
                                       _ptr(av0), _ptr(dE), float(tol), int(max_iters), C.byref(it), C.byref(res)))
        return ax0, av0, it.value, res.value

    def intersections(self, x):
        return int(_load().or_intersections(self._m, _ptr(_f64(x))))
