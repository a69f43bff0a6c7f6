"""ctypes binding of libpncg.so with the names of the C ABI in include/pncg.h (argument marshalling only).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA device); both must be C-contiguous and of the
documented dtype.  Every solver step runs in the library's CUDA kernels: there is no Python or CPU compute path,
and loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpncg.so")

SIM_OK, SIM_ERR_INVALID_ARG, SIM_ERR_CUDA, SIM_ERR_OOM, SIM_ERR_INVERTED, SIM_ERR_PENETRATION, \
    SIM_ERR_NONFINITE, SIM_ERR_TIMEOUT, SIM_ERR_CAPACITY = range(9)
SIM_FP64, SIM_FP32_MIXED = 0, 1
SIM_BETA_PR_PLUS, SIM_BETA_DK = 0, 1
SIM_MAT_NH, SIM_MAT_SNH, SIM_MAT_FCR, SIM_MAT_ARAP = 0, 1, 2, 3
SIM_PNORM_VERTEX2, SIM_PNORM_COMPONENT_INF = 0, 1
SIM_SCATTER_ATOMIC, SIM_SCATTER_SEGMENTED, SIM_SCATTER_BLOCK, SIM_SCATTER_COLOR = 0, 1, 2, 3
TRACE_COLUMNS = ("beta", "gp", "pHp", "pmax", "alpha", "dE", "n_active", "capped")


class sim_mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("rest_x", C.c_void_p), ("tets", C.c_void_p),
                ("x0", C.c_void_p), ("v0", C.c_void_p), ("fixed", C.c_void_p), ("scene_of_vert", C.c_void_p)]


class sim_material(C.Structure):
    _fields_ = [("density", C.c_double), ("youngs", C.c_double), ("poisson", C.c_double),
                ("youngs_per_tet", C.c_void_p), ("model", C.c_int32)]


class sim_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("beta", C.c_int32), ("iters", C.c_int32), ("eps", C.c_double),
                ("gravity", C.c_double * 3), ("has_plane", C.c_int32), ("plane_n", C.c_double * 3),
                ("plane_o", C.c_double), ("pad_r", C.c_double), ("pnorm", C.c_int32), ("scatter", C.c_int32),
                ("excl_factor", C.c_double), ("cuda_stream", C.c_void_p), ("use_graph", C.c_int32),
                ("candidate_capacity", C.c_int32), ("persistent", C.c_int32), ("split_objects", C.c_int32),
                ("block_shape", C.c_int32)]


class sim_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("iters_done", C.c_int32), ("n_candidates", C.c_int32),
                ("n_active", C.c_int32), ("n_rebuilds", C.c_int32), ("n_capped", C.c_int32),
                ("n_surface_tris", C.c_int32), ("n_surface_edges", C.c_int32), ("n_surface_verts", C.c_int32),
                ("dE0", C.c_double), ("dE_last", C.c_double), ("launch_form", C.c_int32), ("n_scenes", C.c_int32),
                ("n_near_fp64", C.c_int32), ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("n_colors", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class sim_iter_scalars(C.Structure):
    _fields_ = [("k", C.c_int32), ("restarted", C.c_int32), ("capped", C.c_int32), ("n_active", C.c_int32),
                ("beta", C.c_double), ("gp", C.c_double), ("pHp", C.c_double), ("pmax", C.c_double),
                ("alpha_bar", C.c_double), ("alpha_up", C.c_double), ("alpha", C.c_double), ("dE", C.c_double),
                ("dE0", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__(f"{_status_name(status)}: {msg}")


_lib = None


ABI_VERSION = 4


def load():
    """Loads libpncg.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2405_08001_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I32, D = C.c_void_p, C.c_int32, C.c_double
    sigs = {
        "sim_abi_version": (I32, []),
        "sim_status_string": (C.c_char_p, [C.c_int]),
        "sim_default_options": (C.c_int, [P]),
        "sim_create": (C.c_int, [P, P, D, D, D, P, P]),
        "sim_step": (C.c_int, [P, I32, P]),
        "sim_step_async": (C.c_int, [P, I32, P]),
        "sim_get_state": (C.c_int, [P, P, P, P]),
        "sim_set_state": (C.c_int, [P, P, P]),
        "sim_begin_step": (C.c_int, [P, P]),
        "sim_iterate": (C.c_int, [P, I32]),
        "sim_end_step": (C.c_int, [P]),
        "sim_get_iterate": (C.c_int, [P, P, P, P, P, P, P]),
        "sim_set_iterate": (C.c_int, [P, P, P, P, P, I32, D]),
        "sim_eval_gradient": (C.c_int, [P, P, P, P, P]),
        "sim_eval_pHp": (C.c_int, [P, P, P, P]),
        "sim_eval_energy": (C.c_int, [P, P, P, P, P]),
        "sim_get_contacts": (C.c_int, [P, P, P, I32, P]),
        "sim_get_candidates": (C.c_int, [P, P, I32, P]),
        "sim_get_trace": (C.c_int, [P, P, I32, P]),
        "sim_profile_step": (C.c_int, [P, P, P, P, I32]),
        "sim_profile_barriers": (C.c_int, [P, P, P, P, P, I32, P, P]),
        "sim_get_scene_scalars": (C.c_int, [P, P, I32, P]),
        "sim_get_groups": (C.c_int, [P, P]),
        "sim_eval_hvp": (C.c_int, [P, P, P, P]),
        "sim_adjoint_step": (C.c_int, [P, P, P, P, P, P, P, D, I32, P, P]),
        "sim_kernel_count": (I32, []),
        "sim_kernel_name": (C.c_char_p, [I32]),
        "sim_get_sizes": (C.c_int, [P, P]),
        "sim_destroy": (None, [P]),
        "sim_last_error": (C.c_char_p, [P]),
        "sim_selftest_wait": (C.c_int, [D]),
        "sim_pHp_noalloc": (C.c_int, [I32, I32, P, P, P, P, P, D, D, D, P, P]),
        "sim_noalloc_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.sim_abi_version() != ABI_VERSION:   # the structures below describe this version's layouts
        raise ImportError(f"{LIB_PATH} has ABI version {lib.sim_abi_version()}, this binding {ABI_VERSION}: rebuild it")
    _lib = lib
    return lib


def _status_name(st):
    try:
        return load().sim_status_string(st).decode()
    except Exception:
        return f"status {st}"


def _check(st, h=None):
    if st != SIM_OK:
        raise SimError(st, load().sim_last_error(h).decode())


def _ptr(a, dtype=np.float64, n=None):
    """Address of a C-contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):   # torch tensor
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        if n is not None and a.numel() < n:
            raise ValueError(f"tensor has {a.numel()} elements, {n} needed")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if n is not None and arr.size < n:
        raise ValueError(f"array has {arr.size} elements, {n} needed")
    return arr.ctypes.data, arr


def sim_default_options() -> sim_options:
    o = sim_options()
    _check(load().sim_default_options(C.byref(o)))
    return o


def sim_create(rest_x, tets, *, density, youngs, poisson, dt, dhat, kappa, x0=None, v0=None, fixed=None,
               youngs_per_tet=None, scene_of_vert=None, options: sim_options | None = None, model: int = SIM_MAT_NH):
    """sim_create with host arrays; returns the opaque handle (a c_void_p value)."""
    lib = load()
    rx = np.ascontiguousarray(rest_x, dtype=np.float64).reshape(-1, 3)
    nv = rx.shape[0]
    tt = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    keep = [rx, tt]
    m = sim_mesh()
    m.n_verts, m.n_tets = nv, tt.shape[0]
    m.rest_x, m.tets = rx.ctypes.data, tt.ctypes.data
    for name, arr, dt_ in (("x0", x0, np.float64), ("v0", v0, np.float64), ("fixed", fixed, np.uint8),
                           ("scene_of_vert", scene_of_vert, np.int32)):
        if arr is not None:
            a = np.ascontiguousarray(arr, dtype=dt_)
            keep.append(a)
            setattr(m, name, a.ctypes.data)
    mat = sim_material()
    mat.density, mat.youngs, mat.poisson, mat.model = density, youngs, poisson, int(model)
    if youngs_per_tet is not None:
        e = np.ascontiguousarray(youngs_per_tet, dtype=np.float64)
        keep.append(e)
        mat.youngs_per_tet = e.ctypes.data
    h = C.c_void_p()
    st = lib.sim_create(C.byref(m), C.byref(mat), float(dt), float(dhat), float(kappa),
                        None if options is None else C.byref(options), C.byref(h))
    _check(st)
    return h.value


def sim_step(h, n_steps: int = 1, targets=None):
    p, keep = _ptr(targets)
    _check(load().sim_step(h, int(n_steps), p), h)


def sim_step_async(h, n_steps: int = 1, targets=None):
    p, keep = _ptr(targets)
    _check(load().sim_step_async(h, int(n_steps), p), h)
    return keep


def sim_get_sizes(h):
    out = np.zeros(6, np.int32)
    _check(load().sim_get_sizes(h, out.ctypes.data), h)
    return dict(zip(["n_verts", "n_tets", "n_surface_tris", "n_surface_edges", "n_surface_verts", "n_excluded"],
                    out.tolist()))


def _out(a, nv):
    if a is None:
        a = np.zeros((nv, 3))
    p, arr = _ptr(a, n=3 * nv)
    return p, arr


def sim_get_state(h, x_out=None, v_out=None, want_x=True, want_v=True):
    nv = sim_get_sizes(h)["n_verts"]
    px, x = _out(x_out, nv) if want_x else (None, None)
    pv, v = _out(v_out, nv) if want_v else (None, None)
    st = sim_stats()
    _check(load().sim_get_state(h, px, pv, C.byref(st)), h)
    return x, v, st.as_dict()


def sim_set_state(h, x=None, v=None):
    nv = sim_get_sizes(h)["n_verts"]
    px, kx = _ptr(x, n=3 * nv)
    pv, kv = _ptr(v, n=3 * nv)
    _check(load().sim_set_state(h, px, pv), h)


def sim_begin_step(h, targets=None):
    p, keep = _ptr(targets)
    _check(load().sim_begin_step(h, p), h)


def sim_iterate(h, n: int = 1):
    _check(load().sim_iterate(h, int(n)), h)


def sim_end_step(h):
    _check(load().sim_end_step(h), h)


def sim_get_iterate(h):
    """(x, g, P, p, xtilde, scalars) after the most recent iteration, as numpy arrays."""
    nv = sim_get_sizes(h)["n_verts"]
    arrs = [np.zeros((nv, 3)) for _ in range(5)]
    s = sim_iter_scalars()
    _check(load().sim_get_iterate(h, *[a.ctypes.data for a in arrs], C.byref(s)), h)
    return (*arrs, s.as_dict())


def sim_set_iterate(h, x=None, g=None, P=None, p=None, k: int = 0, gPg: float = 0.0):
    nv = sim_get_sizes(h)["n_verts"]
    ptrs = [_ptr(a, n=3 * nv) for a in (x, g, P, p)]
    _check(load().sim_set_iterate(h, *[q[0] for q in ptrs], int(k), float(gPg)), h)


def sim_eval_gradient(h, x, xtilde):
    nv = sim_get_sizes(h)["n_verts"]
    px, kx = _ptr(x, n=3 * nv)
    pt, kt = _ptr(xtilde, n=3 * nv)
    g = np.zeros((nv, 3))
    d = np.zeros((nv, 3))
    _check(load().sim_eval_gradient(h, px, pt, g.ctypes.data, d.ctypes.data), h)
    return g, d


def sim_eval_pHp(h, x, p):
    nv = sim_get_sizes(h)["n_verts"]
    px, kx = _ptr(x, n=3 * nv)
    pp, kp = _ptr(p, n=3 * nv)
    out = C.c_double()
    _check(load().sim_eval_pHp(h, px, pp, C.byref(out)), h)
    return out.value


def sim_eval_energy(h, x, xtilde):
    nv = sim_get_sizes(h)["n_verts"]
    px, kx = _ptr(x, n=3 * nv)
    pt, kt = _ptr(xtilde, n=3 * nv)
    out = C.c_double()
    parts = np.zeros(4)
    _check(load().sim_eval_energy(h, px, pt, C.byref(out), parts.ctypes.data), h)
    return out.value, parts


def sim_get_contacts(h):
    cnt = C.c_int32()
    _check(load().sim_get_contacts(h, None, None, 0, C.byref(cnt)), h)
    n = cnt.value
    idx = np.zeros((max(n, 1), 5), np.int32)
    d = np.zeros(max(n, 1))
    _check(load().sim_get_contacts(h, idx.ctypes.data, d.ctypes.data, n, C.byref(cnt)), h)
    return idx[:n], d[:n]


def sim_get_candidates(h):
    cnt = C.c_int32()
    _check(load().sim_get_candidates(h, None, 0, C.byref(cnt)), h)
    n = cnt.value
    idx = np.zeros((max(n, 1), 5), np.int32)
    _check(load().sim_get_candidates(h, idx.ctypes.data, n, C.byref(cnt)), h)
    return idx[:n]


def sim_get_trace(h, max_iters: int = 4096):
    buf = np.zeros((max_iters, len(TRACE_COLUMNS)))
    n = C.c_int32()
    _check(load().sim_get_trace(h, buf.ctypes.data, max_iters, C.byref(n)), h)
    return buf[:n.value]


def sim_kernel_names():
    lib = load()
    return [lib.sim_kernel_name(i).decode() for i in range(lib.sim_kernel_count())]


def sim_profile_step(h, targets=None):
    """One time step timed kernel by kernel on the GPU: {kernel: (milliseconds over the step, launches)}."""
    names = sim_kernel_names()
    ms = np.zeros(len(names), np.float32)
    n = np.zeros(len(names), np.int32)
    p, keep = _ptr(targets)
    _check(load().sim_profile_step(h, p, ms.ctypes.data, n.ctypes.data, len(names)), h)
    return {k: (float(a), int(b)) for k, a, b in zip(names, ms, n)}


def sim_profile_barriers(h, targets=None, max_barriers=4096, max_blocks=4096):
    """Persistent form: one time step with every block's arrival and departure time (ns) at every grid barrier.
    Returns (arrive [n_barriers, n_blocks] uint64, depart [n_barriers, n_blocks] uint64, phase names [n_barriers])."""
    names = sim_kernel_names()
    arrive = np.zeros((max_barriers, max_blocks), np.uint64)
    depart = np.zeros((max_barriers, max_blocks), np.uint64)
    kind = np.zeros(max_barriers, np.int32)
    nb = C.c_int32(0)
    ng = C.c_int32(0)
    p, keep = _ptr(targets)
    _check(load().sim_profile_barriers(h, p, arrive.ctypes.data, depart.ctypes.data, kind.ctypes.data, max_barriers,
                                       C.byref(nb), C.byref(ng)), h)
    n, g = nb.value, ng.value
    if g > max_blocks:
        raise ValueError(f"the launch has {g} blocks, more than max_blocks = {max_blocks}")
    # the library wrote rows of g blocks contiguously
    flat_a = arrive.reshape(-1)[: n * g].reshape(n, g).copy()
    flat_d = depart.reshape(-1)[: n * g].reshape(n, g).copy()
    return flat_a, flat_d, [names[k] for k in kind[:n]]


def sim_eval_hvp(h, x, v, out=None):
    """H(x) v (the incremental potential's Hessian with frozen contact closest points) -> [n_verts, 3]."""
    nv = sim_get_sizes(h)["n_verts"]
    px, kx = _ptr(x, n=3 * nv)
    pv, kv = _ptr(v, n=3 * nv)
    po, o = _out(out, nv)
    _check(load().sim_eval_hvp(h, px, pv, po), h)
    return o


def sim_adjoint_step(h, x1, ax1, av1, dE=None, tol=1e-10, max_iters=2000, ax0=None, av0=None):
    """Reverse of one time step ending at x1: returns (dL/dx_t, dL/dv_t, CG iterations, relative residual) and adds
    dL/dE_e to dE (a float64 [n_tets] array or tensor, updated in place) when given."""
    sz = sim_get_sizes(h)
    nv = sz["n_verts"]
    px, kx = _ptr(x1, n=3 * nv)
    pa, ka = _ptr(ax1, n=3 * nv)
    pb, kb = _ptr(av1, n=3 * nv)
    p0, a0 = _out(ax0, nv)
    p1, a1 = _out(av0, nv)
    pe, ke = (None, None) if dE is None else _ptr(dE, n=sz["n_tets"])
    if dE is not None and not hasattr(dE, "data_ptr") and ke is not dE:
        raise TypeError("dE must be a C-contiguous float64 array (it is updated in place)")
    it = C.c_int32(0)
    res = C.c_double(0.0)
    _check(load().sim_adjoint_step(h, px, pa, pb, p0, p1, pe, float(tol), int(max_iters), C.byref(it), C.byref(res)), h)
    return a0, a1, it.value, res.value


SCENE_SCALAR_COLS = ("beta", "gp", "pHp", "pmax", "alpha", "dE", "dE0", "converged", "iters_done", "restarted",
                     "capped")


def sim_get_groups(h):
    """The group label of every vertex in the current time step (int32 [n_verts])."""
    nv = sim_get_sizes(h)["n_verts"]
    out = np.zeros(nv, np.int32)
    _check(load().sim_get_groups(h, out.ctypes.data), h)
    return out


def sim_get_scene_scalars(h, max_scenes=1024):
    """Per-scene scalars of the most recent iteration: a dict of arrays [n_scenes] named by SCENE_SCALAR_COLS."""
    out = np.zeros((max_scenes, len(SCENE_SCALAR_COLS)))
    n = C.c_int32(0)
    _check(load().sim_get_scene_scalars(h, out.ctypes.data, max_scenes, C.byref(n)), h)
    return {c: out[: n.value, i].copy() for i, c in enumerate(SCENE_SCALAR_COLS)}


def _noalloc_args(x, p, rest_x, tets, mass, out, stream):
    """Checks sim_pHp_noalloc's arguments on the host, before anything reaches the device: every array a contiguous
    CUDA tensor of the right type on one device (the stream's, if one is given), matching sizes.  Returns
    (device, n_verts, n_tets)."""
    import torch
    named = (("x", x, torch.float64), ("p", p, torch.float64), ("rest_x", rest_x, torch.float64),
             ("tets", tets, torch.int32), ("mass", mass, torch.float64), ("out", out, torch.float64))
    for name, a, dt in named:
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"sim_pHp_noalloc: {name} must be a CUDA tensor, not {type(a).__name__}")
        if not a.is_cuda:
            raise TypeError(f"sim_pHp_noalloc: {name} must be a CUDA tensor (it is on {a.device})")
        if a.dtype != dt or not a.is_contiguous():
            raise TypeError(f"sim_pHp_noalloc: {name} must be a contiguous {dt} tensor")
    dev = x.device
    for name, a, _ in named:
        if a.device != dev:
            raise ValueError(f"sim_pHp_noalloc: {name} is on {a.device}, x on {dev}")
    if stream is not None and stream.device != dev:
        raise ValueError(f"sim_pHp_noalloc: the stream belongs to {stream.device}, the tensors to {dev}")
    if x.numel() == 0 or x.numel() % 3:
        raise ValueError("sim_pHp_noalloc: x must hold n_verts x 3 values, n_verts > 0")
    nv = x.numel() // 3
    for name, a, n in (("p", p, 3 * nv), ("rest_x", rest_x, 3 * nv), ("mass", mass, nv)):
        if a.numel() != n:
            raise ValueError(f"sim_pHp_noalloc: {name} has {a.numel()} values, {n} expected")
    if tets.numel() == 0 or tets.numel() % 4:
        raise ValueError("sim_pHp_noalloc: tets must hold n_tets x 4 indices, n_tets > 0")
    if out.numel() < 1:
        raise ValueError("sim_pHp_noalloc: out must hold one value")
    return dev, nv, tets.numel() // 4


def sim_pHp_noalloc(x, p, rest_x, tets, mass, youngs, poisson, dt, out, stream=None):
    """Allocation-free p^T H p (inertia + elastic, no contact) on caller-owned CUDA tensors; asynchronous on
    `stream` (a torch.cuda.Stream or None).  x, p, rest_x: float64 [n_verts, 3]; tets: int32 [n_tets, 4] with
    indices in [0, n_verts); mass: float64 [n_verts]; out: a 1-element float64 tensor.  All on one device; the call
    is made with that device current.  Host arrays, CPU tensors or mismatched sizes raise TypeError / ValueError
    before anything is launched."""
    import torch
    dev, nv, nt = _noalloc_args(x, p, rest_x, tets, mass, out, stream)
    with torch.cuda.device(dev):
        st = load().sim_pHp_noalloc(nv, nt, x.data_ptr(), p.data_ptr(), rest_x.data_ptr(), tets.data_ptr(),
                                    mass.data_ptr(), float(youngs), float(poisson), float(dt), out.data_ptr(),
                                    None if stream is None else stream.cuda_stream)
    if st != SIM_OK:
        raise SimError(st, load().sim_noalloc_last_error().decode())


def sim_noalloc_last_error() -> str:
    return load().sim_noalloc_last_error().decode()


def sim_selftest_wait(limit_s: float = 0.05):
    """The failure-detection self-test (a bounded device wait that nothing completes): (status, message).  The
    expected status is SIM_ERR_TIMEOUT."""
    lib = load()
    st = lib.sim_selftest_wait(float(limit_s))
    return st, lib.sim_last_error(None).decode()


def sim_destroy(h):
    if h:
        load().sim_destroy(h)


def options_for(scene, precision=SIM_FP64, **kw) -> sim_options:
    """Default options filled from a scenes.Scene (gravity, plane, iterations), overridden by keyword arguments."""
    o = sim_default_options()
    o.precision = precision
    o.iters = scene.iters
    o.gravity[:] = list(scene.gravity)
    if scene.plane is not None:
        o.has_plane = 1
        o.plane_n[:] = list(scene.plane[0])
        o.plane_o = float(scene.plane[1])
    for k, v in kw.items():
        if k == "gravity":
            o.gravity[:] = list(v)
        else:
            setattr(o, k, v)
    return o


class Sim:
    """Owning wrapper of a handle: Sim(scene, precision=..., **options)."""

    def __init__(self, scene, precision=SIM_FP64, options: sim_options | None = None, model: int = SIM_MAT_NH, **kw):
        self.scene = scene
        self.options = options if options is not None else options_for(scene, precision, **kw)
        self.h = sim_create(scene.rest_x, scene.tets, density=scene.density, youngs=scene.youngs,
                            poisson=scene.poisson, dt=scene.dt, dhat=scene.dhat, kappa=scene.kappa, x0=scene.x0,
                            v0=scene.v0, fixed=scene.fixed, youngs_per_tet=scene.youngs_per_tet,
                            scene_of_vert=scene.scene_of_vert, options=self.options, model=model)
        self.nv = scene.n_verts
        self.n_fixed = 0 if scene.fixed is None else int(np.count_nonzero(scene.fixed))

    def close(self):
        if getattr(self, "h", None):
            sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, targets=None):
        """n time steps; targets: [n][n_fixed][3] positions of the kinematic vertices (or None to keep them)."""
        if targets is not None and np.size(targets) < 3 * self.n_fixed * n:
            raise ValueError(f"targets has {np.size(targets)} values, {3 * self.n_fixed * n} needed")
        sim_step(self.h, n, targets)

    def state(self):
        return sim_get_state(self.h)

    def sizes(self):
        return sim_get_sizes(self.h)
