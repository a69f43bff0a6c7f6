"""Seeded synthetic scenes for the PNCG solver (inputs only).

This module builds the inputs both sides consume -- rest positions, tetrahedra, initial state, kinematic
(Dirichlet) targets and material / contact parameters -- and holds none of the method's arithmetic: no
deformation gradients, masses, distances or energies are computed here.  The CUDA library and the FP64 CPU
oracle each derive everything else from these arrays on their own.

Meshes are regular hex grids with every cell split into six tetrahedra along the cell's main diagonal (the
Kuhn / Freudenthal split), which is conforming across cells.  The paper's own scenes use meshes that are not
available here (Section 6, Table 1); these grids stand in for them at the same sizes (27K-202K tets).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

# The six monotone lattice paths from corner (0,0,0) to (1,1,1) of a unit cell; each path gives one tetrahedron.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_PERM_ODD = [False, True, True, False, False, True]


def kuhn_grid(nx: int, ny: int, nz: int, size=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)):
    """Vertices [V,3] (float64) and positively oriented tetrahedra [T,4] (int32) of an nx*ny*nz Kuhn grid.

    Vertex (i,j,k) has index i + (nx+1)*(j + (ny+1)*k).
    """
    nx, ny, nz = int(nx), int(ny), int(nz)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid needs at least one cell per axis")
    xs = origin[0] + np.linspace(0.0, size[0], nx + 1)
    ys = origin[1] + np.linspace(0.0, size[1], ny + 1)
    zs = origin[2] + np.linspace(0.0, size[2], nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(order="F"), cj.ravel(order="F"), ck.ravel(order="F")
    tets = []
    for perm, odd in zip(_PERMS, _PERM_ODD):
        step = [np.zeros(3, dtype=np.int64) for _ in range(4)]
        c = np.zeros(3, dtype=np.int64)
        path = [c.copy()]
        for ax in perm:
            c[ax] += 1
            path.append(c.copy())
        v = [vid(ci + p[0], cj + p[1], ck + p[2]) for p in path]
        if odd:  # odd permutations give negative volume; swap two vertices to fix the orientation
            v[1], v[2] = v[2], v[1]
        tets.append(np.stack(v, axis=1))
    # interleave so the six tets of a cell are adjacent in memory (cell-major order)
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return verts, tets


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation in SO(3) from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def rot_z(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


@dataclasses.dataclass
class Scene:
    """One simulation problem: mesh, state, material and contact parameters (SI units)."""
    name: str
    rest_x: np.ndarray                 # [V,3] float64 rest positions
    tets: np.ndarray                   # [T,4] int32
    x0: np.ndarray                     # [V,3] float64 initial positions
    v0: np.ndarray                     # [V,3] float64 initial velocities
    youngs: float
    poisson: float
    density: float
    dt: float
    dhat: float
    kappa: float
    gravity: tuple = (0.0, 0.0, 0.0)
    plane: Optional[tuple] = None      # (normal[3], offset): half-space n.x >= offset
    fixed: Optional[np.ndarray] = None  # [V] uint8, 1 = kinematic vertex
    youngs_per_tet: Optional[np.ndarray] = None
    scene_of_vert: Optional[np.ndarray] = None
    iters: int = 50
    steps: int = 10
    target_fn: Optional[Callable[[int], np.ndarray]] = None  # step -> [n_fixed,3] positions at t_{step+1}

    @property
    def n_verts(self) -> int:
        return int(self.rest_x.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def fixed_indices(self) -> np.ndarray:
        if self.fixed is None:
            return np.zeros(0, dtype=np.int64)
        return np.nonzero(self.fixed)[0]

    def targets(self, step: int) -> Optional[np.ndarray]:
        """Kinematic targets [n_fixed,3] for the end of time step `step` (0-based), or None."""
        if self.target_fn is None:
            return None
        return np.ascontiguousarray(self.target_fn(step), dtype=np.float64)

    def all_targets(self, n_steps: int, first_step: int = 0) -> Optional[np.ndarray]:
        if self.target_fn is None:
            return None
        return np.ascontiguousarray(np.stack([self.targets(first_step + s) for s in range(n_steps)]))

    @property
    def n_scenes(self) -> int:
        return 1 if self.scene_of_vert is None else int(self.scene_of_vert[-1]) + 1

    def scene_ranges(self):
        """Per scene: (first vertex, end vertex, first tet, end tet) of a batch (scenes are contiguous)."""
        if self.scene_of_vert is None:
            return [(0, self.n_verts, 0, self.n_tets)]
        sv = self.scene_of_vert
        st = sv[self.tets[:, 0]]
        out = []
        for s in range(self.n_scenes):
            v = np.nonzero(sv == s)[0]
            t = np.nonzero(st == s)[0]
            out.append((int(v[0]), int(v[-1]) + 1, int(t[0]), int(t[-1]) + 1))
        return out

    def subscene(self, s: int) -> "Scene":
        """Scene s of a batch as a problem of its own (vertex indices rebased)."""
        v0, v1, t0, t1 = self.scene_ranges()[s]
        return Scene(name=f"{self.name}[{s}]", rest_x=self.rest_x[v0:v1].copy(), tets=(self.tets[t0:t1] - v0).astype(np.int32),
                     x0=self.x0[v0:v1].copy(), v0=self.v0[v0:v1].copy(), youngs=self.youngs, poisson=self.poisson,
                     density=self.density, dt=self.dt, dhat=self.dhat, kappa=self.kappa, gravity=self.gravity,
                     plane=self.plane, fixed=None if self.fixed is None else self.fixed[v0:v1].copy(),
                     youngs_per_tet=None if self.youngs_per_tet is None else self.youngs_per_tet[t0:t1].copy(),
                     iters=self.iters, steps=self.steps)


def cube_drop(n: int = 8, side: float = 0.1, drop: float = 0.02, youngs: float = 1e5, poisson: float = 0.4,
              density: float = 1000.0, dt: float = 1.0 / 60.0, dhat: float = 1e-3, kappa: float = 1e4,
              iters: int = 50, steps: int = 10, seed: int = 0, cells=None) -> Scene:
    """A cube of n^3 Kuhn-split cells dropped `drop` metres onto the plane z = 0 under gravity.

    `cells=(nx,ny,nz)` gives a box with uneven cell counts (same cell size), for ragged launch tails.
    """
    nx, ny, nz = cells if cells is not None else (n, n, n)
    h = side / n
    X, T = kuhn_grid(nx, ny, nz, size=(nx * h, ny * h, nz * h), origin=(0.0, 0.0, drop))
    rng = np.random.default_rng(seed)
    x0 = X.copy()
    v0 = np.zeros_like(X)
    del rng
    return Scene(name=f"cube{nx}x{ny}x{nz}", rest_x=X, tets=T, x0=x0, v0=v0, youngs=youngs, poisson=poisson,
                 density=density, dt=dt, dhat=dhat, kappa=kappa, gravity=(0.0, 0.0, -9.8),
                 plane=((0.0, 0.0, 1.0), 0.0), iters=iters, steps=steps)


def twisted_bar(nx: int = 16, ny: int = 16, nz: int = 64, size=(0.1, 0.1, 0.4), youngs: float = 1e5,
                poisson: float = 0.45, density: float = 1000.0, dt: float = 1.0 / 30.0, dhat: float = 5e-4,
                kappa: float = 1e4, omega: float = 2.0, iters: int = 50, steps: int = 120) -> Scene:
    """A bar along z whose two end caps (z = 0 and z = L) turn in opposite directions at `omega` rad/s.

    No gravity and no plane.  Cap vertices are kinematic: at the end of step s (time (s+1)*dt) the z = 0 cap is
    its rest layout turned by -omega*t about the bar axis and the z = L cap by +omega*t.
    """
    X, T = kuhn_grid(nx, ny, nz, size=size)
    zc = X[:, 2]
    lo = np.isclose(zc, 0.0)
    hi = np.isclose(zc, size[2])
    fixed = (lo | hi).astype(np.uint8)
    fidx = np.nonzero(fixed)[0]
    sign = np.where(hi[fidx], 1.0, -1.0)
    axis = np.array([0.5 * size[0], 0.5 * size[1], 0.0])
    rest_f = X[fidx] - axis

    def target_fn(step: int) -> np.ndarray:
        t = (step + 1) * dt
        out = np.empty_like(rest_f)
        for s in (-1.0, 1.0):
            m = sign == s
            out[m] = rest_f[m] @ rot_z(s * omega * t).T
        return out + axis

    return Scene(name=f"twisted_bar{nx}x{ny}x{nz}", rest_x=X, tets=T, x0=X.copy(), v0=np.zeros_like(X),
                 youngs=youngs, poisson=poisson, density=density, dt=dt, dhat=dhat, kappa=kappa,
                 gravity=(0.0, 0.0, 0.0), plane=None, fixed=fixed, iters=iters, steps=steps, target_fn=target_fn)


def two_blocks(seed: int = 0, n: int = 3, side: float = 0.03, gap: float = 0.5, dhat: float = 2e-3,
               kappa: float = 1e4, youngs: float = 1e5, poisson: float = 0.4, dt: float = 1.0 / 60.0,
               iters: int = 20, steps: int = 3, speed: float = 0.3, plane: bool = True) -> Scene:
    """Two small Kuhn-grid blocks, the upper one randomly rotated, with a corner hovering `gap`*dhat above
    the lower block's top face and moving towards it; both above the plane z = 0.

    Generic (non-parallel) point-triangle and edge-edge proximity for contact tests.
    """
    rng = np.random.default_rng(seed)
    Xa, Ta = kuhn_grid(n, n, n, size=(side, side, side), origin=(0.0, 0.0, 0.5 * dhat + 0.004))
    Xb, Tb = kuhn_grid(n, n, n, size=(side, side, side))
    R = random_rotation(rng)
    Xb = (Xb - 0.5 * side) @ R.T
    # put the lowest vertex of block b just above the middle of a's top face
    low = int(np.argmin(Xb[:, 2]))
    top = Xa[:, 2].max()
    jitter = rng.uniform(-0.2, 0.2, size=2) * side
    target = np.array([0.5 * side + jitter[0], 0.5 * side + jitter[1], top + gap * dhat])
    Xb = Xb - Xb[low] + target
    X = np.concatenate([Xa, Xb])
    T = np.concatenate([Ta, Tb + Xa.shape[0]]).astype(np.int32)
    v0 = np.zeros_like(X)
    v0[Xa.shape[0]:, 2] = -speed
    v0[Xa.shape[0]:, :2] = rng.normal(scale=0.05, size=2)
    return Scene(name=f"two_blocks{seed}", rest_x=X, tets=T, x0=X.copy(), v0=v0, youngs=youngs, poisson=poisson,
                 density=1000.0, dt=dt, dhat=dhat, kappa=kappa, gravity=(0.0, 0.0, -9.8),
                 plane=((0.0, 0.0, 1.0), 0.0) if plane else None, iters=iters, steps=steps)


def objects(seed: int = 0, n: int = 3, side: float = 0.03, dhat: float = 2e-3, iters: int = 20) -> Scene:
    """Three objects of one scene for per-object splitting (Sec. 5.2): the two blocks of `two_blocks(seed)` (the
    rotated upper block falling onto the lower one, which rests a little above the plane) and a third block
    falling freely well away from both.  scene_of_vert holds the object of each vertex (0, 1, 2)."""
    ab = two_blocks(seed, n=n, side=side, dhat=dhat, iters=iters)
    Xc, Tc = kuhn_grid(n, n, n, size=(side, side, side), origin=(4.0 * side, 0.0, 0.02))
    na = kuhn_grid(n, n, n)[0].shape[0]
    X = np.concatenate([ab.rest_x, Xc])
    T = np.concatenate([ab.tets, Tc + ab.n_verts]).astype(np.int32)
    v0 = np.concatenate([ab.v0, np.zeros_like(Xc)])
    obj = np.concatenate([np.zeros(na), np.ones(ab.n_verts - na), np.full(Xc.shape[0], 2)]).astype(np.int32)
    return Scene(name=f"objects{seed}", rest_x=X, tets=T, x0=X.copy(), v0=v0, youngs=ab.youngs, poisson=ab.poisson,
                 density=ab.density, dt=ab.dt, dhat=dhat, kappa=ab.kappa, gravity=ab.gravity, plane=ab.plane,
                 scene_of_vert=obj, iters=iters, steps=3)


def toss(n: int = 24, side: float = 0.1, dt: float = 1.0 / 60.0, steps: int = 20, seed: int = 3,
         youngs: float = 1e5, poisson: float = 0.4, dhat: float = 1e-3, kappa: float = 1e4, iters: int = 50,
         height: float = 0.02) -> Scene:
    """A cube of n^3 cells tossed with a seeded velocity onto the plane z = 0."""
    X, T = kuhn_grid(n, n, n, size=(side, side, side), origin=(0.0, 0.0, height))
    rng = np.random.default_rng(seed)
    v = rng.normal(scale=0.5, size=3) + np.array([0.5, 0.0, 1.0])
    v0 = np.tile(v, (X.shape[0], 1))
    return Scene(name=f"toss{n}", rest_x=X, tets=T, x0=X.copy(), v0=v0, youngs=youngs, poisson=poisson,
                 density=1000.0, dt=dt, dhat=dhat, kappa=kappa, gravity=(0.0, 0.0, -9.8),
                 plane=((0.0, 0.0, 1.0), 0.0), iters=iters, steps=steps)


def pile(n_bars: int = 10, cells=(16, 16, 64), size=(0.1, 0.1, 0.4), seed: int = 4, youngs: float = 2e5,
         poisson: float = 0.4, dt: float = 1.0 / 30.0, dhat: float = 5e-4, kappa: float = 1e4, iters: int = 50,
         steps: int = 200, gap: float = 2.0, jitter: bool = True) -> Scene:
    """Bars stacked criss-cross in layers of two (alternating along x and y), gap*dhat vertical gaps, seeded
    jitter of +-1 mm and +-2 degrees (none with jitter=False), dropped onto the plane z = 0.  With gap < 1 and no
    jitter every crossing starts face to face within dhat: a contact-dominated stack."""
    rng = np.random.default_rng(seed)
    Xb, Tb = kuhn_grid(*cells, size=size)
    Xb = Xb - np.array([0.5 * size[0], 0.5 * size[1], 0.5 * size[2]])  # centred, long axis z
    # lay the bar along x: (x,y,z) -> (z, y, -x) keeps orientation (proper rotation)
    lay_x = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    thick = size[0]
    Xs, Ts = [], []
    off = 0
    for b in range(n_bars):
        layer, slot = divmod(b, 2)
        R = lay_x if layer % 2 == 0 else rot_z(math.pi / 2) @ lay_x
        ang = math.radians(rng.uniform(-2.0, 2.0))
        R = rot_z(ang if jitter else 0.0) @ R
        Y = Xb @ R.T
        lateral = (slot - 0.5) * 1.5 * size[1]
        shift = np.array([0.0, lateral, 0.0]) if layer % 2 == 0 else np.array([lateral, 0.0, 0.0])
        jit = rng.uniform(-1e-3, 1e-3, size=2)
        shift = shift + np.append(jit if jitter else np.zeros(2), 0.0)
        Y = Y + shift
        Y[:, 2] += -Y[:, 2].min() + gap * dhat + layer * (thick + gap * dhat)
        Xs.append(Y)
        Ts.append(Tb + off)
        off += Y.shape[0]
    X = np.concatenate(Xs)
    T = np.concatenate(Ts).astype(np.int32)
    return Scene(name=f"pile{n_bars}", rest_x=X, tets=T, x0=X.copy(), v0=np.zeros_like(X), youngs=youngs,
                 poisson=poisson, density=1000.0, dt=dt, dhat=dhat, kappa=kappa, gravity=(0.0, 0.0, -9.8),
                 plane=((0.0, 0.0, 1.0), 0.0), iters=iters, steps=steps)


def batched(n_scenes: int = 256, seed: int = 2, n_min: int = 4, n_max: int = 16, cell: float = 0.0125,
            e_min: float = 5e4, e_max: float = 5e5, poisson: float = 0.4, dt: float = 1.0 / 60.0, dhat: float = 1e-3,
            kappa: float = 1e4, iters: int = 50, steps: int = 60, spacing: float = 0.5) -> Scene:
    """Independent cubes of n^3 Kuhn cells, n ~ U{n_min..n_max}, each with a uniform-random rotation (normalised
    Gaussian quaternion), its lowest vertex U[0.01, 0.05] m above the plane z = 0 and its own Young's modulus
    E ~ U[e_min, e_max]; laid out on a square grid `spacing` apart so that no two scenes overlap.  Vertices and
    tets are ordered scene by scene (scene_of_vert)."""
    rng = np.random.default_rng(seed)
    cols = int(math.ceil(math.sqrt(n_scenes)))
    Xs, Ts, Es, Ss = [], [], [], []
    off = 0
    for s in range(n_scenes):
        n = int(rng.integers(n_min, n_max + 1))
        side = n * cell
        X, T = kuhn_grid(n, n, n, size=(side, side, side))
        R = random_rotation(rng)
        X = (X - 0.5 * side) @ R.T
        h = rng.uniform(0.01, 0.05)
        r, q = divmod(s, cols)
        X = X - np.array([0.0, 0.0, X[:, 2].min()]) + np.array([q * spacing, r * spacing, h])
        Xs.append(X)
        Ts.append(T + off)
        Es.append(np.full(T.shape[0], rng.uniform(e_min, e_max)))
        Ss.append(np.full(X.shape[0], s, dtype=np.int32))
        off += X.shape[0]
    X = np.concatenate(Xs)
    return Scene(name=f"batched{n_scenes}", rest_x=X, tets=np.concatenate(Ts).astype(np.int32), x0=X.copy(),
                 v0=np.zeros_like(X), youngs=1.0, poisson=poisson, density=1000.0, dt=dt, dhat=dhat, kappa=kappa,
                 gravity=(0.0, 0.0, -9.8), plane=((0.0, 0.0, 1.0), 0.0), youngs_per_tet=np.concatenate(Es),
                 scene_of_vert=np.concatenate(Ss), iters=iters, steps=steps)


def perturbed(scene: Scene, seed: int, scale: float) -> np.ndarray:
    """Seeded copy of the scene's initial positions with N(0, scale^2) noise on free vertices."""
    rng = np.random.default_rng(seed)
    x = scene.x0 + rng.normal(scale=scale, size=scene.x0.shape)
    if scene.fixed is not None:
        x[scene.fixed.astype(bool)] = scene.x0[scene.fixed.astype(bool)]
    return x
