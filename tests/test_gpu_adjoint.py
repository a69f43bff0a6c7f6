"""GPU tests of the differentiation form: the Hessian-vector kernel against the oracle's p^T H p (polarisation),
the adjoint gradients (per-tet Young's modulus, initial velocity) against central finite differences of the
oracle's own forward run, and every reverse step against the oracle's own adjoint step (on the 3-cell drop and on a
two-step slice of the 82,944-tet differentiation config)."""
import numpy as np
import pytest

from paper_2405_08001_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2405_08001_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def lowered_cube():
    sc = S.cube_drop(n=8, cells=(5, 4, 6), drop=0.0)
    sc.x0 = sc.x0 + np.array([0.0, 0.0, 0.4 * sc.dhat])
    sc.rest_x = sc.x0.copy()
    return sc


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("make", [lowered_cube, lambda: S.two_blocks(0)])
def test_hvp_is_the_oracle_bilinear_form(B, O, make, prec):
    """p . (H v) from the kernel equals the oracle's bilinear form (p^T H p by polarisation: the oracle's quadratic
    form is pinned by finite differences on the CPU), for several p and v; H is symmetric."""
    sc = make()
    sim = B.Sim(sc, precision=prec)
    o = O.Oracle.from_scene(sc)
    rng = np.random.default_rng(3)
    x = sc.x0 + 2e-5 * rng.normal(size=sc.x0.shape)
    tol = 1e-10 if prec == 0 else 1e-5
    for _ in range(3):
        v = rng.normal(size=x.shape)
        Hv = B.sim_eval_hvp(sim.h, x, v)
        for _ in range(3):
            p = rng.normal(size=x.shape)
            ref = 0.25 * (o.pHp(x, p + v) - o.pHp(x, p - v))
            scale = 0.25 * (abs(o.pHp(x, p + v)) + abs(o.pHp(x, p - v)))
            assert abs(np.vdot(p, Hv) - ref) / scale < tol
        Hp = B.sim_eval_hvp(sim.h, x, p)
        assert abs(np.vdot(p, Hv) - np.vdot(v, Hp)) / abs(np.vdot(v, Hp)) < tol
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("model", [1, 2, 3])
def test_hvp_other_densities(B, O, model, prec):
    """The Hessian-vector kernel for the stable Neo-Hookean, fixed corotated and as-rigid-as-possible densities
    against the oracle's H v (its I1 term from the polar decomposition), on the lowered cube at a strained state:
    the rest shape stretched by 3 % along x and sheared, plus noise, so that S differs from I and R from a plain
    rotation; and p . (H v) = v . (H p)."""
    sc = lowered_cube()
    sim = B.Sim(sc, precision=prec, model=model)
    o = O.Oracle.from_scene(sc, model=model)
    rng = np.random.default_rng(31 + model)
    c = sc.x0.mean(axis=0)
    A = np.array([[1.03, 0.02, 0.0], [0.0, 0.99, 0.015], [0.0, 0.0, 1.0]])
    x = (sc.x0 - c) @ A.T + c + 2e-5 * rng.normal(size=sc.x0.shape)
    tol = 1e-10 if prec == 0 else 1e-5
    for _ in range(3):
        v = rng.normal(size=x.shape)
        Hv = B.sim_eval_hvp(sim.h, x, v)
        ref = o.hvp(x, v)
        assert np.linalg.norm(Hv - ref) <= tol * np.linalg.norm(ref)
        p = rng.normal(size=x.shape)
        Hp = B.sim_eval_hvp(sim.h, x, p)
        assert abs(np.vdot(p, Hv) - np.vdot(v, Hp)) <= tol * abs(np.vdot(v, Hp))
    sim.close()


def drop_scene(iters=1000, steps=5):
    """A 3-cell cube 1.5 mm above the plane, falling and tipping: the barrier is active from the first step.  1000
    iterations per step converge every step to rounding (200 leave 3e-9 m, which biases central differences of
    the run by a few percent)."""
    sc = S.cube_drop(n=3, drop=0.0015, iters=iters, steps=steps)
    sc.v0 = np.tile(np.array([0.05, -0.02, -0.2]), (sc.n_verts, 1))
    return sc


def centroid_loss(x, target):
    d = x.mean(axis=0) - target
    return float(d @ d)


def oracle_forward(O, sc, youngs, v0, steps):
    import dataclasses
    s2 = dataclasses.replace(sc, youngs=1.0, youngs_per_tet=youngs, v0=v0)
    o = O.Oracle.from_scene(s2)
    x, v = s2.x0.copy(), s2.v0.copy()
    for t in range(steps):
        o.step(x, v, s2.targets(t), iters=s2.iters)
    return x


def test_adjoint_gradients_match_oracle_finite_differences(B, O):
    """FP64: dL/dE (per tet) and dL/dv0 from the adjoint equal central differences (relative step 1e-4) of the loss
    computed with the oracle's forward run, along random directions."""
    import torch
    from paper_2405_08001_gb300 import diff
    sc = drop_scene()
    steps = sc.steps
    rng = np.random.default_rng(11)
    E0 = np.full(sc.n_tets, 1e5) * (1.0 + 0.2 * rng.uniform(-1, 1, sc.n_tets))
    target = sc.x0.mean(axis=0) + np.array([0.01, 0.0, -0.005])
    Et = torch.tensor(E0, dtype=torch.float64, requires_grad=True)
    vt = torch.tensor(sc.v0, dtype=torch.float64, requires_grad=True)
    xT = diff.simulate(Et, vt, sc, steps)
    tt = torch.tensor(target, dtype=torch.float64)
    L = ((xT.mean(dim=0) - tt) ** 2).sum()
    L.backward()
    gE, gv = Et.grad.numpy(), vt.grad.numpy()
    # the GPU forward agrees with the oracle's
    x_or = oracle_forward(O, sc, E0, sc.v0, steps)
    assert np.abs(xT.detach().numpy() - x_or).max() < 1e-10
    for _ in range(2):
        uE = rng.normal(size=E0.shape) * E0
        eps = 1e-4
        Lp = centroid_loss(oracle_forward(O, sc, E0 + eps * uE, sc.v0, steps), target)
        Lm = centroid_loss(oracle_forward(O, sc, E0 - eps * uE, sc.v0, steps), target)
        fd = (Lp - Lm) / (2 * eps)
        ad = float(gE @ uE)
        assert abs(ad - fd) <= 1e-3 * abs(fd) + 1e-12, (ad, fd)
        uv = rng.normal(size=sc.v0.shape)
        h = 1e-4 * np.abs(sc.v0).max()
        Lp = centroid_loss(oracle_forward(O, sc, E0, sc.v0 + h * uv, steps), target)
        Lm = centroid_loss(oracle_forward(O, sc, E0, sc.v0 - h * uv, steps), target)
        fd = (Lp - Lm) / (2 * h)
        ad = float(np.vdot(gv, uv))
        assert abs(ad - fd) <= 1e-3 * abs(fd) + 1e-12, (ad, fd)


def test_adjoint_fp32_matches_fp64(B):
    """The FP32-mixed form's adjoint gradients agree with the FP64 form's (relative 2-norm 1e-3)."""
    import torch
    from paper_2405_08001_gb300 import diff
    sc = drop_scene()
    rng = np.random.default_rng(12)
    E0 = np.full(sc.n_tets, 1e5) * (1.0 + 0.2 * rng.uniform(-1, 1, sc.n_tets))
    target = torch.tensor(sc.x0.mean(axis=0) + np.array([0.01, 0.0, -0.005]))
    out = {}
    for prec in (0, 1):
        Et = torch.tensor(E0, dtype=torch.float64, requires_grad=True)
        vt = torch.tensor(sc.v0, dtype=torch.float64, requires_grad=True)
        xT = diff.simulate(Et, vt, sc, sc.steps, precision=prec, tol=1e-10 if prec == 0 else 1e-6)
        ((xT.mean(dim=0) - target) ** 2).sum().backward()
        out[prec] = (Et.grad.numpy(), vt.grad.numpy())
    for a, b in zip(out[1], out[0]):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3


def test_differentiation_config_full_size(B, O):
    """The differentiation config's cube at full size (24^3 cells, 82,944 tets, the seeded toss velocity).

    The adjoint differentiates the minimiser of each step.  PNCG converges slowly on this mesh once the cube
    vibrates (300 iterations reduce Delta E by only ~1e-3 from the second step on) and its step cap (d^/2 per
    iteration) needs many iterations for a fast toss, so finite differences of a multi-step run measure the
    truncated iteration, not the minimiser.  Checked instead: (a) one step from a tenth of the toss velocity plus a
    seeded random velocity field (so that elastic forces act), 4000 iterations: directional derivatives for E_e
    (vertex-wise loss) and v0 (the config's centroid loss) against central differences of the GPU's FP64 forward;
    (b) six steps of flight at the toss velocity with the config's loss: the implicit step conserves momentum and
    the centroid mode of H is the mass, so dL/dv0_i = 2 (c_T - target) T h m_i / sum m exactly, and dL/dE
    vanishes."""
    import torch
    from paper_2405_08001_gb300 import diff
    sc = S.toss(iters=300)
    rng = np.random.default_rng(13)
    E0 = np.full(sc.n_tets, sc.youngs)
    target = sc.x0.mean(axis=0) + rng.uniform(-0.02, 0.02, 3)
    tt = torch.tensor(target)
    shape = torch.tensor(sc.x0 + rng.normal(scale=1e-3, size=sc.x0.shape))
    mass = O.Oracle.from_scene(sc).mass()

    def centroid(x):
        m = torch.tensor(mass)
        return (m[:, None] * x).sum(dim=0) / m.sum()

    def losses(x):
        return ((centroid(x) - tt) ** 2).sum(), ((x - shape) ** 2).sum()

    import dataclasses
    sc1 = dataclasses.replace(sc, iters=4000)

    def grad(which, steps, v0, scene=sc):
        Et = torch.tensor(E0, dtype=torch.float64, requires_grad=True)
        vt = torch.tensor(v0, dtype=torch.float64, requires_grad=True)
        x = diff.simulate(Et, vt, scene, steps)
        losses(x)[which].backward()
        return Et.grad.numpy().copy(), vt.grad.numpy().copy(), x.detach()

    def loss(E, v0, which, steps, scene=sc1):
        with torch.no_grad():
            return float(losses(diff.simulate(torch.tensor(E), torch.tensor(v0), scene, steps))[which])

    # (a) one converged step
    slow = 0.1 * sc.v0 + 0.1 * rng.normal(size=sc.v0.shape)
    gE, _, _ = grad(1, 1, slow, sc1)
    uE = rng.normal(size=E0.shape) * E0
    fd = (loss(E0 + 1e-4 * uE, slow, 1, 1) - loss(E0 - 1e-4 * uE, slow, 1, 1)) / 2e-4
    # the difference resolves Delta L ~ 2e-11 against L ~ 0.05 (rounding of L ~ 1e-17 per term over 47K terms,
    # and FP64 atomics vary the forward's last bits from run to run): about 1e-3 of noise in fd
    assert abs(float(gE @ uE) - fd) <= 5e-3 * abs(fd), (float(gE @ uE), fd)
    _, gv, _ = grad(0, 1, slow, sc1)
    uv = rng.normal(size=sc.v0.shape)
    h = 1e-4 * np.abs(slow).max()
    fd = (loss(E0, slow + h * uv, 0, 1) - loss(E0, slow - h * uv, 0, 1)) / (2 * h)
    assert abs(float(np.vdot(gv, uv)) - fd) <= 1e-3 * abs(fd), (float(np.vdot(gv, uv)), fd)
    # (b) six steps of flight: momentum
    steps = 6
    gE, gv, xT = grad(0, steps, sc.v0)
    assert xT[:, 2].min() > 2 * sc.dhat
    cT = centroid(xT).numpy()
    exact = 2.0 * (cT - target)[None, :] * steps * sc.dt * mass[:, None] / mass.sum()
    assert np.linalg.norm(gv - exact) / np.linalg.norm(exact) < 1e-6
    assert abs(float(gE @ uE)) < 1e-6 * np.linalg.norm(exact) * np.linalg.norm(uE) / np.sqrt(sc.n_tets)


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_adjoint_steps_match_the_oracle_adjoint(B, O, model):
    """Each reverse step of the library (sim_adjoint_step) against the oracle's own adjoint step (its CG on its
    Hessian-vector product, pinned on the CPU) from the same end state and adjoints, along the 3-cell drop's run:
    dL/dx_t, dL/dv_t and the accumulated dL/dE_e; for each of the four densities."""
    sc = drop_scene()
    rng = np.random.default_rng(21)
    E0 = np.full(sc.n_tets, 1e5) * (1.0 + 0.2 * rng.uniform(-1, 1, sc.n_tets))
    import dataclasses
    s2 = dataclasses.replace(sc, youngs=1.0, youngs_per_tet=E0)
    sim = B.Sim(s2, precision=0, model=model)
    o = O.Oracle.from_scene(s2, model=model)
    xs = [s2.x0.copy()]
    for t in range(s2.steps):
        sim.step(1)
        xs.append(sim.state()[0])
    ax = rng.normal(size=s2.x0.shape)
    av = rng.normal(size=s2.x0.shape)
    axo, avo = ax.copy(), av.copy()
    dE, dEo = np.zeros(s2.n_tets), np.zeros(s2.n_tets)
    for t in range(s2.steps, 0, -1):
        ax, av, it, res = B.sim_adjoint_step(sim.h, xs[t], ax, av, dE=dE, tol=1e-13, max_iters=20000)
        axo, avo, ito, reso = o.adjoint_step(xs[t], axo, avo, dE=dEo, tol=1e-13, max_iters=20000)
        assert res < 1e-12 and reso < 1e-12
        for a, b in ((ax, axo), (av, avo), (dE, dEo)):
            assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b), (t, np.linalg.norm(a - b) / np.linalg.norm(b))
    sim.close()


def test_differentiation_config_two_step_slice_matches_the_oracle_adjoint(B, O):
    """The differentiation config at full size (24^3 cells, 82,944 tets, seeded toss velocity, per-tet Young's
    moduli): two FP64 forward steps through the library, then the two reverse steps of the library and of the oracle
    from the same checkpoints: dL/dx_0, dL/dv_0 and dL/dE_e agree to the CG tolerance.  The loss adds to the
    config's |centroid - target|^2 a vertex-wise |x - s|^2 to a seeded shape s: in flight the centroid loss has no
    elastic part (dL/dE vanishes by momentum conservation), the vertex-wise one does."""
    import dataclasses
    sc = S.toss()
    rng = np.random.default_rng(22)
    E0 = np.full(sc.n_tets, sc.youngs) * (1.0 + 0.2 * rng.uniform(-1, 1, sc.n_tets))
    s2 = dataclasses.replace(sc, youngs=1.0, youngs_per_tet=E0)
    sim = B.Sim(s2, precision=0)
    o = O.Oracle.from_scene(s2)
    xs = [s2.x0.copy()]
    for t in range(2):
        sim.step(1)
        xs.append(sim.state()[0])
    mass = o.mass()
    target = sc.x0.mean(axis=0) + rng.uniform(-0.02, 0.02, 3)
    c = (mass[:, None] * xs[-1]).sum(axis=0) / mass.sum()
    shape = sc.x0 + rng.normal(scale=1e-3, size=sc.x0.shape)
    ax = 2.0 * (c - target)[None, :] * mass[:, None] / mass.sum() + 2.0 * (xs[-1] - shape)
    av = np.zeros_like(ax)
    axo, avo = ax.copy(), av.copy()
    dE, dEo = np.zeros(s2.n_tets), np.zeros(s2.n_tets)
    for t in (2, 1):
        ax, av, it, res = B.sim_adjoint_step(sim.h, xs[t], ax, av, dE=dE, tol=1e-10, max_iters=20000)
        axo, avo, ito, reso = O.Oracle.adjoint_step(o, xs[t], axo, avo, dE=dEo, tol=1e-10, max_iters=20000)
        assert res <= 1e-10 and reso <= 1e-10, (res, reso)
    for a, b in ((ax, axo), (av, avo), (dE, dEo)):
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(b), np.linalg.norm(a - b) / np.linalg.norm(b)
    sim.close()


def test_differentiation_config_twenty_converged_steps(B):
    """All twenty steps of the differentiation config (82,944-tet cube, dt = 1/60) with every step converged: the
    initial-velocity gradient against central differences of the GPU's FP64 forward.  The toss is given 0.7 m/s more
    upward speed and a seeded random velocity field (0.1 m/s per component): the cube then stays airborne for the
    twenty steps, spinning and vibrating, and PNCG converges each step to Delta E < 1e-14 Delta E_0 in about 1,500
    iterations.  (On the plane it does not converge within 3,000 iterations, so differences there measure the
    truncation, not the minimiser.)  Every step runs a fixed 2,500 iterations (an eps rule would stop the two runs
    of a difference at different iterations, a jump in x_T that the difference would see), and the forward uses the
    segmented scatter, whose sums are bitwise reproducible.
    Loss: the vertex-wise distance of x_T to a seeded shape.  The Young's-modulus gradient is not checked here: implicit
    Euler at this dt damps the cube's vibration within a few steps (its lowest modes have omega dt of about 5), so
    x_T depends on E by about 1e-6 of the loss, below what the eps rule's truncation lets a difference resolve; it is
    checked on a converged single step of this config above, against the oracle's adjoint on a two-step slice, and
    against the oracle's differences on the 3-cell drop."""
    import dataclasses
    import torch
    from paper_2405_08001_gb300 import diff
    sc = S.toss(iters=2500)
    rng = np.random.default_rng(29)
    v0 = sc.v0 + np.array([0.0, 0.0, 0.7]) + 0.1 * rng.normal(size=sc.v0.shape)
    E0 = np.full(sc.n_tets, sc.youngs)
    shape = torch.tensor(sc.x0 + rng.normal(scale=1e-3, size=sc.x0.shape))
    opts = {"scatter": B.SIM_SCATTER_SEGMENTED}
    # every step converged and airborne
    sim = B.Sim(dataclasses.replace(sc, v0=v0), precision=B.SIM_FP64, **opts)
    for t in range(sc.steps):
        sim.step(1, sc.targets(t))
        x, _, st = sim.state()
        assert abs(st["dE_last"]) <= 1e-14 * st["dE0"], (t, st["dE_last"], st["dE0"])
        assert x[:, 2].min() > 10 * sc.dhat
    sim.close()

    def loss(v):
        with torch.no_grad():
            xT = diff.simulate(torch.tensor(E0), torch.tensor(v), sc, sc.steps, options=opts)
            return float(((xT - shape) ** 2).sum())

    vt = torch.tensor(v0, dtype=torch.float64, requires_grad=True)
    ((diff.simulate(torch.tensor(E0), vt, sc, sc.steps, options=opts) - shape) ** 2).sum().backward()
    gv = vt.grad.numpy()
    uv = rng.normal(size=v0.shape)
    hv = 1e-3 * np.abs(v0).max()
    fd = (loss(v0 + hv * uv) - loss(v0 - hv * uv)) / (2 * hv)
    assert abs(float(np.vdot(gv, uv)) - fd) <= 1e-3 * abs(fd), (float(np.vdot(gv, uv)), fd)


def test_fp32_adjoint_steps_match_the_oracle_adjoint(B, O):
    """The FP32 form's reverse steps against the oracle's (FP64) adjoint steps along the 3-cell drop's run (its
    states from the FP64 form).  A linear solve turns an operator error of relative size eps into a solution error
    of at most cond(H) eps, and each reverse step starts from the previous one's result: the bound after k reverse
    steps is 10 k cond(H) eps, with cond(H) from the oracle's dense Hessian at the state (its columns are H e_j) and
    eps the FP32 Hessian-vector kernel's measured error there, max over random v of |H v - H_oracle v| / (|H| |v|)."""
    sc = drop_scene()
    rng = np.random.default_rng(23)
    sim64 = B.Sim(sc, precision=0)
    xs = [sc.x0.copy()]
    for t in range(sc.steps):
        sim64.step(1)
        xs.append(sim64.state()[0])
    sim64.close()
    sim = B.Sim(sc, precision=1)
    o = O.Oracle.from_scene(sc)
    ax = rng.normal(size=sc.x0.shape)
    av = rng.normal(size=sc.x0.shape)
    axo, avo = ax.copy(), av.copy()
    dE, dEo = np.zeros(sc.n_tets), np.zeros(sc.n_tets)
    n = 3 * sc.n_verts
    for k, t in enumerate(range(sc.steps, 0, -1), start=1):
        H = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            H[:, j] = o.hvp(xs[t], e.reshape(-1, 3)).ravel()
        ev = np.abs(np.linalg.eigvalsh(0.5 * (H + H.T)))
        cond = ev.max() / ev.min()
        eps = 0.0
        for _ in range(4):
            v = rng.normal(size=sc.x0.shape)
            hv = B.sim_eval_hvp(sim.h, xs[t], v)
            eps = max(eps, np.linalg.norm(hv - o.hvp(xs[t], v)) / (ev.max() * np.linalg.norm(v)))
        ax, av, it, res = B.sim_adjoint_step(sim.h, xs[t], ax, av, dE=dE, tol=1e-9, max_iters=20000)
        axo, avo, ito, reso = o.adjoint_step(xs[t], axo, avo, dE=dEo, tol=1e-13, max_iters=20000)
        bound = 10 * k * cond * eps
        for a, b in ((ax, axo), (av, avo), (dE, dEo)):
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err <= bound, (t, err, cond, eps)
    sim.close()
