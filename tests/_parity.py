"""Error measures shared by the GPU parity tests (the oracle's values are the reference).

Besides the relative 2-norm over all entries, every vector is checked entry by entry against a per-entry scale:
the sum of the lengths of the contributions (3-vectors) that make up that vertex's entries (the oracle's
grad_diag_scale for g and diag(H)), the bound a rounding error of each contribution is relative to, plus 1e-6 of
the largest entry's scale
(FLOOR), for entries whose contributions vanish in exact arithmetic (a tet at rest has zero stress in the oracle and
a stress of rounding size in any other evaluation).  A global 2-norm can hide a large error on the few entries of
contact vertices; the entry-wise bound and the 2-norm restricted to contact vertices cannot.
"""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


FLOOR = 1e-6


def entrywise(a, ref, scale, floor=None):
    """max_i max(|a_i - ref_i| - floor_i, 0) / (scale_i + FLOOR max_j scale_j); where every scale is zero the
    entries must match exactly."""
    a, ref, scale = (np.asarray(v, dtype=np.float64).ravel() for v in (a, ref, scale))
    if scale.size:
        scale = scale + FLOOR * scale.max()
    d = np.abs(a - ref)
    if floor is not None:
        d = np.maximum(d - np.asarray(floor, dtype=np.float64).ravel(), 0.0)
    pos = scale > 0
    if np.any(d[~pos] > 0):
        return float("inf")
    return float(np.max(d[pos] / scale[pos])) if pos.any() else 0.0


def contact_mask(o, x, fixed=None):
    """Entries [nv, 3] of the vertices of active pairs and of vertices within dhat of the plane (free ones)."""
    m = o.contact_vertices(x).astype(bool)
    if fixed is not None:
        m &= ~fixed
    return np.repeat(m[:, None], 3, axis=1)


def grad_errors(o, x, xt, g, go, diag=None, diago=None, P=None, Po=None, fixed=None):
    """Entry-wise and contact-restricted errors of the GPU's g (and diag, P) against the oracle's at x.  P's scale
    follows from diag's: |dP| / P = |d diag| / diag <= tol * scale(diag) / |diag|."""
    gs, ds = o.grad_diag_scale(x, xt)
    _, do, _ = o.grad_diag(x, xt)
    free = np.ones(x.shape, bool) if fixed is None else np.repeat(~fixed[:, None], 3, axis=1)
    cm = contact_mask(o, x, fixed)
    out = {"g_entry": entrywise(g[free], go[free], gs[free]),
           "g_contact": rel(g[cm], go[cm]) if cm.any() else 0.0}
    if diag is not None:
        out["diag_entry"] = entrywise(diag[free], diago[free], ds[free])
        out["diag_contact"] = rel(diag[cm], diago[cm]) if cm.any() else 0.0
    if P is not None:
        sP = np.abs(Po) * ds / np.maximum(np.abs(do), 1e-300)
        out["P_entry"] = entrywise(P[free], Po[free], sP[free])
        out["P_contact"] = rel(P[cm], Po[cm]) if cm.any() else 0.0
    return out


def direction_entry(p1, P1, g1, beta, p0):
    """Entry-wise error of the GPU direction p1 against -P1 g1 + beta p0 formed in double from the GPU's own P1, g1,
    p0 and beta, relative to |P1 g1| + |beta p0|.  (beta itself, a ratio of reductions that can cancel, is checked
    against the oracle's through the 2-norm of the direction.)"""
    P1, g1, p0 = (np.asarray(a, dtype=np.float64).ravel() for a in (P1, g1, p0))
    ref = -P1 * g1 + beta * p0
    scale = np.abs(P1 * g1) + abs(beta) * np.abs(p0)
    return entrywise(np.asarray(p1).ravel(), ref, scale)


def beta_scale(g1, P1, g0, P0, p0, k, rule=0):
    """The magnitude of beta's terms (Sec. 4.1): for beta = N / D formed from sums of per-entry products, rounding of
    relative size u in each product (the FP32 form's inputs g, P and y = g1 - g0 are float) moves beta by up to
    u (sum |n_i| + |beta| sum |d_i|) / |D|.  PR+: N = g1 P1 y, D = g0 P0 g0.  DK: beta = gPy / yp - yPy pg / yp^2, the
    same first-order bound over its four sums.  Zero at k = 0 (beta = 0 on both sides)."""
    if k == 0:
        return 0.0
    g1, P1, g0, P0, p0 = (np.asarray(a, dtype=np.float64).ravel() for a in (g1, P1, g0, P0, p0))
    y = g1 - g0
    if rule == 0:
        D = float(np.dot(g0 * P0, g0))
        if not D > 0.0:
            return 0.0
        beta = max(float(np.dot(g1 * P1, y)) / D, 0.0)
        return float(np.abs(g1 * P1 * y).sum()) / D + beta
    S1, S2, S3, S4 = (float(np.dot(g1 * P1, y)), float(np.dot(y * P1, y)), float(np.dot(y, p0)), float(np.dot(p0, g1)))
    if abs(S3) < 1e-30:
        return 0.0
    A1, A3, A4 = float(np.abs(g1 * P1 * y).sum()), float(np.abs(y * p0).sum()), float(np.abs(p0 * g1).sum())
    return (A1 / abs(S3) + abs(S1) * A3 / S3 ** 2 + (S2 * abs(S4) + S2 * A4) / S3 ** 2 +
            2.0 * S2 * abs(S4) * A3 / abs(S3) ** 3)


def direction_error(p1, pd, g1, P1, g0, P0, p0, k, rule=0):
    """|p1 - pd| / (|pd| + beta_scale |p0|): the GPU direction against the oracle's (-P1 g1 + beta p0 with the
    oracle's beta from the same g1, P1, g0, P0, p0), relative to the direction plus what beta's rounding can move
    it by."""
    p1, pd, p0 = (np.asarray(a, dtype=np.float64).ravel() for a in (p1, pd, p0))
    den = np.linalg.norm(pd) + beta_scale(g1, P1, g0, P0, p0, k, rule) * np.linalg.norm(p0)
    return float(np.linalg.norm(p1 - pd) / max(den, 1e-300))


def update_entry(x1, x, alpha, p1):
    """Entry-wise error of the update x1 - x against alpha p1, relative to |alpha p1| beyond 4 ulp of x."""
    ref = alpha * np.asarray(p1)
    floor = 4 * np.spacing(np.abs(np.asarray(x1))) + 4 * np.spacing(np.abs(np.asarray(x)))
    return entrywise(np.asarray(x1) - np.asarray(x), ref, np.abs(ref), floor)


def pHp_pair_scale(O, o, x, p, dhat, kappa):
    """The magnitude of the barrier terms of p^T H p at x (Eqs. 12-13): the sum over the active pairs of
    |A (c.p . t)^2| + |B |c.p|^2|, A = kappa (b''/d^2 - b'/d^3), B = kappa b'/d, with c.p = sum_i c_i p_i.  The two
    terms have opposite signs (b' < 0) and the pairs' sum can cancel, so a float evaluation's rounding is relative to
    this, not to the net p^T H p."""
    idx, _, _ = o.active_pairs(x)
    s = 0.0
    for row in idx:
        t, vv = int(row[0]), [int(v) for v in row[1:]]
        d, c, tt = O.pair_geometry(t, x[vv])
        b = O.barrier_fn(d, dhat)
        cp = (c[:, None] * p[vv]).sum(axis=0)
        A = kappa * (b[2] / d ** 2 - b[1] / d ** 3)
        B = kappa * b[1] / d
        s += abs(A) * float(cp @ tt) ** 2 + abs(B) * float(cp @ cp)
    return s
