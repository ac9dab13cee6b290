"""Pins of the FP64 oracle against what the paper and geometry fix.

None of these re-types the oracle's residual: each check uses a different
route to the same answer (image method, Keller's equal-angle closed form, the
paraboloid focus property, Fermat grid search, dense sampling of segments,
networkx path counting, published SplitMix64 outputs, central differences).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2301_06399_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FULL2 = S.SequenceSpec(quota=(-1, -1, 0, 0))


# ----------------------------------------------------------------- helpers --
def image_method(tx, rx, planes):
    """Image method (Sec. III-A): forward images (Eq. 5), backward points
    (Eq. 6).  planes: list of (n, P) with unit normal n and a point P.
    Returns (points, lambdas); the path exists when every lambda is in (-1, 0)
    (X_k strictly between X_{k+1} and the image I_k)."""
    imgs = [np.asarray(tx, float)]
    for (n, P) in planes:
        I = imgs[-1]
        imgs.append(I - 2.0 * np.dot(I - P, n) * n)
    X = [None] * (len(planes) + 2)
    X[-1] = np.asarray(rx, float)
    lams = [0.0] * len(planes)
    for k in range(len(planes), 0, -1):
        n, P = planes[k - 1]
        Xn, I = X[k + 1], imgs[k]
        den = np.dot(Xn - I, n)
        lam = np.dot(P - Xn, n) / den if den != 0 else np.inf
        lams[k - 1] = lam
        X[k] = Xn + lam * (Xn - I)
    return np.array(X[1:-1]), np.array(lams), imgs


def plane_of(scene, obj):
    p = scene.obj_param[obj]
    n = p[0:3]
    return n, n * p[3]


def solve_one(scene, ids, begin_pair=None):
    """Oracle solve + validate of every pair for one explicit sequence."""
    ids = list(ids) + [-1] * (4 - len(ids))
    table = oracle.SequenceTable(np.array([sum(i >= 0 for i in ids)], np.int32),
                                 np.array([ids], np.int32), np.zeros(1, np.int32))
    return oracle.candidate_range(scene, table, 0, scene.n_pairs)


def _builder():
    return S._Builder()


# --------------------------------------------------------------- Fig. 4 ----
def test_fig4_images_match_printed_values():
    g = json.load(open(os.path.join(GOLDEN, "fig4.json")))
    sc = S.fig4_scene(bs=g["BS"], ue=g["UE"], w1=g["W1"], w2=g["W2"])
    planes = [plane_of(sc, 0), plane_of(sc, 1)]
    _, _, imgs = image_method(sc.tx[0], sc.rx[0], planes)
    assert np.allclose(imgs[1][:2], g["I1"], atol=1e-12)
    assert np.allclose(imgs[2][:2], g["I2"], atol=1e-12)


def test_fig4_oracle_path_equals_image_method():
    g = json.load(open(os.path.join(GOLDEN, "fig4.json")))
    sc = S.fig4_scene(bs=g["BS"], ue=g["UE"], w1=g["W1"], w2=g["W2"])
    # backward pass (Eq. 6) from the printed images
    ue = np.array(g["UE"] + [0.0])
    I1 = np.array(g["I1"] + [0.0])
    I2 = np.array(g["I2"] + [0.0])
    n1, P1 = plane_of(sc, 0)
    n2, P2 = plane_of(sc, 1)
    X2 = ue + np.dot(P2 - ue, n2) / np.dot(ue - I2, n2) * (ue - I2)
    X1 = X2 + np.dot(P1 - X2, n1) / np.dot(X2 - I1, n1) * (X2 - I1)
    sol, ver = solve_one(sc, [0, 1])
    assert sol.cost[0] < 1e-28
    assert np.allclose(sol.X[0, 0:3], X1, atol=1e-10)
    assert np.allclose(sol.X[0, 3:6], X2, atol=1e-10)
    # unfolded length equals the distance from the last image to UE
    assert abs(ver.length[0] - np.linalg.norm(ue - I2)) < 1e-10
    assert ver.valid[0] == 1 and ver.ambiguous[0] == 0


def test_fig4_only_the_drawn_path_is_valid():
    """Fig. 4 states the W1 -> W2 path is the only valid one.  Checked facts:
    W1 alone: BS and UE lie on opposite sides of y = x (no reflection);
    W2 alone: the reflected leg from (5, 1.5) to UE crosses W1;
    W2 -> W1: no valid geometry."""
    sc = S.fig4_scene()
    table = oracle.enumerate_sequences(sc, 2, FULL2)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table))
    got = {tuple(table.ids[i][:table.order[i]]): int(ver.valid[i]) for i in range(len(table))}
    assert got == {(0,): 0, (1,): 0, (0, 1): 1, (1, 0): 0}
    # W2 alone does converge (cost ~ 0) but is blocked by W1
    i = [k for k in range(len(table)) if tuple(table.ids[k][:table.order[k]]) == (1,)][0]
    assert sol.cost[i] < 1e-28 and np.allclose(sol.X[i, :3], [5.0, 1.5, 0.0], atol=1e-9)


# ------------------------------------------------------ image method ------
def test_street_canyon_every_candidate_matches_image_method():
    sc = S.street_canyon()
    table = oracle.enumerate_sequences(sc, 2, FULL2)
    assert len(table) == 9
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    checked = 0
    for e in range(len(table)):
        ids = table.ids[e][:table.order[e]]
        planes = [plane_of(sc, o) for o in ids]
        for p in range(sc.n_pairs):
            c = e * sc.n_pairs + p
            tx, rx = sc.pair_points(p)
            X, lam, _ = image_method(tx, rx, planes)
            exists = bool(np.all((lam > -1.0) & (lam < 0.0)))
            margin = np.min(np.minimum(np.abs(lam), np.abs(lam + 1.0)))
            if margin < 1e-6:
                continue
            assert (sol.cost[c] < oracle.TAU) == exists, (ids, p, lam, sol.cost[c])
            if exists:
                assert np.abs(sol.X[c, :3 * len(ids)] - X.reshape(-1)).max() < 1e-9
                checked += 1
    assert checked > 300


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_planar_sequences_match_image_method(seed):
    rng = np.random.default_rng(100 + seed)
    b = _builder()
    for _ in range(3):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u = np.cross(n, [0.3, 0.5, 0.8])
        u /= np.linalg.norm(u)
        v = np.cross(n, u)
        O = rng.uniform(-20, 20, 3) - 500 * u - 500 * v
        b.rect_plane(O, u, v, 1000.0, 1000.0)
    tx = rng.uniform(-30, 30, (1, 3))
    rx = rng.uniform(-30, 30, (24, 3))
    sc = b.build("planes", 100.0, tx, rx)
    spec = S.SequenceSpec(quota=(-1, -1, -1, 0))
    table = oracle.enumerate_sequences(sc, 3, spec)
    sol = oracle.solve(sc, table)
    agree = 0
    for e in range(len(table)):
        ids = table.ids[e][:table.order[e]]
        planes = [plane_of(sc, o) for o in ids]
        for p in range(sc.n_pairs):
            c = e * sc.n_pairs + p
            X, lam, _ = image_method(*sc.pair_points(p), planes)
            exists = bool(np.all((lam > -1.0) & (lam < 0.0)))
            if np.min(np.minimum(np.abs(lam), np.abs(lam + 1.0))) < 1e-3:
                continue
            assert (sol.cost[c] < oracle.TAU) == exists
            if exists:
                assert np.abs(sol.X[c, :3 * len(ids)] - X.reshape(-1)).max() < 1e-8
                agree += 1
    assert agree > 10


# --------------------------------------------------------- Keller ---------
def test_single_straight_edge_matches_keller_closed_form():
    """Equal angles with the edge (Eq. 3, Fig. 2: h_i/|i| = h_d/|d|) give
    t* = (a h_d + b h_i) / (h_i + h_d) along the edge."""
    rng = np.random.default_rng(7)
    b = _builder()
    for _ in range(6):
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        a1 = np.cross(e, [0.2, 0.9, 0.1])
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(e, a1)
        b.line_edge(rng.uniform(-10, 10, 3), e, -1e3, 1e3, a1, a2)
    sc = b.build("edges", 100.0, rng.uniform(-40, 40, (1, 3)), rng.uniform(-40, 40, (32, 3)))
    table = oracle.enumerate_sequences(sc, 1, S.SequenceSpec(quota=(-1, 0, 0, 0)))
    sol = oracle.solve(sc, table)
    for e in range(len(table)):
        p = sc.obj_param[table.ids[e][0]]
        P, ed = p[0:3], p[3:6]
        for q in range(sc.n_pairs):
            tx, rx = sc.pair_points(q)
            a, bb = np.dot(tx - P, ed), np.dot(rx - P, ed)
            hi = np.linalg.norm(tx - P - a * ed)
            hd = np.linalg.norm(rx - P - bb * ed)
            t = (a * hd + bb * hi) / (hi + hd)
            c = e * sc.n_pairs + q
            assert sol.cost[c] < 1e-26
            assert np.linalg.norm(sol.X[c, :3] - (P + t * ed)) < 1e-9


# ------------------------------------------------------ paraboloid --------
def _one_paraboloid(f, R, t):
    b = _builder()
    b.paraboloid(R, t, f, 2.0)
    return b


@pytest.mark.parametrize("reverse", [False, True])
def test_paraboloid_focus_property(reverse):
    """Rays parallel to the axis reflect through the focus (0, 0, f) of
    z = (x^2 + y^2) / (4 f): with one end at the focus and the other on the
    axis-parallel line through (x0, y0), the reflection point is
    (x0, y0, (x0^2 + y0^2) / (4 f))."""
    rng = np.random.default_rng(3)
    R = S._random_rotation(rng)
    t = rng.uniform(-5, 5, 3)
    f = 1.3
    pts = []
    far = []
    for _ in range(12):
        r = 1.8 * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        x0, y0 = r * math.cos(th), r * math.sin(th)
        pts.append(t + R @ np.array([x0, y0, (x0 * x0 + y0 * y0) / (4 * f)]))
        far.append(t + R @ np.array([x0, y0, rng.uniform(6.0, 30.0)]))
    focus = t + R @ np.array([0.0, 0.0, f])
    b = _one_paraboloid(f, R, t)
    if reverse:
        sc = b.build("parab", 100.0, np.array(far), np.repeat(focus[None], 12, 0), pair_mode=1)
    else:
        sc = b.build("parab", 100.0, np.repeat(focus[None], 12, 0), np.array(far), pair_mode=1)
    spec = S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=8)
    table = oracle.enumerate_sequences(sc, 1, spec)
    assert len(table) == 8
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    for q in range(sc.n_pairs):
        cands = [e * sc.n_pairs + q for e in range(len(table))]
        found = [np.linalg.norm(sol.X[c, :3] - pts[q]) for c in cands if sol.cost[c] < oracle.TAU]
        assert found and min(found) < 1e-9


# ------------------------------------------------------- Fermat -----------
def _grid_min(fun, lo, hi, n, iters=6):
    lo, hi = np.array(lo, float), np.array(hi, float)
    best = None
    for _ in range(iters):
        axes = [np.linspace(l, h, n) for l, h in zip(lo, hi)]
        grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, len(lo))
        vals = fun(grid)
        best = grid[np.argmin(vals)]
        span = (hi - lo) / (n - 1) * 2
        lo, hi = best - span, best + span
    return best


def test_fermat_grid_single_reflection_and_two_edges():
    """Fermat: the path length is stationary (here: minimal) at the solution.
    Grid search over object parameters, independent of the residuals."""
    rng = np.random.default_rng(11)
    b = _builder()
    ez = np.array([0, 0, 1.0])
    b.rect_plane([-50, -50, 0], [1, 0, 0], [0, 1, 0], 100, 100)  # ground
    e1 = np.array([1.0, 0.2, 0.3]); e1 /= np.linalg.norm(e1)
    e2 = np.array([-0.3, 1.0, 0.1]); e2 /= np.linalg.norm(e2)
    for e in (e1, e2):
        a1 = np.cross(e, ez); a1 /= np.linalg.norm(a1)
        b.line_edge(rng.uniform(-5, 5, 3) + [0, 0, 8], e, -100, 100, a1, np.cross(e, a1))
    tx = np.array([[-12.0, 3.0, 9.0]])
    rx = np.array([[14.0, -6.0, 4.0]])
    sc = b.build("fermat", 100.0, tx, rx)
    A, B = tx[0], rx[0]
    # single reflection on the ground
    sol, _ = solve_one(sc, [0])
    X = sol.X[0, :3]
    L = lambda g: (np.linalg.norm(np.c_[g, np.zeros(len(g))] - A, axis=1)
                   + np.linalg.norm(B - np.c_[g, np.zeros(len(g))], axis=1))
    best = _grid_min(L, [-30, -30], [30, 30], 201)
    assert np.linalg.norm(X[:2] - best) < 1e-6
    # two edges (DD)
    sol, _ = solve_one(sc, [1, 2])
    P1, d1 = sc.obj_param[1][0:3], sc.obj_param[1][3:6]
    P2, d2 = sc.obj_param[2][0:3], sc.obj_param[2][3:6]

    def L2(g):
        X1 = P1 + g[:, :1] * d1
        X2 = P2 + g[:, 1:2] * d2
        return (np.linalg.norm(X1 - A, axis=1) + np.linalg.norm(X2 - X1, axis=1)
                + np.linalg.norm(B - X2, axis=1))

    best = _grid_min(L2, [-60, -60], [60, 60], 241)
    assert sol.cost[0] < 1e-26
    assert np.linalg.norm(sol.X[0, 0:3] - (P1 + best[0] * d1)) < 1e-6
    assert np.linalg.norm(sol.X[0, 3:6] - (P2 + best[1] * d2)) < 1e-6
    # reflection on the ground, then an edge (RD)
    sol, _ = solve_one(sc, [0, 1])

    def L3(g):
        X1 = np.c_[g[:, :2], np.zeros(len(g))]
        X2 = P1 + g[:, 2:3] * d1
        return (np.linalg.norm(X1 - A, axis=1) + np.linalg.norm(X2 - X1, axis=1)
                + np.linalg.norm(B - X2, axis=1))

    best = _grid_min(L3, [-40, -40, -40], [40, 40, 40], 61, iters=10)
    assert sol.cost[0] < 1e-26
    assert np.linalg.norm(sol.X[0, 0:2] - best[:2]) < 1e-5
    assert np.linalg.norm(sol.X[0, 3:6] - (P1 + best[2] * d1)) < 1e-5


# ------------------------------------------- curved order-1 completeness --
def _paraboloid_stationary_points(R, t0, f, rho, A, B, n=40):
    """Every stationary point of L(s, t) = |X - A| + |B - X| over the disc of
    z = (s^2 + t^2) / (4 f) (Fermat: the reflection points are among them),
    by damped Newton on the gradient of L from a dense grid of starts; the
    Hessian by central differences of the gradient."""
    g = np.linspace(-rho, rho, n)
    U = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    U = U[(U ** 2).sum(1) <= (1.05 * rho) ** 2]

    def grad(U):
        s, t = U[:, 0], U[:, 1]
        X = np.stack([s, t, (s * s + t * t) / (4 * f)], 1) @ R.T + t0
        d, e = X - A, B - X
        w = d / np.linalg.norm(d, axis=1, keepdims=True) - e / np.linalg.norm(e, axis=1, keepdims=True)
        dx = np.stack([np.ones_like(s), np.zeros_like(s), s / (2 * f)], 1) @ R.T
        dy = np.stack([np.zeros_like(s), np.ones_like(s), t / (2 * f)], 1) @ R.T
        return np.stack([(w * dx).sum(1), (w * dy).sum(1)], 1)

    h = 1e-7
    for _ in range(60):
        G = grad(U)
        H = np.stack([(grad(U + [h, 0]) - grad(U - [h, 0])) / (2 * h),
                      (grad(U + [0, h]) - grad(U - [0, h])) / (2 * h)], 2)
        det = H[:, 0, 0] * H[:, 1, 1] - H[:, 0, 1] * H[:, 1, 0]
        ok = np.abs(det) > 1e-14
        step = np.zeros_like(U)
        step[ok, 0] = (H[ok, 1, 1] * G[ok, 0] - H[ok, 0, 1] * G[ok, 1]) / det[ok]
        step[ok, 1] = (-H[ok, 1, 0] * G[ok, 0] + H[ok, 0, 0] * G[ok, 1]) / det[ok]
        nrm = np.linalg.norm(step, axis=1, keepdims=True)
        U = np.clip(U - step * np.minimum(1.0, 0.5 * rho / np.maximum(nrm, 1e-300)), -3 * rho, 3 * rho)
    U = U[np.linalg.norm(grad(U), axis=1) < 1e-11]
    out = []
    for u in U:
        if not any(np.linalg.norm(u - q) < 1e-7 for q in out):
            out.append(u)
    return out


def _distinct(points, tol=1e-6):
    out = []
    for x in points:
        if not any(np.linalg.norm(x - q) < tol for q in out):
            out.append(np.array(x))
    return out


def _same_sets(a, b, tol=1e-6):
    missed = [x for x in a if not any(np.linalg.norm(x - q) < tol for q in b)]
    extra = [x for x in b if not any(np.linalg.norm(x - q) < tol for q in a)]
    return missed, extra


def test_paraboloid_order1_root_set_matches_dense_scan():
    """Order-1 completeness on a paraboloid (Sec. III-B, multi-start guesses
    of Algorithm 1): in deep bowls with both ends inside, where a sequence
    has up to three reflection points, the valid solutions over 64 starts are
    exactly the mirror-law stationary points of the path length found by a
    dense Newton scan of the disc; with the 8 starts of the workloads they
    are a subset (no false roots).  Points within 1 mm of the rim are left
    out on both sides (the bounds band)."""
    rng = np.random.default_rng(1)
    rho, n_multi = 2.0, 0
    totals = {8: 0, 64: 0}
    n_roots = 0
    for _ in range(40):
        R = S._random_rotation(rng)
        t0 = rng.uniform(-3, 3, 3)
        f = rng.uniform(0.5, 1.2)
        A = t0 + R @ np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 2.0)])
        B = t0 + R @ np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 2.0)])
        P = lambda u: t0 + R @ np.array([u[0], u[1], (u[0] ** 2 + u[1] ** 2) / (4 * f)])
        roots = []
        for u in _paraboloid_stationary_points(R, t0, f, rho, A, B):
            if math.hypot(*u) > rho - 1e-3:
                continue
            x = P(u)
            i = (x - A) / np.linalg.norm(x - A)
            r = (B - x) / np.linalg.norm(B - x)
            nm = R @ np.array([u[0] / (2 * f), u[1] / (2 * f), -1.0])
            nm /= np.linalg.norm(nm)
            if np.linalg.norm(r - (i - 2 * np.dot(i, nm) * nm)) < 1e-8:  # a reflection, not a crossing
                roots.append(x)
        n_roots += len(roots)
        n_multi += len(roots) > 1
        b = _builder()
        b.paraboloid(R, t0, f, rho, occluder=False)
        sc = b.build("bowl", 100.0, A[None], B[None], pair_mode=1)
        for starts in (8, 64):
            table = oracle.enumerate_sequences(sc, 1, S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=starts))
            sol, ver = oracle.candidate_range(sc, table, 0, len(table))
            found = []
            for c in range(len(table)):
                loc = R.T @ (sol.X[c, :3] - t0)
                if ver.valid[c] and math.hypot(loc[0], loc[1]) < rho - 1e-3:
                    found.append(sol.X[c, :3])
            missed, extra = _same_sets(roots, _distinct(found))
            assert not extra, "a valid solution that is not a reflection point"
            if starts == 64:
                assert not missed
            totals[starts] += len(roots) - len(missed)
    assert n_multi >= 3 and n_roots >= 30
    print(f"paraboloid order 1: {n_roots} roots; found with 8 starts {totals[8]}, with 64 starts {totals[64]}")


def test_arc_diffraction_order1_root_set_matches_1d_scan():
    """Order-1 completeness on an arc edge (Eq. 9 on Eq. 4's curve): the
    diffraction points are the zeros of dL/dphi along the arc; a 4000-sample
    sign scan with bisection finds them all, and the valid solutions over the
    8 starts of the workloads are exactly that set.  Points within 1 mm (arc
    length) of an end are left out on both sides."""
    from scipy.optimize import brentq

    rng = np.random.default_rng(2)
    n_roots = n_multi = 0
    for _ in range(60):
        R = S._random_rotation(rng)
        C = rng.uniform(-2, 2, 3)
        Rc = rng.uniform(1, 4)
        a, u = R[:, 2], R[:, 0]
        v = np.cross(a, u)
        phi0 = rng.uniform(-math.pi, math.pi)
        phi1 = phi0 + rng.uniform(math.pi / 4, math.pi)
        A = C + rng.uniform(-6, 6, 3)
        B = C + rng.uniform(-6, 6, 3)
        X = lambda p: C + Rc * (math.cos(p) * u + math.sin(p) * v)

        def dL(p):
            x = X(p)
            w = (x - A) / np.linalg.norm(x - A) - (B - x) / np.linalg.norm(B - x)
            return float(np.dot(w, Rc * (-math.sin(p) * u + math.cos(p) * v)))

        ph = np.linspace(phi0, phi1, 4001)
        d = np.array([dL(p) for p in ph])
        band = 1e-3 / Rc
        roots = [X(p) for p in (brentq(dL, ph[k], ph[k + 1], xtol=1e-15) for k in range(len(ph) - 1)
                                if d[k] * d[k + 1] < 0) if phi0 + band < p < phi1 - band]
        n_roots += len(roots)
        n_multi += len(roots) > 1
        b = _builder()
        b.arc_edge(C, a, Rc, u, phi0, phi1)
        sc = b.build("arc", 100.0, A[None], B[None], pair_mode=1)
        table = oracle.enumerate_sequences(sc, 1, S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=8))
        sol, ver = oracle.candidate_range(sc, table, 0, len(table))
        found = []
        for c in range(len(table)):
            ang = phi0 + math.fmod(sol.T[c, 0] - phi0, 2 * math.pi)
            ang += 2 * math.pi if ang < phi0 else 0.0
            if ver.valid[c] and phi0 + band < ang < phi1 - band:
                found.append(sol.X[c, :3])
        missed, extra = _same_sets(roots, _distinct(found))
        assert not missed and not extra
    assert n_multi >= 3 and n_roots >= 40


# ---------------------------------------------------- invariances ---------
def test_solution_invariant_to_normal_and_edge_direction_signs():
    sc = S.urban_block(4)
    flipped = S.urban_block(4)
    op = flipped.obj_param
    for i, k in enumerate(flipped.obj_kind):
        if k == S.PLANE:
            op[i, 0:4] *= -1.0
        elif k == S.LINE_EDGE:
            op[i, 3:6] *= -1.0
    table = oracle.enumerate_sequences(sc, 2, FULL2)
    sel = np.arange(0, len(table), 37)
    sub = oracle.SequenceTable(table.order[sel], table.ids[sel], table.start[sel])
    a = oracle.solve(sc, sub)
    b = oracle.solve(flipped, sub)
    ok = (a.cost < oracle.TAU)
    assert ok.sum() > 20
    assert np.array_equal(ok, b.cost < oracle.TAU)
    # interaction points agree (the parametrisations differ only by the sign
    # of the edge parameter, which the initial projection follows)
    assert np.abs(a.X[ok] - b.X[ok]).max() < 1e-8


# ------------------------------------------------------ visibility --------
def _sampled_blocked_rect(A, B, O, u, v, U, V, n, samples=4001):
    t = np.linspace(0, 1, samples)
    P = A[None] + t[:, None] * (B - A)[None]
    s = (P - O) @ n
    for i in range(samples - 1):
        if s[i] * s[i + 1] < 0 and abs(s[0]) > 1e-6 and abs(s[-1]) > 1e-6:
            # refine by bisection on the sampled bracket
            lo, hi = t[i], t[i + 1]
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                sm = np.dot(A + mid * (B - A) - O, n)
                if np.sign(sm) == np.sign(s[i]):
                    lo = mid
                else:
                    hi = mid
            X = A + lo * (B - A)
            uu, vv = np.dot(X - O, u), np.dot(X - O, v)
            if 0 <= uu <= U and 0 <= vv <= V:
                return True
    return False


def _sampled_blocked_parab(A, B, R, tt, f, rho, samples=20001):
    L = np.linalg.norm(B - A)
    t = np.linspace(0, 1, samples)
    P = A[None] + t[:, None] * (B - A)[None]
    loc = (P - tt) @ R  # rows: R^T (P - t)
    g = (loc[:, 0] ** 2 + loc[:, 1] ** 2) / (4 * f) - loc[:, 2]
    for i in range(samples - 1):
        if g[i] * g[i + 1] < 0:
            tc = t[i] - g[i] * (t[i + 1] - t[i]) / (g[i + 1] - g[i])
            xc = loc[i] + (loc[i + 1] - loc[i]) * (tc - t[i]) / (t[i + 1] - t[i])
            if tc * L > 1e-6 and (1 - tc) * L > 1e-6 and xc[0] ** 2 + xc[1] ** 2 <= rho * rho:
                return True
    return False


def test_visibility_matches_dense_sampling():
    rng = np.random.default_rng(5)
    b = _builder()
    R = S._random_rotation(rng)
    b.rect_plane([-3, -3, 0], [1, 0, 0], [0, 1, 0], 6, 6)
    b.paraboloid(R, [0.5, -0.5, 4.0], 0.8, 2.0)
    sc = b.build("vis", 10.0, np.zeros((1, 3)), np.zeros((1, 3)))
    rect = sc.occ_param[0]
    par = sc.occ_param[1]
    n_blk = 0
    for _ in range(400):
        A = rng.uniform(-6, 6, 3) + [0, 0, 2]
        B = rng.uniform(-6, 6, 3) + [0, 0, 2]
        got, amb = oracle.segment_blocked(sc, A, B)
        if amb:
            continue
        want = (_sampled_blocked_rect(A, B, rect[0:3], rect[3:6], rect[6:9], rect[9], rect[10], rect[11:14])
                or _sampled_blocked_parab(A, B, par[0:9].reshape(3, 3), par[9:12], par[12], par[13]))
        assert got == want, (A, B)
        n_blk += got
    assert n_blk > 40
    # endpoints on the surface never block; a segment lying in the plane never blocks
    assert not oracle.segment_blocked(sc, np.array([0.0, 0.0, 0.0]), np.array([1.0, 2.0, 5.0]))[0]
    assert not oracle.segment_blocked(sc, np.array([-2.0, 0.0, 0.0]), np.array([2.0, 1.0, 0.0]))[0]
    assert oracle.segment_blocked(sc, np.array([0.0, 0.0, -1.0]), np.array([0.0, 0.0, 1.0]))[0]


def test_bounds_rules():
    sc = S.street_canyon()
    # ground: rectangle origin (-50,-10,0), u along x (100 m), v along y (20 m)
    assert oracle.params_in_bounds(sc, 0, [50.0, 10.0])[0]
    assert not oracle.params_in_bounds(sc, 0, [110.0, 10.0])[0]
    # wall y=-10: u along z (20 m), v along x (100 m)
    assert oracle.params_in_bounds(sc, 1, [19.0, 60.0])[0]
    assert not oracle.params_in_bounds(sc, 1, [21.0, 60.0])[0]
    ok, amb = oracle.params_in_bounds(sc, 1, [5.0, 100.0])
    assert ok and amb


# ------------------------------------------------------ enumeration -------
def test_full_enumeration_counts_and_order():
    sc = S.urban_block(2)
    t = oracle.enumerate_sequences(sc, 2, FULL2)
    assert len(t) == 97 + 97 * 96 == 9409
    seqs = [tuple(r[:n]) for r, n in zip(t.ids, t.order)]
    assert len(set(seqs)) == len(seqs)
    assert all(len(set(s)) == len(s) for s in seqs)
    assert seqs[:97] == [(i,) for i in range(97)]
    assert seqs[97:] == sorted(seqs[97:])
    t3 = oracle.enumerate_sequences(S.street_canyon(), 3, S.SequenceSpec(quota=(-1, -1, -1, 0)))
    assert len(t3) == 3 + 6 + 6


def test_sampled_enumeration_is_deterministic_and_forces_edges():
    sc = S.mixed_order_city()
    spec = S.CONFIG_SPECS["mixed_order"]
    a = oracle.enumerate_sequences(sc, 4, spec)
    b = oracle.enumerate_sequences(sc, 4, spec)
    assert len(a) == 49 + 400 + 800 + 799
    assert np.array_equal(a.ids, b.ids)
    is_edge = np.isin(sc.obj_kind, [S.LINE_EDGE, S.ARC_EDGE])
    for i in range(len(a)):
        n = a.order[i]
        ids = a.ids[i][:n]
        assert len(set(ids.tolist())) == n
    # slot 0 of order 3 is forced: two consecutive edges
    first3 = int(np.nonzero(a.order == 3)[0][0])
    ids = a.ids[first3][:3]
    assert any(is_edge[ids[k]] and is_edge[ids[k + 1]] for k in range(2))


def test_adjacency_matrix_of_fig5_counts_like_networkx():
    """Fig. 5 gives G for the Fig. 3 scene; the candidates with the mask are
    the BS -> UE simple paths of NetworkX's all_simple_paths (Algorithm 1).
    Row s1 is printed with one stray empty cell; it is read without it."""
    nx = pytest.importorskip("networkx")
    names = ["BS", "s1", "s2", "s3", "s4", "s5", "s6", "e1", "e2", "e3", "e4", "e5", "e6", "UE"]
    rows = {
        "BS": ["s1", "s6", "e1", "e2", "e4", "e6", "UE"],
        "s1": ["s6", "e4"],
        "s2": ["s6", "e4", "e6", "UE"],
        "s6": ["s1", "s2", "e1", "e2", "e3", "UE"],
        "e1": ["s6", "e4"],
        "e2": ["s6", "e4", "e6", "UE"],
        "e3": ["s6", "e4", "e6", "UE"],
        "e4": ["s1", "s2", "e1", "e2", "e3", "UE"],
        "e6": ["s2", "e2", "e3", "UE"],
    }
    G = nx.DiGraph()
    G.add_nodes_from(names)
    for a, bs in rows.items():
        for b in bs:
            G.add_edge(a, b)
    objs = names[1:-1]
    kinds = np.array([S.PLANE] * 6 + [S.LINE_EDGE] * 6, np.int32)
    adj = np.zeros((12, 12), np.uint8)
    for i, a in enumerate(objs):
        for j, b in enumerate(objs):
            adj[i, j] = G.has_edge(a, b)
    sc = S.Scene("fig3", 1.0, kinds, np.zeros((12, 24)), np.zeros(0, np.int32), np.zeros((0, 24)),
                 np.zeros((1, 3)), np.zeros((1, 3)))
    for nt in (1, 2, 3, 4):
        t = oracle.enumerate_sequences(sc, nt, S.SequenceSpec(quota=(-1, -1, -1, -1)), adj=adj)
        mine = set()
        for r, n in zip(t.ids, t.order):
            seq = [objs[i] for i in r[:n]]
            if G.has_edge("BS", seq[0]) and G.has_edge(seq[-1], "UE"):
                mine.add(tuple(seq))
        ref = {tuple(p[1:-1]) for p in nx.all_simple_paths(G, "BS", "UE", cutoff=nt + 1) if len(p) > 2}
        assert mine == ref


def test_splitmix64_published_outputs():
    """First outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014):
    the generator adds 0x9E3779B97F4A7C15 before mixing, so output k of the
    stream is mix(k * gamma); oracle_splitmix64(x) = mix(x + gamma)."""
    gamma = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(gamma) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * gamma) & (2**64 - 1)) == 0x06C45D188009454F


# ------------------------------------------------------- gradients --------
def _canyon_valid_paths(limit=6):
    sc = S.street_canyon()
    table = oracle.enumerate_sequences(sc, 2, FULL2)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    out = []
    for c in np.nonzero(ver.valid)[0]:
        e, p = divmod(int(c), sc.n_pairs)
        out.append((table.ids[e][:table.order[e]].tolist(), p, sol.X[c, :3 * table.order[e]].copy(),
                    sol.T[c].copy()))
    rng = np.random.default_rng(0)
    pick = rng.choice(len(out), limit, replace=False)
    return sc, [out[i] for i in pick]


def test_gradient_matches_envelope_closed_forms():
    """At a stationary path dL/dTX = -i_hat_1, dL/dRX = r_hat_n and, for a
    reflection on <n, X> = d, dL/dd = 2 <i_hat_k, n> (reflection law)."""
    sc, paths = _canyon_valid_paths(8)
    for ids, p, x, T in paths:
        a, b = sc.pair_points(p)
        dL, _ = oracle.path_grad(sc, ids, a, b, T)
        n = len(ids)
        P = [a] + [x[3 * k:3 * k + 3] for k in range(n)] + [b]
        unit = lambda v: v / np.linalg.norm(v)
        assert np.allclose(dL[0:3], -unit(P[1] - P[0]), atol=1e-9)
        assert np.allclose(dL[3:6], unit(P[n + 1] - P[n]), atol=1e-9)
        for k, o in enumerate(ids):
            nrm = sc.obj_param[o][0:3]
            assert abs(dL[6 + k] - 2 * np.dot(unit(P[k + 1] - P[k]), nrm)) < 1e-9


def test_gradient_matches_central_differences_of_resolve():
    sc, paths = _canyon_valid_paths(4)
    h = 1e-4
    for ids, p, x, T in paths:
        a, b = sc.pair_points(p)
        dL, dX = oracle.path_grad(sc, ids, a, b, T)

        def length_with(mod):
            s2 = S.street_canyon()
            mod(s2)
            sol, ver = solve_one(s2, ids)
            return ver.length[p], sol.X[p, :3 * len(ids)]

        for j in range(3):
            def tx_shift(s2, d, j=j):
                s2.tx[0, j] += d
            Lp, Xp = length_with(lambda s2: tx_shift(s2, h))
            Lm, Xm = length_with(lambda s2: tx_shift(s2, -h))
            assert abs((Lp - Lm) / (2 * h) - dL[j]) < 1e-6
            assert np.abs((Xp - Xm) / (2 * h) - dX[:, j]).max() < 1e-5
        for k, o in enumerate(ids):
            def d_shift(s2, d, o=o):
                # move the plane <n, X> = d along n: offset and rectangle origin
                s2.obj_param[o, 3] += d
                s2.obj_param[o, 4:7] += d * s2.obj_param[o, 0:3]
            Lp, _ = length_with(lambda s2: d_shift(s2, h))
            Lm, _ = length_with(lambda s2: d_shift(s2, -h))
            assert abs((Lp - Lm) / (2 * h) - dL[6 + k]) < 1e-6


# ------------------------------------------------------ degeneracy --------
def test_collapsed_segments_are_not_paths():
    """A reflection on a wall followed by diffraction on that wall's own edge
    has no genuine solution (it would need grazing incidence); the minimiser
    drifts to a collapsed segment that the minimum-length rule rejects."""
    sc = S.urban_block(8)
    # object 0 is the first wall of box 0; object 49 its first corner edge
    assert sc.obj_kind[0] == S.PLANE and sc.obj_kind[49] == S.LINE_EDGE
    sol, ver = solve_one(sc, [0, 49])
    assert ver.valid.sum() == 0


def test_batched_gradient_sums_equal_per_path_gradients():
    """oracle.grad_sums (threads over paths) adds up exactly what
    oracle.path_grad gives path by path, with length and point weights."""
    sc = S.urban_block(2)
    table = oracle.enumerate_sequences(sc, 2, FULL2)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    v = np.nonzero(ver.valid)[0]
    assert len(v) > 50
    rng = np.random.default_rng(0)
    gl = rng.uniform(0.5, 1.5, len(v))
    gp = rng.normal(size=(len(v), 12))
    gtx, grx, gobj = oracle.grad_sums(sc, table, v, sol.T[v], gl, gp)
    wtx, wrx, wobj = np.zeros_like(sc.tx), np.zeros_like(sc.rx), np.zeros(sc.n_obj)
    for j, c in enumerate(v):
        e, p = divmod(int(c), sc.n_pairs)
        ids = table.ids[e][:table.order[e]]
        dL, dX = oracle.path_grad(sc, ids, *sc.pair_points(p), sol.T[c])
        w = gl[j] * dL + gp[j, :3 * len(ids)] @ dX
        wtx[p // sc.rx.shape[0]] += w[:3]
        wrx[p % sc.rx.shape[0]] += w[3:6]
        for kk, o in enumerate(ids):
            wobj[o] += w[6 + kk]
    assert np.abs(gtx - wtx).max() < 1e-9 and np.abs(grx - wrx).max() < 1e-9 and np.abs(gobj - wobj).max() < 1e-9
