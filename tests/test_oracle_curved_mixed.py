"""Completeness of the oracle's root sets for the remaining curved pairings:
a curved object with a plane or a straight edge, two arc edges, and order 3.

Sec. III-B: every distinct root the multi-start minimiser finds is a path.
As in the order-2 paraboloid pins, the independent route is Fermat's
principle: a path is a stationary point of the length
L = sum_k |X_{k+1} - X_k| over the interaction parameters (two per plane or
paraboloid, the position along a straight edge, the angle of an arc), and among the stationary points the paths
are those that obey the reflection law (Eq. 8) at every surface and the
Keller cone (Eq. 9) at every edge, inside the bounds.  A damped Newton
iteration on the gradient of L (Hessian by forward differences) from the
product of dense start grids on every object finds the stationary points.
No occluders, so the oracle's valid set is the laws, the bounds and the
minimum segment.  Points within 1 mm of a bound and paths with a segment
within a factor 3 of the minimum length are left out on both sides.

Bar: every valid oracle solution is in the reference set (no false root),
and with 256 starts (order 2) or 1024 starts (order 3) the two sets are
equal; the counts found with 8 and 64 starts are reported.
"""
import math

import numpy as np

import oracle
from paper_2301_06399_gb300 import scenes as S

BAND = 1e-3  # metres from a bound
LMIN = 1e-5 * 100.0  # the oracle's minimum segment at scene scale 100


# -- objects: parameters -> point and tangents --------------------------------

def _bowl(R, t0, f, rho=2.0):
    return dict(kind="parab", R=R, t0=t0, f=f, rho=rho, dim=2)


def _plane(O, u, v, U, V):
    return dict(kind="plane", O=O, u=u, v=v, U=U, V=V, n=np.cross(u, v), dim=2)


def _arc(C, a, u, Rc, phi0, phi1):
    return dict(kind="arc", C=C, a=a, u=u, v=np.cross(a, u), Rc=Rc, phi0=phi0, phi1=phi1, dim=1)


def _line(P, e, s0, s1):
    return dict(kind="line", P=P, e=e, s0=s0, s1=s1, dim=1)


def _point(o, P):
    """Points (n, 3) and tangent lists [(n, 3)] * dim for parameters P (n, dim)."""
    if o["kind"] == "parab":
        s, t = P[:, 0], P[:, 1]
        X = np.stack([s, t, (s * s + t * t) / (4 * o["f"])], 1) @ o["R"].T + o["t0"]
        T0 = np.stack([np.ones_like(s), np.zeros_like(s), s / (2 * o["f"])], 1) @ o["R"].T
        T1 = np.stack([np.zeros_like(s), np.ones_like(s), t / (2 * o["f"])], 1) @ o["R"].T
        return X, [T0, T1]
    if o["kind"] == "plane":
        X = o["O"] + P[:, 0:1] * o["u"] + P[:, 1:2] * o["v"]
        return X, [np.broadcast_to(o["u"], X.shape), np.broadcast_to(o["v"], X.shape)]
    if o["kind"] == "line":
        X = o["P"] + P[:, 0:1] * o["e"]
        return X, [np.broadcast_to(o["e"], X.shape)]
    c, s = np.cos(P[:, 0])[:, None], np.sin(P[:, 0])[:, None]
    X = o["C"] + o["Rc"] * (c * o["u"] + s * o["v"])
    return X, [o["Rc"] * (-s * o["u"] + c * o["v"])]


def _start_grid(o, n):
    if o["kind"] == "parab":
        g = np.linspace(-o["rho"], o["rho"], n)
        D = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
        return D[(D ** 2).sum(1) <= o["rho"] ** 2]
    if o["kind"] == "plane":
        D = np.stack(np.meshgrid(np.linspace(0, o["U"], n), np.linspace(0, o["V"], n), indexing="ij"), -1)
        return D.reshape(-1, 2)
    if o["kind"] == "line":
        return np.linspace(o["s0"], o["s1"], 3 * n)[:, None]
    return np.linspace(o["phi0"], o["phi1"], 3 * n)[:, None]


def _params_of(o, X):
    """Parameters of a point on the object (inverse of _point)."""
    if o["kind"] == "parab":
        loc = o["R"].T @ (X - o["t0"])
        return loc[:2]
    if o["kind"] == "plane":
        return np.array([np.dot(X - o["O"], o["u"]), np.dot(X - o["O"], o["v"])])
    if o["kind"] == "line":
        return np.array([np.dot(X - o["P"], o["e"])])
    loc = X - o["C"]
    return np.array([math.atan2(np.dot(loc, o["v"]), np.dot(loc, o["u"]))])


def _inside(o, p):
    """Inside the bounds by more than BAND."""
    if o["kind"] == "parab":
        return math.hypot(p[0], p[1]) < o["rho"] - BAND
    if o["kind"] == "plane":
        return BAND < p[0] < o["U"] - BAND and BAND < p[1] < o["V"] - BAND
    if o["kind"] == "line":
        return o["s0"] + BAND < p[0] < o["s1"] - BAND
    d = (p[0] - o["phi0"]) % (2.0 * math.pi)
    return BAND / o["Rc"] < d < (o["phi1"] - o["phi0"]) - BAND / o["Rc"]


def _normal(o, X):
    if o["kind"] == "plane":
        return o["n"] / np.linalg.norm(o["n"])
    loc = o["R"].T @ (X - o["t0"])
    n = o["R"] @ np.array([loc[0] / (2 * o["f"]), loc[1] / (2 * o["f"]), -1.0])
    return n / np.linalg.norm(n)


# -- the reference: stationary points of L obeying the laws -------------------

def _grad(objs, A, B, P):
    pts, tans, off = [A[None].repeat(len(P), 0)], [], 0
    for o in objs:
        X, T = _point(o, P[:, off:off + o["dim"]])
        pts.append(X)
        tans.append(T)
        off += o["dim"]
    pts.append(B[None].repeat(len(P), 0))
    u = [(pts[k + 1] - pts[k]) / np.linalg.norm(pts[k + 1] - pts[k], axis=1, keepdims=True)
         for k in range(len(pts) - 1)]
    cols = []
    for k, T in enumerate(tans):
        w = u[k] - u[k + 1]
        cols += [(w * t).sum(1) for t in T]
    return np.stack(cols, 1)


def _obeys_laws(objs, pts, tol=1e-8):
    for k, o in enumerate(objs, start=1):
        i = (pts[k] - pts[k - 1]) / np.linalg.norm(pts[k] - pts[k - 1])
        r = (pts[k + 1] - pts[k]) / np.linalg.norm(pts[k + 1] - pts[k])
        if o["kind"] in ("arc", "line"):
            _, (T,) = _point(o, _params_of(o, pts[k])[None])
            e = T[0] / np.linalg.norm(T[0])
            if abs(np.dot(i, e) - np.dot(r, e)) > tol:
                return False
        else:
            n = _normal(o, pts[k])
            if np.linalg.norm(r - (i - 2 * np.dot(i, n) * n)) > tol:
                return False
    return True


def _kept(objs, A, B, pts):
    """Inside every bound by more than BAND and every segment clear of the
    minimum-length band."""
    full = [A, *pts, B]
    if any(np.linalg.norm(full[k + 1] - full[k]) < 3.0 * LMIN for k in range(len(full) - 1)):
        return False
    return all(_inside(o, _params_of(o, X)) for o, X in zip(objs, pts))


def _reference_roots(objs, A, B, n_grid):
    grids = [_start_grid(o, n_grid) for o in objs]
    idx = np.stack(np.meshgrid(*[np.arange(len(g)) for g in grids], indexing="ij"), -1).reshape(-1, len(grids))
    P = np.concatenate([g[idx[:, j]] for j, g in enumerate(grids)], 1)
    D = P.shape[1]
    lim = np.concatenate([[o["phi1"] + 10.0] if o["kind"] == "arc" else [20.0] * o["dim"] for o in objs])
    h = 1e-7
    for _ in range(80):
        G = _grad(objs, A, B, P)
        live = np.linalg.norm(G, axis=1) > 1e-13
        if not live.any():
            break
        Q, Gl = P[live], G[live]
        H = np.stack([(_grad(objs, A, B, Q + h * e) - Gl) / h for e in np.eye(D)], 2)
        HtH = np.einsum("nki,nkj->nij", H, H) + 1e-14 * np.eye(D)
        step = np.linalg.solve(HtH, np.einsum("nki,nk->ni", H, Gl)[..., None])[..., 0]
        nrm = np.linalg.norm(step, axis=1, keepdims=True)
        P[live] = np.clip(Q - step * np.minimum(1.0, 0.5 / np.maximum(nrm, 1e-300)), -lim, lim)
    P = P[np.linalg.norm(_grad(objs, A, B, P), axis=1) < 1e-10]
    P = P[np.unique(np.round(P, 7), axis=0, return_index=True)[1]]  # starts that reached one point
    roots = []
    for p in P:
        pts, off = [], 0
        for o in objs:
            pts.append(_point(o, p[None, off:off + o["dim"]])[0][0])
            off += o["dim"]
        if not _kept(objs, A, B, pts) or not _obeys_laws(objs, [A, *pts, B]):
            continue
        x = np.concatenate(pts)
        if not any(np.linalg.norm(x - q) < 1e-6 for q in roots):
            roots.append(x)
    return roots


def _oracle_roots(sc, objs, order, starts, A, B):
    """The oracle's distinct valid roots per sequence, with the same exclusions
    as the reference."""
    q = [0, 0, 0, 0]
    q[order - 1] = -1
    spec = S.SequenceSpec(quota=tuple(q), starts_curved=starts)
    table = oracle.enumerate_sequences(sc, order, spec)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table))
    sets = {}
    for c in range(len(table)):
        ids = tuple(int(i) for i in table.ids[c][:order])
        if not ver.valid[c]:
            continue
        pts = [sol.X[c, 3 * k:3 * k + 3] for k in range(order)]
        if not _kept([objs[i] for i in ids], A, B, pts):
            continue
        x = np.concatenate(pts)
        found = sets.setdefault(ids, [])
        if not any(np.linalg.norm(x - q) < 1e-6 for q in found):
            found.append(x)
    return sets


def _same(a, b, tol=1e-6):
    missed = [x for x in a if not any(np.linalg.norm(x - q) < tol for q in b)]
    extra = [x for x in b if not any(np.linalg.norm(x - q) < tol for q in a)]
    return missed, extra


def _build(objs, A, B):
    b = S._Builder()
    for o in objs:
        if o["kind"] == "parab":
            b.paraboloid(o["R"], o["t0"], o["f"], o["rho"], occluder=False)
        elif o["kind"] == "plane":
            b.rect_plane(o["O"], o["u"], o["v"], o["U"], o["V"], occluder=False)
        elif o["kind"] == "line":
            # wedge faces (any two unit vectors normal to the edge) do not
            # enter the oracle's acceptance
            w = np.eye(3)[np.argmin(np.abs(o["e"]))]
            f1 = np.cross(o["e"], w) / np.linalg.norm(np.cross(o["e"], w))
            b.line_edge(o["P"], o["e"], o["s0"], o["s1"], f1, np.cross(o["e"], f1))
        else:
            b.arc_edge(o["C"], o["a"], o["Rc"], o["u"], o["phi0"], o["phi1"])
    return b.build("pin", 100.0, A[None], B[None], pair_mode=1)


def _run(family, n_inst, order, seqs, n_grid, start_levels, seed):
    """Compares the oracle's valid root sets with the reference over n_inst
    seeded instances of `family`; returns (roots, multi-root sequences,
    {starts: found})."""
    rng = np.random.default_rng(seed)
    totals = {s: 0 for s in start_levels}
    n_roots = n_multi = 0
    for _ in range(n_inst):
        objs, A, B = family(rng)
        sc = _build(objs, A, B)
        refs = {seq: _reference_roots([objs[i] for i in seq], A, B, n_grid) for seq in seqs}
        for ref in refs.values():
            n_roots += len(ref)
            n_multi += len(ref) > 1
        for starts in start_levels:
            sets = _oracle_roots(sc, objs, order, starts, A, B)
            for seq, ref in refs.items():
                missed, extra = _same(ref, sets.get(seq, []))
                assert not extra, ("an oracle root that is not a path", family.__name__, seq, starts, extra)
                if starts == start_levels[-1]:
                    assert not missed, (len(missed), "roots missed", family.__name__, seq, starts, missed)
                totals[starts] += len(ref) - len(missed)
    print(f"{family.__name__}, order {order}: {n_roots} roots ({n_multi} sequences with several); found "
          + ", ".join(f"{totals[s]} with {s} starts" for s in start_levels))
    return n_roots, n_multi, totals


# -- instance families ----------------------------------------------------------

def _frame(rng):
    return S._random_rotation(rng), rng.uniform(-3, 3, 3)


def _endpoints(rng, R, t0, z_lo, z_hi, r=1.0):
    return [t0 + R @ np.array([*rng.uniform(-r, r, 2), rng.uniform(z_lo, z_hi)]) for _ in range(2)]


def flat_lid_over_bowl(rng):
    """A deep bowl and a flat rectangle above it (5 m square, facing it)."""
    R, t0 = _frame(rng)
    h = rng.uniform(1.6, 2.6)
    bowl = _bowl(R, t0, rng.uniform(0.5, 1.2))
    lid = _plane(t0 + R @ np.array([-2.5, -2.5, h]), R[:, 0], R[:, 1], 5.0, 5.0)
    A, B = _endpoints(rng, R, t0, 0.4, h - 0.4)
    return [lid, bowl], A, B


def arc_over_ground(rng):
    """A circular arc edge (radius 1-1.8 m, 90-180 degrees) 1-2 m above a
    6 m square floor, TX and RX above the floor."""
    R, t0 = _frame(rng)
    floor = _plane(t0 + R @ np.array([-3.0, -3.0, 0.0]), R[:, 0], R[:, 1], 6.0, 6.0)
    phi0 = rng.uniform(-math.pi, math.pi)
    arc = _arc(t0 + R @ np.array([0.0, 0.0, rng.uniform(1.0, 2.0)]), R[:, 2], R[:, 0], rng.uniform(1.0, 1.8),
               phi0, phi0 + rng.uniform(math.pi / 2, math.pi))
    A, B = _endpoints(rng, R, t0, 0.3, 2.5, r=1.5)
    return [floor, arc], A, B


def two_arcs(rng):
    """Two arc edges around one axis at different heights and radii, each
    spanning 120-270 degrees; TX and RX near the axis."""
    R, t0 = _frame(rng)
    arcs = []
    for z in (0.0, rng.uniform(0.8, 1.6)):
        phi0 = rng.uniform(-math.pi, math.pi)
        arcs.append(_arc(t0 + R @ np.array([0.0, 0.0, z]), R[:, 2], R[:, 0], rng.uniform(1.0, 2.0),
                         phi0, phi0 + rng.uniform(2 * math.pi / 3, 1.5 * math.pi)))
    A, B = _endpoints(rng, R, t0, -1.0, 2.5, r=0.8)
    return arcs, A, B


def edge_over_bowl(rng):
    """A straight edge (6 m long) 1-2 m above a deep bowl's vertex, crossing
    its axis within 1 m; TX and RX above the bowl."""
    R, t0 = _frame(rng)
    bowl = _bowl(R, t0, rng.uniform(0.5, 1.2))
    a = rng.uniform(0, 2 * math.pi)
    e = R @ np.array([math.cos(a), math.sin(a), 0.0])
    P = t0 + R @ np.array([*rng.uniform(-1.0, 1.0, 2), rng.uniform(1.0, 2.0)])
    A, B = _endpoints(rng, R, t0, 0.4, 2.5)
    return [bowl, _line(P, e, -3.0, 3.0)], A, B


def bowl_rim_and_lid(rng):
    """Three objects for order 3 (a sequence never repeats an object): a deep
    bowl, an arc rim (radius 1-1.8 m, 120-270 degrees) 0.3-0.8 m above the
    bowl's surface at that radius and a flat 5 m square lid 0.8-1.4 m above
    the rim; TX and RX between bowl and lid.  The clearance keeps the rim off
    the bowl: a root whose rim and bowl points lie a few centimetres apart has
    a basin that random starts, even 1024 of them, rarely hit."""
    R, t0 = _frame(rng)
    f = rng.uniform(0.5, 1.2)
    bowl = _bowl(R, t0, f)
    Rc = rng.uniform(1.0, 1.8)
    z_rim = Rc * Rc / (4 * f) + rng.uniform(0.3, 0.8)
    h = z_rim + rng.uniform(0.8, 1.4)
    lid = _plane(t0 + R @ np.array([-2.5, -2.5, h]), R[:, 0], R[:, 1], 5.0, 5.0)
    phi0 = rng.uniform(-math.pi, math.pi)
    rim = _arc(t0 + R @ np.array([0.0, 0.0, z_rim]), R[:, 2], R[:, 0], Rc,
               phi0, phi0 + rng.uniform(2 * math.pi / 3, 1.5 * math.pi))
    A, B = _endpoints(rng, R, t0, 0.4, h - 0.4)
    return [bowl, rim, lid], A, B


def bowl_edge_and_lid(rng):
    """Order 3 with a straight edge: a deep bowl, a 6 m straight edge 0.3-0.8 m
    above the bowl's surface where it crosses the axis (within 0.8 m of it)
    and a flat 5 m square lid 0.8-1.4 m above the edge."""
    R, t0 = _frame(rng)
    f = rng.uniform(0.5, 1.2)
    bowl = _bowl(R, t0, f)
    a = rng.uniform(0, 2 * math.pi)
    e = R @ np.array([math.cos(a), math.sin(a), 0.0])
    off = rng.uniform(-0.8, 0.8, 2)
    z_edge = float(off @ off) / (4 * f) + rng.uniform(0.3, 0.8)
    h = z_edge + rng.uniform(0.8, 1.4)
    lid = _plane(t0 + R @ np.array([-2.5, -2.5, h]), R[:, 0], R[:, 1], 5.0, 5.0)
    edge = _line(t0 + R @ np.array([off[0], off[1], z_edge]), e, -3.0, 3.0)
    A, B = _endpoints(rng, R, t0, 0.4, h - 0.4)
    return [bowl, edge, lid], A, B


def three_mirrors(rng):
    """Order 3 on three paraboloids: a deep bowl, an inverted paraboloid
    1.8-2.6 m above it, and a shallow side mirror (focal length 3-5 m, disc
    radius 1.5 m) 3 m from their axis at mid height, its axis pointing at
    theirs; TX and RX between bowl and lid."""
    R, t0 = _frame(rng)
    h = rng.uniform(1.8, 2.6)
    flip = np.diag([1.0, -1.0, -1.0])
    bowl = _bowl(R, t0, rng.uniform(0.5, 1.2))
    lid = _bowl(R @ flip, t0 + R @ np.array([0.0, 0.0, h]), rng.uniform(0.5, 1.2))
    a = rng.uniform(0, 2 * math.pi)
    d = np.array([math.cos(a), math.sin(a), 0.0])
    up, axis = np.array([0.0, 0.0, 1.0]), -d
    side = _bowl(R @ np.stack([up, np.cross(axis, up), axis], 1), t0 + R @ (3.0 * d + np.array([0.0, 0.0, h / 2])),
                 rng.uniform(3.0, 5.0), rho=1.5)
    A, B = _endpoints(rng, R, t0, 0.4, h - 0.4)
    return [bowl, lid, side], A, B


def two_arcs_over_floor(rng):
    """Order 3 with two edges and a plane: two arc edges around one vertical
    axis, 0.8-1.2 m and 1.8-2.4 m above a 6 m square floor (radii 1-2 m,
    120-270 degrees); TX and RX near the axis."""
    R, t0 = _frame(rng)
    floor = _plane(t0 + R @ np.array([-3.0, -3.0, 0.0]), R[:, 0], R[:, 1], 6.0, 6.0)
    arcs = []
    for z in (rng.uniform(0.8, 1.2), rng.uniform(1.8, 2.4)):
        phi0 = rng.uniform(-math.pi, math.pi)
        arcs.append(_arc(t0 + R @ np.array([0.0, 0.0, z]), R[:, 2], R[:, 0], rng.uniform(1.0, 2.0),
                         phi0, phi0 + rng.uniform(2 * math.pi / 3, 1.5 * math.pi)))
    A, B = _endpoints(rng, R, t0, 0.3, 2.8, r=0.8)
    return [floor, *arcs], A, B


def bowl_between_walls(rng):
    """Order 3 with two planes and a paraboloid: a deep bowl between two
    facing vertical walls (6 m by 4 m, 2.2-3 m from its axis on either
    side); TX and RX above the bowl."""
    R, t0 = _frame(rng)
    bowl = _bowl(R, t0, rng.uniform(0.5, 1.2))
    w = rng.uniform(2.2, 3.0, 2)
    walls = [_plane(t0 + R @ np.array([x, -3.0, -0.5]), R[:, 1], R[:, 2], 6.0, 4.0) for x in (w[0], -w[1])]
    A, B = _endpoints(rng, R, t0, 0.4, 2.5, r=1.5)
    return [bowl, *walls], A, B


def test_plane_with_paraboloid_order2():
    n, multi, found = _run(flat_lid_over_bowl, 30, 2, [(0, 1), (1, 0)], 8, (8, 64, 256), seed=21)
    assert n >= 40 and multi >= 3


def test_plane_with_arc_order2():
    n, multi, found = _run(arc_over_ground, 30, 2, [(0, 1), (1, 0)], 8, (8, 64, 256), seed=22)
    assert n >= 40


def test_straight_edge_with_paraboloid_order2():
    n, multi, found = _run(edge_over_bowl, 30, 2, [(0, 1), (1, 0)], 8, (8, 64, 256), seed=26)
    assert n >= 40


def test_two_arcs_order2():
    n, multi, found = _run(two_arcs, 30, 2, [(0, 1), (1, 0)], 24, (8, 64, 256), seed=23)
    assert n >= 40 and multi >= 3


def test_bowl_rim_and_lid_order3():
    seqs = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)]
    n, multi, found = _run(bowl_rim_and_lid, 8, 3, seqs, 5, (8, 64, 1024), seed=24)
    assert n >= 40 and multi >= 6


def test_bowl_edge_and_lid_order3():
    seqs = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)]
    n, multi, found = _run(bowl_edge_and_lid, 6, 3, seqs, 5, (8, 64, 1024), seed=27)
    assert n >= 25


def test_three_paraboloids_order3():
    seqs = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)]
    n, multi, found = _run(three_mirrors, 12, 3, seqs, 4, (8, 64, 1024), seed=28)
    assert n >= 20


def test_two_arcs_over_floor_order3():
    seqs = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)]
    n, multi, found = _run(two_arcs_over_floor, 8, 3, seqs, 5, (8, 64, 1024), seed=29)
    assert n >= 40 and multi >= 10


def test_bowl_between_walls_order3():
    seqs = [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)]
    n, multi, found = _run(bowl_between_walls, 5, 3, seqs, 5, (8, 64, 1024), seed=30)
    assert n >= 15
