"""Completeness pin of the oracle for every mix of planar reflections and
straight-edge diffractions: the generalised image method.

Route (independent of the MPT residual and minimiser): reflecting everything
that follows a mirror through that mirror (Eq. 5 applied to geometry, not
only to the source) unfolds the path into a polyline whose only bends are at
the diffraction points.  Its length is the path length, every reflection law
holds by straightness, and Eq. 9 at each edge is exactly the derivative of
the length with respect to that edge's parameter.  The length is a sum of
norms of affine functions of the edge parameters, hence convex with a unique
minimiser on infinite edges, found here by damped Newton on dL/dt with the
exact Hessian.  Folding back (the inverse reflections, Eq. 6 in effect) gives
the interaction points.  The path exists when each mirror is crossed between
the polyline's vertices in sequence order and every point lies inside its
object's bounds with no segment shorter than 1e-5 S.  Then, for scenes
without occluders, "the path exists" must equal "the oracle's candidate is
valid", with points equal to 1e-8 m, for every candidate neither side
decides inside its tolerance band.
"""
import numpy as np
import pytest

import oracle
from paper_2301_06399_gb300 import scenes as S

BAND = 1e-6  # metres: geometric decisions closer than this are not compared


def _reflect(X, n, d):
    return X - 2.0 * (X @ n - d) * n


def _reflect_dir(v, n):
    return v - 2.0 * (v @ n) * n


def _unfold(mirrors_before):
    """Apply the mirrors that precede an object (the latest first) to a point
    or direction: returns (point map, direction map)."""
    def pt(X):
        for (n, d) in reversed(mirrors_before):
            X = _reflect(X, n, d)
        return X

    def dr(v):
        for (n, _) in reversed(mirrors_before):
            v = _reflect_dir(v, n)
        return v
    return pt, dr


def _fold(X, mirrors_before):
    """Inverse of _unfold's point map (reflections in the opposite order)."""
    for (n, d) in mirrors_before:
        X = _reflect(X, n, d)
    return X


def _min_length(A, B, lines, max_iter=200):
    """Minimise L(t) = |Y_1 - A| + sum |Y_{j+1} - Y_j| + |B - Y_m| over the
    parameters of the lines Y_j = P_j + t_j e_j (m >= 1) by damped Newton with
    the exact gradient and Hessian.  Returns (t, converged)."""
    m = len(lines)
    P = np.array([l[0] for l in lines])
    E = np.array([l[1] for l in lines])
    # start: the foot of the straight line A-B on each line
    t = np.array([(0.5 * (A + B) - P[j]) @ E[j] for j in range(m)])

    def pts(t):
        return [A] + [P[j] + t[j] * E[j] for j in range(m)] + [B]

    def length(t):
        Q = pts(t)
        return sum(np.linalg.norm(Q[i + 1] - Q[i]) for i in range(m + 1))

    for _ in range(max_iter):
        Q = pts(t)
        g = np.zeros(m)
        H = np.zeros((m, m))
        for i in range(m + 1):
            v = Q[i + 1] - Q[i]
            L = np.linalg.norm(v)
            if L < 1e-300:
                return t, False
            u = v / L
            # v depends on t_{i-1} (start, coefficient -e) and t_i (end, +e)
            cols = []
            if i >= 1:
                cols.append((i - 1, -E[i - 1]))
            if i < m:
                cols.append((i, E[i]))
            for (a, ba) in cols:
                g[a] += ba @ u
                for (b, bb) in cols:
                    H[a, b] += (ba @ bb - (ba @ u) * (bb @ u)) / L
        try:
            step = -np.linalg.solve(H + 1e-14 * np.eye(m) * max(1.0, np.abs(H).max()), g)
        except np.linalg.LinAlgError:
            return t, False
        L0 = length(t)
        alpha = 1.0
        while alpha > 1e-12 and length(t + alpha * step) > L0 + 1e-15 * max(1.0, L0):
            alpha *= 0.5
        t = t + alpha * step
        if np.abs(alpha * step).max() < 1e-13:
            return t, True
    return t, False


def generalised_image_method(scene, ids, A, B):
    """Points of the path of sequence `ids` (planes and straight edges) from
    A to B, and the verdict.  Returns (exists, ambiguous, X [n, 3])."""
    kinds = scene.obj_kind
    par = scene.obj_param
    S_ = scene.scale
    mirrors = []  # (n, d) of the mirrors passed so far, in sequence order
    before = []  # per object: the mirrors that precede it
    for o in ids:
        before.append(list(mirrors))
        if kinds[o] == S.PLANE:
            mirrors.append((par[o, 0:3], par[o, 3]))
    B_hat = _unfold(mirrors)[0](np.asarray(B, float))
    edges = [k for k, o in enumerate(ids) if kinds[o] == S.LINE_EDGE]
    lines = []
    for k in edges:
        pt, dr = _unfold(before[k])
        lines.append((pt(par[ids[k], 0:3]), dr(par[ids[k], 3:6])))
    A = np.asarray(A, float)
    if lines:
        t, conv = _min_length(A, B_hat, lines)
        if not conv:
            return False, True, None
        verts = [A] + [lines[j][0] + t[j] * lines[j][1] for j in range(len(lines))] + [B_hat]
    else:
        t = []
        verts = [A, B_hat]
    # walk the unfolded polyline: mirrors between consecutive vertices are
    # crossed in sequence order strictly inside the segment
    X = [None] * len(ids)
    amb = False
    ok = True
    seg = 0
    last_lam = 0.0
    for k, o in enumerate(ids):
        if kinds[o] == S.LINE_EDGE:
            j = edges.index(k)
            X[k] = par[o, 0:3] + t[j] * par[o, 3:6]
            seg += 1
            last_lam = 0.0
            continue
        Pa, Pb = verts[seg], verts[seg + 1]
        pt, dr = _unfold(before[k])
        n_hat = dr(par[o, 0:3])
        d_hat = pt(par[o, 0:3] * par[o, 3]) @ n_hat
        den = (Pb - Pa) @ n_hat
        if abs(den) < 1e-300:
            return False, True, None
        lam = (d_hat - Pa @ n_hat) / den
        seg_len = np.linalg.norm(Pb - Pa)
        if not (last_lam < lam < 1.0):
            ok = False
        if min(abs(lam - last_lam), abs(1.0 - lam)) * seg_len < BAND:
            amb = True
        last_lam = lam
        X[k] = _fold(Pa + lam * (Pb - Pa), before[k])
    if any(x is None for x in X):
        return False, True, None
    X = np.array(X)
    # bounds (inclusive) and the minimum segment length
    for k, o in enumerate(ids):
        p = par[o]
        if kinds[o] == S.PLANE:
            s_, t_ = (X[k] - p[4:7]) @ p[7:10], (X[k] - p[4:7]) @ p[10:13]
            ok = ok and 0 <= s_ <= p[13] and 0 <= t_ <= p[14]
            amb = amb or min(abs(s_), abs(s_ - p[13]), abs(t_), abs(t_ - p[14])) < BAND
        else:
            tt = (X[k] - p[0:3]) @ p[3:6]
            ok = ok and p[6] <= tt <= p[7]
            amb = amb or min(abs(tt - p[6]), abs(tt - p[7])) < BAND
    chain = [A] + list(X) + [np.asarray(B, float)]
    lmin = 1e-5 * S_
    for i in range(len(chain) - 1):
        L = np.linalg.norm(chain[i + 1] - chain[i])
        ok = ok and L >= lmin
        amb = amb or (lmin / 3 <= L <= 3 * lmin)
    return bool(ok), bool(amb), X


def _without_occluders(sc):
    sc = S.Scene(sc.name, sc.scale, sc.obj_kind, sc.obj_param, np.zeros(0, np.int32), np.zeros((0, S.REC)),
                 sc.tx, sc.rx, sc.pair_mode, sc.meta)
    return sc.contiguous()


def _random_mixed_sequences(kinds, rng, count, orders=(2, 3, 4)):
    planes = np.nonzero(kinds == S.PLANE)[0]
    edges = np.nonzero(kinds == S.LINE_EDGE)[0]
    out = []
    while len(out) < count:
        n = int(rng.choice(orders))
        n_edges = int(rng.integers(1, n + 1))  # at least one diffraction
        pick = list(rng.choice(edges, n_edges, replace=False)) + list(rng.choice(planes, n - n_edges, replace=False))
        rng.shuffle(pick)
        out.append([int(x) for x in pick])
    return out


def _table(seqs):
    ids = np.full((len(seqs), 4), -1, np.int32)
    for i, s in enumerate(seqs):
        ids[i, :len(s)] = s
    return oracle.SequenceTable(np.array([len(s) for s in seqs], np.int32), ids, np.zeros(len(seqs), np.int32))


def _compare(sc, seqs, known_misses=()):
    """Candidate by candidate: generalised image method vs oracle verdict.
    known_misses: (sequence, pair) the oracle's minimiser is known to miss
    (each must still be one: an existing path the oracle stops short of)."""
    table = _table(seqs)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    stats = dict(exists=0, absent=0, skipped=0, max_err=0.0, misses=[])
    for e, ids in enumerate(seqs):
        for p in range(sc.n_pairs):
            c = e * sc.n_pairs + p
            a, b = sc.pair_points(p)
            exists, amb, X = generalised_image_method(sc, ids, a, b)
            if amb or ver.ambiguous[c]:
                stats["skipped"] += 1
                continue
            if (tuple(ids), p) in known_misses:
                # the minimiser stalls far from the path (status 3: stalled)
                assert exists and not ver.valid[c] and sol.status[c] == 3 and sol.cost[c] > 0.1, (ids, p)
                stats["misses"].append((tuple(ids), p))
                continue
            assert exists == bool(ver.valid[c]), (
                f"sequence {ids} kinds {[int(sc.obj_kind[i]) for i in ids]} pair {p}: generalised image method "
                f"{exists}, oracle valid {bool(ver.valid[c])} (cost {sol.cost[c]:.2e}, status {sol.status[c]}, "
                f"iters {sol.iters[c]})")
            if exists:
                err = np.abs(sol.X[c, :3 * len(ids)] - X.reshape(-1)).max()
                assert err < 1e-8, (ids, p, err)
                stats["max_err"] = max(stats["max_err"], err)
                stats["exists"] += 1
            else:
                stats["absent"] += 1
    return stats


@pytest.mark.parametrize("tx", [0, 3])
def test_box_city_mixed_sequences_match_generalised_image_method(tx):
    """The mixed-order city's walls, ground and vertical wedge edges (no
    occluders; the geometry of the box-city workloads): 300 random sequences
    of orders 2-4 with at least one edge (consecutive diffractions included)
    x 16 receivers, for two of its transmitters.  No exception."""
    base = S.mixed_order_city()
    rng = np.random.default_rng(21 + tx)
    sc = _without_occluders(base)
    sc.tx = base.tx[tx:tx + 1].copy()
    sc.rx = np.ascontiguousarray(base.rx[rng.choice(base.rx.shape[0], 16, replace=False)])
    sc = sc.contiguous()
    seqs = _random_mixed_sequences(sc.obj_kind, rng, 300)
    st = _compare(sc, seqs)
    print(st)
    assert st["exists"] >= 300 and st["absent"] >= 1000 and st["skipped"] <= 0.15 * len(seqs) * sc.n_pairs


def _random_scene(rng, n_planes=6, n_edges=6):
    b = S._Builder()
    for _ in range(n_planes):
        R = S._random_rotation(rng)
        U, V = rng.uniform(40.0, 90.0, 2)
        c = rng.uniform(-20, 20, 3)
        b.rect_plane(c - 0.5 * U * R[:, 0] - 0.5 * V * R[:, 1], R[:, 0], R[:, 1], U, V, occluder=False)
    for _ in range(n_edges):
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        a1 = np.cross(e, [1.0, 0, 0] if abs(e[0]) < 0.9 else [0, 1.0, 0])
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(e, a1)
        P = rng.uniform(-20, 20, 3)
        b.line_edge(P, e, -30.0, 30.0, a1, a2)
    tx = rng.uniform(-25, 25, (8, 3))
    rx = rng.uniform(-25, 25, (8, 3))
    return b.build("random_mixed", 100.0, tx, rx, pair_mode=1)


# Existing paths on skew geometry that Gauss-Newton from the initial guess of
# reading R5 stops short of (seed, sequence, pair): chains of skew edges whose
# "ends" guess puts the directions nearly anti-parallel to the edges, where
# every Eq. 9 residual saturates near +-2 and the line search stalls (cost
# 0.47, 3.93 and 3.99).  Without the early exits the first and third are
# found, the second is not.  On the box-city geometry there are none.
KNOWN_MISSES = {1: {((10, 7, 0, 8), 3)}, 2: {((6, 9, 10, 8), 2)}, 3: {((10, 9, 8, 6), 4)}}


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_skew_geometry_matches_generalised_image_method(seed):
    """Randomly posed large mirrors and skew edges in every direction, TX and
    RX anywhere: 120 random mixed sequences of orders 2-4 x 8 pairs.  Every
    oracle-valid candidate is a path; every existing path is oracle-valid
    except the named minimiser stalls above."""
    rng = np.random.default_rng(100 + seed)
    sc = _random_scene(rng)
    seqs = _random_mixed_sequences(sc.obj_kind, rng, 120)
    st = _compare(sc, seqs, KNOWN_MISSES[seed])
    print(st)
    assert set(st["misses"]) == KNOWN_MISSES[seed]
    assert st["exists"] >= 300 and st["absent"] >= 350
