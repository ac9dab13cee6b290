"""Whole-workload comparison of the GPU's valid paths with the FP64 oracle's.

Test infrastructure: imports the oracle.  The oracle solves and validates
every candidate of a workload in chunks (threads = all host cores); the GPU
side is the compacted path list of one mpt_validate call.  The bar
(Algorithm 1: "C < threshold and X is valid"):

  - every candidate the oracle finds valid and does not flag as ambiguous is
    valid on the GPU (nothing missing);
  - every GPU-valid candidate is oracle-valid or oracle-ambiguous (nothing
    extra);
  - interaction points of the common paths agree within 1e-6 m.

Ambiguous = a decision of the oracle fell inside its tolerance band (cost
within a factor 100 of tau, a segment within a factor 3 of the minimum
length, a point within 1e-6 m of a bound, a crossing within the visibility
band); those candidates may go either way and are counted, not compared.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

POINT_TOL = 1e-6  # metres


@dataclasses.dataclass
class GpuSide:
    cand: np.ndarray  # int64 [n] valid candidates, ascending
    X: np.ndarray  # float64 [n, 12]
    status: np.ndarray | None = None  # uint8 [n_cand] solver status of every candidate
    cost: np.ndarray | None = None  # float64 [n_cand]
    iters: np.ndarray | None = None
    evals: np.ndarray | None = None


def gpu_side(paths, sols=None) -> GpuSide:
    n = paths.n()
    cand = paths.cand[:n].cpu().numpy().astype(np.int64)
    X = paths.X[:, :n].cpu().numpy().T.copy()
    g = GpuSide(cand, X)
    if sols is not None:
        g.status = sols.status.cpu().numpy()
        g.cost = sols.cost.cpu().numpy()
        g.iters = sols.iters.cpu().numpy()
        g.evals = sols.evals.cpu().numpy()
    return g


@dataclasses.dataclass
class Report:
    n_candidates: int = 0
    n_oracle_valid: int = 0  # valid and not ambiguous
    n_ambiguous: int = 0
    n_gpu_valid: int = 0
    n_common: int = 0
    max_err: float = 0.0
    missing: list = dataclasses.field(default_factory=list)  # details of oracle-valid, GPU-invalid
    extra: list = dataclasses.field(default_factory=list)  # details of GPU-valid, oracle-invalid
    n_missing: int = 0
    n_extra: int = 0
    # per-candidate oracle verdicts kept for root-set comparisons (optional)
    valid_idx: np.ndarray | None = None
    amb_idx: np.ndarray | None = None
    valid_X: np.ndarray | None = None
    amb_X: np.ndarray | None = None

    def ok(self) -> bool:
        return self.n_missing == 0 and self.n_extra == 0 and self.max_err < POINT_TOL

    def summary(self) -> str:
        s = (f"{self.n_candidates} candidates: oracle {self.n_oracle_valid} valid (+{self.n_ambiguous} ambiguous), "
             f"gpu {self.n_gpu_valid} valid, {self.n_common} common, max point error {self.max_err:.2e} m, "
             f"missing {self.n_missing}, extra {self.n_extra}")
        for tag, lst in (("missing", self.missing), ("extra", self.extra)):
            for d in lst[:12]:
                s += f"\n  {tag}: " + ", ".join(f"{k}={v}" for k, v in d.items())
        return s


def _detail(sc, table, c, sol, i, ver, gpu: GpuSide):
    e, p = divmod(int(c), sc.n_pairs)
    n = int(table.order[e])
    d = {"cand": int(c), "ids": tuple(int(x) for x in table.ids[e][:n]),
         "kinds": tuple(int(sc.obj_kind[x]) for x in table.ids[e][:n]), "pair": p, "start": int(table.start[e]),
         "o_status": int(sol.status[i]), "o_iters": int(sol.iters[i]), "o_cost": f"{sol.cost[i]:.2e}",
         "o_valid": int(ver.valid[i]), "o_amb": int(ver.ambiguous[i])}
    if gpu.status is not None:
        d.update({"g_status": hex(int(gpu.status[c])), "g_iters": int(gpu.iters[c]), "g_evals": int(gpu.evals[c]),
                  "g_cost": f"{gpu.cost[c]:.2e}"})
    return d


def compare_workload(sc, table, gpu: GpuSide, chunk: int = 1 << 21, keep_sets: bool = False,
                     max_details: int = 50) -> Report:
    total = len(table) * sc.n_pairs
    rep = Report(n_candidates=total, n_gpu_valid=len(gpu.cand))
    g_cand = gpu.cand
    assert np.all(np.diff(g_cand) > 0), "GPU path list is not in ascending candidate order"
    vidx, aidx, vX, aX = [], [], [], []
    for b in range(0, total, chunk):
        e = min(total, b + chunk)
        sol, ver = oracle.candidate_range(sc, table, b, e)
        valid = ver.valid.astype(bool)
        amb = ver.ambiguous.astype(bool)
        ok = valid & ~amb
        rep.n_oracle_valid += int(ok.sum())
        rep.n_ambiguous += int(amb.sum())
        lo, hi = np.searchsorted(g_cand, [b, e])
        gc = g_cand[lo:hi] - b
        gmask = np.zeros(e - b, bool)
        gmask[gc] = True
        miss = np.nonzero(ok & ~gmask)[0]
        extra = np.nonzero(gmask & ~valid & ~amb)[0]
        rep.n_missing += len(miss)
        rep.n_extra += len(extra)
        for i in miss[:max(0, max_details - len(rep.missing))]:
            rep.missing.append(_detail(sc, table, b + i, sol, i, ver, gpu))
        for i in extra[:max(0, max_details - len(rep.extra))]:
            rep.extra.append(_detail(sc, table, b + i, sol, i, ver, gpu))
        common = np.nonzero(ok & gmask)[0]
        if len(common):
            gpos = lo + np.searchsorted(gc, common)
            order = table.order[(b + common) // sc.n_pairs]
            k = 3 * order
            diff = np.abs(gpu.X[gpos] - sol.X[common])
            col = np.arange(12)[None, :] < k[:, None]
            rep.max_err = max(rep.max_err, float(np.where(col, diff, 0.0).max()))
            rep.n_common += len(common)
        if keep_sets:
            vidx.append(b + np.nonzero(ok)[0])
            vX.append(sol.X[ok])
            aidx.append(b + np.nonzero(amb)[0])
            aX.append(sol.X[amb])
    if keep_sets:
        rep.valid_idx = np.concatenate(vidx) if vidx else np.zeros(0, np.int64)
        rep.amb_idx = np.concatenate(aidx) if aidx else np.zeros(0, np.int64)
        rep.valid_X = np.concatenate(vX) if vX else np.zeros((0, 12))
        rep.amb_X = np.concatenate(aX) if aX else np.zeros((0, 12))
    return rep


def _dedup(points: list, tol: float) -> list:
    roots = []
    for x in points:
        if not any(np.abs(x - r).max() < tol for r in roots):
            roots.append(x)
    return roots


def root_set_differences(sc, table, gpu: GpuSide, rep: Report, tol: float = POINT_TOL, group_tol: float = 1e-4):
    """Per (TX/RX pair, object sequence) sets of distinct valid roots over all
    starts of the sequence (Sec. III-B: several starts for curved objects,
    every distinct root is a path).  Returns the groups whose sets differ:
    an oracle root (valid, not ambiguous) the GPU lacks, or a GPU root that
    is neither an oracle root nor the point of an ambiguous oracle candidate."""
    # first entry of each run of equal id tuples (the starts of one sequence)
    first = np.zeros(len(table), np.int64)
    for e in range(1, len(table)):
        first[e] = first[e - 1] if np.array_equal(table.ids[e], table.ids[e - 1]) else e
    n_pairs = sc.n_pairs

    def key(c):
        e, p = divmod(int(c), n_pairs)
        return int(first[e]), p

    o_roots, a_roots, g_roots = {}, {}, {}
    for c, x in zip(rep.valid_idx, rep.valid_X):
        o_roots.setdefault(key(c), []).append(x)
    for c, x in zip(rep.amb_idx, rep.amb_X):
        a_roots.setdefault(key(c), []).append(x)
    for c, x in zip(gpu.cand, gpu.X):
        g_roots.setdefault(key(c), []).append(x)
    diffs = []
    n_groups = 0
    for k in set(o_roots) | set(g_roots):
        n_groups += 1
        o = _dedup(o_roots.get(k, []), group_tol)
        g = _dedup(g_roots.get(k, []), group_tol)
        a = a_roots.get(k, [])
        lack = [x for x in o if not any(np.abs(x - y).max() < tol for y in g)]
        more = [y for y in g if not any(np.abs(x - y).max() < tol for x in o)
                and not any(np.abs(x - y).max() < 1e-4 for x in a)]
        if lack or more:
            diffs.append({"entry": k[0], "pair": k[1], "ids": tuple(int(v) for v in table.ids[k[0]] if v >= 0),
                          "oracle_roots": len(o), "gpu_roots": len(g), "lack": len(lack), "more": len(more)})
    return n_groups, diffs


def points_from_params(sc, table, cand: np.ndarray, T_slots: np.ndarray) -> np.ndarray:
    """Interaction points [n, 12] of candidates from their parameters in two
    slots per interaction (an edge uses slot 2k), by the parametrisations of
    Eqs. 13-14 on the scene records: plane O + s u + t v; paraboloid
    t0 + R (s, t, (s^2 + t^2) / (4 f)); line P + t e; arc
    C + Rc (cos t u + sin t (a x u)).  Unused slots are 0."""
    cand = np.asarray(cand, np.int64)
    ent = cand // sc.n_pairs
    ids = table.ids[ent]
    order = table.order[ent]
    X = np.zeros((len(cand), 12))
    for k in range(4):
        has = np.nonzero(order > k)[0]
        if len(has) == 0:
            continue
        o = ids[has, k]
        p = sc.obj_param[o]
        kind = sc.obj_kind[o]
        s = T_slots[has, 2 * k]
        t = T_slots[has, 2 * k + 1]
        P = np.zeros((len(has), 3))
        m = kind == 0
        P[m] = p[m, 4:7] + s[m, None] * p[m, 7:10] + t[m, None] * p[m, 10:13]
        m = kind == 1
        if m.any():
            loc = np.stack([s[m], t[m], (s[m] ** 2 + t[m] ** 2) / (4.0 * p[m, 12])], 1)
            P[m] = p[m, 9:12] + np.einsum("nij,nj->ni", p[m, 0:9].reshape(-1, 3, 3), loc)
        m = kind == 2
        P[m] = p[m, 0:3] + s[m, None] * p[m, 3:6]
        m = kind == 3
        if m.any():
            a, u = p[m, 3:6], p[m, 7:10]
            v = np.cross(a, u)
            P[m] = p[m, 0:3] + p[m, 6:7] * (np.cos(s[m])[:, None] * u + np.sin(s[m])[:, None] * v)
        X[has, 3 * k:3 * k + 3] = P
    return X


def fp32_point_error(sc, table, rep: Report, T32: np.ndarray):
    """Max distance between the FP32 solver's points (parameters before the
    refinement, T32 [8, n_cand]) and the oracle's, over the oracle-valid
    candidates (rep.valid_idx, rep.valid_X)."""
    c = rep.valid_idx
    if len(c) == 0:
        return float("nan")
    X32 = points_from_params(sc, table, c, T32[:, c].T.astype(np.float64))
    order = table.order[c // sc.n_pairs]
    col = np.arange(12)[None, :] < 3 * order[:, None]
    return float(np.where(col, np.abs(X32 - rep.valid_X), 0.0).max())


def _beams(sc, points: np.ndarray, h_min: float):
    """For every point P and plane i: the four faces of the pyramid from P's
    mirror image through rectangle i (unit normals pointing inwards, offsets
    <n, image>) and whether the pyramid is used (P more than h_min from the
    plane).  Returns faces [n_points, n_obj, 4, 4] and ok [n_points, n_obj]."""
    kinds = np.asarray(sc.obj_kind)
    par = np.asarray(sc.obj_param, np.float64)
    n = len(kinds)
    faces = np.zeros((len(points), n, 4, 4))
    ok = np.zeros((len(points), n), bool)
    for i in range(n):
        if kinds[i] != 0:
            continue
        nrm, O, u, v, U, V = par[i][0:3], par[i][4:7], par[i][7:10], par[i][10:13], par[i][13], par[i][14]
        h = (points - O) @ nrm
        img = points - 2.0 * h[:, None] * nrm
        C = [O, O + U * u, O + U * u + V * v, O + V * v]
        cen = O + 0.5 * U * u + 0.5 * V * v
        for f in range(4):
            nn = np.cross(C[f] - img, C[(f + 1) % 4] - img)
            flip = np.einsum("ij,ij->i", nn, cen - img) < 0
            nn[flip] *= -1.0
            nn /= np.linalg.norm(nn, axis=1, keepdims=True)
            faces[:, i, f, :3] = nn
            faces[:, i, f, 3] = np.einsum("ij,ij->i", nn, img)
        ok[:, i] = np.abs(h) > h_min
    return faces, ok


def exclusion_mask(sc, table, m_tx: float = 1e-5, m_obj: float = 1e-6, m_beam: float = 1e-5,
                   h_min: float = 1e-2, beam: bool = True) -> np.ndarray:
    """Candidates (c = entry * n_pairs + pair) that the reflection law (Eq. 8)
    rules out before any iteration, written with numpy from the law,
    independently of the solver's code (margins in units of the scene scale
    S):

      - half-space: the segment after a reflection leaves on the side of the
        plane that the segment before it came from.  Excluded: the first
        reflection with TX more than m_tx from its plane and the next object
        wholly (every vertex of oracle._object_vertices) more than m_obj on
        the other side (RX for a single reflection); the last reflection
        likewise with RX and the previous object; an inner reflection with
        its two neighbouring objects on opposite sides;
      - beam (beam=True): the outgoing ray of the first reflection is the ray
        from TX's mirror image through the reflection point, so the next
        object (RX for a single reflection) must meet the pyramid from that
        image through the rectangle; likewise backwards from RX for the last
        reflection.  Excluded: every vertex more than m_beam outside one face
        of the pyramid, for an endpoint more than h_min from the plane."""
    kinds = np.asarray(sc.obj_kind)
    par = np.asarray(sc.obj_param, np.float64)
    n = len(kinds)
    verts = [np.asarray(oracle._object_vertices(int(kinds[i]), par[i])) for i in range(n)]
    tx, rx = np.asarray(sc.tx, np.float64), np.asarray(sc.rx, np.float64)
    if sc.pair_mode == 0:
        it = np.repeat(np.arange(len(tx)), len(rx))
        ir = np.tile(np.arange(len(rx)), len(tx))
    else:
        it = ir = np.arange(len(tx))
    A, B = tx[it], rx[ir]
    S = sc.scale
    mt, mo, mb = m_tx * S, m_obj * S, m_beam * S
    if beam:
        fa, oka = _beams(sc, tx, h_min * S)
        fb, okb = _beams(sc, rx, h_min * S)

    def dist(i, X):  # signed distance to plane i: <n, X - O>
        return (X - par[i][4:7]) @ par[i][0:3]

    def outside(faces, ok, X):
        """faces [k, 4, 4], ok [k], X [k, m, 3] or [m, 3]: all points more
        than mb outside one face."""
        d = np.einsum("kfj,mj->kfm", faces[:, :, :3], X) if X.ndim == 2 else \
            np.einsum("kfj,kmj->kfm", faces[:, :, :3], X)
        d = d - faces[:, :, 3][:, :, None]
        return ok & np.any(np.all(d < -mb, axis=2), axis=1)

    side = np.zeros((n, n), np.int8)  # +1 / -1: object j wholly in front of / behind plane i
    for i in range(n):
        if kinds[i] != 0:
            continue
        for j in range(n):
            if j != i:
                d = dist(i, verts[j])
                side[i, j] = 1 if d.min() > mo else (-1 if d.max() < -mo else 0)
    out = np.zeros(len(table) * len(A), bool)
    for e in range(len(table)):
        o = int(table.order[e])
        ids = [int(x) for x in table.ids[e][:o]]
        ex = np.zeros(len(A), bool)
        if kinds[ids[0]] == 0:
            a = dist(ids[0], A)
            if o == 1:
                b = dist(ids[0], B)
                ex |= ((a > mt) & (b < -mt)) | ((a < -mt) & (b > mt))
                if beam:
                    ex |= outside(fa[it, ids[0]], oka[it, ids[0]], B[:, None, :])
            else:
                s = side[ids[0], ids[1]]
                ex |= ((a > mt) & (s < 0)) | ((a < -mt) & (s > 0))
                if beam:
                    ex |= outside(fa[it, ids[0]], oka[it, ids[0]], verts[ids[1]])
        if o >= 2 and kinds[ids[-1]] == 0:
            b = dist(ids[-1], B)
            s = side[ids[-1], ids[-2]]
            ex |= ((b > mt) & (s < 0)) | ((b < -mt) & (s > 0))
            if beam:
                ex |= outside(fb[ir, ids[-1]], okb[ir, ids[-1]], verts[ids[-2]])
        for k in range(1, o - 1):
            if kinds[ids[k]] == 0 and int(side[ids[k], ids[k - 1]]) * int(side[ids[k], ids[k + 1]]) < 0:
                ex[:] = True
        out[e * len(A):(e + 1) * len(A)] = ex
    return out
