"""FP64 CPU oracle for Min-Path-Tracing.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never touch it.  The arithmetic lives in ``mpt_oracle.cpp`` (plain
FP64 C++, see its header for the paper passages each part follows); this
module only compiles it with g++ and marshals numpy arrays.

Completeness of the multi-root solution sets is pinned by dense scans of
the path length's stationary points: curved sequences of every object
kind at orders 1 and 2, and at order 3 five three-object families in all
six orders (every kind in every position); other order-3 combinations run
the same per-interaction code and are compared by multi-start agreement
only.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpt_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TAU = 1e-20  # acceptance threshold on the normalised cost (Algorithm 1)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (host code only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [
        ("n_obj", C.c_int32), ("obj_kind", C.c_void_p), ("obj_param", C.c_void_p),
        ("n_occ", C.c_int32), ("occ_kind", C.c_void_p), ("occ_param", C.c_void_p),
        ("scale", C.c_double), ("tx", C.c_void_p), ("n_tx", C.c_int32),
        ("rx", C.c_void_p), ("n_rx", C.c_int32), ("pair_mode", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            L.oracle_enumerate.restype = I64
            L.oracle_enumerate.argtypes = [I32, P, I32, P, U64, I32, I32, P, P, P, P, I64]
            L.oracle_solve.restype = C.c_int
            L.oracle_solve.argtypes = [P, I64, P, P, P, I64, I64, I64, U64, P, P, P, P, P, C.c_int]
            L.oracle_validate.restype = C.c_int
            L.oracle_validate.argtypes = [P, I64, P, P, I64, I64, I64, P, P, P, D, P, P, P, C.c_int]
            L.oracle_path_grad.restype = C.c_int
            L.oracle_path_grad.argtypes = [P, I32, P, P, P, P, P, P]
            L.oracle_path_grad_many.restype = C.c_int
            L.oracle_path_grad_many.argtypes = [P, I64, P, P, I64, P, P, P, P, P, C.c_int]
            L.oracle_residual.restype = C.c_int
            L.oracle_residual.argtypes = [P, I32, P, P, P, P, P, P]
            L.oracle_segment_blocked.restype = C.c_int
            L.oracle_segment_blocked.argtypes = [P, P, P, P]
            L.oracle_params_in_bounds.restype = C.c_int
            L.oracle_params_in_bounds.argtypes = [P, I32, P, P]
            L.oracle_abi_version.restype = C.c_int
            L.oracle_splitmix64.restype = U64
            L.oracle_splitmix64.argtypes = [U64]
            L.oracle_set_rules.restype = None
            L.oracle_set_rules.argtypes = [I32, I32, D, I32]
            L.oracle_threads.restype = C.c_int
            L.oracle_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class SceneRef:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.scene = scene.contiguous()
        s = self.scene
        self.struct = _Scene(s.n_obj, _p(s.obj_kind).value, _p(s.obj_param).value, s.n_occ,
                             _p(s.occ_kind).value, _p(s.occ_param).value, s.scale, _p(s.tx).value,
                             s.tx.shape[0], _p(s.rx).value, s.rx.shape[0], s.pair_mode)

    @property
    def ptr(self):
        return C.cast(C.pointer(self.struct), C.c_void_p)


@dataclasses.dataclass
class SequenceTable:
    order: np.ndarray  # int32 [E]
    ids: np.ndarray  # int32 [E, 4] (-1 padded)
    start: np.ndarray  # int32 [E]

    def __len__(self):
        return int(self.order.shape[0])


def enumerate_sequences(scene, max_order: int, spec, adj: np.ndarray | None = None) -> SequenceTable:
    """Sequence table of Algorithm 1 (all_simple_paths / seeded quotas)."""
    L = lib()
    kinds = np.ascontiguousarray(scene.obj_kind, np.int32)
    quota = np.ascontiguousarray(spec.as_array(), np.int64)
    adj_p = None
    if adj is not None:
        adj = np.ascontiguousarray(adj, np.uint8)
        adj_p = _p(adj)
    args = (scene.n_obj, _p(kinds), max_order, _p(quota), spec.seed, spec.starts_curved,
            spec.force_edges_every, adj_p)
    e = np.zeros(1, np.int32)
    n = L.oracle_enumerate(*args, _p(e), _p(np.zeros(4, np.int32)), _p(e), 0)
    order = np.zeros(n, np.int32)
    ids = np.zeros((n, 4), np.int32)
    start = np.zeros(n, np.int32)
    n2 = L.oracle_enumerate(*args, _p(order), _p(ids), _p(start), n)
    assert n2 == n
    return SequenceTable(order, ids, start)


@dataclasses.dataclass
class Solutions:
    X: np.ndarray  # float64 [n, 12] interaction points
    T: np.ndarray  # float64 [n, 8] object parameters (Eqs. 13-14)
    cost: np.ndarray  # float64 [n]
    status: np.ndarray  # int32 [n]
    iters: np.ndarray  # int32 [n]
    begin: int = 0


def solve(scene, table: SequenceTable, begin: int = 0, end: int | None = None, init_seed: int = 0,
          threads: int = 0) -> Solutions:
    """Gauss-Newton solve of candidates [begin, end) (c = entry * n_pairs + pair)."""
    L = lib()
    ref = SceneRef(scene)
    n_pairs = scene.n_pairs
    total = len(table) * n_pairs
    end = total if end is None else min(end, total)
    n = max(end - begin, 0)
    X = np.zeros((n, 12), np.float64)
    T = np.zeros((n, 8), np.float64)
    cost = np.zeros(n, np.float64)
    status = np.zeros(n, np.int32)
    iters = np.zeros(n, np.int32)
    if n:
        L.oracle_solve(ref.ptr, len(table), _p(table.order), _p(table.ids), _p(table.start), n_pairs,
                       begin, end, init_seed, _p(X), _p(T), _p(cost), _p(status), _p(iters), threads)
    return Solutions(X, T, cost, status, iters, begin)


@dataclasses.dataclass
class Verdicts:
    valid: np.ndarray  # int32 [n]
    ambiguous: np.ndarray  # int32 [n]
    length: np.ndarray  # float64 [n]


def validate(scene, table: SequenceTable, sol: Solutions, tau: float = TAU, threads: int = 0) -> Verdicts:
    L = lib()
    ref = SceneRef(scene)
    n = sol.X.shape[0]
    valid = np.zeros(n, np.int32)
    amb = np.zeros(n, np.int32)
    length = np.zeros(n, np.float64)
    if n:
        X = np.ascontiguousarray(sol.X)
        T = np.ascontiguousarray(sol.T)
        cost = np.ascontiguousarray(sol.cost)
        L.oracle_validate(ref.ptr, len(table), _p(table.order), _p(table.ids), scene.n_pairs, sol.begin,
                          sol.begin + n, _p(X), _p(T), _p(cost), tau, _p(valid), _p(amb), _p(length),
                          threads)
    return Verdicts(valid, amb, length)


def candidate_range(scene, table: SequenceTable, begin: int, end: int, init_seed: int = 0,
                    threads: int = 0):
    sol = solve(scene, table, begin, end, init_seed, threads)
    ver = validate(scene, table, sol, threads=threads)
    return sol, ver


def _n_params(scene, ids):
    return sum(1 if scene.obj_kind[i] in (2, 3) else 2 for i in ids)


def path_grad(scene, ids, a, b, T):
    """dL/dtheta (theta = TX[3], RX[3], plane offsets d_k) and dX/dtheta at
    a converged path with parameters T."""
    L = lib()
    ref = SceneRef(scene)
    ids = np.asarray([i for i in ids if i >= 0], np.int32)
    n = len(ids)
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(-1)[:_n_params(scene, ids)])
    dL = np.zeros(6 + n, np.float64)
    dX = np.zeros((3 * n, 6 + n), np.float64)
    rc = L.oracle_path_grad(ref.ptr, n, _p(ids), _p(a), _p(b), _p(T), _p(dL), _p(dX))
    if rc != 0:
        raise RuntimeError("oracle_path_grad: singular normal matrix")
    return dL, dX


def pack_params(scene, table: SequenceTable, cand: np.ndarray, T_slots: np.ndarray) -> np.ndarray:
    """Parameters given in two slots per interaction (slot 2k, 2k + 1; an
    edge uses slot 2k only) packed in the oracle's order (an edge takes one
    parameter, a surface two).  T_slots: float64 [n, 8]; returns [n, 8]."""
    n = len(cand)
    ent = np.asarray(cand, np.int64) // scene.n_pairs
    ids = table.ids[ent]
    order = table.order[ent]
    kinds = np.asarray(scene.obj_kind)
    out = np.zeros((n, 8), np.float64)
    pos = np.zeros(n, np.int64)
    rows = np.arange(n)
    for k in range(4):
        has = order > k
        edge = np.zeros(n, bool)
        edge[has] = np.isin(kinds[ids[has, k]], (2, 3))
        r = rows[has]
        out[r, pos[has]] = T_slots[r, 2 * k]
        two = has & ~edge
        out[rows[two], pos[two] + 1] = T_slots[rows[two], 2 * k + 1]
        pos = pos + np.where(has, np.where(edge, 1, 2), 0)
    return out


def grad_sums(scene, table: SequenceTable, cand: np.ndarray, T_packed: np.ndarray, g_len: np.ndarray,
              g_pts: np.ndarray | None = None, threads: int = 0):
    """Sums over paths of the upstream-weighted implicit-function-theorem
    gradient (oracle_path_grad per path): d/dTX [n_tx, 3], d/dRX [n_rx, 3]
    and d/d(plane offset) [n_obj] (non-planar interactions add 0)."""
    L = lib()
    ref = SceneRef(scene)
    cand = np.ascontiguousarray(cand, np.int64)
    n = len(cand)
    T = np.ascontiguousarray(T_packed, np.float64)
    gl = np.ascontiguousarray(g_len, np.float64)
    gp = None if g_pts is None else np.ascontiguousarray(g_pts, np.float64)
    w = np.zeros((n, 10), np.float64)
    bad = L.oracle_path_grad_many(ref.ptr, n, _p(table.order), _p(table.ids), scene.n_pairs, _p(cand), _p(T),
                                  _p(gl), None if gp is None else _p(gp), _p(w), threads)
    if bad:
        raise RuntimeError(f"oracle_path_grad_many: {bad} singular normal matrices")
    ent, pair = np.divmod(cand, scene.n_pairs)
    n_rx = scene.rx.shape[0]
    it, ir = (pair // n_rx, pair % n_rx) if scene.pair_mode == 0 else (pair, pair)
    gtx = np.zeros_like(scene.tx)
    grx = np.zeros_like(scene.rx)
    gobj = np.zeros(scene.n_obj)
    np.add.at(gtx, it, w[:, 0:3])
    np.add.at(grx, ir, w[:, 3:6])
    order = table.order[ent]
    ids = table.ids[ent]
    for k in range(4):
        has = order > k
        np.add.at(gobj, ids[has, k], w[has, 6 + k])
    return gtx, grx, gobj


def residual(scene, ids, a, b, T):
    """Stacked law residual (Eq. 10) and the points X(T)."""
    L = lib()
    ref = SceneRef(scene)
    ids = np.asarray([i for i in ids if i >= 0], np.int32)
    n = len(ids)
    out = np.zeros(12, np.float64)
    X = np.zeros(3 * n, np.float64)
    T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(-1)[:_n_params(scene, ids)])
    m = L.oracle_residual(ref.ptr, n, _p(ids), _p(np.ascontiguousarray(a, np.float64)),
                          _p(np.ascontiguousarray(b, np.float64)), _p(T), _p(out), _p(X))
    return out[:m], X


def cost(scene, ids, a, b, T) -> float:
    return float(np.sum(residual(scene, ids, a, b, T)[0] ** 2))


def segment_blocked(scene, A, B) -> tuple[bool, bool]:
    L = lib()
    ref = SceneRef(scene)
    amb = np.zeros(1, np.int32)
    r = L.oracle_segment_blocked(ref.ptr, _p(np.ascontiguousarray(A, np.float64)),
                                 _p(np.ascontiguousarray(B, np.float64)), _p(amb))
    return bool(r), bool(amb[0])


def params_in_bounds(scene, obj, u) -> tuple[bool, bool]:
    L = lib()
    ref = SceneRef(scene)
    amb = np.zeros(1, np.int32)
    u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(-1))
    r = L.oracle_params_in_bounds(ref.ptr, int(obj), _p(u), _p(amb))
    return bool(r), bool(amb[0])


DEFAULT_RULES = dict(max_iters=24, max_evals=40, min_alpha=1.0 / 16.0, localmin_exit=True)


def set_rules(max_iters: int = 24, max_evals: int = 40, min_alpha: float = 1.0 / 16.0,
              localmin_exit: bool = True) -> None:
    """Stopping rules of the oracle's minimiser (reading R15's values by
    default).  A test hook: the rules apply to every later solve."""
    lib().oracle_set_rules(int(max_iters), int(max_evals), float(min_alpha), int(bool(localmin_exit)))


def splitmix64(x: int) -> int:
    return int(lib().oracle_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def threads(n: int = 0) -> int:
    return int(lib().oracle_threads(n))


# ------------------------------------------------------- visibility matrix --
def _object_vertices(kind: int, p: np.ndarray) -> np.ndarray:
    """Points whose convex hull holds every point the object can put on a path
    (record layouts of include/mpt.h): a rectangle's four corners, a line
    edge's two ends, the eight corners of the local box [-rho, rho]^2 x
    [0, rho^2 / (4f)] of a paraboloid patch, the four corners of the square
    of half-side Rc around an arc's centre in its plane."""
    if kind == 0:  # plane
        O, Ua, Va, U, V = p[4:7], p[7:10], p[10:13], p[13], p[14]
        return np.array([O, O + U * Ua, O + V * Va, O + U * Ua + V * Va])
    if kind == 2:  # line edge
        P, e, t0, t1 = p[0:3], p[3:6], p[6], p[7]
        return np.array([P + t0 * e, P + t1 * e])
    if kind == 1:  # paraboloid: X = t0 + R (s, t, (s^2 + t^2) / (4 f))
        R = p[0:9].reshape(3, 3)
        t0, f, rho = p[9:12], p[12], p[13]
        out = []
        for sx in (-rho, rho):
            for sy in (-rho, rho):
                for sz in (0.0, rho * rho / (4.0 * f)):
                    out.append(t0 + R @ np.array([sx, sy, sz]))
        return np.array(out)
    # arc edge: X = C + Rc (cos t u + sin t (a x u))
    C, a, Rc, u = p[0:3], p[3:6], p[6], p[7:10]
    v = np.cross(a, u)
    return np.array([C + Rc * (sx * u + sy * v) for sx in (-1.0, 1.0) for sy in (-1.0, 1.0)])


def visibility_matrix(scene) -> np.ndarray:
    """Object visibility matrix V of Algorithm 1 (its first line; Sec. III,
    Fig. 5), under the reading that a planar facet reflects on the side its
    normal points to: V[i, j] = 0 when i == j, or when one of the two objects
    is a plane and every vertex of the other lies more than 1e-6 S behind
    that plane (<n, X - O> < -1e-6 S); otherwise 1.  Edges and paraboloids
    are seen from every side.  Used as the adjacency mask of the
    enumeration.  Plain double loops over the object pairs."""
    kinds = np.asarray(scene.obj_kind)
    par = np.asarray(scene.obj_param, np.float64)
    n = len(kinds)
    delta = 1e-6 * float(scene.scale)
    verts = [_object_vertices(int(kinds[i]), par[i]) for i in range(n)]

    def hidden_behind(i: int, j: int) -> bool:
        # every vertex of object j strictly behind plane i
        nrm, O = par[i][0:3], par[i][4:7]
        return all(float(np.dot(nrm, x - O)) < -delta for x in verts[j])

    V = np.ones((n, n), np.uint8)
    for i in range(n):
        V[i, i] = 0
        for j in range(n):
            if i == j:
                continue
            if (kinds[i] == 0 and hidden_behind(i, j)) or (kinds[j] == 0 and hidden_behind(j, i)):
                V[i, j] = 0
    return V


# -------------------------------------------------------------- path field --
def path_field(scene, table: SequenceTable, sol: Solutions, ver: Verdicts, wavenumber: float, e0: float = 1.0,
               refl: complex = -1.0, diff: complex = 1.0) -> np.ndarray:
    """Received field per TX/RX pair (Sec. V, Eqs. 16-19), scalar form: every
    valid path with segment lengths d_0..d_n (total L) adds
    E0 e^{-jkL} / d_0 * prod_k C_k, where interaction k, reached after
    r_k = d_0 + ... + d_{k-1}, has C = refl * r_k / (r_k + d_k) (reflection,
    Eq. 17) or C = diff * sqrt(r_k / (d_k (r_k + d_k))) (diffraction, Eq.
    18).  Returns complex128 [n_pairs].  Plain loops over the valid paths."""
    n_pairs = scene.n_pairs
    out = np.zeros(n_pairs, np.complex128)
    kinds = np.asarray(scene.obj_kind)
    tx, rx = np.asarray(scene.tx), np.asarray(scene.rx)
    for i in np.nonzero(ver.valid)[0]:
        c = sol.begin + int(i)
        e, p = divmod(c, n_pairs)
        n = int(table.order[e])
        ids = table.ids[e][:n]
        if scene.pair_mode == 0:
            a, b = tx[p // len(rx)], rx[p % len(rx)]
        else:
            a, b = tx[p], rx[p]
        pts = [a] + [sol.X[i, 3 * k:3 * k + 3] for k in range(n)] + [b]
        d = [float(np.linalg.norm(pts[k + 1] - pts[k])) for k in range(n + 1)]
        amp = complex(e0) / d[0]
        r = d[0]
        for k in range(n):
            s = d[k + 1]
            if kinds[ids[k]] in (2, 3):
                amp *= diff * np.sqrt(r / (s * (r + s)))
            else:
                amp *= refl * r / (r + s)
            r += s
        out[p] += amp * np.exp(-1j * wavenumber * sum(d))
    return out
