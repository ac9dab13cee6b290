"""Seeded synthetic scenes for Min-Path-Tracing workloads.

This module only *builds inputs*: implicit objects, occluders and TX/RX
positions, as plain float64 arrays.  It contains none of the method's
arithmetic (no residuals, no minimisation, no visibility), so both the FP64
CPU oracle and the CUDA library consume the same scenes without sharing any
computation.

Object model (Sec. II of the paper: every facet has an implicit equation
f(x, y, z) = 0, every edge an implicit description plus a direction vector,
and bounds are applied only when a path is validated):

  kind 0  plane      <n, X> = d, bounded by the rectangle O + u*U_ax + v*V_ax,
                     u in [0, U], v in [0, V]
  kind 1  paraboloid local z = (x^2 + y^2) / (4 f) in the frame X = t + R x_loc,
                     bounded by the disc x^2 + y^2 <= rho^2
  kind 2  line edge  X = P + s e, s in [s0, s1]; two unit normals a1, a2 (both
                     orthogonal to e) describe it implicitly: <a_j, X - P> = 0
  kind 3  arc edge   circle of radius Rc around C in the plane normal to the
                     axis a; angle phi measured from the unit reference u_ref
                     toward a x u_ref, phi in [phi0, phi1]

Parameter records are float64[24] per object (layout in ``OBJ_LAYOUT``).
Occluders (surfaces a segment may not cross) are kind 0 rectangles and kind 1
paraboloid patches, also float64[24] (layout in ``OCC_LAYOUT``).  Edges never
occlude.  Roofs of box buildings are occluder-only rectangles.

TX/RX pairs: ``pair_mode`` 0 = every (tx, rx) combination, pair p = t * n_rx + r;
``pair_mode`` 1 = zipped, pair p = (tx[p], rx[p]).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PLANE, PARABOLOID, LINE_EDGE, ARC_EDGE = 0, 1, 2, 3
OCC_RECT, OCC_PARABOLOID = 0, 1
REC = 24

# Field offsets inside an object record.
OBJ_LAYOUT = {
    PLANE: {"n": 0, "d": 3, "O": 4, "u": 7, "v": 10, "U": 13, "V": 14},
    PARABOLOID: {"R": 0, "t": 9, "f": 12, "rho": 13},
    LINE_EDGE: {"P": 0, "e": 3, "s0": 6, "s1": 7, "a1": 8, "a2": 11},
    ARC_EDGE: {"C": 0, "a": 3, "Rc": 6, "u": 7, "phi0": 10, "phi1": 11},
}
# Field offsets inside an occluder record.
OCC_LAYOUT = {
    OCC_RECT: {"O": 0, "u": 3, "v": 6, "U": 9, "V": 10, "n": 11},
    OCC_PARABOLOID: {"R": 0, "t": 9, "f": 12, "rho": 13},
}


@dataclasses.dataclass
class Scene:
    """A scene plus its TX/RX layout.  All arrays are float64 / int32 numpy."""

    name: str
    scale: float
    obj_kind: np.ndarray  # int32 [n_obj]
    obj_param: np.ndarray  # float64 [n_obj, 24]
    occ_kind: np.ndarray  # int32 [n_occ]
    occ_param: np.ndarray  # float64 [n_occ, 24]
    tx: np.ndarray  # float64 [n_tx, 3]
    rx: np.ndarray  # float64 [n_rx, 3]
    pair_mode: int = 0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_obj(self) -> int:
        return int(self.obj_kind.shape[0])

    @property
    def n_occ(self) -> int:
        return int(self.occ_kind.shape[0])

    @property
    def n_pairs(self) -> int:
        if self.pair_mode == 0:
            return int(self.tx.shape[0] * self.rx.shape[0])
        return int(self.tx.shape[0])

    def pair_points(self, p: int) -> tuple[np.ndarray, np.ndarray]:
        if self.pair_mode == 0:
            n_rx = self.rx.shape[0]
            return self.tx[p // n_rx], self.rx[p % n_rx]
        return self.tx[p], self.rx[p]

    def contiguous(self) -> "Scene":
        for f in ("obj_kind", "occ_kind"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.int32))
        for f in ("obj_param", "occ_param", "tx", "rx"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        return self


class _Builder:
    def __init__(self):
        self.kind: list[int] = []
        self.param: list[np.ndarray] = []
        self.okind: list[int] = []
        self.oparam: list[np.ndarray] = []

    # -- objects -------------------------------------------------------
    def rect_plane(self, O, u_ax, v_ax, U, V, occluder=True):
        """Rectangle O + u*u_ax + v*v_ax with unit axes; plane normal u_ax x v_ax."""
        O, u_ax, v_ax = (np.asarray(a, np.float64) for a in (O, u_ax, v_ax))
        n = np.cross(u_ax, v_ax)
        n = n / np.linalg.norm(n)
        r = np.zeros(REC)
        L = OBJ_LAYOUT[PLANE]
        r[L["n"]:L["n"] + 3] = n
        r[L["d"]] = float(n @ O)
        r[L["O"]:L["O"] + 3] = O
        r[L["u"]:L["u"] + 3] = u_ax
        r[L["v"]:L["v"] + 3] = v_ax
        r[L["U"]] = U
        r[L["V"]] = V
        self.kind.append(PLANE)
        self.param.append(r)
        if occluder:
            self.occ_rect(O, u_ax, v_ax, U, V)
        return len(self.kind) - 1

    def paraboloid(self, R, t, f, rho, occluder=True):
        r = np.zeros(REC)
        L = OBJ_LAYOUT[PARABOLOID]
        r[L["R"]:L["R"] + 9] = np.asarray(R, np.float64).reshape(9)
        r[L["t"]:L["t"] + 3] = t
        r[L["f"]] = f
        r[L["rho"]] = rho
        self.kind.append(PARABOLOID)
        self.param.append(r)
        if occluder:
            o = np.zeros(REC)
            o[:14] = r[:14]
            self.okind.append(OCC_PARABOLOID)
            self.oparam.append(o)
        return len(self.kind) - 1

    def line_edge(self, P, e, s0, s1, a1, a2):
        r = np.zeros(REC)
        L = OBJ_LAYOUT[LINE_EDGE]
        r[L["P"]:L["P"] + 3] = P
        r[L["e"]:L["e"] + 3] = e
        r[L["s0"]] = s0
        r[L["s1"]] = s1
        r[L["a1"]:L["a1"] + 3] = a1
        r[L["a2"]:L["a2"] + 3] = a2
        self.kind.append(LINE_EDGE)
        self.param.append(r)
        return len(self.kind) - 1

    def arc_edge(self, C, a, Rc, u_ref, phi0, phi1):
        r = np.zeros(REC)
        L = OBJ_LAYOUT[ARC_EDGE]
        r[L["C"]:L["C"] + 3] = C
        r[L["a"]:L["a"] + 3] = a
        r[L["Rc"]] = Rc
        r[L["u"]:L["u"] + 3] = u_ref
        r[L["phi0"]] = phi0
        r[L["phi1"]] = phi1
        self.kind.append(ARC_EDGE)
        self.param.append(r)
        return len(self.kind) - 1

    # -- occluders -----------------------------------------------------
    def occ_rect(self, O, u_ax, v_ax, U, V):
        O, u_ax, v_ax = (np.asarray(a, np.float64) for a in (O, u_ax, v_ax))
        n = np.cross(u_ax, v_ax)
        n = n / np.linalg.norm(n)
        o = np.zeros(REC)
        L = OCC_LAYOUT[OCC_RECT]
        o[L["O"]:L["O"] + 3] = O
        o[L["u"]:L["u"] + 3] = u_ax
        o[L["v"]:L["v"] + 3] = v_ax
        o[L["U"]] = U
        o[L["V"]] = V
        o[L["n"]:L["n"] + 3] = n
        self.okind.append(OCC_RECT)
        self.oparam.append(o)

    def build(self, name, scale, tx, rx, pair_mode=0, meta=None) -> Scene:
        return Scene(
            name=name,
            scale=float(scale),
            obj_kind=np.asarray(self.kind, np.int32),
            obj_param=np.asarray(self.param, np.float64).reshape(-1, REC),
            occ_kind=np.asarray(self.okind, np.int32),
            occ_param=np.asarray(self.oparam, np.float64).reshape(-1, REC),
            tx=np.asarray(tx, np.float64).reshape(-1, 3),
            rx=np.asarray(rx, np.float64).reshape(-1, 3),
            pair_mode=pair_mode,
            meta=dict(meta or {}),
        ).contiguous()


# ---------------------------------------------------------------------------
# Worked example of Fig. 4 (image method on two mirrors), embedded in 3-D.
# ---------------------------------------------------------------------------

def fig4_scene(bs=(2.0, -1.0), ue=(2.0, 4.0), w1=((0.0, 0.0), (3.5, 3.5)),
               w2=((5.0, 0.5), (5.0, 4.0)), half_height=1.0) -> Scene:
    """Two vertical mirrors in the z=0 plane (Fig. 4): W1 on y = x, W2 on x = 5.

    Mirror k is the rectangle spanned by its 2-D segment and z in
    [-half_height, half_height]; BS and UE sit at z = 0.  The plane normals
    point toward the side BS and UE are on (irrelevant to the residuals, which
    are invariant to the sign of n).
    """
    b = _Builder()
    z = np.array([0.0, 0.0, 1.0])
    for (p, q) in (w1, w2):
        p = np.array([p[0], p[1], -half_height])
        q = np.array([q[0], q[1], -half_height])
        seg = q - p
        L = float(np.linalg.norm(seg))
        u_ax = seg / L
        b.rect_plane(p, u_ax, z, L, 2 * half_height)
    tx = [bs[0], bs[1], 0.0]
    rx = [ue[0], ue[1], 0.0]
    return b.build("fig4", 10.0, [tx], [rx])


# ---------------------------------------------------------------------------
# Street canyon: ground plus two parallel walls (the canyon workload).
# ---------------------------------------------------------------------------

def street_canyon() -> Scene:
    """Ground z=0 (x in [-50,50], y in [-10,10]) and walls y=-10 / y=+10
    (x in [-50,50], z in [0,20]); TX (0,-5,10); 8x8 RX grid over
    x in [-40,40], y in [-8,8] at z = 1.5 m.  576 reflection-only solves at
    order <= 2."""
    b = _Builder()
    ex, ey, ez = np.eye(3)
    b.rect_plane([-50.0, -10.0, 0.0], ex, ey, 100.0, 20.0)  # ground, normal +z
    b.rect_plane([-50.0, -10.0, 0.0], ez, ex, 20.0, 100.0)  # wall y=-10, normal +y
    b.rect_plane([-50.0, 10.0, 0.0], ex, ez, 100.0, 20.0)  # wall y=+10, normal -y
    gx = np.linspace(-40.0, 40.0, 8)
    gy = np.linspace(-8.0, 8.0, 8)
    rx = np.array([[x, y, 1.5] for y in gy for x in gx])
    return b.build("street_canyon", 100.0, [[0.0, -5.0, 10.0]], rx)


# ---------------------------------------------------------------------------
# Box city: axis-aligned buildings, walls + vertical edges + ground + roofs.
# ---------------------------------------------------------------------------

def _place_boxes(rng, n_boxes, half_extent, side_lo, side_hi, h_lo, h_hi, keep_clear, clear_radius,
                 gap):
    boxes = []
    tries = 0
    while len(boxes) < n_boxes:
        tries += 1
        if tries > 100000:
            raise RuntimeError("box placement failed")
        sx = rng.uniform(side_lo, side_hi)
        sy = rng.uniform(side_lo, side_hi)
        h = rng.uniform(h_lo, h_hi)
        x0 = rng.uniform(-half_extent, half_extent - sx)
        y0 = rng.uniform(-half_extent, half_extent - sy)
        x1, y1 = x0 + sx, y0 + sy
        ok = True
        for (a0, b0, a1, b1, _) in boxes:
            if not (x1 + gap <= a0 or a1 + gap <= x0 or y1 + gap <= b0 or b1 + gap <= y0):
                ok = False
                break
        if ok:
            for (cx, cy) in keep_clear:
                dx = max(x0 - cx, 0.0, cx - x1)
                dy = max(y0 - cy, 0.0, cy - y1)
                if dx * dx + dy * dy < clear_radius * clear_radius:
                    ok = False
                    break
        if ok:
            boxes.append((x0, y0, x1, y1, h))
    return boxes


def box_city(seed: int, n_boxes: int, tx, rx_grid: int, rx_half: float = 95.0, rx_z: float = 1.5,
             half_extent: float = 100.0, name: str = "box_city") -> Scene:
    """Seeded box city (the urban-block workload).

    Buildings: footprint sides U[10,30] m, heights U[10,40] m, rejection-placed
    without overlap (2 m minimum gap) in [-half_extent, half_extent]^2, keeping a
    15 m clear radius around every TX.  Objects, in this order: for each box its
    4 walls (outward normals -y, +x, +y, -x), then the ground z=0 bounded to the
    square, then each box's 4 vertical edges (corners in the same order).
    Occluders: the walls, the ground and one roof rectangle per box.
    RX: rx_grid x rx_grid points over [-rx_half, rx_half]^2 at height rx_z;
    points falling inside a footprint are kept (validity decides).
    """
    rng = np.random.default_rng(seed)
    tx = np.asarray(tx, np.float64).reshape(-1, 3)
    boxes = _place_boxes(rng, n_boxes, half_extent, 10.0, 30.0, 10.0, 40.0,
                         [(t[0], t[1]) for t in tx], 15.0, 2.0)
    b = _Builder()
    ex, ey, ez = np.eye(3)
    for (x0, y0, x1, y1, h) in boxes:
        sx, sy = x1 - x0, y1 - y0
        # wall normals are u x v: choose axes so the normal points outward.
        b.rect_plane([x0, y0, 0.0], ex, ez, sx, h)  # y = y0, normal ex x ez = -y
        b.rect_plane([x1, y0, 0.0], ey, ez, sy, h)  # x = x1, normal ey x ez = +x
        b.rect_plane([x0, y1, 0.0], ez, ex, h, sx)  # y = y1, normal ez x ex = +y
        b.rect_plane([x0, y0, 0.0], ez, ey, h, sy)  # x = x0, normal ez x ey = -x
    b.rect_plane([-half_extent, -half_extent, 0.0], ex, ey, 2 * half_extent, 2 * half_extent)
    for (x0, y0, x1, y1, h) in boxes:
        # each corner edge: a1, a2 = outward normals of the two adjacent walls
        for (cx, cy, a1, a2) in ((x0, y0, -ey, -ex), (x1, y0, -ey, ex), (x1, y1, ey, ex),
                                 (x0, y1, ey, -ex)):
            b.line_edge([cx, cy, 0.0], ez, 0.0, h, a1, a2)
    for (x0, y0, x1, y1, h) in boxes:
        b.occ_rect([x0, y0, h], ex, ey, x1 - x0, y1 - y0)
    g = np.linspace(-rx_half, rx_half, rx_grid)
    rx = np.array([[x, y, rx_z] for y in g for x in g])
    return b.build(name, 100.0, tx, rx, meta={"seed": seed, "boxes": boxes})


def urban_block(n_rx_side: int = 32) -> Scene:
    """12-box city, seed 0, TX (0,0,30), n_rx_side^2 RX at 1.5 m: 97 objects
    (48 walls, ground, 48 edges), 61 occluders (48 walls, ground, 12 roofs)."""
    return box_city(0, 12, [[0.0, 0.0, 30.0]], n_rx_side, name=f"urban_block_{n_rx_side}x{n_rx_side}")


def mixed_order_city() -> Scene:
    """6-box city, seed 1, 4 TX at (+-40, +-40, 30) and 16x16 RX: 49 objects."""
    tx = [[-40.0, -40.0, 30.0], [40.0, -40.0, 30.0], [-40.0, 40.0, 30.0], [40.0, 40.0, 30.0]]
    return box_city(1, 6, tx, 16, name="mixed_order_city")


# ---------------------------------------------------------------------------
# Curved geometry: paraboloid mirrors, arc edges, randomly posed walls.
# ---------------------------------------------------------------------------

def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def curved_scene(seed: int = 2, n_pairs: int = 4096, n_parab: int = 8, n_arc: int = 8,
                 n_wall: int = 16, half: float = 25.0) -> Scene:
    """Curved-geometry study: n_parab paraboloid mirrors (f ~ U[0.5,5] m, disc
    radius 2 m, uniform random rigid pose), n_arc circular-arc edges (radius
    U[1,4] m, angular extent U[pi/4, pi]), n_wall randomly posed rectangles
    (sides U[5,20] m); all placed in [-half, half]^3; n_pairs zipped TX/RX
    pairs uniform in the same cube.  Objects: walls, then paraboloids, then arcs."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    for _ in range(n_wall):
        R = _random_rotation(rng)
        U, V = rng.uniform(5.0, 20.0, size=2)
        c = rng.uniform(-half, half, size=3)
        O = c - 0.5 * U * R[:, 0] - 0.5 * V * R[:, 1]
        b.rect_plane(O, R[:, 0], R[:, 1], U, V)
    for _ in range(n_parab):
        R = _random_rotation(rng)
        f = rng.uniform(0.5, 5.0)
        t = rng.uniform(-half, half, size=3)
        b.paraboloid(R, t, f, 2.0)
    for _ in range(n_arc):
        R = _random_rotation(rng)
        Rc = rng.uniform(1.0, 4.0)
        C = rng.uniform(-half, half, size=3)
        ext = rng.uniform(math.pi / 4, math.pi)
        phi0 = rng.uniform(-math.pi, math.pi)
        b.arc_edge(C, R[:, 2], Rc, R[:, 0], phi0, phi0 + ext)
    tx = rng.uniform(-half, half, size=(n_pairs, 3))
    rx = rng.uniform(-half, half, size=(n_pairs, 3))
    return b.build("curved", 100.0, tx, rx, pair_mode=1, meta={"seed": seed})


# ---------------------------------------------------------------------------
# Candidate-sequence specifications (consumed by both enumerators).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SequenceSpec:
    """Which ordered simple sequences of objects to solve.

    quota[n-1] for order n: -1 = every ordered sequence of n distinct objects
    (Algorithm 1, all_simple_paths); 0 = none; q > 0 = q sequences drawn with
    the counter-based SplitMix64 rule documented with the enumerators.
    ``starts_curved``: number of initial guesses for sequences that contain a
    paraboloid or an arc (1 for everything else).
    ``force_edges_every``: for orders >= 3, every k-th drawn slot forces two
    consecutive edges (0 disables).
    """

    quota: tuple = (-1, -1, 0, 0)
    seed: int = 0
    starts_curved: int = 1
    force_edges_every: int = 0

    def as_array(self) -> np.ndarray:
        q = list(self.quota) + [0] * (4 - len(self.quota))
        return np.asarray(q[:4], np.int64)


CONFIG_SPECS = {
    "street_canyon": SequenceSpec(quota=(-1, -1, 0, 0)),
    "urban_block": SequenceSpec(quota=(-1, -1, 0, 0)),
    "mixed_order": SequenceSpec(quota=(-1, 400, 800, 799), seed=11, force_edges_every=10),
    "curved": SequenceSpec(quota=(-1, 96, 128, 0), seed=12, starts_curved=8),
    "differentiable": SequenceSpec(quota=(-1, -1, 0, 0)),
}


def config_scene(name: str) -> Scene:
    if name == "street_canyon":
        return street_canyon()
    if name == "urban_block":
        return urban_block(32)
    if name == "mixed_order":
        return mixed_order_city()
    if name == "curved":
        return curved_scene()
    if name == "differentiable":
        return urban_block(64)
    raise KeyError(name)
