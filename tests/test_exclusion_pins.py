"""The solver's exclusion of candidates by two conditions of Eq. 8 removes
no path.

Eq. 8 makes the outgoing direction of a reflection r = i - 2 <i, n> n, so
<r, n> = -<i, n> and r is the direction from the mirror image of the
previous point through the reflection point.  Hence (half-space) the
segment after a reflection leaves on the side of the plane that the segment
before it came from, and (beam) after the first reflection the next point
lies in the pyramid from TX's mirror image through the reflecting rectangle
(backwards from RX for the last reflection).  The solver skips a candidate
that fails either with a margin (tests/fullset.exclusion_mask states them):
with every point inside its object's bounds its cost cannot fall below
about (1e-5 S / L)^2 ~ 1e-11 for path legs L of a few hundred metres.  The
oracle does not use the conditions, so it checks them: on reduced versions
of the workloads, no candidate the oracle accepts is excluded, the excluded
candidates that the oracle drives to a zero cost (on the unbounded planes
and lines of the parametrisation) have a point outside its object's
bounds, and the exclusion is not empty.
"""
import numpy as np
import pytest

import fullset as F
import oracle
from paper_2301_06399_gb300 import scenes as S


def _reduced(name):
    if name == "urban_block_8x8rx":
        return S.urban_block(8), S.CONFIG_SPECS["urban_block"], 2
    if name == "mixed_orders_1tx_64rx":
        sc = S.mixed_order_city()
        sc.tx = sc.tx[:1].copy()
        sc.rx = np.ascontiguousarray(sc.rx[::4])
        return sc.contiguous(), S.CONFIG_SPECS["mixed_order"], 4
    return S.curved_scene(n_pairs=256), S.CONFIG_SPECS["curved"], 3


def _outside(sc, i, s, t, tol=1e-6):
    """Parameters (s, t) of object i outside its bounds by more than tol
    (metres; parameters of planes, lines and paraboloids are lengths, an
    arc's is an angle, taken over its radius)."""
    p = np.asarray(sc.obj_param[i], np.float64)
    kind = int(sc.obj_kind[i])
    if kind == 0:
        return s < -tol or s > p[13] + tol or t < -tol or t > p[14] + tol
    if kind == 2:
        return s < p[6] - tol or s > p[7] + tol
    if kind == 1:
        return np.hypot(s, t) > p[13] + tol
    d = (s - p[10]) % (2.0 * np.pi)
    return d > (p[11] - p[10]) + tol / p[6] and d < 2.0 * np.pi - tol / p[6]


@pytest.mark.parametrize("name", ["urban_block_8x8rx", "mixed_orders_1tx_64rx", "curved_256pairs"])
def test_excluded_candidates_have_no_path(name):
    sc, spec, mo = _reduced(name)
    table = oracle.enumerate_sequences(sc, mo, spec)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    ex = F.exclusion_mask(sc, table)
    assert len(ex) == len(sol.cost)
    valid = ver.valid > 0
    print(f"{name}: {len(ex)} candidates, {int(ex.sum())} excluded, {int(valid.sum())} oracle-valid, "
          f"{int((ex & (ver.ambiguous > 0)).sum())} excluded and ambiguous")
    assert not np.any(ex & valid), np.nonzero(ex & valid)[0][:10]
    # a zero cost is reached only on the unbounded surfaces, with a point
    # outside its object's bounds (the condition holds for bounded objects)
    zero = np.nonzero(ex & np.isfinite(sol.cost) & (sol.cost < 1e-12))[0]
    for c in zero:
        e = c // sc.n_pairs
        ids = [int(i) for i in table.ids[e][:int(table.order[e])]]
        # the oracle's parameters are packed: one per edge, two per surface
        q, out = 0, False
        for i in ids:
            edge = int(sc.obj_kind[i]) in (2, 3)
            out = out or _outside(sc, i, sol.T[c, q], 0.0 if edge else sol.T[c, q + 1])
            q += 1 if edge else 2
        assert out, c
    print(f"  {len(zero)} excluded candidates reach a zero cost outside their objects' bounds")
    assert ex.mean() > 0.3


def test_single_reflection_across_a_plane_is_excluded_and_has_no_path():
    """TX and RX on opposite sides of one plane: the only candidate is
    excluded, and the oracle finds no path for it."""
    sc = S.street_canyon()
    sc.tx = np.array([[0.0, -5.0, 10.0]])
    sc.rx = np.array([[0.0, 15.0, 1.5]])  # beyond the wall y = +10
    sc = sc.contiguous()
    spec = S.SequenceSpec(quota=(-1, 0, 0, 0))
    table = oracle.enumerate_sequences(sc, 1, spec)
    ex = F.exclusion_mask(sc, table)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    ids = [int(table.ids[e][0]) for e in range(len(table))]
    # the wall y = +10 (normal along y, origin at y = 10) separates TX and RX
    wall = [e for e, i in enumerate(ids) if abs(abs(sc.obj_param[i][1]) - 1.0) < 1e-12 and sc.obj_param[i][5] == 10.0]
    assert len(wall) == 1
    assert ex[wall[0]] and not ver.valid[wall[0]]
    assert not np.isfinite(sol.cost[wall[0]]) or sol.cost[wall[0]] > 1e-6


@pytest.mark.parametrize("x_rx,expect_path", [(40.0, True), (80.0, False)])
def test_beam_condition_on_a_single_wall_agrees_with_the_image_method(x_rx, expect_path):
    """Street canyon, order 1, the wall y = +10 (x in [-50, 50]): TX (0, -5,
    10) and RX (x_rx, 5, 10), both on its inner side.  The image method
    (Eqs. 5-6) puts the reflection point where the segment from TX's image
    (0, 25, 10) to RX crosses y = 10: x = 0.75 x_rx, 30 m for RX at 40 m
    (inside the wall: a path) and 60 m for RX at 80 m (outside: no path).
    The half-space test keeps both (same side); the beam test excludes
    exactly the second, as the image method and the oracle decide."""
    sc = S.street_canyon()
    sc.tx = np.array([[0.0, -5.0, 10.0]])
    sc.rx = np.array([[x_rx, 5.0, 10.0]])
    sc = sc.contiguous()
    table = oracle.enumerate_sequences(sc, 1, S.SequenceSpec(quota=(-1, 0, 0, 0)))
    ex = F.exclusion_mask(sc, table)
    half = F.exclusion_mask(sc, table, beam=False)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    wall = [e for e in range(len(table))
            if abs(abs(sc.obj_param[int(table.ids[e][0])][1]) - 1.0) < 1e-12
            and sc.obj_param[int(table.ids[e][0])][5] == 10.0]
    assert len(wall) == 1
    e = wall[0]
    crossing = 0.75 * x_rx  # the image-method reflection point's x
    assert (abs(crossing) <= 50.0) == expect_path
    assert not half[e]
    assert bool(ex[e]) == (not expect_path)
    assert bool(ver.valid[e]) == expect_path
