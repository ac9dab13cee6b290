"""Pins of the oracle's received field (Sec. V, Eqs. 16-19, scalar form).

For reflections alone the spreading factors r/(r+s) of Eq. 17 telescope to
the field of the image source, E0 coef^n e^{-jkL} / L with L the distance
from the image of the TX to the RX: checked against that closed form for one
reflection on a floor and two reflections in a corridor.  A single
diffraction (Eq. 18) is reciprocal: swapping TX and RX gives the same
field."""
import numpy as np

import oracle as O
from paper_2301_06399_gb300 import scenes as S

K = 2 * np.pi / 0.3  # 1 GHz
SPEC = S.SequenceSpec(quota=(-1, -1, 0, 0))


def _field_of(sc, entry_ids=None, refl=-1.0, diff=1.0):
    table = O.enumerate_sequences(sc, 2, SPEC)
    sol, ver = O.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    if entry_ids is not None:
        keep = np.zeros_like(ver.valid)
        for e in range(len(table)):
            n = int(table.order[e])
            if tuple(int(x) for x in table.ids[e][:n]) == tuple(entry_ids):
                keep[e * sc.n_pairs:(e + 1) * sc.n_pairs] = ver.valid[e * sc.n_pairs:(e + 1) * sc.n_pairs]
        ver = O.Verdicts(keep, ver.ambiguous, ver.length)
    return O.path_field(sc, table, sol, ver, K, 1.0, refl, diff), ver


def test_single_reflection_is_the_image_source():
    b = S._Builder()
    ex, ey, ez = np.eye(3)
    b.rect_plane([-50, -50, 0], ex, ey, 100, 100)  # floor, normal +z
    tx, rx = np.array([0.0, 0.0, 10.0]), np.array([20.0, 0.0, 5.0])
    sc = b.build("floor", 100.0, [tx], [rx])
    f, ver = _field_of(sc)
    assert int(ver.valid.sum()) == 1
    d = np.linalg.norm(rx - np.array([0.0, 0.0, -10.0]))
    want = -np.exp(-1j * K * d) / d
    assert abs(f[0] - want) < 1e-12 * abs(want)


def test_double_reflection_is_the_twice_mirrored_source():
    b = S._Builder()
    ex, ey, ez = np.eye(3)
    a = b.rect_plane([-10, 0, -10], ez, ex, 30, 60)   # y = 0, normal ez x ex = +y
    c = b.rect_plane([-10, 10, -10], ex, ez, 60, 30)  # y = 10, normal ex x ez = -y
    tx, rx = np.array([0.0, 2.0, 1.0]), np.array([30.0, 7.0, 1.0])
    sc = b.build("corridor", 100.0, [tx], [rx])
    f, ver = _field_of(sc, entry_ids=(a, c))
    assert int(ver.valid.sum()) == 1
    image = np.array([0.0, 22.0, 1.0])  # TX mirrored in y = 0, then in y = 10
    L = np.linalg.norm(rx - image)
    want = (-1.0) ** 2 * np.exp(-1j * K * L) / L
    assert abs(f[0] - want) < 1e-12 * abs(want)


def test_single_diffraction_is_reciprocal():
    ex, ey, ez = np.eye(3)

    def scene(tx, rx):
        b = S._Builder()
        b.line_edge([0, 0, 0], ez, 0.0, 20.0, -ey, -ex)
        return b.build("edge", 100.0, [tx], [rx])

    tx, rx = np.array([10.0, -5.0, 3.0]), np.array([-8.0, 6.0, 9.0])
    f1, v1 = _field_of(scene(tx, rx), diff=0.3 - 0.2j)
    f2, v2 = _field_of(scene(rx, tx), diff=0.3 - 0.2j)
    assert int(v1.valid.sum()) == 1 and int(v2.valid.sum()) == 1
    assert abs(f1[0] - f2[0]) < 1e-12 * abs(f1[0])
