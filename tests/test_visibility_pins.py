"""Pins of the oracle's visibility matrix (Algorithm 1, its first line;
Sec. III, Fig. 5) on small scenes whose answer follows from the geometry
alone: facets that face each other see each other, facets back to back do
not, the opposite walls of one box do not, adjacent walls (sharing an edge,
so not strictly behind each other) do, and the matrix is symmetric with an
empty diagonal."""
import numpy as np

import oracle as O
from paper_2301_06399_gb300 import scenes as S


def _facets():
    b = S._Builder()
    ex, ey, ez = np.eye(3)
    # two 10 x 10 facets at y = 0 and y = 20; normal u x v
    a = b.rect_plane([0, 0, 0], ex, ez, 10, 10)          # normal ex x ez = -y (faces y < 0)
    f = b.rect_plane([0, 20, 0], ez, ex, 10, 10)         # normal ez x ex = +y (faces y > 20)
    c = b.rect_plane([0, 30, 0], ex, ez, 10, 10)         # normal -y: faces the facet at y = 20
    e = b.line_edge([5, 25, 0], ez, 0, 10, -ey, ey)      # between f and c
    return b.build("facets", 100.0, [[5, 10, 5]], [[5, 40, 5]]), (a, f, c, e)


def test_facing_back_to_back_and_edges():
    sc, (a, f, c, e) = _facets()
    V = O.visibility_matrix(sc)
    assert (np.diag(V) == 0).all() and (V == V.T).all()
    # a faces -y, f faces +y from y = 20: each lies behind the other
    assert V[a, f] == 0
    # f (y = 20, normal +y) and c (y = 30, normal -y) face each other
    assert V[f, c] == 1
    # a (y = 0, normal -y): c at y = 30 is behind a
    assert V[a, c] == 0
    # the edge at y = 25 is in front of f and of c, behind a
    assert V[f, e] == 1 and V[c, e] == 1 and V[a, e] == 0


def test_one_box():
    sc = S.box_city(3, 1, [[0, 0, 30]], 2)
    V = O.visibility_matrix(sc)
    walls = [i for i in range(4)]
    # walls in the order -y, +x, +y, -x: opposite pairs (0, 2), (1, 3)
    assert V[walls[0], walls[2]] == 0 and V[walls[1], walls[3]] == 0
    # adjacent walls share an edge (distance 0, not strictly behind)
    assert V[walls[0], walls[1]] == 1 and V[walls[1], walls[2]] == 1
    # the ground (index 4, normal +z) sees every wall and the walls see it
    assert all(V[4, w] == 1 and V[w, 4] == 1 for w in walls)
