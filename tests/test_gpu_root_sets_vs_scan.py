"""The CUDA path's curved root sets against the independent reference.

The CPU pins (test_oracle_curved_mixed.py, test_oracle_curved_order2.py)
compare the oracle's valid solutions with the stationary points of the path
length found by a dense scan (Fermat's principle; Eq. 8 and Eq. 9 checked
at every point).  Here the same seeded instances go through the CUDA path
(enumerate, FP32 solve with float-float refinement, validate) and its valid
paths, sequence by sequence, are compared with that reference directly:
with 255 starts (the most a candidate record holds; on these instances the
oracle finds every reference root with them) the sets are equal; with 8
starts every GPU root is a reference root.  Points within
1 mm of a bound and paths with a segment within a factor 3 of the minimum
length are left out on both sides, as in the CPU pins.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_06399_gb300 import scenes as S

import test_oracle_curved_mixed as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpt():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_06399_gb300 import mpt as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return m


@pytest.fixture(scope="module")
def ctx(mpt):
    return mpt.Context(0)


def _gpu_sets(mpt, ctx, sc, objs, order, starts, A, B):
    q = [0, 0, 0, 0]
    q[order - 1] = -1
    spec = S.SequenceSpec(quota=tuple(q), starts_curved=starts)
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, order, spec)
    sols = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
    paths = mpt.validate(ds, cands, sols, capacity=cands.capacity)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    table = oracle.enumerate_sequences(sc, order, spec)  # bit-exact with the GPU's table
    n = paths.n()
    cand = paths.cand[:n].cpu().numpy()
    X = paths.X[:, :n].cpu().numpy().T
    sets = {}
    for i, c in enumerate(cand):
        ids = tuple(int(v) for v in table.ids[int(c) // sc.n_pairs][:order])
        pts = [X[i, 3 * k:3 * k + 3] for k in range(order)]
        if not M._kept([objs[j] for j in ids], A, B, pts):
            continue
        x = np.concatenate(pts)
        found = sets.setdefault(ids, [])
        if not any(np.linalg.norm(x - y) < 1e-6 for y in found):
            found.append(x)
    return sets


CASES = [
    (M.flat_lid_over_bowl, 8, 2, 21),
    (M.arc_over_ground, 8, 2, 22),
    (M.edge_over_bowl, 8, 2, 26),
    (M.two_arcs, 8, 2, 23),
    (M.bowl_rim_and_lid, 2, 3, 24),
    (M.bowl_edge_and_lid, 2, 3, 27),
]


@pytest.mark.parametrize("family,n_inst,order,seed", CASES, ids=[c[0].__name__ for c in CASES])
def test_gpu_root_sets_equal_the_scan(mpt, ctx, family, n_inst, order, seed):
    rng = np.random.default_rng(seed)  # the CPU pin's first instances
    most = 255
    n_roots = 0
    for _ in range(n_inst):
        objs, A, B = family(rng)
        sc = M._build(objs, A, B)
        seqs = ([(0, 1), (1, 0)] if order == 2 else
                [(0, 1, 2), (2, 1, 0), (1, 0, 2), (0, 2, 1), (2, 0, 1), (1, 2, 0)])
        grid = 24 if family is M.two_arcs else (8 if order == 2 else 5)
        refs = {seq: M._reference_roots([objs[i] for i in seq], A, B, grid) for seq in seqs}
        for starts in (8, most):
            sets = _gpu_sets(mpt, ctx, sc, objs, order, starts, A, B)
            for seq, ref in refs.items():
                missed, extra = M._same(ref, sets.get(seq, []))
                assert not extra, ("a GPU root that is not a path", family.__name__, seq, starts, extra)
                if starts == most:
                    assert not missed, ("roots the GPU missed", family.__name__, seq, starts, missed)
        n_roots += sum(len(r) for r in refs.values())
    print(f"{family.__name__}: {n_roots} reference roots, GPU sets equal with {most} starts")
    assert n_roots >= 4
