"""The minimiser's early exits lose no valid path.

Reading R15 ends a Gauss-Newton search early at a non-zero local minimum
(after two accepted steps, the model's predicted decrease below a fraction of
a large cost) and caps it at 24 accepted steps and 40 evaluations.  Those
rules set the valid-path set that the GPU is compared with, so they are
checked here against the same oracle with the local-minimum exit off and the
caps raised to 200 steps and 400 evaluations, on reduced versions of the
workloads: the valid sets must be identical (per candidate for planes and
straight edges; per TX/RX pair and sequence, over all starts, for curved
objects, where Sec. III-B makes every distinct root a path).
"""
import numpy as np
import pytest

import fullset as F
import oracle
from paper_2301_06399_gb300 import scenes as S


@pytest.fixture
def rules_restored():
    yield
    oracle.set_rules(**oracle.DEFAULT_RULES)


def _run(sc, table, **rules):
    oracle.set_rules(**rules)
    return oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)


def _valid_sets(sc, spec, max_order):
    table = oracle.enumerate_sequences(sc, max_order, spec)
    s0, v0 = _run(sc, table, **oracle.DEFAULT_RULES)
    s1, v1 = _run(sc, table, max_iters=200, max_evals=400, min_alpha=1.0 / 16.0, localmin_exit=False)
    oracle.set_rules(**oracle.DEFAULT_RULES)
    return table, (s0, v0), (s1, v1)


@pytest.mark.parametrize("name", ["urban_block_8x8rx", "mixed_orders_1tx_64rx"])
def test_early_exits_keep_every_valid_candidate(name, rules_restored):
    if name == "urban_block_8x8rx":
        sc, spec, mo = S.urban_block(8), S.CONFIG_SPECS["urban_block"], 2
    else:
        sc = S.mixed_order_city()
        sc.tx = sc.tx[:1].copy()
        sc.rx = np.ascontiguousarray(sc.rx[::4])
        sc, spec, mo = sc.contiguous(), S.CONFIG_SPECS["mixed_order"], 4
    table, (s0, v0), (s1, v1) = _valid_sets(sc, spec, mo)
    a = (v0.valid > 0) & (v0.ambiguous == 0)
    b = (v1.valid > 0) & (v1.ambiguous == 0)
    amb = (v0.ambiguous > 0) | (v1.ambiguous > 0)
    differ = np.nonzero((a != b) & ~amb)[0]
    print(f"{name}: {len(a)} candidates, {int(a.sum())} valid with the early exits, {int(b.sum())} without; "
          f"mean accepted steps {s0.iters.mean():.2f} vs {s1.iters.mean():.2f}")
    assert len(differ) == 0, [(int(c), table.ids[c // sc.n_pairs].tolist()) for c in differ[:10]]
    assert a.sum() > 1000
    both = np.nonzero(a & b)[0]
    assert np.abs(s0.X[both] - s1.X[both]).max() < 1e-8


def test_early_exits_keep_every_curved_root(rules_restored):
    """Curved scene, 256 pairs, 8 starts: the local-minimum exit stops some
    starts on a plateau (cost near 4, the direction reversed) that would
    reach a root, but another start finds the same root, so the root set of
    every (pair, sequence) is the same with and without the early exits."""
    sc = S.curved_scene(n_pairs=256)
    table, (s0, v0), (s1, v1) = _valid_sets(sc, S.CONFIG_SPECS["curved"], 3)
    ref = F.Report()
    ok = (v1.valid > 0) & (v1.ambiguous == 0)
    amb = v1.ambiguous > 0
    ref.valid_idx, ref.valid_X = np.nonzero(ok)[0], s1.X[ok]
    ref.amb_idx, ref.amb_X = np.nonzero(amb)[0], s1.X[amb]
    tested = F.GpuSide(np.nonzero(v0.valid > 0)[0].astype(np.int64), s0.X[v0.valid > 0])
    n_groups, diffs = F.root_set_differences(sc, table, tested, ref)
    print(f"curved: {n_groups} (pair, sequence) groups, {int(ok.sum())} valid without the early exits, "
          f"{int((v0.valid > 0).sum())} with")
    assert n_groups > 1000 and not diffs, diffs[:5]
