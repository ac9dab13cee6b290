"""Whole-workload parity of the GPU path with the FP64 oracle, at the full
sizes of every workload, in the launch configurations the benchmark times.

Bar (Algorithm 1, "C < threshold and X is valid"): the GPU's valid set equals
the oracle's on every candidate the oracle does not flag as ambiguous, and
interaction points agree within 1e-6 m.  For curved sequences solved from
several starts (Sec. III-B) the bar is per (TX/RX pair, object sequence): the
sets of distinct valid roots over all starts are identical.  Each test also
prints the FP32-only point error against the oracle (the same solver without
the refinement, accepted at a looser cost), reported, not a pass criterion.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_06399_gb300 import scenes as S
import fullset as F

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


def _trace(mpt, ds, max_order, spec, precision, schedule=None):
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    sols = mpt.solve(ds, cands, precision, schedule, keep_fp32=True)
    paths = mpt.validate(ds, cands, sols, capacity=1 << 22)
    torch.cuda.synchronize()
    assert paths.n() < paths.capacity
    return cands, sols, paths


def _check_full_set(mpt, ctx, sc, spec, max_order, label, schedule=None):
    ds = mpt.DeviceScene(ctx, sc)
    cands, sols, paths = _trace(mpt, ds, max_order, spec, mpt.FP32_FP64REFINE, schedule)
    assert ctx.check() == 0
    table = oracle.enumerate_sequences(sc, max_order, spec)
    assert int(cands.count.item()) == len(table) * sc.n_pairs
    gpu = F.gpu_side(paths, sols)
    rep = F.compare_workload(sc, table, gpu, keep_sets=True)
    err32 = F.fp32_point_error(sc, table, rep, sols.T32.cpu().numpy())
    print(f"\nPER-CONFIG {label}: {rep.summary()}; FP32-only max point error {err32:.2e} m")
    assert rep.ok(), rep.summary()
    return ds, cands, sols, paths, table, rep


def test_urban_block_every_candidate(mpt, ctx):
    """The benchmark workload: 9,634,816 candidates, every one compared."""
    sc = S.urban_block(32)
    _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["urban_block"], 2, "urban_block_32x32rx_order2")


@pytest.mark.parametrize("mixed", [0, 1])
def test_mixed_orders_every_candidate(mpt, ctx, mixed):
    """Orders 1-4 mixed (2,097,152 candidates, consecutive edge diffractions
    included), per-order launches and the single persistent launch over
    every order, each compared with the oracle candidate by candidate."""
    sc = S.mixed_order_city()
    sched = mpt.schedule_struct(mixed_orders=mixed)
    _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["mixed_order"], 4,
                    f"mixed_orders_{'single_launch' if mixed else 'per_order'}", sched)


def test_curved_root_sets_at_full_size(mpt, ctx):
    """Paraboloids, arcs and posed rectangles, 4,096 TX/RX pairs, orders 1-3,
    8 starts for curved sequences: for every (pair, sequence) the sets of
    distinct valid roots of the GPU and of the oracle are identical."""
    sc = S.curved_scene(n_pairs=4096)
    spec = S.CONFIG_SPECS["curved"]
    ds = mpt.DeviceScene(ctx, sc)
    cands, sols, paths = _trace(mpt, ds, 3, spec, mpt.FP32_FP64REFINE)
    table = oracle.enumerate_sequences(sc, 3, spec)
    gpu = F.gpu_side(paths, sols)
    rep = F.compare_workload(sc, table, gpu, keep_sets=True)
    n_groups, diffs = F.root_set_differences(sc, table, gpu, rep)
    # FP32-only error over the candidates whose start reaches the oracle's root
    same = np.intersect1d(rep.valid_idx, gpu.cand)
    keep = np.isin(rep.valid_idx, same)
    sub = F.Report(valid_idx=rep.valid_idx[keep], valid_X=rep.valid_X[keep])
    err32 = F.fp32_point_error(sc, table, sub, sols.T32.cpu().numpy())
    print(f"\nPER-CONFIG curved_4096pairs_order3: {rep.summary()}; root-set groups {n_groups}, differing "
          f"{len(diffs)}; FP32-only max point error {err32:.2e} m")
    for d in diffs[:20]:
        print("  root-set difference:", d)
    assert not diffs


def test_differentiable_block_every_candidate_and_adjoint(mpt, ctx):
    """The urban block with 64x64 RX (38,539,264 candidates): valid set
    against the oracle, then the adjoint of the valid paths (length and point
    weights) against the oracle's implicit-function-theorem gradient
    evaluated at the GPU's converged parameters, summed per TX, RX and plane."""
    sc = S.urban_block(64)
    ds, cands, sols, paths, table, rep = _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["differentiable"], 2,
                                                         "differentiable_64x64rx_order2")
    n = paths.n()
    rng = np.random.default_rng(4)
    g_len = torch.as_tensor(rng.uniform(0.5, 1.5, paths.capacity)).cuda()
    g_pts = torch.as_tensor(rng.normal(size=(12, paths.capacity)) * 0.1).cuda()
    cand = paths.cand[:n].cpu().numpy()
    T = oracle.pack_params(sc, table, cand, paths.T[:, :n].cpu().numpy().T)
    for with_pts in (False, True):
        gtx, grx, gobj = mpt.grad(ds, cands, paths, g_len, g_pts if with_pts else None)
        torch.cuda.synchronize()
        wtx, wrx, wobj = oracle.grad_sums(sc, table, cand, T, g_len[:n].cpu().numpy(),
                                          g_pts[:, :n].cpu().numpy().T if with_pts else None)
        planes = sc.obj_kind == 0
        e_tx = np.abs(gtx.cpu().numpy() - wtx).max() / max(1.0, np.abs(wtx).max())
        e_rx = np.abs(grx.cpu().numpy() - wrx).max() / max(1.0, np.abs(wrx).max())
        e_obj = np.abs(gobj.cpu().numpy()[planes] - wobj[planes]).max() / max(1.0, np.abs(wobj).max())
        print(f"adjoint over {n} paths ({'length and point' if with_pts else 'length'} weights): relative error "
              f"TX {e_tx:.1e}, RX {e_rx:.1e}, plane offsets {e_obj:.1e}")
        assert e_tx < 1e-6 and e_rx < 1e-6 and e_obj < 1e-6
