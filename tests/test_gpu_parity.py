"""GPU path (through the C ABI) against the FP64 CPU oracle.

Bar: bit-exact candidate records; identical valid-path sets on every
candidate the oracle does not flag as ambiguous (tolerance bands of the
acceptance rules); interaction points within 1e-6 m of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_06399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

POINT_TOL = 1e-6  # metres, FP64-refined points vs the oracle


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


def expand_oracle(table, n_pairs):
    E = len(table)
    pair = np.tile(np.arange(n_pairs), E)
    ids = np.repeat(table.ids, n_pairs, axis=0)
    order = np.repeat(table.order, n_pairs)
    start = np.repeat(table.start, n_pairs)
    return pair, ids, order, start


def gpu_trace(mpt, ctx, sc, max_order, spec, precision=None, schedule=None, keep_fp32=False, path_cap=None):
    ds = mpt.DeviceScene(ctx, sc)
    prec = mpt.FP32_FP64REFINE if precision is None else precision
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    sols = mpt.solve(ds, cands, prec, schedule, keep_fp32=keep_fp32)
    cap = path_cap if path_cap is not None else cands.capacity
    paths = mpt.validate(ds, cands, sols, capacity=cap)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return ds, cands, sols, paths


def compare_entries(sc, table, paths, entries, n_pairs):
    """Oracle on whole entries (one object sequence x every pair) vs GPU."""
    n = paths.n()
    gcand = paths.cand[:n].cpu().numpy()
    gX = paths.X[:, :n].cpu().numpy().T
    gpos = {int(c): i for i, c in enumerate(gcand)}
    n_valid = n_amb = n_amb_gpu = 0
    max_err = 0.0
    for e in entries:
        b, en = int(e) * n_pairs, (int(e) + 1) * n_pairs
        sol, ver = oracle.candidate_range(sc, table, b, en)
        for i in range(en - b):
            c = b + i
            if ver.ambiguous[i]:
                n_amb += 1
                n_amb_gpu += c in gpos
                continue
            want = bool(ver.valid[i])
            got = c in gpos
            assert want == got, f"candidate {c} (entry {e}, ids {table.ids[e]}): oracle {want}, gpu {got}, " \
                                f"oracle cost {sol.cost[i]:.3e}"
            if want:
                n_valid += 1
                k = 3 * int(table.order[e])
                err = np.abs(gX[gpos[c], :k] - sol.X[i, :k]).max()
                max_err = max(max_err, err)
    assert max_err < POINT_TOL, max_err
    return n_valid, n_amb, max_err, n_amb_gpu


# ------------------------------------------------------------ enumeration --
@pytest.mark.parametrize("name,max_order", [("street_canyon", 2), ("mixed_order", 4), ("curved", 3)])
def test_enumeration_bit_exact(mpt, ctx, name, max_order):
    sc = S.config_scene(name)
    spec = S.CONFIG_SPECS[name]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, max_order, spec)
    n = int(cands.count.item())
    assert n == len(table) * sc.n_pairs == cands.capacity
    pair, ids, order, start = mpt.decode_candidates(cands, n)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(pair, p2) and np.array_equal(ids, i2)
    assert np.array_equal(order, o2) and np.array_equal(start, s2)
    ob = cands.order_begin.cpu().numpy()
    for k in range(1, 5):
        first = np.nonzero(o2 >= k)[0]
        assert ob[k - 1] == (first[0] if len(first) else n)
    assert ob[4] == n


def test_enumeration_urban_block_entries(mpt, ctx):
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, spec)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec)
    pair, ids, order, start = mpt.decode_candidates(cands)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(ids, i2) and np.array_equal(pair, p2) and np.array_equal(order, o2)


def test_enumeration_adjacency_mask(mpt, ctx):
    sc = S.urban_block(2)
    rng = np.random.default_rng(3)
    adj = (rng.uniform(size=(sc.n_obj, sc.n_obj)) < 0.3).astype(np.uint8)
    spec = S.SequenceSpec(quota=(-1, -1, 0, 0))
    ds = mpt.DeviceScene(ctx, sc)
    cap = mpt.candidate_count(ds, 2, spec)
    cands = mpt.enumerate_candidates(ds, 2, spec, adj=torch.as_tensor(adj).cuda(), capacity=cap)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec, adj=adj)
    n = int(cands.count.item())
    assert n == len(table) * sc.n_pairs
    pair, ids, order, start = mpt.decode_candidates(cands, n)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(ids, i2) and np.array_equal(pair, p2)


def test_enumeration_capacity_error(mpt, ctx):
    sc = S.street_canyon()
    ds = mpt.DeviceScene(ctx, sc)
    with pytest.raises(RuntimeError, match="CAPACITY"):
        mpt.enumerate_candidates(ds, 2, S.CONFIG_SPECS["street_canyon"], capacity=100)


def test_start_count_limit(mpt, ctx):
    """A candidate record holds the start index in 8 bits: 255 starts are
    accepted, 256 are an argument error of both the count and the
    enumeration, which enqueue nothing."""
    sc = S.curved_scene(n_pairs=4)
    ds = mpt.DeviceScene(ctx, sc)
    ok = S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=255)
    n = mpt.candidate_count(ds, 1, ok)
    n_curved = int(np.isin(sc.obj_kind, (S.PARABOLOID, S.ARC_EDGE)).sum())
    assert n == ((sc.n_obj - n_curved) + 255 * n_curved) * sc.n_pairs
    bad = S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=256)
    with pytest.raises(RuntimeError, match="bad arguments"):
        mpt.candidate_count(ds, 1, bad)
    with pytest.raises(RuntimeError, match="ARG"):
        mpt.enumerate_candidates(ds, 1, bad, capacity=n)
    assert ctx.check() == 0


# ------------------------------------------------------------------ Fig. 4 --
@pytest.mark.parametrize("prec", ["FP64_PLAIN", "FP32_FP64REFINE"])
def test_fig4_gpu_path(mpt, ctx, prec):
    sc = S.fig4_scene()
    spec = S.SequenceSpec(quota=(-1, -1, 0, 0))
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, getattr(mpt, prec))
    assert paths.n() == 1
    _, ids, _, _ = mpt.decode_candidates(cands)
    c = int(paths.cand[0].item())
    assert list(ids[c][:2]) == [0, 1]
    X = paths.X[:6, 0].cpu().numpy()
    assert np.allclose(X, [20 / 7, 20 / 7, 0, 5, 10 / 3, 0], atol=1e-9)
    assert abs(paths.length[0].item() - np.sqrt(85.0)) < 1e-9


# ---------------------------------------------------------- street canyon --
@pytest.mark.parametrize("prec", ["FP64_PLAIN", "FP32_FP64REFINE"])
def test_street_canyon_parity(mpt, ctx, prec):
    sc = S.street_canyon()
    spec = S.CONFIG_SPECS["street_canyon"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, getattr(mpt, prec))
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_valid, n_amb, err, n_amb_gpu = compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)
    assert n_valid == paths.n() and n_valid > 300
    print(f"canyon {prec}: {n_valid} valid, {n_amb} ambiguous, max err {err:.2e} m")


def test_street_canyon_ragged_pairs(mpt, ctx):
    """37 RX: tiles and warps straddle sequence boundaries."""
    sc = S.street_canyon()
    rng = np.random.default_rng(9)
    sc.rx = np.ascontiguousarray(np.c_[rng.uniform(-40, 40, 37), rng.uniform(-8, 8, 37), np.full(37, 1.5)])
    spec = S.CONFIG_SPECS["street_canyon"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    table = oracle.enumerate_sequences(sc, 2, spec)
    compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)


def test_validation_with_unaligned_status_buffer(mpt, ctx):
    """Caller buffers need no alignment: the same solutions validated with
    their status bytes at an odd address (the acceptance's flag pass then
    reads them one byte at a time) give the same valid paths."""
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    n = paths.n()
    raw = torch.zeros(sols.capacity + 8, dtype=torch.uint8, device="cuda")
    odd = raw[3:3 + sols.capacity]
    odd.copy_(sols.status)
    shifted = mpt.Solutions(sols.T, sols.cost, odd, sols.iters, sols.evals, sols.T32, sols.capacity)
    assert shifted.status.data_ptr() % 8 == 3
    p2 = mpt.validate(ds, cands, shifted, capacity=cands.capacity)
    torch.cuda.synchronize()
    assert p2.n() == n > 0
    assert torch.equal(p2.cand[:n], paths.cand[:n])
    assert torch.equal(p2.X[:, :n], paths.X[:, :n])


# ------------------------------------------------------------- urban block --
def test_urban_block_small_all_candidates(mpt, ctx):
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, keep_fp32=True)
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_valid, n_amb, err, n_amb_gpu = compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)
    # every GPU path is a compared candidate: an oracle-valid one or one the
    # oracle flags as ambiguous (either verdict allowed there)
    assert n_valid + n_amb_gpu == paths.n()
    print(f"urban 4x4: {n_valid} valid, {n_amb} ambiguous, max err {err:.2e} m")


def test_urban_block_full_size_adjoint(mpt, ctx):
    """The adjoint in the benchmark's launch configuration (length weights,
    157,792 paths): the accumulated dL/dTX, dL/dRX and plane-offset sums equal
    the explicit gradient written out in numpy from the returned FP64 points
    (-u_0 per path for TX, u_n for its RX, <u_m - u_m+1, n> for a reflection
    on plane m), a property that holds at any size."""
    sc = S.urban_block(32)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, path_cap=1 << 20)
    n = paths.n()
    g_len = torch.ones(paths.capacity, dtype=torch.float64, device="cuda")
    gtx, grx, gobj = mpt.grad(ds, cands, paths, g_len)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec)
    cand = paths.cand[:n].cpu().numpy()
    X = paths.X[:, :n].cpu().numpy().T
    ent, pair = np.divmod(cand, sc.n_pairs)
    order = table.order[ent]
    A = np.repeat(sc.tx[:1], n, 0)
    B = sc.rx[pair]
    def unit(v):
        with np.errstate(invalid="ignore", divide="ignore"):  # order-1 rows of u2 are unused
            return v / np.linalg.norm(v, axis=1, keepdims=True)

    P1 = X[:, 0:3]
    P2 = np.where((order == 2)[:, None], X[:, 3:6], B)
    u0, u1 = unit(P1 - A), unit(P2 - P1)
    u2 = unit(B - P2)
    want_tx = -u0.sum(0)
    last = np.where((order == 2)[:, None], u2, u1)
    want_rx = np.zeros_like(sc.rx)
    np.add.at(want_rx, pair, last)
    want_obj = np.zeros(sc.n_obj)
    planes = sc.obj_kind == 0
    for k, (ui, uo) in enumerate(((u0, u1), (u1, u2))):
        has = order > k
        ids = table.ids[ent[has], k]
        keep = planes[ids]
        nrm = sc.obj_param[ids[keep], 0:3]
        np.add.at(want_obj, ids[keep], ((ui[has][keep] - uo[has][keep]) * nrm).sum(1))
    assert n == 157792
    assert np.abs(gtx.cpu().numpy()[0] - want_tx).max() < 1e-9 * max(1.0, np.abs(want_tx).max())
    assert np.abs(grx.cpu().numpy() - want_rx).max() < 1e-9 * max(1.0, np.abs(want_rx).max())
    assert np.abs(gobj.cpu().numpy() - want_obj).max() < 1e-9 * max(1.0, np.abs(want_obj).max())


# ------------------------------------------------------------ mixed orders --
def test_mixed_orders_single_launch_matches_per_order(mpt, ctx):
    sc = S.mixed_order_city()
    spec = S.CONFIG_SPECS["mixed_order"]
    _, _, _, p1 = gpu_trace(mpt, ctx, sc, 4, spec, path_cap=1 << 20)
    sched = mpt.schedule_struct(mixed_orders=1)
    _, _, _, p2 = gpu_trace(mpt, ctx, sc, 4, spec, schedule=sched, path_cap=1 << 20)
    a = p1.cand[:p1.n()].cpu().numpy()
    b = p2.cand[:p2.n()].cpu().numpy()
    assert np.array_equal(a, b)
    assert torch.allclose(p1.X[:, :p1.n()], p2.X[:, :p2.n()], atol=1e-9, rtol=0)


@pytest.mark.parametrize("prec", ["FP32_FP64REFINE", "FP64_PLAIN"])
@pytest.mark.parametrize("name", ["urban_block", "mixed_order", "curved"])
def test_excluded_candidates_match_the_half_space_condition(mpt, ctx, name, prec):
    """The solver's MPT_PATH_EXCLUDED candidates (the half-space and beam
    conditions of Eq. 8, tested before iterating) against the conditions
    written with numpy in FP64 (fullset.exclusion_mask): the GPU set lies
    between the masks with every margin and threshold 10% smaller and 10%
    larger (the GPU tests in FP32), and is about two thirds of the
    candidates."""
    import fullset as F
    if name == "urban_block":
        sc, order = S.urban_block(32), 2
    elif name == "mixed_order":
        sc, order = S.mixed_order_city(), 4
    else:
        sc, order = S.curved_scene(), 3
    if prec == "FP64_PLAIN" and name != "mixed_order":
        pytest.skip("the plain FP64 method is checked on the mixed-order city")
    spec = S.CONFIG_SPECS[name]
    _, cands, sols, _ = gpu_trace(mpt, ctx, sc, order, spec, precision=getattr(mpt, prec), path_cap=1 << 21)
    n = int(cands.count.item())
    got = ((sols.status[:n] & 0x0F) == mpt.PATH_EXCLUDED).cpu().numpy()
    table = oracle.enumerate_sequences(sc, order, spec)
    wide = F.exclusion_mask(sc, table, m_tx=0.9e-5, m_obj=0.9e-6, m_beam=0.9e-5, h_min=0.9e-2)
    narrow = F.exclusion_mask(sc, table, m_tx=1.1e-5, m_obj=1.1e-6, m_beam=1.1e-5, h_min=1.1e-2)
    print(f"{name} {prec}: {int(got.sum())} of {n} excluded (numpy {int(narrow.sum())}..{int(wide.sum())})")
    assert not np.any(narrow & ~got), np.nonzero(narrow & ~got)[0][:10]
    assert not np.any(got & ~wide), np.nonzero(got & ~wide)[0][:10]
    assert got.mean() > 0.5
    assert np.all(np.isinf(sols.cost[:n].cpu().numpy()[got]))


@pytest.mark.parametrize("name", ["urban_block", "curved"])
def test_warp_fallback_equals_single_lane_fallback(mpt, ctx, name):
    """The refinement's fallback with its FP64 evaluation spread over a warp
    (the default) against the same Gauss-Newton on one lane: the same queued
    candidates, the same valid paths, points within 1e-9 m (J^T J is summed
    in another order)."""
    if name == "urban_block":
        sc, spec, order = S.urban_block(32), S.CONFIG_SPECS["urban_block"], 2
    else:
        sc, spec, order = S.curved_scene(), S.CONFIG_SPECS["curved"], 3
    _, _, s1, p1 = gpu_trace(mpt, ctx, sc, order, spec, path_cap=1 << 21)
    sched = mpt.schedule_struct(fallback=3)
    _, _, s2, p2 = gpu_trace(mpt, ctx, sc, order, spec, schedule=sched, path_cap=1 << 21)
    fb1 = (s1.status & mpt.PATH_FALLBACK) != 0
    fb2 = (s2.status & mpt.PATH_FALLBACK) != 0
    assert torch.equal(fb1, fb2)
    n_fb = int(fb1.sum().item())
    if name == "urban_block":
        assert n_fb >= 50, n_fb
    a = p1.cand[:p1.n()].cpu().numpy()
    b = p2.cand[:p2.n()].cpu().numpy()
    assert np.array_equal(a, b)
    assert torch.allclose(p1.X[:, :p1.n()], p2.X[:, :p2.n()], atol=1e-9, rtol=0)
    both = fb1 & torch.isfinite(s1.cost) & torch.isfinite(s2.cost) & (s1.cost < 1e-20) & (s2.cost < 1e-20)
    print(f"{name}: {n_fb} fallback candidates, {int(both.sum().item())} converged in both")


def test_cuda_graph_replay_matches_eager(mpt, ctx):
    sc = S.mixed_order_city()
    spec = S.CONFIG_SPECS["mixed_order"]
    ds = mpt.DeviceScene(ctx, sc)
    n = mpt.candidate_count(ds, 4, spec)
    dev = ds.tx.device
    cands = mpt.alloc_candidates(n, dev)
    sols = mpt.alloc_solutions(n, dev)
    paths = mpt.alloc_paths(1 << 20, dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        def step():
            mpt.enumerate_candidates(ds, 4, spec, out=cands, stream=s)
            mpt.solve(ds, cands, mpt.FP32_FP64REFINE, out=sols, stream=s)
            mpt.validate(ds, cands, sols, out=paths, stream=s)
        step()
        s.synchronize()
        eager = paths.cand[:paths.n()].clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            step()
        paths.count.zero_()
        g.replay()
        s.synchronize()
    assert torch.equal(paths.cand[:paths.n()], eager)


# ------------------------------------------------------------------ curved --
def _root_sets(Xs, tol=1e-4):
    roots = []
    for x in Xs:
        if not any(np.abs(x - r).max() < tol for r in roots):
            roots.append(x)
    return roots


def test_curved_geometry_gpu_paths_are_oracle_roots(mpt, ctx):
    """Paraboloids, arcs and posed rectangles with 8 starts for curved
    sequences: every GPU-valid path is a root of the oracle's own cost, and
    the oracle's point map of the GPU parameters gives the GPU's points.
    (Root sets are compared in full at 4,096 pairs by the full-size tests.)"""
    sc = S.curved_scene(n_pairs=512)
    spec = S.CONFIG_SPECS["curved"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 3, spec, path_cap=1 << 20)
    table = oracle.enumerate_sequences(sc, 3, spec)
    n = paths.n()
    assert n > 0
    gcand = paths.cand[:n].cpu().numpy()
    gT = paths.T[:, :n].cpu().numpy().T
    gX = paths.X[:, :n].cpu().numpy().T
    checked = 0
    for i, c in enumerate(gcand):
        e, p = divmod(int(c), sc.n_pairs)
        ids = table.ids[e][:table.order[e]]
        k = int(table.order[e])
        # repack GPU slots (edges use slot 2k) into the oracle's packed order
        tp = []
        for kk, o in enumerate(ids):
            tp.append(gT[i, 2 * kk])
            if sc.obj_kind[o] not in (2, 3):
                tp.append(gT[i, 2 * kk + 1])
        cst = oracle.cost(sc, ids, *sc.pair_points(p), tp)
        assert cst < oracle.TAU * 100, (c, cst)
        _, Xo = oracle.residual(sc, ids, *sc.pair_points(p), tp)
        assert np.abs(Xo - gX[i, :3 * k]).max() < 1e-9
        checked += 1
    print(f"curved: {checked} GPU-valid paths confirmed by the oracle's own cost and point map")


def test_deep_bowl_root_sets(mpt, ctx):
    """Order-1 reflections in deep paraboloid bowls with both ends inside
    (up to three reflection points per sequence): with 64 starts the GPU's
    distinct valid roots equal the oracle's (which the oracle pins equate to
    a dense scan of the path-length stationary points); with 8 starts every
    GPU root is one of them."""
    rng = np.random.default_rng(1)
    rho = 2.0
    n_roots = 0
    for _ in range(40):
        R = S._random_rotation(rng)
        t0 = rng.uniform(-3, 3, 3)
        f = rng.uniform(0.5, 1.2)
        A = t0 + R @ np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 2.0)])
        B = t0 + R @ np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 2.0)])
        b = S._Builder()
        b.paraboloid(R, t0, f, rho, occluder=False)
        sc = b.build("bowl", 100.0, A[None], B[None], pair_mode=1)

        def inside(x):
            loc = R.T @ (x - t0)
            return np.hypot(loc[0], loc[1]) < rho - 1e-3

        roots = {}
        for starts in (64, 8):
            spec = S.SequenceSpec(quota=(-1, 0, 0, 0), starts_curved=starts)
            _, _, _, paths = gpu_trace(mpt, ctx, sc, 1, spec)
            n = paths.n()
            gX = [x for x in paths.X[:3, :n].cpu().numpy().T if inside(x)]
            table = oracle.enumerate_sequences(sc, 1, spec)
            sol, ver = oracle.candidate_range(sc, table, 0, len(table))
            oX = [sol.X[c, :3] for c in range(len(table)) if ver.valid[c] and inside(sol.X[c, :3])]
            roots[starts] = (_root_sets(gX, 1e-6), _root_sets(oX, 1e-6))
        g64, o64 = roots[64]
        assert len(g64) == len(o64) and all(any(np.abs(x - y).max() < 1e-6 for y in o64) for x in g64)
        g8, _ = roots[8]
        assert all(any(np.abs(x - y).max() < 1e-6 for y in o64) for x in g8)
        n_roots += len(o64)
    assert n_roots >= 30


# --------------------------------------------------------------- adjoint --
def _oracle_grad_sums(sc, table, paths_cand, paths_T, g_len, g_pts):
    gtx = np.zeros_like(sc.tx)
    grx = np.zeros_like(sc.rx)
    gobj = np.zeros(sc.n_obj)
    for i, c in enumerate(paths_cand):
        e, p = divmod(int(c), sc.n_pairs)
        ids = table.ids[e][:table.order[e]]
        tp = []
        for kk, o in enumerate(ids):
            tp.append(paths_T[i, 2 * kk])
            if sc.obj_kind[o] not in (2, 3):
                tp.append(paths_T[i, 2 * kk + 1])
        a, b = sc.pair_points(p)
        dL, dX = oracle.path_grad(sc, ids, a, b, tp)
        k = len(ids)
        w = g_len[i] * dL + g_pts[i, :3 * k] @ dX
        it, ir = (p // sc.rx.shape[0], p % sc.rx.shape[0]) if sc.pair_mode == 0 else (p, p)
        gtx[it] += w[0:3]
        grx[ir] += w[3:6]
        for kk, o in enumerate(ids):
            gobj[o] += w[6 + kk]
    return gtx, grx, gobj


@pytest.mark.parametrize("with_pts", [True, False])
@pytest.mark.parametrize("name", ["street_canyon", "urban4"])
def test_adjoint_matches_oracle_gradient(mpt, ctx, name, with_pts):
    """Full adjoint (length and point weights: the normal-matrix solve), and
    length weights alone (the explicit-gradient path of the library),
    against the oracle's implicit-function-theorem gradient."""
    sc = S.street_canyon() if name == "street_canyon" else S.urban_block(4)
    spec = S.CONFIG_SPECS["street_canyon"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    n = paths.n()
    rng = np.random.default_rng(4)
    g_len = torch.as_tensor(rng.uniform(0.5, 1.5, paths.capacity)).cuda()
    g_pts = torch.as_tensor(rng.normal(size=(12, paths.capacity)) * 0.1).cuda()
    if not with_pts:
        g_pts.zero_()
    gtx, grx, gobj = mpt.grad(ds, cands, paths, g_len, g_pts if with_pts else None)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec)
    cand = paths.cand[:n].cpu().numpy()
    T = paths.T[:, :n].cpu().numpy().T
    wtx, wrx, wobj = _oracle_grad_sums(sc, table, cand, T, g_len[:n].cpu().numpy(), g_pts[:, :n].cpu().numpy().T)
    scale = max(1.0, np.abs(wrx).max())
    assert np.abs(gtx.cpu().numpy() - wtx).max() < 1e-6 * max(1.0, np.abs(wtx).max())
    assert np.abs(grx.cpu().numpy() - wrx).max() < 1e-6 * scale
    # edges (kind 2) have no plane offset: the oracle column is zero
    planes = sc.obj_kind == 0
    assert np.abs(gobj.cpu().numpy()[planes] - wobj[planes]).max() < 1e-6 * max(1.0, np.abs(wobj).max())
    print(f"adjoint {name}: {n} paths, |dL/dTX| {np.abs(wtx).max():.3e}")


def test_autograd_function_matches_central_differences(mpt, ctx):
    """MPT lengths as a torch.autograd.Function: d(sum of lengths)/d(RX, TX,
    plane offsets) against central differences (h = 1e-4 m) of the GPU
    forward, over the paths present in the base and both perturbed runs."""
    from paper_2301_06399_gb300 import autograd as ag

    sc = S.urban_block(4)
    tx = torch.tensor(sc.tx, dtype=torch.float64, device="cuda", requires_grad=True)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda", requires_grad=True)
    dd = torch.zeros(sc.n_obj, dtype=torch.float64, device="cuda", requires_grad=True)
    L, X, cand = ag.path_lengths(ctx, sc, tx, rx, dd)
    assert L.numel() > 100
    h = 1e-4

    def lengths(tx_, rx_, dd_):
        with torch.no_grad():
            l2, _, c2 = ag.path_lengths(ctx, sc, tx_, rx_, dd_)
        return dict(zip(c2.cpu().tolist(), l2.cpu().tolist()))

    base = dict(zip(cand.cpu().tolist(), L.detach().cpu().tolist()))
    rng = np.random.default_rng(3)
    checks = [("rx", int(rng.integers(sc.rx.shape[0])), int(rng.integers(3))) for _ in range(3)]
    checks += [("tx", 0, j) for j in range(3)]
    walls = [int(o) for o in rng.choice(np.nonzero(sc.obj_kind == 0)[0], 3, replace=False)]
    checks += [("dd", o, 0) for o in walls]
    for what, i, j in checks:
        args_p = [tx.detach().clone(), rx.detach().clone(), dd.detach().clone()]
        args_m = [tx.detach().clone(), rx.detach().clone(), dd.detach().clone()]
        k = {"tx": 0, "rx": 1, "dd": 2}[what]
        if what == "dd":
            args_p[k][i] += h
            args_m[k][i] -= h
        else:
            args_p[k][i, j] += h
            args_m[k][i, j] -= h
        lp, lm = lengths(*args_p), lengths(*args_m)
        common = sorted(set(base) & set(lp) & set(lm))
        fd = sum((lp[c] - lm[c]) / (2 * h) for c in common)
        mask = torch.tensor([1.0 if int(c) in set(common) else 0.0 for c in cand.cpu().tolist()],
                            dtype=torch.float64, device="cuda")
        g = torch.autograd.grad(L, [tx, rx, dd], grad_outputs=mask, retain_graph=True)
        ad = g[k][i].item() if what == "dd" else g[k][i, j].item()
        assert abs(ad - fd) < 1e-5 * max(1.0, abs(fd)), (what, i, j, ad, fd)


# ---------------------------------------------------------- FP32 precision --
def test_fp32_only_error_is_reported(mpt, ctx):
    """FP32 iterations alone reach ~1e-5..1e-3 m; the FP64 refinement brings
    the same candidates to the 1e-6 m bar (reported, not a pass criterion
    beyond a sanity bound)."""
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, keep_fp32=True)
    n = paths.n()
    cand = paths.cand[:n].cpu().numpy()
    T32 = sols.T32[:, cand].cpu().numpy().T.astype(np.float64)
    T64 = paths.T[:, :n].cpu().numpy().T
    err32 = np.abs(T32 - T64).max()
    print(f"FP32-only parameter error vs refined (valid paths): max {err32:.2e} m")
    assert err32 < 5e-2


# -------------------------------------------------------------- edge cases --
def test_empty_enumeration(mpt, ctx):
    sc = S.street_canyon()
    spec = S.SequenceSpec(quota=(0, 0, 0, 0))
    ds = mpt.DeviceScene(ctx, sc)
    assert mpt.candidate_count(ds, 2, spec) == 0
    cands = mpt.enumerate_candidates(ds, 2, spec, capacity=1)
    sols = mpt.solve(ds, cands)
    paths = mpt.validate(ds, cands, sols, capacity=4)
    torch.cuda.synchronize()
    assert int(cands.count.item()) == 0 and paths.n() == 0


def test_order_four_full_enumeration_small_scene(mpt, ctx):
    """Every ordered sequence of 1..4 distinct objects on a 5-object scene."""
    b = S._Builder()
    ez = np.array([0, 0, 1.0])
    b.rect_plane([-50, -50, 0], [1, 0, 0], [0, 1, 0], 100, 100)
    b.rect_plane([-20, 10, 0], [1, 0, 0], [0, 0, 1], 40, 20)
    b.rect_plane([-20, -10, 0], [0, 0, 1], [1, 0, 0], 20, 40)
    b.line_edge([20, 10, 0], ez, 0, 20, [1, 0, 0], [0, 1, 0])
    b.line_edge([-20, -10, 0], ez, 0, 20, [-1, 0, 0], [0, -1, 0])
    rng = np.random.default_rng(8)
    sc = b.build("five", 100.0, [[0.0, 0.0, 10.0]],
                 np.c_[rng.uniform(-15, 15, 40), rng.uniform(-8, 8, 40), np.full(40, 1.5)])
    spec = S.SequenceSpec(quota=(-1, -1, -1, -1))
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 4, spec)
    table = oracle.enumerate_sequences(sc, 4, spec)
    assert len(table) == 5 + 20 + 60 + 120
    compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)


@pytest.mark.parametrize("name", ["urban_block", "mixed_order", "curved"])
def test_visibility_matrix_bit_exact(mpt, ctx, name):
    sc = {"urban_block": lambda: S.urban_block(4), "mixed_order": S.mixed_order_city, "curved": S.curved_scene}[name]()
    ds = mpt.DeviceScene(ctx, sc)
    V = mpt.visibility(ds)
    torch.cuda.synchronize()
    want = oracle.visibility_matrix(sc)
    assert np.array_equal(V.cpu().numpy(), want)
    assert 0 < want.sum() < want.size - len(want)  # the test prunes something


def test_visibility_pruning_keeps_every_valid_path_of_the_urban_block(mpt, ctx):
    # closed boxes: a path that used a wall from behind runs inside a box, so
    # pruning the enumeration with V loses only paths to receivers that the
    # workload places inside a footprint (kept there on purpose, validity
    # decides); every path to a receiver outside the boxes survives
    sc = S.urban_block(8)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    V = mpt.visibility(ds)
    cm = mpt.enumerate_candidates(ds, 2, spec, adj=V)
    sm = mpt.solve(ds, cm, mpt.FP32_FP64REFINE)
    pm = mpt.validate(ds, cm, sm, capacity=cm.capacity)
    torch.cuda.synchronize()
    n_full, n_masked = int(cands.count.item()), int(cm.count.item())
    assert n_masked < 0.75 * n_full

    def keys(c, p):
        pair, ids, order, start = mpt.decode_candidates(c, int(c.count.item()))
        sel = p.cand[:p.n()].cpu().numpy()
        return {(int(pair[k]), tuple(int(x) for x in ids[k][:order[k]])) for k in sel}

    full, masked = keys(cands, paths), keys(cm, pm)
    assert masked <= full

    def inside(rx):
        return any(x0 <= rx[0] <= x1 and y0 <= rx[1] <= y1 for (x0, y0, x1, y1, h) in sc.meta["boxes"])

    outside = {k for k in full if not inside(sc.rx[k[0] % sc.rx.shape[0]])}
    assert len(outside) > 100
    assert outside <= masked


def test_received_field_matches_oracle(mpt, ctx):
    # Sec. V, Eqs. 16-19 at 1 GHz; points agree to 1e-6 m, so each path's
    # phase to k * 3e-6 rad: the bound below is that, summed over the paths
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    k = 2 * np.pi / 0.3
    refl, diff = -1.0, 0.25 - 0.1j
    got = mpt.field(ds, cands, paths, k, 1.0, refl, diff)
    torch.cuda.synchronize()
    got = got[:, 0].cpu().numpy() + 1j * got[:, 1].cpu().numpy()
    table = oracle.enumerate_sequences(sc, 2, spec)
    sol, ver = oracle.candidate_range(sc, table, 0, len(table) * sc.n_pairs)
    assert not ver.ambiguous[ver.valid > 0].any()
    want = oracle.path_field(sc, table, sol, ver, k, 1.0, refl, diff)
    mag = oracle.path_field(sc, table, sol, ver, 0.0 + 1e-300, 1.0, abs(refl), abs(diff))  # sum of |contributions|
    assert np.all(np.abs(got - want) <= 2 * k * 3e-6 * np.abs(mag) + 1e-15)
    assert np.abs(want).max() > 0


# ------------------------------------------------------- failure path ---
def test_bounded_wait_reports_timeout_and_the_context_stays_usable(mpt, ctx):
    """A device wait that gives up (a flag nothing sets, bounded spin) raises
    the context's error flag; mpt_ctx_check reports MPT_ERR_TIMEOUT once and
    clears it, and the context keeps working."""
    assert ctx.check() == mpt.MPT_OK
    assert ctx.selftest_wait() == mpt.MPT_OK
    torch.cuda.synchronize()
    assert ctx.check() == mpt.MPT_ERR_TIMEOUT
    assert ctx.check() == mpt.MPT_OK
    sc = S.street_canyon()
    spec = S.CONFIG_SPECS["street_canyon"]
    _, cands, _, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_valid, _, _, _ = compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)
    assert n_valid == paths.n() > 0


def _host_shifted(scene, delta):
    """The scene with plane i moved by delta[i] along its normal, built on the
    host (corner and offset of the plane, corner of its own rectangle)."""
    s = S.Scene(scene.name, scene.scale, scene.obj_kind.copy(), scene.obj_param.copy(), scene.occ_kind.copy(),
                scene.occ_param.copy(), scene.tx.copy(), scene.rx.copy(), scene.pair_mode, dict(scene.meta))
    L, OL = S.OBJ_LAYOUT[S.PLANE], S.OCC_LAYOUT[S.OCC_RECT]
    for i in np.nonzero(delta)[0]:
        if s.obj_kind[i] != S.PLANE:
            continue
        p = s.obj_param[i]
        n, O0 = p[L["n"]:L["n"] + 3].copy(), p[L["O"]:L["O"] + 3].copy()
        for q in range(s.n_occ):
            if s.occ_kind[q] == S.OCC_RECT and np.array_equal(s.occ_param[q, OL["O"]:OL["O"] + 3], O0) and \
                    np.array_equal(s.occ_param[q, OL["u"]:OL["u"] + 3], p[L["u"]:L["u"] + 3]):
                s.occ_param[q, OL["O"]:OL["O"] + 3] = O0 + delta[i] * n
        p[L["d"]] += delta[i]
        p[L["O"]:L["O"] + 3] = O0 + delta[i] * n
    return s.contiguous()


@pytest.mark.parametrize("which", ["ground_and_walls", "ground"])
def test_device_plane_shift_equals_host_shift(mpt, ctx, which):
    """mpt_scene_shift_planes (device) against a host-shifted re-upload: the
    solver's output is bit-identical (same rounding of the shifted records);
    with only the ground moved (no edge lies in its plane, so validation's
    lists of rectangles holding an object agree) the valid paths are too."""
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    delta = np.zeros(sc.n_obj)
    ground = int(np.nonzero(sc.obj_kind == S.PLANE)[0][-1])
    delta[ground] = 0.3
    if which == "ground_and_walls":
        delta[[0, 5, 13, 22]] = [0.25, -0.4, 1.0, 0.05]
    base = mpt.DeviceScene(ctx, sc)
    dst = mpt.DeviceScene(ctx, sc)
    mpt.shift_planes(base, dst, torch.as_tensor(delta).cuda())
    view = mpt.SceneView(ctx, sc, dst.h, base.tx, base.rx)
    r1 = mpt.trace(view, 2, spec, path_capacity=1 << 16)
    r2 = mpt.trace(mpt.DeviceScene(ctx, _host_shifted(sc, delta)), 2, spec, path_capacity=1 << 16)
    torch.cuda.synchronize()
    n = int(r1.cands.count.item())
    assert torch.equal(r1.sols.T[:, :n], r2.sols.T[:, :n]) and torch.equal(r1.sols.cost[:n], r2.sols.cost[:n])
    assert torch.equal(r1.sols.status[:n], r2.sols.status[:n])
    if which == "ground":
        m = r1.paths.n()
        assert m == r2.paths.n() > 100
        assert torch.equal(r1.paths.cand[:m], r2.paths.cand[:m]) and torch.equal(r1.paths.X[:, :m], r2.paths.X[:, :m])


def test_solver_timing_events(mpt, ctx):
    """mpt_ctx_time_solver / mpt_ctx_solver_ms: with timing on, the order-2
    solver launch of the urban block (8x8 RX) has a positive duration and the
    solutions are bit-identical to a solve with timing off."""
    sc = S.urban_block(8)
    spec = S.CONFIG_SPECS["urban_block"]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, spec)
    s_off = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
    ctx.time_solver(True)
    try:
        s_on = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
        torch.cuda.synchronize()
        ms = ctx.solver_ms(2)
    finally:
        ctx.time_solver(False)
    assert 0.0 < ms < 1000.0
    assert torch.equal(s_on.T.view(torch.int64), s_off.T.view(torch.int64))
    assert torch.equal(s_on.status, s_off.status)
    print(f"order-2 solver launch: {ms:.3f} ms")
