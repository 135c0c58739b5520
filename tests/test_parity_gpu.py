"""GPU parity: every step of the CUDA path, called through the C ABI, against the
CPU oracle on the same seeded inputs. Everything on this path is integer, so the
bar is bit-exact equality (the kd tree: equal leaf sets, split dimensions and split
values; the order inside a leaf is unspecified by the ABI)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1508_05151_gb300 import ffapi, synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")
SIZES = [(1, 1), (5, 3), (17, 13), (33, 31), (128, 96), (300, 170)]


def rimg(seed, H, W, flat=False):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
    if flat and H > 4 and W > 4:
        img[H // 4:H // 2, W // 4:W // 2] = 90  # ties
    return img


def tg(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_census(img, n):
    sm = ffapi.ff_smooth(tg(img), n)
    return ffapi.ff_census(sm, n), sm


# ------------------------------------------------------------------ A1/A2 -----
@pytest.mark.parametrize("W,H", SIZES + [(1024, 436)])
def test_smooth_and_census(W, H):
    img = rimg(W * 7 + H, H, W)
    for n in (1, 2, 4, 8):
        C, sm = gpu_census(img, n)
        ref_sm = O.smooth(img, n)
        assert np.array_equal(cpu(sm), ref_sm), (W, H, n)
        assert np.array_equal(cpu(C).view(np.uint32), O.census(ref_sm, n)), (W, H, n)


# --------------------------------------------------------------------- A3 -----
@pytest.mark.parametrize("W,H", SIZES + [(1024, 436)])
def test_features_all_pixels(W, H):
    img = rimg(W + 3 * H, H, W)
    for r in ((8, 6, 2) if W * H < 100000 else (8,)):
        f = cpu(ffapi.ff_features(tg(img), r))
        ref = O.wht_features(img, r)
        assert np.array_equal(f[:, :27], ref), (W, H, r)
        assert (f[:, 27] == 0).all()


def test_features_point_list():
    img = rimg(5, 90, 110)
    pts = np.array([[0, 0], [109, 89], [50, 3], [7, 88], [64, 40]], np.int32)
    for r in (8, 6, 1):
        f = cpu(ffapi.ff_features(tg(img), r, tg(pts)))
        assert np.array_equal(f[:, :27], O.wht_features(img, r, pts))


# --------------------------------------------------------------------- A4 -----
def _leafsets(perm, N, D):
    out = []
    for lf in range(1 << D):
        b, e = O.kd_leaf_range(N, D, lf)
        out.append(np.sort(perm[b:e]))
    return out


@pytest.mark.parametrize("W,H,r,leaf,flat", [(17, 13, 2, 2, False), (33, 31, 3, 8, True),
                                             (128, 96, 8, 8, False), (128, 96, 8, 8, True),
                                             (301, 203, 6, 5, True), (1024, 436, 8, 8, False)])
def test_kdtree_build(W, H, r, leaf, flat):
    img = rimg(W * H, H, W, flat)
    feat_g = ffapi.ff_features(tg(img), r)
    feat = cpu(feat_g)[:, :27]
    T = ffapi.ff_kdtree_build(feat_g, leaf)
    ref = O.kd_build(feat, leaf)
    assert T["D"] == ref["D"]
    assert np.array_equal(cpu(T["split_dim"]), ref["split_dim"])
    assert np.array_equal(cpu(T["split_val"]), ref["split_val"])
    g, o = _leafsets(cpu(T["perm"]), ref["N"], ref["D"]), _leafsets(ref["perm"], ref["N"], ref["D"])
    for a, b in zip(g, o):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N,leaf", [(3000, 4), (70001, 8)])
def test_kdtree_build_arbitrary_features(N, leaf):
    """The public kd build on feature rows that no WHT produces: spreads up to
    2^31 (keys wider than the WHT bound, more radix passes) and heavy ties."""
    rng = np.random.default_rng(N)
    feat = np.zeros((N, 28), np.int32)
    feat[:, :9] = rng.integers(-2**30, 2**30, size=(N, 9))
    feat[:, 9:18] = rng.integers(-3, 4, size=(N, 9)) * (2**28)  # few values, many ties
    feat[:, 18:27] = rng.integers(0, 5, size=(N, 9))
    fg = tg(feat)
    T = ffapi.ff_kdtree_build(fg, leaf)
    ref = O.kd_build(feat[:, :27], leaf)
    assert T["D"] == ref["D"]
    assert np.array_equal(cpu(T["split_dim"]), ref["split_dim"])
    assert np.array_equal(cpu(T["split_val"]), ref["split_val"])
    g, o = _leafsets(cpu(T["perm"]), ref["N"], ref["D"]), _leafsets(ref["perm"], ref["N"], ref["D"])
    for a, b in zip(g, o):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N,leaf", [(1000, 4), (5000, 4)])
def test_kdtree_build_mixed_key_widths(N, leaf):
    """Subtree levels whose nodes need 64-bit sort keys (a split-dimension spread
    >= 2^21) and levels that use 32-bit keys, in one tree. Dimension 0 splits the
    root into its two value groups exactly; dimension 2 spreads exactly 2^21 in one
    child only; all others stay below 2^21. With N = 1000 the whole tree is one
    subtree CTA: levels 0-1 take 64-bit keys (level 1 with one wide and one narrow
    node), the deeper levels 32-bit keys."""
    rng = np.random.default_rng(N + 7)
    feat = np.zeros((N, 28), np.int32)
    hi = rng.permutation(N)[: N - N // 2]
    feat[hi, 0] = 2**25
    lo = np.setdiff1d(np.arange(N), hi)
    feat[rng.permutation(lo)[: len(lo) // 2], 2] = 2**21
    feat[:, 1] = rng.integers(0, 2**21, size=N)
    feat[:, 3:27] = rng.integers(0, 2**19, size=(N, 24))
    T = ffapi.ff_kdtree_build(tg(feat), leaf)
    ref = O.kd_build(feat[:, :27], leaf)
    assert T["D"] == ref["D"]
    assert np.array_equal(cpu(T["split_dim"]), ref["split_dim"])
    assert np.array_equal(cpu(T["split_val"]), ref["split_val"])
    g, o = _leafsets(cpu(T["perm"]), ref["N"], ref["D"]), _leafsets(ref["perm"], ref["N"], ref["D"])
    for a, b in zip(g, o):
        assert np.array_equal(a, b)
    sd = ref["split_dim"]
    assert sd[0] == 0 and 2 in sd[1:3] and (sd[3:] != 0).all() and (sd[3:] != 2).all()


# --------------------------------------------------------------------- A5 -----
@pytest.mark.parametrize("W,H,n,r,leaf,K", [(40, 30, 1, 3, 4, 0), (128, 96, 8, 8, 8, 0),
                                           (128, 96, 8, 8, 8, 3), (130, 97, 4, 6, 8, 2),
                                           (300, 170, 8, 8, 8, 4)])
def test_kdtree_init(W, H, n, r, leaf, K):
    p = synth.pair_shift(W + H, W=W, H=H, max_shift=(8, 8), square=min(16, W, H), square_move=6)
    I1, I2 = p["I1"], p["I2"]
    C1g, _ = gpu_census(I1, n)
    C2g, _ = gpu_census(I2, n)
    feat_g = ffapi.ff_features(tg(I2), r)
    T = ffapi.ff_kdtree_build(feat_g, leaf)
    Gx, Gy = O.grid(W, H, n)
    prop = None
    if K:
        prop = np.random.default_rng(1).integers(-40, 41, size=(Gy, Gx, K, 2)).astype(np.int16)
    f, c = ffapi.ff_kdtree_init(T, leaf, tg(I1), C1g, C2g, n, r,
                                None if prop is None else tg(prop))
    C1 = O.census(O.smooth(I1, n), n)
    C2 = O.census(O.smooth(I2, n), n)
    fr, cr, _ = O.kd_init(cpu(feat_g)[:, :27], I1, r, leaf, C1, C2, n,
                          None if prop is None else prop.astype(np.int32))
    assert np.array_equal(cpu(c), cr)
    assert np.array_equal(cpu(f).astype(np.int32), fr)


def test_kdtree_init_reports_a_corrupt_tree():
    """A caller's tree with a split dimension outside [0, 27) or a leaf entry outside
    [0, N): the query's own checks skip the access and report device status 1
    (DEV_ERR_BOUNDS) with the grid point and the node or leaf position; a sound tree
    reports 0."""
    W, H, n, r, leaf = 64, 48, 4, 4, 8
    p = synth.pair_shift(5, W=W, H=H, max_shift=(6, 6), square=16, square_move=4)
    C1g, _ = gpu_census(p["I1"], n)
    C2g, _ = gpu_census(p["I2"], n)
    T = ffapi.ff_kdtree_build(ffapi.ff_features(tg(p["I2"]), r), leaf)
    _, _, st = ffapi.ff_kdtree_init(T, leaf, tg(p["I1"]), C1g, C2g, n, r, with_status=True)
    assert st == (0, 0, 0)
    N = T["N"]
    sd, _ = T["_keep"]
    sd[0] = 99  # root split dimension out of range: every grid point meets it
    _, _, st = ffapi.ff_kdtree_init(T, leaf, tg(p["I1"]), C1g, C2g, n, r, with_status=True)
    assert st[0] == 1 and st[2] == 0
    T2 = ffapi.ff_kdtree_build(ffapi.ff_features(tg(p["I2"]), r), leaf)
    T2["perm"][:] = N + 7  # every leaf entry out of range
    f, c, st = ffapi.ff_kdtree_init(T2, leaf, tg(p["I1"]), C1g, C2g, n, r, with_status=True)
    assert st[0] == 1 and 0 <= st[2] < N
    assert bool((c == O.COST_UNSET).all())  # no candidate was evaluated
    torch.cuda.synchronize()


# ---------------------------------------------------------------- A7 / A8 -----
@pytest.mark.parametrize("W,H,n,r,tile,n_rs", [(64, 48, 1, 3, 8, 3), (128, 96, 1, 8, 32, 3),
                                               (128, 96, 2, 8, 32, 3), (128, 96, 4, 6, 32, 2),
                                               (97, 71, 2, 4, 6, 3), (200, 150, 1, 6, 16, 1),
                                               (33, 31, 8, 8, 2, 3), (300, 170, 2, 8, 32, 0)])
def test_search_level_seeded(W, H, n, r, tile, n_rs):
    p = synth.pair_shift(W * 3 + H, W=W, H=H, max_shift=(10, 10), square=min(24, W, H),
                         square_move=9)
    I1, I2 = p["I1"], p["I2"]
    C1g, _ = gpu_census(I1, n)
    C2g, _ = gpu_census(I2, n)
    C1, C2 = cpu(C1g).view(np.uint32), cpu(C2g).view(np.uint32)
    Gxc, Gyc = O.grid(W, H, 2 * n)
    rng = np.random.default_rng(n * 100 + r)
    coarse = rng.integers(-12, 13, size=(Gyc, Gxc, 2))
    ys, xs = np.mgrid[0:Gyc, 0:Gxc] * (2 * n)
    coarse[..., 0] = np.clip(xs + coarse[..., 0], 0, W - 1) - xs
    coarse[..., 1] = np.clip(ys + coarse[..., 1], 0, H - 1) - ys
    P = dict(tile=tile, n_rs=n_rs, seed=12345, R=1)
    for fid in (0, 2):
        f, c = ffapi.ff_search_level(C1g, C2g, n, r, P, flow_id=fid,
                                     flow_coarse=tg(coarse.astype(np.int16)))
        fr, cr, _ = O.search_level(C1, C2, n, r, flow_coarse=coarse.astype(np.int32), tile=tile,
                                   n_rs=n_rs, R=1, seed=12345, flow_id=fid)
        assert np.array_equal(cpu(c), cr)
        assert np.array_equal(cpu(f).astype(np.int32), fr)


@pytest.mark.parametrize("W,H,n,r,tile,pw,rs_min_n,wide,split,split2", [
    (128, 96, 1, 8, 16, 1, 1, 0, 0, 0), (200, 150, 4, 6, 16, 8, 2, 0, 0, 0),
    (97, 71, 2, 8, 6, 3, 2, 0, 0, 0), (128, 96, 1, 8, 16, 1, 0, 1, 0, 0),
    (200, 150, 4, 6, 16, 8, 8, 2, 2, 0), (97, 71, 2, 8, 6, 3, 0, 2, 0, 0),
    (300, 170, 8, 8, 10, 4, 2, 8, 8, 0), (130, 97, 1, 3, 14, 4, 0, 1, 1, 0),
    (128, 96, 1, 8, 16, 1, 0, 1, 0, 1), (97, 71, 2, 6, 6, 3, 0, 2, 0, 2),
    (130, 97, 1, 3, 14, 4, 0, 1, 1, 1), (200, 150, 4, 5, 16, 8, 4, 1, 0, 4)])
def test_search_level_execution_variants(W, H, n, r, tile, pw, rs_min_n, wide, split, split2):
    """The random search as a kernel of its own and the CTA-per-tile propagation
    with 2, 4 or 8 threads per candidate (execution parameters) equal the oracle."""
    p = synth.pair_shift(W + 11 * H, W=W, H=H, max_shift=(10, 10), square=min(24, W, H),
                         square_move=9)
    C1g, _ = gpu_census(p["I1"], n)
    C2g, _ = gpu_census(p["I2"], n)
    C1, C2 = cpu(C1g).view(np.uint32), cpu(C2g).view(np.uint32)
    Gxc, Gyc = O.grid(W, H, 2 * n)
    rng = np.random.default_rng(n + r)
    coarse = rng.integers(-12, 13, size=(Gyc, Gxc, 2))
    ys, xs = np.mgrid[0:Gyc, 0:Gxc] * (2 * n)
    coarse[..., 0] = np.clip(xs + coarse[..., 0], 0, W - 1) - xs
    coarse[..., 1] = np.clip(ys + coarse[..., 1], 0, H - 1) - ys
    before = ffapi.get_exec_params()
    try:
        ffapi.set_exec_params(pass_warps=pw, rs_min_n=rs_min_n, wide_min_n=wide, split8_min_n=split,
                              split2_max_n=split2)
        f, c = ffapi.ff_search_level(C1g, C2g, n, r, dict(tile=tile, seed=77), flow_id=1,
                                     flow_coarse=tg(coarse.astype(np.int16)))
        torch.cuda.synchronize()
    finally:
        ffapi.set_exec_params(**before)
    fr, cr, _ = O.search_level(C1, C2, n, r, flow_coarse=coarse.astype(np.int32), tile=tile,
                               seed=77, flow_id=1)
    assert np.array_equal(cpu(c), cr)
    assert np.array_equal(cpu(f).astype(np.int32), fr)


@pytest.mark.parametrize("W,H,n,r,tile", [(128, 96, 8, 8, 32), (80, 60, 1, 3, 10)])
def test_search_level_from_state(W, H, n, r, tile):
    # top-level form: the state (including unset points) is the input
    p = synth.pair_shift(7, W=W, H=H, max_shift=(6, 6), square=16, square_move=5)
    C1g, _ = gpu_census(p["I1"], n)
    C2g, _ = gpu_census(p["I2"], n)
    C1, C2 = cpu(C1g).view(np.uint32), cpu(C2g).view(np.uint32)
    Gx, Gy = O.grid(W, H, n)
    rng = np.random.default_rng(3)
    flow = np.zeros((Gy, Gx, 2), np.int32)
    cost = np.full((Gy, Gx), O.COST_UNSET, np.int32)
    for _ in range(max(2, Gx * Gy // 20)):
        gx, gy = rng.integers(0, Gx), rng.integers(0, Gy)
        x, y = gx * n, gy * n
        tx, ty = np.clip(x + rng.integers(-9, 10), 0, W - 1), np.clip(y + rng.integers(-9, 10), 0, H - 1)
        flow[gy, gx] = (tx - x, ty - y)
        cost[gy, gx] = O.patch_cost(C1, C2, n, r, (x, y), (tx, ty))
    fg, cg = tg(flow.astype(np.int16)), tg(cost)
    ffapi.ff_search_level(C1g, C2g, n, r, dict(tile=tile), flow_id=1, flow=fg, cost=cg)
    fr, cr, _ = O.search_level(C1, C2, n, r, flow=flow, cost=cost, tile=tile, flow_id=1)
    assert np.array_equal(cpu(cg), cr)
    assert np.array_equal(cpu(fg).astype(np.int32), fr)


# ------------------------------------------------------------ A11 - A13 -------
@pytest.mark.parametrize("seed", [1, 2])
def test_consistency_filter(seed):
    p = synth.workload_pair("noise_128x96", seed)
    ref = O.flow_fields(p["I1"], p["I2"])
    flows = ref["flows"].copy()
    rng = np.random.default_rng(seed)
    # perturb: random outliers and small shifts so every branch is exercised
    m = rng.random(flows.shape[1:3]) < 0.05
    flows[0][m] += rng.integers(-6, 7, size=(int(m.sum()), 2)).astype(np.int32)
    H, W = flows.shape[1:3]
    ys, xs = np.mgrid[0:H, 0:W]
    flows[0][..., 0] = np.clip(xs + flows[0][..., 0], 0, W - 1) - xs
    flows[0][..., 1] = np.clip(ys + flows[0][..., 1], 0, H - 1) - ys
    for params in (dict(eps=5, e=4, s=50), dict(eps=1, e=7, s=50), dict(eps=2, e=1, s=500)):
        g = ffapi.ff_consistency_filter(*(tg(flows[j].astype(np.int16)) for j in range(3)), params)
        vcc, err, e1, e2 = O.consistency(flows[0], flows[1], flows[2], params["eps"], errors=True)
        val = O.region_filter(flows[0], vcc, params["s"])
        sp, mask = O.sparsify(val, e1, e2, flows[0], params["e"])
        assert np.array_equal(cpu(g["err_sum"]), err)
        assert np.array_equal(cpu(g["valid"]), val)
        assert np.array_equal(cpu(g["mask"]), mask)
        n = int(cpu(g["n_sparse"])[0])
        assert n == len(sp)
        assert np.array_equal(cpu(g["sparse"])[:n], sp)


# ----------------------------------------------------------- whole path -------
def _compare(out, ref):
    assert np.array_equal(cpu(out["flows"]).astype(np.int32), ref["flows"])
    assert np.array_equal(cpu(out["valid"]), ref["valid"])
    assert np.array_equal(cpu(out["err_sum"]), ref["err_sum"])
    assert np.array_equal(cpu(out["mask"]), ref["mask"])
    n = int(cpu(out["n_sparse"])[0])
    assert n == len(ref["sparse"])
    assert np.array_equal(cpu(out["sparse"])[:n], ref["sparse"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_flow_fields_128x96(seed):
    p = synth.workload_pair("noise_128x96", seed)
    params = dict(seed=seed)
    out = ffapi.ff_flow_fields(tg(p["I1"]), tg(p["I2"]), params)
    _compare(out, O.flow_fields(p["I1"], p["I2"], params=params))


@pytest.mark.parametrize("W,H,params", [(1, 1, dict(k=3)), (5, 3, dict(k=1, r=2, r2=1)),
                                        (37, 29, dict(k=2, r=4, r2=3, tile=6)),
                                        (64, 48, dict(k=0, r=5, r2=5, leaf=3)),
                                        (150, 100, dict(k=4, tile=8, n_rs=1, R=2, leaf=12))])
def test_flow_fields_edge_shapes(W, H, params):
    p = synth.pair_shift(W + 11 * H, W=W, H=H, max_shift=(4, 4), square=min(8, W, H),
                         square_move=3)
    out = ffapi.ff_flow_fields(tg(p["I1"]), tg(p["I2"]), params)
    _compare(out, O.flow_fields(p["I1"], p["I2"], params=params))


def test_flow_fields_1024x436_full_size():
    # the benchmark workload, whole-field bit-exact comparison
    p = synth.workload_pair("layers_1024x436", 1)
    out = ffapi.ff_flow_fields(tg(p["I1"]), tg(p["I2"]))
    _compare(out, O.flow_fields(p["I1"], p["I2"], threads=3))


def test_flow_fields_is_deterministic_and_stream_independent():
    p = synth.workload_pair("noise_128x96", 9)
    ff = ffapi.FlowFields(128, 96)
    a = {k: v.clone() for k, v in ff.run(tg(p["I1"]), tg(p["I2"])).items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())  # calls are ordered only by their stream
    with torch.cuda.stream(s):
        b = ff.run(tg(p["I1"]), tg(p["I2"]))
    s.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert ff.device_status() == (0, 0, 0)


# ------------------------------------------- per-level budget composition -----
def test_forward_flow_levels_composition():
    """The per-level composition used by the random-search budget study: with a
    uniform budget it is ff_flow_fields' forward flow; with a different n_rs per
    level it is bit-exact against the oracle composed the same way."""
    from paper_1508_05151_gb300 import train
    W, H = 150, 101
    p = synth.pair_shift(4242, W=W, H=H, max_shift=(12, 9), square=32, square_move=10)
    I1, I2 = p["I1"], p["I2"]
    a, b = tg(I1), tg(I2)
    full = ffapi.FlowFields(W, H).run(a, b)
    assert torch.equal(train.forward_flow_levels(a, b, (3, 3, 3, 3)), full["flows"][0])
    bud = (1, 3, 0, 2)
    got = cpu(train.forward_flow_levels(a, b, bud)).astype(np.int32)
    P = O.default_params()
    r, leaf = P["r"], P["leaf"]
    feat = O.wht_features(I2, r)
    kw = dict(tile=P["tile"], R=P["R"], seed=P["seed"], flow_id=0)
    flow = None
    for i, n in enumerate((8, 4, 2, 1)):
        C1 = O.census(O.smooth(I1, n) if n > 1 else I1, n)
        C2 = O.census(O.smooth(I2, n) if n > 1 else I2, n)
        if i == 0:
            flow, cost, _ = O.kd_init(feat, I1, r, leaf, C1, C2, n)
            flow, cost, _ = O.search_level(C1, C2, n, r, flow=flow, cost=cost, n_rs=bud[i], **kw)
        else:
            flow, cost, _ = O.search_level(C1, C2, n, r, flow_coarse=flow, n_rs=bud[i], **kw)
    assert np.array_equal(got, flow)


# ------------------------------------------- full sizes of the other workloads --
def test_flow_fields_with_proposals_kitti_full_size():
    """The learned-proposal form at its workload's full size: a 1242x375 KITTI-shaped
    pair with K = 4 proposals per coarsest grid point through the whole path,
    bit-exact against the oracle given the same proposals. Two proposals are the
    rounded ground-truth flow (one jittered by a few pixels), so they often win the
    data term; two are random within +-300 px, so targets are clamped."""
    p = synth.workload_pair("kitti_1242x375", 11)
    H, W = p["I1"].shape[:2]
    Gx, Gy = O.grid(W, H, 8)
    rng = np.random.default_rng(12)
    gt = np.rint(p["flow"][::8, ::8]).astype(np.int64)[:Gy, :Gx]
    prop = np.empty((Gy, Gx, 4, 2), np.int64)
    prop[:, :, 0] = gt
    prop[:, :, 1] = gt + rng.integers(-3, 4, size=(Gy, Gx, 2))
    prop[:, :, 2:] = rng.integers(-300, 301, size=(Gy, Gx, 2, 2))
    prop = prop.astype(np.int16)
    params = dict(K=4)
    out = ffapi.FlowFields(W, H, params).run(tg(p["I1"]), tg(p["I2"]), tg(prop))
    ref = O.flow_fields(p["I1"], p["I2"], params=params, proposals=prop.astype(np.int32),
                        threads=3)
    _compare(out, ref)


def test_batch_64_mixed_full_size_sampled():
    """The benchmark's 64-pair mixed batch (16 each of 640x480, 584x388, 1024x436,
    1242x375, every pair from its own seed) as one graph replay: every pair equals
    the single-pair path, and two distinct pairs of each size are bit-exact against
    the oracle."""
    batch_pairs = synth.mixed_batch()
    sizes = [wh for wh, _ in batch_pairs]
    frames = [(tg(p["I1"]), tg(p["I2"])) for _, p in batch_pairs]
    batch = ffapi.FlowFieldsBatch(sizes, graph=True)
    outs = batch.run(frames)
    torch.cuda.synchronize()
    singles = {}
    for i, ((W, H), (a, b)) in enumerate(zip(sizes, frames)):
        if (W, H) not in singles:
            singles[(W, H)] = ffapi.FlowFields(W, H)
        one = singles[(W, H)].run(a, b)
        torch.cuda.synchronize()
        for key in ("flows", "valid", "err_sum", "mask", "n_sparse"):
            assert torch.equal(outs[i][key], one[key]), (i, key)
    for k in range(4):
        for j in (3, 12):
            i = 16 * k + j
            p = batch_pairs[i][1]
            _compare(outs[i], O.flow_fields(p["I1"], p["I2"], threads=3))


# ------------------------------------------------------------- CIELab ---------
def test_rgb_to_lab_every_colour():
    """ff_rgb_to_lab against the oracle on all 2^24 sRGB colours (a 4096 x 4096
    image holding each once): bit for bit."""
    v = np.arange(1 << 24, dtype=np.uint32)
    img = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], -1).astype(np.uint8)
    img = img.reshape(4096, 4096, 3)
    got = cpu(ffapi.ff_rgb_to_lab(tg(img)))
    assert np.array_equal(got, O.rgb_to_lab(img))


@pytest.mark.parametrize("seed", [4, 5])
def test_flow_fields_lab_128x96(seed):
    """The whole path in CIELab (params.color = 1) against the oracle."""
    p = synth.workload_pair("noise_128x96", seed)
    params = dict(color=1)
    out = ffapi.FlowFields(128, 96, params).run(tg(p["I1"]), tg(p["I2"]))
    torch.cuda.synchronize()
    _compare(out, O.flow_fields(p["I1"], p["I2"], params=params, threads=3))


# ------------------------------------------------- weighted median field ------
@pytest.mark.parametrize("rho", [1, 2, 3])
def test_weighted_median_field(rho):
    """ff_weighted_median against the oracle on the forward field of the whole
    path (128x96) and on a field with random outliers: flows and matching errors
    bit for bit."""
    p = synth.workload_pair("noise_128x96", 8)
    out = ffapi.FlowFields(128, 96).run(tg(p["I1"]), tg(p["I2"]))
    F = out["flows"][0].clone()
    torch.cuda.synchronize()
    Fn = cpu(F).astype(np.int32)
    rng = np.random.default_rng(rho)
    G = Fn.copy()
    m = rng.random(G.shape[:2]) < 0.1
    G[m] += rng.integers(-30, 31, size=(int(m.sum()), 2))
    ys, xs = np.mgrid[0:96, 0:128]
    G[..., 0] = np.clip(xs + G[..., 0], 0, 127) - xs
    G[..., 1] = np.clip(ys + G[..., 1], 0, 95) - ys
    for field in (Fn, G):
        med, E = ffapi.ff_weighted_median(tg(p["I1"]), tg(p["I2"]), tg(field.astype(np.int16)), 8, rho)
        Eo = O.match_errors(p["I1"], p["I2"], field, 8)
        assert np.array_equal(cpu(E), Eo)
        assert np.array_equal(cpu(med).astype(np.int32), O.weighted_median(field, Eo, rho))


# ------------------------------------------------ subpixel random search ------
@pytest.mark.parametrize("q", [2, 4])
def test_flow_fields_subpel_128x96(q):
    """The whole path with subpixel flows (params.subpel = q: interpolated target
    census, offsets and thresholds in 1/q pixel) against the oracle, bit for bit."""
    p = synth.workload_pair("noise_128x96", 9)
    params = dict(subpel=q)
    out = ffapi.FlowFields(128, 96, params).run(tg(p["I1"]), tg(p["I2"]))
    torch.cuda.synchronize()
    _compare(out, O.flow_fields(p["I1"], p["I2"], params=params, threads=3))


def test_flow_fields_subpel_translation_and_batch():
    """A pair whose true flow is half a pixel: GPU == oracle with subpel = 2; the
    batched form, the graph replay and the persistent level kernel give the same
    flows as the single pair."""
    rng = np.random.default_rng(13)
    v = synth.value_noise(rng, 72, 96, lattices=(16, 8, 4), amps=(0.5, 0.25, 0.125))
    I2 = (np.floor(v * 127) * 2).astype(np.int64)
    I1 = ((I2 + np.concatenate([I2[:, 1:], I2[:, -1:]], 1)) // 2).astype(np.uint8)
    I2 = I2.astype(np.uint8)
    params = dict(subpel=2)
    single = ffapi.FlowFields(96, 72, params).run(tg(I1), tg(I2))
    torch.cuda.synchronize()
    _compare(single, O.flow_fields(I1, I2, params=params, threads=3))
    ref = {k: v.clone() for k, v in single.items()}
    before = ffapi.get_exec_params()
    try:
        for persist in (0, 1):
            ffapi.set_exec_params(persist_levels=persist)
            for graph in (False, True):
                outs = ffapi.FlowFieldsBatch([(96, 72), (96, 72)], params, graph=graph).run(
                    [(tg(I1), tg(I2)), (tg(I1), tg(I2))])
                torch.cuda.synchronize()
                for o in outs:
                    for key in ("flows", "valid", "err_sum", "mask", "n_sparse"):
                        assert torch.equal(o[key], ref[key]), (persist, graph, key)
    finally:
        ffapi.set_exec_params(**before)
