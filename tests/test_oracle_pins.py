"""Pins of the CPU oracle to facts fixed outside the oracle itself.

Each test checks the oracle against mathematics, closed forms, published values,
brute force on tiny inputs, or invariants the paper states, chosen so that a
plausible slip (a dropped term, a flipped sign, a swapped index, a wrong tie rule)
fails at least one of them. No GPU is needed.
"""
import os

import numpy as np
import pytest

from paper_1508_05151_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNSET = 2**31 - 1


def rng_img(seed, H, W):
    return np.random.default_rng(seed).integers(0, 256, size=(H, W, 3), dtype=np.uint8)


# ---------------------------------------------------------------- RNG ----------
def test_splitmix64_published_sequence(ffo):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 3
    for state, out in rows:
        assert ffo.splitmix64(int(state, 16)) == int(out, 16)


def test_rs_offsets_uniform_and_bounded(ffo):
    # Lemire multiply-shift gives each value of [-Rn, Rn] with probability
    # 1/(2Rn+1) up to 2^-32; a chi-square over 40k draws must not reject.
    Rn = 4
    d = np.array([ffo.rs_offset(7, 1, 2, 0, x, y, Rn) for y in range(200) for x in range(200)])
    assert d.min() >= -Rn and d.max() <= Rn
    for c in range(2):
        cnt = np.bincount(d[:, c] + Rn, minlength=2 * Rn + 1)
        exp = len(d) / (2 * Rn + 1)
        chi2 = ((cnt - exp) ** 2 / exp).sum()
        assert chi2 < 30.0  # 8 dof, p ~ 2e-4
    # dx and dy are not the same stream
    assert np.mean(d[:, 0] == d[:, 1]) < 0.2
    # every key field changes the draw
    base = ffo.rs_offset(7, 1, 2, 0, 5, 6, 1000)
    for args in [(8, 1, 2, 0, 5, 6), (7, 2, 2, 0, 5, 6), (7, 1, 3, 0, 5, 6),
                 (7, 1, 2, 1, 5, 6), (7, 1, 2, 0, 6, 6), (7, 1, 2, 0, 5, 7)]:
        assert ffo.rs_offset(*args, 1000) != base


# --------------------------------------------------------- census / E_d --------
def test_census_constant_image_is_zero(ffo):
    img = np.full((9, 11, 3), 77, np.uint8)
    for n in (1, 2, 4):
        assert not ffo.census(img, n).any()


def test_census_single_dark_pixel_bit_layout(ffo):
    # One dark pixel in a flat image. Each neighbour at spacing n sees it at the
    # opposite offset, so exactly the bit of that offset is set, in all three
    # channels (offsets in raster order without the centre: bit 8c + o).
    for n in (1, 2):
        img = np.full((15, 15, 3), 100, np.uint8)
        img[7, 7] = 10
        C = ffo.census(img, n)
        offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
        for o, (dx, dy) in enumerate(offs):
            x, y = 7 - n * dx, 7 - n * dy
            assert C[y, x] == (1 << o) * 0x010101, (n, o)
        assert C[7, 7] == 0
        assert C[0, 0] == 0


def test_census_single_bright_pixel_all_bits(ffo):
    img = np.full((8, 8, 3), 50, np.uint8)
    img[3, 4] = (200, 40, 60)  # R and B brighter than the flat 50, G darker
    C = ffo.census(img, 1)
    # centre: neighbours are darker in R (bits 0-7) and B (bits 16-23); in G
    # the centre is darker, so no G bit
    assert C[3, 4] == 0xFF00FF


def test_patch_cost_identities(ffo):
    rng = np.random.default_rng(3)
    I1, I2 = rng_img(1, 20, 24), rng_img(2, 20, 24)
    for n in (1, 2, 4):
        C1, C2 = ffo.census(I1, n), ffo.census(I2, n)
        for r in (1, 3, 6):
            for _ in range(10):
                p1 = (int(rng.integers(0, 24)), int(rng.integers(0, 20)))
                p2 = (int(rng.integers(0, 24)), int(rng.integers(0, 20)))
                e = ffo.patch_cost(C1, C2, n, r, p1, p2)
                assert 0 <= e <= 24 * (2 * r + 1) ** 2
                assert e == ffo.patch_cost(C2, C1, n, r, p2, p1)
                assert ffo.patch_cost(C1, C1, n, r, p1, p1) == 0


def test_patch_cost_counts_clamped_tap_multiplicity(ffo):
    # Ct equals Cs except for one bit at the corner pixel (0, 0). E(p, p) is then
    # the number of taps of P^n_r(p) that clamp onto (0, 0): for p = (x, y) that
    # is #{u : x + n u <= 0} * #{v : y + n v <= 0}.
    W, H = 30, 25
    Cs = np.zeros((H, W), np.uint32)
    Ct = Cs.copy()
    Ct[0, 0] = 1 << 5
    for n, r, x, y in [(1, 3, 0, 0), (1, 3, 2, 1), (2, 3, 3, 4), (4, 2, 5, 9), (1, 8, 4, 7)]:
        cu = sum(1 for u in range(-r, r + 1) if x + n * u <= 0)
        cv = sum(1 for v in range(-r, r + 1) if y + n * v <= 0)
        assert ffo.patch_cost(Cs, Ct, n, r, (x, y), (x, y)) == cu * cv


# -------------------------------------------------------------- WHT ------------
def test_wht_blocks_follow_uneven_split():
    import oracle as O
    # footnote of Sec. 3.1: 2r+1 is split into r and r+1, then again
    assert list(O.wht_blocks(17)) == [4, 4, 4, 5]
    assert list(O.wht_blocks(13)) == [3, 3, 3, 4]
    assert list(O.wht_blocks(4)) == [1, 1, 1, 1]
    # an odd half splits again r | r + 1, the smaller block first
    assert list(O.wht_blocks(7)) == [1, 2, 2, 2]
    assert list(O.wht_blocks(5)) == [1, 1, 1, 2]
    assert list(O.wht_blocks(11)) == [2, 3, 3, 3]


def test_wht_basis_is_walsh_in_sequency_order(ffo):
    Hm = ffo.wht_basis_1d(4, 4)
    assert np.array_equal(Hm @ Hm.T, 4 * np.eye(4, dtype=np.int32))
    # sequency = number of sign changes = row index
    for i in range(4):
        assert int(np.sum(Hm[i, 1:] != Hm[i, :-1])) == i
    # odd windows: each function is constant on the 4 blocks
    for L in (13, 17):
        B = ffo.wht_basis_1d(L, 3)
        sz = ffo.wht_blocks(L)
        edges = np.cumsum(sz)[:-1]
        for i in range(3):
            assert int(np.sum(B[i, 1:] != B[i, :-1])) == i
            assert set(np.flatnonzero(B[i, 1:] != B[i, :-1]) + 1) <= set(edges)


def test_wht_exact_inverse_on_4x4(ffo):
    # Complete 2-D Walsh-Hadamard transform of a 4x4 patch: H H^T = 4 I per axis,
    # so patch = H^T coeff H / 16 exactly in integers.
    img = rng_img(5, 12, 12)
    pts = np.array([[5, 6], [1, 1], [9, 4]], np.int32)
    co = ffo.wht_features_general(img, 4, 4, pts)
    Hm = ffo.wht_basis_1d(4, 4).astype(np.int64)
    for k, (x, y) in enumerate(pts):
        for c in range(3):
            rec = Hm.T @ co[k, c].astype(np.int64) @ Hm
            assert np.all(rec % 16 == 0)
            patch = img[y - 1:y + 3, x - 1:x + 3, c].astype(np.int64)
            assert np.array_equal(rec // 16, patch)


def test_wht_constant_image_closed_form(ffo):
    # On a constant image v the feature (c, i, j) is v * S_i * S_j with S_i the
    # sum of the 1-D function: blocks 4,4,4,5 give S = (17, -1, +1).
    img = np.zeros((30, 30, 3), np.uint8)
    img[..., 0], img[..., 1], img[..., 2] = 10, 20, 30
    f = ffo.wht_features(img, 8, np.array([[15, 15], [0, 0], [29, 3]]))
    S = np.array([17, -1, 1])
    for c, v in enumerate((10, 20, 30)):
        exp = v * np.outer(S, S).ravel()
        for k in range(3):
            assert np.array_equal(f[k, 9 * c:9 * c + 9], exp)


def test_wht_linear_in_image(ffo):
    a, b = rng_img(1, 20, 20) // 2, rng_img(2, 20, 20) // 2
    fa, fb, fab = (ffo.wht_features(x, 6) for x in (a, b, a + b))
    assert np.array_equal(fa + fb, fab)


# ------------------------------------------------------------ kd tree ----------
def test_kd_depth():
    import oracle as O
    assert O.kd_depth(1024 * 436, 8) == 16
    assert O.kd_depth(128 * 96, 8) == 11
    assert O.kd_depth(8, 8) == 0
    assert O.kd_depth(9, 8) == 1


def test_kd_tree_invariants(ffo):
    img = rng_img(9, 23, 31)
    img[5:15, 5:15] = 40  # ties on many dimensions
    feat = ffo.wht_features(img, 3)
    N, leaf = len(feat), 6
    T = ffo.kd_build(feat, leaf)
    D = T["D"]
    leaves = ffo.kd_leaves(T)
    allp = np.concatenate(leaves)
    assert np.array_equal(np.sort(allp), np.arange(N))  # a partition
    sizes = np.array([len(l) for l in leaves])
    assert sizes.max() <= leaf and sizes.max() - sizes.min() <= 1 and sizes.min() >= 1

    # every internal node: split dim has maximal spread over the node (lowest on
    # ties), the left child is the first floor(m/2) under (value, index), the split
    # value is the first right value
    def members(node, depth):
        lo = node - ((1 << depth) - 1)
        span = 1 << (D - depth)
        return np.concatenate(leaves[lo * span:(lo + 1) * span])

    for depth in range(D):
        for i in range(1 << depth):
            node = (1 << depth) - 1 + i
            m = members(node, depth)
            spread = feat[m].max(0).astype(np.int64) - feat[m].min(0)
            d = T["split_dim"][node]
            assert d == int(np.argmax(spread))
            left = members(2 * node + 1, depth + 1)
            right = members(2 * node + 2, depth + 1)
            assert len(left) == len(m) // 2
            kl = sorted((feat[p, d], p) for p in left)
            kr = sorted((feat[p, d], p) for p in right)
            assert kl[-1] < kr[0]
            assert T["split_val"][node] == kr[0][0]


def test_kd_query_reaches_own_leaf_unless_tied(ffo):
    img = rng_img(4, 16, 20)
    feat = ffo.wht_features(img, 2)
    T = ffo.kd_build(feat, 4)
    owner = np.empty(len(feat), np.int64)
    for lf, l in enumerate(ffo.kd_leaves(T)):
        owner[l] = lf
    for p in range(len(feat)):
        got = ffo.kd_query(T, feat[p])
        if got != owner[p]:
            # only possible when p sits left of a split with value == split value
            node, D, tied = 0, T["D"], False
            path = owner[p]
            for d in range(D):
                go_right = (path >> (D - 1 - d)) & 1
                if not go_right and feat[p, T["split_dim"][node]] == T["split_val"][node]:
                    tied = True
                node = 2 * node + 1 + go_right
            assert tied


def test_kd_init_single_leaf_is_exact_nnf(ffo):
    # With l >= N the tree is one leaf holding every target pixel, so the
    # initialisation is the exhaustive nearest neighbour field under E_d
    # (the paper's "NNF", Sec. 4.1) with ties to the lowest pixel index.
    W, H = 16, 12
    I1, I2 = rng_img(11, H, W), rng_img(12, H, W)
    I2[4:8, 4:10] = I1[3:7, 2:8]  # some good matches
    for n, r in [(1, 2), (2, 1), (4, 1)]:
        C1, C2 = ffo.census(ffo.smooth(I1, n), n), ffo.census(ffo.smooth(I2, n), n)
        feat = ffo.wht_features(I2, r)
        flow, cost, ev = ffo.kd_init(feat, I1, r, W * H, C1, C2, n)
        Gx, Gy = ffo.grid(W, H, n)
        assert ev == Gx * Gy * W * H
        for gy in range(Gy):
            for gx in range(Gx):
                p = (gx * n, gy * n)
                best, arg = None, None
                for q in range(W * H):  # brute force in index order
                    e = ffo.patch_cost(C1, C2, n, r, p, (q % W, q // W))
                    if best is None or e < best:
                        best, arg = e, q
                assert cost[gy, gx] == best
                assert tuple(flow[gy, gx]) == (arg % W - p[0], arg // W - p[1])


def test_kd_init_proposals_strict_less(ffo):
    W, H = 20, 14
    I1 = rng_img(21, H, W)
    I2 = np.roll(I1, (2, 3), axis=(0, 1))
    C1, C2 = ffo.census(I1, 1), ffo.census(I2, 1)
    feat = ffo.wht_features(I2, 2)
    f0, c0, _ = ffo.kd_init(feat, I1, 2, 4, C1, C2, 1)
    # proposal 0 = the current winner (tie: must not replace), proposal 1 = far out
    # of the image (clamped), proposal 2 = truth
    prop = np.zeros((H, W, 3, 2), np.int32)
    prop[:, :, 0] = f0
    prop[:, :, 1] = (500, -500)
    prop[:, :, 2] = (3, 2)
    f1, c1, _ = ffo.kd_init(feat, I1, 2, 4, C1, C2, 1, proposals=prop)
    assert np.all(c1 <= c0)
    ys, xs = np.mgrid[0:H, 0:W]
    # the clamped proposal can only land on the right/top border
    tx, ty = xs + f1[..., 0], ys + f1[..., 1]
    assert tx.min() >= 0 and tx.max() < W and ty.min() >= 0 and ty.max() < H
    true_cost = np.array([[ffo.patch_cost(C1, C2, 1, 2, (x, y), (min(x + 3, W - 1), min(y + 2, H - 1)))
                           for x in range(W)] for y in range(H)])
    assert np.all(c1 <= true_cost)


# ------------------------------------------------------------- search ----------
def test_eval_count_matches_schedule_shape(ffo):
    # Sequential schedule, no candidate skipped: per level 4 propagations with 2
    # neighbours each (minus the grid border, where a neighbour is missing) and
    # n_rs random searches per point, plus one re-evaluation per seeded point.
    # For a new level this is the paper's 11 comparisons per point (Sec. 4.1).
    W, H = 37, 29
    I1, I2 = rng_img(31, H, W), rng_img(32, H, W)
    for n in (1, 2, 4):
        C1, C2 = ffo.census(ffo.smooth(I1, n), n), ffo.census(ffo.smooth(I2, n), n)
        Gx, Gy = ffo.grid(W, H, n)
        Gxc, Gyc = ffo.grid(W, H, 2 * n)
        coarse = np.zeros((Gyc, Gxc, 2), np.int32)
        for n_rs in (0, 3):
            _, cost, ev = ffo.search_level(C1, C2, n, 2, flow_coarse=coarse, tile=0, n_rs=n_rs)
            assert ev == 8 * Gx * Gy - 4 * (Gx + Gy) + n_rs * Gx * Gy + Gxc * Gyc
            assert (cost != UNSET).all()
    # 11 per point in the interior
    assert 8 + 3 == 11


def _line_search(ffo, L, vertical, tile):
    """Level search (n = 1, r = 1, no random search) on a line of L grid points
    where only point 0 holds a flow; returns which points hold one afterwards and
    the flows."""
    rng = np.random.default_rng(6)
    W, H = (1, L) if vertical else (L, 1)
    Cs = rng.integers(0, 1 << 24, size=(H, W)).astype(np.uint32)
    Ct = rng.integers(0, 1 << 24, size=(H, W)).astype(np.uint32)
    flow = np.zeros((H, W, 2), np.int32)
    cost = np.full((H, W), 0x7fffffff, np.int32)
    f0 = (0, 1) if vertical else (1, 0)
    flow[0, 0] = f0
    cost[0, 0] = 0
    fl, co, _ = ffo.search_level(Cs, Ct, 1, 1, flow=flow, cost=cost, tile=tile, n_rs=0)
    return [c != 0x7fffffff for c in co.reshape(-1)], fl.reshape(-1, 2), f0


def test_tiled_schedule_two_tile_hand_case(ffo):
    """Sec. 3.1 propagation in the tiled schedule (T = 2, no random search) on a
    line of grid points where only point 0 holds a flow. Worked out by hand from
    the rules: a source in another tile is read from the start-of-pass state, odd
    passes shift the tiles by T / 2. Horizontal sources: pass 0 left, 1 right,
    2 right, 3 left; vertical: 0 up, 1 down, 2 up, 3 down.
    Horizontal line of 4:
      pass 0 (left, tiles {0,1} {2,3}): 1 takes 0's flow; 2 reads 1 from the
             start-of-pass state (unset), so 2 and 3 stay unset.
      passes 1, 2 (right): every right-hand source of 2 and 3 is unset.
      pass 3 (left, tiles {0} {1,2} {3}): 2 takes 1's flow inside its tile; 3
             reads 2 from the start-of-pass state (unset).
      -> 0, 1, 2 set, 3 unset. Without the start-of-pass rule (pass 0) or without
      the shift (pass 3: tiles {0,1} {2,3}) all four would be set.
    Vertical line of 8:
      pass 0 (up, tiles {0,1} {2,3} ...): 1 set; 2 reads 1 from the start-of-pass
             state: unset.
      pass 1 (down): nothing below is set.
      pass 2 (up, tiles {0,1} {2,3} {4,5} {6,7}): 2 reads 1 (set at the start of
             the pass) and 3 follows inside the tile; 4 reads 3 from the
             start-of-pass state: unset.
      pass 3 (down): nothing below is set.
      -> 0..3 set, 4..7 unset.
    The paper's sequential scan sets every point in both cases."""
    got, fl, f0 = _line_search(ffo, 4, False, 2)
    assert got == [True, True, True, False]
    assert all(tuple(fl[i]) == f0 for i in range(3))
    got, fl, f0 = _line_search(ffo, 8, True, 2)
    assert got == [True] * 4 + [False] * 4
    assert all(tuple(fl[i]) == f0 for i in range(4))
    for L, vertical in ((4, False), (8, True)):
        assert all(_line_search(ffo, L, vertical, 0)[0])


def test_random_search_radius_scales_with_the_level(ffo):
    # Sec. 3.2: the random-search radius at spacing n is R_n = R n. From an all-zero
    # field on a pair shifted by 4 px, at n = 4 with R = 1, propagation alone keeps
    # the zero flow; only offsets of up to +-4 px reach the true flow, and
    # propagation then spreads it. With an unscaled radius (+-1) it is never found.
    W, H, n, sh = 128, 96, 4, 4
    canvas = synth._to_u8(synth.value_noise(np.random.default_rng(3), H + 40, W + 40))
    I1 = canvas[20:20 + H, 20:20 + W]
    I2 = canvas[20:20 + H, 20 - sh:20 - sh + W]
    C1, C2 = ffo.census(ffo.smooth(I1, n), n), ffo.census(ffo.smooth(I2, n), n)
    Gxc, Gyc = ffo.grid(W, H, 2 * n)
    Gx, Gy = ffo.grid(W, H, n)
    inner = np.zeros((Gy, Gx), bool)
    inner[2:-2, 2:-3] = True
    for seed in (0, 1):
        f, _, _ = ffo.search_level(C1, C2, n, 2, flow_coarse=np.zeros((Gyc, Gxc, 2), np.int32),
                                   tile=16, n_rs=3, R=1, seed=seed, flow_id=0)
        assert ((f[..., 0] == sh) & (f[..., 1] == 0))[inner].mean() >= 0.9


def test_tiled_schedule_reduces_to_sequential(ffo):
    # tiled(T) with T >= 2 max(Gx, Gy) keeps the whole grid in one tile in every
    # pass (odd passes shift the origin by T/2), so it equals the sequential scan.
    p = synth.pair_shift(5, W=48, H=40, max_shift=(6, 6), square=12, square_move=5)
    for n in (1, 2):
        C1 = ffo.census(ffo.smooth(p["I1"], n), n)
        C2 = ffo.census(ffo.smooth(p["I2"], n), n)
        Gx, Gy = ffo.grid(48, 40, n)
        Gxc, Gyc = ffo.grid(48, 40, 2 * n)
        coarse = np.random.default_rng(n).integers(-5, 6, size=(Gyc, Gxc, 2)).astype(np.int32)
        a = ffo.search_level(C1, C2, n, 3, flow_coarse=coarse, tile=0, seed=9)
        b = ffo.search_level(C1, C2, n, 3, flow_coarse=coarse, tile=2 * max(Gx, Gy), seed=9)
        c = ffo.search_level(C1, C2, n, 3, flow_coarse=coarse, tile=4, seed=9)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert (c[1] != UNSET).all()


def test_search_never_increases_cost_and_costs_are_exact(ffo):
    p = synth.pair_shift(8, W=40, H=36, max_shift=(5, 5), square=10, square_move=6)
    n, r = 2, 3
    C1 = ffo.census(ffo.smooth(p["I1"], n), n)
    C2 = ffo.census(ffo.smooth(p["I2"], n), n)
    Gx, Gy = ffo.grid(40, 36, n)
    rng = np.random.default_rng(0)
    flow = rng.integers(-4, 5, size=(Gy, Gx, 2)).astype(np.int32)
    ys, xs = np.mgrid[0:Gy, 0:Gx] * n
    flow[..., 0] = np.clip(xs + flow[..., 0], 0, 39) - xs
    flow[..., 1] = np.clip(ys + flow[..., 1], 0, 35) - ys
    cost = np.array([[ffo.patch_cost(C1, C2, n, r, (x, y), (x + flow[j, i, 0], y + flow[j, i, 1]))
                      for i, x in enumerate(range(0, 40, n))] for j, y in enumerate(range(0, 36, n))],
                    np.int32)
    f2, c2, _ = ffo.search_level(C1, C2, n, r, flow=flow, cost=cost, tile=8, seed=3)
    assert np.all(c2 <= cost)
    for j in range(Gy):
        for i in range(Gx):
            x, y = i * n, j * n
            tx, ty = x + f2[j, i, 0], y + f2[j, i, 1]
            assert 0 <= tx < 40 and 0 <= ty < 36
            assert c2[j, i] == ffo.patch_cost(C1, C2, n, r, (x, y), (tx, ty))


def test_two_seed_spread(ffo):
    # Fig. 5a analogue: one level initialised with only two flows; propagation
    # and random search spread the true motion over nearly the whole image.
    W, H = 96, 72
    canvas = synth._to_u8(synth.value_noise(np.random.default_rng(4), H + 40, W + 40))
    dx, dy = 7, -5
    I1 = canvas[20:20 + H, 20:20 + W]
    I2 = canvas[20 - dy:20 - dy + H, 20 - dx:20 - dx + W]
    C1, C2 = ffo.census(I1, 1), ffo.census(I2, 1)
    flow = np.zeros((H, W, 2), np.int32)
    cost = np.full((H, W), UNSET, np.int32)
    for (x, y, f) in [(30, 30, (dx, dy)), (60, 50, (dx + 30, dy - 20))]:
        flow[y, x] = f
        cost[y, x] = ffo.patch_cost(C1, C2, 1, 4, (x, y), (x + f[0], y + f[1]))
    f2, c2, _ = ffo.search_level(C1, C2, 1, 4, flow=flow, cost=cost, tile=0, n_rs=3)
    ys, xs = np.mgrid[0:H, 0:W]
    inside = (xs + dx >= 0) & (xs + dx < W) & (ys + dy >= 0) & (ys + dy < H)
    ok = (f2[..., 0] == dx) & (f2[..., 1] == dy)
    assert ok[inside].mean() > 0.9


def test_pure_translation_recovered_and_consistent(ffo):
    # Whole pipeline on a pure integer translation drawn from a larger canvas:
    # the true flow has E_d = 0, so it must be found wherever the patch stays
    # inside both frames, and the consistency check must keep those pixels.
    W, H, dx, dy = 80, 64, 5, -3
    canvas = synth._to_u8(synth.value_noise(np.random.default_rng(1), H + 40, W + 40))
    I1 = canvas[20:20 + H, 20:20 + W]
    I2 = canvas[20 - dy:20 - dy + H, 20 - dx:20 - dx + W]
    res = ffo.flow_fields(I1, I2, params=dict(k=2, r=4, r2=3, tile=16))
    F = res["flows"][0]
    m = 4 * 4  # patch reach at the finest levels used for the decision
    ys, xs = np.mgrid[0:H, 0:W]
    inner = (xs >= m) & (xs < W - m) & (ys >= m) & (ys < H - m) & \
            (xs + dx >= m) & (xs + dx < W - m) & (ys + dy >= m) & (ys + dy < H - m)
    ok = (F[..., 0] == dx) & (F[..., 1] == dy)
    assert ok[inner].mean() >= 0.99
    assert res["valid"][inner & ok].mean() >= 0.99


def test_hierarchy_removes_background_outliers(ffo):
    # Sec. 3.2: hierarchy levels act as outlier sieves, so on the large smoothly
    # moving background the hierarchical search (k=3) leaves no more outliers
    # than the basic approach (k=0). The 32x32 square of these pairs is smaller
    # than the coarse patches (radius 8n), so it is left out of this comparison.
    out = {0: [], 3: []}
    for seed in range(4):
        p = synth.workload_pair("noise_128x96", 100 + seed)
        px, py = p["square_pos"]
        bg = ~p["occ"]
        bg[max(py - 8, 0):py + 40, max(px - 8, 0):px + 40] = False
        for k in (0, 3):
            F = ffo.flow_fields(p["I1"], p["I2"], params=dict(k=k))["flows"][0]
            epe = np.hypot(*(F - p["flow"]).transpose(2, 0, 1))
            out[k].append((epe[bg] > 3).mean())
    assert np.mean(out[3]) <= np.mean(out[0])


# ------------------------------------------------------------- filters ---------
def test_consistency_exact_inverse_and_symmetry(ffo):
    W, H = 20, 16
    ys, xs = np.mgrid[0:H, 0:W]
    F = np.zeros((H, W, 2), np.int32)
    F[..., 0] = np.where(xs < 17, 3, 0)
    Fb = np.zeros_like(F)
    Fb[..., 0] = np.where(xs >= 3, -3, 0)
    v, e = ffo.consistency(F, Fb, Fb, 1)
    # exact inverse wherever the backward flow at the target is -F
    good = (xs < 17)
    assert v[good].all() and (e[good] == 0).all()
    # swapping the two backward flows changes nothing
    Fb2 = Fb.copy()
    Fb2[..., 1] = 1
    a = ffo.consistency(F, Fb, Fb2, 2)
    b = ffo.consistency(F, Fb2, Fb, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # hand values: |(3,0)+(-3,1)|^2 = 1 -> kept for eps 2, dropped for eps 1
    assert a[0][0, 0] == 1 and a[1][0, 0] == 1
    assert ffo.consistency(F, Fb, Fb2, 1)[0][0, 0] == 0
    # strict inequality on the norm: error exactly eps is rejected
    Fb3 = Fb.copy()
    Fb3[..., 1] = 2
    assert ffo.consistency(F, Fb3, Fb3, 2)[0][0, 0] == 0
    # mirrored problem gives the mirrored mask
    Fm, Fbm = F[:, ::-1].copy(), Fb2[:, ::-1].copy()
    Fm[..., 0] *= -1
    Fbm[..., 0] *= -1
    c = ffo.consistency(Fm, Fbm, Fbm, 2)
    d = ffo.consistency(F, Fb2, Fb2, 2)
    assert np.array_equal(c[0], d[0][:, ::-1])


def test_region_filter_hand_cases(ffo):
    W, H = 12, 6
    F = np.zeros((H, W, 2), np.int32)
    vcc = np.ones((H, W), np.uint8)
    # region A: 3 pixels with flow (10, 0), touching a removed outlier whose flow
    # is (11, 1) (|diff|^2 = 2 < 9): deleted
    F[1, 1:4] = (10, 0)
    F[1, 4] = (11, 1)
    vcc[1, 4] = 0
    # region B: 2 pixels with flow (20, 0) next to a removed pixel with flow (0, 0)
    # (far): kept
    F[4, 8:10] = (20, 0)
    vcc[4, 10] = 0
    # region C: 1 pixel (30, 0) touching a close removed pixel only diagonally: kept
    F[4, 1] = (30, 0)
    F[3, 2] = (30, 1)
    vcc[3, 2] = 0
    F[3, 1] = (50, 0)
    F[4, 2] = (60, 0)
    out = ffo.region_filter(F, vcc, 5)
    assert not out[1, 1:4].any()
    assert out[4, 8:10].all()
    assert out[4, 1] == 1
    # the large background region (flow 0) touches removed pixel (4,10) with flow
    # (0,0) but has >= s pixels: kept
    assert out[0, 0] == 1
    # with s = 1 nothing is small enough to be deleted
    assert np.array_equal(ffo.region_filter(F, vcc, 1), vcc)
    # removed pixels stay removed
    assert out[1, 4] == 0 and out[4, 10] == 0


def test_sparsify_hand_cases(ffo):
    W, H = 7, 4  # blocks: 3 x 2, partial ones on the right and bottom
    valid = np.zeros((H, W), np.uint8)
    err = np.full((H, W), 50, np.int32)
    F = np.zeros((H, W, 2), np.int32)
    F[..., 0] = np.arange(W)[None, :]
    F[..., 1] = np.arange(H)[:, None]
    valid[0:3, 0:3] = 1
    err[1, 2] = 3
    err[2, 0] = 3  # tie with (2,1): raster-first wins -> (2, 1)
    valid[0:2, 3:6] = 1  # 6 valid, all err 50 -> first in raster order (3, 0)
    valid[3, 6] = 1  # partial block (6..6, 3..3) with 1 valid: needs e <= 1
    zero = np.zeros_like(err)
    sp, mask = ffo.sparsify(valid, err, zero, F, 4)
    assert sp.tolist() == [[2, 1, 2, 1], [3, 0, 3, 0]]
    assert mask.sum() == 2
    sp1, _ = ffo.sparsify(valid, err, zero, F, 1)
    assert sp1.tolist()[-1] == [6, 3, 6, 3]


def test_sparsify_takes_the_sum_of_the_two_errors(ffo):
    """Sec. 3.5 keeps the sample whose two consistency-check errors |.| (Eq. 5) sum
    to the least: sqrt(e1) + sqrt(e2), not e1 + e2. Blocks where the two readings
    disagree, and exact ties (rational and irrational) that go to raster order."""
    W, H = 9, 3
    valid = np.zeros((H, W), np.uint8)
    e1 = np.zeros((H, W), np.int32)
    e2 = np.zeros((H, W), np.int32)
    F = np.zeros((H, W, 2), np.int32)
    F[..., 0] = np.arange(W)[None, :]
    # block 0: (0, 25) at x = 1 -> 5 beats (9, 9) at x = 0 -> 6, although 25 > 18
    valid[0, 0] = valid[0, 1] = 1
    e1[0, 1], e2[0, 1] = 0, 25
    e1[0, 0], e2[0, 0] = 9, 9
    # block 1: sqrt(4) + sqrt(9) = sqrt(1) + sqrt(16) = 5: tie, raster-first (3, 0)
    valid[0, 3] = valid[0, 4] = 1
    e1[0, 3], e2[0, 3] = 4, 9
    e1[0, 4], e2[0, 4] = 1, 16
    # block 2: sqrt(2) + sqrt(8) = sqrt(18) = 3 sqrt(2): tie, raster-first (7, 0);
    # sqrt(17) < 3 sqrt(2) wins the block from row 2
    valid[0, 7] = valid[0, 8] = valid[2, 6] = 1
    e1[0, 7], e2[0, 7] = 2, 8
    e1[0, 8], e2[0, 8] = 18, 0
    e1[2, 6], e2[2, 6] = 17, 0
    sp, _ = ffo.sparsify(valid, e1, e2, F, 1)
    assert sp[:, :2].tolist() == [[1, 0], [3, 0], [6, 2]]
    e2[2, 6] = 1  # sqrt(17) + 1 > 3 sqrt(2): the tie (7, 0) / (8, 0) decides
    sp, _ = ffo.sparsify(valid, e1, e2, F, 1)
    assert sp[:, :2].tolist() == [[1, 0], [3, 0], [7, 0]]


def test_sqrt_sum_comparator_against_high_precision(ffo):
    """The exact integer comparison of sqrt(a) + sqrt(b) and sqrt(c) + sqrt(d)
    against 60-digit decimal square roots. For integers below 2^20 a nonzero
    difference exceeds 1e-30, so smaller differences are ties."""
    import decimal
    decimal.getcontext().prec = 60
    D = decimal.Decimal

    def ref(a, b, c, d):
        diff = (D(c).sqrt() + D(d).sqrt()) - (D(a).sqrt() + D(b).sqrt())
        return diff > D("1e-30")

    rng = np.random.default_rng(5)
    cases = [tuple(int(v) for v in rng.integers(0, 1 << 20, size=4)) for _ in range(3000)]
    cases += [tuple(int(v) for v in rng.integers(0, 40, size=4)) for _ in range(3000)]
    # near-ties: c, d perturbed around a, b
    for _ in range(2000):
        a, b = (int(v) for v in rng.integers(0, 1 << 20, size=2))
        cases.append((a, b, max(0, a + int(rng.integers(-2, 3))), max(0, b + int(rng.integers(-2, 3)))))
    cases += [(4, 9, 1, 16), (1, 16, 4, 9), (2, 8, 18, 0), (18, 0, 2, 8), (0, 0, 0, 0),
              (12, 3, 27, 0), (27, 0, 12, 3), (5, 5, 20, 0), (0, 20, 5, 5), (50, 0, 2, 32)]
    for a, b, c, d in cases:
        assert ffo.sqrt_sum_less(a, b, c, d) == ref(a, b, c, d), (a, b, c, d)


# ------------------------------------------------------------- smoothing -------
def test_area_down_block_means(ffo):
    W, H = 10, 7
    img = np.zeros((H, W, 3), np.uint8)
    img[..., 0] = np.arange(W)[None, :] * 10
    img[..., 1] = np.arange(H)[:, None] * 20
    img[..., 2] = 7
    d = ffo.area_down(img, 4)
    # block x in [4, 8): mean of 40..70 = 55; last block x in [8, 10): mean 85
    assert d[0, 1, 0] == 55 and d[0, 2, 0] == 85
    # rows [4, 7): mean of 80, 100, 120 = 100
    assert d[1, 0, 1] == 100
    assert (d[..., 2] == 7).all()
    # rounding half up: mean of 0 and 1 over a 2-pixel partial block
    img2 = np.zeros((1, 3, 3), np.uint8)
    img2[0, 2] = 1
    assert ffo.area_down(img2, 2)[0, 1, 0] == 1  # (1 + 0) / 1
    img3 = np.zeros((2, 2, 3), np.uint8)
    img3[0, 0] = 2
    assert ffo.area_down(img3, 2)[0, 0, 0] == 1  # (2 + 2) // 4


def test_lanczos_table_properties(ffo):
    for n in (2, 4, 8):
        base, w = ffo.lanczos_table(n)
        assert (w.sum(1) == 16384).all()
        # mirror symmetry of the phases: phase phi and n-1-phi are reflections
        for phi in range(n):
            assert np.array_equal(w[phi], w[n - 1 - phi][::-1])
        # agrees with the textbook Lanczos-3 kernel sinc(t) sinc(t/3), normalised,
        # to within the Q14 rounding (+ the residual on the largest tap)
        for phi in range(n):
            u = (2 * phi - n + 1) / (2 * n)
            j0 = int(np.floor(u))
            assert base[phi] == j0
            t = (u - j0) - np.arange(-2, 4)
            ref = np.sinc(t) * np.sinc(t / 3)
            ref = 16384 * ref / ref.sum()
            assert np.abs(w[phi] - ref).max() <= 2


def test_smooth_preserves_constants_and_is_a_lowpass(ffo):
    for n in (2, 4, 8):
        img = np.full((21, 34, 3), 123, np.uint8)
        assert (ffo.smooth(img, n) == 123).all()
    # high-frequency checkerboard loses most of its contrast
    ys, xs = np.mgrid[0:32, 0:32]
    chk = np.repeat((((xs + ys) % 2) * 200 + 20).astype(np.uint8)[..., None], 3, 2)
    s = ffo.smooth(chk, 4)
    assert s[8:24, 8:24].std() < 0.05 * chk.std()
    assert abs(int(s[8:24, 8:24].mean()) - 120) <= 2


# ------------------------------------------------------------- CIELab ----------
def test_lab_decoding_table_and_matrix(ffo):
    """Step 1 and 2 of the integer CIELab: the linear branch of the sRGB decoding
    curve in closed form, the end points, monotonicity; matrix rows that sum to
    exactly 16384 and stay within one unit of the published IEC 61966-2-1 matrix
    divided by the D65 white."""
    from fractions import Fraction
    t = ffo.lab_gamma_table()
    assert t[0] == 0 and t[255] == 65536
    assert np.all(np.diff(t) > 0)
    for v in range(11):  # v / 255 <= 0.04045: linear segment c / 12.92
        x = Fraction(65536 * v * 100, 255 * 1292) + Fraction(1, 2)
        assert t[v] == x.numerator // x.denominator
    m = ffo.lab_matrix()
    assert np.all(m.sum(1) == 16384)
    M = np.array([[0.4124, 0.3576, 0.1805], [0.2126, 0.7152, 0.0722], [0.0193, 0.1192, 0.9505]])
    assert np.all(np.abs(m - M / M.sum(1, keepdims=True) * 16384) <= 1.0)


def test_lab_transfer_exact(ffo):
    """Step 3: the cube-root branch is the exact integer cube root of t * 2^32;
    below (6/29)^3 the line t / (3 (6/29)^2) + 4/29 (Q16, rounded)."""
    from fractions import Fraction
    assert ffo.lab_f(65536) == 65536
    assert ffo.lab_f(0) == 9039  # round(65536 * 4 / 29)
    rng = np.random.default_rng(7)
    for t in list(range(570, 600)) + [int(x) for x in rng.integers(581, 65537, size=400)]:
        y = ffo.lab_f(t)
        if t * 29 ** 3 > 6 ** 3 * 65536:
            assert y ** 3 <= t << 32 < (y + 1) ** 3, t
        else:
            x = Fraction(t, 65536) / (3 * Fraction(6, 29) ** 2) + Fraction(4, 29)
            x = x * 65536 + Fraction(1, 2)
            assert y == x.numerator // x.denominator, t


def test_lab_grey_white_black_and_primaries(ffo):
    """Step 4: greys have a = b = 0 exactly (128), white is L = 100 (255), black
    L = 0; the sRGB primaries land within one unit of their published CIELab
    (D65) values: red (53.24, 80.09, 67.20), green (87.73, -86.18, 83.18), blue
    (32.30, 79.19, -107.86)."""
    grey = np.repeat(np.arange(256, dtype=np.uint8)[None, :, None], 3, axis=2)
    lab = ffo.rgb_to_lab(grey)[0]
    assert np.all(lab[:, 1] == 128) and np.all(lab[:, 2] == 128)
    assert lab[0, 0] == 0 and lab[255, 0] == 255
    assert np.all(np.diff(lab[:, 0].astype(int)) >= 0)
    prim = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255]]], np.uint8)
    got = ffo.rgb_to_lab(prim)[0].astype(float)
    want = np.array([[53.24, 80.09, 67.20], [87.73, -86.18, 83.18], [32.30, 79.19, -107.86]])
    enc = np.stack([want[:, 0] * 2.55, want[:, 1] + 128, want[:, 2] + 128], 1)
    assert np.all(np.abs(got - enc) <= 1.0), (got, enc)


def test_lab_against_float_formula(ffo):
    """The integer conversion against the CIELab formulas in float64 on random
    colours: every channel within one unit (the fixed-point rounding)."""
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, size=(64, 128, 3)).astype(np.uint8)
    got = ffo.rgb_to_lab(img).astype(float)
    c = img.astype(float) / 255.0
    lin = np.where(c <= 0.04045, c / 12.92, ((c + 0.055) / 1.055) ** 2.4)
    M = np.array([[0.4124, 0.3576, 0.1805], [0.2126, 0.7152, 0.0722], [0.0193, 0.1192, 0.9505]])
    xyz = lin @ (M / M.sum(1, keepdims=True)).T
    d = 6.0 / 29.0
    f = np.where(xyz > d ** 3, np.cbrt(xyz), xyz / (3 * d * d) + 4.0 / 29.0)
    L = 116 * f[..., 1] - 16
    a = 500 * (f[..., 0] - f[..., 1])
    b = 200 * (f[..., 1] - f[..., 2])
    want = np.stack([np.clip(L * 2.55, 0, 255), np.clip(a + 128, 0, 255), np.clip(b + 128, 0, 255)], -1)
    assert np.max(np.abs(got - want)) <= 1.0


# ------------------------------------------------- weighted median field -------
def test_weighted_median_reduces_to_median_and_follows_weights(ffo):
    """The weighted median of the "k=3+median" field: with equal matching errors
    it is the plain lower median of the in-image window (numpy, brute force); a
    constant field is a fixed point; one pixel whose weight outweighs the rest of
    its window wins it; an isolated outlier in a smooth field is replaced."""
    rng = np.random.default_rng(9)
    H, W = 11, 13
    F = rng.integers(-20, 21, size=(H, W, 2)).astype(np.int32)
    E = np.full((H, W), 37, np.int32)
    got = ffo.weighted_median(F, E, 2)
    for y in range(H):
        for x in range(W):
            win = F[max(0, y - 2):y + 3, max(0, x - 2):x + 3].reshape(-1, 2)
            srt = np.sort(win, axis=0)
            k = (len(win) - 1) // 2  # lower median: first value with 2 * count >= total
            assert tuple(got[y, x]) == (srt[k, 0], srt[k, 1]), (y, x)
    const = np.full((H, W, 2), 7, np.int32)
    assert np.array_equal(ffo.weighted_median(const, E, 2), const)
    E2 = np.full((H, W), 6000, np.int32)
    E2[5, 6] = 0  # weight 65536 against 24 * 10
    got2 = ffo.weighted_median(F, E2, 2)
    assert tuple(got2[5, 6]) == tuple(F[5, 6])
    smooth = np.zeros((H, W, 2), np.int32)
    smooth[..., 0] = 3
    smooth[6, 6] = (40, -30)
    assert np.array_equal(ffo.weighted_median(smooth, E, 1)[6, 6], [3, 0])


def test_match_errors_are_the_data_term(ffo):
    """E(p) is E_d of the pixel's own flow at full resolution: zero for a frame
    paired with itself under the zero flow; equal to patch_cost otherwise."""
    rng = np.random.default_rng(10)
    I1 = rng.integers(0, 256, size=(20, 24, 3)).astype(np.uint8)
    I2 = rng.integers(0, 256, size=(20, 24, 3)).astype(np.uint8)
    Z = np.zeros((20, 24, 2), np.int32)
    assert np.all(ffo.match_errors(I1, I1, Z, 3) == 0)
    F = rng.integers(-4, 5, size=(20, 24, 2)).astype(np.int32)
    F[..., 0] = np.clip(np.arange(24)[None, :] + F[..., 0], 0, 23) - np.arange(24)[None, :]
    F[..., 1] = np.clip(np.arange(20)[:, None] + F[..., 1], 0, 19) - np.arange(20)[:, None]
    E = ffo.match_errors(I1, I2, F, 3)
    C1, C2 = ffo.census(I1, 1), ffo.census(I2, 1)
    for (y, x) in [(0, 0), (5, 7), (19, 23), (10, 12)]:
        assert E[y, x] == ffo.patch_cost(C1, C2, 1, 3, (x, y), (x + F[y, x, 0], y + F[y, x, 1]))


# ------------------------------------------------ subpixel random search -------
def _subpel_pair(q, axis, seed=11, W=96, H=72):
    """Frame 1 is frame 2 sampled 1/q pixel further along `axis` (0: x, 1: y), with
    frame 2 quantised so that the sample ((q - 1) I2(p) + I2(p + e)) / q is an
    exact integer: the forward flow is 1/q pixel, i.e. 1 in units of 1/q."""
    rng = np.random.default_rng(seed)
    v = synth.value_noise(rng, H, W, lattices=(16, 8, 4), amps=(0.5, 0.25, 0.125))
    I2 = (np.floor(v * (255 // q)) * q).astype(np.int64)  # multiples of q
    nxt = np.concatenate([I2[:, 1:], I2[:, -1:]], 1) if axis == 0 else \
        np.concatenate([I2[1:], I2[-1:]], 0)
    I1 = ((q - 1) * I2 + nxt) // q
    return I1.astype(np.uint8), I2.astype(np.uint8)


def test_subpel_census_phase_zero_is_the_census(ffo):
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, size=(17, 23, 3)).astype(np.uint8)
    for n in (1, 2, 4):
        for q in (2, 4):
            assert np.array_equal(ffo.census_subpel(img, n, q, 0, 0), ffo.census(img, n))


@pytest.mark.parametrize("q,axis", [(2, 0), (2, 1), (4, 0)])
def test_subpixel_translation_is_recovered(ffo, q, axis):
    """Sec. 3.1, subpixel random search with bilinear target colours: on a pair
    whose true flow is exactly 1/q pixel, the census of frame 2 interpolated at the
    subpixel target equals frame 1's, so that flow has zero matching error and no
    integer flow has. The search with subpel = q finds it (1 in units of 1/q) at
    interior pixels; with integer flows (subpel = 1) it cannot."""
    I1, I2 = _subpel_pair(q, axis)
    m = np.zeros(I1.shape[:2], bool)
    m[10:-10, 10:-10] = True
    want = np.zeros(2, np.int32)
    want[axis] = 1
    out = ffo.flow_fields(I1, I2, params=dict(subpel=q), threads=3)
    f = out["flows"][0]
    hit = np.all(f == want, axis=-1)[m].mean()
    assert hit > 0.95, hit
    C1 = ffo.census(I1, 1)
    for (y, x) in [(20, 30), (40, 50)]:  # zero matching error at the true subpixel target
        Cq = ffo.census_subpel(I2, 1, q, want[0], want[1])
        assert ffo.patch_cost(C1, Cq, 1, 8, (x, y), (x, y)) == 0
    # integer flows can only take the neighbouring whole pixels, 0 or 1 px along the axis
    f1 = ffo.flow_fields(I1, I2, params=dict(subpel=1), threads=3)["flows"][0]
    assert np.isin(f1[m][:, axis], [0, 1]).mean() > 0.9


def test_subpel_filter_thresholds(ffo):
    """Eq. 5 and the region rule in units of 1/q pixel: a backward flow read at the
    nearest pixel of a half-pixel target, eps and the 3-pixel region threshold
    scaled by q."""
    H, W = 6, 8
    F = np.zeros((H, W, 2), np.int32)
    F[..., 0] = 1  # +0.5 px with q = 2: target x + 0.5 rounds up to x + 1
    Fb = np.zeros((H, W, 2), np.int32)
    Fb[..., 0] = -1
    v, e = ffo.consistency(F, Fb, Fb, 1, subpel=2)
    assert np.all(v[:, :W - 1] == 1) and np.all(e[:, :W - 1] == 0)
    assert np.all(v[:, W - 1] == 0)  # x + 1 = W: outside
    Fb2 = Fb.copy()
    Fb2[..., 0] = -4  # error 3 half pixels = 1.5 px: passes eps = 2, fails eps = 1
    assert np.all(ffo.consistency(F, Fb2, Fb2, 2, subpel=2)[0][:, :W - 1] == 1)
    assert np.all(ffo.consistency(F, Fb2, Fb2, 1, subpel=2)[0][:, :W - 1] == 0)
    # region rule: flows differing by 2.5 px (5 half pixels) are neighbours, 3 px not
    G = np.zeros((1, 3, 2), np.int32)
    G[0, 1, 0] = 5
    G[0, 2, 0] = 11
    vcc = np.array([[1, 1, 0]], np.uint8)
    out = ffo.region_filter(G, vcc, 5, subpel=2)
    assert out.tolist() == [[1, 1, 0]]  # (1, 2) differ by 3 px: no touch, region kept
    G[0, 2, 0] = 10  # 2.5 px: the rejected pixel touches the region -> removed
    assert ffo.region_filter(G, vcc, 5, subpel=2).tolist() == [[0, 0, 0]]


def _assert_filter_composed(ffo, res, eps, s, e):
    """valid, err_sum, sparse and mask of a whole-path result equal Eq. 5 against
    both backward flows, the region filter and the sparsification composed by hand
    on its flows (Sec. 3.4, 3.5)."""
    F, Fb1, Fb2 = res["flows"]
    v, err, e1, e2 = ffo.consistency(F, Fb1, Fb2, eps, errors=True)
    valid = ffo.region_filter(F, v, s)
    sp, mask = ffo.sparsify(valid, e1, e2, F, e)
    assert np.array_equal(valid, res["valid"])
    assert np.array_equal(err, res["err_sum"])
    assert np.array_equal(sp, res["sparse"]) and np.array_equal(mask, res["mask"])


@pytest.mark.parametrize("color", [0, 1])
def test_whole_path_is_the_composition_of_its_steps(ffo, color):
    # Fig. 2 / Sec. 3.4 wiring: (with color = 1 both frames in CIELab first); per
    # level the census of I^n; forward flow I1 -> I2 and first backward flow with
    # radius r, second backward flow with r2, each from a kd tree over the target
    # frame's WHT features, flow ids 0, 1, 2. Each flow must equal its steps
    # composed by hand.
    W, H = 56, 44
    rng = np.random.default_rng(41)
    I1 = synth._to_u8(synth.value_noise(rng, H, W))
    I2 = synth._to_u8(synth.value_noise(rng, H, W))
    P = dict(k=2, r=3, r2=2, tile=8, n_rs=2, R=1, seed=9, color=color)
    res = ffo.flow_fields(I1, I2, params=P)
    A = (ffo.rgb_to_lab(I1), ffo.rgb_to_lab(I2)) if color else (I1, I2)
    Cn = {(f, n): ffo.census(ffo.smooth(A[f], n), n) for f in (0, 1) for n in (1, 2, 4)}
    for j, (src, tgt, r) in enumerate(((0, 1, 3), (1, 0, 3), (1, 0, 2))):
        f, c, _ = ffo.kd_init(ffo.wht_features(A[tgt], r), A[src], r, 8, Cn[(src, 4)],
                              Cn[(tgt, 4)], 4)
        f, c, _ = ffo.search_level(Cn[(src, 4)], Cn[(tgt, 4)], 4, r, flow=f, cost=c, tile=8,
                                   n_rs=2, R=1, seed=9, flow_id=j)
        for n in (2, 1):
            f, c, _ = ffo.search_level(Cn[(src, n)], Cn[(tgt, n)], n, r, flow_coarse=f, tile=8,
                                       n_rs=2, R=1, seed=9, flow_id=j)
        assert np.array_equal(f, res["flows"][j]), j
    _assert_filter_composed(ffo, res, 5, 50, 4)
