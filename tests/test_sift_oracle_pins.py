"""Pins of the oracle's SIFT flow data term (Sec. 3.3) to facts fixed outside it.

The descriptor is checked against closed forms (ramps, constant images), against
the mirror and transpose symmetries any correct layout of cells and orientations
must have, and against an independent float64 statement of Lowe's
normalisation; the moments against brute force; the PCA against the eigen
equation and a planted subspace; the colours against a hand basis; the cost
against the Euclidean norm; the search against a pure translation. No GPU.
"""
import math

import numpy as np

from paper_1508_05151_gb300 import synth

CELL = 3


def rng_img(seed, H, W):
    return np.random.default_rng(seed).integers(0, 256, size=(H, W, 3), dtype=np.uint8)


def smooth_img(seed, H, W):
    return synth._to_u8(synth.value_noise(np.random.default_rng(seed), H, W))


# ------------------------------------------------------------ integer sqrt ----
def test_isqrt_against_math(ffo):
    rng = np.random.default_rng(0)
    xs = [0, 1, 2, 3, 4, 15, 16, 17, 2**32 - 1, 2**32, 2**52 + 1, 2**62, 2**64 - 1]
    xs += [int(v) for v in rng.integers(0, 2**62, 200, dtype=np.int64)]
    xs += [k * k + d for k in (1, 7, 2**20, 3037000499) for d in (-1, 0, 1) if k * k + d >= 0]
    for x in xs:
        assert ffo.isqrt(x) == math.isqrt(x)


# ------------------------------------------------------------- orientation ----
def test_orientations_of_ramps_closed_form(ffo):
    # R = G = B = a x: grey 3 a x, interior gx = 6 a, gy = 0. The rectified
    # derivative along k * 45 degrees is 6 a (256, 181, 0, 0, 0, 0, 0, 181).
    a, W, H = 2, 60, 9
    x = np.arange(W)
    img = np.repeat((a * x).astype(np.uint8)[None, :, None], 3, 2).repeat(H, 0)
    o = ffo.sift_orient(img)
    g = 6 * a
    assert (o[:, 1:-1] == np.array([256, 181, 0, 0, 0, 0, 0, 181]) * g).all()
    assert (o[:, 0] == np.array([256, 181, 0, 0, 0, 0, 0, 181]) * 3 * a).all()  # clamped
    # The same ramp along y (y pointing down) peaks at k = 2.
    o = ffo.sift_orient(np.ascontiguousarray(img.transpose(1, 0, 2)))
    assert (o[1:-1, :] == np.array([0, 181, 256, 181, 0, 0, 0, 0]) * g).all()
    # A falling ramp peaks at k = 4 (180 degrees).
    o = ffo.sift_orient(np.ascontiguousarray(img[:, ::-1]))
    assert (o[:, 1:-1] == np.array([0, 0, 0, 181, 256, 181, 0, 0]) * g).all()


def test_descriptor_of_constant_image_is_zero(ffo):
    img = np.full((20, 30, 3), 77, np.uint8)
    assert (ffo.sift_descriptors(img) == 0).all()


def _dview(d):
    H, W = d.shape[:2]
    return d.reshape(H, W, 4, 4, 8)  # [y][x][cell row j][cell column i][orientation k]


def test_descriptor_mirror_and_transpose_symmetry(ffo):
    # A correct layout maps under a flip of x to: the descriptor one pixel to the
    # right of the mirrored pixel (the 4 x 4 window spans offsets -2c .. 2c-1),
    # cell columns reversed, orientation k -> 4 - k; under a flip of y likewise
    # with rows and k -> -k; under a transpose, cells (i, j) -> (j, i) and
    # k -> 2 - k.
    img = smooth_img(3, 37, 41)
    H, W = img.shape[:2]
    d = _dview(ffo.sift_descriptors(img))
    k = np.arange(8)
    df = _dview(ffo.sift_descriptors(np.ascontiguousarray(img[:, ::-1])))
    for xp in range(1, W):
        assert (df[:, xp] == d[:, W - xp][:, :, ::-1][..., (4 - k) % 8]).all()
    dv = _dview(ffo.sift_descriptors(np.ascontiguousarray(img[::-1])))
    for yp in range(1, H):
        assert (dv[yp] == d[H - yp][:, ::-1][..., (8 - k) % 8]).all()
    dt = _dview(ffo.sift_descriptors(np.ascontiguousarray(img.transpose(1, 0, 2))))
    assert (dt == d.transpose(1, 0, 3, 2, 4)[..., (2 - k) % 8]).all()


def test_descriptor_matches_float_statement_of_lowe_normalisation(ffo):
    # Cell sums by numpy slicing of the orientation responses, then unit length,
    # clip at 0.2, unit length, x 512, floor, clamp 255 in float64. Entries whose
    # float value lies within 1e-6 of an integer (or of the clip threshold) are
    # not compared.
    img = rng_img(5, 30, 34)
    H, W = img.shape[:2]
    o = ffo.sift_orient(img).astype(np.int64)
    pad = 2 * CELL
    yy = np.clip(np.arange(-pad, H + pad), 0, H - 1)
    xx = np.clip(np.arange(-pad, W + pad), 0, W - 1)
    op = o[yy][:, xx]
    h = np.zeros((H, W, 4, 4, 8), np.int64)
    for j in range(4):
        for i in range(4):
            for v in range((j - 2) * CELL, (j - 1) * CELL):
                for u in range((i - 2) * CELL, (i - 1) * CELL):
                    h[:, :, j, i] += op[pad + v:pad + v + H, pad + u:pad + u + W]
    h = h.reshape(H, W, 128).astype(np.float64)
    n1 = np.sqrt((h ** 2).sum(-1, keepdims=True))
    u = np.where(n1 > 0, h / np.where(n1 > 0, n1, 1), 0)
    near_clip = np.abs(u - 0.2) < 1e-9
    u = np.minimum(u, 0.2)
    n2 = np.sqrt((u ** 2).sum(-1, keepdims=True))
    v = np.where(n2 > 0, 512 * u / np.where(n2 > 0, n2, 1), 0)
    want = np.minimum(np.floor(v), 255)
    got = ffo.sift_descriptors(img).astype(np.float64)
    ok = (np.abs(v - np.round(v)) > 1e-6) & ~near_clip.any(-1, keepdims=True)
    assert ok.mean() > 0.95
    assert (got[ok] == want[ok]).all()
    assert (np.abs(got - want) <= 1).all()


# ----------------------------------------------------------------- moments ----
def test_moments_brute_force_and_accumulation(ffo):
    rng = np.random.default_rng(2)
    d = rng.integers(0, 256, size=(7, 9, 128), dtype=np.uint8)
    s, g, n = ffo.sift_moments(d)
    x = d.reshape(-1, 128).astype(np.int64)
    assert n == 63
    assert (s.astype(np.int64) == x.sum(0)).all()
    assert (g.astype(np.int64) == x.T @ x).all()
    s2, g2, n2 = ffo.sift_moments(d[:3], acc=ffo.sift_moments(d[3:]))
    assert n2 == 63 and (s2 == s).all() and (g2 == g).all()


# --------------------------------------------------------------------- PCA ----
def test_pca_eigen_equation_and_order(ffo):
    d = ffo.sift_descriptors(smooth_img(7, 40, 48))
    s, g, n = ffo.sift_moments(d)
    P = ffo.sift_pca(s, g, n, 12)
    mu = s.astype(np.float64) / n
    Cm = g.astype(np.float64) / n - np.outer(mu, mu)
    w = P["eigval"]
    assert (np.diff(w) <= 1e-9 * w[0]).all()
    assert abs(w.sum() - np.trace(Cm)) <= 1e-9 * abs(np.trace(Cm))
    gain = 127.0 / (3.0 * math.sqrt(max(w[0], 1.0)))
    E = P["exact"] / (4096.0 * gain)
    assert np.allclose(E @ E.T, np.eye(12), atol=1e-10)
    for sidx in range(12):
        e = E[sidx]
        assert np.linalg.norm(Cm @ e - w[sidx] * e) <= 1e-8 * w[0]
        assert e[np.argmax(np.abs(e))] > 0
    assert (P["basis"] == np.clip(np.floor(P["exact"] + 0.5), -32767, 32767)).all()


def test_pca_recovers_a_planted_subspace(ffo):
    # Descriptors mu + a e1 + b e2 with large independent a, b and small noise:
    # the first two basis vectors span {e1, e2}.
    rng = np.random.default_rng(4)
    e1 = np.zeros(128)
    e1[:8] = 1 / math.sqrt(8)
    e2 = np.zeros(128)
    e2[40:44] = 0.5
    e2[44:48] = -0.5
    N = 5000
    a = rng.uniform(-200, 200, N)
    b = rng.uniform(-100, 100, N)
    x = 128 + a[:, None] * e1 + b[:, None] * e2 + rng.uniform(-2, 2, (N, 128))
    d = np.clip(np.round(x), 0, 255).astype(np.uint8)
    s, g, n = ffo.sift_moments(d.reshape(N, 1, 128))
    P = ffo.sift_pca(s, g, n, 3)
    E = P["exact"][:2] / np.linalg.norm(P["exact"][:2], axis=1, keepdims=True)
    Q = np.stack([e1, e2])
    assert np.linalg.svd(E @ Q.T, compute_uv=False).min() > 0.999
    assert abs(E[0] @ e1) > 0.999  # the larger variance first


# ----------------------------------------------------------------- colours ----
def test_colors_hand_basis_and_centring(ffo):
    rng = np.random.default_rng(9)
    d = rng.integers(0, 128, size=(5, 6, 128), dtype=np.uint8)
    B = np.zeros((6, 128), np.int16)
    for sidx in range(6):
        B[sidx, 3 * sidx] = 4096  # channel s = descriptor entry 3 s
    col = ffo.sift_colors(d, B, np.zeros(6, np.int32))
    assert col.shape == (2, 5, 6, 3)
    for sidx in range(6):
        assert (col[sidx // 3, :, :, sidx % 3] == np.minimum(128 + d[:, :, 3 * sidx], 255)).all()
    # Offsets centre the mean: a descriptor equal to an integral mean maps to 128.
    mean = rng.integers(0, 256, 128)
    rows = np.stack([mean + t for t in (-3, 3)]).clip(0, 255)
    rows[:, mean < 3] = mean[mean < 3]
    rows[:, mean > 252] = mean[mean > 252]
    s = rows.astype(np.uint64).sum(0)
    Bq = rng.integers(-3000, 3000, (9, 128)).astype(np.int16)
    off = ffo.sift_pca_offset(Bq, s, 2)
    col = ffo.sift_colors(mean.astype(np.uint8).reshape(1, 1, 128), Bq, off)
    assert (col == 128).all()


def test_pca_offsets_centre_a_fractional_mean(ffo):
    # Over the descriptors the offsets were fitted on, the mean unfloored projection
    # B q + o equals B mu + o, which rounding B mu half up puts in (2048 - 1/2,
    # 2048 + 1/2] (exact fractions; 3 descriptors give a mean in thirds).
    from fractions import Fraction
    rng = np.random.default_rng(13)
    rows = rng.integers(0, 256, size=(3, 128))
    s = rows.astype(np.uint64).sum(0)
    B = rng.integers(-3000, 3000, (9, 128)).astype(np.int16)
    off = ffo.sift_pca_offset(B, s, 3)
    fr = []
    for k in range(9):
        m = Fraction(int(np.dot(B[k].astype(np.int64), s.astype(np.int64))), 3) + int(off[k])
        assert Fraction(-1, 2) < m - 2048 <= Fraction(1, 2)
        fr.append(m - 2048)
    assert any(abs(f) > Fraction(1, 4) for f in fr)  # the case is not trivially integral


# -------------------------------------------------------------------- cost ----
def test_tap_is_fixed_point_euclidean_norm(ffo):
    a = np.zeros(12, np.uint8)
    b = np.zeros(12, np.uint8)
    b[0], b[4] = 3, 4
    assert ffo.sift_tap(a, b) == 80
    b[:] = 0
    b[11] = 255
    assert ffo.sift_tap(a, b) == 16 * 255
    rng = np.random.default_rng(1)
    for S in (3, 12, 18, 30):
        for _ in range(200):
            a = rng.integers(0, 256, S, dtype=np.uint8)
            b = rng.integers(0, 256, S, dtype=np.uint8)
            t = ffo.sift_tap(a, b)
            norm = np.linalg.norm(a.astype(np.float64) - b)
            assert t / 16 <= norm + 1e-9 and norm < (t + 1) / 16
            assert ffo.sift_tap(b, a) == t


def test_patch_cost_sums_clamped_taps(ffo):
    rng = np.random.default_rng(3)
    Ks = rng.integers(0, 256, (4, 9, 11, 3), dtype=np.uint8)
    Kt = rng.integers(0, 256, (4, 9, 11, 3), dtype=np.uint8)
    H, W = 9, 11
    for (n, r, p1, p2) in [(1, 1, (0, 0), (10, 8)), (2, 2, (5, 4), (1, 7)), (4, 1, (10, 8), (3, 3))]:
        want = 0
        for v in range(-r, r + 1):
            for u in range(-r, r + 1):
                xs, ys = min(max(p1[0] + n * u, 0), W - 1), min(max(p1[1] + n * v, 0), H - 1)
                xt, yt = min(max(p2[0] + n * u, 0), W - 1), min(max(p2[1] + n * v, 0), H - 1)
                a = Ks[:, ys, xs].reshape(-1)
                b = Kt[:, yt, xt].reshape(-1)
                want += ffo.sift_tap(a, b)
        assert ffo.sift_patch_cost(Ks, Kt, n, r, p1, p2) == want
    assert ffo.sift_patch_cost(Ks, Ks, 2, 3, (4, 4), (4, 4)) == 0


# ------------------------------------------------------------------ search ----
def _basis(ffo, frames, S):
    acc = None
    for f in frames:
        acc = ffo.sift_moments(ffo.sift_descriptors(f), acc=acc)
    P = ffo.sift_pca(*acc, S)
    return P["basis"], P["offset"]


def test_sift_pure_translation_recovered_and_consistent(ffo):
    # SIFT vectors are translation-equivariant away from the border, so the
    # true flow has E_d = 0 wherever the descriptor window and the patch stay
    # inside both frames; the consistency check must keep those pixels.
    W, H, dx, dy = 72, 56, 4, -3
    canvas = synth._to_u8(synth.value_noise(np.random.default_rng(11), H + 40, W + 40))
    I1 = canvas[20:20 + H, 20:20 + W]
    I2 = canvas[20 - dy:20 - dy + H, 20 - dx:20 - dx + W]
    B1, o1 = _basis(ffo, [I1, I2], 12)
    B2, o2 = _basis(ffo, [I1, I2], 18)
    res = ffo.sift_flow_fields(I1, I2, B1, o1, B2, o2,
                               params=dict(k=2, r=3, r2=2, tile=16, eps=1, e=9, s=150))
    F = res["flows"][0]
    m = 2 * CELL + 1 + 4 * 3
    ys, xs = np.mgrid[0:H, 0:W]
    inner = (xs >= m) & (xs < W - m) & (ys >= m) & (ys < H - m) & \
            (xs + dx >= m) & (xs + dx < W - m) & (ys + dy >= m) & (ys + dy < H - m)
    ok = (F[..., 0] == dx) & (F[..., 1] == dy)
    assert ok[inner].mean() >= 0.99
    assert res["valid"][inner & ok].mean() >= 0.99


def test_sift_search_never_increases_cost(ffo):
    I1, I2 = smooth_img(21, 40, 52), smooth_img(22, 40, 52)
    B, o = _basis(ffo, [I1, I2], 12)
    K1 = ffo.sift_colors(ffo.sift_descriptors(I1), B, o)
    K2 = ffo.sift_colors(ffo.sift_descriptors(I2), B, o)
    feat = ffo.wht_features(I2, 3)
    f0, c0, _ = ffo.sift_kd_init(feat, I1, 3, 8, ffo.sift_smooth(K1, 4), ffo.sift_smooth(K2, 4), 4)
    f1, c1, _ = ffo.sift_search_level(ffo.sift_smooth(K1, 4), ffo.sift_smooth(K2, 4), 4, 3,
                                      flow=f0, cost=c0, tile=4)
    assert (c1 <= c0).all()
    Ks, Kt = ffo.sift_smooth(K1, 4), ffo.sift_smooth(K2, 4)
    for gy in range(0, c1.shape[0], 3):
        for gx in range(0, c1.shape[1], 3):
            p = (4 * gx, 4 * gy)
            t = (p[0] + f1[gy, gx, 0], p[1] + f1[gy, gx, 1])
            assert 0 <= t[0] < 52 and 0 <= t[1] < 40
            assert ffo.sift_patch_cost(Ks, Kt, 4, 3, p, t) == c1[gy, gx]


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


def test_sift_whole_path_is_the_composition_of_its_steps(ffo):
    # The whole path wires its inputs as Sec. 3.3 / Sec. 5 prescribe: per level the
    # colours smoothed like I^n; forward (I1 -> I2) and first backward flow with
    # radius r and the first colour set, second backward flow with r2 and the second
    # set (S2 channels); kd trees over the target frame's WHT features. Each flow
    # must equal its steps composed by hand.
    W, H = 48, 40
    I1, I2 = smooth_img(31, H, W), smooth_img(32, H, W)
    B1, o1 = _basis(ffo, [I1, I2], 6)
    B2, o2 = _basis(ffo, [I1, I2], 9)
    P = dict(k=2, r=2, r2=1, tile=8, n_rs=3, R=1, seed=5, eps=1, e=9, s=150)
    res = ffo.sift_flow_fields(I1, I2, B1, o1, B2, o2, params=P)
    col = {(c, f): ffo.sift_colors(ffo.sift_descriptors(img), B, o)
           for c, (B, o) in enumerate(((B1, o1), (B2, o2))) for f, img in enumerate((I1, I2))}
    for j, (src, tgt, r, c) in enumerate(((0, 1, 2, 0), (1, 0, 2, 0), (1, 0, 1, 1))):
        imgs = (I1, I2)
        lv = {n: (ffo.sift_smooth(col[(c, src)], n) if n > 1 else col[(c, src)],
                  ffo.sift_smooth(col[(c, tgt)], n) if n > 1 else col[(c, tgt)]) for n in (1, 2, 4)}
        feat = ffo.wht_features(imgs[tgt], r)
        f, cst, _ = ffo.sift_kd_init(feat, imgs[src], r, 8, lv[4][0], lv[4][1], 4)
        f, cst, _ = ffo.sift_search_level(lv[4][0], lv[4][1], 4, r, flow=f, cost=cst, tile=8,
                                          n_rs=3, R=1, seed=5, flow_id=j)
        for n in (2, 1):
            f, cst, _ = ffo.sift_search_level(lv[n][0], lv[n][1], n, r, flow_coarse=f, tile=8,
                                              n_rs=3, R=1, seed=5, flow_id=j)
        assert np.array_equal(f, res["flows"][j]), j
    _assert_filter_composed(ffo, res, 1, 150, 9)
