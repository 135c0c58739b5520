"""GPU parity of the SIFT flow data term (Sec. 3.3) through the C ABI against the
CPU oracle on the same seeded inputs.

Descriptors, moments, colours, the kd initialisation, the level search and the
whole path are integer: bit-exact. The PCA basis comes out of a float64
eigensolver on each side (Jacobi rotations here, LAPACK in the oracle): the
eigenvalues must agree to 1e-9 of the largest, and the quantised basis and its
offsets exactly wherever the oracle's unrounded value lies at least 1e-6 from a
rounding boundary (every entry in these cases; an fp64 solver's error is far
below that)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1508_05151_gb300 import ffapi, synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")


def tg(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rimg(seed, H, W):
    return np.random.default_rng(seed).integers(0, 256, size=(H, W, 3), dtype=np.uint8)


def vimg(seed, H, W):
    return synth._to_u8(synth.value_noise(np.random.default_rng(seed), H, W))


def oracle_bases(frames, *S):
    """The oracle's quantised bases (basis, offset) for each channel count in S,
    fitted on the descriptors of `frames`."""
    acc = None
    for f in frames:
        acc = O.sift_moments(O.sift_descriptors(f), acc=acc)
    out = []
    for s in S:
        P = O.sift_pca(*acc, s)
        out += [P["basis"], P["offset"]]
    return out


def oracle_basis(frames, S):
    return oracle_bases(frames, S)


@pytest.mark.parametrize("W,H", [(1, 1), (5, 3), (17, 13), (40, 33), (128, 96), (301, 170)])
def test_descriptors_bit_exact(W, H):
    img = rimg(W * 7 + H, H, W) if W < 100 else vimg(W + H, H, W)
    got = cpu(ffapi.ff_sift_descriptors(tg(img)))
    assert np.array_equal(got, O.sift_descriptors(img))


def test_descriptors_full_size_kitti_frame():
    d = synth.workload_pair("kitti_1242x375", 3)
    got = cpu(ffapi.ff_sift_descriptors(tg(d["I1"])))
    assert np.array_equal(got, O.sift_descriptors(d["I1"]))


def test_moments_bit_exact_and_accumulate():
    a, b = vimg(1, 70, 90), rimg(2, 33, 41)
    da, db = ffapi.ff_sift_descriptors(tg(a)), ffapi.ff_sift_descriptors(tg(b))
    s, g, n = ffapi.ff_sift_moments(db, acc=ffapi.ff_sift_moments(da))
    os_, og, on = O.sift_moments(O.sift_descriptors(b), acc=O.sift_moments(O.sift_descriptors(a)))
    assert n == on == 70 * 90 + 33 * 41
    assert np.array_equal(cpu(s).astype(np.uint64), os_)
    assert np.array_equal(cpu(g).astype(np.uint64), og)
    # a chunk boundary of the moments kernel (4096 descriptors) and a ragged tail
    c = rimg(3, 65, 67)
    s, g, n = ffapi.ff_sift_moments(ffapi.ff_sift_descriptors(tg(c)))
    os_, og, _ = O.sift_moments(O.sift_descriptors(c))
    assert np.array_equal(cpu(s).astype(np.uint64), os_) and np.array_equal(cpu(g).astype(np.uint64), og)


@pytest.mark.parametrize("S", [3, 12, 18, 30])
def test_pca_basis(S):
    frames = [vimg(11, 94, 310), vimg(12, 94, 310)]
    acc = None
    oacc = None
    for f in frames:
        acc = ffapi.ff_sift_moments(ffapi.ff_sift_descriptors(tg(f)), acc=acc)
        oacc = O.sift_moments(O.sift_descriptors(f), acc=oacc)
    B, off, eig, st = ffapi.ff_sift_pca(acc[0], acc[1], acc[2], S, with_status=True)
    assert st[0] == 0
    P = O.sift_pca(*oacc, S)
    w = P["eigval"]
    assert np.allclose(cpu(eig), w, rtol=0, atol=1e-9 * w[0])
    exact = P["exact"]
    margin = np.abs(exact - np.floor(exact) - 0.5)
    assert margin.min() >= 1e-6, "an entry sits on a rounding boundary; choose other inputs"
    assert np.array_equal(cpu(B), P["basis"])
    assert np.array_equal(cpu(off), P["offset"])


def test_colors_bit_exact_with_oracle_basis():
    I1 = vimg(21, 80, 104)
    for S in (12, 18):
        B, off = oracle_basis([I1], S)
        got = cpu(ffapi.ff_sift_colors(ffapi.ff_sift_descriptors(tg(I1)), tg(B), tg(off)))
        assert np.array_equal(got, O.sift_colors(O.sift_descriptors(I1), B, off))


def _colours(I, B, off, n):
    col = O.sift_colors(O.sift_descriptors(I), B, off)
    return O.sift_smooth(col, n) if n > 1 else col


@pytest.mark.parametrize("n,r,S", [(8, 3, 12), (4, 2, 18), (2, 3, 3), (8, 8, 30)])
def test_kd_init_bit_exact(n, r, S):
    I1, I2 = vimg(31, 96, 128), vimg(32, 96, 128)
    B, off = oracle_basis([I1, I2], S)
    K1, K2 = _colours(I1, B, off, n), _colours(I2, B, off, n)
    feat = O.wht_features(I2, r)
    of, oc, _ = O.sift_kd_init(feat, I1, r, 8, K1, K2, n)
    tree = ffapi.ff_kdtree_build(ffapi.ff_features(tg(I2), r), 8)
    gf, gc = ffapi.ff_sift_kdtree_init(tree, 8, tg(I1), tg(K1), tg(K2), n, r)
    assert np.array_equal(cpu(gc), oc)
    assert np.array_equal(cpu(gf).astype(np.int32), of)


def test_kd_init_reports_a_corrupt_tree():
    """The SIFT kd query's own checks: a split dimension outside [0, 27) or a leaf
    entry outside [0, N) is skipped and reported as device status 1 with the grid
    point; a sound tree reports 0."""
    I1, I2 = vimg(51, 48, 64), vimg(52, 48, 64)
    n, r, S = 4, 3, 12
    B, off = oracle_basis([I1, I2], S)
    K1, K2 = tg(_colours(I1, B, off, n)), tg(_colours(I2, B, off, n))
    T = ffapi.ff_kdtree_build(ffapi.ff_features(tg(I2), r), 8)
    _, _, st = ffapi.ff_sift_kdtree_init(T, 8, tg(I1), K1, K2, n, r, with_status=True)
    assert st == (0, 0, 0)
    sd, _ = T["_keep"]
    sd[0] = 99
    _, _, st = ffapi.ff_sift_kdtree_init(T, 8, tg(I1), K1, K2, n, r, with_status=True)
    assert st[0] == 1 and st[2] == 0
    T2 = ffapi.ff_kdtree_build(ffapi.ff_features(tg(I2), r), 8)
    T2["perm"][:] = T2["N"] + 7
    _, c, st = ffapi.ff_sift_kdtree_init(T2, 8, tg(I1), K1, K2, n, r, with_status=True)
    assert st[0] == 1 and 0 <= st[2] < T2["N"]
    assert bool((c == O.COST_UNSET).all())


@pytest.mark.parametrize("W,H,n,r,S,tile,n_rs,seeded", [
    (128, 96, 1, 3, 12, 16, 3, True),
    (128, 96, 2, 2, 18, 16, 3, True),
    (128, 96, 8, 3, 12, 16, 3, False),
    (77, 53, 1, 1, 3, 4, 2, True),
    (77, 53, 4, 8, 30, 32, 1, False),
    (150, 100, 1, 3, 12, 2, 0, True),
    (33, 17, 2, 2, 18, 6, 3, True),
    (600, 400, 1, 2, 12, 8, 3, True),   # 3750 tiles, more than one wave of CTAs
])
def test_search_level_bit_exact(W, H, n, r, S, tile, n_rs, seeded):
    I1, I2 = vimg(41 + W, H, W), vimg(42 + W, H, W)
    B, off = oracle_basis([I1, I2], S)
    K1, K2 = _colours(I1, B, off, n), _colours(I2, B, off, n)
    Gx, Gy = (W + n - 1) // n, (H + n - 1) // n
    rng = np.random.default_rng(W + H + n)
    P = dict(tile=tile, n_rs=n_rs, R=1, seed=1234)
    if seeded:
        Gxc, Gyc = (W + 2 * n - 1) // (2 * n), (H + 2 * n - 1) // (2 * n)
        fc = np.stack([rng.integers(-6, 7, (Gyc, Gxc)), rng.integers(-5, 6, (Gyc, Gxc))], -1)
        # coarse flows with targets inside the image, like a real coarser level
        ys, xs = np.mgrid[0:Gyc, 0:Gxc] * (2 * n)
        fc[..., 0] = np.clip(xs + fc[..., 0], 0, W - 1) - xs
        fc[..., 1] = np.clip(ys + fc[..., 1], 0, H - 1) - ys
        fc = fc.astype(np.int32)
        of, oc, _ = O.sift_search_level(K1, K2, n, r, flow_coarse=fc, flow_id=1, **P)
        gf, gc = ffapi.ff_sift_search_level(tg(K1), tg(K2), n, r, params=P, flow_id=1,
                                            flow_coarse=tg(fc.astype(np.int16)))
    else:
        feat = O.wht_features(I2, min(r, 8))
        f0, c0, _ = O.sift_kd_init(feat, I1, r, 8, K1, K2, n)
        of, oc, _ = O.sift_search_level(K1, K2, n, r, flow=f0, cost=c0, flow_id=2, **P)
        gf, gc = ffapi.ff_sift_search_level(tg(K1), tg(K2), n, r, params=P, flow_id=2,
                                            flow=tg(f0.astype(np.int16)), cost=tg(c0))
    assert gf.shape == (Gy, Gx, 2)
    assert np.array_equal(cpu(gc), oc)
    assert np.array_equal(cpu(gf).astype(np.int32), of)


def _whole(I1, I2, S1, S2, params):
    B1, o1, B2, o2 = oracle_bases([I1, I2], S1, S2)
    ref = O.sift_flow_fields(I1, I2, B1, o1, B2, o2, params=params)
    got = ffapi.ff_sift_flow_fields(tg(I1), tg(I2), tg(B1), tg(o1), tg(B2), tg(o2),
                                    params=params)
    assert np.array_equal(cpu(got["flows"]).astype(np.int32), ref["flows"])
    assert np.array_equal(cpu(got["valid"]), ref["valid"])
    assert np.array_equal(cpu(got["err_sum"]), ref["err_sum"])
    ns = int(cpu(got["n_sparse"])[0])
    assert ns == len(ref["sparse"])
    assert np.array_equal(cpu(got["sparse"])[:ns], ref["sparse"])
    assert np.array_equal(cpu(got["mask"]), ref["mask"])
    return ref


KITTI = dict(k=3, r=3, r2=2, eps=1, e=9, s=150)


@pytest.mark.parametrize("seed", [0, 1])
def test_whole_path_bit_exact_128x96(seed):
    d = synth.workload_pair("noise_128x96", 600 + seed)
    _whole(d["I1"], d["I2"], 12, 18, KITTI)


@pytest.mark.parametrize("W,H,k,extra", [(1, 1, 0, {}), (9, 5, 1, {}), (37, 23, 2, dict(color=1)),
                                         (150, 100, 3, dict(tile=8, n_rs=1))])
def test_whole_path_edge_shapes(W, H, k, extra):
    I1, I2 = rimg(W * 3 + 1, H, W), rimg(W * 3 + 2, H, W)
    _whole(I1, I2, 3, 6, dict(KITTI, k=k, **extra))


def test_whole_path_full_size_kitti_pair():
    d = synth.workload_pair("kitti_1242x375", 7)
    ref = _whole(d["I1"], d["I2"], 12, 18, KITTI)
    assert ref["valid"].mean() > 0.2
