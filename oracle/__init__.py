"""Python access to the Flow Fields CPU oracle (``ffo.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the GPU library never imports it. The oracle is a
plain, slow restatement of the paper's method in C; see the comments in ffo.c for
the passage each function follows.

All arrays are numpy. Flows are int32 (..., 2) arrays of (dx, dy); images uint8
(H, W, 3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffo.c")
_LIB = os.path.join(_HERE, "libffo.so")
_lock = threading.Lock()
_lib = None

COST_UNSET = 2**31 - 1


def build(force=False):
    """Compile ffo.c into libffo.so next to it (gcc, portable flags)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm", "-lpthread"])
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [(n, C.c_int32) for n in
                ("k", "r", "r2", "leaf", "R", "eps", "e", "s", "tile", "n_rs", "K", "color",
                 "subpel")] + \
               [("seed", C.c_uint64)]


def default_params(**kw):
    """Sec. 4 parameters (k=3, R=1, l=8, r=8, r2=6; Sintel eps/e/s = 5/4/50),
    tile T=16 for the parallel schedule, 3 random-search steps, no proposals."""
    d = dict(k=3, r=8, r2=6, leaf=8, R=1, eps=5, e=4, s=50, tile=16, n_rs=3, K=0, color=0,
             subpel=1, seed=0)
    d.update(kw)
    return d


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u8, i32, u32, i64 = (C.POINTER(C.c_uint8), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint32), C.POINTER(C.c_int64))
            ci = C.c_int
            L.ffo_area_down.argtypes = [u8, ci, ci, ci, u8]
            L.ffo_lanczos_table.argtypes = [ci, i32, i32]
            L.ffo_smooth.argtypes = [u8, ci, ci, ci, u8]
            L.ffo_census.argtypes = [u8, ci, ci, ci, u32]
            L.ffo_patch_cost.argtypes = [u32, u32, ci, ci, ci, ci, ci, ci, ci, ci]
            L.ffo_patch_cost.restype = C.c_int32
            L.ffo_wht_blocks.argtypes = [ci, i32]
            L.ffo_wht_basis_1d.argtypes = [ci, ci, i32]
            L.ffo_wht_features.argtypes = [u8, ci, ci, ci, i32, ci, i32]
            L.ffo_wht_features_general.argtypes = [u8, ci, ci, ci, ci, i32, ci, i32]
            L.ffo_kd_depth.argtypes = [ci, ci]
            L.ffo_kd_build.argtypes = [i32, ci, ci, i32, i32, i32]
            L.ffo_kd_leaf_range.argtypes = [ci, ci, ci, i32, i32]
            L.ffo_kd_query.argtypes = [i32, i32, ci, i32]
            L.ffo_kd_init.argtypes = [i32, u8, ci, ci, ci, ci, u32, u32, ci, i32, ci, i32, i32]
            L.ffo_kd_init.restype = C.c_int64
            L.ffo_splitmix64.argtypes = [C.c_uint64]
            L.ffo_splitmix64.restype = C.c_uint64
            L.ffo_rs_offset.argtypes = [C.c_uint64, ci, ci, ci, ci, ci, ci, i32]
            L.ffo_search_level.argtypes = [u32, u32, ci, ci, ci, ci, i32, ci, ci, ci,
                                           C.c_uint64, ci, i32, i32]
            L.ffo_search_level.restype = C.c_int64
            L.ffo_consistency.argtypes = [i32, i32, i32, ci, ci, ci, ci, u8, i32, i32, i32]
            L.ffo_census_subpel.argtypes = [u8, ci, ci, ci, ci, ci, ci, u32]
            L.ffo_sqrt_sum_less.argtypes = [C.c_int64] * 4
            L.ffo_lab_gamma_table.argtypes = [i32]
            L.ffo_lab_matrix.argtypes = [i32]
            L.ffo_lab_f.argtypes = [C.c_int32]
            L.ffo_lab_f.restype = C.c_int32
            L.ffo_rgb_to_lab.argtypes = [u8, ci, ci, u8]
            L.ffo_match_errors.argtypes = [u8, u8, i32, ci, ci, ci, i32]
            L.ffo_weighted_median.argtypes = [i32, i32, ci, ci, ci, i32]
            L.ffo_region_filter.argtypes = [i32, u8, ci, ci, ci, ci, u8]
            L.ffo_sparsify.argtypes = [u8, i32, i32, i32, ci, ci, ci, i32, u8]
            L.ffo_flow_fields.argtypes = [u8, u8, ci, ci, C.POINTER(Params), i32, ci, i32, u8,
                                          i32, i32, u8, i64]
            u64, i16 = C.POINTER(C.c_uint64), C.POINTER(C.c_int16)
            L.ffo_isqrt.argtypes = [C.c_uint64]
            L.ffo_isqrt.restype = C.c_uint64
            L.ffo_sift_orient.argtypes = [u8, ci, ci, i32]
            L.ffo_sift_descriptors.argtypes = [u8, ci, ci, u8]
            L.ffo_sift_moments.argtypes = [u8, ci, u64, u64]
            L.ffo_sift_pca_offset.argtypes = [i16, ci, u64, C.c_int64, i32]
            L.ffo_sift_colors.argtypes = [u8, ci, ci, i16, i32, ci, u8]
            L.ffo_sift_tap.argtypes = [u8, u8, ci, C.c_size_t, C.c_size_t, C.c_size_t]
            L.ffo_sift_tap.restype = C.c_int32
            L.ffo_sift_patch_cost.argtypes = [u8, u8, ci, ci, ci, ci, ci, ci, ci, ci, ci]
            L.ffo_sift_patch_cost.restype = C.c_int32
            L.ffo_sift_kd_init.argtypes = [i32, u8, ci, ci, ci, ci, u8, u8, ci, ci, i32, i32]
            L.ffo_sift_kd_init.restype = C.c_int64
            L.ffo_sift_search_level.argtypes = [u8, u8, ci, ci, ci, ci, ci, i32, ci, ci, ci,
                                                C.c_uint64, ci, i32, i32]
            L.ffo_sift_search_level.restype = C.c_int64
            L.ffo_sift_flow_fields.argtypes = [u8, u8, ci, ci, C.POINTER(Params), i16, i32, ci,
                                               i16, i32, ci, ci, i32, u8, i32, i32, u8, i64]
            _lib = L
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def grid(W, H, n):
    return (W + n - 1) // n, (H + n - 1) // n


def area_down(img, n):
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    out = np.empty(((H + n - 1) // n, (W + n - 1) // n, 3), np.uint8)
    lib().ffo_area_down(_p(img, C.c_uint8), W, H, n, _p(out, C.c_uint8))
    return out


def lanczos_table(n):
    base = np.empty(n, np.int32)
    w = np.empty((n, 6), np.int32)
    lib().ffo_lanczos_table(n, _p(base, C.c_int32), _p(w, C.c_int32))
    return base, w


def smooth(img, n):
    img = _c(img, np.uint8)
    out = np.empty_like(img)
    lib().ffo_smooth(_p(img, C.c_uint8), img.shape[1], img.shape[0], n, _p(out, C.c_uint8))
    return out


def census(imgn, n):
    imgn = _c(imgn, np.uint8)
    H, W = imgn.shape[:2]
    out = np.empty((H, W), np.uint32)
    lib().ffo_census(_p(imgn, C.c_uint8), W, H, n, _p(out, C.c_uint32))
    return out


def patch_cost(Cs, Ct, n, r, p1, p2):
    Cs, Ct = _c(Cs, np.uint32), _c(Ct, np.uint32)
    H, W = Cs.shape
    return int(lib().ffo_patch_cost(_p(Cs, C.c_uint32), _p(Ct, C.c_uint32), W, H, n, r,
                                    int(p1[0]), int(p1[1]), int(p2[0]), int(p2[1])))


def wht_blocks(L):
    out = np.empty(4, np.int32)
    lib().ffo_wht_blocks(L, _p(out, C.c_int32))
    return out


def wht_basis_1d(L, nb=3):
    out = np.empty((nb, L), np.int32)
    lib().ffo_wht_basis_1d(L, nb, _p(out, C.c_int32))
    return out


def wht_features(img, r, pts=None):
    """Features (npts or H*W, 27) int32; pts: int32 (npts, 2) of (x, y)."""
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    if pts is None:
        out = np.empty((H * W, 27), np.int32)
        lib().ffo_wht_features(_p(img, C.c_uint8), W, H, r, None, 0, _p(out, C.c_int32))
    else:
        pts = _c(pts, np.int32).reshape(-1, 2)
        out = np.empty((len(pts), 27), np.int32)
        lib().ffo_wht_features(_p(img, C.c_uint8), W, H, r, _p(pts, C.c_int32), len(pts),
                               _p(out, C.c_int32))
    return out


def wht_features_general(img, L, nb, pts):
    """Window of L pixels from x - (L-1)//2, nb x nb bases per channel:
    returns (npts, 3, nb, nb)."""
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    pts = _c(pts, np.int32).reshape(-1, 2)
    out = np.empty((len(pts), 3, nb, nb), np.int32)
    lib().ffo_wht_features_general(_p(img, C.c_uint8), W, H, L, nb, _p(pts, C.c_int32),
                                   len(pts), _p(out, C.c_int32))
    return out


def kd_depth(N, leaf):
    return int(lib().ffo_kd_depth(N, leaf))


def kd_build(feat, leaf):
    feat = _c(feat, np.int32)
    N = feat.shape[0]
    D = kd_depth(N, leaf)
    perm = np.empty(N, np.int32)
    sd = np.zeros((1 << D) + 1, np.int32)
    sv = np.zeros((1 << D) + 1, np.int32)
    lib().ffo_kd_build(_p(feat, C.c_int32), N, leaf, _p(perm, C.c_int32), _p(sd, C.c_int32),
                       _p(sv, C.c_int32))
    return dict(perm=perm, split_dim=sd[:(1 << D) - 1], split_val=sv[:(1 << D) - 1], D=D, N=N)


def kd_leaf_range(N, D, leaf):
    b, e = C.c_int32(), C.c_int32()
    lib().ffo_kd_leaf_range(N, D, leaf, C.byref(b), C.byref(e))
    return b.value, e.value


def kd_query(tree, q):
    q = _c(q, np.int32)
    sd = _c(np.append(tree["split_dim"], 0), np.int32)
    sv = _c(np.append(tree["split_val"], 0), np.int32)
    return int(lib().ffo_kd_query(_p(sd, C.c_int32), _p(sv, C.c_int32), tree["D"],
                                  _p(q, C.c_int32)))


def kd_leaves(tree):
    """List of sorted pixel-index arrays, one per leaf."""
    out = []
    for lf in range(1 << tree["D"]):
        b, e = kd_leaf_range(tree["N"], tree["D"], lf)
        out.append(np.sort(tree["perm"][b:e]))
    return out


def kd_init(tgt_feat, src_img, r, leaf, Cs, Ct, n, proposals=None):
    """Top-level initialisation (Eq. 1/4). Returns flow (Gy, Gx, 2), cost (Gy, Gx), evals."""
    src_img = _c(src_img, np.uint8)
    H, W = src_img.shape[:2]
    Gx, Gy = grid(W, H, n)
    tgt_feat, Cs, Ct = _c(tgt_feat, np.int32), _c(Cs, np.uint32), _c(Ct, np.uint32)
    flow = np.empty((Gy, Gx, 2), np.int32)
    cost = np.empty((Gy, Gx), np.int32)
    K = 0
    if proposals is not None:
        proposals = _c(proposals, np.int32)
        K = proposals.shape[2]
    ev = lib().ffo_kd_init(_p(tgt_feat, C.c_int32), _p(src_img, C.c_uint8), W, H, r, leaf,
                           _p(Cs, C.c_uint32), _p(Ct, C.c_uint32), n,
                           _p(proposals, C.c_int32), K, _p(flow, C.c_int32),
                           _p(cost, C.c_int32))
    return flow, cost, int(ev)


def lab_gamma_table():
    t = np.empty(256, np.int32)
    lib().ffo_lab_gamma_table(_p(t, C.c_int32))
    return t


def lab_matrix():
    m = np.empty(9, np.int32)
    lib().ffo_lab_matrix(_p(m, C.c_int32))
    return m.reshape(3, 3)


def lab_f(t):
    return int(lib().ffo_lab_f(int(t)))


def rgb_to_lab(img):
    """Integer CIELab (L * 255/100, a + 128, b + 128 as uint8) of an sRGB image."""
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    out = np.empty((H, W, 3), np.uint8)
    lib().ffo_rgb_to_lab(_p(img, C.c_uint8), W, H, _p(out, C.c_uint8))
    return out


def match_errors(I1, I2, F, r):
    """E_d of every pixel's own match at full resolution (census spacing 1)."""
    I1, I2, F = _c(I1, np.uint8), _c(I2, np.uint8), _c(F, np.int32)
    H, W = I1.shape[:2]
    E = np.empty((H, W), np.int32)
    lib().ffo_match_errors(_p(I1, C.c_uint8), _p(I2, C.c_uint8), _p(F, C.c_int32), W, H, r,
                           _p(E, C.c_int32))
    return E


def weighted_median(F, E, rho=2):
    """Component-wise median weighted by floor(2^16 / (1 + E)) over the in-image
    (2 rho + 1)^2 window (the lower weighted median)."""
    F, E = _c(F, np.int32), _c(E, np.int32)
    H, W = E.shape
    out = np.empty((H, W, 2), np.int32)
    lib().ffo_weighted_median(_p(F, C.c_int32), _p(E, C.c_int32), W, H, rho, _p(out, C.c_int32))
    return out


def splitmix64(z):
    return int(lib().ffo_splitmix64(C.c_uint64(z)))


def rs_offset(seed, flow_id, level, step, gx, gy, Rn):
    d = np.empty(2, np.int32)
    lib().ffo_rs_offset(C.c_uint64(seed), flow_id, level, step, gx, gy, Rn, _p(d, C.c_int32))
    return int(d[0]), int(d[1])


def search_level(Cs, Ct, n, r, flow_coarse=None, flow=None, cost=None, tile=16, n_rs=3, R=1,
                 seed=0, flow_id=0):
    """One hierarchy level. With flow_coarse the level is seeded from it (Sec. 3.2);
    without, (flow, cost) is the initial state (top level). Returns flow, cost, evals."""
    Cs, Ct = _c(Cs, np.uint32), _c(Ct, np.uint32)
    H, W = Cs.shape
    Gx, Gy = grid(W, H, n)
    if flow_coarse is not None:
        fc = _c(flow_coarse, np.int32)
        flow = np.empty((Gy, Gx, 2), np.int32)
        cost = np.empty((Gy, Gx), np.int32)
    else:
        fc = None
        flow = _c(flow, np.int32).copy()
        cost = _c(cost, np.int32).copy()
    ev = lib().ffo_search_level(_p(Cs, C.c_uint32), _p(Ct, C.c_uint32), W, H, n, r,
                                _p(fc, C.c_int32), tile, n_rs, R, C.c_uint64(seed), flow_id,
                                _p(flow, C.c_int32), _p(cost, C.c_int32))
    return flow, cost, int(ev)


def census_subpel(imgn, n, q, a, b):
    """Census (spacing n) of the image interpolated at (x + a/q, y + b/q)."""
    imgn = _c(imgn, np.uint8)
    H, W = imgn.shape[:2]
    out = np.empty((H, W), np.uint32)
    lib().ffo_census_subpel(_p(imgn, C.c_uint8), W, H, n, q, a, b, _p(out, C.c_uint32))
    return out


def consistency(F, Fb1, Fb2, eps, errors=False, subpel=1):
    """Eq. 5 check: (valid_cc, err_sum = e1 + e2), and with errors=True also the
    squared errors e1, e2 against the two backward flows (flows in 1/subpel px)."""
    F, Fb1, Fb2 = _c(F, np.int32), _c(Fb1, np.int32), _c(Fb2, np.int32)
    H, W = F.shape[:2]
    v = np.empty((H, W), np.uint8)
    e = np.empty((H, W), np.int32)
    e1 = np.empty((H, W), np.int32)
    e2 = np.empty((H, W), np.int32)
    lib().ffo_consistency(_p(F, C.c_int32), _p(Fb1, C.c_int32), _p(Fb2, C.c_int32), W, H, eps,
                          subpel, _p(v, C.c_uint8), _p(e, C.c_int32), _p(e1, C.c_int32),
                          _p(e2, C.c_int32))
    return (v, e, e1, e2) if errors else (v, e)


def sqrt_sum_less(a, b, c, d):
    """sqrt(a) + sqrt(b) < sqrt(c) + sqrt(d), exactly, for integers in [0, 2^28)."""
    return bool(lib().ffo_sqrt_sum_less(int(a), int(b), int(c), int(d)))


def region_filter(F, valid_cc, s, subpel=1):
    F, valid_cc = _c(F, np.int32), _c(valid_cc, np.uint8)
    H, W = valid_cc.shape
    out = np.empty((H, W), np.uint8)
    lib().ffo_region_filter(_p(F, C.c_int32), _p(valid_cc, C.c_uint8), W, H, s, subpel,
                            _p(out, C.c_uint8))
    return out


def sparsify(valid, e1, e2, F, e):
    """Sec. 3.5: per 3x3 block with >= e valid pixels the one with the smallest
    sqrt(e1) + sqrt(e2) (raster-first on ties)."""
    valid, e1, e2, F = _c(valid, np.uint8), _c(e1, np.int32), _c(e2, np.int32), _c(F, np.int32)
    H, W = valid.shape
    sp = np.empty((((W + 2) // 3) * ((H + 2) // 3), 4), np.int32)
    mask = np.empty((H, W), np.uint8)
    n = lib().ffo_sparsify(_p(valid, C.c_uint8), _p(e1, C.c_int32), _p(e2, C.c_int32),
                           _p(F, C.c_int32), W, H, e, _p(sp, C.c_int32), _p(mask, C.c_uint8))
    return sp[:n].copy(), mask


def flow_fields(I1, I2, params=None, proposals=None, threads=3):
    """Whole pipeline. Returns dict(flows (3, H, W, 2), valid, err_sum, sparse, mask, evals)."""
    P = default_params(**(params or {}))
    if proposals is not None:
        P["K"] = proposals.shape[2]
    I1, I2 = _c(I1, np.uint8), _c(I2, np.uint8)
    H, W = I1.shape[:2]
    flows = np.empty((3, H, W, 2), np.int32)
    valid = np.empty((H, W), np.uint8)
    err = np.empty((H, W), np.int32)
    sp = np.empty((((W + 2) // 3) * ((H + 2) // 3), 4), np.int32)
    mask = np.empty((H, W), np.uint8)
    ev = C.c_int64()
    pr = _c(proposals, np.int32) if proposals is not None else None
    n = lib().ffo_flow_fields(_p(I1, C.c_uint8), _p(I2, C.c_uint8), W, H, C.byref(Params(**P)),
                              _p(pr, C.c_int32), threads, _p(flows, C.c_int32),
                              _p(valid, C.c_uint8), _p(err, C.c_int32), _p(sp, C.c_int32),
                              _p(mask, C.c_uint8), C.byref(ev))
    return dict(flows=flows, valid=valid, err_sum=err, sparse=sp[:n].copy(), mask=mask,
                evals=ev.value)


# --------------------------------------------------------------------------
# Sec. 3.3, the SIFT flow data term (readings in ffo.c).

SIFT_DIM = 128
SIFT_SHIFT = 12  # basis components in units of 2^-12


def isqrt(x):
    return int(lib().ffo_isqrt(C.c_uint64(int(x))))


def sift_orient(img):
    """The 8 rectified orientation responses per pixel, (H, W, 8) int32."""
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    out = np.empty((H, W, 8), np.int32)
    lib().ffo_sift_orient(_p(img, C.c_uint8), W, H, _p(out, C.c_int32))
    return out


def sift_descriptors(img):
    """Dense SIFT vectors, (H, W, 128) uint8."""
    img = _c(img, np.uint8)
    H, W = img.shape[:2]
    out = np.empty((H, W, SIFT_DIM), np.uint8)
    lib().ffo_sift_descriptors(_p(img, C.c_uint8), W, H, _p(out, C.c_uint8))
    return out


def sift_moments(desc, acc=None):
    """Exact sums and Gram matrix of the descriptors (added to acc = (sum, gram)
    when given). Returns (sum uint64 [128], gram uint64 [128, 128], count)."""
    d = _c(desc, np.uint8).reshape(-1, SIFT_DIM)
    if acc is None:
        sm, gram, count = np.zeros(SIFT_DIM, np.uint64), np.zeros((SIFT_DIM, SIFT_DIM), np.uint64), 0
    else:
        sm, gram, count = acc[0].copy(), acc[1].copy(), acc[2]
    lib().ffo_sift_moments(_p(d, C.c_uint8), d.shape[0], _p(sm, C.c_uint64), _p(gram, C.c_uint64))
    return sm, gram, count + d.shape[0]


def sift_pca(sm, gram, count, S):
    """Sec. 3.3: PCA of the descriptors from their moments, reduced to S
    dimensions and quantised. Readings: covariance C = gram / count - mu mu^T
    (mu = sum / count) in float64; its eigenvectors by eigenvalue, largest first
    (numpy's symmetric eigensolver), each signed so that its entry of largest
    magnitude (lowest index on ties) is positive; one gain for all components,
    g = 127 / (3 sqrt(max(lambda_1, 1))), so that distances between colours stay
    proportional to distances between descriptors; B_si = clamp(floor(2^12 g e_si
    + 1/2), -32767, 32767); offsets from ffo_sift_pca_offset. Returns dict(basis
    int16 [S, 128], offset int32 [S], eigval float64 [128] (descending), exact
    float64 [S, 128] = the unrounded 2^12 g e_si)."""
    sm = np.asarray(sm, np.uint64)
    gram = np.asarray(gram, np.uint64)
    mu = sm.astype(np.float64) / count
    Cm = gram.astype(np.float64) / count - np.outer(mu, mu)
    w, V = np.linalg.eigh(Cm)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    E = V[:, :S].T.copy()
    for s in range(S):
        i = int(np.argmax(np.abs(E[s])))
        if E[s, i] < 0:
            E[s] = -E[s]
    g = 127.0 / (3.0 * np.sqrt(max(float(w[0]), 1.0)))
    exact = float(1 << SIFT_SHIFT) * g * E
    B = np.clip(np.floor(exact + 0.5), -32767, 32767).astype(np.int16)
    off = sift_pca_offset(B, sm, count)
    return dict(basis=B, offset=off, eigval=w, exact=exact)


def sift_pca_offset(B, sm, count):
    B = _c(B, np.int16)
    sm = _c(sm, np.uint64)
    off = np.empty(B.shape[0], np.int32)
    lib().ffo_sift_pca_offset(_p(B, C.c_int16), B.shape[0], _p(sm, C.c_uint64), int(count),
                              _p(off, C.c_int32))
    return off


def sift_colors(desc, B, off):
    """SIFT flow colours in S/3 groups: (S/3, H, W, 3) uint8."""
    desc = _c(desc, np.uint8)
    H, W = desc.shape[:2]
    B, off = _c(B, np.int16), _c(off, np.int32)
    S = B.shape[0]
    out = np.empty((S // 3, H, W, 3), np.uint8)
    lib().ffo_sift_colors(_p(desc, C.c_uint8), W, H, _p(B, C.c_int16), _p(off, C.c_int32), S,
                          _p(out, C.c_uint8))
    return out


def sift_smooth(col, n):
    """Each colour group smoothed like I^n (Sec. 3.2)."""
    return np.stack([smooth(g, n) for g in col])


def sift_tap(a, b):
    """Distance of two colours given as length-S uint8 vectors."""
    a, b = _c(a, np.uint8), _c(b, np.uint8)
    S = a.shape[0]
    ga = _c(a.reshape(S // 3, 1, 3), np.uint8)
    gb = _c(b.reshape(S // 3, 1, 3), np.uint8)
    return int(lib().ffo_sift_tap(_p(ga, C.c_uint8), _p(gb, C.c_uint8), S, 1, 0, 0))


def sift_patch_cost(Ks, Kt, n, r, p1, p2):
    Ks, Kt = _c(Ks, np.uint8), _c(Kt, np.uint8)
    G, H, W = Ks.shape[:3]
    return int(lib().ffo_sift_patch_cost(_p(Ks, C.c_uint8), _p(Kt, C.c_uint8), 3 * G, W, H, n, r,
                                         p1[0], p1[1], p2[0], p2[1]))


def sift_kd_init(tgt_feat, src_img, r, leaf, Ks, Kt, n):
    """Top-level initialisation (Eq. 1/4) with the SIFT flow data term."""
    src_img = _c(src_img, np.uint8)
    H, W = src_img.shape[:2]
    Gx, Gy = grid(W, H, n)
    tgt_feat, Ks, Kt = _c(tgt_feat, np.int32), _c(Ks, np.uint8), _c(Kt, np.uint8)
    flow = np.empty((Gy, Gx, 2), np.int32)
    cost = np.empty((Gy, Gx), np.int32)
    ev = lib().ffo_sift_kd_init(_p(tgt_feat, C.c_int32), _p(src_img, C.c_uint8), W, H, r, leaf,
                                _p(Ks, C.c_uint8), _p(Kt, C.c_uint8), 3 * Ks.shape[0], n,
                                _p(flow, C.c_int32), _p(cost, C.c_int32))
    return flow, cost, int(ev)


def sift_search_level(Ks, Kt, n, r, flow_coarse=None, flow=None, cost=None, tile=16, n_rs=3, R=1,
                      seed=0, flow_id=0):
    """One hierarchy level with the SIFT flow data term (as search_level)."""
    Ks, Kt = _c(Ks, np.uint8), _c(Kt, np.uint8)
    G, H, W = Ks.shape[:3]
    Gx, Gy = grid(W, H, n)
    if flow_coarse is not None:
        fc = _c(flow_coarse, np.int32)
        flow = np.empty((Gy, Gx, 2), np.int32)
        cost = np.empty((Gy, Gx), np.int32)
    else:
        fc = None
        flow = _c(flow, np.int32).copy()
        cost = _c(cost, np.int32).copy()
    ev = lib().ffo_sift_search_level(_p(Ks, C.c_uint8), _p(Kt, C.c_uint8), 3 * G, W, H, n, r,
                                     _p(fc, C.c_int32), tile, n_rs, R, C.c_uint64(seed), flow_id,
                                     _p(flow, C.c_int32), _p(cost, C.c_int32))
    return flow, cost, int(ev)


def sift_flow_fields(I1, I2, B1, off1, B2, off2, params=None, threads=3):
    """Whole pipeline with the SIFT flow data term. Returns the dict of flow_fields."""
    P = default_params(**(params or {}))
    I1, I2 = _c(I1, np.uint8), _c(I2, np.uint8)
    H, W = I1.shape[:2]
    B1, B2 = _c(B1, np.int16), _c(B2, np.int16)
    off1, off2 = _c(off1, np.int32), _c(off2, np.int32)
    flows = np.empty((3, H, W, 2), np.int32)
    valid = np.empty((H, W), np.uint8)
    err = np.empty((H, W), np.int32)
    sp = np.empty((((W + 2) // 3) * ((H + 2) // 3), 4), np.int32)
    mask = np.empty((H, W), np.uint8)
    ev = C.c_int64()
    n = lib().ffo_sift_flow_fields(_p(I1, C.c_uint8), _p(I2, C.c_uint8), W, H,
                                   C.byref(Params(**P)), _p(B1, C.c_int16), _p(off1, C.c_int32),
                                   B1.shape[0], _p(B2, C.c_int16), _p(off2, C.c_int32),
                                   B2.shape[0], threads, _p(flows, C.c_int32),
                                   _p(valid, C.c_uint8), _p(err, C.c_int32), _p(sp, C.c_int32),
                                   _p(mask, C.c_uint8), C.byref(ev))
    return dict(flows=flows, valid=valid, err_sum=err, sparse=sp[:n].copy(), mask=mask,
                evals=ev.value)
