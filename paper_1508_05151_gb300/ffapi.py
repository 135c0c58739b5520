"""Thin Python binding of the C ABI in include/flowfields.h.

Functions carry the ABI's names. They take and return torch CUDA tensors, which
serve only as device memory; every step runs in the library's CUDA kernels on
torch's current stream. There is no CPU path: if the library is missing or no
GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import torch

from . import _build

FF_OK = 0
COST_UNSET = 2**31 - 1
_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported image shape",
           3: "workspace missing, misaligned or too small", 4: "CUDA error",
           5: "device-side check failed"}


class FFError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {_STATUS.get(code, code)} ({code})")
        self.code = code


class Pair(C.Structure):
    """ff_pair: one image pair of a batch (device pointers)."""
    _fields_ = [("I1", C.c_void_p), ("I2", C.c_void_p), ("W", C.c_int), ("H", C.c_int),
                ("proposals", C.c_void_p), ("flows", C.c_void_p), ("valid", C.c_void_p),
                ("err_sum", C.c_void_p), ("sparse", C.c_void_p), ("n_sparse", C.c_void_p),
                ("mask", C.c_void_p)]


class ExecParams(C.Structure):
    """ff_exec_params: launch shapes that never change results."""
    _fields_ = [("pass_warps", C.c_int32), ("rs_min_n", C.c_int32), ("wide_min_n", C.c_int32),
                ("split8_min_n", C.c_int32), ("serial_flows", C.c_int32),
                ("kd_merge", C.c_int32), ("persist_levels", C.c_int32),
                ("split2_max_n", C.c_int32)]


class NetDesc(C.Structure):
    """ff_net_desc: proposal-net shape."""
    _fields_ = [("cin", C.c_int32), ("c1", C.c_int32), ("c2", C.c_int32), ("c3", C.c_int32),
                ("k", C.c_int32), ("dil", C.c_int32 * 4)]


class Params(C.Structure):
    """ff_params; defaults are the Sintel preset of Sec. 4."""
    _fields_ = [(n, C.c_int32) for n in
                ("k", "r", "r2", "leaf", "R", "eps", "e", "s", "tile", "n_rs", "K", "color",
                 "subpel")] + [("seed", C.c_uint64)]

    def __init__(self, **kw):
        d = dict(k=3, r=8, r2=6, leaf=8, R=1, eps=5, e=4, s=50, tile=16, n_rs=3, K=0, color=0,
                 subpel=1, seed=0)
        unknown = set(kw) - set(d)
        if unknown:
            raise TypeError(f"unknown parameters {sorted(unknown)}")
        d.update(kw)
        super().__init__(**d)

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def header_functions():
    """Names of the entry points declared in include/flowfields.h."""
    with open(os.path.join(_build.INCLUDE, "flowfields.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:ff_status|const char \*)\s*(ff_\w+)\s*\(", txt, re.M)))


def lib():
    """Load libflowfields.so (building it first when sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, sz, i32, u64 = C.c_void_p, C.c_size_t, C.c_int, C.c_uint64
        P = C.POINTER(Params)
        sig = {
            "ff_status_str": ([i32], C.c_char_p),
            "ff_params_preset": ([P, i32], i32),
            "ff_workspace_size": ([i32, i32, P, C.POINTER(sz)], i32),
            "ff_smooth_workspace_size": ([i32, i32, i32, C.POINTER(sz)], i32),
            "ff_smooth": ([vp, i32, i32, i32, vp, vp, sz, vp], i32),
            "ff_census": ([vp, i32, i32, i32, vp, vp], i32),
            "ff_rgb_to_lab": ([vp, i32, i32, vp, vp], i32),
            "ff_median_workspace_size": ([i32, i32, C.POINTER(sz)], i32),
            "ff_weighted_median": ([vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, sz, vp], i32),
            "ff_features": ([vp, i32, i32, i32, vp, i32, vp, vp], i32),
            "ff_kdtree_size": ([i32, i32, C.POINTER(C.c_int), C.POINTER(sz)], i32),
            "ff_kdtree_build": ([vp, i32, i32, vp, vp, vp, vp, sz, vp], i32),
            "ff_kdtree_init": ([vp, vp, vp, i32, vp, vp, vp, i32, i32, i32, i32, vp, i32, vp, vp,
                                vp, sz, vp], i32),
            "ff_level_workspace_size": ([i32, i32, i32, C.POINTER(sz)], i32),
            "ff_search_level": ([vp, vp, i32, i32, i32, i32, vp, P, i32, vp, vp, vp, sz, vp], i32),
            "ff_filter_workspace_size": ([i32, i32, C.POINTER(sz)], i32),
            "ff_consistency_filter": ([vp, vp, vp, i32, i32, P, vp, vp, vp, vp, vp, vp, sz, vp],
                                      i32),
            "ff_consistency_filter_static": ([vp, vp, vp, i32, i32, P, vp, vp, vp, vp, vp, vp],
                                             i32),
            "ff_flow_fields": ([vp, vp, i32, i32, P, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], i32),
            "ff_batch_workspace_size": ([i32, C.POINTER(Pair), P, C.POINTER(sz)], i32),
            "ff_flow_fields_batch": ([i32, C.POINTER(Pair), P, vp, sz, vp], i32),
            "ff_graph_create": ([i32, C.POINTER(Pair), P, vp, sz, vp, C.POINTER(vp)], i32),
            "ff_graph_launch": ([vp, vp], i32),
            "ff_graph_kernel_count": ([vp, C.POINTER(u64)], i32),
            "ff_graph_destroy": ([vp], i32),
            "ff_set_exec_params": ([C.POINTER(ExecParams)], i32),
            "ff_net_param_count": ([C.POINTER(NetDesc), C.POINTER(sz)], i32),
            "ff_net_workspace_size": ([C.POINTER(NetDesc), i32, i32, i32, C.POINTER(sz)], i32),
            "ff_net_input": ([vp, vp, i32, i32, i32, vp, vp], i32),
            "ff_net_forward": ([C.POINTER(NetDesc), vp, vp, i32, i32, i32, vp, vp, sz, vp], i32),
            "ff_net_loss": ([C.POINTER(NetDesc), vp, vp, vp, i32, i32, i32, C.c_float, C.c_float,
                             vp, vp, vp, vp], i32),
            "ff_net_backward": ([C.POINTER(NetDesc), vp, vp, i32, i32, i32, vp, vp, sz, vp], i32),
            "ff_net_adam": ([sz, vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float,
                             vp], i32),
            "ff_net_proposals": ([C.POINTER(NetDesc), vp, i32, i32, i32, C.c_float, vp, vp], i32),
            "ff_get_exec_params": ([C.POINTER(ExecParams)], i32),
            "ff_set_wait_test": ([C.c_longlong, i32, i32], i32),
            "ff_device_status": ([vp, C.POINTER(C.c_uint32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), vp], i32),
            "ff_profile_enable": ([i32], i32),
            "ff_profile_reset": ([], i32),
            "ff_profile_read": ([C.POINTER(u64), C.POINTER(C.c_double), C.POINTER(u64)], i32),
            "ff_profile_levels": ([C.POINTER(C.c_double), C.POINTER(u64)], i32),
            "ff_profile_evals": ([C.POINTER(u64)], i32),
            "ff_profile_marks": ([C.POINTER(C.c_int32), C.POINTER(C.c_double), i32,
                                  C.POINTER(C.c_int)], i32),
            "ff_sift_descriptors": ([vp, i32, i32, vp, vp], i32),
            "ff_sift_moments": ([vp, i32, vp, vp, vp], i32),
            "ff_sift_pca_workspace_size": ([C.POINTER(sz)], i32),
            "ff_sift_pca": ([vp, vp, C.c_int64, i32, vp, vp, vp, vp, sz, vp], i32),
            "ff_sift_colors": ([vp, i32, i32, vp, vp, i32, vp, vp], i32),
            "ff_sift_level_workspace_size": ([i32, i32, i32, i32, C.POINTER(sz)], i32),
            "ff_sift_kdtree_init": ([vp, vp, vp, i32, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp,
                                     vp, sz, vp], i32),
            "ff_sift_search_level": ([vp, vp, i32, i32, i32, i32, i32, vp, P, i32, vp, vp, vp, sz,
                                      vp], i32),
            "ff_sift_workspace_size": ([i32, i32, P, i32, i32, C.POINTER(sz)], i32),
            "ff_sift_flow_fields": ([vp, vp, i32, i32, P, vp, vp, i32, vp, vp, i32, vp, vp, vp,
                                     vp, vp, vp, vp, sz, vp], i32),
            "ff_probe_popc": ([vp, i32, i32, vp], i32),
            "ff_probe_smem_taps": ([vp, i32, i32, vp], i32),
            "ff_probe_l2_gather": ([vp, sz, i32, vp, i32, i32, C.POINTER(u64), vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(fn, code):
    if code != FF_OK:
        raise FFError(fn, code)


def _dev(t):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _opt(t):
    return C.c_void_p(None) if t is None else _dev(t)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ws(nbytes, device):
    # torch's allocator returns 512-byte aligned blocks; +256 guards the rounding
    return torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)


def _ws_ptr(ws):
    p = ws.data_ptr()
    return C.c_void_p((p + 255) & ~255), ws.numel() - (((p + 255) & ~255) - p)


def _size(fn, *args):
    out = C.c_size_t()
    _check(fn, getattr(lib(), fn)(*args, C.byref(out)))
    return out.value


def _params(p):
    if p is None:
        return Params()
    if isinstance(p, dict):
        return Params(**p)
    return p


# ------------------------------------------------------------------ steps ----
def ff_smooth(img, n):
    H, W = img.shape[:2]
    out = torch.empty_like(img)
    ws = _ws(_size("ff_smooth_workspace_size", W, H, n), img.device)
    wp, wn = _ws_ptr(ws)
    _check("ff_smooth", lib().ff_smooth(_dev(img), W, H, n, _dev(out), wp, wn, _stream()))
    return out


def ff_rgb_to_lab(img):
    """Integer CIELab (uint8 L*255/100, a+128, b+128) of an (H, W, 3) sRGB image."""
    H, W = img.shape[:2]
    out = torch.empty_like(img)
    _check("ff_rgb_to_lab", lib().ff_rgb_to_lab(_dev(img), W, H, _dev(out), _stream()))
    return out


def ff_weighted_median(I1, I2, flow, r=8, rho=2):
    """The raw forward field filtered by the matching-error-weighted median
    ("k=3+median" of Table 1). Returns (filtered flow int16 (H, W, 2), E int32)."""
    H, W = I1.shape[:2]
    nb = _size("ff_median_workspace_size", W, H)
    ws = _ws(nb, I1.device)
    wp, wn = _ws_ptr(ws)
    out = torch.empty((H, W, 2), dtype=torch.int16, device=I1.device)
    E = torch.empty((H, W), dtype=torch.int32, device=I1.device)
    _check("ff_weighted_median", lib().ff_weighted_median(
        _dev(I1), _dev(I2), _dev(flow), W, H, r, rho, _dev(out), _dev(E), wp, wn, _stream()))
    return out, E


def ff_census(img_n, n):
    H, W = img_n.shape[:2]
    out = torch.empty((H, W), dtype=torch.int32, device=img_n.device)
    _check("ff_census", lib().ff_census(_dev(img_n), W, H, n, _dev(out), _stream()))
    return out


def ff_features(img, r, pts=None):
    H, W = img.shape[:2]
    npts = H * W if pts is None else int(pts.shape[0])
    out = torch.empty((max(npts, 1), 28), dtype=torch.int32, device=img.device)
    _check("ff_features", lib().ff_features(_dev(img), W, H, r, _opt(pts), npts, _dev(out),
                                            _stream()))
    return out[:npts]


def ff_kdtree_build(feat, leaf):
    N = int(feat.shape[0])
    D = C.c_int()
    nbytes = C.c_size_t()
    _check("ff_kdtree_size", lib().ff_kdtree_size(N, leaf, C.byref(D), C.byref(nbytes)))
    dev = feat.device
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    nn = max((1 << D.value) - 1, 1)
    sd = torch.zeros(nn, dtype=torch.int32, device=dev)
    sv = torch.zeros(nn, dtype=torch.int32, device=dev)
    ws = _ws(nbytes.value, dev)
    wp, wn = _ws_ptr(ws)
    _check("ff_kdtree_build", lib().ff_kdtree_build(_dev(feat), N, leaf, _dev(perm), _dev(sd),
                                                    _dev(sv), wp, wn, _stream()))
    return dict(perm=perm, split_dim=sd[:(1 << D.value) - 1], split_val=sv[:(1 << D.value) - 1],
                D=D.value, N=N, _keep=(sd, sv))


def _grid(W, H, n):
    return (W + n - 1) // n, (H + n - 1) // n


def ff_kdtree_init(tree, leaf, src_img, census_src, census_tgt, n, r, proposals=None,
                   with_status=False):
    """Initial flow at the grid of spacing n from a kd tree (Eq. 1 / Eq. 4).
    Returns (flow, cost), plus the device status (code, x, y) with with_status."""
    H, W = src_img.shape[:2]
    Gx, Gy = _grid(W, H, n)
    dev = src_img.device
    flow = torch.empty((Gy, Gx, 2), dtype=torch.int16, device=dev)
    cost = torch.empty((Gy, Gx), dtype=torch.int32, device=dev)
    ws = _ws(_size("ff_level_workspace_size", W, H, n), dev)
    wp, wn = _ws_ptr(ws)
    K = 0 if proposals is None else int(proposals.shape[2])
    sd, sv = tree["_keep"]
    _check("ff_kdtree_init", lib().ff_kdtree_init(
        _dev(tree["perm"]), _dev(sd), _dev(sv), leaf, _dev(src_img), _dev(census_src),
        _dev(census_tgt), W, H, n, r, _opt(proposals), K, _dev(flow), _dev(cost), wp, wn,
        _stream()))
    if with_status:
        code, x, y = C.c_uint32(), C.c_int32(), C.c_int32()
        # the call itself returns an error status when a device check failed
        lib().ff_device_status(wp, C.byref(code), C.byref(x), C.byref(y), _stream())
        return flow, cost, (code.value, x.value, y.value)
    return flow, cost


def ff_search_level(census_src, census_tgt, n, r, params=None, flow_id=0, flow_coarse=None,
                    flow=None, cost=None):
    """One level. With flow_coarse: seeded from it; else (flow, cost) is the initial
    state and is updated in place. Returns (flow, cost)."""
    H, W = census_src.shape
    Gx, Gy = _grid(W, H, n)
    dev = census_src.device
    if flow_coarse is not None:
        flow = torch.empty((Gy, Gx, 2), dtype=torch.int16, device=dev)
        cost = torch.empty((Gy, Gx), dtype=torch.int32, device=dev)
    P = _params(params)
    ws = _ws(_size("ff_level_workspace_size", W, H, n), dev)
    wp, wn = _ws_ptr(ws)
    _check("ff_search_level", lib().ff_search_level(
        _dev(census_src), _dev(census_tgt), W, H, n, r, _opt(flow_coarse), C.byref(P), flow_id,
        _dev(flow), _dev(cost), wp, wn, _stream()))
    return flow, cost


def ff_consistency_filter(F, Fb1, Fb2, params=None):
    H, W = F.shape[:2]
    dev = F.device
    P = _params(params)
    valid = torch.empty((H, W), dtype=torch.uint8, device=dev)
    err = torch.empty((H, W), dtype=torch.int32, device=dev)
    nb = ((W + 2) // 3) * ((H + 2) // 3)
    sparse = torch.empty((nb, 4), dtype=torch.int32, device=dev)
    ns = torch.zeros(1, dtype=torch.int32, device=dev)
    mask = torch.empty((H, W), dtype=torch.uint8, device=dev)
    ws = _ws(_size("ff_filter_workspace_size", W, H), dev)
    wp, wn = _ws_ptr(ws)
    _check("ff_consistency_filter", lib().ff_consistency_filter(
        _dev(F), _dev(Fb1), _dev(Fb2), W, H, C.byref(P), _dev(valid), _dev(err), _dev(sparse),
        _dev(ns), _dev(mask), wp, wn, _stream()))
    return dict(valid=valid, err_sum=err, sparse=sparse, n_sparse=ns, mask=mask)


def ff_consistency_filter_static(F, Fb1, Fb2, params=None, out=None):
    """ff_consistency_filter without a workspace: the library's static scratch
    array is used (images up to 2^20 pixels; calls must not overlap on the GPU).
    Outputs may be passed preallocated in ``out`` (same keys as the result)."""
    H, W = F.shape[:2]
    dev = F.device
    P = _params(params)
    if out is None:
        nb = ((W + 2) // 3) * ((H + 2) // 3)
        out = dict(valid=torch.empty((H, W), dtype=torch.uint8, device=dev),
                   err_sum=torch.empty((H, W), dtype=torch.int32, device=dev),
                   sparse=torch.empty((nb, 4), dtype=torch.int32, device=dev),
                   n_sparse=torch.zeros(1, dtype=torch.int32, device=dev),
                   mask=torch.empty((H, W), dtype=torch.uint8, device=dev))
    _check("ff_consistency_filter_static", lib().ff_consistency_filter_static(
        _dev(F), _dev(Fb1), _dev(Fb2), W, H, C.byref(P), _dev(out["valid"]),
        _dev(out["err_sum"]), _dev(out["sparse"]), _dev(out["n_sparse"]), _dev(out["mask"]),
        _stream()))
    return out


class FlowFields:
    """The whole path for W x H pairs with one reusable workspace.

    ``run(I1, I2)`` takes uint8 (H, W, 3) CUDA tensors and returns device tensors:
    flows int16 (3, H, W, 2) (forward, backward r, backward r2), valid, err_sum,
    sparse int32 (rows, 4) with the row count in n_sparse, mask.
    """

    def __init__(self, W, H, params=None, device="cuda"):
        self.W, self.H = W, H
        self.params = _params(params)
        self.device = torch.device(device)
        self.ws_bytes = _size("ff_workspace_size", W, H, C.byref(self.params))
        self.ws = _ws(self.ws_bytes, self.device)
        nb = ((W + 2) // 3) * ((H + 2) // 3)
        d = self.device
        self.flows = torch.empty((3, H, W, 2), dtype=torch.int16, device=d)
        self.valid = torch.empty((H, W), dtype=torch.uint8, device=d)
        self.err_sum = torch.empty((H, W), dtype=torch.int32, device=d)
        self.sparse = torch.empty((nb, 4), dtype=torch.int32, device=d)
        self.n_sparse = torch.zeros(1, dtype=torch.int32, device=d)
        self.mask = torch.empty((H, W), dtype=torch.uint8, device=d)

    def run(self, I1, I2, proposals=None):
        wp, wn = _ws_ptr(self.ws)
        _check("ff_flow_fields", lib().ff_flow_fields(
            _dev(I1), _dev(I2), self.W, self.H, C.byref(self.params), _opt(proposals),
            _dev(self.flows), _dev(self.valid), _dev(self.err_sum), _dev(self.sparse),
            _dev(self.n_sparse), _dev(self.mask), wp, wn, _stream()))
        return dict(flows=self.flows, valid=self.valid, err_sum=self.err_sum,
                    sparse=self.sparse, n_sparse=self.n_sparse, mask=self.mask)

    def device_status(self):
        wp, _ = _ws_ptr(self.ws)
        code, x, y = C.c_uint32(), C.c_int32(), C.c_int32()
        lib().ff_device_status(wp, C.byref(code), C.byref(x), C.byref(y), _stream())
        return code.value, x.value, y.value


def ff_flow_fields(I1, I2, params=None, proposals=None):
    H, W = I1.shape[:2]
    return FlowFields(W, H, params, I1.device).run(I1, I2, proposals)


# ------------------------------------------------------------ SIFT flow ----
# Sec. 3.3, the second data term. Colours are uint8 (S/3, H, W, 3) groups.

def ff_sift_descriptors(img):
    """Dense SIFT vectors of an RGB frame: uint8 (H, W, 128)."""
    H, W = img.shape[:2]
    desc = torch.empty((H, W, 128), dtype=torch.uint8, device=img.device)
    _check("ff_sift_descriptors", lib().ff_sift_descriptors(_dev(img), W, H, _dev(desc),
                                                            _stream()))
    return desc


def ff_sift_moments(desc, acc=None):
    """Exact PCA statistics of the descriptors, added to acc = (sum, gram, count)
    when given. Returns (sum uint64 [128] as int64, gram [128, 128], count)."""
    dev = desc.device
    if acc is None:
        sm = torch.zeros(128, dtype=torch.int64, device=dev)
        gram = torch.zeros((128, 128), dtype=torch.int64, device=dev)
        count = 0
    else:
        sm, gram, count = acc
    N = desc.numel() // 128
    _check("ff_sift_moments", lib().ff_sift_moments(_dev(desc), N, _dev(sm), _dev(gram),
                                                    _stream()))
    return sm, gram, count + N


def ff_sift_pca(sm, gram, count, S, with_status=False):
    """PCA basis (int16 [S, 128]), offsets (int32 [S]) and eigenvalues (float64
    [128], descending) from the moments."""
    dev = sm.device
    basis = torch.empty((S, 128), dtype=torch.int16, device=dev)
    off = torch.empty(S, dtype=torch.int32, device=dev)
    eig = torch.empty(128, dtype=torch.float64, device=dev)
    ws = _ws(_size("ff_sift_pca_workspace_size"), dev)
    wp, wn = _ws_ptr(ws)
    _check("ff_sift_pca", lib().ff_sift_pca(_dev(sm), _dev(gram), int(count), S, _dev(basis),
                                            _dev(off), _dev(eig), wp, wn, _stream()))
    if with_status:
        code, x, y = C.c_uint32(), C.c_int32(), C.c_int32()
        lib().ff_device_status(wp, C.byref(code), C.byref(x), C.byref(y), _stream())
        return basis, off, eig, (code.value, x.value, y.value)
    return basis, off, eig


def ff_sift_colors(desc, basis, offset):
    H, W = desc.shape[:2]
    S = int(basis.shape[0])
    col = torch.empty((S // 3, H, W, 3), dtype=torch.uint8, device=desc.device)
    _check("ff_sift_colors", lib().ff_sift_colors(_dev(desc), W, H, _dev(basis), _dev(offset), S,
                                                  _dev(col), _stream()))
    return col


def ff_sift_smooth(col, n):
    """Every colour group smoothed like I^n (Sec. 3.2), by ff_smooth."""
    return torch.stack([ff_smooth(g.contiguous(), n) for g in col])


def ff_sift_kdtree_init(tree, leaf, src_img, col_src, col_tgt, n, r, with_status=False):
    """Initial flow at the grid of spacing n with the SIFT flow data term. Returns
    (flow, cost), plus the device status (code, x, y) with with_status."""
    G3, H, W = col_src.shape[:3]
    Gx, Gy = _grid(W, H, n)
    dev = src_img.device
    flow = torch.empty((Gy, Gx, 2), dtype=torch.int16, device=dev)
    cost = torch.empty((Gy, Gx), dtype=torch.int32, device=dev)
    ws = _ws(_size("ff_sift_level_workspace_size", W, H, n, 3 * G3), dev)
    wp, wn = _ws_ptr(ws)
    sd, sv = tree["_keep"]
    _check("ff_sift_kdtree_init", lib().ff_sift_kdtree_init(
        _dev(tree["perm"]), _dev(sd), _dev(sv), leaf, _dev(src_img), _dev(col_src),
        _dev(col_tgt), 3 * G3, W, H, n, r, _dev(flow), _dev(cost), wp, wn, _stream()))
    if with_status:
        code, x, y = C.c_uint32(), C.c_int32(), C.c_int32()
        lib().ff_device_status(wp, C.byref(code), C.byref(x), C.byref(y), _stream())
        return flow, cost, (code.value, x.value, y.value)
    return flow, cost


def ff_sift_search_level(col_src, col_tgt, n, r, params=None, flow_id=0, flow_coarse=None,
                         flow=None, cost=None):
    """One level with the SIFT flow data term (as ff_search_level)."""
    G3, H, W = col_src.shape[:3]
    Gx, Gy = _grid(W, H, n)
    dev = col_src.device
    if flow_coarse is not None:
        flow = torch.empty((Gy, Gx, 2), dtype=torch.int16, device=dev)
        cost = torch.empty((Gy, Gx), dtype=torch.int32, device=dev)
    P = _params(params)
    ws = _ws(_size("ff_sift_level_workspace_size", W, H, n, 3 * G3), dev)
    wp, wn = _ws_ptr(ws)
    _check("ff_sift_search_level", lib().ff_sift_search_level(
        _dev(col_src), _dev(col_tgt), 3 * G3, W, H, n, r, _opt(flow_coarse), C.byref(P), flow_id,
        _dev(flow), _dev(cost), wp, wn, _stream()))
    return flow, cost


class SiftFlowFields:
    """The whole path with the SIFT flow data term for W x H pairs: bases
    (basis, offset) of S1 channels for the forward and first backward flow and of
    S2 channels for the second backward flow. ``run`` returns the dict of
    FlowFields.run."""

    def __init__(self, W, H, basis1, offset1, basis2, offset2, params=None, device="cuda"):
        self.W, self.H = W, H
        self.params = _params(params)
        self.device = torch.device(device)
        self.b = (basis1.contiguous(), offset1.contiguous(), basis2.contiguous(),
                  offset2.contiguous())
        self.S1, self.S2 = int(basis1.shape[0]), int(basis2.shape[0])
        self.ws_bytes = _size("ff_sift_workspace_size", W, H, C.byref(self.params), self.S1,
                              self.S2)
        self.ws = _ws(self.ws_bytes, self.device)
        nb = ((W + 2) // 3) * ((H + 2) // 3)
        d = self.device
        self.flows = torch.empty((3, H, W, 2), dtype=torch.int16, device=d)
        self.valid = torch.empty((H, W), dtype=torch.uint8, device=d)
        self.err_sum = torch.empty((H, W), dtype=torch.int32, device=d)
        self.sparse = torch.empty((nb, 4), dtype=torch.int32, device=d)
        self.n_sparse = torch.zeros(1, dtype=torch.int32, device=d)
        self.mask = torch.empty((H, W), dtype=torch.uint8, device=d)

    def run(self, I1, I2):
        wp, wn = _ws_ptr(self.ws)
        b1, o1, b2, o2 = self.b
        _check("ff_sift_flow_fields", lib().ff_sift_flow_fields(
            _dev(I1), _dev(I2), self.W, self.H, C.byref(self.params), _dev(b1), _dev(o1),
            self.S1, _dev(b2), _dev(o2), self.S2, _dev(self.flows), _dev(self.valid),
            _dev(self.err_sum), _dev(self.sparse), _dev(self.n_sparse), _dev(self.mask), wp, wn,
            _stream()))
        return dict(flows=self.flows, valid=self.valid, err_sum=self.err_sum,
                    sparse=self.sparse, n_sparse=self.n_sparse, mask=self.mask)


def ff_sift_flow_fields(I1, I2, basis1, offset1, basis2, offset2, params=None):
    H, W = I1.shape[:2]
    return SiftFlowFields(W, H, basis1, offset1, basis2, offset2, params, I1.device).run(I1, I2)


def profile_enable(on=True, count_evals=False, marks=False):
    """Events around every propagation launch (on), device counters of the
    propagation kernels' candidate evaluations (count_evals), timing events at the
    phase boundaries of a pair (marks)."""
    _check("ff_profile_enable", lib().ff_profile_enable(
        (1 if on else 0) | (2 if count_evals else 0) | (4 if marks else 0)))


MARK_PHASES = {0: "start", 1: "pyramid", 2: "features", 3: "kd_build", 4: "kd_query",
               20: "joined", 21: "filter"}
MARK_GROUPS = {0: "fwd", 1: "bwd1", 2: "bwd2", 3: "shared"}


def profile_marks(cap=4096):
    """Recorded phase marks: list of (group, phase, ms since the first mark)."""
    tags = (C.c_int32 * cap)()
    ms = (C.c_double * cap)()
    n = C.c_int()
    _check("ff_profile_marks", lib().ff_profile_marks(tags, ms, cap, C.byref(n)))
    out = []
    for i in range(min(n.value, cap)):
        g, ph = divmod(tags[i], 100)
        name = MARK_PHASES.get(ph, f"level{1 << (ph - 10)}" if 10 <= ph < 20 else str(ph))
        out.append((MARK_GROUPS.get(g, str(g)), name, ms[i]))
    return out


def profile_reset():
    _check("ff_profile_reset", lib().ff_profile_reset())


def profile_read():
    n, ms, pn = C.c_uint64(), C.c_double(), C.c_uint64()
    _check("ff_profile_read", lib().ff_profile_read(C.byref(n), C.byref(ms), C.byref(pn)))
    return dict(launches=n.value, prop_ms=ms.value, prop_launches=pn.value)


def profile_levels():
    """Per level l (spacing 2^l, l = 0..4): summed propagation-launch ms, launches."""
    ms = (C.c_double * 5)()
    n = (C.c_uint64 * 5)()
    _check("ff_profile_levels", lib().ff_profile_levels(ms, n))
    return [dict(ms=ms[l], launches=n[l]) for l in range(5)]


EVAL_KINDS = ("inc_window", "inc_planes", "full_window", "full_planes")


def profile_evals():
    """Candidate evaluations counted since the last reset: {(r, l): {kind: count}}
    for every radius r and level l (spacing 2^l) with a non-zero count."""
    c = (C.c_uint64 * (9 * 5 * 4))()
    _check("ff_profile_evals", lib().ff_profile_evals(c))
    out = {}
    for r in range(9):
        for l in range(5):
            v = [c[(r * 5 + l) * 4 + k] for k in range(4)]
            if any(v):
                out[(r, l)] = dict(zip(EVAL_KINDS, v))
    return out


def eval_taps(r, counts):
    """Target taps read for evaluation counts of radius r: an incremental
    evaluation reads two patch lines (2 (2r+1) taps), a full one (2r+1)^2."""
    L = 2 * r + 1
    inc = counts["inc_window"] + counts["inc_planes"]
    full = counts["full_window"] + counts["full_planes"]
    planes = 2 * L * counts["inc_planes"] + L * L * counts["full_planes"]
    return dict(taps=2 * L * inc + L * L * full, taps_from_planes=planes)


def probe_popc(sink, blocks, iters):
    _check("ff_probe_popc", lib().ff_probe_popc(_dev(sink), blocks, iters, _stream()))
    return 4096 * iters * blocks


def probe_smem_taps(sink, blocks, iters):
    _check("ff_probe_smem_taps", lib().ff_probe_smem_taps(_dev(sink), blocks, iters, _stream()))
    return 4096 * iters * blocks


def probe_l2_gather(buf, mode, sink, blocks, iters):
    nb = C.c_uint64()
    _check("ff_probe_l2_gather", lib().ff_probe_l2_gather(_dev(buf), buf.numel(), mode, _dev(sink),
                                                          blocks, iters, C.byref(nb), _stream()))
    return nb.value


EXEC_FIELDS = ("pass_warps", "rs_min_n", "wide_min_n", "split8_min_n", "serial_flows",
               "kd_merge", "persist_levels", "split2_max_n")


def set_exec_params(**kw):
    """Set execution parameters (names of EXEC_FIELDS); the others keep their value."""
    unknown = set(kw) - set(EXEC_FIELDS)
    if unknown:
        raise TypeError(f"unknown execution parameters {sorted(unknown)}")
    cur = get_exec_params()
    cur.update({k: v for k, v in kw.items() if v is not None})
    e = ExecParams(**cur)
    _check("ff_set_exec_params", lib().ff_set_exec_params(C.byref(e)))


def get_exec_params():
    e = ExecParams()
    _check("ff_get_exec_params", lib().ff_get_exec_params(C.byref(e)))
    return {k: getattr(e, k) for k in EXEC_FIELDS}


class FlowFieldsBatch:
    """Batched form: many pairs of (possibly) different sizes per call.

    ``sizes``: list of (W, H). ``run(frames)`` takes a list of (I1, I2) uint8 CUDA
    tensors and returns one result dict per pair (views of preallocated output
    tensors). With ``graph=True`` the first run captures the whole batch into a
    CUDA graph bound to internal input buffers and later runs replay it; inputs
    (and, when ``params.K > 0``, the proposals) are copied into those buffers.
    """

    def __init__(self, sizes, params=None, device="cuda", graph=False):
        self.sizes = [tuple(map(int, s)) for s in sizes]
        self.params = _params(params)
        self.device = torch.device(device)
        d = self.device
        self.out = []
        self.inp = []
        for (W, H) in self.sizes:
            nb = ((W + 2) // 3) * ((H + 2) // 3)
            self.out.append(dict(
                flows=torch.empty((3, H, W, 2), dtype=torch.int16, device=d),
                valid=torch.empty((H, W), dtype=torch.uint8, device=d),
                err_sum=torch.empty((H, W), dtype=torch.int32, device=d),
                sparse=torch.empty((nb, 4), dtype=torch.int32, device=d),
                n_sparse=torch.zeros(1, dtype=torch.int32, device=d),
                mask=torch.empty((H, W), dtype=torch.uint8, device=d)))
            self.inp.append((torch.empty((H, W, 3), dtype=torch.uint8, device=d),
                             torch.empty((H, W, 3), dtype=torch.uint8, device=d)))
        # graph mode binds proposal buffers too when the forward flow takes K of them
        K, n = self.params.K, 1 << self.params.k
        self.prop = [torch.zeros(((H + n - 1) // n, (W + n - 1) // n, K, 2), dtype=torch.int16,
                                 device=d) for (W, H) in self.sizes] if (graph and K > 0) else None
        self.pairs = (Pair * len(self.sizes))()
        self._fill_pairs(self.inp, self.prop)
        n = C.c_size_t()
        _check("ff_batch_workspace_size", lib().ff_batch_workspace_size(
            len(self.sizes), self.pairs, C.byref(self.params), C.byref(n)))
        self.ws = _ws(n.value, d)
        self.use_graph = graph
        self.graph = None
        # graphs are captured and replayed on a stream of their own (the legacy
        # default stream cannot be captured), ordered after the caller's stream
        self.stream = torch.cuda.Stream(device=d) if graph else None

    def _fill_pairs(self, frames, proposals=None):
        for i, ((W, H), (a, b)) in enumerate(zip(self.sizes, frames)):
            o = self.out[i]
            if tuple(a.shape[:2]) != (H, W) or tuple(b.shape[:2]) != (H, W):
                raise ValueError(f"pair {i}: expected {W}x{H}")
            pr = proposals[i] if proposals is not None else None
            self.pairs[i] = Pair(a.data_ptr(), b.data_ptr(), W, H,
                                 pr.data_ptr() if pr is not None else None,
                                 o["flows"].data_ptr(), o["valid"].data_ptr(),
                                 o["err_sum"].data_ptr(), o["sparse"].data_ptr(),
                                 o["n_sparse"].data_ptr(), o["mask"].data_ptr())

    def run(self, frames, proposals=None):
        wp, wn = _ws_ptr(self.ws)
        if self.use_graph:
            if (proposals is None) != (self.prop is None):
                raise ValueError("graph mode takes proposals exactly when params.K > 0")
            caller = torch.cuda.current_stream()
            self.stream.wait_stream(caller)
            with torch.cuda.stream(self.stream):
                for (a, b), (da, db) in zip(frames, self.inp):
                    da.copy_(a, non_blocking=True)
                    db.copy_(b, non_blocking=True)
                if proposals is not None:
                    for src, dst in zip(proposals, self.prop):
                        dst.copy_(src.reshape(dst.shape), non_blocking=True)
                if self.graph is None:
                    self._fill_pairs(self.inp, self.prop)
                    g = C.c_void_p()
                    _check("ff_graph_create", lib().ff_graph_create(
                        len(self.sizes), self.pairs, C.byref(self.params), wp, wn, _stream(),
                        C.byref(g)))
                    self.graph = g
                _check("ff_graph_launch", lib().ff_graph_launch(self.graph, _stream()))
            caller.wait_stream(self.stream)
        else:
            self._fill_pairs(frames, proposals)
            _check("ff_flow_fields_batch", lib().ff_flow_fields_batch(
                len(self.sizes), self.pairs, C.byref(self.params), wp, wn, _stream()))
        return self.out

    def graph_kernels(self):
        if self.graph is None:
            return 0
        k = C.c_uint64()
        _check("ff_graph_kernel_count", lib().ff_graph_kernel_count(self.graph, C.byref(k)))
        return k.value

    def __del__(self):
        if getattr(self, "graph", None) is not None and _lib is not None:
            _lib.ff_graph_destroy(self.graph)
            self.graph = None


# ------------------------------------------------------------- proposal net ----
def net_desc(c1=32, c2=64, c3=64, k=4, dil=(1, 2, 4, 8)):
    return NetDesc(6, c1, c2, c3, k, (C.c_int32 * 4)(*dil))


def ff_net_param_count(desc):
    n = C.c_size_t()
    _check("ff_net_param_count", lib().ff_net_param_count(C.byref(desc), C.byref(n)))
    return n.value


def ff_net_input(I1, I2):
    """I1, I2: uint8 [B][H][W][3] CUDA tensors -> x float32 [B][6][Gy][Gx]."""
    B, H, W = I1.shape[:3]
    x = torch.empty((B, 6, (H + 7) // 8, (W + 7) // 8), dtype=torch.float32, device=I1.device)
    _check("ff_net_input", lib().ff_net_input(_dev(I1), _dev(I2), B, W, H, _dev(x), _stream()))
    return x


class NetRunner:
    """Workspace-holding wrapper of the net entry points for one batch shape."""

    def __init__(self, desc, B, Gx, Gy, device="cuda"):
        self.desc, self.B, self.Gx, self.Gy = desc, B, Gx, Gy
        n = C.c_size_t()
        _check("ff_net_workspace_size", lib().ff_net_workspace_size(C.byref(desc), B, Gx, Gy,
                                                                    C.byref(n)))
        self.ws = _ws(n.value, device)
        d = torch.device(device)
        self.out = torch.empty((B, 2 * desc.k, Gy, Gx), dtype=torch.float32, device=d)
        self.dout = torch.empty_like(self.out)
        self.loss = torch.zeros(1, dtype=torch.float32, device=d)
        self.count = torch.zeros(1, dtype=torch.int32, device=d)

    def forward(self, params, x):
        wp, wn = _ws_ptr(self.ws)
        _check("ff_net_forward", lib().ff_net_forward(
            C.byref(self.desc), _dev(params), _dev(x), self.B, self.Gx, self.Gy, _dev(self.out),
            wp, wn, _stream()))
        return self.out

    def loss_grad(self, label, valid, flow_scale, alpha):
        _check("ff_net_loss", lib().ff_net_loss(
            C.byref(self.desc), _dev(self.out), _dev(label), _dev(valid), self.B, self.Gx,
            self.Gy, flow_scale, alpha, _dev(self.loss), _dev(self.dout), _dev(self.count),
            _stream()))
        return self.loss, self.dout

    def backward(self, params, grads, dout=None):
        wp, wn = _ws_ptr(self.ws)
        _check("ff_net_backward", lib().ff_net_backward(
            C.byref(self.desc), _dev(params), _dev(self.dout if dout is None else dout), self.B,
            self.Gx, self.Gy, _dev(grads), wp, wn, _stream()))
        return grads

    def device_status(self):
        wp, _ = _ws_ptr(self.ws)
        code, x, y = C.c_uint32(), C.c_int32(), C.c_int32()
        lib().ff_device_status(wp, C.byref(code), C.byref(x), C.byref(y), _stream())
        return code.value, x.value, y.value

    def proposals(self, flow_scale, out=None):
        o = self.out if out is None else out
        prop = torch.empty((self.B, self.Gy, self.Gx, self.desc.k, 2), dtype=torch.int16,
                           device=o.device)
        _check("ff_net_proposals", lib().ff_net_proposals(
            C.byref(self.desc), _dev(o), self.B, self.Gx, self.Gy, flow_scale, _dev(prop),
            _stream()))
        return prop


def ff_net_adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    _check("ff_net_adam", lib().ff_net_adam(params.numel(), _dev(params), _dev(grads), _dev(m),
                                            _dev(v), step, lr, b1, b2, eps, _stream()))
