"""The allocation-free filter entry point against the workspace one.

ff_consistency_filter_static serves callers that cannot allocate device memory
(a plugin inside a framework that owns the memory pool, or a real-time loop that
must not call cudaMalloc after start-up): it takes its scratch from a static
device array inside the library. This test calls it through the C ABI twice in a
row, on different inputs, and checks every output against ff_consistency_filter
on the same inputs. The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1508_05151_gb300 import ffapi, synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _flows(seed, W, H):
    """Three consistent-ish flows with a sprinkling of outliers (int16)."""
    rng = np.random.default_rng(seed)
    p = synth.pair_shift(seed, W=W, H=H, max_shift=(6, 6), square=min(24, W, H),
                         square_move=8)
    F = p["flow"].astype(np.int32)
    ys, xs = np.mgrid[0:H, 0:W]
    out = []
    for j in range(3):
        f = (-F if j else F).copy()
        m = rng.random((H, W)) < 0.08
        f[m] += rng.integers(-7, 8, size=(int(m.sum()), 2))
        f[..., 0] = np.clip(xs + f[..., 0], 0, W - 1) - xs
        f[..., 1] = np.clip(ys + f[..., 1], 0, H - 1) - ys
        out.append(torch.from_numpy(f.astype(np.int16)).cuda())
    return out


@pytest.mark.parametrize("W,H,seeds", [(128, 96, (3, 4)), (1024, 436, (5, 6))])
def test_static_filter_matches_workspace_filter_twice(W, H, seeds):
    params = dict(eps=2, e=3, s=40)
    for seed in seeds:  # two calls in a row: the shared array keeps old contents
        F, Fb1, Fb2 = _flows(seed, W, H)
        ref = ffapi.ff_consistency_filter(F, Fb1, Fb2, params)
        got = ffapi.ff_consistency_filter_static(F, Fb1, Fb2, params)
        torch.cuda.synchronize()
        for k in ("valid", "err_sum", "mask", "n_sparse"):
            assert torch.equal(got[k], ref[k]), (seed, k)
        n = int(ref["n_sparse"].item())
        assert n > 0
        assert torch.equal(got["sparse"][:n], ref["sparse"][:n])


def test_static_filter_rejects_what_the_workspace_filter_rejects():
    L = ffapi.lib()
    p = ffapi.Params()
    fake = C.c_void_p(0x1000)
    # refused on the host, nothing enqueued: 2^20 + 1 pixels, a width above 16384,
    # and parameters ff_consistency_filter refuses (odd tile)
    assert L.ff_consistency_filter_static(fake, fake, fake, 1025, 1024, C.byref(p), fake, fake,
                                          fake, fake, fake, None) == 2
    assert L.ff_consistency_filter_static(fake, fake, fake, 20000, 1, C.byref(p), fake, fake,
                                          fake, fake, fake, None) == 2
    bad = ffapi.Params(tile=31)
    assert L.ff_consistency_filter_static(fake, fake, fake, 64, 48, C.byref(bad), fake, fake,
                                          fake, fake, fake, None) == 1
