"""The C-ABI library builds, loads and exports every declared entry point; host-side
argument checks and workspace planning behave as documented. No GPU needed."""
import ctypes as C
import re
import subprocess

import pytest

from paper_1508_05151_gb300 import ffapi, _build


@pytest.fixture(scope="module")
def L():
    return ffapi.lib()


def test_header_declares_the_boundary():
    names = ffapi.header_functions()
    for must in ("ff_features", "ff_kdtree_build", "ff_kdtree_init", "ff_search_level",
                 "ff_consistency_filter", "ff_flow_fields", "ff_smooth", "ff_census"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(ff_\w+)", out))
    missing = set(ffapi.header_functions()) - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for n in ffapi.header_functions():
        assert hasattr(L, n)


def test_library_is_built_for_sm_103a():
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", _build.LIB],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_presets(L):
    p = ffapi.Params()
    assert L.ff_params_preset(C.byref(p), 0) == 0
    assert (p.k, p.r, p.r2, p.leaf, p.R, p.eps, p.e, p.s) == (3, 8, 6, 8, 1, 5, 4, 50)
    assert L.ff_params_preset(C.byref(p), 1) == 0 and (p.eps, p.e, p.s) == (1, 7, 50)
    assert L.ff_params_preset(C.byref(p), 2) == 0 and (p.eps, p.e, p.s) == (1, 9, 150)
    assert L.ff_params_preset(C.byref(p), 7) == 1
    assert L.ff_params_preset(None, 0) == 1
    assert L.ff_status_str(3) == b"workspace missing, misaligned or too small"


def test_parameter_and_shape_checks(L):
    sz = C.c_size_t()
    ok = ffapi.Params()
    assert L.ff_workspace_size(1024, 436, C.byref(ok), C.byref(sz)) == 0
    assert sz.value > 0
    for bad in [dict(k=5), dict(r=9), dict(r2=0), dict(leaf=1), dict(tile=31), dict(tile=64),
                dict(n_rs=4), dict(K=9), dict(eps=0), dict(e=10), dict(R=-1)]:
        p = ffapi.Params(**bad)
        assert L.ff_workspace_size(64, 64, C.byref(p), C.byref(sz)) == 1, bad
    for W, H in [(0, 5), (5, 0), (20000, 10), (5000, 5000)]:
        assert L.ff_workspace_size(W, H, C.byref(ok), C.byref(sz)) == 2
    assert L.ff_workspace_size(64, 64, None, C.byref(sz)) == 1


def test_workspace_grows_with_size_and_levels(L):
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    p = ffapi.Params()
    L.ff_workspace_size(128, 96, C.byref(p), C.byref(a))
    L.ff_workspace_size(1024, 436, C.byref(p), C.byref(b))
    p0 = ffapi.Params(k=0)
    L.ff_workspace_size(1024, 436, C.byref(p0), C.byref(c))
    assert a.value < b.value
    # 3 feature tables of 112 B per pixel dominate; the basic approach (k = 0)
    # also queries every pixel, so it needs 3 more tables
    assert b.value > 3 * 112 * 1024 * 436
    assert c.value > b.value


def test_calls_reject_null_and_unaligned_workspace_before_any_launch(L):
    p = ffapi.Params()
    fake = C.c_void_p(0x1000)
    # null inputs
    assert L.ff_flow_fields(None, fake, 64, 64, C.byref(p), None, fake, fake, fake, fake, fake,
                            fake, fake, 1 << 30, None) == 1
    # misaligned workspace
    assert L.ff_flow_fields(fake, fake, 64, 64, C.byref(p), None, fake, fake, fake, fake, fake,
                            fake, C.c_void_p(0x1001), 1 << 30, None) == 3
    # too small workspace
    assert L.ff_flow_fields(fake, fake, 64, 64, C.byref(p), None, fake, fake, fake, fake, fake,
                            fake, C.c_void_p(0x100000), 16, None) == 3
    # proposals required when K > 0
    pk = ffapi.Params(K=2)
    assert L.ff_flow_fields(fake, fake, 64, 64, C.byref(pk), None, fake, fake, fake, fake, fake,
                            fake, C.c_void_p(0x100000), 1 << 40, None) == 1
    # smooth: n must be a power of two
    assert L.ff_smooth(fake, 64, 64, 3, fake, fake, 1 << 20, None) == 1
    assert L.ff_census(fake, 64, 64, 0, fake, None) == 1
    # kd: leaf range
    d = C.c_int()
    assert L.ff_kdtree_size(100, 1, C.byref(d), None) == 1
    assert L.ff_kdtree_size(1024 * 436, 8, C.byref(d), None) == 0 and d.value == 16


def test_kd_depth_matches_definition(L):
    d = C.c_int()
    for N, leaf in [(1, 2), (2, 2), (3, 2), (9, 8), (12288, 8), (446464, 8), (465750, 8),
                    (1000, 31)]:
        assert L.ff_kdtree_size(N, leaf, C.byref(d), None) == 0
        D = d.value
        assert -(-N // (1 << D)) <= leaf
        assert D == 0 or -(-N // (1 << (D - 1))) > leaf


def test_batch_argument_checks(L):
    p = ffapi.Params()
    sz = C.c_size_t()
    pairs = (ffapi.Pair * 2)()
    for i in range(2):
        pairs[i] = ffapi.Pair(0x1000, 0x1000, 128, 96, None, 0x1000, 0x1000, 0x1000, 0x1000,
                              0x1000, 0x1000)
    assert L.ff_batch_workspace_size(2, pairs, C.byref(p), C.byref(sz)) == 0
    one = C.c_size_t()
    L.ff_workspace_size(128, 96, C.byref(p), C.byref(one))
    assert sz.value > one.value
    assert L.ff_batch_workspace_size(0, pairs, C.byref(p), C.byref(sz)) == 1
    assert L.ff_batch_workspace_size(2, None, C.byref(p), C.byref(sz)) == 1
    pairs[1].W = 0
    assert L.ff_batch_workspace_size(2, pairs, C.byref(p), C.byref(sz)) == 2
    pairs[1].W = 128
    pairs[0].I1 = None
    assert L.ff_flow_fields_batch(2, pairs, C.byref(p), C.c_void_p(0x100000), 1 << 40, None) == 1
    g = C.c_void_p()
    assert L.ff_graph_create(2, pairs, C.byref(p), C.c_void_p(0x100000), 1 << 40, None,
                             C.byref(g)) == 1
    assert L.ff_graph_destroy(None) == 0


def test_exec_params_checks(L):
    e = ffapi.ExecParams()
    assert L.ff_get_exec_params(C.byref(e)) == 0 and 1 <= e.pass_warps <= 8
    bad = ffapi.ExecParams(pass_warps=9)
    assert L.ff_set_exec_params(C.byref(bad)) == 1
    for rs in (-1, 3, 256):  # not a power of two in 0..128
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, rs_min_n=rs))) == 1
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, wide_min_n=rs))) == 1
    for sp in (-1, 3, 256):
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, split8_min_n=sp))) == 1
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, split2_max_n=sp))) == 1
    for v in (-1, 2):
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, serial_flows=v))) == 1
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, kd_merge=v))) == 1
        assert L.ff_set_exec_params(C.byref(ffapi.ExecParams(pass_warps=2, persist_levels=v))) == 1
    assert L.ff_set_wait_test(-1, -1, 0) == 1 and L.ff_set_wait_test(0, -2, 0) == 1
    assert L.ff_set_wait_test(0, -1, -1) == 1
    assert L.ff_set_wait_test(0, -1, 0) == 0
    assert L.ff_set_exec_params(None) == 1
    ok = ffapi.ExecParams(pass_warps=e.pass_warps, rs_min_n=4, wide_min_n=2, split8_min_n=8)
    assert L.ff_set_exec_params(C.byref(ok)) == 0
    assert L.ff_set_exec_params(C.byref(e)) == 0  # restore


def test_static_filter_applies_the_workspace_filters_checks(L):
    """ff_consistency_filter_static refuses what ff_consistency_filter refuses (shape and
    parameter checks run first, on the host, before any CUDA call), then its own
    2^20-pixel limit."""
    fake = C.c_void_p(0x1000)
    ok = ffapi.Params()

    def call(W, H, p):
        return L.ff_consistency_filter_static(fake, fake, fake, W, H, C.byref(p), fake, fake,
                                              fake, fake, fake, None)

    assert call(20000, 1, ok) == 2          # W above 16384
    assert call(1, 20000, ok) == 2          # H above 16384
    assert call(0, 5, ok) == 2
    assert call(1025, 1024, ok) == 2        # 2^20 + 1 pixels
    for bad in [dict(tile=31), dict(k=5), dict(r=9), dict(leaf=1), dict(n_rs=4), dict(K=9),
                dict(eps=0), dict(e=10)]:
        assert call(64, 48, ffapi.Params(**bad)) == 1, bad
    assert L.ff_consistency_filter_static(None, fake, fake, 64, 48, C.byref(ok), fake, fake, fake,
                                          fake, fake, None) == 1


def test_sift_argument_checks(L):
    """The SIFT flow entry points refuse bad channel counts, sizes and pointers on
    the host, before any CUDA call."""
    fake = C.c_void_p(0x1000)
    sz = C.c_size_t()
    assert L.ff_sift_pca_workspace_size(None) == 1
    assert L.ff_sift_pca_workspace_size(C.byref(sz)) == 0 and sz.value >= 128 * 128 * 8
    for S in (0, 2, 4, 33):
        assert L.ff_sift_pca(fake, fake, 10, S, fake, fake, None, C.c_void_p(0x100000), 1 << 30,
                             None) == 1, S
        assert L.ff_sift_colors(C.c_void_p(0x1000), 64, 48, fake, fake, S, fake, None) == 1, S
        assert L.ff_sift_level_workspace_size(64, 48, 2, S, C.byref(sz)) == 1, S
    assert L.ff_sift_pca(fake, fake, 0, 12, fake, fake, None, C.c_void_p(0x100000), 1 << 30,
                         None) == 1
    assert L.ff_sift_pca(fake, fake, 10, 12, fake, fake, None, C.c_void_p(0x100001), 1 << 30,
                         None) == 3
    assert L.ff_sift_descriptors(fake, 64, 48, C.c_void_p(0x1008), None) == 1  # desc not 16-aligned
    assert L.ff_sift_descriptors(fake, 0, 48, fake, None) == 2
    assert L.ff_sift_moments(fake, -1, fake, fake, None) == 1
    assert L.ff_sift_level_workspace_size(64, 48, 3, 12, C.byref(sz)) == 1
    assert L.ff_sift_level_workspace_size(64, 48, 4, 12, C.byref(sz)) == 0
    p = ffapi.Params(k=3, r=3, r2=2)
    a, b = C.c_size_t(), C.c_size_t()
    assert L.ff_sift_workspace_size(1242, 375, C.byref(p), 12, 18, C.byref(a)) == 0
    assert L.ff_sift_workspace_size(1242, 375, C.byref(p), 3, 3, C.byref(b)) == 0
    assert a.value > b.value > 128 * 1242 * 375 * 2  # two frames of SIFT vectors at least
    assert L.ff_sift_workspace_size(1242, 375, C.byref(p), 12, 19, C.byref(a)) == 1
    ps = ffapi.Params(k=3, r=3, r2=2, subpel=2)
    args = (fake, fake, 12, fake, fake, 18, fake, fake, fake, fake, fake, fake)
    assert L.ff_sift_flow_fields(fake, fake, 64, 48, C.byref(ps), *args, C.c_void_p(0x100000),
                                 1 << 40, None) == 1
    assert L.ff_sift_flow_fields(None, fake, 64, 48, C.byref(p), *args, C.c_void_p(0x100000),
                                 1 << 40, None) == 1
    assert L.ff_sift_flow_fields(fake, fake, 64, 48, C.byref(p), *args, C.c_void_p(0x100001),
                                 1 << 40, None) == 3
    assert L.ff_sift_search_level(fake, fake, 12, 64, 48, 1, 3, None, C.byref(ps), 0, fake, fake,
                                  C.c_void_p(0x100000), 1 << 30, None) == 1
    assert L.ff_sift_kdtree_init(fake, fake, fake, 8, fake, fake, fake, 12, 64, 48, 1, 9, fake,
                                 fake, C.c_void_p(0x100000), 1 << 30, None) == 1
