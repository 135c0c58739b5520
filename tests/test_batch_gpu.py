"""Batched form (mixed sizes, one launch set per level), CUDA-graph replay and the
autotuner's execution parameters: every result equals the single-pair path and
the CPU oracle bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1508_05151_gb300 import ffapi, synth, tune

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SIZES = [(128, 96), (97, 71), (160, 120), (64, 48)]


def _frames(seed0=0):
    pairs = [synth.pair_shift(seed0 + i, W=W, H=H, max_shift=(W // 6, H // 6), square=min(24, W, H),
                              square_move=8) for i, (W, H) in enumerate(SIZES)]
    frames = [(torch.from_numpy(p["I1"]).cuda(), torch.from_numpy(p["I2"]).cuda()) for p in pairs]
    return pairs, frames


def _same(a, b):
    torch.cuda.synchronize()
    for k in ("flows", "valid", "err_sum", "mask", "n_sparse"):
        assert torch.equal(a[k], b[k]), k
    n = int(a["n_sparse"].item())
    assert torch.equal(a["sparse"][:n], b["sparse"][:n])


def test_batch_equals_single_pairs_and_oracle():
    pairs, frames = _frames(10)
    batch = ffapi.FlowFieldsBatch(SIZES)
    outs = batch.run(frames)
    torch.cuda.synchronize()
    for i, ((W, H), (a, b)) in enumerate(zip(SIZES, frames)):
        single = ffapi.FlowFields(W, H).run(a, b)
        _same(outs[i], single)
    for i in (0, 2):  # oracle on two of the pairs
        ref = O.flow_fields(pairs[i]["I1"], pairs[i]["I2"])
        assert np.array_equal(outs[i]["flows"].cpu().numpy().astype(np.int32), ref["flows"])
        assert np.array_equal(outs[i]["valid"].cpu().numpy(), ref["valid"])


def test_graph_replay_equals_direct_run():
    _, frames1 = _frames(20)
    _, frames2 = _frames(30)
    direct = ffapi.FlowFieldsBatch(SIZES)
    graphed = ffapi.FlowFieldsBatch(SIZES, graph=True)
    for frames in (frames1, frames2, frames1):  # capture on first run, then replay
        d = [{k: v.clone() for k, v in o.items()} for o in direct.run(frames)]
        g = graphed.run(frames)
        for a, b in zip(d, g):
            _same(a, b)
    assert graphed.graph_kernels() > 50


def test_execution_parameters_do_not_change_results():
    _, frames = _frames(40)
    batch = ffapi.FlowFieldsBatch(SIZES)
    ref = [{k: v.clone() for k, v in o.items()} for o in batch.run(frames)]
    before = ffapi.get_exec_params()
    try:
        # tiles per CTA, and the random search inside the pass kernel or as its
        # own kernel from some level on
        for pw, rs, wide, s8 in ((1, 0, 0, 0), (2, 1, 0, 0), (8, 2, 0, 0), (4, 8, 1, 0),
                                 (4, 64, 2, 2), (8, 0, 4, 0), (4, 0, 1, 1), (4, 0, 1, 4)):
            ffapi.set_exec_params(pass_warps=pw, rs_min_n=rs, wide_min_n=wide, split8_min_n=s8)
            got = batch.run(frames)
            for a, b in zip(ref, got):
                _same(a, b)
        # 2 threads per candidate at the finest levels (with 8 above, and with the
        # persistent launch, which runs them as 4)
        for s2, s8, persist in ((1, 0, 0), (2, 4, 0), (128, 0, 0), (2, 4, 1)):
            ffapi.set_exec_params(split2_max_n=s2, split8_min_n=s8, persist_levels=persist)
            got = batch.run(frames)
            for a, b in zip(ref, got):
                _same(a, b)
        # stream layouts: flows serialised on one stream, kd trees of all flows in
        # one launch chain, both
        ffapi.set_exec_params(**before)
        for serial, merge in ((1, 0), (0, 1), (1, 1)):
            ffapi.set_exec_params(serial_flows=serial, kd_merge=merge)
            got = batch.run(frames)
            for a, b in zip(ref, got):
                _same(a, b)
        # one persistent launch per level (4 and 8 threads per candidate), alone and
        # with the other stream layouts
        for s8, serial, merge in ((0, 0, 0), (1, 0, 0), (2, 0, 1), (4, 1, 0)):
            ffapi.set_exec_params(persist_levels=1, split8_min_n=s8, serial_flows=serial,
                                  kd_merge=merge)
            got = batch.run(frames)
            for a, b in zip(ref, got):
                _same(a, b)
    finally:
        ffapi.set_exec_params(**before)


def test_autotuner_picks_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "_CACHE", str(tmp_path / "t.json"))
    before = ffapi.get_exec_params()
    try:
        r = tune.tune([(128, 96), (97, 71)], reps=1)
        assert not r["cached"]
        assert r["choice"]["pass_warps"] in tune.CANDIDATES["pass_warps"]
        assert r["choice"]["rs_min_n"] in tune.CANDIDATES["rs_min_n"]
        assert r["choice"]["wide_min_n"] in tune.CANDIDATES["wide_min_n"]
        assert r["choice"]["split8_min_n"] in tune.CANDIDATES["split8_min_n"]
        assert r["choice"]["serial_flows"] in tune.CANDIDATES["serial_flows"]
        assert r["choice"]["kd_merge"] in tune.CANDIDATES["kd_merge"]
        assert r["choice"]["persist_levels"] in tune.CANDIDATES["persist_levels"]
        assert r["choice"]["split2_max_n"] in tune.CANDIDATES["split2_max_n"]
        assert ffapi.get_exec_params() == r["choice"]
        r2 = tune.tune([(128, 96), (97, 71)], reps=1)
        assert r2["cached"] and r2["choice"] == r["choice"]
    finally:
        ffapi.set_exec_params(**before)


def test_persistent_levels_graph_and_radius_mix():
    """The persistent level kernel inside a captured graph equals the direct
    per-pass form, for the paper's radii (8, 6: one fused launch per level) and
    for a radius pair without a fused kernel (5, 3: one launch per radius)."""
    _, frames = _frames(50)
    before = ffapi.get_exec_params()
    try:
        for params in (None, dict(r=5, r2=3)):
            ffapi.set_exec_params(**before)
            ref = [{k: v.clone() for k, v in o.items()}
                   for o in ffapi.FlowFieldsBatch(SIZES, params).run(frames)]
            ffapi.set_exec_params(persist_levels=1)
            g = ffapi.FlowFieldsBatch(SIZES, params, graph=True)
            for _ in range(2):  # capture, then replay
                got = g.run(frames)
                for a, b in zip(ref, got):
                    _same(a, b)
    finally:
        ffapi.set_exec_params(**before)


def test_persistent_barrier_wait_runs_out_and_reports():
    """Bounded-wait path of the persistent level kernel: the test hook keeps one
    block away from the first grid barrier and sets a tiny wait limit, so every
    other block's wait runs out. The launch must return, the device status word
    must say timeout (code 3), and the GPU must stay usable: the next run without
    the hook is correct again."""
    p = synth.pair_shift(60, W=128, H=96)
    I1, I2 = torch.from_numpy(p["I1"]).cuda(), torch.from_numpy(p["I2"]).cuda()
    ff = ffapi.FlowFields(128, 96)
    ref = {k: v.clone() for k, v in ff.run(I1, I2).items()}
    torch.cuda.synchronize()
    before = ffapi.get_exec_params()
    L = ffapi.lib()
    try:
        ffapi.set_exec_params(persist_levels=1)
        assert L.ff_set_wait_test(200000, 0, 0) == 0  # ~0.1 ms at 2 GHz
        ff.run(I1, I2)
        code, x, y = ff.device_status()
        assert code == 3, (code, x, y)
        assert L.ff_set_wait_test(0, -1, 0) == 0
        got = ff.run(I1, I2)
        code, _, _ = ff.device_status()
        assert code == 0
        _same(ref, got)
    finally:
        L.ff_set_wait_test(0, -1, 0)
        ffapi.set_exec_params(**before)
