"""Proposal net on the GPU against the float64 oracle of oracle/net.py.

Tolerances. Both sides round the convolution operands to BF16 at the same points;
they differ only in the accumulation (FP32 in the tensor cores, float64 in the
oracle) and, through it, in the rare activation whose BF16 rounding flips (one
BF16 ulp, 2^-8 relative). Over <= 576-term dot products the FP32 error is about
1e-6 relative, so flips touch a few activations in 10^5 and the outputs agree to
about 1e-4 in relative L2 norm; the tests allow 2e-3 (relative L2) and 2e-2 of
the largest magnitude per element. Weight gradients are summed with FP32
atomics over all pixels: the same bounds apply per layer.
Integer steps (net input, proposals) are exact.
"""
import numpy as np
import pytest
import torch

from oracle import net as N
from paper_1508_05151_gb300 import ffapi, synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DESCS = [
    dict(cin=6, c1=32, c2=64, c3=64, k=4, dil=(1, 2, 4, 8)),
    dict(cin=6, c1=20, c2=40, c3=24, k=3, dil=(1, 3, 2, 1)),  # ragged channel counts
]


def _desc(d):
    return ffapi.net_desc(d["c1"], d["c2"], d["c3"], d["k"], d["dil"])


def _params(d, seed):
    sh, n = N.shapes(d)
    rng = np.random.default_rng(seed)
    p = np.zeros(n, np.float32)
    for s in sh:
        p[s["woff"]:s["boff"]] = rng.normal(scale=np.sqrt(2.0 / (9 * s["cin"])),
                                            size=s["boff"] - s["woff"])
        p[s["boff"]:s["boff"] + s["cout"]] = rng.normal(scale=0.05, size=s["cout"])
    return p


def _frames(B, W, H, seed):
    I1, I2 = [], []
    for i in range(B):
        pr = synth.pair_shift(seed + i, W=W, H=H, max_shift=(24, 16), square=min(48, W, H))
        I1.append(pr["I1"])
        I2.append(pr["I2"])
    return np.stack(I1), np.stack(I2)


def _close(got, ref, rel_l2=2e-3, rel_max=2e-2):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(), 1e-30)
    assert np.linalg.norm(got - ref) <= rel_l2 * max(np.linalg.norm(ref), 1e-30), \
        (np.linalg.norm(got - ref), np.linalg.norm(ref))
    assert np.abs(got - ref).max() <= rel_max * scale, (np.abs(got - ref).max(), scale)


def test_net_input_exact():
    I1, I2 = _frames(3, 203, 117, 1)  # partial blocks on both axes
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    torch.cuda.synchronize()
    for b in range(3):
        ref = N.net_input(I1[b], I2[b]).astype(np.float32)
        assert np.array_equal(x[b].cpu().numpy(), ref)


@pytest.mark.parametrize("di", range(len(DESCS)))
def test_forward_backward_match_oracle(di):
    d = DESCS[di]
    desc = _desc(d)
    B, W, H = 2, 300, 205  # Gx 38, Gy 26: 1976 pixels = 30 full 64-row tiles + a ragged one
    I1, I2 = _frames(B, W, H, 10 + di)
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    Gy, Gx = x.shape[2:]
    p = _params(d, 20 + di)
    params = torch.from_numpy(p).cuda()
    run = ffapi.NetRunner(desc, B, Gx, Gy)
    out = run.forward(params, x).cpu().numpy()
    ref, cache = N.forward(p.astype(np.float64), x.cpu().numpy().astype(np.float64), d)
    _close(out, ref)

    rng = np.random.default_rng(30 + di)
    dout = rng.normal(size=out.shape).astype(np.float32)
    grads = torch.empty_like(params)
    run.backward(params, grads, torch.from_numpy(dout).cuda())
    g = grads.cpu().numpy()
    gref = N.backward(p.astype(np.float64), dout.astype(np.float64), cache, d)
    sh, _ = N.shapes(d)
    for s in sh:
        _close(g[s["woff"]:s["boff"]], gref[s["woff"]:s["boff"]])
        _close(g[s["boff"]:s["boff"] + s["cout"]], gref[s["boff"]:s["boff"] + s["cout"]])


def test_loss_and_gradient_of_loss():
    d = DESCS[0]
    K, B, Gy, Gx = d["k"], 3, 17, 29
    rng = np.random.default_rng(40)
    out = rng.normal(scale=3.0, size=(B, 2 * K, Gy, Gx)).astype(np.float32)
    label = rng.integers(-40, 41, size=(B, Gy, Gx, 2)).astype(np.int16)
    valid = (rng.random((B, Gy, Gx)) < 0.6).astype(np.uint8)
    run = ffapi.NetRunner(_desc(d), B, Gx, Gy)
    run.out.copy_(torch.from_numpy(out))
    loss, dout = run.loss_grad(torch.from_numpy(label).cuda(), torch.from_numpy(valid).cuda(),
                               8.0, 0.05)
    lref, dref = N.wta_loss(out.astype(np.float64), label, valid, K, 8.0, 0.05)
    assert abs(float(loss.item()) - lref) <= 1e-5 * abs(lref)
    assert int(run.count.item()) == int(valid.sum())
    assert np.allclose(dout.cpu().numpy(), dref, rtol=1e-6, atol=1e-9)


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(50)
    n = 10007
    p, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = (rng.normal(size=n) * 0.1).astype(np.float32), (rng.random(n) * 0.1).astype(np.float32)
    tp, tg, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    ffapi.ff_net_adam(tp, tg, tm, tv, 7, 1e-3)
    # the kernel receives binary32 hyperparameters (0.999f is 0.99900001...): the
    # oracle takes the same values so that only the arithmetic precision differs
    f32 = lambda a: float(np.float32(a))
    pr, mr, vr = N.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                        v.astype(np.float64), 7, f32(1e-3), f32(0.9), f32(0.999), f32(1e-8))
    assert np.allclose(tp.cpu().numpy(), pr, rtol=0, atol=1e-6)
    assert np.allclose(tm.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)
    assert np.allclose(tv.cpu().numpy(), vr, rtol=1e-5, atol=1e-9)


def test_proposals_are_rounded_outputs():
    d = DESCS[0]
    K, B, Gy, Gx = d["k"], 2, 9, 13
    rng = np.random.default_rng(60)
    out = (rng.normal(scale=10.0, size=(B, 2 * K, Gy, Gx))).astype(np.float32)
    out[0, 0, 0, :4] = [0.0625, 0.1875, -0.3125, 2500.0]  # exact halves and a clamp
    run = ffapi.NetRunner(_desc(d), B, Gx, Gy)
    prop = run.proposals(8.0, torch.from_numpy(out).cuda()).cpu().numpy()
    ref = np.clip(np.rint(out * np.float32(8.0)), -16000, 16000)   # ties to even, as rintf
    ref = ref.reshape(B, K, 2, Gy, Gx).transpose(0, 3, 4, 1, 2)
    assert np.array_equal(prop, ref.astype(np.int16))


def test_training_reduces_the_loss():
    d = DESCS[0]
    desc = _desc(d)
    B, W, H = 8, 256, 128
    I1, I2 = _frames(B, W, H, 70)
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    Gy, Gx = x.shape[2:]
    lab = np.zeros((B, Gy, Gx, 2), np.int16)
    for b in range(B):
        pr = synth.pair_shift(70 + b, W=W, H=H, max_shift=(24, 16), square=min(48, W, H))
        lab[b] = pr["flow"][::8, ::8]
    label = torch.from_numpy(lab).cuda()
    valid = torch.ones((B, Gy, Gx), dtype=torch.uint8, device="cuda")
    params = torch.from_numpy(_params(d, 71)).cuda()
    grads, m, v = (torch.zeros_like(params) for _ in range(3))
    run = ffapi.NetRunner(desc, B, Gx, Gy)
    losses = []
    for step in range(1, 201):
        run.forward(params, x)
        loss, _ = run.loss_grad(label, valid, 8.0, 0.05)
        losses.append(float(loss.item()))
        run.backward(params, grads)
        ffapi.ff_net_adam(params, grads, m, v, step, 2e-3)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10]), losses[::20]


def test_learned_proposals_lower_the_coarse_data_cost():
    """Gain test: a net trained briefly on plain-search labels proposes candidates
    that win the exact data term at the coarsest level on held-out pairs. The cost
    with proposals can never be higher (strict-less acceptance); measured on these
    pairs they win at ~24% of grid points and lower the summed cost by ~13%."""
    from paper_1508_05151_gb300 import train

    def pairs(seed0, n, W=256, H=128):
        ps = [synth.pair_shift(seed0 + i, W=W, H=H, max_shift=(24, 16), square=min(48, W, H))
              for i in range(n)]
        return tuple(np.stack([p[k] for p in ps]) for k in ("I1", "I2", "flow", "occ"))

    I1, I2, _, _ = pairs(5000, 192)
    label, valid = train.plain_labels(I1, I2)
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    net = train.ProposalNet(seed=3)
    losses = net.train(x, label, valid, epochs=15, batch=32)
    assert losses[-5:].mean() < 0.6 * losses[:5].mean()
    E1, E2, _, _ = pairs(9000, 32)
    d = train.coarse_cost_delta(net, E1, E2)
    assert d["never_worse"]
    assert d["frac_won"] > 0.10, d
    assert d["cost_reduction"] > 0.05, d


def test_net_bounded_waits_run_out_and_report():
    """Bounded-wait path of the tensor-core kernels: with the test hook every
    kernel first waits on an mbarrier that nothing completes; the wait must run out,
    the forward and backward calls must return with device status 3 (timeout), and
    the next calls without the hook must give the same results as before."""
    d = DESCS[0]
    desc = _desc(d)
    B, W, H = 2, 160, 120
    I1, I2 = _frames(B, W, H, 70)
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    Gy, Gx = x.shape[2:]
    params = torch.from_numpy(_params(d, 71)).cuda()
    run = ffapi.NetRunner(desc, B, Gx, Gy)
    ref = run.forward(params, x).clone()
    assert run.device_status()[0] == 0
    dout = torch.ones_like(ref)
    gref = run.backward(params, torch.empty_like(params), dout).clone()
    assert run.device_status()[0] == 0
    L = ffapi.lib()
    try:
        assert L.ff_set_wait_test(0, -1, 64) == 0
        run.forward(params, x)
        assert run.device_status()[0] == 3
        run.backward(params, torch.empty_like(params), dout)
        assert run.device_status()[0] == 3
    finally:
        assert L.ff_set_wait_test(0, -1, 0) == 0
    out = run.forward(params, x)
    assert run.device_status()[0] == 0
    assert torch.equal(out, ref)
    g = run.backward(params, torch.empty_like(params), dout)
    assert run.device_status()[0] == 0
    _close(g.cpu().numpy(), gref.cpu().numpy())
