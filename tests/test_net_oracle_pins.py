"""Pins of the proposal-net oracle: BF16 rounding from the binary32 layout, the
convolution against a brute-force loop, backward passes against central finite
differences, the WTA loss on hand cases, and the first Adam step in closed form."""
import numpy as np

from oracle import net as N

DESC = dict(cin=6, c1=5, c2=4, c3=3, k=2, dil=(1, 2, 1, 3))


def test_bf16_round_to_nearest_even():
    e = 2.0 ** -7  # bf16 spacing at 1.0
    vals = np.array([1.0, 1 + e / 2, 1 + 1.5 * e, 1 + e / 2 + 2 ** -20, -1 - e / 2, 3.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 * e, 1 + e, -1.0, 3.0, 0.0])
    assert np.array_equal(N.bf16(vals), want)
    # every bf16 value is exactly representable: rounding is idempotent
    r = N.bf16(np.random.default_rng(0).normal(size=1000))
    assert np.array_equal(N.bf16(r), r)
    # relative error bound: the unit roundoff 2^-8 (half the spacing 2^-7 at 1.0)
    x = np.random.default_rng(1).uniform(-10, 10, size=10000)
    assert np.max(np.abs(N.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_conv_matches_brute_force():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(2, 3, 5, 7))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    for d in (1, 2, 3):
        out = N.conv(a, W, b, d)
        ref = np.zeros_like(out)
        for bb in range(2):
            for n in range(4):
                for y in range(5):
                    for x in range(7):
                        s = b[n]
                        for c in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    yy, xx = y + (ky - 1) * d, x + (kx - 1) * d
                                    if 0 <= yy < 5 and 0 <= xx < 7:
                                        s += W[n, c, ky, kx] * a[bb, c, yy, xx]
                        ref[bb, n, y, x] = s
        assert np.allclose(out, ref)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    _, n = N.shapes(DESC)
    p = rng.normal(scale=0.4, size=n)
    x = rng.normal(size=(2, 6, 5, 6))
    R = rng.normal(size=(2, 4, 5, 6))
    out, cache = N.forward(p, x, DESC, rounding=False)
    g = N.backward(p, R, cache, DESC, rounding=False)
    h = 1e-6
    for i in rng.choice(n, size=40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fp = (N.forward(pp, x, DESC, rounding=False)[0] * R).sum()
        fm = (N.forward(pm, x, DESC, rounding=False)[0] * R).sum()
        assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-5 * (1 + abs(g[i]))


def test_wta_loss_hand_case_and_gradient():
    # K=2, one point, label (4, -2) px, scale 2 -> (2, -1); candidates (2.5, -1) and (0, 0)
    out = np.array([2.5, -1.0, 0.0, 0.0]).reshape(1, 4, 1, 1)
    label = np.array([[[[4, -2]]]])
    valid = np.ones((1, 1, 1), np.uint8)
    loss, d = N.wta_loss(out, label, valid, 2, 2.0, 0.1)
    # errors 0.5 and 3.0; best is k=0: 0.9*0.5 + 0.1*3 = 0.75
    assert abs(loss - 0.75) < 1e-12
    assert np.allclose(d.ravel(), [0.9, 0.0, -0.1, 0.1])
    # away from ties and kinks the gradient is the finite difference
    rng = np.random.default_rng(4)
    out = rng.normal(size=(2, 6, 3, 4))
    label = rng.integers(-5, 6, size=(2, 3, 4, 2))
    valid = rng.random((2, 3, 4)) < 0.7
    _, d = N.wta_loss(out, label, valid, 3, 4.0, 0.2)
    h = 1e-7
    for i in range(out.size):
        o1, o2 = out.copy().ravel(), out.copy().ravel()
        o1[i] += h
        o2[i] -= h
        l1 = N.wta_loss(o1.reshape(out.shape), label, valid, 3, 4.0, 0.2)[0]
        l2 = N.wta_loss(o2.reshape(out.shape), label, valid, 3, 4.0, 0.2)[0]
        assert abs((l1 - l2) / (2 * h) - d.ravel()[i]) < 1e-5


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p, g = rng.normal(size=50), rng.normal(size=50)
    p1, m, v = N.adam(p, g, np.zeros(50), np.zeros(50), 1, 0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(g))
    # epsilon is added to sqrt(v_hat) (Kingma & Ba): with |g| = eps the first step is
    # g / (|g| + eps) = 1/2 of the learning rate
    e = 1e-8
    p1, _, _ = N.adam(np.zeros(2), np.array([e, -e]), np.zeros(2), np.zeros(2), 1, 0.01, eps=e)
    assert np.allclose(p1, [-0.005, 0.005], rtol=1e-9, atol=0)


def test_net_input_block_means():
    I1 = np.zeros((10, 9, 3), np.uint8)
    I1[:8, :8, 0] = 255
    I2 = np.full((10, 9, 3), 51, np.uint8)
    x = N.net_input(I1, I2)
    assert x.shape == (6, 2, 2)
    assert x[0, 0, 0] == np.float32(0.5) and x[0, 1, 1] == np.float32(-0.5)
    assert np.allclose(x[3:], np.float32(51) / np.float32(255) - np.float32(0.5))
