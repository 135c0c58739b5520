"""Seeded synthetic image pairs with exact ground-truth flow.

The paper evaluates on MPI-Sintel, Middlebury and KITTI (Sec. 4). None of them is
available here, so these generators stand in with the same shapes and the same kind
of content: textured layers, large displacements, occlusions, brightness changes and
blur. Every pair is a pure function of its seed.

This module holds only image synthesis. It contains none of the Flow Fields
arithmetic, so that both the CUDA path and the CPU oracle can be fed from it.

Ground truth convention: ``flow[y, x] = (u, v)`` means that the frame-1 pixel (x, y)
shows up at (x + u, y + v) in frame 2. ``occ[y, x]`` is True where that point is not
visible in frame 2 (covered by another layer or outside the frame).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "value_noise",
    "pair_shift",
    "pair_layers",
    "pair_kitti",
    "workload_pair",
    "WORKLOADS",
    "mixed_batch",
    "BATCH_SIZES",
]

# Image sizes of the mixed-size batch (16 pairs of each).
BATCH_SIZES = ((640, 480), (584, 388), (1024, 436), (1242, 375))


def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise(rng, h, w, c=3, lattices=(32, 16, 8, 4),
                amps=(0.5, 0.25, 0.125, 0.0625)):
    """Multi-octave value noise in [0, 1], shape (h, w, c), float64.

    Each octave places uniform random values on a square lattice of the given
    spacing and interpolates them with smoothstep weights.
    """
    out = np.zeros((h, w, c))
    ys = np.arange(h, dtype=np.float64)
    xs = np.arange(w, dtype=np.float64)
    for s, a in zip(lattices, amps):
        g = rng.random((h // s + 2, w // s + 2, c))
        fy, fx = ys / s, xs / s
        iy, ix = np.floor(fy).astype(np.int64), np.floor(fx).astype(np.int64)
        ty, tx = _smooth(fy - iy)[:, None, None], _smooth(fx - ix)[None, :, None]
        # separable: interpolate every lattice row along x, then rows along y
        gx = g[:, ix] * (1 - tx) + g[:, ix + 1] * tx
        out += a * (gx[iy] * (1 - ty) + gx[iy + 1] * ty)
    lo = out.min(axis=(0, 1), keepdims=True)
    hi = out.max(axis=(0, 1), keepdims=True)
    return (out - lo) / np.maximum(hi - lo, 1e-12)


def _to_u8(x):
    return np.clip(np.rint(x * 255.0), 0, 255).astype(np.uint8)


def pair_shift(seed, W=128, H=96, max_shift=(16, 16), square=32, square_move=24,
               margin=None):
    """Textured background moved by one integer shift, plus an occluding square.

    frame1 is a window of a 4-octave value-noise canvas. frame2 is the same canvas
    shifted by an integer (dx, dy), each uniform in [-max_shift, max_shift]. A
    square with its own texture moves independently by an integer vector with
    max-norm <= square_move and is drawn on top in both frames.

    Returns dict(I1, I2 uint8 [H, W, 3], flow int32 [H, W, 2], occ bool [H, W],
    shift, square_pos, square_move).
    """
    rng = np.random.default_rng(np.uint64(seed))
    sx_max, sy_max = (max_shift, max_shift) if np.isscalar(max_shift) else max_shift
    M = margin if margin is not None else max(64, sx_max, sy_max)
    canvas = _to_u8(value_noise(rng, H + 2 * M, W + 2 * M))
    dx = int(rng.integers(-sx_max, sx_max + 1))
    dy = int(rng.integers(-sy_max, sy_max + 1))
    I1 = canvas[M:M + H, M:M + W].copy()
    I2 = canvas[M - dy:M - dy + H, M - dx:M - dx + W].copy()
    flow = np.empty((H, W, 2), np.int32)
    flow[..., 0], flow[..., 1] = dx, dy

    S = min(square, W, H)
    tex = _to_u8(value_noise(rng, S, S, lattices=(8, 4, 2), amps=(0.5, 0.3, 0.2)))
    px = int(rng.integers(0, W - S + 1))
    py = int(rng.integers(0, H - S + 1))
    mx = int(rng.integers(-square_move, square_move + 1))
    my = int(rng.integers(-square_move, square_move + 1))
    I1[py:py + S, px:px + S] = tex
    flow[py:py + S, px:px + S] = (mx, my)
    # draw the moved square in frame 2, clipped to the frame
    qx, qy = px + mx, py + my
    x0, x1 = max(qx, 0), min(qx + S, W)
    y0, y1 = max(qy, 0), min(qy + S, H)
    if x0 < x1 and y0 < y1:
        I2[y0:y1, x0:x1] = tex[y0 - qy:y1 - qy, x0 - qx:x1 - qx]

    ys, xs = np.mgrid[0:H, 0:W]
    tx, ty = xs + flow[..., 0], ys + flow[..., 1]
    occ = (tx < 0) | (tx >= W) | (ty < 0) | (ty >= H)
    in_sq1 = (xs >= px) & (xs < px + S) & (ys >= py) & (ys < py + S)
    covered = (tx >= qx) & (tx < qx + S) & (ty >= qy) & (ty < qy + S)
    occ |= (~in_sq1) & covered
    return dict(I1=I1, I2=I2, flow=flow, occ=occ, shift=(dx, dy),
                square_pos=(px, py), square_move=(mx, my))


def _bilinear(img, x, y):
    """Sample img (h, w, c) float at real positions with edge clamping."""
    h, w = img.shape[:2]
    x = np.clip(x, 0, w - 1.000001)
    y = np.clip(y, 0, h - 1.000001)
    x0, y0 = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64)
    tx, ty = (x - x0)[..., None], (y - y0)[..., None]
    a = img[y0, x0] * (1 - tx) + img[y0, x0 + 1] * tx
    b = img[y0 + 1, x0] * (1 - tx) + img[y0 + 1, x0 + 1] * tx
    return a * (1 - ty) + b * ty


def _star_mask(x, y, cx, cy, radii):
    """Inside test for a star-shaped polygon with vertex radii at equal angles."""
    ang = np.arctan2(y - cy, x - cx) % (2 * np.pi)
    k = len(radii)
    f = ang / (2 * np.pi) * k
    i0 = np.floor(f).astype(np.int64) % k
    t = f - np.floor(f)
    rr = radii[i0] * (1 - t) + radii[(i0 + 1) % k] * t
    return np.hypot(x - cx, y - cy) < rr


def _ellipse_mask(x, y, cx, cy, a, b, th):
    c, s = np.cos(th), np.sin(th)
    u = (x - cx) * c + (y - cy) * s
    v = -(x - cx) * s + (y - cy) * c
    return (u / a) ** 2 + (v / b) ** 2 < 1.0


def _random_shapes(rng, W, H, count, rmin, rmax):
    shapes = []
    for _ in range(count):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        if rng.random() < 0.5:
            a, b = rng.uniform(rmin, rmax), rng.uniform(rmin, rmax)
            shapes.append(("e", cx, cy, a, b, rng.uniform(0, np.pi)))
        else:
            k = int(rng.integers(5, 9))
            shapes.append(("p", cx, cy, rng.uniform(rmin, rmax, size=k)))
    return shapes


def _shapes_mask(shapes, x, y):
    m = np.zeros(np.broadcast(x, y).shape, bool)
    for sh in shapes:
        if sh[0] == "e":
            m |= _ellipse_mask(x, y, *sh[1:])
        else:
            m |= _star_mask(x, y, sh[1], sh[2], sh[3])
    return m


def _box3(img):
    """3x3 box blur with replicated borders, (sum + 4) // 9 per channel."""
    p = np.pad(img.astype(np.int32), ((1, 1), (1, 1), (0, 0)), mode="edge")
    s = sum(p[dy:dy + img.shape[0], dx:dx + img.shape[1]]
            for dy in range(3) for dx in range(3))
    return ((s + 4) // 9).astype(np.uint8)


def pair_layers(seed, W=1024, H=436, max_disp=200.0):
    """Sintel-shaped pair: 3 textured layers with affine motion and occlusions.

    Layer 0 is a full background. Layers 1 and 2 are unions of random ellipses and
    star polygons. Each layer has its own affine motion (scale, rotation about its
    centre, translation) whose displacement over the frame is capped at max_disp.
    Each frame gets a brightness gain from U[0.9, 1.1]; frame 2 is box-blurred with
    probability 0.3.

    Returns dict(I1, I2 uint8 [H, W, 3], flow float32 [H, W, 2], occ bool [H, W]).
    """
    rng = np.random.default_rng(np.uint64(seed))
    M = 256
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    layers = []
    for li in range(3):
        tex = value_noise(rng, H + 2 * M, W + 2 * M,
                          lattices=(64, 24, 8, 3), amps=(0.45, 0.3, 0.15, 0.1))
        tint = rng.uniform(0.3, 1.0, size=3)
        tex = tex * tint
        # painted shapes give sharp edges inside the texture
        for sh in _random_shapes(rng, W + 2 * M, H + 2 * M, 12 if li == 0 else 4, 10, 60):
            ext = 61 if sh[0] == "e" else int(np.ceil(max(sh[3]))) + 1
            x0, y0 = max(int(sh[1]) - ext, 0), max(int(sh[2]) - ext, 0)
            x1, y1 = min(int(sh[1]) + ext, W + 2 * M), min(int(sh[2]) + ext, H + 2 * M)
            ty, tx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
            m = _shapes_mask([sh], tx, ty)
            sub = tex[y0:y1, x0:x1]
            sub[m] = sub[m] * 0.4 + 0.6 * rng.uniform(0, 1, size=3)
        if li == 0:
            shapes = None
            cx, cy = W / 2, H / 2
            tmax = 40.0
        else:
            shapes = _random_shapes(rng, W, H, int(rng.integers(1, 4)), 40, 140)
            cx = float(np.mean([s[1] for s in shapes]))
            cy = float(np.mean([s[2] for s in shapes]))
            tmax = 160.0
        sc = rng.uniform(0.93, 1.07)
        th = np.deg2rad(rng.uniform(-4, 4))
        t = rng.uniform(-tmax, tmax, size=2)
        A = sc * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        # displacement field d(x) = (A - I)(x - c) + t, capped over the frame
        corners = np.array([[0, 0], [W - 1, 0], [0, H - 1], [W - 1, H - 1]], np.float64)
        d = (corners - [cx, cy]) @ (A - np.eye(2)).T + t
        alpha = min(1.0, max_disp / max(np.hypot(d[:, 0], d[:, 1]).max(), 1e-9))
        B = np.eye(2) + alpha * (A - np.eye(2))
        t = alpha * t
        layers.append(dict(tex=tex, shapes=shapes, c=np.array([cx, cy]), B=B, t=t))

    def fwd(L, x, y):
        p = np.stack([x - L["c"][0], y - L["c"][1]], -1) @ L["B"].T
        return p[..., 0] + L["c"][0] + L["t"][0], p[..., 1] + L["c"][1] + L["t"][1]

    def inv(L, x, y):
        Bi = np.linalg.inv(L["B"])
        p = np.stack([x - L["c"][0] - L["t"][0], y - L["c"][1] - L["t"][1]], -1) @ Bi.T
        return p[..., 0] + L["c"][0], p[..., 1] + L["c"][1]

    def render(frame):
        img = np.zeros((H, W, 3))
        top = np.zeros((H, W), np.int32)
        for li, L in enumerate(layers):
            if frame == 0:
                lx, ly = xs, ys
            else:
                lx, ly = inv(L, xs, ys)
            inside = np.ones((H, W), bool) if L["shapes"] is None else _shapes_mask(L["shapes"], lx, ly)
            col = _bilinear(L["tex"], lx + M, ly + M)
            img[inside] = col[inside]
            top[inside] = li
        return img, top

    f1, top1 = render(0)
    f2, top2 = render(1)
    g1, g2 = rng.uniform(0.9, 1.1, size=2)
    I1 = _to_u8(f1 * g1)
    I2 = _to_u8(f2 * g2)
    if rng.random() < 0.3:
        I2 = _box3(I2)

    flow = np.zeros((H, W, 2))
    occ = np.zeros((H, W), bool)
    for li, L in enumerate(layers):
        m = top1 == li
        fx, fy = fwd(L, xs, ys)
        flow[..., 0][m] = (fx - xs)[m]
        flow[..., 1][m] = (fy - ys)[m]
    tx = xs + flow[..., 0]
    ty = ys + flow[..., 1]
    out = (tx < 0) | (tx > W - 1) | (ty < 0) | (ty > H - 1)
    rx = np.clip(np.rint(tx), 0, W - 1).astype(np.int64)
    ry = np.clip(np.rint(ty), 0, H - 1).astype(np.int64)
    occ = out | (top2[ry, rx] != top1)
    return dict(I1=I1, I2=I2, flow=flow.astype(np.float32), occ=occ)


def pair_kitti(seed, W=1242, H=375, max_disp=300.0):
    """KITTI-shaped pair: ground plane under forward motion, sky band, cuboids.

    The camera moves forward, so the ground flows radially away from the focus
    of expansion with magnitude growing towards the bottom of the frame (capped at
    max_disp). The sky band above the horizon is constant up to +-2 noise. A few
    textured boxes move independently and occlude the ground.

    Returns dict(I1, I2 uint8 [H, W, 3], flow float32 [H, W, 2], occ bool [H, W]).
    """
    rng = np.random.default_rng(np.uint64(seed))
    M = 320
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    hor = H * rng.uniform(0.3, 0.4)
    foe = np.array([W * rng.uniform(0.4, 0.6), hor])
    ground_tex = value_noise(rng, H + 2 * M, W + 2 * M,
                             lattices=(48, 16, 6, 2), amps=(0.4, 0.3, 0.2, 0.1))
    sky_col = rng.uniform(0.55, 0.9, size=3)
    # ground flow: d(x) = k (x - foe) * depth-like factor ((y - hor) / (H - hor))
    kmax = max_disp / np.hypot(max(foe[0], W - foe[0]), H - hor)
    k = rng.uniform(0.5, 1.0) * kmax

    def ground_fwd(x, y):
        s = np.clip((y - hor) / (H - hor), 0, None)
        return x + k * s * (x - foe[0]) * 1.0, y + k * s * (y - foe[1])

    boxes = []
    for _ in range(int(rng.integers(2, 5))):
        bw, bh = rng.uniform(60, 220), rng.uniform(40, 140)
        bx, by = rng.uniform(0, W - bw), rng.uniform(hor - bh * 0.5, H - bh)
        tex = value_noise(rng, int(bh) + 4, int(bw) + 4, lattices=(16, 8, 4, 2))
        mv = rng.uniform(-max_disp / 3, max_disp / 3, size=2)
        boxes.append(dict(x=bx, y=by, w=bw, h=bh, tex=tex, mv=mv))

    def render(frame):
        img = np.zeros((H, W, 3))
        top = np.zeros((H, W), np.int32)  # 0 sky, 1 ground, 2+ boxes
        # ground: frame 2 samples the ground texture at the pre-image, found by
        # fixed-point iteration of the forward map (it is monotone per row).
        if frame == 0:
            gx, gy = xs, ys
        else:
            gx, gy = xs.copy(), ys.copy()
            for _ in range(30):
                fx, fy = ground_fwd(gx, gy)
                gx, gy = gx - (fx - xs) * 0.5, gy - (fy - ys) * 0.5
        gmask = gy > hor
        col = _bilinear(ground_tex, gx + M, gy + M)
        img[gmask] = col[gmask]
        top[gmask] = 1
        sky = ~gmask
        noise = rng.integers(-2, 3, size=(H, W, 3)) / 255.0
        img[sky] = (sky_col + noise)[sky]
        for bi, b in enumerate(boxes):
            ox, oy = (b["x"], b["y"]) if frame == 0 else (b["x"] + b["mv"][0], b["y"] + b["mv"][1])
            m = (xs >= ox) & (xs < ox + b["w"]) & (ys >= oy) & (ys < oy + b["h"])
            col = _bilinear(b["tex"], xs - ox, ys - oy)
            img[m] = col[m]
            top[m] = 2 + bi
        return img, top

    f1, top1 = render(0)
    f2, top2 = render(1)
    I1, I2 = _to_u8(f1), _to_u8(f2)
    flow = np.zeros((H, W, 2))
    fx, fy = ground_fwd(xs, ys)
    g = top1 == 1
    flow[..., 0][g] = (fx - xs)[g]
    flow[..., 1][g] = (fy - ys)[g]
    for bi, b in enumerate(boxes):
        m = top1 == 2 + bi
        flow[..., 0][m] = b["mv"][0]
        flow[..., 1][m] = b["mv"][1]
    tx, ty = xs + flow[..., 0], ys + flow[..., 1]
    out = (tx < 0) | (tx > W - 1) | (ty < 0) | (ty > H - 1)
    rx = np.clip(np.rint(tx), 0, W - 1).astype(np.int64)
    ry = np.clip(np.rint(ty), 0, H - 1).astype(np.int64)
    occ = out | (top2[ry, rx] != top1) | (top1 == 0)
    return dict(I1=I1, I2=I2, flow=flow.astype(np.float32), occ=occ)


WORKLOADS = ("noise_128x96", "layers_1024x436", "mixed", "noise_512x218", "kitti_1242x375")


def workload_pair(workload, seed, size=None):
    """A generated pair of one evaluation workload:

    noise_128x96     128x96 shifted value noise with an occluding square;
    layers_1024x436  Sintel-shaped 1024x436 three-layer affine scene;
    mixed            a pair of the mixed-size batch, ``size`` = (W, H) from
                     BATCH_SIZES, shift bounds 0.2 W horizontally, 0.2 H vertically;
    noise_512x218    512x218 shifted value noise (proposal-net training data);
    kitti_1242x375   KITTI-shaped 1242x375 ground plane with radial expansion.
    """
    if workload == "noise_128x96":
        return pair_shift(seed)
    if workload == "layers_1024x436":
        return pair_layers(seed)
    if workload == "mixed":
        W, H = size
        return pair_shift(seed, W=W, H=H,
                          max_shift=(int(round(0.2 * W)), int(round(0.2 * H))))
    if workload == "noise_512x218":
        return pair_shift(seed, W=512, H=218)
    if workload == "kitti_1242x375":
        return pair_kitti(seed)
    raise ValueError(f"unknown workload {workload}")


def mixed_batch(seed0=500, per_size=16):
    """The mixed-size batch: ``per_size`` pairs of each size in BATCH_SIZES, every
    pair generated from its own seed (seed0 + 100 k + i for the i-th pair of the
    k-th size). Returns a list of ((W, H), pair) in size order."""
    out = []
    for k, (W, H) in enumerate(BATCH_SIZES):
        for i in range(per_size):
            out.append(((W, H), workload_pair("mixed", seed0 + 100 * k + i, (W, H))))
    return out
