"""Training and inference driver of the learned proposal net (not in the paper).

The net (ff_net_* entry points) reads the 1/8-scale RGB of both frames and emits
K flow candidates per point of the coarsest search grid (spacing 2^k = 8). It is
trained on labels that plain Flow Fields produces itself: the forward flow of
ff_flow_fields at the coarsest grid points, masked by the filter's valid mask
(Sec. 3.3: only points that survive the consistency check and region filter
are labelled). The loss is the relaxed winner-takes-all L1 over the K
candidates; Adam updates the FP32 master weights. Everything runs in the
library's kernels; this module only schedules calls (no autograd).

At inference the candidates become the `proposals` input of the search (params.K
= K). They are tried after the kd-tree candidates under the exact integer data
term and replace the kd result only on a strictly lower E_d (Eq. 1/4 rerank), so
the plain search stays both the fallback and the arbiter of every candidate.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import torch

from . import ffapi, synth

GRID = 8           # coarsest grid spacing 2^k, k = 3
FLOW_SCALE = 8.0   # net outputs are in units of grid cells (8 px)


def _gen(args):
    workload, seed, size = args
    p = synth.workload_pair(workload, seed, size)
    return p["I1"], p["I2"], p["flow"], p["occ"]


def make_pairs(workload, seeds, size=None, workers=None):
    """Generate pairs of one workload with a spawn pool (safe after CUDA init).

    Returns (I1, I2, flow, occ) stacked over the seeds: uint8 [N][H][W][3] x2,
    flow [N][H][W][2] (the generator's ground truth), occ bool [N][H][W]."""
    seeds = list(seeds)
    workers = workers or min(len(seeds), os.cpu_count() or 1, 16)
    args = [(workload, s, size) for s in seeds]
    if workers <= 1:
        res = [_gen(a) for a in args]
    else:
        # a dead worker raises BrokenProcessPool instead of being respawned
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_gen, args, chunksize=max(1, len(args) // (4 * workers))))
    return tuple(np.stack([r[i] for r in res]) for i in range(4))


def plain_labels(I1, I2, params=None, batch=64, device="cuda"):
    """Labels from plain Flow Fields: forward flow and filter mask at the grid points.

    I1, I2: uint8 [N][H][W][3] (host numpy or CUDA tensors, all one size).
    Returns label int16 [N][Gy][Gx][2] and valid uint8 [N][Gy][Gx] as CUDA tensors."""
    N, H, W = I1.shape[:3]
    P = ffapi._params(params).as_dict()
    P["K"] = 0
    nb = min(batch, N)
    run = ffapi.FlowFieldsBatch([(W, H)] * nb, P, device=device, graph=True)
    Gy, Gx = (H + GRID - 1) // GRID, (W + GRID - 1) // GRID
    label = torch.empty((N, Gy, Gx, 2), dtype=torch.int16, device=device)
    valid = torch.empty((N, Gy, Gx), dtype=torch.uint8, device=device)
    for i0 in range(0, N, nb):
        idx = [min(i, N - 1) for i in range(i0, i0 + nb)]  # last chunk: repeat the tail pair
        frames = [(torch.as_tensor(I1[i]).to(device, non_blocking=True),
                   torch.as_tensor(I2[i]).to(device, non_blocking=True)) for i in idx]
        outs = run.run(frames)
        for j, i in enumerate(range(i0, min(i0 + nb, N))):
            label[i] = outs[j]["flows"][0, ::GRID, ::GRID]
            valid[i] = outs[j]["valid"][::GRID, ::GRID]
    return label, valid


class ProposalNet:
    """FP32 master weights, Adam state and per-batch-shape runners of the net."""

    def __init__(self, desc=None, seed=0, device="cuda"):
        self.desc = desc if desc is not None else ffapi.net_desc()
        self.device = torch.device(device)
        self.K = self.desc.k
        n = ffapi.ff_net_param_count(self.desc)
        ch = [self.desc.cin, self.desc.c1, self.desc.c2, self.desc.c3, 2 * self.desc.k]
        rng = np.random.default_rng(seed)
        p = np.zeros(n, np.float32)
        off = 0
        for l in range(4):
            cin, cout = ch[l], ch[l + 1]
            nw = cout * cin * 9
            # He initialisation; the last layer starts small so that early
            # candidates stay near zero flow
            std = np.sqrt(2.0 / (9 * cin)) * (0.1 if l == 3 else 1.0)
            p[off:off + nw] = rng.normal(scale=std, size=nw)
            off += nw + cout
        self.params = torch.from_numpy(p).to(self.device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._runners = {}

    def runner(self, B, Gx, Gy):
        key = (B, Gx, Gy)
        if key not in self._runners:
            self._runners[key] = ffapi.NetRunner(self.desc, B, Gx, Gy, self.device)
        return self._runners[key]

    # ------------------------------------------------------------ training --
    def train(self, x, label, valid, epochs=10, batch=64, lr=2e-3, alpha=0.05, seed=0,
              log_every=0):
        """x float32 [N][6][Gy][Gx] (ff_net_input), label/valid as from plain_labels.
        Returns the per-step losses (host floats, read once at the end)."""
        N, _, Gy, Gx = x.shape
        B = min(batch, N)
        run = self.runner(B, Gx, Gy)
        rng = np.random.default_rng(seed)
        losses = torch.empty(epochs * (N // B), dtype=torch.float32, device=self.device)
        it = 0
        for ep in range(epochs):
            order = torch.from_numpy(rng.permutation(N)).to(self.device)
            for b0 in range(0, N - B + 1, B):
                idx = order[b0:b0 + B]
                xb = x.index_select(0, idx).contiguous()
                lb = label.index_select(0, idx).contiguous()
                vb = valid.index_select(0, idx).contiguous()
                run.forward(self.params, xb)
                loss, _ = run.loss_grad(lb, vb, FLOW_SCALE, alpha)
                losses[it:it + 1].copy_(loss)
                run.backward(self.params, self.grads)
                self.step += 1
                ffapi.ff_net_adam(self.params, self.grads, self.m, self.v, self.step, lr)
                it += 1
                if log_every and it % log_every == 0:
                    print(f"epoch {ep} step {it} loss {float(loss.item()):.4f}", flush=True)
        return losses[:it].cpu().numpy()

    # ----------------------------------------------------------- inference --
    def infer(self, I1, I2):
        """I1, I2: uint8 [B][H][W][3] CUDA tensors -> proposals int16 [B][Gy][Gx][K][2]."""
        x = ffapi.ff_net_input(I1, I2)
        B, _, Gy, Gx = x.shape
        run = self.runner(B, Gx, Gy)
        run.forward(self.params, x)
        return run.proposals(FLOW_SCALE)

    # --------------------------------------------------------- checkpoints --
    def save(self, path):
        d = self.desc
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(),
                 v=self.v.cpu().numpy(), step=self.step,
                 desc=np.array([d.cin, d.c1, d.c2, d.c3, d.k, *d.dil], np.int32))

    @classmethod
    def load(cls, path, device="cuda"):
        z = np.load(path)
        dd = [int(v) for v in z["desc"]]
        net = cls(ffapi.net_desc(dd[1], dd[2], dd[3], dd[4], tuple(dd[5:9])), device=device)
        net.params.copy_(torch.from_numpy(z["params"]))
        net.m.copy_(torch.from_numpy(z["m"]))
        net.v.copy_(torch.from_numpy(z["v"]))
        net.step = int(z["step"])
        return net


# ------------------------------------------------------------- evaluation ----
def flow_quality(flow, gt, occ):
    """inliers@3px (EPE <= 3, reading of Table 1's measure) and mean EPE of the raw
    forward flow over non-occluded ground-truth pixels. flow: [N][H][W][2]."""
    f = np.asarray(flow, np.float64)
    e = np.sqrt(((f - gt) ** 2).sum(-1))
    m = ~np.asarray(occ, bool)
    return float((e[m] <= 3.0).mean()), float(e[m].mean())


def paired_inlier_delta(flow_a, flow_b, gt, occ):
    """Per-pair difference of inliers@3px, arm a minus arm b, over the same pairs:
    mean and standard error of the mean (n - 1 in the variance; 0 for one pair)."""
    d = []
    for j in range(len(gt)):
        d.append(flow_quality(flow_a[j:j + 1], gt[j:j + 1], occ[j:j + 1])[0]
                 - flow_quality(flow_b[j:j + 1], gt[j:j + 1], occ[j:j + 1])[0])
    d = np.asarray(d, np.float64)
    se = float(d.std(ddof=1) / np.sqrt(len(d))) if len(d) > 1 else 0.0
    return dict(mean=float(d.mean()), se=se, pairs=len(d))


def run_arm(net, I1, I2, params, batch=32, device="cuda", reps=5):
    """Forward flows of all pairs with one arm (plain if params.K == 0, else with
    the net's proposals) and the device time per pair (ms, CUDA events, median over
    batches of `reps` graph replays; the learned arm includes the net)."""
    N, H, W = I1.shape[:3]
    B = min(batch, N)
    P = ffapi._params(params).as_dict()
    learned = P["K"] > 0
    if learned and P["K"] != net.K:
        raise ValueError("params.K differs from the net's K")
    run = ffapi.FlowFieldsBatch([(W, H)] * B, P, device=device, graph=True)
    flows, ms = [], []
    for i0 in range(0, N - B + 1, B):
        a = torch.as_tensor(I1[i0:i0 + B]).to(device)
        b = torch.as_tensor(I2[i0:i0 + B]).to(device)
        frames = [(a[j], b[j]) for j in range(B)]

        def step():
            prop = None
            if learned:
                pr = net.infer(a, b)
                prop = [pr[j] for j in range(B)]
            return run.run(frames, prop)

        step()  # capture / warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            outs = step()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1) / reps / B)
        flows.append(torch.stack([o["flows"][0] for o in outs]).cpu().numpy())
    return np.concatenate(flows), float(np.median(ms))


def coarse_cost_delta(net, I1, I2, params=None, device="cuda"):
    """Data-cost delta of the proposals at the coarsest level (Eq. 4 init).

    For every pair the kd-tree init runs twice through ff_kdtree_init, without and
    with the net's K candidates. Strict-less acceptance makes the cost with
    proposals <= the cost without at every grid point. Returns the fraction of
    grid points where a proposal won, the mean relative cost reduction, and
    whether the <= property held everywhere."""
    P = ffapi._params(params).as_dict()
    n, r, leaf = 1 << P["k"], P["r"], P["leaf"]
    a = torch.as_tensor(I1).to(device)
    b = torch.as_tensor(I2).to(device)
    prop = net.infer(a, b)
    won, tot, c0s, c1s, ok = 0, 0, 0.0, 0.0, True
    for j in range(a.shape[0]):
        C1 = ffapi.ff_census(ffapi.ff_smooth(a[j], n), n)
        C2 = ffapi.ff_census(ffapi.ff_smooth(b[j], n), n)
        T = ffapi.ff_kdtree_build(ffapi.ff_features(b[j], r), leaf)
        _, c0 = ffapi.ff_kdtree_init(T, leaf, a[j], C1, C2, n, r)
        _, c1 = ffapi.ff_kdtree_init(T, leaf, a[j], C1, C2, n, r, prop[j].contiguous())
        c0, c1 = c0.cpu().numpy().astype(np.int64), c1.cpu().numpy().astype(np.int64)
        ok &= bool((c1 <= c0).all())
        won += int((c1 < c0).sum())
        tot += c0.size
        c0s += float(c0.sum())
        c1s += float(c1.sum())
    return dict(frac_won=won / max(tot, 1), cost_reduction=1.0 - c1s / max(c0s, 1.0),
                never_worse=ok)


def evaluate(net, I1, I2, gt, occ, n_rs_list=(1, 2, 3), params=None, batch=32,
             device="cuda", reps=5):
    """Plain search vs search with the net's proposals on the same pairs, at each
    random-search budget n_rs. Per arm and budget: ms per pair, inliers@3px, EPE;
    per budget the fraction of pixels where the two forward flows differ and the
    per-pair inlier difference (learned - plain, mean and standard error); and the
    proposals' data-cost delta at the coarsest level."""
    base = ffapi._params(params).as_dict()
    out = dict(coarse=coarse_cost_delta(net, I1, I2, base, device), arms={})
    for n_rs in n_rs_list:
        fl = {}
        for name, K in (("plain", 0), ("learned", net.K)):
            f, ms = run_arm(net, I1, I2, dict(base, n_rs=n_rs, K=K), batch, device, reps)
            m = f.shape[0]
            inl, epe = flow_quality(f, gt[:m], occ[:m])
            out["arms"][f"{name}_rs{n_rs}"] = dict(ms_per_pair=round(ms, 4),
                                                   inliers_3px=round(inl, 5), epe=round(epe, 4))
            fl[name] = f
        d = np.abs(fl["learned"].astype(np.int32) - fl["plain"].astype(np.int32)).sum(-1)
        out["arms"][f"changed_rs{n_rs}"] = round(float((d > 0).mean()), 5)
        m = fl["plain"].shape[0]
        dl = paired_inlier_delta(fl["learned"], fl["plain"], gt[:m], occ[:m])
        out["arms"][f"inlier_delta_rs{n_rs}"] = {k: (round(v, 6) if isinstance(v, float) else v)
                                                 for k, v in dl.items()}
    return out


def equal_inlier_point(ev, ref=None):
    """The cheapest learned arm whose inliers@3px reach the reference arm's; None
    if no learned budget reaches it. The reference defaults to the plain arm with
    the largest random-search budget evaluated."""
    arms = ev["arms"]
    if ref is None:
        plain = [k for k in arms if k.startswith("plain_rs")]
        ref = max(plain, key=lambda k: int(k[len("plain_rs"):]))
    target = arms[ref]["inliers_3px"]
    ok = [(v["ms_per_pair"], k) for k, v in arms.items()
          if k.startswith("learned_") and v["inliers_3px"] >= target]
    if not ok:
        return None
    ms, k = min(ok)
    return dict(arm=k, ms_per_pair=ms, ref=ref, ref_ms_per_pair=arms[ref]["ms_per_pair"],
                speedup=round(arms[ref]["ms_per_pair"] / ms, 4))


def forward_flow_levels(I1, I2, budgets, proposals=None, params=None):
    """Forward flow of one pair (uint8 [H][W][3] CUDA tensors) composed from the
    per-level entry points, with its own random-search budget per level:
    budgets[i] is n_rs at the level of spacing 2^(k-i) (coarsest first). Features
    of I2, the kd tree, the kd init (with the net's proposals if given) and the
    top level in place, then each finer level seeded from the one above (Sec. 3.2,
    Fig. 2). With a uniform budget this is ff_flow_fields' forward flow."""
    P = ffapi._params(params).as_dict()
    k, r, leaf = P["k"], P["r"], P["leaf"]
    if len(budgets) != k + 1:
        raise ValueError(f"need {k + 1} budgets, one per level")
    tree = ffapi.ff_kdtree_build(ffapi.ff_features(I2, r), leaf)
    flow = cost = None
    for i in range(k + 1):
        n = 1 << (k - i)
        a = ffapi.ff_smooth(I1, n) if n > 1 else I1
        b = ffapi.ff_smooth(I2, n) if n > 1 else I2
        C1, C2 = ffapi.ff_census(a, n), ffapi.ff_census(b, n)
        Pl = dict(P, n_rs=int(budgets[i]))
        if i == 0:
            flow, cost = ffapi.ff_kdtree_init(tree, leaf, I1, C1, C2, n, r, proposals)
            ffapi.ff_search_level(C1, C2, n, r, Pl, flow_id=0, flow=flow, cost=cost)
        else:
            flow, _ = ffapi.ff_search_level(C1, C2, n, r, Pl, flow_id=0, flow_coarse=flow)
    return flow


def level_budget_study(net, I1, I2, gt, occ, budgets, params=None, device="cuda"):
    """Inliers@3px and EPE of the forward flow for per-level random-search budgets
    (tuples, coarsest level first), plain and with the net's proposals. Shows
    which levels' random search the flow quality depends on."""
    a = torch.as_tensor(I1).to(device)
    b = torch.as_tensor(I2).to(device)
    prop = net.infer(a, b) if net is not None else None
    out = {}
    for bud in budgets:
        arms = (("plain", None),) + ((("learned", prop),) if prop is not None else ())
        for name, pr in arms:
            fl = [forward_flow_levels(a[j], b[j], bud, None if pr is None else pr[j].contiguous(),
                                      params).cpu().numpy() for j in range(a.shape[0])]
            inl, epe = flow_quality(np.stack(fl), gt, occ)
            out[f"{name}_{''.join(str(int(v)) for v in bud)}"] = dict(
                inliers_3px=round(inl, 5), epe=round(epe, 4))
    return out


def train_for(workload, n_train, epochs, batch=64, lr=2e-3, seed=1000, size=None, log=None):
    """Generate pairs, label them with plain Flow Fields and train a net."""
    import time
    t0 = time.time()
    I1, I2, _, _ = make_pairs(workload, range(seed, seed + n_train), size)
    t1 = time.time()
    label, valid = plain_labels(I1, I2)
    x = ffapi.ff_net_input(torch.from_numpy(I1).cuda(), torch.from_numpy(I2).cuda())
    torch.cuda.synchronize()
    t2 = time.time()
    net = ProposalNet(seed=seed)
    losses = net.train(x, label, valid, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    t3 = time.time()
    info = dict(workload=workload, pairs=n_train, epochs=epochs, batch=min(batch, n_train),
                steps=len(losses), gen_s=round(t1 - t0, 2), label_s=round(t2 - t1, 2),
                train_s=round(t3 - t2, 2), loss_first=round(float(losses[:10].mean()), 4),
                loss_last=round(float(losses[-10:].mean()), 4))
    return net, info


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the proposal net on plain-FF labels")
    ap.add_argument("--workload", default="noise_512x218", choices=[w for w in synth.WORKLOADS if w != "mixed"])
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--eval", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--n-rs", default="1,2,3", help="random-search budgets to compare")
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--save", default=None, help="checkpoint path (.npz)")
    ap.add_argument("--load", default=None, help="skip training, load this checkpoint")
    ap.add_argument("--level-budgets", default=None,
                    help="per-level n_rs study on the eval pairs, e.g. 3333,1333,3331 "
                         "(coarsest level first)")
    a = ap.parse_args(argv)
    if a.load:
        net, info = ProposalNet.load(a.load), dict(loaded=a.load)
    else:
        net, info = train_for(a.workload, a.train, a.epochs, a.batch, a.lr, a.seed)
    if a.save:
        net.save(a.save)
    E1, E2, Egt, Eocc = make_pairs(a.workload, range(a.seed + 10**6, a.seed + 10**6 + a.eval))
    ev = evaluate(net, E1, E2, Egt, Eocc, tuple(int(v) for v in a.n_rs.split(",")))
    res = dict(train=info, eval=ev, equal_inliers=equal_inlier_point(ev))
    if a.level_budgets:
        buds = [tuple(int(c) for c in w) for w in a.level_budgets.split(",")]
        res["level_budgets"] = level_budget_study(net, E1, E2, Egt, Eocc, buds)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
