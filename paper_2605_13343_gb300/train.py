"""Train the hierarchical-transformer preconditioner with hmpcg_train_step (Sec. 6; Supp. C).

Systems are drawn from two seeded pools assembled on the device once (the cached
training contexts of Sec. 6.3 / Supp. D): 16^3 boxes with contrast log-uniform in
[1, 100] and 32x16x16 boxes with 5-12 spheres of contrast 100.  Each step takes a
random batch from one pool (every `--big-every`-th step from the larger grid),
16 probes per system (Rademacher, or with `--probe-kind gaussian` the paper's Gaussian
probes smoothed by two damped-Jacobi sweeps, Sec. 6.2), AdamW with global-norm clipping (inside the
step) and a reduce-on-plateau learning-rate schedule (factor 0.5, patience 5 log
steps, relative threshold 5e-3, floor max(lr * 1e-3, 1e-6); Supp. C).  With
`--auto-stop` training ends once the rate is at its floor and the loss has not
improved for 10 log steps (Supp. C, "Auto-stop").  Every `--eval-every` steps the PCG
iteration count on held-out 32x16x16 frames is measured (inference + PCG, BF16
factors, rtol 1e-6) next to Jacobi PCG; the best checkpoint by mean iterations
is written to `--out` as a flat float32 file in the weight-blob order.

    python -m paper_2605_13343_gb300.train --steps 3000 --out weights.f32
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402
import paper_2605_13343_gb300 as h  # noqa: E402

CFG = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)


class Plateau:
    """Reduce-on-plateau on a minimised quantity (relative threshold), Supp. C: factor 0.5,
    patience 5 log steps, threshold 5e-3, floor max(lr0 * 1e-3, 1e-6)."""

    def __init__(self, lr, factor=0.5, patience=5, threshold=5e-3, min_lr=None):
        if min_lr is None:
            min_lr = max(lr * 1e-3, 1e-6)
        self.lr, self.factor, self.patience, self.threshold, self.min_lr = lr, factor, patience, threshold, min_lr
        self.best = float("inf")
        self.bad = 0

    def step(self, value):
        if value < self.best * (1.0 - self.threshold):
            self.best = value
            self.bad = 0
        else:
            self.bad += 1
            if self.bad > self.patience:
                self.lr = max(self.min_lr, self.lr * self.factor)
                self.bad = 0
        return self.lr


class AutoStop:
    """Early termination of Supp. C: stop once the learning rate sits at its floor and the loss
    has not improved by the relative threshold for ``patience`` consecutive log steps (twice
    the scheduler's patience)."""

    def __init__(self, patience=10, threshold=5e-3):
        self.patience, self.threshold = patience, threshold
        self.best = float("inf")
        self.bad = 0

    def step(self, value, lr, min_lr):
        if value < self.best * (1.0 - self.threshold):
            self.best = value
            self.bad = 0
        else:
            self.bad += 1
        return lr <= min_lr and self.bad >= self.patience


def make_pool(family, seeds):
    out = []
    for s in seeds:
        fr = inputs.frame(family, s)
        sg = h.System(fr["dims"])
        bc = h.BC_NEUMANN if fr["bc"] == "neumann" else h.BC_DIRICHLET
        face = h.FACE_RHO if fr["face"] == "rho" else h.FACE_INV_RHO
        h.assemble(torch.from_numpy(fr["rho"]).cuda(), sg, bc=bc, face=face)
        out.append((sg, torch.from_numpy(fr["b"]).cuda()))
    return out


def split_pools(family, n_train, n_test, seed):
    """The per-scale split of Supp. D: n_train training and n_test test frames of one family
    with disjoint seeds, assembled on the device once (cached contexts, Sec. 6.3)."""
    tr, te = inputs.split_seeds(seed, n_train, n_test)
    return make_pool(family, tr), make_pool(family, te)


def evaluate_detail(ctx, frames, rtol):
    """Mean and standard deviation of learned-H and Jacobi PCG iterations over frames."""
    n = frames[0][0].n
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    fac = h.factors(h.PRE_LEARNED, packed, n, 64, 16)
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it_l, it_j, failed = [], [], 0
    for sg, b in frames:
        h.infer_factors(ctx, [sg], packed)
        info = h.solve(ctx, sg, fac, b, x, rtol=rtol, allow=(h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN, h.E_NAN))
        if info.status == h.OK:
            it_l.append(info.iters)
        else:
            failed += 1
        it_j.append(h.solve(ctx, sg, jac, b, x, rtol=rtol).iters)
    return dict(iters_learned=float(np.mean(it_l)) if it_l else None,
                iters_learned_std=float(np.std(it_l)) if it_l else None, failed=failed,
                iters_jacobi=float(np.mean(it_j)), iters_jacobi_std=float(np.std(it_j)), frames=len(frames))


def evaluate(ctx, frames, rtol=1e-6):
    n = frames[0][0].n
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    fac = h.factors(h.PRE_LEARNED, packed, n, 64, 16)
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    it_l, it_j, ok = [], [], True
    for sg, b in frames:
        h.infer_factors(ctx, [sg], packed)
        info = h.solve(ctx, sg, fac, b, x, rtol=rtol, allow=(h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN, h.E_NAN))
        ok = ok and info.status == h.OK
        it_l.append(info.iters if info.status == h.OK else 10 ** 6)
        it_j.append(h.solve(ctx, sg, jac, b, x, rtol=rtol).iters)
    return float(np.mean(it_l)), float(np.mean(it_j)), ok


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3000, help="step limit (the paper's is 1e5, with --auto-stop)")
    ap.add_argument("--auto-stop", action="store_true",
                    help="stop early once the learning rate is at its floor and the loss has stalled")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--probes", type=int, default=16)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--big-every", type=int, default=4)
    ap.add_argument("--eval-every", type=int, default=250)
    ap.add_argument("--log-every", type=int, default=50)
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--init", default=None)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "hmpcg_d128_l4.f32"))
    ap.add_argument("--log", default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--probe-kind", choices=["rademacher", "gaussian"], default="rademacher")
    ap.add_argument("--omega", type=float, default=0.6)
    ap.add_argument("--smooth-steps", type=int, default=2)
    ap.add_argument("--loss", choices=["cosine", "sai"], default="cosine",
                    help="cosine: Eq. 7; sai: the SAI-loss ablation of Sec. 6.1")
    ap.add_argument("--no-highways", action="store_true", help="highway channels held at zero (ablation)")
    ap.add_argument("--family", default=None,
                    help="train and test on frame families (comma-separated, e.g. barriers2d_1024,barriers2d_4096) "
                         "with the --split of Supp. D instead of the two 3D pools; steps cycle through the "
                         "families, a family of N > 4096 takes a batch of --batch * 4096 / N systems")
    ap.add_argument("--split", default="100/20", help="training/test frame counts with --family")
    args = ap.parse_args()

    w0 = np.fromfile(args.init, dtype=np.float32) if args.init else inputs.network_blob(args.seed, **CFG)
    max_n = 8192
    if args.family:
        max_n = max(max_n, max(int(np.prod(inputs.frame(f, 0)["dims"])) for f in args.family.split(",")))
    ctx = h.Context(max_n=max_n, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                    max_batch=args.batch, weights=w0)
    if args.probe_kind == "gaussian":
        h.set_train_probes(ctx, h.PROBES_GAUSSIAN_SMOOTHED, args.omega, args.smooth_steps)
    if args.loss == "sai":
        h.set_train_loss(ctx, h.LOSS_SAI)
    if args.no_highways:
        h.set_highways(ctx, False)
    rtol = 1e-6
    fam_pools = None
    if args.family:
        n_train, n_test = (int(v) for v in args.split.split("/"))
        fams = args.family.split(",")
        fam_pools = []
        for fam in fams:
            tr, te = split_pools(fam, n_train, n_test, args.seed)
            nb = max(1, min(n_train, args.batch * 4096 // max(4096, tr[0][0].n)))
            fam_pools.append((fam, tr, te, nb))
        rtol = inputs.frame(fams[0], 0)["rtol"]
        # held-out evaluation during training: the largest family's test frames
        small, held, big = fam_pools[-1][1], fam_pools[-1][2], []
    else:
        small = make_pool("spheres3d_4096_lu", range(args.pool))
        big = make_pool("spheres3d_8192", range(10000, 10000 + args.pool // 2))
        held = make_pool("spheres3d_8192", range(20000, 20008))
    rng = np.random.default_rng(args.seed)
    sched = Plateau(args.lr)
    stopper = AutoStop() if args.auto_stop else None
    lr = args.lr
    logf = open(args.log, "w") if args.log else None
    best = float("inf")
    t0 = time.time()
    window = []
    cycle = []
    nfam = len(fam_pools) if fam_pools is not None else 1
    nsample = min(args.log_every, nfam * max(1, 10 // nfam))
    it_l, it_j, ok = evaluate(ctx, held, rtol)
    rec = dict(step=0, iters_learned=it_l, iters_jacobi=it_j, ok=ok, lr=lr, t=0.0)
    print(json.dumps(rec), flush=True)
    for step in range(1, args.steps + 1):
        if fam_pools is not None:
            _, pool, _, nb = fam_pools[step % len(fam_pools)]
            pick = rng.choice(len(pool), size=nb, replace=False)
            batch = [pool[i][0] for i in pick]
        elif big and args.big_every and step % args.big_every == 0:
            pick = rng.choice(len(big), size=max(1, args.batch // 2), replace=False)
            batch = [big[i][0] for i in pick]
        else:
            pick = rng.choice(len(small), size=args.batch, replace=False)
            batch = [small[i][0] for i in pick]
        # the logged loss: the mean over the last `nsample` steps of each log cycle (a multiple of
        # the number of scales, so that every scale is sampled equally): one batch alone is too
        # noisy for the plateau rule, and one scale alone would make it react to the scale
        into_cycle = (-step) % args.log_every
        want = into_cycle < nsample
        loss = h.train_step(ctx, batch, args.probes, lr, int(rng.integers(1 << 62)), want_loss=want)
        stop = False
        if want:
            cycle.append(loss)
        if step % args.log_every == 0:
            loss = float(np.mean(cycle))
            cycle = []
            window.append(loss)
            lr = sched.step(loss)
            stop = stopper is not None and stopper.step(loss, lr, sched.min_lr)
            rec = dict(step=step, loss=loss, lr=lr, t=time.time() - t0)
            if logf:
                logf.write(json.dumps(rec) + "\n")
                logf.flush()
        if step % args.eval_every == 0 or step == args.steps or stop:
            it_l, it_j, ok = evaluate(ctx, held, rtol)
            rec = dict(step=step, iters_learned=it_l, iters_jacobi=it_j, ok=ok, lr=lr, loss=window[-1] if window else None,
                       t=time.time() - t0)
            print(json.dumps(rec), flush=True)
            if logf:
                logf.write(json.dumps(rec) + "\n")
                logf.flush()
            if ok and it_l < best:
                best = it_l
                os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
                h.get_weights(ctx, w0.size).tofile(args.out)
        if stop:
            print(json.dumps(dict(auto_stop=step, lr=lr)), flush=True)
            break
    final = ({fam: evaluate_detail(ctx, te, rtol) for fam, _, te, _ in fam_pools} if fam_pools is not None
             else evaluate_detail(ctx, held, rtol))
    print(json.dumps(dict(done=True, best_iters=best, seconds=time.time() - t0, steps=step, loss_kind=args.loss,
                          highways=not args.no_highways, family=args.family or "spheres3d pools",
                          test_final=final)), flush=True)


if __name__ == "__main__":
    main()
