"""Per-frame benchmark: learned-H PCG (inference + solve) at N = 8192.

Workload: 3D 32x16x16 Dirichlet grids, density 1 with 100 inside 5-12 seeded
spheres (radii 2-6), b ~ N(0, I) minus its mean; leaf 64, rank 16; network
d=128, 4 layers, 4 heads, MLP 512 (seeded init, or a trained checkpoint with
--weights); BF16 factors and apply, FP64 PCG scalars, rtol 1e-6.

A step is one frame: hmpcg_infer_factors + hmpcg_solve on that frame's system
(the paper's per-frame "Total = Infer + Solve").  Systems and right-hand sides
of all frames are assembled on the device before timing; L2 is flushed (a
256 MiB write) before every frame outside its CUDA-event bracket.

Prints one JSON line (see the design notes for every key).  `--impl reference`
times the FP64 CPU oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/frame to rtol 1e-6 at N=8192 (learned-H vs Jacobi PCG); apply/SpMV %HBM roof"
FAMILY = "spheres3d_8192"
CFG = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)
# dram__bytes_read.sum + dram__bytes_write.sum of one pcg_cluster_kernel<bf16, H-matrix> launch of
# this workload (ncu, --clock-control none); the factors and the system are read from HBM once
PCG_TRAFFIC_BYTES = 2253824


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self):
        self.rows = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", "0", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reference_arm(args):
    """The FP64 CPU oracle on a bounded sample: oracle network forward + oracle PCG."""
    import numpy as np
    import torch
    import inputs
    from oracle import grid, hmatrix, network, pcg
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    torch.set_num_threads(os.cpu_count() or 1)
    blob = _weights_blob(args.weights, inputs)
    p = network.unflatten(blob, inputs.network_layout(**CFG))
    times, iters = [], []
    nframes = max(1, min(args.steps, 2))
    for k in range(nframes):
        fr = inputs.frame(FAMILY, 1000 + k)
        sys_ = grid.assemble(fr["rho"], fr["dims"])
        a = grid.sparse_matrix(sys_)
        t0 = time.perf_counter()
        with torch.no_grad():
            f = network.to_numpy_factors(network.forward(p, sys_, CFG))
        out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(f, v), fr["b"], rtol=1e-6)
        times.append((time.perf_counter() - t0) * 1e3)
        iters.append(out["iters"])
    v = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/frame", "n_gpus": args.gpus,
            "steps": len(times), "warmup": 0, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "learned-H PCG, 3D 32x16x16 spheres 1:100, N=8192, rtol 1e-6",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "ms/frame", "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": f"{len(times)} frames (seeds 1000+), oracle "
                             "network forward (torch FP64) + oracle PCG (numpy/scipy FP64)"},
            "e2e": {"value": v, "unit": "ms/frame", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters_mean": statistics.mean(iters)}
    print(json.dumps(line), flush=True)


def frame_seeds(rank, nframes):
    """Seeds of one rank's frames.  Replicas process disjoint frames (weak scaling), so no
    frame is timed twice across ranks and no data-path collective is needed."""
    if not 0 <= nframes <= 100000:
        raise ValueError("at most 100000 frames per rank")
    return [rank * 100000 + k for k in range(nframes)]


def whole_job_ms_per_unit(dist, device, step_ms, units_per_step=1):
    """Whole-job value of a time-like metric over replicas.

    Every rank times the same number of steps.  The job's time is the slowest rank's total
    (a MAX all-reduce when a process group is up; `device` is where the reduced tensor lives:
    cuda for NCCL, cpu for gloo), and the job processed world x steps x units_per_step units.
    Returns (job ms per unit, slowest rank's ms per step).  With one process both equal the
    mean step time divided by units_per_step, resp. the mean step time.
    """
    steps = len(step_ms)
    if steps == 0:
        raise ValueError("no timed steps")
    total = float(sum(step_ms))
    world = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total / (world * steps * units_per_step), total / steps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_2605_13343_gb300", "weights",
                                                      "hmpcg_d128_l4.f32"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the training-step and batch measurements")
    ap.add_argument("--workload", default="frame8192", choices=["frame8192", "batch64", "precision16384", "svdh8192", "bandwidth", "train4096",
                             "barriers"],
                    help="frame8192: the per-frame headline; batch64: 64 ragged systems in one graph; "
                         "precision16384: FP32/BF16/FP8 apply sweep with SVD-H factors")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    import inputs
    import paper_2605_13343_gb300 as h

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hbm_peak, bf16_peak, peak_kind = _peaks()

    # weights: trained checkpoint if present, else the seeded init
    if os.path.exists(args.weights):
        w = np.fromfile(args.weights, dtype=np.float32)
        wsrc = os.path.basename(args.weights)
    else:
        w = inputs.network_blob(0, **CFG)
        wsrc = "seeded init"
    if args.workload == "precision16384":
        return bench_precision(args, h, torch, np, inputs, hbm_peak, peak_kind)
    if args.workload == "train4096":
        return bench_train(args, h, torch, np, inputs, bf16_peak, peak_kind)
    if args.workload == "bandwidth":
        return bench_bandwidth(args, h, torch, np, hbm_peak, peak_kind)
    if args.workload == "barriers":
        return bench_barriers(args, h, torch, np, inputs)
    if args.workload == "svdh8192":
        return bench_precision(args, h, torch, np, inputs, hbm_peak, peak_kind, family=FAMILY)
    if args.workload == "batch64":
        return bench_batch(args, h, torch, np, inputs, w, wsrc)
    n = 8192
    ctx = h.Context(max_n=n, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                    max_batch=1, weights=w)
    nfr = args.warmup + args.steps
    seeds = frame_seeds(rank, nfr)
    frames = [inputs.frame(FAMILY, s) for s in seeds]
    systems, bs = [], []
    for fr in frames:
        s = h.System(fr["dims"])
        h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
        systems.append(s)
        bs.append(torch.from_numpy(fr["b"]).cuda())
    P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    packed = torch.empty(P, dtype=torch.bfloat16, device="cuda")
    fac = h.factors(h.PRE_LEARNED, packed, n, 64, 16)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    graph_error = None
    stream = torch.cuda.current_stream()
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI

    # One frame = inputs copied into a fixed device slot, then assemble + infer + solve,
    # all captured once into a CUDA graph and replayed per frame.
    slot_rho = torch.empty(n, dtype=torch.float64, device="cuda")
    slot_b = torch.empty(n, dtype=torch.float64, device="cuda")
    slot_sys = h.System(frames[0]["dims"])
    rho_dev = [torch.from_numpy(fr["rho"]).cuda() for fr in frames]

    def body():
        h.assemble(slot_rho, slot_sys)
        h.infer_factors(ctx, [slot_sys], packed)
        h.solve(ctx, slot_sys, fac, slot_b, x, rtol=1e-6, info=False)

    for _ in range(2):   # warm-up outside capture (first-use attributes, tensor-map encoders)
        slot_rho.copy_(rho_dev[0]); slot_b.copy_(bs[0]); body()
    torch.cuda.synchronize()
    graph = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            body()
        graph = g
    except Exception as exc:  # fall back to direct launches
        graph_error = str(exc)
    torch.cuda.synchronize()

    def frame_learned(k):
        slot_rho.copy_(rho_dev[k], non_blocking=True)
        slot_b.copy_(bs[k], non_blocking=True)
        if graph is not None:
            graph.replay()
        else:
            body()

    def timed(fn, ks):
        ev = []
        for k in ks:
            flush.fill_(k & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    # warm-up frames (untimed)
    for k in range(args.warmup):
        frame_learned(k)
    torch.cuda.synchronize()
    ks = list(range(args.warmup, nfr))
    clk = ClockSampler()
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_learned = timed(frame_learned, ks)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    # value: the job's ms per frame (slowest rank's time over all ranks' frames);
    # ms_per_step: the slowest rank's ms per frame
    value_ms, ms = whole_job_ms_per_unit(dist if world > 1 else None, "cuda", t_learned)

    # iteration counts and accuracy of the learned frames; Jacobi on the same frames
    it_l, it_j, res_l, ms_inf, ms_sol = [], [], [], [], []
    for k in ks:
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        h.infer_factors(ctx, [systems[k]], packed)
        e1.record(stream)
        inf = h.solve(ctx, systems[k], fac, bs[k], x, rtol=1e-6)
        e2.record(stream)
        torch.cuda.synchronize()
        ms_inf.append(e0.elapsed_time(e1))
        ms_sol.append(e1.elapsed_time(e2))
        it_l.append(inf.iters)
        res_l.append(inf.rel_res_true)
    t_jac = timed(lambda k: h.solve(ctx, systems[k], jac, bs[k], x, rtol=1e-6, info=False), ks)
    for k in ks:
        it_j.append(h.solve(ctx, systems[k], jac, bs[k], x, rtol=1e-6).iters)

    # the same frames with the factors emitted and applied in FP8-E4M3 (one scale per block),
    # captured as a graph like the BF16 frame
    K = n // 64
    packed8 = torch.empty(P, dtype=torch.float8_e4m3fn, device="cuda")
    sc8 = torch.empty(4 * K + K - 1, dtype=torch.float32, device="cuda")
    fac8 = h.factors(h.PRE_LEARNED, packed8, n, 64, 16, sc8)

    def body8():
        h.assemble(slot_rho, slot_sys)
        h.infer_factors(ctx, [slot_sys], packed8, scales=sc8)
        h.solve(ctx, slot_sys, fac8, slot_b, x, rtol=1e-6, info=False)

    slot_rho.copy_(rho_dev[0]); slot_b.copy_(bs[0]); body8()
    torch.cuda.synchronize()
    graph8 = None
    try:
        g8 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g8, capture_error_mode="relaxed"):
            body8()
        graph8 = g8
    except Exception:
        graph8 = None
    torch.cuda.synchronize()

    def frame_fp8(k):
        slot_rho.copy_(rho_dev[k], non_blocking=True)
        slot_b.copy_(bs[k], non_blocking=True)
        if graph8 is not None:
            graph8.replay()
        else:
            body8()

    t_fp8 = timed(frame_fp8, ks)
    it_8, res_8 = [], []
    for k in ks:
        h.infer_factors(ctx, [systems[k]], packed8, scales=sc8)
        inf8 = h.solve(ctx, systems[k], fac8, bs[k], x, rtol=1e-6, allow=(h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN))
        it_8.append(inf8.iters)
        res_8.append(inf8.rel_res_true)

    # end to end through the public API with host buffers: H2D of rho and b into the slot,
    # the captured frame, D2H of x
    rho_h = [torch.from_numpy(fr["rho"]).pin_memory() for fr in frames]
    b_h = [torch.from_numpy(fr["b"]).pin_memory() for fr in frames]
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()

    def frame_e2e(k):
        slot_rho.copy_(rho_h[k], non_blocking=True)
        slot_b.copy_(b_h[k], non_blocking=True)
        if graph is not None:
            graph.replay()
        else:
            body()
        x_h.copy_(x, non_blocking=True)

    for k in range(args.warmup):
        frame_e2e(k)
    t_e2e = timed(frame_e2e, ks)
    e2e_ms, _ = whole_job_ms_per_unit(dist if world > 1 else None, "cuda", t_e2e)

    # launches per frame: capture one frame's calls into a CUDA graph with the driver API and
    # count its kernel nodes (every kernel of a frame is ours: assembly, inference, solve)
    launches = _count_kernel_nodes(torch, body)

    # roofline of the dominant kernel: the persistent PCG kernel (solve share of the frame)
    # algorithmic bytes per iteration (FP32 vectors, BF16 factors): SpMV 24 N + apply
    # (2 P + 12 N) + vector passes 40 N
    iters_mean = statistics.mean(it_l)
    bytes_iter = 24 * n + (2 * P + 12 * n) + 40 * n
    sol_ms = statistics.mean(ms_sol)
    achieved = bytes_iter * iters_mean / (sol_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "pcg_kernel<bf16, H-matrix> (whole solve)", "achieved": achieved,
            "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": PCG_TRAFFIC_BYTES,
            "peak_kind": f"{peak_kind} (copy bandwidth)",
            "note": "latency-bound at N=8192: the per-iteration working set (~2 MB) is L2-resident"}

    # HBM rooflines of the bandwidth kernels (SpMV, H-apply) at sizes above L2, measured after
    # the timed region so that the frame numbers are unaffected
    bw_rows = None
    if rank == 0:
        try:
            bw_rows = [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r_.items()}
                       for r_ in bandwidth_rows(h, torch, np, hbm_peak, 10, 3)]
        except Exception as exc:  # reported, not fatal
            bw_rows = [{"error": str(exc)[:200]}]

    # secondary workloads, after the timed region so that the frame numbers are unaffected: the
    # training step and the 64-system ragged batch (their own --workload runs print full lines)
    secondary = None
    if rank == 0 and not args.no_secondary:
        secondary = {}
        small = argparse.Namespace(**vars(args))
        small.steps, small.warmup = 5, 2
        try:
            t = bench_train(small, h, torch, np, inputs, bf16_peak, peak_kind, emit=False)
            secondary["train4096"] = {"ms_per_step": t["value"], "steps": t["steps"], "workload": t["config"]["workload"]}
        except Exception as exc:  # reported, not fatal
            secondary["train4096"] = {"error": str(exc)[:200]}
        try:
            bt = bench_batch(small, h, torch, np, inputs, w, wsrc, emit=False)
            secondary["batch64"] = {"solves_per_s": bt["value"], "ms_per_batch": bt["ms_per_step"],
                                    "learned_converged": bt["learned_converged"],
                                    "jacobi_fallbacks": bt["jacobi_fallbacks"], "iters_mean": bt["iters_mean"],
                                    "jacobi": bt["jacobi"], "steps": bt["steps"]}
        except Exception as exc:
            secondary["batch64"] = {"error": str(exc)[:200]}
        try:
            br = bench_barriers(small, h, torch, np, inputs, emit=False)
            secondary["barriers_rtol1e-8"] = {"weights": br["config"]["weights"], "sizes": br["sizes"],
                                              "paper_size_model": br["paper_size_model"]}
        except Exception as exc:
            secondary["barriers_rtol1e-8"] = {"error": str(exc)[:200]}
        torch.cuda.synchronize()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = _cpu_baseline(args.weights)
        except Exception as e:  # pragma: no cover - reported, not fatal
            cpu = {"error": str(e)}

    line = {
        "metric": METRIC, "value": value_ms, "unit": "ms/frame", "n_gpus": world, "steps": len(ks),
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned-H PCG (infer + solve), 3D 32x16x16 spheres 1:100, N=8192, "
                               "leaf 64, rank 16, d128 4 layers 4 heads MLP 512, BF16 factors, rtol 1e-6",
                   "weights": wsrc, "l2": "flushed (256 MiB write) before every frame, outside the timing",
                   "parallelism": f"replicas x{world}"},
        "breakdown": {"ms_per_frame_std": statistics.pstdev(t_learned), "e2e_ms_std": statistics.pstdev(t_e2e),
                      "infer_ms": statistics.mean(ms_inf), "solve_ms": sol_ms,
                      "iters_learned": iters_mean, "true_rel_res_max": max(res_l),
                      "jacobi_ms_per_frame": statistics.mean(t_jac), "iters_jacobi": statistics.mean(it_j),
                      "jacobi_speedup": statistics.mean(t_jac) / ms,
                      "fp8_factors": {"ms_per_frame": statistics.mean(t_fp8), "iters": statistics.mean(it_8),
                                      "true_rel_res_max": max(res_8), "cuda_graph": graph8 is not None}},
        "roofline": roof,
        "roofline_bandwidth_kernels": bw_rows,
        "e2e": {"value": e2e_ms, "unit": "ms/frame", "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": (launches * len(ks)) if launches else None,
        "cuda_graph": graph is not None if graph_error is None else f"direct launches ({graph_error[:80]})",
        "clocks": clocks,
        "cpu_baseline": cpu,
        "secondary": secondary,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- secondary workloads
def _dense_from_system(torch, s):
    """Dense FP64 A (Morton order) from an assembled system, on the device."""
    n, dims = s.n, s.dims
    dev = s.diag.device
    perm = s.perm.long()
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(n, device=dev)
    a = torch.zeros(n, n, dtype=torch.float64, device=dev)
    ar = torch.arange(n, device=dev)
    a[ar, ar] = s.diag
    stride = 1
    for ax, d in enumerate(dims):
        c = (perm // stride) % d
        has = c < d - 1
        i = ar[has]
        j = inv[perm[has] + stride]
        w = s.wplus(ax)[has]
        a[i, j] = -w
        a[j, i] = -w
        stride *= d
    return a


def _svdh_torch(torch, ainv, leaf, rank):
    """SVD-H factors of a dense inverse (leaves (A^-1)_kk, tiles' truncated SVD), packed in the
    SVD-H layout [G][Sigma][W per level].  Tiles wider than 1024 use a randomized truncated
    SVD (8 extra columns, 6 power iterations)."""
    n = ainv.shape[0]
    K = n // leaf
    levels = K.bit_length() - 1
    G = ainv.reshape(K, leaf, K, leaf).diagonal(dim1=0, dim2=2).permute(2, 0, 1).contiguous()
    sig = torch.zeros(K - 1, rank, rank, dtype=torch.float64, device=ainv.device)
    W = torch.zeros(levels, n, rank, dtype=torch.float64, device=ainv.device)
    for lev in range(1, levels + 1):
        S = (K >> lev) * leaf
        for t in range(1 << (lev - 1)):
            m = (1 << (lev - 1)) - 1 + t
            r0, c0 = 2 * t * S, (2 * t + 1) * S
            X = ainv[r0:r0 + S, c0:c0 + S]
            rr = min(rank, S)
            if S <= 1024:
                U, sv, Vh = torch.linalg.svd(X)
                V = Vh.mH
            else:
                U, sv, V = torch.svd_lowrank(X, q=rr + 8, niter=6)
            sig[m, torch.arange(rr), torch.arange(rr)] = sv[:rr]
            W[lev - 1, r0:r0 + S, :rr] = U[:, :rr]
            W[lev - 1, c0:c0 + S, :rr] = V[:, :rr]
    return G, sig, W


def _fp8_blocks(torch, blocks):
    """Per-block FP8-E4M3 quantisation: (stored, scale) with value = stored * scale."""
    flat = blocks.reshape(blocks.shape[0], -1)
    amax = flat.abs().amax(dim=1).clamp_min(1e-300)
    sc = amax / 448.0
    q = (flat / sc[:, None]).to(torch.float32).to(torch.float8_e4m3fn)
    return q.flatten(), sc.to(torch.float32)


def bench_precision(args, h, torch, np, inputs, hbm_peak, peak_kind, family="discs2d_16384"):
    """SVD-H PCG by apply precision.  discs2d_16384 (the precision sweep): 2D 128x128, 20 discs
    of contrast 100, leaf 64, rank 32; spheres3d_8192: the per-frame workload's grid with SVD-H
    leaf 64, rank 16.  PCG with the apply in FP32, BF16 and FP8-E4M3 (per-block scales), FP64
    scalars, true residual every 10 iterations.  A step is one solve."""
    fr = inputs.frame(family, 0)
    n, leaf, rank = int(np.prod(fr["dims"])), fr["leaf"], fr["rank"]
    s = h.System(fr["dims"])
    h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
    b = torch.from_numpy(fr["b"]).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a = _dense_from_system(torch, s)
    ainv = torch.cholesky_inverse(torch.linalg.cholesky(a))
    xstar = ainv @ b
    G, sig, W = _svdh_torch(torch, ainv, leaf, rank)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    K = n // leaf
    ctx = h.Context(max_n=n, leaf=leaf, rank=rank)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    keep = []

    def run(fac, label):
        for _ in range(args.warmup):
            h.solve(ctx, s, fac, b, x, rtol=1e-6, info=False)
        ts = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.solve(ctx, s, fac, b, x, rtol=1e-6, info=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        info = h.solve(ctx, s, fac, b, x, rtol=1e-6, allow=(h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN, h.E_NAN))
        err = float(torch.linalg.norm(x - xstar) / torch.linalg.norm(xstar))
        out[label] = {"ms_per_solve": statistics.mean(ts), "iters": info.iters, "status": info.status,
                      "true_rel_res": info.rel_res_true, "rel_err_vs_fp64_direct": err}

    for label, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        packed = torch.cat([G.flatten(), sig.flatten(), W.flatten()]).to(dt)
        keep.append(packed)
        run(h.factors(h.PRE_SVDH, packed, n, leaf, rank), label)
    gq, gs = _fp8_blocks(torch, G)
    cq, cs = _fp8_blocks(torch, sig)
    wq, ws = _fp8_blocks(torch, W.reshape(-1, leaf, rank))
    packed8 = torch.cat([gq, cq, wq])
    sc8 = torch.cat([gs, cs, ws]).cuda()
    keep += [packed8, sc8]
    run(h.factors(h.PRE_SVDH, packed8, n, leaf, rank, sc8), "fp8e4m3")
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    run(jac, "jacobi")
    line = {"metric": f"ms/solve and iterations by apply precision, {family} (N={n}), SVD-H leaf {leaf} "
                      f"rank {rank}, rtol 1e-6", "value": out["bf16"]["ms_per_solve"], "unit": "ms/solve",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["bf16"]["ms_per_solve"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"SVD-H precision sweep: {family} seed 0, SVD-H from the dense FP64 inverse "
                                   "on the device (torch, setup outside the timing), apply FP32/BF16/FP8",
                       "l2": "flushed (256 MiB write) before every solve, outside the timing",
                       "svdh_build_seconds": build_s},
            "sweep": out}
    print(json.dumps(line), flush=True)


BARRIER_SIZES = (1024, 2048, 4096, 8192, 16384)
BARRIER_WEIGHTS = os.path.join(ROOT, "paper_2605_13343_gb300", "weights", "hmpcg_d128_l4_barriers.f32")


def bench_barriers(args, h, torch, np, inputs, emit=True, frames_per_size=20):
    """The paper's benchmark distribution (Supp. D): 2D barrier frames with zero-flux boundaries,
    face rule 2 rho_i rho_j / (rho_i + rho_j), PCG to rtol 1e-8, at N = 1024 ... 16384; the 20 test
    frames of each scale from the disjoint-seed split (seed 1) the barrier checkpoint was trained
    on.  Per size: learned-H frame (assemble + infer + solve, one CUDA graph per size) and Jacobi
    PCG frame (assemble + solve), CUDA events per frame, L2 flushed between frames.  A step is
    one frame."""
    wsrc = os.path.basename(BARRIER_WEIGHTS) if os.path.exists(BARRIER_WEIGHTS) else "seeded init"
    w = np.fromfile(BARRIER_WEIGHTS, dtype=np.float32) if os.path.exists(BARRIER_WEIGHTS) else \
        inputs.network_blob(0, **CFG)
    ctx = h.Context(max_n=max(BARRIER_SIZES), leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                    max_batch=1, weights=w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    _, test_seeds = inputs.split_seeds(1, 100, frames_per_size)
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    rows = {}
    for n in BARRIER_SIZES:
        fam = f"barriers2d_{n}"
        frs = [inputs.frame(fam, s) for s in test_seeds]
        rtol = frs[0]["rtol"]
        rho_dev = [torch.from_numpy(fr["rho"]).cuda() for fr in frs]
        b_dev = [torch.from_numpy(fr["b"]).cuda() for fr in frs]
        slot_rho = torch.empty(n, dtype=torch.float64, device="cuda")
        slot_b = torch.empty(n, dtype=torch.float64, device="cuda")
        slot = h.System(frs[0]["dims"])
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        packed = torch.empty(h.packed_width(n, 64, 16, h.PRE_LEARNED), dtype=torch.bfloat16, device="cuda")
        fac = h.factors(h.PRE_LEARNED, packed, n, 64, 16)

        def asm():
            h.assemble(slot_rho, slot, bc=h.BC_NEUMANN, face=h.FACE_RHO)

        def body_l():
            asm()
            h.infer_factors(ctx, [slot], packed)
            h.solve(ctx, slot, fac, slot_b, x, rtol=rtol, info=False)

        def body_j():
            asm()
            h.solve(ctx, slot, jac, slot_b, x, rtol=rtol, info=False)

        graphs = {}
        for name, body in (("learned", body_l), ("jacobi", body_j)):
            slot_rho.copy_(rho_dev[0]); slot_b.copy_(b_dev[0])
            body(); body()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                body()
            graphs[name] = g
        torch.cuda.synchronize()
        out = {}
        for name in ("learned", "jacobi"):
            ts, its, fails = [], [], 0
            for k in range(len(frs)):
                slot_rho.copy_(rho_dev[k]); slot_b.copy_(b_dev[k])
                flush.fill_(k & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                graphs[name].replay()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                # iterations and status of the same frame through the public calls
                f = fac if name == "learned" else jac
                if name == "learned":
                    h.infer_factors(ctx, [slot], packed)
                inf = h.solve(ctx, slot, f, slot_b, x, rtol=rtol, allow=(h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN, h.E_NAN))
                if inf.status != h.OK:
                    fails += 1
                its.append(inf.iters)
            out[name] = {"ms_per_frame": statistics.mean(ts), "ms_std": statistics.pstdev(ts),
                         "iters": statistics.mean(its), "iters_std": statistics.pstdev(its), "not_ok": fails}
        out["speedup_vs_jacobi"] = out["jacobi"]["ms_per_frame"] / out["learned"]["ms_per_frame"]
        rows[str(n)] = out
        del graphs
        torch.cuda.synchronize()
    # the paper's model size (d 128, 3 layers, 8 heads of 16, leaf 128, rank 32; seeded weights)
    # on the N = 8192 frames: inference time through the layered kernels (Table S5 reports the
    # H200's inference at this size and N)
    paper = None
    try:
        pc = dict(d=128, n_layers=3, n_heads=8, d_mlp=512, leaf=128, rank=32)
        pw = inputs.network_blob(0, **pc)
        pctx = h.Context(max_n=8192, leaf=128, rank=32, d_model=128, n_layers=3, n_heads=8, d_mlp=512,
                         max_batch=1, weights=pw)
        frs = [inputs.frame("barriers2d_8192", s_) for s_ in test_seeds[:5]]
        psys = []
        for fr in frs:
            sg = h.System(fr["dims"])
            h.assemble(torch.from_numpy(fr["rho"]).cuda(), sg, bc=h.BC_NEUMANN, face=h.FACE_RHO)
            psys.append(sg)
        ppk = torch.empty(h.packed_width(8192, 128, 32, h.PRE_LEARNED), dtype=torch.bfloat16, device="cuda")
        for sg in psys[:2]:
            h.infer_factors(pctx, [sg], ppk)
        ts = []
        for k, sg in enumerate(psys):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.infer_factors(pctx, [sg], ppk)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        paper = {"infer_ms_n8192": statistics.mean(ts), "frames": len(ts), "path": "layered kernels",
                 "config": "d128, 3 layers, 8 heads of 16, leaf 128, rank 32, seeded weights"}
        pctx.close()
    except Exception as exc:  # reported, not fatal
        paper = {"error": str(exc)[:200]}
    line = {"metric": "ms/frame to rtol 1e-8 on the paper's barrier distribution (learned-H vs Jacobi PCG)",
            "value": rows["8192"]["learned"]["ms_per_frame"], "unit": "ms/frame", "n_gpus": 1,
            "steps": frames_per_size, "warmup": 2, "ms_per_step": rows["8192"]["learned"]["ms_per_frame"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "barriers2d_N (Supp. D generator: 1-3 barriers, contrast log-uniform [5,100], "
                                   "5% jitter, zero-flux), N=1024..16384, 20 test frames each (split seed 1), "
                                   "leaf 64 rank 16 d128 4 layers, BF16 factors, rtol 1e-8",
                       "weights": wsrc, "l2": "flushed (256 MiB write) before every frame, outside the timing"},
            "sizes": rows, "paper_size_model": paper}
    ctx.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def bench_batch(args, h, torch, np, inputs, w, wsrc, emit=True):
    """64 ragged systems (N uniform over {1024 ... 16384}, 2D and 3D alternating, 1:100): learned-H
    inference per grid shape plus one hmpcg_solve_batch, captured as one CUDA graph; Jacobi batch
    beside it.  A step is one whole batch."""
    count = 64
    dims = inputs.batch_mixed_dims(7, count)
    frames = []
    for i, d in enumerate(dims):
        n = int(np.prod(d))
        frames.append(dict(dims=d, n=n, rho=inputs.density_for_dims(7000 + i, d), b=inputs.rhs(7000 + i, n)))
    groups = {}
    for i, fr in enumerate(frames):
        groups.setdefault(tuple(fr["dims"]), []).append(i)
    gmax = max(len(v) for v in groups.values())
    ctx = h.Context(max_n=16384, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                    max_batch=gmax, weights=w)
    systems, bs, xs = [], [], []
    for fr in frames:
        s = h.System(fr["dims"])
        h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
        systems.append(s)
        bs.append(torch.from_numpy(fr["b"]).cuda())
        xs.append(torch.zeros(fr["n"], dtype=torch.float64, device="cuda"))
    facs = [None] * count
    gbufs = {}
    for key, ids in groups.items():
        n = frames[ids[0]]["n"]
        P = h.packed_width(n, 64, 16, h.PRE_LEARNED)
        buf = torch.empty(len(ids) * P, dtype=torch.bfloat16, device="cuda")
        gbufs[key] = buf
        for j, i in enumerate(ids):
            facs[i] = h.factors(h.PRE_LEARNED, buf[j * P:(j + 1) * P], n, 64, 16)
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    jacs = [jac] * count

    def infer_all():
        for key, ids in groups.items():
            h.infer_factors(ctx, [systems[i] for i in ids], gbufs[key])

    infer_all()
    csz = h.autotune_batch(ctx, systems, facs, bs, xs, rtol=1e-6)
    h.autotune_batch(ctx, systems, jacs, bs, xs, rtol=1e-6)
    allow = (h.OK, h.NOT_CONVERGED, h.E_BREAKDOWN, h.E_NAN)

    def learned_body():
        infer_all()
        h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6, info=False, allow=allow, fallback=True)

    def jacobi_body():
        h.solve_batch(ctx, systems, jacs, bs, xs, rtol=1e-6, info=False, allow=allow)

    graphs = {}
    for name, fn in (("learned", learned_body), ("jacobi", jacobi_body)):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            fn()
        graphs[name] = g
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(g):
        for _ in range(args.warmup):
            g.replay()
        ts = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    clk = ClockSampler()
    clk.start()
    ms_l = timed(graphs["learned"])
    ms_j = timed(graphs["jacobi"])
    clocks = clk.stop()
    infer_all()
    inf_l = h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6, allow=allow, fallback=True)
    inf_j = h.solve_batch(ctx, systems, jacs, bs, xs, rtol=1e-6, allow=allow)
    per = [{"n": fr["n"], "dims": list(fr["dims"]), "cluster": c, "iters_learned": a.iters, "status_learned": a.status,
            "fallback": a.fallback, "iters_jacobi": j.iters, "status_jacobi": j.status}
           for fr, c, a, j in zip(frames, csz, inf_l, inf_j)]
    ok_l = sum(1 for a in inf_l if a.status == h.OK)
    line = {"metric": "solves/s, 64 ragged systems N in {1024..16384} 2D/3D 1:100, learned-H (infer + PCG) "
                      "to rtol 1e-6", "value": count / (ms_l * 1e-3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "batch of 64 (inputs.batch_mixed_dims seed 7), one CUDA graph: inference "
                                   "per grid shape + hmpcg_solve_batch (persistent cluster kernels, tuned "
                                   "cluster sizes, Jacobi fallback on breakdown)", "weights": wsrc,
                       "l2": "flushed (256 MiB write) before every batch, outside the timing"},
            "jacobi": {"solves_per_s": count / (ms_j * 1e-3), "ms_per_batch": ms_j,
                       "converged": sum(1 for j in inf_j if j.status == h.OK)},
            "learned_converged": ok_l, "jacobi_fallbacks": sum(1 for a in inf_l if a.fallback),
            "iters_mean": {"learned": statistics.mean(a.iters for a in inf_l),
                           "jacobi": statistics.mean(j.iters for j in inf_j)},
            "clocks": clocks, "systems": per}
    if not emit:
        return line
    print(json.dumps(line), flush=True)


def bench_bandwidth(args, h, torch, np, hbm_peak, peak_kind):
    """HBM roofline of the bandwidth-bound kernels at sizes larger than L2: the 7/5-point SpMV
    (algorithmic bytes 24 N in 3D, 20 N in 2D: x, y, faces, diag in FP32) and the BF16 learned
    H-apply (2 P + 12 N bytes: the packed factors once, r, z and the diagonal-stage vector).
    A step is one call; CUDA events around `steps` calls after `warmup` calls."""
    rows = bandwidth_rows(h, torch, np, hbm_peak, args.steps, args.warmup)
    top = rows[-1]
    line = {"metric": "HBM roofline fraction of SpMV and BF16 learned H-apply (algorithmic bytes / time)",
            "value": top["frac"], "unit": f"fraction of {peak_kind} HBM {hbm_peak:.0f} GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": top["us"] / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "SpMV 256^3 and 4096^2 (rho = 1), apply N = 2^20..2^22 leaf 64 rank 16 with "
                                   "random BF16 factors", "l2": "inputs larger than L2"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def bandwidth_rows(h, torch, np, hbm_peak, steps, warmup):
    """SpMV (256^3, 4096^2) and BF16 learned apply (N = 2^20..2^22) timings and HBM fractions."""
    stream = torch.cuda.current_stream()
    args = argparse.Namespace(steps=steps, warmup=warmup)

    def timeit(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    rows = []
    for dims in [(256, 256, 256), (4096, 4096)]:
        n = int(np.prod(dims))
        s = h.System(dims)
        h.assemble(torch.ones(n, dtype=torch.float64, device="cuda"), s)
        x = torch.randn(n, device="cuda")
        y = torch.empty_like(x)
        ms = timeit(lambda: h.spmv(s, x, y))
        byts = (24 if len(dims) == 3 else 20) * n
        rows.append({"kernel": "spmv", "dims": list(dims), "n": n, "us": ms * 1e3, "bytes": byts,
                     "GBps": byts / ms / 1e6, "frac": byts / ms / 1e6 / hbm_peak})
        del s, x, y
    ctx = h.Context(max_n=1 << 22, leaf=64, rank=16)
    for n in [1 << 20, 1 << 21, 1 << 22]:
        w = h.packed_width(n, 64, 16, h.PRE_LEARNED)
        pk = (torch.randn(w, device="cuda") * 0.01).to(torch.bfloat16)
        fac = h.factors(h.PRE_LEARNED, pk, n, 64, 16)
        r = torch.randn(n, device="cuda")
        z = torch.empty_like(r)
        ms = timeit(lambda: h.apply(ctx, fac, r, z))
        byts = 2 * w + 12 * n
        rows.append({"kernel": "apply_bf16_learned", "n": n, "us": ms * 1e3, "bytes": byts,
                     "GBps": byts / ms / 1e6, "frac": byts / ms / 1e6 / hbm_peak})
        del pk, r, z
    # FP8-E4M3 learned factors (one FP32 scale per block) at the largest size
    n = 1 << 22
    K = n // 64
    w = h.packed_width(n, 64, 16, h.PRE_LEARNED)
    pk8 = (torch.randn(w, device="cuda") * 64.0).clamp(-448, 448).to(torch.float8_e4m3fn)
    sc8 = torch.full((4 * K + K - 1,), 1e-3, dtype=torch.float32, device="cuda")
    fac8 = h.factors(h.PRE_LEARNED, pk8, n, 64, 16, sc8)
    r = torch.randn(n, device="cuda")
    z = torch.empty_like(r)
    ms = timeit(lambda: h.apply(ctx, fac8, r, z))
    byts = w + 4 * sc8.numel() + 12 * n
    rows.append({"kernel": "apply_fp8_learned", "n": n, "us": ms * 1e3, "bytes": byts,
                 "GBps": byts / ms / 1e6, "frac": byts / ms / 1e6 / hbm_peak})
    del pk8, sc8, r, z
    del ctx
    torch.cuda.synchronize()
    return rows


def _count_kernel_nodes(torch, fn):
    """Kernel nodes of a driver-API stream capture of fn() (None if the capture fails)."""
    import ctypes
    try:
        cu = ctypes.CDLL("libcuda.so.1")
        st = torch.cuda.Stream()
        torch.cuda.synchronize()
        h = ctypes.c_void_p(st.cuda_stream)
        if cu.cuStreamBeginCapture_v2(h, ctypes.c_int(2)) != 0:      # relaxed capture mode
            return None
        with torch.cuda.stream(st):
            fn()
        graph = ctypes.c_void_p()
        if cu.cuStreamEndCapture(h, ctypes.byref(graph)) != 0:
            return None
        n = ctypes.c_size_t(0)
        cu.cuGraphGetNodes(graph, None, ctypes.byref(n))
        nodes = (ctypes.c_void_p * n.value)()
        cu.cuGraphGetNodes(graph, nodes, ctypes.byref(n))
        kernels = 0
        for i in range(n.value):
            t = ctypes.c_int(-1)
            cu.cuGraphNodeGetType(ctypes.c_void_p(nodes[i]), ctypes.byref(t))
            kernels += 1 if t.value == 0 else 0                       # CU_GRAPH_NODE_TYPE_KERNEL
        cu.cuGraphDestroy(graph)
        torch.cuda.synchronize()
        return kernels
    except Exception as exc:  # reported, not fatal
        print(f"gpu_launches: capture failed: {exc}", file=sys.stderr)
        return None


def bench_train(args, h, torch, np, inputs, bf16_peak, peak_kind, emit=True):
    """Training step of the cosine-Hutchinson objective: 32 systems 16^3 (density ratio
    log-uniform in [1, 100]), 16 Rademacher probes each, BF16 forward, hand-written backward,
    global-norm clip, AdamW (lr 3e-4).  A step is one hmpcg_train_step."""
    B = 32
    ctx = h.Context(max_n=4096, leaf=64, rank=16, d_model=128, n_layers=4, n_heads=4, d_mlp=512,
                    max_batch=B, weights=inputs.network_blob(0, **CFG))
    pool = []
    for k in range(4 * B):
        fr = inputs.frame("spheres3d_4096_lu", k)
        sg = h.System(fr["dims"])
        h.assemble(torch.from_numpy(fr["rho"]).cuda(), sg)
        pool.append(sg)
    stream = torch.cuda.current_stream()
    batches = [pool[(i % 4) * B:(i % 4 + 1) * B] for i in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        h.train_step(ctx, batches[i], 16, 3e-4, i, want_loss=False)
    torch.cuda.synchronize()
    clk = ClockSampler()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.warmup, args.warmup + args.steps):
        h.train_step(ctx, batches[i], 16, 3e-4, i, want_loss=False)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    loss = h.train_step(ctx, batches[0], 16, 0.0, 0)
    tokens = B * 4096
    line = {"metric": "ms per training step (32 systems of N=4096, 16 probes, AdamW)", "value": ms, "unit": "ms/step",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "hmpcg_train_step on spheres3d_4096_lu (16^3, contrast log-uniform 1..100), "
                                   "batch 32, 16 Rademacher probes, d128 4 layers 4 heads MLP 512, seeded init",
                       "tokens_per_step": tokens, "l2": "working set (activations ~1 GB) larger than L2"},
            "loss_after": loss, "clocks": clocks}
    if not emit:
        return line
    print(json.dumps(line), flush=True)


def _weights_blob(path, inputs):
    """The network weights of the workload: the trained checkpoint if present, else the seeded init."""
    import numpy as np
    if path and os.path.exists(path):
        return np.fromfile(path, dtype=np.float32)
    return inputs.network_blob(0, **CFG)


def _cpu_baseline(weights):
    """Oracle (FP64, CPU) on one frame of the same workload, in a spawned process
    so that no process pool is forked after CUDA initialisation."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        return pool.apply(_cpu_baseline_worker, (weights,))


def _cpu_baseline_worker(weights, nframes=5):
    """The oracle as it stands, timed on the host cores over `nframes` frames of the headline
    workload (seeds 1000..): learned-H frame (FP64 network forward + FP64 PCG), its PCG alone,
    and Jacobi PCG on the same frames."""
    import numpy as np
    import torch
    import inputs
    from oracle import grid, hmatrix, network, pcg
    torch.set_num_threads(os.cpu_count() or 1)
    p = network.unflatten(_weights_blob(weights, inputs), inputs.network_layout(**CFG))
    t_frame, t_solve, t_jac, it_l, it_j = [], [], [], [], []
    for k in range(nframes):
        fr = inputs.frame(FAMILY, 1000 + k)
        sys_ = grid.assemble(fr["rho"], fr["dims"])
        a = grid.sparse_matrix(sys_)
        t0 = time.perf_counter()
        with torch.no_grad():
            f = network.to_numpy_factors(network.forward(p, sys_, CFG))
        t1 = time.perf_counter()
        out = pcg.pcg(lambda v: a @ v, lambda v: hmatrix.apply(f, v), fr["b"], rtol=1e-6)
        t2 = time.perf_counter()
        d = sys_["diag"]
        outj = pcg.pcg(lambda v: a @ v, lambda v: v / d, fr["b"], rtol=1e-6)
        t3 = time.perf_counter()
        t_frame.append((t2 - t0) * 1e3)
        t_solve.append((t2 - t1) * 1e3)
        t_jac.append((t3 - t2) * 1e3)
        it_l.append(out["iters"])
        it_j.append(outj["iters"])
    return {"value": statistics.mean(t_frame), "unit": "ms/frame", "cores": torch.get_num_threads(), "kind": "oracle",
            "std": statistics.pstdev(t_frame),
            "sample": f"{nframes} frames (seeds 1000..{1000 + nframes - 1}): oracle network forward (torch FP64, "
                      f"{torch.get_num_threads()} threads) + oracle PCG (numpy/scipy FP64, one thread)",
            "learned_solve_ms": statistics.mean(t_solve), "learned_iters": statistics.mean(it_l),
            "jacobi_ms": statistics.mean(t_jac), "jacobi_iters": statistics.mean(it_j)}


if __name__ == "__main__":
    main()
