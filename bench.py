"""Benchmark: paired rotated-rectangle IoU forward + backward on GB300.

Workload: the IoU-loss recipe with 1,000,000 pairs of rotated rectangles
(K = 4, FP32): target center ~ U[0,10]^2, w,h ~ U[0.5,4], theta ~ U[-pi,pi);
prediction = target + center N(0,0.5)^2, log-size N(0,0.2), angle N(0,0.2);
dL/dIoU = 1.  One step = forward (IoU, nx, xflags saved) + backward from the
saved flags, i.e. every step of the hot path.  "Plain" = the same pairs
through the plain form (FP32 only, no flags saved, backward recomputes).

Prints one JSON line (rank 0).  Options: --gpus N --steps K --warmup W
[--impl reference] [--n PAIRS] [--workload NAME] [--no-configs].  The default
line also carries, under "configs", the other workloads measured in the same
run: 4096 rectangle pairs, the 2000 x 2000 pairwise matrix, the 64-scene
ragged batch and the 4M convex pairs (each with its plain form, a parity
sample against the FP64 oracle and the oracle's own rate).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IoU pairs/s fwd+bwd, batched vs plain on one GB300, ≤1e-5 err vs FP64 oracle"
UNIT = "pairs/s"
WORKLOAD = ("paired rotated-rectangle IoU forward+backward (IoU-loss recipe), 1,000,000 pairs, K=4, FP32, "
            "flags saved in the forward and consumed by the backward")
WORKLOADS = {
    "loss1m": WORKLOAD,
    "rect4096": "paired rotated-rectangle IoU forward+backward, 4096 pairs, K=4, FP32 (L2-resident, launch-bound)",
    "convex": "paired general convex polygons (hulls of 3-8 points, counts, K=8) forward+backward, 4,000,000 pairs, "
              "5% constructed near-degenerate, FP64 refinement on",
    "pairwise2000": "pairwise IoU matrix, 2000 x 2000 bird's-eye boxes (K=4), forward, IoU + nx",
    "ragged64": "ragged batch, 64 scenes N_i in [50,3000] x M_i in [5,200] (K=4), forward, one persistent launch "
                "in a CUDA graph vs one launch per scene",
    "nms2000": "greedy rotated NMS over 2000 bird's-eye boxes (K=4), scores U[0,1), IoU threshold 0.2: visiting "
               "order, suppression bitmask, greedy pass",
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_run(d, threads):
    """One fwd+bwd pass of the FP64 oracle over the arrays in d; returns seconds."""
    import oracle

    c1, c2 = d.get("c1"), d.get("c2")
    grad = d["grad"].astype(np.float64) if "grad" in d else np.ones(d["p1"].shape[0])
    t0 = time.perf_counter()
    o = oracle.iou_paired(d["p1"], d["p2"], c1, c2, threads=threads)
    oracle.iou_backward_paired(d["p1"], d["p2"], grad, o["nx"], o["xflags"], c1, c2, threads=threads)
    return time.perf_counter() - t0


def reference_arm(args):
    """The reference arm: the FP64 oracle (plain C, all host cores) on bounded
    samples of the same workload, timed per step."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    from paper_2011_11134_gb300 import workloads as W

    threads = os.cpu_count() or 1
    sample = args.ref_sample
    d = W.loss_pairs_1m(seed=0, n=sample)
    for _ in range(args.warmup):
        cpu_oracle_run(d, threads)
    times = [cpu_oracle_run(d, threads) for _ in range(args.steps)]
    total = sum(times)
    value = sample * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_step": sample, "K": 4,
                   "note": "each step is a bounded sample of the 1M-pair workload"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"first {sample} pairs of the workload per step, fwd+bwd"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def matrix_workload(args):
    print(json.dumps(matrix_measure(args, args.workload)), flush=True)


def matrix_measure(args, workload, parity=False):
    """Forward-only matrix workloads: the 2000 x 2000 pairwise matrix, and the
    64-scene ragged batch (persistent launch in a CUDA graph; plain = one
    launch per scene).  Unit: IoU entries/s.  Returns the JSON line; with
    parity, also checks sampled rows / scenes against the FP64 oracle and times
    the oracle on them (its cpu_baseline)."""
    import torch

    import paper_2011_11134_gb300 as dg
    from paper_2011_11134_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    if workload == "pairwise2000":
        d = W.pairwise_bev_2000(seed=0)
        a, b = torch.from_numpy(d["a"]).to(dev), torch.from_numpy(d["b"]).to(dev)
        N, M = a.shape[0], b.shape[0]
        out = (torch.empty((N, M), device=dev), torch.empty((N, M), device=dev, dtype=torch.uint8))
        entries = N * M
        tuned = None
        fast = lambda: dg.dgal_iou_pairwise(a, b, out=out)
        plain = lambda: dg.dgal_iou_pairwise(a, b, out=out, flags=dg.DGAL_PLAIN)
        launches = 1
        out_bytes = 5 * entries
    elif workload == "ragged64":
        d = W.ragged_scenes_64(seed=0)
        a, b = torch.from_numpy(d["a"]).to(dev), torch.from_numpy(d["b"]).to(dev)
        ao, bo, oo = (torch.from_numpy(d[k]).to(dev) for k in ("a_off", "b_off", "out_off"))
        entries = int(d["out_off"][-1])
        tuned = dg.dgal_autotune(4)  # untimed: picks entries per tile, threads per block, blocks per SM
        g = dg.BatchedGraph(a, b, ao, bo, oo, entries)
        out = (torch.empty(entries, device=dev), torch.empty(entries, device=dev, dtype=torch.uint8))
        fast = lambda: g.launch()
        plain = lambda: dg.dgal_iou_pairwise_per_scene(a, b, d["a_off"], d["b_off"], d["out_off"], out=out,
                                                       flags=dg.DGAL_PLAIN)
        launches = 2
        out_bytes = 5 * entries
    elif workload == "nms2000":
        d = W.pairwise_bev_2000(seed=0)
        a = torch.from_numpy(d["a"]).to(dev)
        N = a.shape[0]
        scores = torch.from_numpy(np.random.default_rng(0).uniform(0, 1, N).astype(np.float32)).to(dev)
        ws = torch.empty(dg.dgal_nms_workspace_bytes(N, 4), device=dev, dtype=torch.uint8)
        entries = N * (N - 1) // 2  # pairs b > a of the visiting order
        tuned = None
        fast = lambda: dg.dgal_nms_rotated(a, scores, 0.2, workspace=ws, sync=False)
        plain = None
        launches = 3
        out_bytes = 8 * N * ((N + 63) // 64) // 2  # suppression words on and right of the diagonal
    for _ in range(args.warmup):
        fast()
        if plain:
            plain()
    torch.cuda.synchronize(dev)

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for _ in range(max(3, args.warmup)):  # untimed, right before the timed steps: clocks up after idle
            flush.fill_(0)
            fn()
        for s_ in range(args.steps):
            flush.fill_(s_ & 0xFF)
            ev[s_][0].record(stream)
            fn()
            ev[s_][1].record(stream)
        torch.cuda.synchronize(dev)
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    t_fast = timed(fast)
    clocks = sampler.stop()
    t_plain = timed(plain) if plain else None
    ms = statistics.mean(t_fast)
    value = entries / (ms * 1e-3)
    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    gbs = out_bytes / (ms * 1e-3) / 1e9
    line = {
        "metric": "IoU matrix entries/s, forward", "value": value, "unit": "entries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[workload], "entries": entries,
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "plain": {"value": entries / (statistics.mean(t_plain) * 1e-3), "unit": "entries/s",
                  "ms_per_step": statistics.mean(t_plain)} if t_plain else None,
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "traffic": None, "alg_bytes_per_entry": 5},
        "gpu_launches": launches * args.steps, "clocks": clocks,
    }
    if workload == "ragged64":
        line["config"]["autotuned"] = tuned
    if parity and workload in ("pairwise2000", "ragged64"):
        line.update(_matrix_parity(workload, d, out, entries))
    if workload == "nms2000":
        line["metric"] = "NMS pair tests/s (IoU > threshold decisions, upper triangle)"
        line["unit"] = "pairs/s"
        line["config"]["boxes"] = N
        line["config"]["kept"] = int(dg.dgal_nms_rotated(a, scores, 0.2, workspace=ws).numel())
        line["roofline"]["alg_bytes_per_entry"] = 1 / 8
        line["roofline"]["note"] = "latency-bound (one sequential greedy block); not an HBM-bound size"
    return line


def _matrix_parity(workload, d, out, entries):
    """Sampled parity of a matrix workload against the FP64 oracle (the first
    200 rows of the 2000 x 2000 matrix; 4 of the 64 scenes), and the oracle's
    rate on that sample (all host cores)."""
    import oracle

    threads = os.cpu_count() or 1
    iou = out[0].cpu().numpy().ravel()
    nx = out[1].cpu().numpy().ravel()
    t0 = time.perf_counter()
    if workload == "pairwise2000":
        rows = 200
        ref_iou, ref_nx = oracle.iou_pairwise(d["a"][:rows], d["b"], threads=threads)
        got_iou = iou[: rows * d["b"].shape[0]]
        got_nx = nx[: rows * d["b"].shape[0]]
        sample = f"first {rows} rows ({rows * d['b'].shape[0]:,} entries)"
        ref_iou, ref_nx = ref_iou.ravel(), ref_nx.ravel()
    else:
        got, gnx, ri, rn = [], [], [], []
        for s_ in (0, 21, 42, 63):
            a = d["a"][d["a_off"][s_]:d["a_off"][s_ + 1]]
            b = d["b"][d["b_off"][s_]:d["b_off"][s_ + 1]]
            r_iou, r_nx = oracle.iou_pairwise(a, b, threads=threads)
            ri.append(r_iou.ravel())
            rn.append(r_nx.ravel())
            got.append(iou[d["out_off"][s_]:d["out_off"][s_ + 1]])
            gnx.append(nx[d["out_off"][s_]:d["out_off"][s_ + 1]])
        ref_iou, ref_nx, got_iou, got_nx = map(np.concatenate, (ri, rn, got, gnx))
        sample = f"scenes 0, 21, 42, 63 ({ref_iou.size:,} entries)"
    secs = time.perf_counter() - t0
    return {"parity": {"iou_max_abs": float(np.abs(got_iou.astype(np.float64) - ref_iou).max()),
                       "nx_mismatch_entries": int((got_nx != ref_nx).sum()), "sample": sample},
            "cpu_baseline": {"value": ref_iou.size / secs, "unit": "entries/s", "cores": threads, "kind": "oracle",
                             "sample": sample + ", forward"}}


def fused_workload(args):
    """The 1M-pair IoU-loss workload through dgal_iou_loss: the loss-mode
    forward and the loss-mode backward, which also sums the partials (unit:
    pairs/s, forward + backward), with the separate calls timed beside it."""
    import torch

    import paper_2011_11134_gb300 as dg
    from paper_2011_11134_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d = W.loss_pairs_1m(seed=0, n=args.n)
    n = d["p1"].shape[0]
    p1, p2 = torch.from_numpy(d["p1"]).to(dev), torch.from_numpy(d["p2"]).to(dev)
    ws = torch.empty(dg.dgal_iou_loss_workspace_bytes(n), device=dev, dtype=torch.uint8)
    out = (torch.empty(1, device=dev), torch.empty_like(p1), torch.empty_like(p2), None)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    L = dg._lib
    lib = L.lib()
    sp = L.stream_ptr(stream)
    # direct C-ABI calls with prepared pointers: the timed region holds device
    # work, not Python argument checks
    loss_args = (L.ptr(p1), None, L.ptr(p2), None, n, 4, None, 1.0 / n, L.ptr(out[0]), None, L.ptr(out[1]),
                 L.ptr(out[2]), L.ptr(ws), ws.numel(), dg.DGAL_FP64_REFINE, sp)

    def run():
        st = lib.dgal_iou_loss(*loss_args)
        assert st == 0, dg.dgal_last_error()

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for _ in range(max(3, args.warmup)):  # untimed, right before the timed steps: clocks up after idle
        flush.fill_(0)
        run()
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        ev[s_][0].record(stream)
        run()
        ev[s_][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    # the same loss through the separate forward and backward calls
    g_iou = torch.full((n,), -1.0 / n, device=dev)
    iv = torch.empty(n, device=dev)
    nx_ = torch.empty(n, device=dev, dtype=torch.uint8)
    xf_ = torch.empty((n, 8), device=dev, dtype=torch.uint8)
    g1_, g2_ = torch.empty_like(p1), torch.empty_like(p2)
    fwd_args = (L.ptr(p1), None, L.ptr(p2), None, n, 4, L.ptr(iv), L.ptr(nx_), L.ptr(xf_), None, dg.DGAL_FP64_REFINE,
                sp)
    bwd_args = (L.ptr(p1), None, L.ptr(p2), None, n, 4, L.ptr(g_iou), L.ptr(nx_), L.ptr(xf_), L.ptr(g1_), L.ptr(g2_),
                dg.DGAL_FP64_REFINE, sp)

    def unfused():
        assert lib.dgal_iou_paired(*fwd_args) == 0
        assert lib.dgal_iou_backward(*bwd_args) == 0
        return (1.0 - iv).sum() / n

    for _ in range(args.warmup):
        unfused()
    torch.cuda.synchronize(dev)
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        ev[s_][0].record(stream)
        unfused()
        ev[s_][1].record(stream)
    torch.cuda.synchronize(dev)
    ms_unfused = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    # the GIoU and DIoU forms of the same loss (one more kernel in each pass:
    # the hull / centre / diameter terms)
    variants = {}
    for name, bit in (("giou", dg.DGAL_LOSS_GIOU), ("diou", dg.DGAL_LOSS_DIOU)):
        vargs = loss_args[:-2] + (dg.DGAL_FP64_REFINE | bit, sp)

        def vrun():
            st = lib.dgal_iou_loss(*vargs)
            assert st == 0, dg.dgal_last_error()

        for _ in range(args.warmup):
            vrun()
        torch.cuda.synchronize(dev)
        for s_ in range(args.steps):
            flush.fill_(s_ & 0xFF)
            ev[s_][0].record(stream)
            vrun()
            ev[s_][1].record(stream)
        torch.cuda.synchronize(dev)
        vms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
        variants[name] = {"value": n / (vms * 1e-3), "unit": UNIT, "ms_per_step": vms,
                          "loss": float(out[0].item()), "gpu_launches_per_step": 4}
    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    # forward: polygons 64 B + flags 9 B out; backward: polygons 64 B + flags
    # 9 B in, gradients 64 B out
    alg = 64 + 9 + 64 + 9 + 64
    gbs = alg * n / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "IoU loss (mean of 1 - IoU) and its gradient through dgal_iou_loss, 1,000,000 pairs, K=4",
                   "l2": "flushed between steps"},
        "roofline": {"bound": "hbm", "kernel": "k_paired_fwd + k_paired_bwd (loss mode)", "achieved": gbs,
                     "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "alg_bytes_per_pair": alg},
        "unfused": {"value": n / (ms_unfused * 1e-3), "unit": UNIT, "ms_per_step": ms_unfused,
                    "what": "dgal_iou_paired + torch sum + dgal_iou_backward"},
        "variants": variants,
        "gpu_launches": 2 * args.steps, "clocks": clocks,  # forward, backward (with the partial sum in its block 0)
    }
    print(json.dumps(line), flush=True)


def iou3d_workload(args):
    """1M paired rotated 3D boxes (bird's-eye-view quadrilateral + vertical
    extent): dgal_iou3d_paired + dgal_iou3d_backward per step (pairs/s,
    forward + backward), parity of a sample against the FP64 oracle."""
    import torch

    import oracle
    import paper_2011_11134_gb300 as dg
    from paper_2011_11134_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d = W.loss3d_pairs_1m(seed=0, n=args.n)
    n = d["p1"].shape[0]
    p1, p2, z1, z2 = (torch.from_numpy(d[k]).to(dev) for k in ("p1", "p2", "z1", "z2"))
    grad = torch.ones(n, device=dev)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    iou3 = torch.empty(n, device=dev)
    nx3 = torch.empty(n, device=dev, dtype=torch.uint8)
    xf3 = torch.empty((n, 8), device=dev, dtype=torch.uint8)
    g1, g2 = torch.empty_like(p1), torch.empty_like(p2)
    gz1, gz2 = torch.empty_like(z1), torch.empty_like(z2)
    state = {"f": (iou3, nx3, xf3, None), "b": (g1, gz1, g2, gz2)}
    L = dg._lib
    lib = L.lib()
    sp = L.stream_ptr(stream)
    # direct C-ABI calls with prepared pointers (device work only in the timed region)
    f_args = (L.ptr(p1), None, L.ptr(z1), L.ptr(p2), None, L.ptr(z2), n, 4, L.ptr(iou3), L.ptr(nx3), L.ptr(xf3), None,
              dg.DGAL_FP64_REFINE, sp)
    b_args = (L.ptr(p1), None, L.ptr(z1), L.ptr(p2), None, L.ptr(z2), n, 4, L.ptr(grad), L.ptr(nx3), L.ptr(xf3),
              L.ptr(g1), L.ptr(gz1), L.ptr(g2), L.ptr(gz2), dg.DGAL_FP64_REFINE, sp)

    def fwd():
        assert lib.dgal_iou3d_paired(*f_args) == 0, dg.dgal_last_error()

    def bwd():
        assert lib.dgal_iou3d_backward(*b_args) == 0, dg.dgal_last_error()

    for _ in range(args.warmup):
        fwd()
        bwd()
    torch.cuda.synchronize(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for _ in range(max(3, args.warmup)):  # untimed, right before the timed steps: clocks up after idle
        flush.fill_(0)
        fwd()
        bwd()
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        ev[s_][0].record(stream)
        fwd()
        ev[s_][1].record(stream)
        bwd()
        ev[s_][2].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    fw = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    bw = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    ms = fw + bw
    m = min(n, 20_000)
    iou = state["f"][0][:m].cpu().numpy()
    g1, gz1, g2, gz2 = (t[:m].cpu().numpy() for t in state["b"])
    sub = {k: v[:m] for k, v in d.items()}
    ref = oracle.iou3d_paired(sub["p1"], sub["p2"], sub["z1"], sub["z2"], threads=os.cpu_count() or 1)
    r1, rz1, r2, rz2 = oracle.iou3d_backward_paired(sub["p1"], sub["p2"], sub["z1"], sub["z2"], np.ones(m), ref["nx"],
                                                    ref["xflags"], threads=os.cpu_count() or 1)
    gen = ref["degen"] == 0
    G = np.concatenate([g1.reshape(m, -1), g2.reshape(m, -1), gz1, gz2], 1)[gen]
    R = np.concatenate([r1.reshape(m, -1), r2.reshape(m, -1), rz1, rz2], 1)[gen]
    grad_rel = float((np.abs(G - R).max(1) / np.maximum(np.abs(R).max(1), 1e-6)).max())
    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    alg_f, alg_b = 64 + 16 + 13, 64 + 16 + 9 + 4 + 64 + 16
    line = {
        "metric": "3D IoU pairs/s fwd+bwd", "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "paired rotated 3D boxes (bird's-eye-view quadrilateral + (z, h)), 3D IoU "
                               "forward+backward, 1,000,000 pairs, K=4, FP64 refinement on",
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "roofline": {"bound": "hbm", "kernel": "k_paired_fwd<4> (3D)" if fw >= bw else "k_paired_bwd<4> (3D)",
                     "achieved": (alg_f / fw if fw >= bw else alg_b / bw) * n / 1e-3 / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": (alg_f / fw if fw >= bw else alg_b / bw) * n / 1e-3 / 1e9 / hbm, "traffic": None,
                     "per_kernel": {"forward": {"ms": fw, "alg_bytes_per_pair": alg_f},
                                    "backward": {"ms": bw, "alg_bytes_per_pair": alg_b}}},
        "parity": {"iou_max_abs": float(np.abs(iou - ref["iou"]).max()), "grad_max_rel": grad_rel,
                   "sample_pairs": m},
        "gpu_launches": 2 * args.steps, "clocks": clocks,  # 3D forward, 3D backward
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=0, help="pairs of a paired workload (default: its own size)")
    ap.add_argument("--ref-sample", type=int, default=200_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="headline line only (skip the other configurations' measurements)")
    ap.add_argument("--launch-only", action="store_true",
                    help="paired workloads: run the batched forward + backward warmup + steps times and exit, "
                         "with no timing, oracle or host-memory pass (a short program to run under a profiler)")
    ap.add_argument("--workload", default="loss1m",
                    choices=["loss1m", "rect4096", "convex", "pairwise2000", "ragged64", "fused1m", "iou3d1m",
                             "nms2000"],
                    help="loss1m (default) is the headline line; the others measure the remaining workloads")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload in ("pairwise2000", "ragged64", "nms2000"):
        matrix_workload(args)
        return
    if args.workload == "fused1m":
        args.n = args.n or 1_000_000
        fused_workload(args)
        return
    if args.workload == "iou3d1m":
        args.n = args.n or 1_000_000
        iou3d_workload(args)
        return

    import torch
    import torch.distributed as dist

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    line = paired_measure(args, args.workload, args.n, with_e2e=True,
                          with_cpu=(not args.no_cpu_baseline and world == 1))
    if rank == 0 and not args.launch_only:
        if args.workload == "loss1m" and world == 1 and not args.no_configs and not args.n:
            line["configs"] = other_configs(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def paired_measure(args, workload, n_pairs, with_e2e, with_cpu, use_graph=False):
    """One paired workload (loss1m, rect4096 or convex): forward (saving the
    flags) + backward (reading them) timed over args.steps steps, the plain
    form timed on the same pairs, parity of a sample against the FP64 oracle,
    and optionally the host-resident call (e2e) and the oracle's own rate
    (cpu_baseline).  With use_graph (small batches) the batched step is also
    timed captured in a CUDA graph (forward + backward, replayed once per
    step) and as one dgal_iou_fwd_bwd call (dL/dIoU given up front: one
    kernel for K = 4); the line's value is the one-call form's, and the
    graph's and the eager calls' rates are kept beside it.  Returns the JSON
    line on rank 0, None on the others."""
    import torch
    import torch.distributed as dist

    import paper_2011_11134_gb300 as dg
    from paper_2011_11134_gb300 import workloads as W
    from paper_2011_11134_gb300.replicas import max_over_ranks, replica_seed

    rank, world, local = _dist_env()
    dev = torch.device("cuda", local)
    seed = replica_seed(rank)  # weak scaling: every replica runs its own seeded workload
    if workload == "rect4096":
        d = W.paired_rect_4096(seed=seed)
    elif workload == "convex":
        d = W.convex_pairs_4m(seed=seed, n=n_pairs or 4_000_000)
    else:
        d = W.loss_pairs_1m(seed=seed, n=n_pairs or 1_000_000)
    n = d["p1"].shape[0]
    K = d["p1"].shape[1]
    workload_name = WORKLOADS[workload]
    if n_pairs and workload in ("loss1m", "convex"):
        workload_name += f" (resized by --n to {n:,} pairs)"
    p1 = torch.from_numpy(d["p1"]).to(dev)
    p2 = torch.from_numpy(d["p2"]).to(dev)
    c1 = torch.from_numpy(d["c1"]).to(dev) if "c1" in d else None
    c2 = torch.from_numpy(d["c2"]).to(dev) if "c2" in d else None
    grad = torch.ones(n, device=dev)
    iou = torch.empty(n, device=dev)
    nx = torch.empty(n, device=dev, dtype=torch.uint8)
    xf = torch.empty((n, 2 * K), device=dev, dtype=torch.uint8)
    g1 = torch.empty_like(p1)
    g2 = torch.empty_like(p2)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)
    stream = torch.cuda.current_stream(dev)
    L = dg._lib
    lib = L.lib()
    sp = L.stream_ptr(stream)
    FLAGS = dg.DGAL_FP64_REFINE

    def fwd(s=None):
        st = lib.dgal_iou_paired(L.ptr(p1), L.ptr(c1), L.ptr(p2), L.ptr(c2), n, K, L.ptr(iou), L.ptr(nx), L.ptr(xf), None,
                                 FLAGS, s or sp)
        assert st == 0, dg.dgal_last_error()

    def bwd(s=None):
        st = lib.dgal_iou_backward(L.ptr(p1), L.ptr(c1), L.ptr(p2), L.ptr(c2), n, K, L.ptr(grad), L.ptr(nx), L.ptr(xf),
                                   L.ptr(g1), L.ptr(g2), FLAGS, s or sp)
        assert st == 0, dg.dgal_last_error()

    def fwd_plain():
        st = lib.dgal_iou_paired(L.ptr(p1), L.ptr(c1), L.ptr(p2), L.ptr(c2), n, K, L.ptr(iou), None, None, None,
                                 dg.DGAL_PLAIN, sp)
        assert st == 0, dg.dgal_last_error()

    def bwd_plain():
        st = lib.dgal_iou_backward(L.ptr(p1), L.ptr(c1), L.ptr(p2), L.ptr(c2), n, K, L.ptr(grad), None, None, L.ptr(g1),
                                   L.ptr(g2), dg.DGAL_PLAIN, sp)
        assert st == 0, dg.dgal_last_error()

    def timed(steps, f, b):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for _ in range(max(3, args.warmup)):  # untimed, right before the timed steps: clocks up after idle
            flush.fill_(0)
            f()
            b()
        for s in range(steps):
            flush.fill_(s & 0xFF)  # evict the inputs from L2 between steps (outside the timed events)
            ev[s][0].record(stream)
            f()
            ev[s][1].record(stream)
            b()
            ev[s][2].record(stream)
        torch.cuda.synchronize(dev)
        fw = [ev[s][0].elapsed_time(ev[s][1]) for s in range(steps)]
        bw = [ev[s][1].elapsed_time(ev[s][2]) for s in range(steps)]
        return fw, bw

    if args.launch_only:
        for _ in range(args.warmup + args.steps):
            fwd()
            bwd()
        torch.cuda.synchronize(dev)
        assert dg.dgal_get_device_status() == 0
        return None

    # warm-up (untimed)
    for _ in range(args.warmup):
        fwd()
        bwd()
        fwd_plain()
        bwd_plain()
    torch.cuda.synchronize(dev)

    graph = None
    if use_graph:
        # the batched forward + backward captured once, on a side stream
        cs = torch.cuda.Stream(dev)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            csp = L.stream_ptr(cs)
            fwd(csp)
            bwd(csp)
            torch.cuda.synchronize(dev)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=cs):
                fwd(csp)
                bwd(csp)
        stream.wait_stream(cs)
        torch.cuda.synchronize(dev)

    def onecall():
        st = lib.dgal_iou_fwd_bwd(L.ptr(p1), L.ptr(c1), L.ptr(p2), L.ptr(c2), L.ptr(grad), n, K, L.ptr(iou), L.ptr(g1),
                                  L.ptr(g2), L.ptr(nx), L.ptr(xf), FLAGS, sp)
        assert st == 0, dg.dgal_last_error()

    def timed_one(steps, f):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        for _ in range(max(3, args.warmup)):
            flush.fill_(0)
            f()
        for s in range(steps):
            flush.fill_(s & 0xFF)
            ev[s][0].record(stream)
            f()
            ev[s][1].record(stream)
        torch.cuda.synchronize(dev)
        return [ev[s][0].elapsed_time(ev[s][1]) for s in range(steps)]

    def timed_graph(steps):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        for _ in range(max(3, args.warmup)):
            flush.fill_(0)
            graph.replay()
        for s in range(steps):
            flush.fill_(s & 0xFF)
            ev[s][0].record(stream)
            graph.replay()
            ev[s][1].record(stream)
        torch.cuda.synchronize(dev)
        return [ev[s][0].elapsed_time(ev[s][1]) for s in range(steps)]

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    # per-kernel durations (an event between the two kernels, which also keeps
    # the backward from starting during the forward's last wave), then the
    # steps themselves with events around each step only
    fw, bw = timed(args.steps, fwd, bwd)

    def step():
        fwd()
        bwd()

    ssteps = timed_one(args.steps, step)
    gsteps = timed_graph(args.steps) if graph is not None else None
    osteps = timed_one(args.steps, onecall) if graph is not None else None  # last: parity reads its outputs
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    eager_ms = max_over_ranks(sum(ssteps), dev)
    eager_value = n * world * args.steps / (eager_ms / 1e3)
    graph_ms = max_over_ranks(sum(gsteps), dev) if gsteps is not None else None
    total_ms = max_over_ranks(sum(osteps), dev) if osteps is not None else eager_ms
    value = n * world * args.steps / (total_ms / 1e3)

    # parity of the timed outputs on a sample (FP64 oracle): 20,000 random
    # pairs, plus 2,000 constructed near-degenerate ones where the workload has them
    err = None
    if rank == 0:
        import oracle

        rng = np.random.Generator(np.random.PCG64(7))
        idx = rng.choice(n, size=min(n, 20000), replace=False)
        if "kind" in d and (d["kind"] > 0).any():
            deg = np.flatnonzero(d["kind"] > 0)
            idx = np.union1d(idx, rng.choice(deg, size=min(2000, deg.size), replace=False))
        idx.sort()
        sc1 = d["c1"][idx] if "c1" in d else None
        sc2 = d["c2"][idx] if "c2" in d else None
        ref = oracle.iou_paired(d["p1"][idx], d["p2"][idx], sc1, sc2, threads=os.cpu_count() or 1)
        r1, r2 = oracle.iou_backward_paired(d["p1"][idx], d["p2"][idx], np.ones(len(idx)), ref["nx"],
                                            ref["xflags"], sc1, sc2, threads=os.cpu_count() or 1)
        gi = iou.cpu().numpy()[idx].astype(np.float64)
        G = np.concatenate([g1.cpu().numpy()[idx], g2.cpu().numpy()[idx]], 1).astype(np.float64)
        R = np.concatenate([r1, r2], 1)
        gen = ref["degen"] == 0
        rel = np.abs(G - R).max(axis=(1, 2)) / np.maximum(np.abs(R).max(axis=(1, 2)), 1e-6)
        flags_ok = bool(((xf.cpu().numpy()[idx] == ref["xflags"]).all(1) | ~gen).all())
        err = {"iou_max_abs": float(np.abs(gi - ref["iou"]).max()), "grad_max_rel": float(rel[gen].max()),
               "xflags_bit_exact_generic": flags_ok, "sample_pairs": int(len(idx))}
        if "kind" in d:
            kd = d["kind"][idx] > 0
            ie = np.abs(gi - ref["iou"])
            err["iou_max_abs_constructed_degenerate"] = float(ie[kd].max()) if kd.any() else None
            err["iou_max_abs_other"] = float(ie[~kd].max())
            err["grad_max_rel_generic"] = float(rel[gen].max())
            err["constructed_degenerate_in_sample"] = int(kd.sum())

    # plain form on the same pairs, timed like the steps
    def plain_step():
        fwd_plain()
        bwd_plain()

    plain_ms = sum(timed_one(args.steps, plain_step))
    plain_value = n * world * args.steps / (plain_ms / 1e3)

    e2e = _paired_e2e(args, dg, d, n, K, world, dev, stream) if with_e2e else None
    if rank != 0:
        return None

    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    fw_ms, bw_ms = statistics.mean(fw), statistics.mean(bw)
    cb = 2 if c1 is not None else 0  # count bytes read per pair
    fwd_bytes = 2 * 8 * K + cb + 4 + 1 + 2 * K
    bwd_bytes = 2 * 8 * K + cb + 4 + 1 + 2 * K + 2 * 8 * K
    fw_gbs = fwd_bytes * n / (fw_ms * 1e-3) / 1e9
    bw_gbs = bwd_bytes * n / (bw_ms * 1e-3) / 1e9
    dom = "forward" if fw_ms >= bw_ms else "backward"
    ach = fw_gbs if dom == "forward" else bw_gbs
    # DRAM bytes per pair (dram__bytes_read.sum + dram__bytes_write.sum) of the
    # K = 4 forward and backward from one ncu capture of 4,000,000 IoU-loss
    # pairs (the current kernels), scaled to this launch by its pairs
    traffic = None
    if K == 4 and c1 is None and workload == "loss1m":
        traffic = (DRAM_BYTES_PER_PAIR_K4["forward" if dom == "forward" else "backward"]) * n
    roofline = {"bound": "hbm", "kernel": f"k_paired_{'fwd' if dom == 'forward' else 'bwd'}<{K}>", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
                "traffic_source": ("ncu DRAM bytes per pair of a 4M-pair capture of the same kernel, x pairs per "
                                   "launch") if traffic else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "per_kernel": {"forward": {"ms": fw_ms, "alg_bytes_per_pair": fwd_bytes, "GB_s": fw_gbs},
                               "backward": {"ms": bw_ms, "alg_bytes_per_pair": bwd_bytes, "GB_s": bw_gbs},
                               "timing": "CUDA events before, between and after the two kernels of each step, in a "
                                         "pass of its own; the step time comes from events around each step only"},
                "step": {"ms": total_ms / args.steps, "alg_bytes_per_pair": fwd_bytes + bwd_bytes,
                         "frac": (fwd_bytes + bwd_bytes) * n / (total_ms / args.steps * 1e-3) / 1e9 / hbm}}
    if K == 8:
        # 2.7 kflop per pair (an FP32 operation count of the clip: 64 crossings and 128
        # orientations forward, the shape derivative backward) against the derived FP32 peak
        roofline["fp32"] = {"achieved_tflops": 2.7e3 * n / (total_ms / args.steps * 1e-3) / 1e12,
                            "peak_tflops": FP32_PEAK_TFLOPS,
                            "frac": 2.7e3 * n / (total_ms / args.steps * 1e-3) / 1e12 / FP32_PEAK_TFLOPS}
    cpu = None
    if with_cpu:
        threads = os.cpu_count() or 1
        if "kind" in d:
            # every constructed near-degenerate pair of the first 2M, plus the first 100,000 pairs
            deg = np.flatnonzero(d["kind"][: min(n, 2_000_000)] > 0)
            sidx = np.union1d(np.arange(min(n, 100_000)), deg)
            ds = {k: v[sidx] for k, v in d.items()}
            desc = f"{sidx.size:,} pairs: the first 100,000 and all {deg.size:,} constructed near-degenerate " \
                   f"pairs of the first 2M, fwd+bwd, FP64 C oracle on all host cores"
        else:
            sample = min(n, args.ref_sample)
            ds = {k: v[:sample] for k, v in d.items()}
            desc = f"first {sample} pairs of the workload, fwd+bwd, FP64 C oracle on all host cores"
        m = ds["p1"].shape[0]
        cpu_oracle_run(ds, threads)
        secs = cpu_oracle_run(ds, threads)
        one = min(m, 20_000)  # single-thread rate on a smaller sample (about a second)
        secs1 = cpu_oracle_run({k: v[:one] for k, v in ds.items()}, 1)
        cpu = {"value": m / secs, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "single_thread": {"value": one / secs1, "unit": UNIT, "cores": 1, "sample": f"first {one} pairs"}}
    launches = 3 if K == 8 else 2  # K = 8: forward, its hard-pair finish, backward
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name, "pairs_per_gpu": n, "K": K,
                   "parallelism": f"replicas x{world}",
                   "l2": f"flushed between steps (256 MiB write outside the timed events); inputs {2 * n * 8 * K / 1e6:.0f} MB"},
        "plain": {"value": plain_value, "unit": UNIT, "ms_per_step": plain_ms / args.steps,
                  "form": "FP32 only, no saved flags, backward recomputes the clip",
                  "batched_over_plain": value / plain_value},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,  # forward (saves the flags), backward (reads them)
        "clocks": clocks,
        "parity": err,
    }
    if graph is not None:
        graph_value = n * world * args.steps / (graph_ms / 1e3)
        line["form"] = ("one dgal_iou_fwd_bwd call per step (dL/dIoU = 1 given up front): forward and backward in one "
                        "kernel, the clip state kept in registers between them")
        line["graph"] = {"value": graph_value, "unit": UNIT, "ms_per_step": graph_ms / args.steps,
                         "form": "dgal_iou_paired (flags saved) + dgal_iou_backward (flags read) captured in one CUDA "
                                 "graph, replayed once per step"}
        line["eager"] = {"value": eager_value, "unit": UNIT, "ms_per_step": eager_ms / args.steps,
                         "form": "the same two calls launched eagerly"}
        line["gpu_launches"] = args.steps  # the one-call form: one kernel per step
        line["plain"]["batched_over_plain"] = value / plain_value
        line["plain"]["graph_over_plain"] = graph_value / plain_value
        line["plain"]["eager_over_plain"] = eager_value / plain_value
    return line


# DRAM bytes per pair of the K = 4 paired kernels (forward saving the flags,
# backward reading them), measured by ncu on 4,000,000 IoU-loss pairs
DRAM_BYTES_PER_PAIR_K4 = {"forward": 74.03, "backward": 130.75}

# FP32 non-tensor peak of GB300, derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _paired_e2e(args, dg, d, n, K, world, dev, stream):
    """End to end through the C ABI on pinned host buffers:
    dgal_iou_fwd_bwd_host reads the polygons (and counts) and dL/dIoU from
    host memory and writes IoU and the gradients back, all inside the timed
    region: K = 4 in its direct form (one kernel on the pinned buffers in
    place), K = 8 staged (chunks copied in and out, overlapping the kernels)."""
    import torch

    L = dg._lib
    lib = L.lib()
    sp = L.stream_ptr(stream)
    h_p1 = torch.from_numpy(d["p1"]).pin_memory()
    h_p2 = torch.from_numpy(d["p2"]).pin_memory()
    h_c1 = torch.from_numpy(d["c1"]).pin_memory() if "c1" in d else None
    h_c2 = torch.from_numpy(d["c2"]).pin_memory() if "c2" in d else None
    h_grad = torch.ones(n).pin_memory()
    h_iou = torch.empty(n).pin_memory()
    h_g1 = torch.empty((n, K, 2)).pin_memory()
    h_g2 = torch.empty((n, K, 2)).pin_memory()
    chunk = 262144
    direct = K == 4  # every buffer is pinned
    ws_e2e = None
    if not direct:
        ws_e2e = torch.empty(dg.dgal_iou_host_workspace_bytes(chunk, K) + 256, device=dev, dtype=torch.uint8)
        ws_e2e = ws_e2e[(-ws_e2e.data_ptr()) % 256:]
    host_args = (L.ptr(h_p1), L.ptr(h_c1), L.ptr(h_p2), L.ptr(h_c2), L.ptr(h_grad), n, K, L.ptr(h_iou), L.ptr(h_g1),
                 L.ptr(h_g2), L.ptr(ws_e2e), ws_e2e.numel() if ws_e2e is not None else 0, chunk,
                 dg.DGAL_FP64_REFINE, sp)

    def e2e_step():
        assert lib.dgal_iou_fwd_bwd_host(*host_args) == 0, dg.dgal_last_error()

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    h2d = 2 * n * 8 * K + 4 * n + (2 * n if h_c1 is not None else 0)
    d2h = 4 * n + 2 * n * 8 * K
    return {"value": n * world * args.steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "path": "dgal_iou_fwd_bwd_host on pinned host buffers, " + (
                "direct form: one kernel reads and writes them in place over the host link" if direct else
                f"staged form: {chunk}-pair chunks copied in and out, overlapping the kernels")}


def _summary(line, keys=("value", "unit", "ms_per_step", "plain", "roofline", "parity", "cpu_baseline", "clocks",
                         "gpu_launches")):
    out = {"workload": line["config"]["workload"]}
    out.update({k: line.get(k) for k in keys})
    if isinstance(out.get("roofline"), dict):
        out["roofline"] = {k: v for k, v in out["roofline"].items() if k != "per_kernel"} | {
            "per_kernel": line["roofline"].get("per_kernel")}
    return out


def other_configs(args):
    """The configurations other than the headline, measured in the same run
    (each with its own timing, plain form, parity sample and oracle rate):
    1 the 4096 rotated-rectangle pairs, 2 the 2000 x 2000 pairwise matrix,
    3 the 64-scene ragged batch in a CUDA graph, 5 the 4M convex pairs with 5%
    constructed near-degenerate ones."""
    import paper_2011_11134_gb300 as dg

    out = {}
    dg.dgal_autotune(4, config_class=1)  # the paired launch shape (untimed)
    c1 = paired_measure(args, "rect4096", 0, with_e2e=False, with_cpu=True, use_graph=True)
    c1["roofline"]["note"] = "0.9 MB per step stays in L2: launch/latency-bound, the HBM fraction is not meaningful"
    c1["config"]["paired_shape"] = dg.dgal_get_paired_config(4)
    out["1_rect4096_fwd_bwd"] = _summary(c1) | {"paired_shape": c1["config"]["paired_shape"], "form": c1["form"],
                                                "graph": c1["graph"], "eager": c1["eager"]}
    out["2_pairwise2000_fwd"] = _summary(matrix_measure(args, "pairwise2000", parity=True))
    out["3_ragged64_fwd_graph"] = _summary(matrix_measure(args, "ragged64", parity=True))
    c5 = paired_measure(args, "convex", 0, with_e2e=False, with_cpu=True)
    out["5_convex4m_fwd_bwd"] = _summary(c5)
    return out


if __name__ == "__main__":
    main()
