"""Benchmark of the neural-bounding hot path on one GB300 (or N replicas).

Workload (3D ray queries, BF16 tensor-core inference): a union of 64 spheres
(radii 0.02-0.2) in [-1,1]^3; rays with origin uniform on the radius-2 sphere and
direction uniform on S^2; MLP 6 -> 128 x4 -> 1 (ReLU); trained with the asymmetric
BCE (FN weight ramped 1 -> 100, beta 1) for 20k Adam steps of 65,536 rays; threshold
calibrated in FP64 on a 16M-ray evaluation set (FN = 0 on it).

One timed step = nb_query over the 16M evaluation rays (BF16 tcgen05 forward, FP32 /
float-float re-check of the margin band), inputs resident in HBM (384 MB per step,
larger than L2, so no flush is needed).  value = rays/s over all ranks.
Also reported: FN / FP of the decisions, the plain FP32 single-object forward on the
same weights, training samples/s, the roofline of the forward kernel, an end-to-end
number through the public API with host buffers, and the FP64 CPU oracle.
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

WIDTHS = [6, 128, 128, 128, 128, 1]
N_SPHERES, R_LO, R_HI = 64, 0.02, 0.2
BATCH, TRAIN_STEPS = 65536, 20000
N_EVAL = 16 << 20
MARGIN = 0.05
MARGIN32 = 1e-2  # FP32 form: re-check band above its own logit error
SEED_SCENE, SEED_QUERY, SEED_INIT = 1001, 2001, 4001
# DRAM bytes (read + write) per ray of the forward kernel, from one ncu capture of
# fwd_split_kernel at 1,048,576 rays (25,459,968 bytes); None once the kernel changes
TRAFFIC_BYTES_PER_RAY = 25459968 / 1048576
METRIC = "neural-bound queries/s at 0 FN (3D rays, split-FP16 tcgen05 forward + FP32 re-check)"
WORKLOAD = "3D ray queries: 64-sphere union, MLP 6->128x4->1, tensor-core 16-bit, 16M eval rays (configs[1])"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(params, q_host, seconds=12.0):
    """FP64 oracle forward on a bounded sample, on the host cores."""
    from oracle import oracle as O
    nthreads = os.cpu_count() or 1
    n = 4096
    t0 = time.perf_counter()
    O.forward(WIDTHS, params, q_host[:n], nthreads)
    dt = time.perf_counter() - t0
    n = int(min(len(q_host), max(4096, n * seconds / max(dt, 1e-6) * 0.5)))
    t0 = time.perf_counter()
    O.forward(WIDTHS, params, q_host[:n], nthreads)
    dt = time.perf_counter() - t0
    return n / dt, nthreads, n


def reference_arm(args):
    """The oracle as it stands (FP64 forward of the same network), timed on host cores."""
    from oracle import oracle as O
    from paper_2310_06822_gb300 import inputs as I
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = I.init_params(SEED_INIT, WIDTHS)
    nthreads = os.cpu_count() or 1
    sample = 150_000
    q = I.sample_queries(I.RAY3, SEED_QUERY, sample)
    for _ in range(args.warmup):
        O.forward(WIDTHS, p, q[:4096], nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.forward(WIDTHS, p, q, nthreads)
    dt = time.perf_counter() - t0
    v = args.steps * sample / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": sample},
        "cpu_baseline": {"value": v, "unit": "queries/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"{sample} rays per step through the FP64 oracle forward"},
        "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--train-steps", type=int, default=TRAIN_STEPS)
    ap.add_argument("--n-eval", type=int, default=N_EVAL, help="evaluation rays (smaller only for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    n_eval = args.n_eval
    import torch
    import torch.distributed as dist

    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- setup (untimed)
    sc = I.make_scene(SEED_SCENE, N_SPHERES, 3, R_LO, R_HI)
    shape = nb.Shape(sc, dev)
    pool_n = 8 << 20
    pool = torch.as_tensor(I.sample_queries(I.RAY3, SEED_QUERY + 17, pool_n), device=dev)
    pool_bits = nb.label(shape, I.RAY3, pool)
    eval_q_host = I.sample_queries(I.RAY3, SEED_QUERY + 1000 * rank, n_eval)
    eval_q = torch.as_tensor(eval_q_host, device=dev)
    eval_bits, lst = nb.label(shape, I.RAY3, eval_q, stats=True)

    p0 = I.init_params(SEED_INIT, WIDTHS)
    trainer = nb.Model(WIDTHS, infer_prec="f32", train_prec="f32")
    trainer.set_params(p0)
    T = args.train_steps
    per = pool_n // BATCH
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_train0 = time.perf_counter()
    train_ms = None
    ta, tb = min(100, T - 1), min(T - 1, 300)  # steps timed with events inside training
    for t in range(T):
        j = t % per
        alpha = 1.0 + 99.0 * t / max(T - 1, 1)
        if t == ta:
            e0.record()
        trainer.train_step(pool[j * BATCH:(j + 1) * BATCH], pool_bits[j * (BATCH // 32):(j + 1) * (BATCH // 32)],
                           alpha, 1.0)
        if t == tb:
            e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / (tb - ta + 1)
    t_train = time.perf_counter() - t_train0
    params = trainer.get_params()

    model = nb.Model(WIDTHS, infer_prec="f16x3", train_prec="f32")
    model.set_params(params)
    tau = model.calibrate(eval_q, eval_bits, eps=1e-5)
    plain = nb.Model(WIDTHS, infer_prec="f32")
    plain.set_params(params)
    plain.tau = tau

    out = torch.empty(nb.n_words(n_eval), dtype=torch.int32, device=dev)
    bits, qst = model.query(eval_q, margin=MARGIN, out=out, stats=True)
    y = nb.bits_to_numpy(eval_bits, n_eval)
    dec = nb.bits_to_numpy(bits, n_eval)
    fn = int(np.sum(y & ~dec))
    fp = int(np.sum(~y & dec))
    bits32 = plain.query(eval_q, margin=MARGIN32)
    dec32 = nb.bits_to_numpy(bits32, n_eval)
    differ = int(np.sum(dec != dec32))

    # ---------------------------------------------------------------- timed region
    for _ in range(max(args.warmup, 3)):
        model.query(eval_q, margin=MARGIN, out=out)
    barrier()
    with Clocks(local) as clk:
        e0.record()
        for _ in range(args.steps):
            model.query(eval_q, margin=MARGIN, out=out)
        e1.record()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t_ = torch.tensor([ms], device=dev)
        dist.all_reduce(t_, op=dist.ReduceOp.MAX)
        ms = float(t_.item())
    value = world * n_eval / (ms / 1000.0)

    # forward kernel alone (margin 0: the re-check kernels find an empty band)
    for _ in range(2):
        model.query(eval_q, margin=0.0, out=out)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        model.query(eval_q, margin=0.0, out=out)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / args.steps

    # plain FP32 single-object form on the same weights and threshold
    e0.record()
    for _ in range(3):
        plain.query(eval_q, margin=MARGIN32, out=out)
    e1.record()
    torch.cuda.synchronize()
    f32_ms = e0.elapsed_time(e1) / 3

    # plain single-product BF16 on the same weights: margin = 4x its largest logit
    # deviation from the FP32 form on the evaluation set
    bf = nb.Model(WIDTHS, infer_prec="bf16")
    bf.set_params(params)
    bf.tau = tau
    _, zbf = bf.query(eval_q, logits=True)
    _, z32 = plain.query(eval_q, logits=True)
    bf_dev = float((zbf - z32).abs().max().item())
    bf_margin = 4 * bf_dev + 1e-3
    bbits, bst = bf.query(eval_q, margin=bf_margin, out=out, stats=True)
    bf_fn = int(np.sum(y & ~nb.bits_to_numpy(bbits, n_eval)))
    e0.record()
    for _ in range(5):
        bf.query(eval_q, margin=bf_margin, out=out)
    e1.record()
    torch.cuda.synchronize()
    bf_ms = e0.elapsed_time(e1) / 5
    _, zsp = model.query(eval_q, logits=True)
    split_dev = float((zsp - z32).abs().max().item())

    # end to end through the public API: pinned host rays -> device -> bits -> host
    host_q = torch.empty((n_eval, 6), dtype=torch.float32, pin_memory=True)
    host_q.copy_(torch.as_tensor(eval_q_host))
    host_bits = torch.empty(nb.n_words(n_eval), dtype=torch.int32, pin_memory=True)
    dq = torch.empty_like(eval_q)
    for _ in range(2):
        dq.copy_(host_q, non_blocking=True)
        model.query(dq, margin=MARGIN, out=out)
        host_bits.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 4)
    e0.record()
    for _ in range(e2e_steps):
        dq.copy_(host_q, non_blocking=True)
        model.query(dq, margin=MARGIN, out=out)
        host_bits.copy_(out, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    if rank != 0:
        if world > 1:
            dist.barrier()
        return

    pk, pk_kind = peaks()
    macs = sum(WIDTHS[i] * WIDTHS[i + 1] for i in range(len(WIDTHS) - 1))
    flops = 2.0 * macs * n_eval
    achieved = flops / (fwd_ms / 1000.0) / 1e12
    peak = float(pk.get("bf16_tflops", 1900.0))
    cpu_v, cores, cpu_n = cpu_oracle_rate(params, eval_q_host)
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x3 (split fp16, fp32 accumulate)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_eval": n_eval, "batch": BATCH, "train_steps": T, "margin": MARGIN,
                   "l2": "inputs 384 MB per step > 129 MB L2, no flush", "parallelism": f"replicas{world}"},
        "fn": fn, "fp": fp, "fp_rate": fp / n_eval, "positives": int(y.sum()), "tau": tau,
        "decisions_differing_from_fp32_form": differ,
        "band": {"flagged": qst["n_flagged"], "resolved_f32": qst["n_resolved_f32"],
                 "resolved_ff": qst["n_resolved_ff"], "unresolved": qst["n_unresolved"]},
        "fp32_plain_queries_per_s": n_eval / (f32_ms / 1000.0),
        "max_logit_dev_vs_fp32_form": {"f16x3": split_dev, "bf16": bf_dev},
        "bf16_plain": {"queries_per_s": n_eval / (bf_ms / 1000.0), "margin": bf_margin, "fn": bf_fn,
                       "flagged": bst["n_flagged"], "unresolved": bst["n_unresolved"]},
        "speedup_vs_fp32_plain": f32_ms / ms,
        "train_samples_per_s_fp32": (BATCH / (train_ms / 1000.0)) if train_ms else None,
        "train_wall_s": t_train,
        "roofline": {"kernel": "fwd_split_kernel (tcgen05, 3 products per k-step)", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC_BYTES_PER_RAY * n_eval) if TRAFFIC_BYTES_PER_RAY else None,
                     "peak_kind": f"{pk_kind} bf16 burst", "fwd_ms": fwd_ms,
                     "algorithmic_flops_per_launch": flops},
        "cpu_baseline": {"value": cpu_v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cpu_n} of the evaluation rays through the FP64 oracle forward"},
        "e2e": {"value": world * n_eval / (e2e_ms / 1000.0), "unit": "queries/s",
                "h2d_bytes_per_step": n_eval * 6 * 4, "d2h_bytes_per_step": nb.n_words(n_eval) * 4},
        "gpu_launches": args.steps * 3,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()


if __name__ == "__main__":
    main()
