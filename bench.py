"""Benchmark of the neural-bounding hot path on one GB300 (or N replicas).

Default workload (configuration of the headline metric): 3D ray queries against a union
of 64 spheres (radii 0.02-0.2) in [-1,1]^3; rays with origin uniform on the radius-2
sphere and direction uniform on S^2; MLP 6 -> 128 x4 -> 1 (ReLU); 20k BF16 tensor-core
training steps, each on a fresh batch of 65,536 rays sampled and labelled on the GPU, with
the asymmetric BCE (FN weight ramped 1 -> 100, beta 1);
threshold calibrated in FP64 on the 16M-ray evaluation set (FN = 0 on it).
One timed step = nb_query over the 16M evaluation rays (split-FP16 tcgen05 forward,
FP32 / extended-precision re-check of the margin band), inputs resident in HBM (384 MB
per step, more than the 129 MB L2, so no flush is needed); value = rays/s over all ranks.

Other configurations (--config): c1 (2D points, plain FP32), c3 (3D boxes and planes,
256 spheres, 256-wide networks, 20k BF16 training steps, FP8 E4M3 inference), c2e (3D points behind the neural
early-out of Sec. 3.3), c4 (256 objects of moving
spheres, 4D points, grouped training under a CUDA graph and grouped queries), c5 (1024
objects, 64M world rays through the learned-culler cascade, against box + exact).
Every line also carries the FP64 oracle timed on the host cores, an end-to-end figure
through the public API with host buffers, the SM clocks seen during the timed region
and, where it applies, the roofline of the dominant kernel.
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

# 3D rays (default)
WIDTHS = [6, 128, 128, 128, 128, 1]
N_SPHERES, R_LO, R_HI = 64, 0.02, 0.2
BATCH, TRAIN_STEPS = 65536, 20000
N_EVAL = 16 << 20
MARGIN = 0.05
MARGIN32 = 1e-2  # FP32 form: re-check band above its own logit error
# margins of the low-precision forms are measured on a calibration sample of other queries
# (this many, from stream SEED_CAL + kind), never on the evaluation queries they certify
CAL_N, SEED_CAL = 4 << 20, 2101
SEED_SCENE, SEED_QUERY, SEED_INIT, SEED_TRAIN = 1001, 2001, 4001, 2018
# DRAM bytes (read + write) per ray of the forward kernel, from one ncu capture of
# fwd_split_kernel at 1,048,576 rays (25,464,832 bytes); None once the kernel changes
TRAFFIC_BYTES_PER_RAY = 25464832 / 1048576
# the same for fwd_fp8_kernel at 1,048,576 boxes (25,698,816 bytes: 24 B per box and the
# weight image once per capture; scaled by boxes it slightly overcounts the image)
TRAFFIC_BYTES_PER_BOX = 25698816 / 1048576
METRIC = "neural-bound queries/s at 0 FN (3D rays, split-FP16 tcgen05 forward + FP32 re-check)"
WORKLOAD = "3D ray queries: 64-sphere union, MLP 6->128x4->1, tensor-core 16-bit, 16M eval rays"


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


def cpu_oracle_rate(widths, params, q_host, seconds=12.0):
    """FP64 oracle forward on a bounded sample, on the host cores."""
    from oracle import oracle as O
    nthreads = os.cpu_count() or 1
    n = 4096
    t0 = time.perf_counter()
    O.forward(widths, params, q_host[:n], nthreads)
    dt = time.perf_counter() - t0
    n = int(min(len(q_host), max(4096, n * seconds / max(dt, 1e-6) * 0.5)))
    t0 = time.perf_counter()
    O.forward(widths, params, q_host[:n], nthreads)
    dt = time.perf_counter() - t0
    return n / dt, nthreads, n


def cpu_oracle_label_rate(kind, q_host, scene, seconds=4.0):
    """The oracle's exact labeller on a bounded sample, on the host cores."""
    from oracle import oracle as O
    nthreads = os.cpu_count() or 1
    n = 4096
    t0 = time.perf_counter()
    O.label(kind, q_host[:n], scene, nthreads)
    dt = time.perf_counter() - t0
    n = int(min(len(q_host), max(4096, n * seconds / max(dt, 1e-6) * 0.5)))
    t0 = time.perf_counter()
    O.label(kind, q_host[:n], scene, nthreads)
    return n / (time.perf_counter() - t0), n


def rank_seed(seed: int, rank: int) -> int:
    """Each replica evaluates its own queries: rank r draws the stream seed + 1000 r."""
    return seed + 1000 * rank


def max_over_ranks(ms: float, dist, world: int, device="cpu") -> float:
    """The job's time is the slowest replica's (all-reduce MAX; identity on one rank)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units of every replica over the slowest replica's time."""
    return world * units_per_rank / (ms / 1000.0)


class Ctx:
    """Device, ranks, CUDA events and the JSON line common to every configuration."""

    def __init__(self, args):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.args = args
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(self.local)
        if self.world > 1:
            dist.init_process_group("nccl")
        self.dev = torch.device("cuda", self.local)
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()
        self.torch.cuda.synchronize()

    def time_ms(self, fn, reps):
        self.torch.cuda.synchronize()
        self.e0.record()
        for _ in range(reps):
            fn()
        self.e1.record()
        self.torch.cuda.synchronize()
        return self.e0.elapsed_time(self.e1) / reps

    def timed(self, fn, steps, warmup):
        """W warm-up steps, then K steps between barriers; max over ranks."""
        for _ in range(max(warmup, 3)):
            fn()
        self.barrier()
        with Clocks(self.local) as clk:
            self.e0.record()
            for _ in range(steps):
                fn()
            self.e1.record()
            self.barrier()
        ms = max_over_ranks(self.e0.elapsed_time(self.e1) / steps, self.dist, self.world, self.dev)
        return ms, clk.summary()

    def emit(self, line):
        if self.rank == 0:
            print(json.dumps(line), flush=True)
        if self.world > 1:
            self.dist.barrier()


def base_line(ctx, metric, value, unit, ms, steps, warmup, dtype, config, clocks, launches):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": ctx.world, "steps": steps,
            "warmup": max(warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config, "gpu_launches": launches,
            "clocks": clocks}


# ---------------------------------------------------------------------------------- 3D rays
def run_c2(args):
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    n_eval = args.n_eval
    sc = I.make_scene(SEED_SCENE, N_SPHERES, 3, R_LO, R_HI)
    shape = nb.Shape(sc, dev)
    eval_q_host = I.sample_queries(I.RAY3, rank_seed(SEED_QUERY, ctx.rank), n_eval)
    eval_q = torch.as_tensor(eval_q_host, device=dev)
    eval_bits = nb.label(shape, I.RAY3, eval_q)
    # the sampler and the exact labeller over the evaluation set on their own (steps a2, a3)
    label_ms = ctx.time_ms(lambda: nb.label(shape, I.RAY3, eval_q, out=eval_bits), 5)
    sample_buf = torch.empty_like(eval_q)
    nb.sample(I.RAY3, n_eval, SEED_TRAIN, out=sample_buf)
    sample_ms = ctx.time_ms(lambda: nb.sample(I.RAY3, n_eval, SEED_TRAIN, out=sample_buf), 5)
    del sample_buf

    # training on the tensor cores (BF16 operands, FP32 accumulation, FP32 master weights),
    # a fresh batch every iteration as in Alg. 1: sampled and labelled on the GPU
    T = args.train_steps
    trainer = nb.Model(WIDTHS, infer_prec="f32", train_prec="bf16")
    trainer.set_params(I.init_params(SEED_INIT, WIDTHS))
    qb = torch.empty((BATCH, 6), dtype=torch.float32, device=dev)
    yb = torch.empty(nb.n_words(BATCH), dtype=torch.int32, device=dev)

    def fresh(t, model_, alpha):
        nb.sample(I.RAY3, BATCH, SEED_TRAIN, first=t * BATCH, out=qb)
        nb.label(shape, I.RAY3, qb, out=yb)
        model_.train_step(qb, yb, alpha, 1.0)

    t_train0 = time.perf_counter()
    ta, tb = min(100, T - 1), min(T - 1, 600)
    for t in range(T):
        if t == ta:
            ctx.e0.record()
        fresh(t, trainer, 1.0 + 99.0 * t / max(T - 1, 1))
        if t == tb:
            ctx.e1.record()
    torch.cuda.synchronize()
    loop_ms = ctx.e0.elapsed_time(ctx.e1) / (tb - ta + 1)
    t_train = time.perf_counter() - t_train0
    params = trainer.get_params()
    # the training step alone (BF16 tensor cores), and the plain FP32 step, on one batch
    bft = nb.Model(WIDTHS, infer_prec="f32", train_prec="bf16")
    bft.set_params(params)
    bf16_step_ms = ctx.time_ms(lambda: bft.train_step(qb, yb, 50.0), 50)
    f32t = nb.Model(WIDTHS)
    f32t.set_params(params)
    f32_step_ms = ctx.time_ms(lambda: f32t.train_step(qb, yb, 50.0), 20)
    del bft, f32t

    model = nb.Model(WIDTHS, infer_prec="f16x3")
    model.set_params(params)
    tau = model.calibrate(eval_q, eval_bits, eps=1e-5)
    plain = nb.Model(WIDTHS, infer_prec="f32")
    plain.set_params(params)
    plain.tau = tau

    out = torch.empty(nb.n_words(n_eval), dtype=torch.int32, device=dev)
    bits, qst = model.query(eval_q, margin=MARGIN, out=out, stats=True)
    y = nb.bits_to_numpy(eval_bits, n_eval)
    dec = nb.bits_to_numpy(bits, n_eval)
    fn, fp = int(np.sum(y & ~dec)), int(np.sum(~y & dec))
    dec32 = nb.bits_to_numpy(plain.query(eval_q, margin=MARGIN32), n_eval)
    differ = int(np.sum(dec != dec32))

    ms, clocks = ctx.timed(lambda: model.query(eval_q, margin=MARGIN, out=out), args.steps, args.warmup)
    value = job_value(n_eval, ctx.world, ms)
    fwd_ms = ctx.time_ms(lambda: model.query(eval_q, margin=0.0, out=out), args.steps)
    f32_ms = ctx.time_ms(lambda: plain.query(eval_q, margin=MARGIN32, out=out), 3)

    # plain single-product BF16 on the same weights: margin = 4x its largest logit
    # deviation from the FP32 form, measured on a calibration sample of other rays (so the
    # decisions on the evaluation rays check the margin on queries it was not fitted to)
    cal_q = nb.sample(I.RAY3, CAL_N, rank_seed(SEED_CAL, ctx.rank), device=dev)
    bf = nb.Model(WIDTHS, infer_prec="bf16")
    bf.set_params(params)
    bf.tau = tau
    _, zbf = bf.query(cal_q, logits=True)
    _, z32c = plain.query(cal_q, logits=True)
    bf_dev = float((zbf - z32c).abs().max().item())
    _, zspc = model.query(cal_q, logits=True)
    split_dev_cal = float((zspc - z32c).abs().max().item())
    del zbf, zspc, z32c
    bf_margin = 4 * bf_dev + 1e-3
    bbits, bst = bf.query(eval_q, margin=bf_margin, out=out, stats=True)
    bdec = nb.bits_to_numpy(bbits, n_eval)
    bf_fn = int(np.sum(y & ~bdec))
    bf_differ = int(np.sum(bdec != dec32))
    bf_ms = ctx.time_ms(lambda: bf.query(eval_q, margin=bf_margin, out=out), 5)
    _, zsp = model.query(eval_q, logits=True)
    _, z32 = plain.query(eval_q, logits=True)
    split_dev = float((zsp - z32).abs().max().item())
    del zsp, z32

    # end to end through the public API: pinned host rays in, bits back in host memory
    # (nb_query_host: the forward reads the rays in place over NVLink-C2C; for comparison
    # the staged form, 4M-ray chunks copied in on a second stream while the previous runs)
    host_q = torch.empty((n_eval, 6), dtype=torch.float32, pin_memory=True)
    host_q.copy_(torch.as_tensor(eval_q_host))
    host_bits = torch.empty(nb.n_words(n_eval), dtype=torch.int32, pin_memory=True)

    def e2e_step():
        model.query_host(host_q, margin=MARGIN, out=host_bits)

    for _ in range(3):
        e2e_step()
    e2e_ms = ctx.time_ms(e2e_step, max(5, args.steps // 4))
    e2e_equal = bool(np.array_equal(nb.bits_to_numpy(host_bits, n_eval), nb.bits_to_numpy(model.query(eval_q, margin=MARGIN), n_eval)))
    staged_ms = ctx.time_ms(lambda: model.query_host(host_q, margin=MARGIN, out=host_bits, chunk_rows=1 << 22),
                            max(5, args.steps // 4))

    if ctx.rank != 0:
        return ctx.emit(None)
    pk, pk_kind = peaks()
    macs = sum(WIDTHS[i] * WIDTHS[i + 1] for i in range(len(WIDTHS) - 1))
    flops = 2.0 * macs * n_eval
    achieved = flops / (fwd_ms / 1000.0) / 1e12
    peak = float(pk.get("bf16_tflops", 1900.0))
    cpu_v, cores, cpu_n = cpu_oracle_rate(WIDTHS, params, eval_q_host)
    cpu_label_v, cpu_label_n = cpu_oracle_label_rate(I.RAY3, eval_q_host, sc)
    line = base_line(ctx, METRIC, value, "queries/s", ms, args.steps, args.warmup,
                     "f16x3 (split fp16 operands, fp32 accumulate)",
                     {"workload": WORKLOAD, "n_eval": n_eval, "batch": BATCH, "train_steps": T, "margin": MARGIN,
                      "l2": "inputs 384 MB per step > 129 MB L2, no flush", "parallelism": f"replicas{ctx.world}"},
                     clocks, args.steps * 4)  # forward, stage 1, Dot2, three-word
    line.update({
        "fn": fn, "fp": fp, "fp_rate": fp / n_eval, "positives": int(y.sum()), "tau": tau,
        "decisions_differing_from_fp32_form": differ,
        "band": {"flagged": qst["n_flagged"], "resolved_f32": qst["n_resolved_f32"],
                 "resolved_ff": qst["n_resolved_ff"], "unresolved": qst["n_unresolved"]},
        "fp32_plain_queries_per_s": n_eval / (f32_ms / 1000.0),
        "speedup_vs_fp32_plain": f32_ms / ms,
        "max_logit_dev_vs_fp32_form": {"f16x3_eval": split_dev, "f16x3_calibration_sample": split_dev_cal,
                                       "bf16_calibration_sample": bf_dev},
        "margins_measured_on": f"{CAL_N} calibration rays of another stream, not the evaluation rays",
        "bf16_plain": {"queries_per_s": n_eval / (bf_ms / 1000.0), "margin": bf_margin, "fn": bf_fn,
                       "decisions_differing_from_fp32_form": bf_differ,
                       "flagged": bst["n_flagged"], "unresolved": bst["n_unresolved"]},
        "train_samples_per_s": {"bf16_tensor_core": BATCH / (bf16_step_ms / 1000.0),
                                "bf16_incl_gpu_sampling_and_labelling": BATCH / (loop_ms / 1000.0),
                                "fp32": BATCH / (f32_step_ms / 1000.0)},
        "train_wall_s": t_train,
        "roofline": {"kernel": "fwd_split_kernel (tcgen05, 3 products per k-step)", "bound": "tensor",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC_BYTES_PER_RAY * n_eval) if TRAFFIC_BYTES_PER_RAY else None,
                     "peak_kind": f"{pk_kind} bf16 burst", "fwd_ms": fwd_ms, "algorithmic_flops_per_launch": flops},
        "cpu_baseline": {"value": cpu_v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cpu_n} of the evaluation rays through the FP64 oracle forward"},
        "label_queries_per_s": n_eval / (label_ms / 1000.0),
        "label_sphere_predicates_per_s": n_eval * N_SPHERES / (label_ms / 1000.0),
        "sample_queries_per_s": n_eval / (sample_ms / 1000.0),
        "cpu_oracle_label_queries_per_s": {"value": cpu_label_v, "cores": cores,
                                           "sample": f"{cpu_label_n} of the evaluation rays, 64 spheres"},
        "e2e": {"value": ctx.world * n_eval / (e2e_ms / 1000.0), "unit": "queries/s",
                "h2d_bytes_per_step": n_eval * 6 * 4, "d2h_bytes_per_step": nb.n_words(n_eval) * 4,
                "call": "nb_query_host (pinned host rays read in place by the forward over NVLink-C2C, "
                        "bits copied back)",
                "bits_equal_device_query": e2e_equal,
                "staged_value": ctx.world * n_eval / (staged_ms / 1000.0),
                "staged_call": "nb_query_host with chunk_rows 2^22 (chunks copied in while the previous runs)"},
    })
    ctx.emit(line)


# ---------------------------------------------------------------------------------- 3D boxes, planes (FP8)
def run_c3(args):
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    sc = I.make_scene(1003, 256, 3, R_LO, R_HI)
    shape = nb.Shape(sc, dev)
    T = args.train_steps
    B = 131072
    n_eval = args.n_eval if args.n_eval != N_EVAL else (64 << 20)
    res = {}
    for kind, w0 in ((I.BOX3, 6), (I.PLANE3, 4)):
        widths = [w0, 256, 256, 256, 256, 1]
        # BF16 tensor-core training (weights streamed per half layer), a fresh GPU-sampled
        # and labelled batch per step
        tr = nb.Model(widths, infer_prec="f32", train_prec="bf16")
        tr.set_params(I.init_params(4003 + kind, widths))
        qb = torch.empty((B, w0), dtype=torch.float32, device=dev)
        yb = torch.empty(nb.n_words(B), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(T):
            nb.sample(kind, B, 2003 + kind, first=t * B, out=qb)
            nb.label(shape, kind, qb, out=yb)
            tr.train_step(qb, yb, 1.0 + 99.0 * t / max(T - 1, 1), 1.0)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        params = tr.get_params()
        # evaluation queries drawn by the GPU sampler (another stream), exact labels
        eq = nb.sample(kind, n_eval, rank_seed(3003 + kind, ctx.rank))
        ey = nb.label(shape, kind, eq)
        f32 = nb.Model(widths)
        f32.set_params(params)
        tau = f32.calibrate(eq, ey, eps=1e-5)
        f8 = nb.Model(widths, infer_prec="fp8")
        f8.set_params(params)
        f8.tau = tau
        # the margin: 2x the largest FP8 deviation from the FP32 form on a calibration sample
        # of other queries; the evaluation queries then check it
        cq = nb.sample(kind, CAL_N, rank_seed(SEED_CAL + kind, ctx.rank))
        _, z8 = f8.query(cq, logits=True)
        _, z32 = f32.query(cq, logits=True)
        dcal = (z8 - z32).abs()
        err = float(dcal.max().item())
        err999 = float(torch.quantile(dcal[:1 << 24].double(), 0.999).item())
        del z8, z32, dcal, cq
        _, z8 = f8.query(eq, logits=True)
        _, z32 = f32.query(eq, logits=True)
        err_eval = float((z8 - z32).abs().max().item())
        del z8, z32
        margin = max(2.0 * err, 0.05)
        out = torch.empty(nb.n_words(n_eval), dtype=torch.int32, device=dev)
        bits, qst = f8.query(eq, margin=margin, out=out, stats=True)
        y = nb.bits_to_numpy(ey, n_eval)
        dec = nb.bits_to_numpy(bits, n_eval)
        dec32 = nb.bits_to_numpy(f32.query(eq, margin=1e-2), n_eval)
        res[kind] = dict(widths=widths, params=params, eq=eq, f8=f8, f32=f32, out=out, margin=margin, err=err,
                         err999=err999, err_eval=err_eval,
                         fn=int(np.sum(y & ~dec)), fp=int(np.sum(~y & dec)), differ=int(np.sum(dec != dec32)),
                         qst=qst, tau=tau, train_s=train_s, pos=int(y.sum()))
        torch.cuda.empty_cache()
    box = res[I.BOX3]
    ms, clocks = ctx.timed(lambda: box["f8"].query(box["eq"], margin=box["margin"], out=box["out"]), args.steps,
                           args.warmup)
    value = ctx.world * n_eval / (ms / 1000.0)
    fwd_ms = ctx.time_ms(lambda: box["f8"].query(box["eq"], margin=0.0, out=box["out"]), max(3, args.steps // 4))
    f32_ms = ctx.time_ms(lambda: box["f32"].query(box["eq"], margin=1e-2, out=box["out"]), 2)
    # end to end through the public API: pinned host boxes in, bits back in host memory
    host_q = torch.empty((n_eval, 6), dtype=torch.float32, pin_memory=True)
    host_q.copy_(box["eq"].cpu())
    host_bits = torch.empty(nb.n_words(n_eval), dtype=torch.int32, pin_memory=True)

    def e2e_step():
        box["f8"].query_host(host_q, margin=box["margin"], out=host_bits)

    for _ in range(3):
        e2e_step()
    e2e_ms = ctx.time_ms(e2e_step, max(5, args.steps // 4))
    e2e_equal = bool(torch.equal(host_bits, box["f8"].query(box["eq"], margin=box["margin"]).cpu()))
    staged_ms = ctx.time_ms(lambda: box["f8"].query_host(host_q, margin=box["margin"], out=host_bits,
                                                         chunk_rows=1 << 22), max(5, args.steps // 4))
    del host_q
    pl = res[I.PLANE3]
    pl_ms = ctx.time_ms(lambda: pl["f8"].query(pl["eq"], margin=pl["margin"], out=pl["out"]), max(3, args.steps // 4))
    pl32_ms = ctx.time_ms(lambda: pl["f32"].query(pl["eq"], margin=1e-2, out=pl["out"]), 2)
    tr_ms, tr32_ms = {}, {}
    for kind, r in res.items():
        qb = nb.sample(kind, B, 9)
        yb = nb.label(shape, kind, qb)
        m = nb.Model(r["widths"], infer_prec="f32", train_prec="bf16")
        m.set_params(r["params"])
        tr_ms[kind] = ctx.time_ms(lambda: m.train_step(qb, yb, 50.0), 20)
        m32 = nb.Model(r["widths"])
        m32.set_params(r["params"])
        tr32_ms[kind] = ctx.time_ms(lambda: m32.train_step(qb, yb, 50.0), 3)
    if ctx.rank != 0:
        return ctx.emit(None)
    pk, pk_kind = peaks()
    macs = sum(box["widths"][i] * box["widths"][i + 1] for i in range(5))
    flops = 2.0 * macs * n_eval
    achieved = flops / (fwd_ms / 1000.0) / 1e12
    peak = 2.0 * float(pk.get("bf16_tflops", 1900.0))  # E4M3 dense rate = 2x BF16 (nominal 4.5 vs 2.25 PF)
    cpu_v, cores, cpu_n = cpu_oracle_rate(box["widths"], box["params"], box["eq"][:200000].cpu().numpy(), seconds=8.0)

    def summary(r, q_ms, q32_ms):
        return {"fn": r["fn"], "fp": r["fp"], "fp_rate": r["fp"] / n_eval, "positives": r["pos"], "tau": r["tau"],
                "margin": r["margin"],
                "margin_measured_on": f"{CAL_N} calibration queries of another stream (2x their max deviation)",
                "max_logit_dev_fp8_vs_fp32_form": {"calibration_max": r["err"], "calibration_p99.9": r["err999"],
                                                   "evaluation_max": r["err_eval"]},
                "band_fraction": r["qst"]["n_flagged"] / n_eval,
                "decisions_differing_from_fp32_form": r["differ"],
                "band": {"flagged": r["qst"]["n_flagged"], "resolved_f32": r["qst"]["n_resolved_f32"],
                         "resolved_ff": r["qst"]["n_resolved_ff"], "unresolved": r["qst"]["n_unresolved"]},
                "fp8_queries_per_s": n_eval / (q_ms / 1000.0), "fp32_plain_queries_per_s": n_eval / (q32_ms / 1000.0),
                "train_s_bf16": r["train_s"]}

    line = base_line(ctx, "neural-bound queries/s at 0 FN (3D boxes, FP8 E4M3 tcgen05 forward + FP32 re-check)",
                     value, "queries/s", ms, args.steps, args.warmup,
                     "e4m3 (two-term fp8 operands, 3 products per k-step, fp32 accumulate)",
                     {"workload": "3D box and plane queries: 256-sphere union, MLP in->256x4->1, FP8 inference, "
                                  "64M eval queries", "n_eval": n_eval, "batch": B, "train_steps": T,
                      "train_precision": "bf16 tensor cores (weights streamed per half layer), fp32 master weights",
                      "l2": f"inputs {n_eval * 24 >> 20} MB per step > L2"},
                     clocks, args.steps * 4)  # FP8 forward, stage 1, Dot2, three-word
    line.update({"box": summary(box, ms, f32_ms), "plane": summary(pl, pl_ms, pl32_ms),
                 "speedup_vs_fp32_plain": f32_ms / ms,
                 "train_samples_per_s": {"bf16_box": B / (tr_ms[I.BOX3] / 1000.0),
                                         "bf16_plane": B / (tr_ms[I.PLANE3] / 1000.0),
                                         "fp32_box": B / (tr32_ms[I.BOX3] / 1000.0),
                                         "fp32_plane": B / (tr32_ms[I.PLANE3] / 1000.0)},
                 "roofline": {"kernel": "fwd_fp8_kernel (tcgen05 kind::f8f6f4)", "bound": "tensor",
                              "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                              "traffic": (TRAFFIC_BYTES_PER_BOX * n_eval) if TRAFFIC_BYTES_PER_BOX else None,
                              "peak_kind": f"{pk_kind} bf16 burst x 2 (E4M3 nominal ratio)",
                              "fwd_ms": fwd_ms, "algorithmic_flops_per_launch": flops},
                 "cpu_baseline": {"value": cpu_v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                  "sample": f"{cpu_n} box queries through the FP64 oracle forward"},
                 "e2e": {"value": ctx.world * n_eval / (e2e_ms / 1000.0), "unit": "queries/s",
                         "h2d_bytes_per_step": n_eval * 6 * 4, "d2h_bytes_per_step": nb.n_words(n_eval) * 4,
                         "call": "nb_query_host (pinned host boxes read in place by the forward over "
                                 "NVLink-C2C, bits copied back)", "bits_equal_device_query": e2e_equal,
                         "staged_value": ctx.world * n_eval / (staged_ms / 1000.0),
                         "staged_call": "nb_query_host with chunk_rows 2^22 (chunks copied in while the "
                                        "previous runs)"}})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- early-out
EARLY_STEPS_FACTOR = 8
# the one-pass settle test is certified by its own rounding bound: no extra margin
MARGIN_EARLY = 0.0


def run_c2e(args):
    """3D point queries against a solid object (16 spheres of radius 0.2-0.5), the late
    network 3->128x4->1 (split-FP16) behind the neural early-out of Sec. 3.3: an early
    network of one hidden layer (the paper's early exit), trained on the complement 1 - g,
    evaluated in FP32 with a rigorous error bound in the one-pass stage that settles rows
    and gathers the others for the late network."""
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    sc = I.make_scene(SEED_SCENE + 10, 16, 3, 0.2, 0.5)
    shape = nb.Shape(sc, dev)
    late_w, early_w = [3, 128, 128, 128, 128, 1], [3, args.early_hidden, 1]
    T = args.train_steps if args.train_steps != TRAIN_STEPS else 10000
    late_t = nb.Model(late_w, infer_prec="f32", train_prec="bf16")
    late_t.set_params(I.init_params(SEED_INIT, late_w))
    early = nb.Model(early_w, train_prec="bf16")
    early.set_params(I.init_params(SEED_INIT + 1, early_w))
    for t in range(T):
        q = nb.sample(I.POINT3, BATCH, SEED_TRAIN, first=t * BATCH)
        y = nb.label(shape, I.POINT3, q)
        late_t.train_step(q, y, 1.0 + 99.0 * t / max(T - 1, 1))
    # the one-hidden-layer early network costs little to train: it gets --early-steps-factor
    # times the late network's steps (the share of rows it settles grows with them)
    TE = args.early_steps_factor * T
    for t in range(TE):
        q = nb.sample(I.POINT3, BATCH, SEED_TRAIN, first=t * BATCH)
        y = nb.label(shape, I.POINT3, q)
        early.train_step(q, nb.bits_not(y, BATCH), 1.0 + 99.0 * t / max(TE - 1, 1))
    late = nb.Model(late_w, infer_prec="f16x3")
    late.set_params(late_t.get_params())
    early_q = nb.Model(early_w, infer_prec="f32")  # FP32: the one-pass settle stage
    early_q.set_params(early.get_params())
    early = early_q
    n = args.n_eval
    eq = nb.sample(I.POINT3, n, rank_seed(SEED_QUERY, ctx.rank))
    ey = nb.label(shape, I.POINT3, eq)
    late.calibrate(eq, ey)
    early.calibrate(eq, nb.bits_not(ey, n))
    out = torch.empty(nb.n_words(n), dtype=torch.int32, device=dev)
    bits, est = nb.query_early_out(early, late, eq, margin_early=MARGIN_EARLY, margin_late=MARGIN, out=out)
    y = nb.bits_to_numpy(ey, n)
    dec = nb.bits_to_numpy(bits, n)
    ms, clocks = ctx.timed(lambda: nb.query_early_out(early, late, eq, margin_early=MARGIN_EARLY, margin_late=MARGIN,
                                                      out=out), args.steps, args.warmup)
    plain_ms = ctx.time_ms(lambda: late.query(eq, margin=MARGIN, out=out), max(3, args.steps // 4))
    early_ms = ctx.time_ms(lambda: early.query(eq, margin=1e-3, out=out), max(3, args.steps // 4))
    dplain = nb.bits_to_numpy(late.query(eq, margin=MARGIN), n)
    # the same two networks as a bound and an inverted bound: the broad-phase three-way
    # class of Sec. 4.4 (certainly outside / certainly inside / neither)
    codes = torch.empty(n, dtype=torch.uint8, device=dev)
    tw_stats = torch.zeros(4, dtype=torch.int64, device=dev)
    nb.query_three_way(late, early, eq, margin_outer=MARGIN, margin_inner=1e-3, out=codes, stats=tw_stats)
    tw = tw_stats.cpu().numpy()
    tc = codes.cpu().numpy()
    tw_ms = ctx.time_ms(lambda: nb.query_three_way(late, early, eq, margin_outer=MARGIN, margin_inner=1e-3,
                                                   out=codes), max(3, args.steps // 4))
    if ctx.rank != 0:
        return ctx.emit(None)
    line = base_line(ctx, "neural-bound queries/s at 0 FN (3D points, neural early-out + split-FP16 late network)",
                     ctx.world * n / (ms / 1000.0), "queries/s", ms, args.steps, args.warmup,
                     "f32 early network, f16x3 late network",
                     {"workload": f"3D points: 16-sphere solid (radii 0.2-0.5), late MLP 3->128x4->1, early MLP "
                                  f"3->{args.early_hidden}->1 on 1 - g, 16M eval points (Sec. 3.3 early-out)",
                      "n_eval": n, "train_steps": T, "early_train_steps": TE},
                     clocks, args.steps * 6)  # settle stage, late query (4), merge
    line.update({"fn": int(np.sum(y & ~dec)), "fp_rate": float(np.mean(~y & dec)),
                 "fp_rate_without_early_out": float(np.mean(~y & dplain)),
                 "early_inside_fraction": est["n_early_inside"] / n,
                 "without_early_out_queries_per_s": n / (plain_ms / 1000.0),
                 "speedup_vs_without": plain_ms / ms, "cpu_baseline": None, "e2e": None,
                 "inside_fraction": float(y.mean()), "early_network_alone_ms": early_ms, "late_network_alone_ms": plain_ms,
                 # the early-out saves f T_late and costs the early network plus the compaction,
                 # gather, scatter and host hand-over, C = T_total - (1 - f) T_late: it pays once the
                 # settled fraction f exceeds C / T_late
                 "break_even_settled_fraction": (ms - (1.0 - est["n_early_inside"] / n) * plain_ms) / plain_ms,
                 "three_way": {"queries_per_s": n / (tw_ms / 1000.0), "certainly_out": int(tw[0]),
                               "certainly_in": int(tw[1]), "neither": int(tw[2]), "conflicts": int(tw[3]),
                               "certain_and_wrong": int(np.sum((tc == 0) & y) + np.sum((tc == 1) & ~y)),
                               "launches": 9}})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- 2D points
def run_c1(args):
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    widths = [2, 32, 32, 32, 1]
    sc = I.make_scene(1000, 8, 2, 0.05, 0.3)
    shape = nb.Shape(sc, dev)
    T, B = 1000, 1024
    pool = torch.as_tensor(I.sample_queries(I.POINT2, 2000, T * B), device=dev)
    bits = nb.label(shape, I.POINT2, pool)
    m = nb.Model(widths)
    m.set_params(I.init_params(1001, widths))
    ctx.e0.record()
    for t in range(T):
        m.train_step(pool[t * B:(t + 1) * B], bits[t * B // 32:(t + 1) * B // 32], 1.0 + 99.0 * t / (T - 1), 1.0)
    ctx.e1.record()
    torch.cuda.synchronize()
    train_ms = ctx.e0.elapsed_time(ctx.e1) / T
    grid = torch.as_tensor(I.grid_points_2d(256), device=dev)
    yg = nb.label(shape, I.POINT2, grid)
    tau = m.calibrate(grid, yg)
    out = torch.empty(nb.n_words(grid.shape[0]), dtype=torch.int32, device=dev)
    m.query(grid, margin=1e-3, out=out)
    y = nb.bits_to_numpy(yg, grid.shape[0])
    dec = nb.bits_to_numpy(out, grid.shape[0])
    # the 65,536-point grid is one step; repeated to get a measurable region
    reps = 50
    # a 65,536-point query is launch-bound: the 50 queries of a step are one CUDA graph
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        with torch.cuda.graph(graph, stream=s_cap):
            for _ in range(reps):
                m.query(grid, margin=1e-3, out=out)
    torch.cuda.current_stream().wait_stream(s_cap)
    torch.cuda.synchronize()
    eager_ms = ctx.time_ms(lambda: [m.query(grid, margin=1e-3, out=out) for _ in range(reps)], 3)
    # end to end through the public API: the pinned host grid read in place, bits back
    hgrid = torch.empty(grid.shape, dtype=torch.float32, pin_memory=True)
    hgrid.copy_(grid.cpu())
    hbits = torch.empty(nb.n_words(grid.shape[0]), dtype=torch.int32, pin_memory=True)
    for _ in range(3):
        m.query_host(hgrid, margin=1e-3, out=hbits)
    e2e_ms = ctx.time_ms(lambda: [m.query_host(hgrid, margin=1e-3, out=hbits) for _ in range(reps)], 3)
    e2e_equal = bool(np.array_equal(nb.bits_to_numpy(hbits, grid.shape[0]), dec))
    ms, clocks = ctx.timed(graph.replay, args.steps, args.warmup)
    value = job_value(reps * grid.shape[0], ctx.world, ms)
    assert np.array_equal(nb.bits_to_numpy(out, grid.shape[0]), dec)
    cpu_v, cores, cpu_n = cpu_oracle_rate(widths, m.get_params(), I.grid_points_2d(256))
    line = base_line(ctx, "neural-bound queries/s at 0 FN (2D points, plain FP32)", value, "queries/s", ms,
                     args.steps, args.warmup, "f32",
                     {"workload": "2D points: 8-disk union, MLP 2->32x3->1 FP32, 1000 steps x 1024, 256x256 grid",
                      "reps_of_grid_per_step": reps, "cuda_graph": True,
                      "l2": "grid resident in L2 (256 KB); small-case configuration"},
                     clocks, args.steps * reps * 4)  # forward, stage 1, Dot2, three-word
    line.update({"fn": int(np.sum(y & ~dec)), "fp": int(np.sum(~y & dec)), "fp_rate": float(np.mean(~y & dec)),
                 "tau": tau, "train_samples_per_s_fp32": B / (train_ms / 1000.0),
                 "without_graph_queries_per_s": reps * grid.shape[0] / (eager_ms / 1000.0),
                 "cpu_baseline": {"value": cpu_v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                  "sample": f"{cpu_n} grid points through the FP64 oracle forward"},
                 "e2e": {"value": ctx.world * reps * grid.shape[0] / (e2e_ms / 1000.0), "unit": "queries/s",
                         "h2d_bytes_per_step": reps * grid.shape[0] * 2 * 4,
                         "d2h_bytes_per_step": reps * nb.n_words(grid.shape[0]) * 4,
                         "call": "nb_query_host per grid (pinned host points read in place over NVLink-C2C, bits "
                                 "copied back; one synchronous call per grid)", "bits_equal_device_query": e2e_equal}})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- 4D grouped
def run_c4(args):
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    widths = [4, 64, 64, 64, 1]
    K = 256
    rng = np.random.default_rng(4000)
    counts = [int(c) for c in rng.integers(4096 // 32, 65536 // 32 + 1, size=K) * 32]
    scenes = [I.make_scene(4100 + o, int(rng.integers(16, 65)), 3, 0.02, 0.2, moving=True) for o in range(K)]
    shapes = [nb.Shape(s, dev) for s in scenes]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    W = 4
    batches = []
    for j in range(W):
        qs = [torch.as_tensor(I.sample_queries(I.POINT4T, 5000 + 10 * o + j, counts[o]), device=dev) for o in range(K)]
        bs = [nb.label(shapes[o], I.POINT4T, qs[o]) for o in range(K)]
        batches.append((torch.cat(qs).contiguous(), torch.cat(bs).contiguous()))
    g = nb.Group(widths, K, infer_prec="f16x3", train_prec="bf16")
    g.set_params(np.stack([I.init_params(6000 + o, widths) for o in range(K)]))
    # rows per work item of the grouped launches, measured by the autotuner
    cands = (1024, 2048, 4096, 8192, 16384)
    chunk_train, ms_train = g.autotune(off, *batches[0], op="train", candidates=cands)
    plan = nb.Plan(off, chunk_rows=chunk_train)
    T = args.train_steps if args.train_steps != TRAIN_STEPS else 2000
    alpha = (1.0 + 99.0 * np.arange(T) / max(T - 1, 1)).astype(np.float32)
    g.set_schedule(alpha)
    g.reserve(plan)
    # one CUDA graph per pool batch, each replaying a training step with the device schedule
    graphs = []
    for j in range(W):
        g.train_step(plan, *batches[j], -1.0)  # eager first steps initialise kernel attributes
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for j in range(W):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(gr, stream=s):
                g.train_step(plan, *batches[j], -1.0)
        graphs.append(gr)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ctx.e0.record()
    for t in range(W, T):
        graphs[t % W].replay()
    ctx.e1.record()
    torch.cuda.synchronize()
    step_ms = ctx.e0.elapsed_time(ctx.e1) / max(T - W, 1)
    g.sync_schedule()
    # evaluation: 1M space-time points per object
    NE = args.n_eval if args.n_eval != N_EVAL else (1 << 20)
    eoff = np.arange(K + 1, dtype=np.int64) * NE
    eq = torch.empty((K * NE, 4), dtype=torch.float32, device=dev)
    ebits = torch.empty(nb.n_words(K * NE), dtype=torch.int32, device=dev)
    for o in range(K):
        eq[o * NE:(o + 1) * NE] = torch.as_tensor(I.sample_queries(I.POINT4T, 7000 + o, NE), device=dev)
        ebits[o * NE // 32:(o + 1) * NE // 32] = nb.label(shapes[o], I.POINT4T, eq[o * NE:(o + 1) * NE])
    chunk_query, ms_query = g.autotune(eoff, eq, op="query", candidates=cands + (32768,))
    eplan = nb.Plan(eoff, chunk_rows=chunk_query)
    taus = g.calibrate(eplan, eq, ebits)
    out = torch.empty_like(ebits)
    _, qst = g.query(eplan, eq, margin=MARGIN, out=out, stats=True)
    y = nb.bits_to_numpy(ebits, K * NE)
    dec = nb.bits_to_numpy(out, K * NE)
    ms, clocks = ctx.timed(lambda: g.query(eplan, eq, margin=MARGIN, out=out), args.steps, args.warmup)
    value = ctx.world * K * NE / (ms / 1000.0)
    # the grouped forward alone (margin 0: the re-check launches find an empty band)
    fwd_ms = ctx.time_ms(lambda: g.query(eplan, eq, margin=0.0, out=out), max(3, args.steps // 4))
    g.query(eplan, eq, margin=MARGIN, out=out)
    # plain FP32 single-object form: one network at a time, same weights and thresholds
    P = g.get_params()
    single = nb.Model(widths)
    o_ms = []
    for o in range(0, K, 32):
        single.set_params(P[o])
        single.tau = float(taus[o])
        o_ms.append(ctx.time_ms(lambda: single.query(eq[o * NE:(o + 1) * NE], margin=1e-2,
                                                     out=out[o * NE // 32:(o + 1) * NE // 32]), 2))
    f32_ms = float(np.mean(o_ms)) * K
    cpu_v, cores, cpu_n = cpu_oracle_rate(widths, P[0], eq[:NE].cpu().numpy())
    pk, pk_kind = peaks()
    macs = sum(widths[i] * widths[i + 1] for i in range(len(widths) - 1))
    flops = 2.0 * macs * K * NE
    achieved = flops / (fwd_ms / 1000.0) / 1e12
    roof_c4 = {"kernel": "fwd_split_group_kernel (tcgen05, 3 products per k-step)", "bound": "tensor",
               "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops"],
               "traffic": None, "peak_kind": f"{pk_kind} bf16 burst", "fwd_ms": fwd_ms,
               "algorithmic_flops_per_launch": flops}
    line = base_line(ctx, "grouped neural-bound queries/s at 0 FN (4D points, 256 objects, split-FP16)", value,
                     "queries/s", ms, args.steps, args.warmup, "f16x3 (split fp16 operands, fp32 accumulate)",
                     {"workload": "4D space-time points: 256 objects of 16-64 moving spheres, 4->64x3->1 per object, "
                                  "uneven 4096-65536 samples per object", "train_steps": T,
                      "eval_per_object": NE, "l2": f"inputs {K * NE * 16 >> 20} MB per step > L2"},
                     clocks, args.steps * 3)  # grouped forward, Dot2, three-word
    line.update({"fn": int(np.sum(y & ~dec)), "fp_rate": float(np.mean(~y & dec)),
                 "band": {"flagged": qst["n_flagged"], "unresolved": qst["n_unresolved"]},
                 "fp32_single_object_queries_per_s": K * NE / (f32_ms / 1000.0),
                 "speedup_vs_fp32_single_object": f32_ms / ms,
                 "grouped_train_samples_per_s_bf16_graph": sum(counts) / (step_ms / 1000.0),
                 "autotune": {"train_chunk_rows": chunk_train, "train_ms": ms_train,
                              "query_chunk_rows": chunk_query, "query_ms": ms_query},
                 "roofline": roof_c4,
                 "cpu_baseline": {"value": cpu_v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                  "sample": f"{cpu_n} points of object 0 through the FP64 oracle forward"},
                 "e2e": None})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- cascade
def run_c5(args):
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    widths = [6, 128, 128, 128, 1]
    K = 1024
    ms_ = I.make_multi_scene(5000, K, 32)
    ws = nb.WorldScene(ms_, dev)
    ix = nb.CascadeIndex(ws)  # stage 1 walks the 4-wide tree of object boxes
    T = args.train_steps if args.train_steps != TRAIN_STEPS else 2000
    # training pairs from the deployment distribution: world rays binned and moved into
    # each object's frame by the cascade's own first stage, labelled by the exact stage
    # (uneven pair counts per object, one grouped launch per step)
    n_pools, pool_rays = 16, 1 << 18
    pools = []
    for j in range(n_pools):
        r = torch.as_tensor(I.sample_world_rays(5100 + j, pool_rays), device=dev)
        off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, r, canonical=True, index=ix)
        rows = int(off[-1])
        lab = torch.zeros(nb.n_words(rows), dtype=torch.int32, device=dev)
        nb.cascade_exact(ws, r, pair_ray, off_d, rows, pair_hits=lab)
        pools.append((nb.Plan(off, chunk_rows=2048), pair_q, lab))
        del r, off_d, pair_ray
    g = nb.Group(widths, K, infer_prec="f16x3", train_prec="bf16")
    g.set_params(np.stack([I.init_params(5200 + k, widths) for k in range(K)]))
    t0 = time.perf_counter()
    for t in range(T):
        pl, pq, pb = pools[t % n_pools]
        g.train_step(pl, pq, pb, 1.0 + 99.0 * t / max(T - 1, 1))
    torch.cuda.synchronize()
    train_pairs_per_step = int(np.mean([p[0].n_rows for p in pools]))
    train_s = time.perf_counter() - t0
    NR = args.n_eval if args.n_eval != N_EVAL else (64 << 20)
    CH = min(NR, 16 << 20)
    rays = torch.empty((NR, 6), dtype=torch.float32, device=dev)
    for c in range(0, NR, CH):
        rays[c:c + CH] = torch.as_tensor(I.sample_world_rays(5300 + c // CH, min(CH, NR - c)), device=dev)
    chunks = [rays[c:c + CH] for c in range(0, NR, CH)]
    # thresholds calibrated on the benchmark rays' own pairs, chunk by chunk: the minimum
    # over chunks of (zmin - eps rounded down) is the threshold of all pairs together
    taus = np.full(K, np.inf)
    for ch in chunks:
        off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, ch, canonical=True, index=ix)
        rows = int(off[-1])
        lab = torch.zeros(nb.n_words(rows), dtype=torch.int32, device=dev)
        nb.cascade_exact(ws, ch, pair_ray, off_d, rows, pair_hits=lab)
        taus = np.minimum(taus, g.calibrate(nb.Plan(off, chunk_rows=2048), pair_q, lab))
        del off_d, pair_ray, pair_q, lab
    g.tau = taus
    hits_c = torch.zeros(nb.n_words(NR), dtype=torch.int32, device=dev)
    hits_p = torch.zeros(nb.n_words(NR), dtype=torch.int32, device=dev)
    est = torch.zeros(nb.CASCADE_STATS.itemsize, dtype=torch.uint8, device=dev)
    pst = torch.zeros(nb.CASCADE_STATS.itemsize, dtype=torch.uint8, device=dev)
    nst = torch.zeros(nb.QUERY_STATS.itemsize, dtype=torch.uint8, device=dev)

    bin_stats = {"aabb_pairs": 0, "ball_pairs": 0}

    def cascade_step(collect=False):
        # box + ball binning, neural bound per object, exact test of the survivors
        for ci, ch in enumerate(chunks):
            off, off_d, pair_ray, pair_q, st = nb.cascade_bin(ws, ch, canonical=True, index=ix)
            if collect:
                for k in bin_stats:
                    bin_stats[k] += int(st[k])
            plan_c = nb.Plan(off, chunk_rows=2048)
            neural = g.query(plan_c, pair_q, margin=MARGIN)
            nb.cascade_exact(ws, ch, pair_ray, off_d, int(off[-1]), pass_bits=neural,
                             ray_hits=hits_c[ci * CH // 32:], stats=est)

    def plain_step():
        for ci, ch in enumerate(chunks):
            off, off_d, pair_ray, _, st = nb.cascade_bin(ws, ch, canonical=False, index=ix)
            nb.cascade_exact(ws, ch, pair_ray, off_d, int(off[-1]), ray_hits=hits_p[ci * CH // 32:], stats=pst)

    est.zero_()
    cascade_step(collect=True)
    pst.zero_()
    plain_step()
    e = nb._read(est, nb.CASCADE_STATS)
    pe = nb._read(pst, nb.CASCADE_STATS)
    hc = nb.bits_to_numpy(hits_c, NR)
    hp = nb.bits_to_numpy(hits_p, NR)
    ms, clocks = ctx.timed(cascade_step, args.steps, args.warmup)
    plain_ms = ctx.time_ms(plain_step, max(2, args.steps))
    # per-stage times on the first chunk, for Eq. (Benefit): with the box (and ball) test
    # alone every pair goes to the exact test (p_b = 1); with the network in front a
    # fraction p_a does, at t_nn more per pair.  The network pays off when an exact pair
    # test costs more than t_nn / (1 - p_a).
    ch = chunks[0]
    off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, ch, canonical=True, index=ix)
    rows = int(off[-1])
    plan_c = nb.Plan(off, chunk_rows=2048)
    hb = torch.zeros(nb.n_words(ch.shape[0]), dtype=torch.int32, device=dev)
    neural = g.query(plan_c, pair_q, margin=MARGIN)
    t_bin = ctx.time_ms(lambda: nb.cascade_bin(ws, ch, canonical=True, index=ix), 2)
    # the same stage without the index: every ray against every object's box
    t_bin_all = ctx.time_ms(lambda: nb.cascade_bin(ws, ch, canonical=True), 2)
    t_bin_plain = ctx.time_ms(lambda: nb.cascade_bin(ws, ch, canonical=False, index=ix), 2)
    t_bin_plain_all = ctx.time_ms(lambda: nb.cascade_bin(ws, ch, canonical=False), 2)
    same_pairs = bool(np.array_equal(nb.cascade_bin(ws, ch, canonical=True)[0], off))
    t_nn = ctx.time_ms(lambda: g.query(plan_c, pair_q, margin=MARGIN, out=neural), 3)
    t_exact_all = ctx.time_ms(lambda: nb.cascade_exact(ws, ch, pair_ray, off_d, rows, ray_hits=hb), 3)
    t_exact_pass = ctx.time_ms(lambda: nb.cascade_exact(ws, ch, pair_ray, off_d, rows, pass_bits=neural,
                                                        ray_hits=hb), 3)
    live = int((pair_ray != -1).sum().item())
    p_a = e["exact_pairs"] / max(bin_stats["ball_pairs"], 1)
    t_nn_pair = t_nn / max(live, 1)
    t_exact_pair = t_exact_all / max(live, 1)
    break_even = t_nn_pair / max(1.0 - p_a, 1e-12)
    del off_d, pair_ray, pair_q, neural, plan_c
    # held-out rays: FN of the calibrated bounds on rays they were not calibrated on
    held = torch.as_tensor(I.sample_world_rays(5999, min(NR, 4 << 20)), device=dev)
    hh_c = torch.zeros(nb.n_words(held.shape[0]), dtype=torch.int32, device=dev)
    hh_p = torch.zeros_like(hh_c)
    off, off_d, pair_ray, pair_q, _ = nb.cascade_bin(ws, held, canonical=True, index=ix)
    neural = g.query(nb.Plan(off, chunk_rows=2048), pair_q, margin=MARGIN)
    nb.cascade_exact(ws, held, pair_ray, off_d, int(off[-1]), pass_bits=neural, ray_hits=hh_c)
    off, off_d, pair_ray, _, _ = nb.cascade_bin(ws, held, canonical=False, index=ix)
    nb.cascade_exact(ws, held, pair_ray, off_d, int(off[-1]), ray_hits=hh_p)
    held_fn = int(np.sum(nb.bits_to_numpy(hh_p, held.shape[0]) & ~nb.bits_to_numpy(hh_c, held.shape[0])))
    # cost of one exact pair test relative to one network query at which the cascade pays
    # off (Eq. (Benefit) with p = fraction of pairs sent to the exact test)
    line = base_line(ctx, "cascade rays/s at 0 FN (1024 objects, box -> neural bound -> exact)",
                     ctx.world * NR / (ms / 1000.0), "queries/s", ms, args.steps, args.warmup,
                     "f16x3 (split fp16 operands, fp32 accumulate)",
                     {"workload": "learned-culler cascade: 1024 objects of 32 spheres in [-10,10]^3, 6->128x3->1 per "
                                  "object, 64M rays", "n_rays": NR, "train_steps": T,
                      "stage1": "4-wide tree of object boxes (Morton order, median splits), 2 walks per call",
                      "training": f"{n_pools} x {pool_rays} world rays through the box/ball stage, exact labels",
                      "calibration": "thresholds calibrated on the benchmark rays' own pairs"},
                     clocks, args.steps * len(chunks) * 6)  # bin x2, grouped query (3), exact
    line.update({"fn_vs_plain": int(np.sum(hp & ~hc)), "hits_equal_plain": bool(np.array_equal(hc, hp)),
                 "stages_first_chunk_ms": {"bin": t_bin, "neural": t_nn, "exact_all_pairs": t_exact_all,
                                           "exact_passed_pairs": t_exact_pass},
                 "stage1_first_chunk_ms": {"box_ball_index": t_bin, "box_ball_every_object": t_bin_all,
                                           "box_index": t_bin_plain, "box_every_object": t_bin_plain_all,
                                           "index_counts_equal_every_object": same_pairs},
                 "benefit": {"p_a": p_a, "t_nn_per_pair_ns": 1e6 * t_nn_pair, "t_exact_per_pair_ns": 1e6 * t_exact_pair,
                             "break_even_exact_ns": 1e6 * break_even,
                             "exact_cost_factor_needed": break_even / max(t_exact_pair, 1e-30)},
                 "plain_box_exact_rays_per_s": NR / (plain_ms / 1000.0),
                 "pairs": {"box": bin_stats["aabb_pairs"], "ball": bin_stats["ball_pairs"], "exact_plain": pe["exact_pairs"], "exact_cascade": e["exact_pairs"],
                           "hit": pe["hit_pairs"]},
                 "exact_tests_avoided": pe["exact_pairs"] - e["exact_pairs"],
                 "exact_sphere_tests": {"plain": pe["sphere_tests"], "cascade": e["sphere_tests"]},
                 "held_out_fn": held_fn, "held_out_rays": int(held.shape[0]), "grouped_train_s_bf16": train_s,
                 "train_pairs_per_step": train_pairs_per_step,
                 "cpu_baseline": None, "e2e": None})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- paper sizes
def run_c6(args):
    """The paper's own network sizes (its supplementary architecture table: two hidden
    layers of 25 / 50 / 75 neurons for 2D / 3D / 4D indicators), each trained in FP32 on a
    sphere union of its dimension, calibrated on its evaluation queries and queried on the
    FP32 form and on the split-FP16 tensor-core form, zero-padded to 64 / 128 neurons.
    --activation sine gives every network the paper's sinusoidal hidden activation."""
    act = args.activation
    from paper_2310_06822_gb300 import inputs as I
    from paper_2310_06822_gb300 import nb
    ctx = Ctx(args)
    torch, dev = ctx.torch, ctx.dev
    T = args.train_steps if args.train_steps != TRAIN_STEPS else 2000
    n = args.n_eval if args.n_eval != N_EVAL else (16 << 20)
    B = 8192
    rows = [("2d_point", I.POINT2, [2, 25, 25, 1], I.make_scene(6000, 8, 2, 0.05, 0.3)),
            ("3d_point", I.POINT3, [3, 50, 50, 1], I.make_scene(6001, 64, 3, R_LO, R_HI)),
            ("3d_ray", I.RAY3, [6, 50, 50, 1], I.make_scene(6001, 64, 3, R_LO, R_HI)),
            ("3d_plane", I.PLANE3, [4, 50, 50, 1], I.make_scene(6001, 64, 3, R_LO, R_HI)),
            ("3d_box", I.BOX3, [6, 50, 50, 1], I.make_scene(6001, 64, 3, R_LO, R_HI)),
            ("4d_point", I.POINT4T, [4, 75, 75, 1], I.make_scene(6002, 32, 3, 0.02, 0.2, moving=True))]
    table = {}
    head = None
    for name, kind, widths, sc in rows:
        shape = nb.Shape(sc, dev)
        m = nb.Model(widths, activation=act)
        m.set_params(I.init_params(6100 + kind, widths))
        for t in range(T):
            q = nb.sample(kind, B, seed=rank_seed(6200 + kind, ctx.rank), first=t * B, device=dev)
            m.train_step(q, nb.label(shape, kind, q), 1.0 + 99.0 * t / max(T - 1, 1), 1.0)
        eq = nb.sample(kind, n, seed=rank_seed(6300 + kind, ctx.rank), device=dev)
        ey = nb.label(shape, kind, eq)
        tau = m.calibrate(eq, ey)
        f = nb.Model(widths, infer_prec="f16x3", activation=act)
        f.set_params(m.get_params())
        f.tau = tau
        out = torch.empty(nb.n_words(n), dtype=torch.int32, device=dev)
        d32 = nb.bits_to_numpy(m.query(eq, margin=MARGIN32), n)
        # margin: 4x the split form's largest deviation from the FP32 form on calibration
        # queries of another stream
        cq = nb.sample(kind, 1 << 20, seed=rank_seed(SEED_CAL + 100 + kind, ctx.rank), device=dev)
        _, zf = f.query(cq, logits=True)
        dev_f = float(np.max(np.abs(zf.cpu().numpy().astype(np.float64) - m.query(cq, logits=True)[1].cpu().numpy())))
        del cq, zf
        margin = max(MARGIN, 4.0 * dev_f)
        df = nb.bits_to_numpy(f.query(eq, margin=margin, out=out), n)
        y = nb.bits_to_numpy(ey, n)
        reps = max(3, args.steps // 4)
        ms32 = ctx.time_ms(lambda: m.query(eq, margin=MARGIN32, out=out), reps)
        if name == "3d_ray":
            msf, clocks = ctx.timed(lambda: f.query(eq, margin=margin, out=out), args.steps, args.warmup)
            # end to end through the public API: pinned host rays read in place, bits back
            hq = torch.empty((n, 6), dtype=torch.float32, pin_memory=True)
            hq.copy_(eq.cpu())
            hb = torch.empty(nb.n_words(n), dtype=torch.int32, pin_memory=True)
            for _ in range(3):
                f.query_host(hq, margin=margin, out=hb)
            e2e_ms = ctx.time_ms(lambda: f.query_host(hq, margin=margin, out=hb), reps)
            e2e_equal = bool(np.array_equal(nb.bits_to_numpy(hb, n), df))
            head = (msf, clocks, e2e_ms, e2e_equal)
            del hq, hb
        else:
            msf = ctx.time_ms(lambda: f.query(eq, margin=margin, out=out), reps)
        table[name] = {"widths": widths, "fp32_queries_per_s": n / (ms32 / 1000.0),
                       "f16x3_padded_queries_per_s": n / (msf / 1000.0), "speedup": ms32 / msf,
                       "fn": int(np.sum(y & ~df)), "fp_rate": float(np.mean(~y & df)),
                       "decisions_equal_fp32_form": bool(np.array_equal(d32, df)), "margin": margin}
        m.close()
        f.close()
    msf, clocks, e2e_ms, e2e_equal = head
    line = base_line(ctx, "neural-bound queries/s at 0 FN (3D rays, the paper's 6->50->50->1%s, split-FP16 padded)"
                     % (", sine activations" if act == "sine" else ""),
                     job_value(n, ctx.world, msf), "queries/s", msf, args.steps, args.warmup,
                     "f16x3 (split fp16 operands, fp32 accumulate)",
                     {"workload": "the paper's network sizes: 2D 2->25x2->1, 3D 3/6/4->50x2->1, 4D 4->75x2->1, "
                                  "FP32 training, 16M eval queries each", "n_eval": n, "train_steps": T,
                      "batch": B, "padding": "hidden widths zero-padded to 64 (25, 50) and 128 (75)",
                      "activation": act},
                     clocks, args.steps * 4)
    line.update({"sizes": table, "cpu_baseline": None,
                 "e2e": {"value": ctx.world * n / (e2e_ms / 1000.0), "unit": "queries/s",
                         "h2d_bytes_per_step": n * 6 * 4, "d2h_bytes_per_step": nb.n_words(n) * 4,
                         "call": "nb_query_host on the 3D-ray network (pinned host rays read in place over "
                                 "NVLink-C2C, bits copied back)", "bits_equal_device_query": e2e_equal}})
    ctx.emit(line)


# ---------------------------------------------------------------------------------- reference arm
def reference_arm(args):
    """The oracle as it stands (FP64 forward of the same network), timed on host cores."""
    from oracle import oracle as O
    from paper_2310_06822_gb300 import inputs as I
    if int(os.environ.get("RANK", "0")) != 0:
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
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c2e", "c3", "c4", "c5", "c6"])
    ap.add_argument("--train-steps", type=int, default=TRAIN_STEPS)
    ap.add_argument("--n-eval", type=int, default=N_EVAL, help="evaluation size (smaller only for profiling)")
    ap.add_argument("--early-hidden", type=int, default=64,
                    help="c2e: hidden width of the one-hidden-layer early network")
    ap.add_argument("--early-steps-factor", type=int, default=EARLY_STEPS_FACTOR,
                    help="c2e: the early network's training steps as a multiple of the late network's")
    ap.add_argument("--activation", default="relu", choices=["relu", "sine"],
                    help="hidden activation of the c6 networks (sine: the paper's sinusoidal activation)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    {"c1": run_c1, "c2": run_c2, "c2e": run_c2e, "c3": run_c3, "c4": run_c4, "c5": run_c5,
     "c6": run_c6}[args.config](args)


if __name__ == "__main__":
    main()
