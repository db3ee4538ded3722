"""Benchmark of the hot path: LLG right-hand-side evaluations per second.

Workload (default): the standard-problem-4 film 500 x 125 x 3 nm as
200 x 50 x 1 tiles (n = 10,000), tensor assembled in FP64 on the GPU and
stored in FP32 (2.43 GB, larger than L2), one simulation, field 1
(mu0 H = (-24.6, 4.3, 0) mT), alpha = 0.02.  A step is one attempted
Dormand-Prince step: 6 right-hand sides (streaming demag product +
exchange + Zeeman + LLG), the embedded error, accept/reject and step-size
control, all on the device (one CUDA-graph replay).

Printed: one JSON line (rank 0).  `value` = RHS evaluations per second over
all ranks, device-resident inputs, timed with CUDA events on the
integrator's stream.  `e2e` = the same through the public API with host
buffers (pinned host -> device state copy, one step, device -> host copy
every step).  `roofline` = the streaming demag kernel against the measured
HBM bandwidth.  `cpu_baseline` = the FP64 CPU oracle on the same workload.

--impl reference runs the FP64 CPU oracle instead (the reference arm), on
this machine's host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_05364_gb300 import workloads as wl  # noqa: E402

MU0 = 4e-7 * math.pi
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the streaming FP32 product at the film workload below (n = 10,000), from one
# ncu capture of a full launch of the current kernels.  Every block stored, 4
# planes (the single-layer film): 1,618,117,632 read + 2,918,912 written
# (1.0132 x the 1.6e9 algorithmic bytes: the zero padding of the last chunk
# row).  Valid while k_matvec<f32> reads the same bytes (since the capture,
# only the order of the split panels' loads of their parked parts changed).
MATVEC_F32_N10000_TRAFFIC = {4: 1618117632 + 2918912}  # tensors storing every block
# The same film with the tensor stored half (upper triangle of chunks, in
# super-row order) and traceless (3 planes: xx, xy, yy), one ncu capture of
# each kernel of a product: k_matvec_half<f32, 3 planes> read 621,368,064 and
# wrote 4,680,192 bytes, k_half_cols read 4,864,000 (the column sums of the
# groups above the diagonal) and wrote 15,360 -- 1.051 x the 0.60 GB
# algorithmic bytes.  Valid while both kernels are unchanged.
MATVEC_F32_HALF_N10000_TRAFFIC = {3: 621368064 + 4680192 + 4864000 + 15360}


def f32_alg_bytes(info, n):
    """Algorithmic bytes of one FP32 streaming product: every unique stored
    value read once -- the stored entry planes of every block, or of the
    upper triangle (n (n + 1) / 2 blocks) when the tensor of a tile set of
    one shape is stored half (N_ij = N_ji)."""
    blocks = n * (n + 1) / 2.0 if info.get("half") else float(n) * n
    return 4.0 * info["planes"] * blocks
# The tensor-core products at n = 8,000 read 1.0040 (split) and 1.0028 (BF16)
# x their stored tensors and wrote their fields (one ncu capture each of the
# current kernels); the batched line scales that per stored byte.
GEMM_READ_PER_STORED_BYTE = {"split": 1.0040, "bf16": 1.0028}
FIELD1 = np.array([-24.6e-3, 4.3e-3, 0.0]) / MU0
WORKLOAD = "sp4_film_200x50x1_n10000_f32"
METRIC = "LLG RHS evals/s"
UNIT = "RHS evals/s"


def film_config(n, world):
    """The workload description both arms print (the reference arm runs the
    same workload on the host cores)."""
    return {"workload": WORKLOAD, "tiles": n, "sims_per_gpu": 1, "step": "one Dormand-Prince attempt = 6 RHS",
            "l2": "inputs larger than L2 (FP32 tensor 1.62 GB, L2 129 MB)",
            "parallelism": "replicas" if world > 1 else "single"}


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_rhs_baseline(t, m0, n_evals=3):
    """The FP64 oracle as it stands: dense FP64 tensor (assembled once,
    untimed), then n_evals right-hand sides timed on all host cores."""
    import oracle
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=0.02, Ha=FIELD1)
    oracle.llg_rhs(md, m0, p)  # warm
    t0 = time.perf_counter()
    for _ in range(n_evals):
        oracle.llg_rhs(md, m0, p)
    dt = time.perf_counter() - t0
    return {"value": n_evals / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "n=%d film, FP64 tensor assembled once (untimed), %d RHS evaluations timed" % (t.n, n_evals)}


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (the job is done when every replica is)."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all replicas per second of the slowest one."""
    return units_per_rank * world / (ms * 1e-3)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle's RK(4,5) on the same workload."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    import oracle
    t = wl.film(200, 50, 1)
    m0 = wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=0)
    md = oracle.Model.from_tiles(t)
    p = oracle.llg_params(alpha=0.02, Ha=FIELD1)
    h = 1e-13
    m = m0.copy()
    for _ in range(args.warmup):
        st, m, _, _ = oracle.integrate(md, m, p, oracle.ode_opts(fixed_h=h), 0.0, h, 1)
    t0 = time.perf_counter()
    n_rhs = 0
    for _ in range(args.steps):
        st, m, _, s = oracle.integrate(md, m, p, oracle.ode_opts(fixed_h=h), 0.0, h, 1)
        n_rhs += s["n_rhs"] - 1  # the first evaluation of each call is the FSAL restart
    dt = time.perf_counter() - t0
    val = n_rhs / dt
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": film_config(t.n, world), "precision": "f64 (oracle: stored FP64 tensor)",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one fixed-size RK(4,5) step (6 RHS) per timed step, n=%d" % t.n},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = _rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2107_05364_gb300 import binding as mt

    t = wl.film(200, 50, 1)
    n = t.n
    m0 = wl.m_noisy(n, (1, 1, 1), 1e-3, seed=rank).astype(np.float32)
    ctx = mt.mt_ctx_create(dev)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    info = T.info()
    p, keep = mt.llg_params(1, alpha=0.02, Ha=FIELD1)
    I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11))
    I.set_state(m0.ravel())
    stream = torch.cuda.ExternalStream(I.stream_handle())

    # warm-up
    I.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device-resident state --------------------
    s0 = I.stats()[0]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        I.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    s1 = I.stats()[0]
    n_rhs = s1["n_rhs"] - s0["n_rhs"]
    assert n_rhs == 6 * args.steps, (n_rhs, args.steps)
    ms = max_over_ranks(ms, dist, "cuda")
    value = whole_job_rate(n_rhs, world, ms)

    # ---- dominant kernel: the streaming demag product, standalone and as
    # the step runs it (six back to back in one CUDA graph) ----------------
    mg = torch.tensor(m0.ravel(), device="cuda")
    H = torch.empty_like(mg)
    field_ms, graph_ms = _product_times(mt, T, mg, H, 1, reps=max(10, min(args.steps, 100)))
    # the stored FP32 entries of a 3x3 block, each read once: 6, or 4 for a
    # single-layer film (xz and yz vanish)
    planes = info["planes"]
    alg_bytes = f32_alg_bytes(info, n)
    peaks, kind = _peaks()
    # the product's duration inside the timed step: at most the step time
    # over its six products (the stage kernels take the rest), so the
    # bandwidth from it is a lower bound of what the product streams at
    launch_ms = ms / args.steps / 6.0
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))

    # ---- end to end through the public API with host buffers ------------
    pinned_in = torch.from_numpy(m0.ravel().copy()).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    I.set_state(pinned_in.numpy())
    I.step(1)
    I.get_state(pinned_out.numpy().reshape(1, n, 3))
    torch.cuda.synchronize()
    tw0 = time.perf_counter()
    for _ in range(e2e_steps):
        I.set_state(pinned_in.numpy())
        I.step(1)
        I.get_state(pinned_out.numpy().reshape(1, n, 3))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - tw0
    # counted as `value` counts: 6 RHS per attempted step (a state loaded from
    # the host also needs its first derivative: that restart is overhead
    # inside the timed region, not counted)
    e2e_val = 6.0 * e2e_steps * world / e2e_s if e2e_s > 0 else None

    if dist:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = _oracle_rhs_baseline(t, m0.astype(np.float64))
    # the other two hot-path rows, compact: batched tensor-core product and
    # serving (full versions: --workload batched / --workload serving)
    extra = {}
    if world == 1 and not args.no_extras:
        # the same film, one simulation, with the tensor stored in the other
        # streaming precisions (BF16 with per-block scales, split BF16)
        prec_rows = {}
        for pname in ("f32_every_block", "f32_six_planes", "bf16", "split"):
            if pname == "f32_every_block":  # 4 planes, every block stored (no use of N_ij = N_ji)
                Tp = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)
            elif pname == "f32_six_planes":  # 6 planes, every block stored
                Tp = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM6)
            else:
                Tp = mt.mt_demag_assemble(tiles, pname)
            Ip = mt.Integrator(Tp, p, mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11))
            Ip.set_state(m0.ravel())
            Ip.step(3)
            sp = torch.cuda.ExternalStream(Ip.stream_handle())
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            nst = max(20, min(args.steps, 200))
            torch.cuda.synchronize()
            k0.record(sp)
            Ip.step(nst)
            k1.record(sp)
            torch.cuda.synchronize()
            prec_rows[pname] = {"rhs_evals_per_s": 6.0 * nst / (k0.elapsed_time(k1) * 1e-3),
                                "tensor_gb": Tp.info()["bytes"] / 1e9}
            Ip.close()
            Tp.close()
        extra["stored_precisions_same_workload"] = prec_rows
        for h in (I, T, tiles):
            h.close()
        import argparse as _ap
        try:
            b = run_batched(_ap.Namespace(batch=64, prec="split", steps=5, warmup=3), quiet=True)
            extra["batched"] = {k: b[k] for k in ("value", "unit", "vs_plain_fp32", "plain_fp32_evals_per_s",
                                                  "dtype", "config", "roofline")}
        except Exception as e:  # reported, never hides the main line
            extra["batched"] = {"error": str(e)}
        try:
            extra["serving"] = run_serving(_ap.Namespace(
                requests=args.requests, rate=args.rate, t_cap=args.t_cap, batch_slots=args.batch_slots,
                serve_prec=args.serve_prec, serve_budget_gb=args.serve_budget_gb, serve_rtol=args.serve_rtol,
                serve_limit=args.serve_limit), quiet=True)
        except Exception as e:
            extra["serving"] = {"error": str(e)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": film_config(n, world),
        "precision": "f32 storage, f32 accumulate, f64 assembly", "stored_planes": planes,
        "stored_half": bool(info["half"]),
        "sms": torch.cuda.get_device_properties(dev).multi_processor_count,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": None if n != 10000 else (MATVEC_F32_HALF_N10000_TRAFFIC if info["half"]
                                                         else MATVEC_F32_N10000_TRAFFIC).get(planes),
                     "kernel": (("k_matvec_half<f32" if info["half"] else "k_matvec<f32") +
                                (", %d planes" % planes if planes != 6 else "") +
                                ("> + k_half_cols" if info["half"] else ">")),
                     "stored": "upper triangle of blocks (N_ij = N_ji: tiles of one shape)" if info["half"]
                     else "every block",
                     "peak_kind": kind, "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": launch_ms,
                     "launch_ms_source": "timed step (CUDA events) / 6 products: an upper bound of the "
                                         "product's in-step duration, so frac is a lower bound",
                     "standalone_launch_ms": field_ms,
                     "standalone_frac": alg_bytes / (field_ms * 1e-3) / 1e9 / peak,
                     "graph6_launch_ms": graph_ms,
                     "graph6_frac": None if graph_ms is None else alg_bytes / (graph_ms * 1e-3) / 1e9 / peak,
                     "graph6_note": "six mt_demag_field calls in one CUDA graph (each with its operand prep)"},
        "demag_gbs": achieved,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 12 * n, "d2h_bytes_per_step": 12 * n,
                "note": "set_state(pinned host) + 1 step + get_state(host); 6 RHS counted per step"},
        "gpu_launches": 13 * args.steps,
        "clocks": clk.summary(),
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batched(args, quiet=False):
    """Batched workload: film 200 x 50 x 2 (n = 20,000), B simulations (field
    sweep +-50 mT along a seeded in-plane direction, alpha in {0.02, 0.1,
    0.5}) on a dense BF16 / split BF16 tensor multiplied on the tensor cores;
    against the same steps of the plain FP32 streaming path run one simulation
    at a time."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    t = wl.film(200, 50, 2)
    n, B = t.n, args.batch
    Ha, d = wl.sweep_fields(B, 50.0, seed=0)
    alphas = wl.sweep_alphas(B)
    m0 = np.stack([wl.m_noisy(n, d + np.array([0, 0, 0.05]), 1e-2, seed=b) for b in range(B)]).astype(np.float32)
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    peaks, kind = _peaks()
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11)

    def time_steps(I, steps):
        stream = torch.cuda.ExternalStream(I.stream_handle())
        I.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        I.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # batched path on the tensor cores
    Td = mt.mt_demag_assemble_ex(tiles, args.prec, mt.MT_LAYOUT_DENSE)
    info = Td.info()
    p, keep = mt.llg_params(B, alpha=alphas, Ha=Ha)
    I = mt.Integrator(Td, p, opts, B=B)
    I.set_state(m0.ravel())
    with ClockSampler(0) as clk:
        ms = time_steps(I, args.steps)
    value = 6.0 * args.steps * B / (ms * 1e-3)
    # the batched product alone (prep + tcgen05 GEMM + FP64 near blocks)
    mg = torch.tensor(m0.ravel(), device="cuda")
    H = torch.empty_like(mg)
    cur = torch.cuda.current_stream()
    for _ in range(3):
        mt.mt_demag_field(Td, mg, H, B=B, stream=cur)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(reps):
        mt.mt_demag_field(Td, mg, H, B=B, stream=cur)
    e1.record(cur)
    torch.cuda.synchronize()
    gemm_ms = e0.elapsed_time(e1) / reps
    Kp = int(math.ceil(3 * n / 128) * 128)
    stored = info["bytes"]
    flops = 2.0 * Kp * Kp * mt_pad(B) * (3 if args.prec == "split" else 1)
    Td.close()
    I.close()
    # plain FP32 path, one simulation at a time
    Ts = mt.mt_demag_assemble(tiles, "f32")
    p1, keep1 = mt.llg_params(1, alpha=alphas[0], Ha=Ha[0])
    I1 = mt.Integrator(Ts, p1, opts, B=1)
    I1.set_state(m0[0].ravel())
    ms1 = time_steps(I1, max(3, args.steps // 2))
    plain = 6.0 * max(3, args.steps // 2) / (ms1 * 1e-3)
    line = {
        "metric": METRIC + " (batched, tensor cores)", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": "sp4_film_200x50x2_n20000_B%d_%s_dense" % (B, args.prec), "tiles": n, "sims": B,
                   "l2": "inputs larger than L2 (tensor %.1f GB)" % (stored / 1e9)},
        "vs_plain_fp32": value / plain, "plain_fp32_evals_per_s": plain,
        "roofline": {"bound": "hbm", "achieved": stored / (gemm_ms * 1e-3) / 1e9, "peak": float(peaks["hbm_gbs"]),
                     "unit": "GB/s", "frac": stored / (gemm_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"]),
                     "traffic": round(GEMM_READ_PER_STORED_BYTE[args.prec] * stored + 12 * n * B),
                     "traffic_note": "scaled from an n = 8,000 capture",
                     "kernel": "k_gemm<%s>" % args.prec, "launch_ms": gemm_ms,
                     "tensor_tflops": flops / (gemm_ms * 1e-3) / 1e12,
                     "tensor_frac_of_bf16_peak": flops / (gemm_ms * 1e-3) / 1e12 / float(peaks["bf16_tflops"]),
                     "peak_kind": kind},
        "gpu_launches": 19 * args.steps, "clocks": clk.summary(),
    }
    for h in (Ts, I1, tiles):
        h.close()
    if not quiet:
        print(json.dumps(line), flush=True)
    return line


def run_serving(args, quiet=False):
    """Serving workload: a Poisson stream (mean `rate` req/s, seed 0) of
    relax-to-equilibrium jobs over 12 synthetic geometries (films and prisms,
    n log-uniform in [500, 40,000], Ms 4e5-1.2e6 A/m), |mu0 H| <= 100 mT,
    each job from its own random m0 (random unit vector per tile), relaxed at
    alpha = 0.5 to a torque below 1e-4 or stopped at the simulated-time cap.
    Tensors are cached on the device under an HBM budget, evicted least
    recently used; assembly on first use (and after an eviction) is part of
    the served time.  Two passes over the same requests: continuous batching
    (`batch_slots` per geometry, engines of different geometries overlapping)
    and one job at a time in arrival order (one slot, a server-wide limit of
    one running job).  A pass stops `serve_limit` seconds after the last
    arrival; jobs still running then are reported as unfinished, with their
    latency bounded below by that time."""
    import threading as th
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    geoms = wl.serving_geometries(12, 500, 40000, seed=0)
    reqs = wl.serving_requests(args.requests, args.rate, 12, seed=0)
    ctx = mt.mt_ctx_create(0)
    layout = mt.MT_LAYOUT_STREAM if args.serve_prec == "f32" else mt.MT_LAYOUT_DENSE
    budget = int(args.serve_budget_gb * (1 << 30))
    opts = mt.ode_opts(rtol=args.serve_rtol, atol=args.serve_rtol, h0=1e-14, hmax=1e-11)
    m0s = [wl.m_random(geoms[r.geometry].n, seed=r.m0_seed).astype(np.float32) for r in reqs]

    def one_pass(max_batch, max_running):
        S = mt.Server(ctx, max_batch=max_batch, prec=args.serve_prec, layout=layout, hbm_budget_bytes=budget,
                      opts=opts, replays_per_poll=8, max_running=max_running)
        gids = [S.add_geometry(g) for g in geoms]
        # warm the context and the graph machinery on the smallest geometry
        small = int(np.argmin([g.n for g in geoms]))
        w = S.submit(gids[small], wl.m_random(geoms[small].n, seed=7), alpha=0.5, tol=1e-4, t_max=1e-14)
        S.wait(w, 600.0)
        ids = [None] * len(reqs)
        t0 = time.perf_counter()

        def feeder():
            for k, r in enumerate(reqs):
                dt = r.arrival_s - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids[k] = S.submit(gids[r.geometry], m0s[k], alpha=0.5, Ha=r.Ha, tol=1e-4, t_max=args.t_cap)

        f = th.Thread(target=feeder)
        f.start()
        f.join()
        deadline = time.perf_counter() + args.serve_limit
        res, unfinished = [], []
        for k in range(len(reqs)):
            s, r, _ = S.wait(ids[k], max(0.0, deadline - time.perf_counter()))
            if s == mt.MT_OK:
                res.append(r)
            else:
                unfinished.append(k)
        wall = time.perf_counter() - t0
        st = S.stats()
        S.close()  # drops the unfinished jobs
        lat = np.array([r["t_done"] - r["t_submit"] for r in res])
        # an unfinished job's latency is at least the pass's end minus its arrival
        lat_lb = np.concatenate([lat, [wall - reqs[k].arrival_s for k in unfinished]])
        status = [r["status"] for r in res]
        out = {"finished": len(res), "unfinished": len(unfinished),
               "converged": int(sum(1 for x in status if x == 0)),
               "capped": int(sum(1 for x in status if x == 4)),
               "failed": int(sum(1 for x in status if x not in (0, 4))),
               "p50_s": float(np.percentile(lat_lb, 50)), "p99_s": float(np.percentile(lat_lb, 99)),
               "latency_note": "over all requests; unfinished ones at their lower bound" if unfinished else
               "over all requests",
               "jobs_per_s": len(res) / wall, "wall_s": wall,
               "rhs_evals": int(sum(r["n_rhs"] for r in res)),
               "assemblies": st["assemblies"], "evictions": st["evictions"]}
        if len(res):
            out["p50_finished_s"] = float(np.percentile(lat, 50))
            out["p99_finished_s"] = float(np.percentile(lat, 99))
        return out

    batched = one_pass(args.batch_slots, 0)
    single = one_pass(1, 1)
    tensor_gb = [mt_tensor_gb(g, args.serve_prec) for g in geoms]
    out = {"requests": len(reqs), "rate_hz": args.rate, "geometries": len(geoms),
           "n_range": [int(min(g.n for g in geoms)), int(max(g.n for g in geoms))],
           "precision": args.serve_prec + (" streaming" if layout == mt.MT_LAYOUT_STREAM else " dense (tensor cores)"),
           "budget_gb": args.serve_budget_gb, "tensors_gb_total": float(sum(tensor_gb)),
           "slots": args.batch_slots, "t_cap_s": args.t_cap, "tol": 1e-4, "rtol_atol": args.serve_rtol,
           "limit_after_last_arrival_s": args.serve_limit, "m0": "random unit vector per tile",
           "continuous_batching": batched, "one_by_one": single}
    if not quiet:
        line = {"metric": "serving p50/p99 latency (relax jobs)", "value": batched["p99_s"], "unit": "s (p99)",
                "n_gpus": 1, "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 * batched["wall_s"] / len(reqs),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.serve_prec,
                "data": "synthetic", "config": {"workload": "serving_12geoms_poisson%g_%dreq" % (args.rate, len(reqs))},
                "serving": out}
        print(json.dumps(line), flush=True)
    return out


def mt_tensor_gb(t, prec):
    """Stored bytes of a geometry's tensor (GB): streaming FP32 16 B (one
    layer of tiles) or 24 B per block, dense BF16 2 B / split 4 B per entry
    of the padded 3n x 3n matrix."""
    n = t.n
    if prec == "f32":
        return (16.0 if t.shape[2] == 1 else 24.0) * n * n / 1e9
    kp = math.ceil(3 * n / 128) * 128
    return (2.0 if prec == "bf16" else 4.0) * kp * kp / 1e9


def run_threshold(args):
    """Sec. 4.3.1 experiment: time versus error when the smallest fraction of
    the tensor elements is dropped, on the standard-problem-4 film at the
    paper's converged resolution 160 x 40 x 1 (n = 6,400).  For each fraction:
    kept elements, time of one product, field error against the unthresholded
    FP64 product at a relaxed state, and the largest deviation of <m>(t) over
    0.5 ns of field-1 dynamics from the unthresholded FP32 run."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    t = wl.film(160, 40, 1)
    n = t.n
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    # thresholding works on a tensor with every block stored; the half
    # storage of this film (N_ij = N_ji) is timed beside it at the end
    T = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM_FULL)
    # a relaxed start (the s-state route: relax from near (1,1,1))
    p0, k0 = mt.llg_params(1, alpha=0.5)
    I = mt.Integrator(T, p0, mt.ode_opts(rtol=1e-5, atol=1e-5))
    I.set_state(wl.m_noisy(n, (1, 1, 1), 1e-3, seed=0).astype(np.float32).ravel())
    I.relax(1e-4, 10e-9, check=False)
    m_rel = I.get_state()[0].copy()
    I.close()
    mg = torch.tensor(m_rel.ravel(), device="cuda")
    H0 = torch.empty_like(mg)
    # reference field: the unthresholded tensor stored and applied in FP64
    T64 = mt.mt_demag_assemble(tiles, "f64")
    Hd = torch.empty(mg.numel(), dtype=torch.float64, device="cuda")
    mt.mt_demag_field_f64(T64, mg.double(), Hd)
    torch.cuda.synchronize()
    H0n = Hd.cpu().numpy()
    T64.close()
    mt.mt_demag_field(T, mg, H0)
    torch.cuda.synchronize()
    dense_err = float(np.linalg.norm(H0.cpu().numpy() - H0n) / np.linalg.norm(H0n))
    p1, k1 = mt.llg_params(1, alpha=0.02, Ha=FIELD1)
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11)

    def dynamics(tensor):
        J = mt.Integrator(tensor, p1, opts)
        J.set_state(m_rel.ravel())
        tw = time.perf_counter()
        _, mavg, st = J.run(0.5e-9, 100, check=False)
        wall = time.perf_counter() - tw
        J.close()
        return mavg[:, 0, :], wall, st[0]["n_rhs"]

    ref_trace, ref_wall, _ = dynamics(T)
    rows = []
    for f in (0.0, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8):
        S, thr, kept = mt.mt_tensor_threshold(T, f)
        H = torch.empty_like(mg)
        for _ in range(3):
            mt.mt_demag_field(S, mg, H)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            mt.mt_demag_field(S, mg, H)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        err = float(np.linalg.norm(H.cpu().numpy() - H0n) / np.linalg.norm(H0n))
        trace, wall, nrhs = dynamics(S)
        info = S.info()
        rows.append({"fraction": f, "kept_elements": kept, "sparse_bytes": info["bytes"],
                     "row_warps": info["row_warps"], "product_ms": ms,
                     "field_rel_err": err, "mavg_max_dev": float(np.abs(trace - ref_trace).max()),
                     "dynamics_s": wall, "rhs": nrhs})
        S.close()
    # the dense FP32 streaming product for comparison
    for _ in range(3):
        mt.mt_demag_field(T, mg, H0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        mt.mt_demag_field(T, mg, H0)
    e1.record()
    torch.cuda.synchronize()
    dense_ms = e0.elapsed_time(e1) / 20
    # the default storage of this film: the upper triangle only
    Th = mt.mt_demag_assemble(tiles, "f32")
    Hh = torch.empty_like(mg)
    for _ in range(3):
        mt.mt_demag_field(Th, mg, Hh)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        mt.mt_demag_field(Th, mg, Hh)
    e1.record()
    torch.cuda.synchronize()
    half_ms = e0.elapsed_time(e1) / 20
    half_err = float(np.linalg.norm(Hh.cpu().numpy() - H0n) / np.linalg.norm(H0n))
    half_info = Th.info()
    Th.close()
    line = {"metric": "thresholded tensor: product time vs field error", "value": rows[3]["product_ms"],
            "unit": "ms (40 % threshold)", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "sp4_film_160x40x1_n6400_threshold"},
            "dense_fp32_product_ms": dense_ms, "dense_fp32_field_rel_err": dense_err,
            "dense_fp32_bytes": T.info()["bytes"],
            "half_fp32_product_ms": half_ms, "half_fp32_field_rel_err": half_err,
            "half_fp32_bytes": half_info["bytes"], "half_stored": bool(half_info["half"]),
            "dense_dynamics_s": ref_wall, "rows": rows}
    print(json.dumps(line), flush=True)


def run_hysteresis(args):
    """Standard problem 2 (Sec. 4.1): film L x L/5 x L/50 as 100 x 20 x 3
    tiles (n = 6,000), field along [1,1,1] descending from 0.08 Ms to -0.08 Ms
    in 4,000 steps, each value held 40 ns, LL form with the precession term
    dropped and alpha = 4000, as the paper.  One tensor serves the whole
    d / l_ex sweep (the point tensor is scale-invariant; exchange enters as
    (d_ref / d)^2), so the B = 8 films d / l_ex = 10 ... 45 run as one batch.
    Timed: the first `--values` values of the paper's schedule for each
    product (FP32 streaming, split BF16 and BF16 on the tensor cores); then a
    coarse loop (17 values, relaxed to torque 1e-3 or 40 ns) for the
    coercivity and remanence of each film."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    t = wl.sp2_film(100, 20, 3, d_lex=10.0)
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    d_lex = np.array([10.0, 15.0, 20.0, 25.0, 30.0, 35.0, 40.0, 45.0])
    B = len(d_lex)
    H = wl.sp2_fields(4001)
    opts = mt.ode_opts(rtol=1e-5, atol=1e-5, h0=1e-14, hmax=1e-10)
    m0 = np.tile(wl.m_noisy(t.n, wl.SP2_DIR, 1e-3, seed=0).astype(np.float32).ravel(), B)
    K = args.values
    rows = []
    # (8 simulations per pass: the FP32 tensor stores every block, the half
    # storage's product being faster for 1 or 2 simulations only)
    for prec, layout in (("f32", mt.MT_LAYOUT_STREAM_FULL), ("split", 1), ("bf16", 1)):
        T = mt.mt_demag_assemble_ex(tiles, prec, layout)
        p, keep = mt.llg_params(B, alpha=4000.0, form=mt.MT_FORM_LL, precess=0, exch_scale=(10.0 / d_lex) ** 2)
        I = mt.Integrator(T, p, opts, B=B)
        I.set_state(m0)
        I.hysteresis(wl.SP2_DIR, H[:1], 1e-12)  # warm-up: graph, first products
        I.set_state(m0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mavg, tau, hc, mr, st = I.hysteresis(wl.SP2_DIR, H[:K], 40e-9)
        wall = time.perf_counter() - t0
        rhs = sum(x["n_rhs"] for x in st)
        rows.append({"product": "%s_%s" % (prec, "dense" if layout == mt.MT_LAYOUT_DENSE else "stream"),
                     "wall_s": wall,
                     "values_x_sims_per_s": K * B / wall, "rhs_evals_per_s": rhs / wall,
                     "attempts_stiffest": st[0]["n_accept"] + st[0]["n_reject"],
                     "full_loop_hours": wall / K * len(H) / 3600.0})
        I.close()
        T.close()
    # coarse loop for coercivity and remanence (split BF16 products)
    T = mt.mt_demag_assemble_ex(tiles, "split", 1)
    p, keep = mt.llg_params(B, alpha=4000.0, form=mt.MT_FORM_LL, precess=0, exch_scale=(10.0 / d_lex) ** 2)
    I = mt.Integrator(T, p, opts, B=B)
    I.set_state(m0)
    Hc = wl.sp2_fields(args.coarse)
    t0 = time.perf_counter()
    mavg, tau, hc, mr, st = I.hysteresis(wl.SP2_DIR, Hc, 40e-9, tol=1e-3)
    coarse_wall = time.perf_counter() - t0
    loop = [{"d_lex": float(d_lex[b]), "hc_over_Ms": float(-hc[b] / wl.SP4_MS), "mr": [float(x) for x in mr[b]]}
            for b in range(B)]
    best = max(rows, key=lambda r: r["values_x_sims_per_s"])
    line = {"metric": "SP2 hysteresis field values x films per second (40 ns per value)",
            "value": best["values_x_sims_per_s"], "unit": "values*films/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "sp2_film_100x20x3_n6000_B8_dlex10-45", "tiles": t.n, "films": B,
                       "values_timed": K, "product": best["product"]},
            "rows": rows, "coarse_loop": {"values": int(args.coarse), "tol": 1e-3, "wall_s": coarse_wall,
                                          "films": loop}}
    print(json.dumps(line), flush=True)


def run_crossover(args):
    """Standard problem 3 (Sec. 4.2): cube with K_u = 0.1 K_m along z, the
    size at which the flower and the vortex state have equal energy, at
    several resolutions N^3, extrapolated by a fit L_cross = a N^b + c (the
    paper: c = L_inf = 8.477 +- 0.007 l_ex).  For each N one tensor serves all
    sizes (exchange factors), and each scan relaxes flower seeds (along z) and
    vortex seeds (core along x, across the easy axis; a core along z unwinds
    into the twisted flower at these sizes) at 8 sizes as one batch of 16 on
    the tensor cores (split BF16): a coarse scan
    over 7.5 ... 9.5 l_ex, then a fine one over +-0.15 l_ex around its
    crossing."""
    import torch
    from scipy.optimize import curve_fit
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    ctx = mt.mt_ctx_create(0)
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-10)
    res = [int(x) for x in args.resolutions.split(",")]
    rows = []
    t_all = time.perf_counter()
    for N in res:
        t = wl.cube(N, 1.0)
        tiles = mt.mt_tiles_create(ctx, t)
        tw = time.perf_counter()
        T = mt.mt_demag_assemble_ex(tiles, "split", 1)
        t_asm = time.perf_counter() - tw
        p, keep = mt.llg_params(16, alpha=4000.0, form=mt.MT_FORM_LL, precess=0)
        I = mt.Integrator(T, p, opts, B=16)
        lam = np.linspace(7.5, 9.5, 8)
        tw = time.perf_counter()
        eA, eB, lc, _, st = I.crossover(lam, wl.m_flower(t), wl.m_vortex(t, axis=0), 1e-4, 20e-9)
        rhs = sum(x["n_rhs"] for x in st)
        if not np.isfinite(lc):
            rows.append({"N": N, "tiles": t.n, "crossing": None})
            continue
        lam2 = np.linspace(lc - 0.15, lc + 0.15, 8)
        eA2, eB2, lc2, _, st2 = I.crossover(lam2, wl.m_flower(t), wl.m_vortex(t, axis=0), 1e-4, 20e-9)
        wall = time.perf_counter() - tw
        rhs += sum(x["n_rhs"] for x in st2)
        km = 0.5 * MU0 * float(t.Ms[0]) ** 2
        rows.append({"N": N, "tiles": t.n, "crossing": lc2 if np.isfinite(lc2) else lc, "coarse_crossing": lc,
                     "assemble_s": t_asm, "scan_s": wall, "rhs_evals": rhs, "rhs_evals_per_s": rhs / wall,
                     "e_flower_at_crossing_over_Km": float(np.interp(lc2, lam2, eA2) / km)
                     if np.isfinite(lc2) else None})
        I.close()
        T.close()
        print("N=%d: crossing %.4f l_ex (%.1f s)" % (N, rows[-1]["crossing"], wall), file=sys.stderr, flush=True)
    total = time.perf_counter() - t_all
    ok = [r for r in rows if r.get("crossing") is not None]
    fit = None
    if len(ok) >= 4:
        x = np.array([r["N"] for r in ok], np.float64)
        y = np.array([r["crossing"] for r in ok])
        try:
            popt, pcov = curve_fit(lambda n, a, b, c: a * n ** b + c, x, y, p0=(1.0, -1.0, 8.5), maxfev=20000)
            fit = {"a": float(popt[0]), "b": float(popt[1]), "L_inf": float(popt[2]),
                   "L_inf_sigma": float(np.sqrt(pcov[2, 2])), "paper_L_inf": 8.477, "paper_sigma": 0.007}
        except RuntimeError as e:
            fit = {"error": str(e)}
    line = {"metric": "SP3 flower/vortex crossover", "value": fit["L_inf"] if fit and "L_inf" in fit else None,
            "unit": "l_ex (L_inf of the fit)", "n_gpus": 1, "higher_is_better": None, "data": "synthetic",
            "config": {"workload": "sp3_cube_N%s_split_dense" % "-".join(map(str, res)), "sizes_per_scan": 8,
                       "scans_per_N": 2},
            "wall_s": total, "rows": rows, "fit": fit}
    print(json.dumps(line), flush=True)


def run_tetra(args):
    """Tetrahedral tiles (Sec. 3): a box of 20 x 20 x 10 cells, 6 jittered
    tetrahedra each (n = 24,000), against the cuboid film of the same tile
    count: FP64 assembly rate of the face-charge tensor, the FP32 streaming
    product on the tetrahedral tensor (the same kernel: layouts do not care
    about the tile shape), and RHS evals/s of the integrator."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    ctx = mt.mt_ctx_create(0)
    verts, tets = wl.tetra_box(20, 20, 10, size=(200e-9, 200e-9, 50e-9), jitter=0.1, seed=9)
    n = len(tets)
    out = {}
    for name, make in (("tetra", lambda: mt.mt_tiles_create_tetra(ctx, verts, tets, wl.SP4_MS, wl.SP4_AEX, 0.0)),
                       ("cuboid", lambda: mt.mt_tiles_create(ctx, wl.film(240, 100, 1, size=(600e-9, 250e-9,
                                                                                              3e-9))))):
        tiles = make()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # all 6 entry planes for both: the single-layer film would store 4
        T = mt.mt_demag_assemble_ex(tiles, "f32", mt.MT_LAYOUT_STREAM6)
        torch.cuda.synchronize()
        t_asm = time.perf_counter() - t0
        m = torch.tensor(wl.m_random(tiles.n, seed=1).astype(np.float32).ravel(), device="cuda")
        H = torch.empty_like(m)
        for _ in range(3):
            mt.mt_demag_field(T, m, H)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            mt.mt_demag_field(T, m, H)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        p, keep = mt.llg_params(1, alpha=0.1)
        I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-5, atol=1e-5, h0=1e-15, hmax=1e-11))
        I.set_state(wl.m_noisy(tiles.n, (1, 1, 1), 1e-2, seed=1).astype(np.float32).ravel())
        I.step(5)
        torch.cuda.synchronize()
        s = torch.cuda.ExternalStream(I.stream_handle())
        e0.record(s)
        I.step(100)
        e1.record(s)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / 100
        out[name] = {"tiles": tiles.n, "assemble_s": t_asm, "blocks_per_s": tiles.n ** 2 / t_asm,
                     "product_ms": ms, "product_gbs": f32_alg_bytes(T.info(), tiles.n) / (ms * 1e-3) / 1e9,
                     "stored_half": bool(T.info()["half"]),
                     "rhs_evals_per_s": 6.0 / (step_ms * 1e-3)}
        I.close()
        T.close()
    line = {"metric": "tetrahedral tiles: RHS evals/s", "value": out["tetra"]["rhs_evals_per_s"],
            "unit": "RHS evals/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "tetra_box_20x20x10x6_n%d_f32" % n}, "tetra": out["tetra"],
            "cuboid_same_n": out["cuboid"]}
    print(json.dumps(line), flush=True)


def run_sp4(args):
    """Standard problem 4 as the paper times it (Sec. 4.3): the film
    500 x 125 x 3 nm on grids [20n, 5n, 1], n = 1 ... 9; the s-state is
    relaxed first (untimed), then the dynamic part -- 1 ns under field 1 and
    under field 2, LL form with the paper's gamma = 2.21e5 and
    alpha = 4.42e3, rtol = atol = 1e-6 -- is timed: each field as its own
    simulation (as the paper runs them), both fields as one batch of 2, and
    the FP64 oracle on the host cores for the smallest grids."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    ctx = mt.mt_ctx_create(0)
    fields = np.stack([FIELD1, np.array([-35.5e-3, -6.3e-3, 0.0]) / MU0])
    opts = dict(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11)
    rows = []
    for k in range(1, args.sp4_max + 1):
        t = wl.film(20 * k, 5 * k, 1)
        tiles = mt.mt_tiles_create(ctx, t)
        T = mt.mt_demag_assemble(tiles, "f32")
        p0, k0 = mt.llg_params(1, alpha=0.5)
        I = mt.Integrator(T, p0, mt.ode_opts(rtol=1e-5, atol=1e-5))
        I.set_state(wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=0).astype(np.float32).ravel())
        I.run(5e-9, 1, check=False)
        s_state = I.get_state()[0].copy()
        I.close()
        row = {"n": k, "grid": [20 * k, 5 * k, 1], "tiles": t.n}
        single = 0.0
        rhs = 0
        for f in range(2):
            p, keep = mt.llg_params(1, gamma=2.21e5, alpha=4.42e3, Ha=fields[f], form=mt.MT_FORM_LL)
            J = mt.Integrator(T, p, mt.ode_opts(**opts))
            J.set_state(s_state.ravel())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, mavg, st = J.run(1e-9, 100, check=False)
            single += time.perf_counter() - t0
            rhs += st[0]["n_rhs"]
            if f == 0:
                row["mavg_1ns_field1"] = [float(x) for x in mavg[-1, 0]]
            J.close()
        p, keep = mt.llg_params(2, gamma=2.21e5, alpha=4.42e3, Ha=fields, form=mt.MT_FORM_LL)
        J = mt.Integrator(T, p, mt.ode_opts(**opts), B=2)
        J.set_state(np.tile(s_state.ravel(), 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J.run(1e-9, 100, check=False)
        batched = time.perf_counter() - t0
        J.close()
        row.update({"gpu_fields_one_by_one_s": single, "gpu_fields_batched_s": batched, "rhs_evals": rhs})
        if k <= args.sp4_cpu_max:
            # CPU baseline of this workload: the FP64 oracle, as it stands
            import oracle
            md = oracle.Model.from_tiles(t)
            t0 = time.perf_counter()
            for f in range(2):
                oracle.integrate(md, s_state.astype(np.float64),
                                 oracle.llg_params(gamma=2.21e5, alpha=4.42e3, Ha=fields[f], form=1),
                                 oracle.ode_opts(**opts), 0.0, 1e-9, 1)
            row["cpu_baseline"] = {"value": time.perf_counter() - t0, "unit": "s", "cores": oracle.num_threads(),
                                   "kind": "oracle", "sample": "fields 1 and 2, 1 ns each, FP64 stored tensor"}
        rows.append(row)
        print("SP4 n=%d (%d tiles): GPU %.2f s (batched %.2f s)%s" % (
            k, t.n, single, batched,
            "" if "cpu_baseline" not in row else ", CPU oracle %.1f s" % row["cpu_baseline"]["value"]),
            file=sys.stderr, flush=True)
        T.close()
    line = {"metric": "SP4 dynamic part wall time (fields 1 and 2, 1 ns each)", "value": rows[-1]["gpu_fields_one_by_one_s"],
            "unit": "s (n = %d)" % rows[-1]["n"], "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "dtype": "f32", "config": {"workload": "sp4_film_grids_20n_5n_1_n1-%d" % args.sp4_max}, "rows": rows}
    print(json.dumps(line), flush=True)


def run_c1(args):
    """The plain method at its smallest: the film 500 x 125 x 3 nm as
    40 x 10 x 1 tiles (n = 400, FP32 tensor 3.8 MB, resident in L2), the
    seed-0 state relaxed at alpha = 0.5 to a torque below 1e-6, then 1 ns of
    Gilbert dynamics at alpha = 0.02 under field 1 with <m> every 1 ps.  At
    this size a right-hand side is bound by kernel launch and grid-wide
    dependency latency, not by HBM: reported as RHS evals/s and time per
    step, beside the FP64 oracle running the same two phases on the host."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    ctx = mt.mt_ctx_create(0)
    t = wl.film(40, 10, 1)
    m0 = wl.m_noisy(t.n, (1, 1, 1), 1e-3, seed=0).astype(np.float32)
    tiles = mt.mt_tiles_create(ctx, t)
    t0 = time.perf_counter()
    T = mt.mt_demag_assemble(tiles, "f32")
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    relax_o = dict(rtol=1e-5, atol=1e-5)
    dyn_o = dict(rtol=1e-6, atol=1e-6)
    p_r, k_r = mt.llg_params(1, alpha=0.5)
    p_d, k_d = mt.llg_params(1, alpha=0.02, Ha=FIELD1)

    def phases(path):
        res = {}
        for rep in range(2):  # the first pass warms up (graph capture, autotuning)
            I = mt.Integrator(T, p_r, mt.ode_opts(**relax_o))
            I.set_path(path)
            I.set_state(m0.ravel())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s_r, st_r = I.relax(1e-6, 5e-9, check=False)
            t_relax = time.perf_counter() - t0
            m_rel = I.get_state()[0].copy()
            I.close()
            J = mt.Integrator(T, p_d, mt.ode_opts(**dyn_o))
            J.set_path(path)
            J.set_state(m_rel.ravel())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, mavg, st_d = J.run(1e-9, 1000, check=False)
            t_dyn = time.perf_counter() - t0
            J.close()
            res = {"relax_s": t_relax, "relax_status": int(s_r), "relax_tau": st_r[0]["tau"],
                   "relax_rhs": st_r[0]["n_rhs"], "dynamics_s": t_dyn, "dynamics_rhs": st_d[0]["n_rhs"],
                   "dynamics_accepted": st_d[0]["n_accept"]}
        # the step itself: fixed steps back to back
        F = mt.Integrator(T, p_d, mt.ode_opts(fixed_h=1e-13))
        F.set_path(path)
        F.set_state(m0.ravel())
        F.step(args.warmup)
        torch.cuda.synchronize()
        steps = max(args.steps, 100)
        t0 = time.perf_counter()
        F.step(steps)
        torch.cuda.synchronize()
        res["ms_per_fixed_step"] = (time.perf_counter() - t0) * 1e3 / steps
        res["fixed_step_rhs_evals_per_s"] = 6e3 / res["ms_per_fixed_step"]
        F.close()
        res["rhs_evals_per_s"] = (res["relax_rhs"] + res["dynamics_rhs"]) / (res["relax_s"] + res["dynamics_s"])
        return res, mavg

    res, mavg = phases(mt.MT_PATH_PERSISTENT)
    graph, _ = phases(mt.MT_PATH_GRAPH)
    line = {"metric": "LLG RHS evals/s", "value": res["rhs_evals_per_s"], "unit": "RHS evals/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "film_40x10x1_n400_relax_then_1ns", "n": t.n, "path": "persistent"},
            "assembly_s": t_asm, **res, "graph_path": graph}
    if not args.no_cpu_baseline:
        # CPU baseline of this workload: the FP64 oracle, as it stands
        import oracle
        md = oracle.Model.from_tiles(t)
        t0 = time.perf_counter()
        s1, m_o, st1 = oracle.relax(md, m0.astype(np.float64), oracle.llg_params(alpha=0.5),
                                       oracle.ode_opts(**relax_o), 1e-6, 5e-9)
        s2, _, trace, st2 = oracle.integrate(md, m_o, oracle.llg_params(alpha=0.02, Ha=FIELD1),
                                             oracle.ode_opts(**dyn_o), 0.0, 1e-9, 1000)
        wall = time.perf_counter() - t0
        n_rhs = st1["n_rhs"] + st2["n_rhs"]
        line["cpu_baseline"] = {"value": n_rhs / wall, "unit": "RHS evals/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": "the whole workload (relax + 1 ns), FP64 stored tensor",
                                "wall_s": wall, "mavg_trace_max_dev_vs_gpu": float(np.abs(trace[:, :] - mavg[:, 0]).max())}
    print(json.dumps(line), flush=True)


def _product_times(mt, T, mg, H, B, reps=20):
    """Average time of one product (CUDA events): standalone calls, and six
    back to back inside one CUDA graph as the step graph holds them (None
    if the capture fails)."""
    import torch
    cur = torch.cuda.current_stream()
    for _ in range(3):
        mt.mt_demag_field(T, mg, H, B=B, stream=cur)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(reps):
        mt.mt_demag_field(T, mg, H, B=B, stream=cur)
    e1.record(cur)
    torch.cuda.synchronize()
    alone = e0.elapsed_time(e1) / reps
    graph = None
    try:
        gs = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs, capture_error_mode="thread_local"):
            for _ in range(6):
                mt.mt_demag_field(T, mg, H, B=B, stream=gs)
        with torch.cuda.stream(gs):
            g.replay()
            torch.cuda.synchronize()
            e0.record(gs)
            for _ in range(max(3, reps // 2)):
                g.replay()
            e1.record(gs)
        torch.cuda.synchronize()
        graph = e0.elapsed_time(e1) / (6 * max(3, reps // 2))
        del g
        if graph < 0.5 * alone:
            graph = None
    except Exception as e:
        print("in-graph product timing unavailable: %s" % e, file=sys.stderr)
    return alone, graph


def _time_attempts(I, steps, warmup):
    """Device time (ms) of `steps` RK(4,5) attempts on the integrator's stream."""
    import torch
    stream = torch.cuda.ExternalStream(I.stream_handle())
    I.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    I.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_cube(args):
    """Config 2's cube (standard problem 3 shape, Sec. 4.2): edge 20 l_ex as
    20 x 20 x 20 tiles (n = 8,000), K_u = 0.1 K_m along z, FP32 streaming
    tensor (6 entry planes, 1.54 GB, larger than L2).  The flower seed and the
    vortex seed (core across the easy axis) run as one batch of 2, so every
    tensor chunk read serves both.  Timed on the device: RK(4,5) attempts
    (6 RHS each) -> RHS evals/s, and the product alone (standalone and six in
    a CUDA graph) against the HBM roofline.  Then both states are relaxed to
    a torque below --tol (1e-6 asked by the workload; an explicit integrator
    in FP32 state has a torque floor near 10 x atol, so the call either
    converges or returns MT_ENOCONV at the time cap with the attained torque),
    and their energies are reported.  CPU baseline: the FP64 oracle's RHS with
    its stored tensor on the host cores."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    t = wl.cube(20, 20.0)
    n = t.n
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    tw = time.perf_counter()
    T = mt.mt_demag_assemble(tiles, "f32")
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - tw
    info = T.info()
    m0 = np.stack([wl.m_flower(t), wl.m_vortex(t, axis=0)]).astype(np.float32)
    B = 2
    p, keep = mt.llg_params(B, alpha=0.5)
    opts = mt.ode_opts(rtol=args.cube_rtol, atol=args.cube_rtol, h0=1e-14, hmax=1e-11)
    I = mt.Integrator(T, p, opts, B=B)
    I.set_state(m0.ravel())
    with ClockSampler(0) as clk:
        ms = _time_attempts(I, args.steps, args.warmup)
    value = 6.0 * args.steps * B / (ms * 1e-3)
    mg = torch.tensor(m0.ravel(), device="cuda")
    H = torch.empty_like(mg)
    alone, graph = _product_times(mt, T, mg, H, B)
    alg = f32_alg_bytes(info, n)  # the stored FP32 entries, read once per group of <= 4 simulations
    peaks, kind = _peaks()
    peak = float(peaks["hbm_gbs"])
    launch = graph if graph is not None else alone
    # relax both states
    I.set_state(m0.ravel())
    tw = time.perf_counter()
    s, st = I.relax(args.tol, args.cube_tmax, check=False)
    relax_wall = time.perf_counter() - tw
    m_rel = I.get_state()
    E = mt.mt_energy(T, p, torch.tensor(m_rel.ravel(), device="cuda"), B=B)
    km = 0.5 * MU0 * float(t.Ms[0]) ** 2
    vol = float(np.prod(t.edge, axis=1).sum())
    states = []
    for b, name in enumerate(("flower", "vortex")):
        states.append({"seed": name, "status": int(st[b]["status"]),
                       "converged": st[b]["status"] == mt.MT_OK, "tau": st[b]["tau"], "t_s": st[b]["t"],
                       "attempts": st[b]["n_accept"] + st[b]["n_reject"],
                       "energy_density_over_Km": float(E[b, 0] / vol / km),
                       "mean_m": [float(x) for x in np.mean(m_rel[b], axis=0)]})
    I.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        md = oracle.Model.from_tiles(t)
        pp = oracle.llg_params(alpha=0.5)
        x = m0[0].astype(np.float64)
        oracle.llg_rhs(md, x, pp)
        tw = time.perf_counter()
        for _ in range(3):
            oracle.llg_rhs(md, x, pp)
        cpu = {"value": 3.0 / (time.perf_counter() - tw), "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "3 RHS of the n=8,000 cube, FP64 tensor assembled once (untimed)"}
    line = {"metric": METRIC + " (cube, 2 simulations)", "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sp3_cube_20x20x20_n8000_f32_flower_vortex", "tiles": n, "sims": B,
                       "step": "one Dormand-Prince attempt of both simulations = 12 RHS",
                       "l2": "inputs larger than L2 (tensor %.2f GB)" % (info["bytes"] / 1e9)},
            "assemble_s": t_asm,
            "roofline": {"bound": "hbm", "achieved": alg / (launch * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (launch * 1e-3) / 1e9 / peak, "traffic": None,
                         "kernel": "k_matvec_half<f32> + k_half_cols" if info["half"] else "k_matvec<f32>",
                         "stored": "upper triangle of blocks (N_ij = N_ji: tiles of one shape)" if info["half"]
                         else "every block",
                         "algorithmic_bytes_per_launch": alg, "launch_ms": launch,
                         "launch_ms_source": "six products in one CUDA graph" if graph is not None else "standalone",
                         "standalone_launch_ms": alone, "peak_kind": kind},
            "relax": {"tol": args.tol, "t_max_s": args.cube_tmax, "rtol_atol": args.cube_rtol, "alpha": 0.5,
                      "wall_s": relax_wall, "status": int(s), "states": states},
            "cpu_baseline": cpu, "gpu_launches": 13 * args.steps, "clocks": clk.summary()}
    T.close()
    tiles.close()
    print(json.dumps(line), flush=True)


def run_graded(args):
    """Config 3: the graded film 1000 x 250 x 5 nm as 200 x 50 x 3 tiles
    (n = 30,000; column, row and layer widths varied 2^u, u ~ U(-1, 1), so no
    translation invariance: every block is evaluated, 9e8 of them).  For each
    storage precision of the streaming layout (FP32; BF16 with per-block
    scales; split BF16 hi + lo): FP64 assembly time, stored bytes, the product
    alone (standalone and six in a CUDA graph) against the HBM roofline,
    RHS evals/s of RK(4,5) attempts (device events), and the field error
    against the FP64 oracle on sampled rows (uniform and random m), which the
    matrix-free oracle computes one by one (the FP64 tensor, 43 GB, is not
    stored on the host).  CPU baseline: those oracle rows, timed and scaled to
    one whole product."""
    import torch
    torch.cuda.set_device(0)
    import oracle
    from paper_2107_05364_gb300 import binding as mt
    t = wl.graded_film(200, 50, 3, seed=0)
    n = t.n
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    rows = np.unique(np.concatenate([[0, n - 1, 15000], np.random.default_rng(4).integers(0, n, 36)]))
    cases = {"uniform": np.tile(np.array([[0.6, 0.48, 0.64]]), (n, 1)).astype(np.float32),
             "random": wl.m_random(n, seed=1).astype(np.float32)}
    tw = time.perf_counter()
    refs = {k: oracle.demag_field_rows(t.centre, t.edge, t.Ms, m.astype(np.float64), rows) for k, m in cases.items()}
    t_rows = (time.perf_counter() - tw) / (2 * len(rows))
    m0 = wl.m_noisy(n, (1, 1, 1), 1e-3, seed=0).astype(np.float32)
    p, keep = mt.llg_params(1, alpha=0.02, Ha=FIELD1)
    peaks, kind = _peaks()
    peak = float(peaks["hbm_gbs"])
    out = {}
    for prec in ("f32", "bf16", "split"):
        torch.cuda.synchronize()
        tw = time.perf_counter()
        T = mt.mt_demag_assemble(tiles, prec)
        torch.cuda.synchronize()
        t_asm = time.perf_counter() - tw
        info = T.info()
        errs = {}
        for name, m in cases.items():
            mg = torch.tensor(m.ravel(), device="cuda")
            H = torch.empty_like(mg)
            mt.mt_demag_field(T, mg, H)
            torch.cuda.synchronize()
            Hg = H.cpu().numpy().reshape(-1, 3)[rows]
            errs[name] = float(np.linalg.norm(Hg - refs[name]) / np.linalg.norm(refs[name]))
        mg = torch.tensor(m0.ravel(), device="cuda")
        H = torch.empty_like(mg)
        alone, graph = _product_times(mt, T, mg, H, 1, reps=10)
        launch = graph if graph is not None else alone
        # algorithmic bytes: every stored value (and BF16 scale byte) read once
        per_block = {"f32": 4.0, "bf16": 2.0, "split": 4.0}[prec] * (6 if info["planes"] in (6, 12) else 4)
        if prec == "bf16":
            per_block += 1.0
        alg = per_block * n * n
        I = mt.Integrator(T, p, mt.ode_opts(rtol=1e-6, atol=1e-6, h0=1e-14, hmax=1e-11))
        I.set_state(m0.ravel())
        steps = max(5, args.steps // 4)
        ms = _time_attempts(I, steps, 3)
        I.close()
        out[prec] = {"assemble_s": t_asm, "blocks_per_s": n * n / t_asm, "tensor_gb": info["bytes"] / 1e9,
                     "planes": info["planes"], "near_blocks": info["near_blocks"],
                     "rhs_evals_per_s": 6.0 * steps / (ms * 1e-3), "ms_per_attempt": ms / steps,
                     "product_ms": launch, "product_ms_standalone": alone,
                     "algorithmic_bytes_per_launch": alg, "hbm_frac": alg / (launch * 1e-3) / 1e9 / peak,
                     "field_rel_err_sampled_rows": errs}
        T.close()
        print("graded %s: %.0f RHS/s, product %.3f ms (%.2f of HBM), field err %s" % (
            prec, out[prec]["rhs_evals_per_s"], launch, out[prec]["hbm_frac"], errs), file=sys.stderr, flush=True)
    f = out["f32"]
    line = {"metric": METRIC + " (graded film, by storage precision)", "value": f["rhs_evals_per_s"],
            "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "graded_film_200x50x3_n30000", "tiles": n, "sims": 1,
                       "l2": "inputs larger than L2 (FP32 tensor %.1f GB)" % f["tensor_gb"]},
            "roofline": {"bound": "hbm", "achieved": f["algorithmic_bytes_per_launch"] / (f["product_ms"] * 1e-3) / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": f["hbm_frac"], "traffic": None,
                         "kernel": "k_matvec<f32>", "launch_ms": f["product_ms"], "peak_kind": kind},
            "by_precision": out, "sampled_rows": int(len(rows)),
            "cpu_baseline": {"value": 1.0 / (t_rows * n), "unit": UNIT + " (demag part, estimated)",
                             "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d rows of the matrix-free FP64 product, timed and scaled to n = %d rows"
                                       % (2 * len(rows), n)}}
    tiles.close()
    print(json.dumps(line), flush=True)


def run_profile(args):
    """One kernel family on a chosen film, for profiler captures: the
    2.5 x 2.5 x 3 nm cell film of nx x ny x nz tiles; --what field (the
    product, `--reps` calls), step (RK(4,5) attempts through the integrator,
    on --path), or assemble; --layout stream / full (stream without the
    half storage) / stream6 / dense; --threshold F applies the Sec. 4.3.1
    sparse tensor.  Prints the average time per call from CUDA events
    (meaningless under a profiler)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2107_05364_gb300 import binding as mt
    prec = args.prec or "f32"
    t = wl.film(args.nx, args.ny, args.nz, size=(2.5e-9 * args.nx, 2.5e-9 * args.ny, 3e-9 * args.nz))
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.what == "assemble":
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.reps):
            mt.mt_demag_assemble(tiles, prec).close()
        e1.record()
        torch.cuda.synchronize()
        print("assemble n=%d: %.3f ms" % (t.n, e0.elapsed_time(e1) / args.reps))
        return
    layout = {"stream": mt.MT_LAYOUT_STREAM, "full": mt.MT_LAYOUT_STREAM_FULL, "half": mt.MT_LAYOUT_STREAM_HALF,
              "dense": mt.MT_LAYOUT_DENSE, "stream6": mt.MT_LAYOUT_STREAM6}[args.layout]
    if args.threshold is not None and layout == mt.MT_LAYOUT_STREAM:
        layout = mt.MT_LAYOUT_STREAM_FULL  # thresholding needs every block stored
    T = mt.mt_demag_assemble_ex(tiles, prec, layout)
    if args.threshold is not None:
        S, thr, kept = mt.mt_tensor_threshold(T, args.threshold)
        T.close()
        T = S
        print("threshold %.2f: t = %.4g, kept elements %d, sparse bytes %d" % (args.threshold, thr, kept,
                                                                                T.info()["bytes"]))
    B = args.sims
    m = np.stack([wl.m_random(t.n, seed=b) for b in range(B)]).astype(np.float32)
    if args.what == "field":
        mg = torch.tensor(m.ravel(), device="cuda")
        H = torch.empty_like(mg)
        mt.mt_demag_field(T, mg, H, B=B)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.reps):
            mt.mt_demag_field(T, mg, H, B=B)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        print("field n=%d B=%d prec=%s: %.4f ms/call (%.0f GB/s of stored bytes)" % (
            t.n, B, prec, ms, T.info()["bytes"] / (ms * 1e-3) / 1e9))
    else:
        p, keep = mt.llg_params(B, alpha=0.02, Ha=FIELD1)
        I = mt.Integrator(T, p, mt.ode_opts(), B=B)
        if args.path != "auto":
            I.set_path(mt.MT_PATH_GRAPH if args.path == "graph" else mt.MT_PATH_PERSISTENT)
        I.set_state(m.ravel())
        ms = _time_attempts(I, args.reps, 1)
        print("step n=%d B=%d path=%d: %.4f ms/attempt" % (t.n, B, I.path(), ms / args.reps))


def mt_pad(B):
    bp = 16
    while bp < B and bp < 128:
        bp *= 2
    return bp


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the compact batched and serving legs")
    ap.add_argument("--workload", default="film", choices=["film", "batched", "serving", "threshold", "hysteresis",
                                                                   "crossover", "tetra", "sp4", "c1", "cube",
                                                                   "graded", "profile"])
    ap.add_argument("--sp4-max", type=int, default=9, help="sp4: largest n of the [20n, 5n, 1] grids")
    ap.add_argument("--sp4-cpu-max", type=int, default=3, help="sp4: largest n the CPU oracle runs")
    ap.add_argument("--resolutions", default="8,10,12,16,20,24", help="crossover: cube tiles per edge")
    ap.add_argument("--values", type=int, default=2, help="hysteresis: field values of the paper's schedule timed")
    ap.add_argument("--coarse", type=int, default=17, help="hysteresis: values of the coarse loop")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests of the Poisson stream")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--t-cap", type=float, default=1e-9, help="serving: simulated-time cap per job, s")
    ap.add_argument("--batch-slots", type=int, default=4, help="serving: slots per resident geometry")
    ap.add_argument("--serve-prec", default="f32", choices=["f32", "bf16", "split"],
                    help="serving: f32 streaming engines, or bf16 / split dense (tensor cores)")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0, help="serving: HBM budget of the cache")
    ap.add_argument("--serve-rtol", type=float, default=1e-6, help="serving: rtol = atol of the integrator")
    ap.add_argument("--serve-limit", type=float, default=60.0,
                    help="serving: seconds after the last arrival a pass may run")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--prec", default=None, choices=["f32", "split", "bf16"],
                    help="batched: split (default) or bf16; profile: f32 (default), bf16 or split")
    ap.add_argument("--tol", type=float, default=1e-6, help="cube: relax torque tolerance")
    ap.add_argument("--cube-tmax", type=float, default=5e-9, help="cube: relax time cap, s")
    ap.add_argument("--cube-rtol", type=float, default=1e-7, help="cube: rtol = atol of the integrator")
    # profile: one kernel family on a chosen film (for ncu captures)
    ap.add_argument("--nx", type=int, default=100)
    ap.add_argument("--ny", type=int, default=40)
    ap.add_argument("--nz", type=int, default=1)
    ap.add_argument("--what", default="field", choices=["field", "step", "assemble"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sims", type=int, default=1)
    ap.add_argument("--layout", default="stream", choices=["stream", "full", "half", "dense", "stream6"])
    ap.add_argument("--threshold", type=float, default=None)
    ap.add_argument("--path", default="auto", choices=["auto", "graph", "persistent"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        args.prec = args.prec or "split"
        if args.prec == "f32":
            ap.error("--workload batched runs the tensor-core product: --prec split or bf16")
        run_batched(args)
    elif args.workload == "cube":
        run_cube(args)
    elif args.workload == "graded":
        run_graded(args)
    elif args.workload == "profile":
        run_profile(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "threshold":
        run_threshold(args)
    elif args.workload == "hysteresis":
        run_hysteresis(args)
    elif args.workload == "crossover":
        run_crossover(args)
    elif args.workload == "tetra":
        run_tetra(args)
    elif args.workload == "sp4":
        run_sp4(args)
    elif args.workload == "c1":
        run_c1(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
