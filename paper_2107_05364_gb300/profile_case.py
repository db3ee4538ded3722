"""Small driver for profiling one kernel family on a chosen film size.

    python -m paper_2107_05364_gb300.profile_case --nx 100 --ny 40 --prec f32 --what field --reps 3

--what field    : mt_demag_field R times (prep + streaming product [+ near])
--what step     : R Runge-Kutta attempts through the integrator
--path P        : step execution: auto (default), graph (one CUDA-graph replay
                  per attempt) or persistent (one cooperative kernel per call)
--what assemble : tensor assembly only
--layout dense  : 9-entry BF16 / split tensor for the batched tensor-core product
--layout stream6: the streaming layout with all 6 entry planes even for a
                  single-layer film (which otherwise stores 4)
--threshold F   : drop the smallest fraction F of the elements (Sec. 4.3.1) and
                  apply the sparse tensor (FP32, streaming layout first)
Prints the average time per call measured with CUDA events (not meaningful
under a profiler).
"""
from __future__ import annotations

import argparse
import math

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=100)
    ap.add_argument("--ny", type=int, default=40)
    ap.add_argument("--nz", type=int, default=1)
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--what", default="field", choices=["field", "step", "assemble"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--B", type=int, default=1)
    ap.add_argument("--layout", default="stream", choices=["stream", "dense", "stream6"])
    ap.add_argument("--threshold", type=float, default=None)
    ap.add_argument("--path", default="auto", choices=["auto", "graph", "persistent"])
    a = ap.parse_args()

    import torch

    from . import binding as mt
    from . import workloads as wl

    t = wl.film(a.nx, a.ny, a.nz, size=(2.5e-9 * a.nx, 2.5e-9 * a.ny, 3e-9 * a.nz))
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.what == "assemble":
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            T = mt.mt_demag_assemble(tiles, a.prec)
            T.close()
        e1.record()
        torch.cuda.synchronize()
        print("assemble n=%d: %.3f ms" % (t.n, e0.elapsed_time(e1) / a.reps))
        return
    layout = {"stream": mt.MT_LAYOUT_STREAM, "dense": mt.MT_LAYOUT_DENSE, "stream6": mt.MT_LAYOUT_STREAM6}[a.layout]
    T = mt.mt_demag_assemble_ex(tiles, a.prec, layout)
    if a.threshold is not None:
        S, thr, kept = mt.mt_tensor_threshold(T, a.threshold)
        T.close()
        T = S
        print("threshold %.2f: t = %.4g, kept elements %d, sparse bytes %d" % (a.threshold, thr, kept, T.info()["bytes"]))
    m = np.stack([wl.m_random(t.n, seed=b) for b in range(a.B)]).astype(np.float32)
    if a.what == "field":
        mg = torch.tensor(m.ravel(), device="cuda")
        H = torch.empty_like(mg)
        mt.mt_demag_field(T, mg, H, B=a.B)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            mt.mt_demag_field(T, mg, H, B=a.B)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        gbs = 4.0 * T.info()["planes"] * t.n * t.n * a.B / (ms * 1e-3) / 1e9 if a.prec == "f32" else float("nan")
        if a.threshold is not None:
            gbs = T.info()["bytes"] * a.B / (ms * 1e-3) / 1e9
        print("field n=%d B=%d prec=%s: %.4f ms/call (%.0f GB/s algorithmic for f32)" % (t.n, a.B, a.prec, ms, gbs))
    else:
        p, keep = mt.llg_params(a.B, alpha=0.02, Ha=np.array([-24.6e-3, 4.3e-3, 0.0]) / (4e-7 * math.pi))
        I = mt.Integrator(T, p, mt.ode_opts(), B=a.B)
        if a.path != "auto":
            I.set_path(mt.MT_PATH_GRAPH if a.path == "graph" else mt.MT_PATH_PERSISTENT)
        I.set_state(m.ravel())
        I.step(1)
        torch.cuda.synchronize()
        s = torch.cuda.ExternalStream(I.stream_handle())
        e0.record(s)
        I.step(a.reps)
        e1.record(s)
        torch.cuda.synchronize()
        print("step n=%d B=%d path=%d: %.4f ms/attempt" % (t.n, a.B, I.path(), e0.elapsed_time(e1) / a.reps))


if __name__ == "__main__":
    main()
