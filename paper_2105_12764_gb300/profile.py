"""Per-kernel timing of one decomposition + recomposition.

    python -m paper_2105_12764_gb300.profile --form fp64 --shape 513 [--reps 3]

prints every kernel role (level pass, solves, interpolation, ...) with its
CUDA-event time and the achieved bandwidth / flop rate of its algorithmic
work (mgr_profile), then the graph-replayed decompose and recompose times.
With --plain it only runs the operations (no event brackets): a clean target
for an external profiler.

    python -m paper_2105_12764_gb300.profile --fp64-rate

measures the FP64 FMA throughput of cuda:0 (mgr_fp64_fma_rate), the
denominator of the plain FP64 form's roofline.

    python -m paper_2105_12764_gb300.profile --batch 4096 [--form fp32] [--reps 1]

submits the batched workload (the given number of uneven 2D / 3D fields,
element counts log-uniform on [17^2, 129^3], half on stretched coordinates)
once to autotune and capture it, then times `reps` decompose + recompose
submits; only those submits run between cudaProfilerStart and
cudaProfilerStop (an external profiler started with profiling off captures
exactly their launches).
"""
import argparse
import os
import sys

sys.path.append(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import paper_2105_12764_gb300 as mgr

    ap = argparse.ArgumentParser()
    ap.add_argument("--form", choices=["fp64", "fp32", "mixed"], default="fp64")
    ap.add_argument("--shape", default="513", help="n (cube) or n0,n1,n2")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--plain", action="store_true")
    ap.add_argument("--packed", action="store_true", help="class-packed decompose / recompose")
    ap.add_argument("--batch", type=int, default=0, help="batched workload of this many fields")
    ap.add_argument("--fp64-rate", action="store_true", help="measured FP64 FMA throughput of cuda:0")
    a = ap.parse_args()
    if a.fp64_rate:
        rates = [mgr.fp64_fma_rate(0) for _ in range(3)]
        print(f"FP64 FMA rate: {max(rates) / 1e12:.4f} T FMA/s = {2 * max(rates) / 1e12:.4f} TFLOP/s "
              f"(three measurements: {', '.join(f'{r / 1e12:.4f}' for r in rates)} T FMA/s)")
        return
    if a.batch:
        return batch_main(a)
    shape = tuple(int(v) for v in a.shape.split(","))
    if len(shape) == 1:
        shape = shape * 3
    dtype = mgr.MGR_F64 if a.form == "fp64" else mgr.MGR_F32
    prec = mgr.MGR_PREC_MIXED if a.form == "mixed" else mgr.MGR_PREC_NATIVE
    td = torch.float64 if dtype == mgr.MGR_F64 else torch.float32
    ctx = mgr.Context(0)
    plan = mgr.Plan(ctx, shape, None, -1, dtype, prec)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(shape, dtype=td, device="cuda", generator=g)
    y, z = torch.empty_like(x), torch.empty_like(x)
    ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    L = plan.levels
    if a.packed:
        dec = lambda: plan.decompose_packed(x, y, ws)  # noqa: E731
        rec = lambda: plan.recompose_packed(y, L + 1, z, ws)  # noqa: E731
        ops = ((mgr.MGR_OP_DECOMPOSE_PACKED, (x, y)), (mgr.MGR_OP_RECOMPOSE_PACKED, (y, z)))
    else:
        dec = lambda: plan.decompose(x, y, ws)  # noqa: E731
        rec = lambda: plan.recompose(y, z, ws)  # noqa: E731
        ops = ((0, (x, y)), (1, (y, z)))
    if a.plain:
        for _ in range(a.reps):
            dec()
            rec()
        torch.cuda.synchronize()
        print(f"done: round trip max error {float((z - x).abs().max()):.3e}")
        return
    for _ in range(2):
        dec()
        rec()
    torch.cuda.synchronize()
    agg = {}
    for _ in range(a.reps):
        for op, (src, dst) in ops:
            for r in plan.profile(op, src, dst, ws):
                e = agg.setdefault((r["name"], r["level"]), [0.0, 0, r["bytes"], r["flops"]])
                e[0] += r["ms"]
                e[1] += 1
    tot = sum(v[0] / v[1] for v in agg.values())
    print(f"form {a.form}{' packed' if a.packed else ''} shape {shape} levels {plan.levels}: {tot:.3f} ms per decompose + recompose "
          f"(sum of event-bracketed launches)")
    for (name, lvl), v in sorted(agg.items(), key=lambda kv: -kv[1][0])[:24]:
        ms = v[0] / v[1]
        print(f"  {name:16s} L{lvl:<2d} {ms:8.4f} ms {v[2] / ms / 1e6:9.1f} GB/s {v[3] / ms / 1e9:7.3f} TFLOP/s "
              f"share {ms / tot:.3f}")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(a.reps):
        dec()
    ev[1].record()
    for _ in range(a.reps):
        rec()
    ev[2].record()
    torch.cuda.synchronize()
    print(f"graph-replayed: decompose {ev[0].elapsed_time(ev[1]) / a.reps:.3f} ms, "
          f"recompose {ev[1].elapsed_time(ev[2]) / a.reps:.3f} ms")
    plan.close()
    ctx.close()


def batch_main(a):
    import time

    import torch

    import paper_2105_12764_gb300 as mgr
    from paper_2105_12764_gb300 import synth

    dtype = mgr.MGR_F64 if a.form == "fp64" else mgr.MGR_F32
    prec = mgr.MGR_PREC_MIXED if a.form == "mixed" else mgr.MGR_PREC_NATIVE
    ctx = mgr.Context(0)
    specs = synth.batch_field_specs(a.batch, seed=0)
    plans, xs, ys, zs = [], [], [], []
    for i, (shape, st) in enumerate(specs):
        coords = [synth.stretched_coords(n) for n in shape] if st else None
        plans.append(mgr.Plan(ctx, shape, coords, -1, dtype, prec))
        u = synth.grf_field_torch(shape, seed=1000 + i)
        xs.append(u if dtype == mgr.MGR_F64 else u.float())
        ys.append(torch.empty_like(xs[-1]))
        zs.append(torch.empty_like(xs[-1]))
    dec = ctx.batch_prepare([(mgr.MGR_OP_DECOMPOSE, p, x, y) for p, x, y in zip(plans, xs, ys)])
    rec = ctx.batch_prepare([(mgr.MGR_OP_RECOMPOSE, p, y, z) for p, y, z in zip(plans, ys, zs)])

    def step():
        ctx.batch_poll(ctx.batch_submit(dec), -1)
        ctx.batch_poll(ctx.batch_submit(rec), -1)

    step()  # autotune + graph capture
    step()
    torch.cuda.synchronize()
    cudart = torch.cuda.cudart()
    cudart.cudaProfilerStart()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        step()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / a.reps
    cudart.cudaProfilerStop()
    elems = sum(x.numel() for x in xs)
    print(f"batch of {len(specs)} fields ({a.form}), {elems} elements: {ms:.3f} ms per decompose + recompose "
          f"submit pair; {ctx.batch_tuning().strip()[:300]}")
    for p in plans:
        p.close()
    ctx.close()


if __name__ == "__main__":
    main()
