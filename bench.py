#!/usr/bin/env python
"""Time to the lowest 16 vertical excitation energies on one GB300.

Workload ("medium"): cubic cell L = 20 bohr, 72^3 grid, 20,479 plane waves, 256
localised orbitals, 512 PDEP vectors with lambda_i = -0.8 exp(-i/100), overlap
threshold keeping 15% of the v <= w pairs, 16 excitations with Davidson block 32,
mixed precision (FP32 FFTs / pair products / tau streaming, FP64 Davidson algebra).
A step is one whole solve: screened-integral build (bse_build_tau) followed by the
Davidson solve (bse_davidson) to ||r|| <= 2e-4 Ha, inputs resident in HBM. The
FP64 plain path solves the same system once: the step is valid when every mixed
excitation energy is within 1 meV of it. Inputs (tau 7.4 GB, r-space workspaces
24 GB) are far larger than L2, so no separate L2 flush is done.

--impl reference times the CPU FP64 oracle on a bounded sample of the same workload.
Under torchrun each rank solves an independent replica (seed + rank): no collective
on the data path; the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the batched solves run one CUDA stream per system: give the streams more hardware queues
# than the default 8 so independent systems do not serialise behind one another
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

MEV = 3.6749322e-5
N_EIG, BLOCK, MAX_SUB = 16, 32, 128
# trial vectors the medium mixed solve passes through the operator (measured on the GPU);
# the CPU reference arm scales its samples to this many applications
N_APPLY_MEDIUM = 528
TOL_MIXED, TOL_FP64 = 2e-4, 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="medium")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--apply-only", action="store_true",
                    help="time bse_apply_liouville alone on --nvec vectors (operator GB/s)")
    ap.add_argument("--nvec", type=int, default=32)
    ap.add_argument("--batch", type=int, default=0,
                    help="solve this many uneven systems of the batch family together (bse_solve_batch)")
    ap.add_argument("--lanczos", type=int, default=0,
                    help="time a Lanczos absorption chain of this many steps for x, y, z (bse_lanczos)")
    ap.add_argument("--no-batch-line", action="store_true",
                    help="skip the 64-system batched solve that the default line reports under 'batch'")
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(device_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, reasons = [], set()
        mx = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if sm:
            sm.sort()
            out.update(sm_mhz=sm[len(sm) // 2], sm_max_mhz=mx, reasons=sorted(reasons),
                       samples=len(sm))
        return out


# --------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------------------
def cpu_oracle_setup(inst, seed: int = 0):
    """FP64 oracle set-up for the CPU baseline (not counted in the solve time): the operator
    (orbitals on the grid, overlaps, pair mask) and, timed once, the per-vector work of one
    operator application (one vector's orbitals to the grid and its Hartree potential)."""
    import numpy as np
    from oracle import liouville, pairs as opairs
    t0 = time.perf_counter()
    Lop = liouville.Liouville(inst)
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    A1 = Lop.project(rng.standard_normal((1, inst.n_occ, inst.n_pw)))
    t0 = time.perf_counter()
    ua, VH = Lop.fields(A1)
    t_fixed = time.perf_counter() - t0
    plist = opairs.pair_list(Lop.mask)
    return dict(inst=inst, Lop=Lop, A1=A1, ua=ua, VH=VH, t_fixed=t_fixed, setup_s=setup_s,
                plist=plist, P=int(plist.shape[0]), cores=len(os.sched_getaffinity(0)))


def cpu_oracle_step(S, i: int, n_apply_vectors: int, pairs_per_step: int = 4, rows_per_step: int = 2):
    """One bounded sample of the FP64 oracle's solve, scaled to the whole solve.

    Sample i times, with the oracle as it stands, tau_vw for `pairs_per_step` pairs spread
    over the pair list (each computed afresh) and the K1d / local / exchange / forward
    transform work of `rows_per_step` orbital rows of one vector (Liouville.apply_rows; the
    rows' tau come from the cache or are built untimed first). With the per-vector work
    t_fixed of the set-up, one solve is modelled as
        P t_pair + n_apply (t_fixed + N_occ t_row),
    the same sum the solve performs (every pair's tau once, every applied vector through
    every row), checked against a timed complete oracle solve of a small system.
    """
    import numpy as np
    Lop, P, plist, inst = S["Lop"], S["P"], S["plist"], S["inst"]
    n = inst.n_occ
    stride = max(1, P // 97)
    t_pair = 0.0
    for q in range(pairs_per_step):
        v, w = (int(x) for x in plist[((i * pairs_per_step + q) * stride) % P])
        Lop._tau.pop((v, w), None)
        t0 = time.perf_counter()
        Lop.tau(v, w)
        t_pair += time.perf_counter() - t0
    t_pair /= pairs_per_step
    rows = [((i * rows_per_step + q) * 37) % n for q in range(rows_per_step)]
    for v in rows:
        for w in np.nonzero(Lop.mask[v])[0]:
            Lop.tau(v, int(w))
    t0 = time.perf_counter()
    Lop.apply_rows(S["A1"], S["ua"], S["VH"], rows)
    t_row = (time.perf_counter() - t0) / rows_per_step
    value = P * t_pair + n_apply_vectors * (S["t_fixed"] + n * t_row)
    return dict(value=value, t_pair_s=t_pair, t_row_s=t_row)


def cpu_model_check(seed: int = 0):
    """Times a complete FP64 oracle solve (tau build + block Davidson to 1e-5 Ha) of a small
    localised system (32^3 grid, 16 orbitals, 4 excitations) and the model's prediction for
    it from the same kind of samples: (measured s, predicted s)."""
    import numpy as np
    from synth import make_localized
    from oracle import davidson
    inst = make_localized(6, 20.0 * 32 / 72, 32, 16, 2.5, 32, n_eig=4, block=4)
    S = cpu_oracle_setup(inst, seed)
    S["Lop"]._tau.clear()
    Lop = S["Lop"]
    t0 = time.perf_counter()
    Lop.build_tau()
    om, _, info = davidson.davidson(Lop.apply, Lop.diagonal(), Lop.project, 4, 4, 32, 1e-5)
    measured = time.perf_counter() - t0
    n_apply = int(info.get("n_apply", 0)) or None
    preds = [cpu_oracle_step(S, i, n_apply or 1)["value"] for i in range(4)]
    return measured, float(np.median(preds)), n_apply


def cpu_baseline_run(inst, n_apply_vectors: int, steps: int, warmup: int = 0):
    """Set-up, then `warmup` + `steps` samples; returns the baseline entry (value = mean of
    the timed samples, with their spread) and the per-sample values."""
    import numpy as np
    S = cpu_oracle_setup(inst)
    vals = []
    for i in range(warmup + steps):
        r = cpu_oracle_step(S, i, n_apply_vectors)
        if i >= warmup:
            vals.append(r["value"])
    meas, pred, nap = cpu_model_check()
    v = float(np.mean(vals))
    sample = (f"FP64 oracle, {steps} samples of 4 tau pairs (of {S['P']}) + 2 operator rows (of "
              f"{inst.n_occ}) each, with one vector's grid transforms + Hartree ({S['t_fixed']:.2f} s, "
              f"timed once); scaled to {S['P']} pairs + {n_apply_vectors} vectors x {inst.n_occ} rows. "
              f"Model check on a complete oracle solve (32^3, 16 orbitals, {nap} vectors): "
              f"measured {meas:.2f} s, model {pred:.2f} s. Oracle set-up {S['setup_s']:.1f} s not counted")
    return {"value": v, "unit": "s", "cores": S["cores"], "kind": "oracle", "sample": sample,
            "spread": {"min": float(np.min(vals)), "max": float(np.max(vals)), "n": len(vals)},
            "model_check": {"measured_s": meas, "model_s": pred}}


# --------------------------------------------------------------------------------------
def batch_run(binding, Context, PREC_MIXED, PREC_FP64, n_systems, warmup=1, steps=1):
    """Many independent systems (grids 32/48/64^3, N_occ 32..192, N_pdep = 2 N_occ, 8 VEEs
    each), one context and CUDA stream per system, solved together by bse_solve_batch (mixed
    precision); the same systems one after another on one stream; the FP64 plain solves as a
    batch too, the reference of every system's energies."""
    import numpy as np
    import torch
    from synth.instance import make_batched_member
    systems = [make_batched_member(300 + i) for i in range(n_systems)]
    n_eig, block, max_sub = 8, 8, 64

    def run_batch(prec, tol):
        streams = [torch.cuda.Stream() for _ in systems]
        ctxs = [Context(s, prec, stream=st.cuda_stream) for s, st in zip(systems, streams)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, stats, rc = binding.solve_batch(ctxs, n_eig, block, max_sub, res_tol=tol)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        return t, om, stats, rc

    for _ in range(max(1, warmup)):
        run_batch(PREC_MIXED, TOL_MIXED)
    tb, om, stats, rc = min((run_batch(PREC_MIXED, TOL_MIXED) for _ in range(max(1, steps))), key=lambda x: x[0])
    # sequential: the same solves, one system at a time on one stream
    ctxs = [Context(s, PREC_MIXED) for s in systems]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in ctxs:
        c.build_tau()
        c.davidson(n_eig, block, max_sub, res_tol=TOL_MIXED)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    # FP64 plain reference: the same batched solve, 16 systems at a time (64 FP64 contexts do
    # not fit the device together)
    t64, ref, rc64 = 0.0, np.zeros_like(om), []
    for i0 in range(0, len(systems), 16):
        sub = systems[i0:i0 + 16]
        streams = [torch.cuda.Stream() for _ in sub]
        ctxs = [Context(s_, PREC_FP64, stream=st.cuda_stream) for s_, st in zip(sub, streams)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o64, _, r64 = binding.solve_batch(ctxs, n_eig, block, max_sub, res_tol=TOL_FP64)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t0
        for c in ctxs:
            c.close()
        ref[i0:i0 + len(sub)] = o64
        rc64 += r64
        torch.cuda.empty_cache()
    err = np.abs(om - ref).max(1) / MEV
    return {"n_systems": len(systems), "batch_s": tb, "sequential_s": ts, "speedup_vs_sequential": ts / tb,
            "fp64_plain_batch_s": t64, "fp64_plain_batch": "16 systems at a time", "speedup_vs_fp64_plain": t64 / tb,
            "max_err_meV_vs_fp64_every_system": float(err.max()), "valid_1meV": bool(err.max() <= 1.0),
            "grids": [s.n_grid for s in systems], "n_occ": [s.n_occ for s in systems],
            "status": rc, "status_fp64": rc64, "iterations": [st.iterations for st in stats]}


def cufft_comparison(n_grid: int, n_fields: int, ours_inv_us: float, ours_fwd_us: float, reps: int = 10):
    """cuFFT (through torch.fft) on the unpruned transforms of the same real fields, for comparison.

    Both library forms are timed per real field: r2c/c2r on the half spectrum, and c2c with two real
    fields packed in one complex transform (the packing the library's own transforms use). cuFFT
    starts from a full grid of coefficients: it has no sphere scatter or pruning, so it moves more
    bytes per field than the sphere-to-grid transforms it is compared with."""
    import torch
    n = n_grid
    nb = max(2, min(n_fields, int(1.5e9 // (n ** 3 * 4 * 3))) // 2 * 2)
    dev = "cuda"
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn(nb, n, n, n, device=dev, generator=g)
    xh = torch.fft.rfftn(x, dim=(1, 2, 3))
    z = torch.complex(x[0::2], x[1::2])
    st = torch.cuda.current_stream()

    def timed(f):
        for _ in range(3):
            f()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            f()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2] * 1e3 / nb         # median, us per real field

    r = {"grid": n, "fields_per_launch": nb,
         "c2r_us_per_field": timed(lambda: torch.fft.irfftn(xh, s=(n, n, n), dim=(1, 2, 3))),
         "r2c_us_per_field": timed(lambda: torch.fft.rfftn(x, dim=(1, 2, 3))),
         "c2c_inverse_us_per_field": timed(lambda: torch.fft.ifftn(z, dim=(1, 2, 3))),
         "c2c_forward_us_per_field": timed(lambda: torch.fft.fftn(z, dim=(1, 2, 3))),
         "ours_inverse_us_per_field": ours_inv_us, "ours_forward_us_per_field": ours_fwd_us}
    r["inverse_speedup_vs_c2r"] = r["c2r_us_per_field"] / ours_inv_us if ours_inv_us else None
    r["forward_speedup_vs_r2c"] = r["r2c_us_per_field"] / ours_fwd_us if ours_fwd_us else None
    del x, xh, z
    torch.cuda.empty_cache()
    return r


def batch_mode(args, binding, Context, PREC_MIXED, PREC_FP64):
    r = batch_run(binding, Context, PREC_MIXED, PREC_FP64, args.batch, args.warmup, args.steps)
    print(json.dumps({"mode": "batch", **r}), flush=True)


def apply_only(args, inst, ctx, stream, binding):
    """Operator-only timing: one bse_apply_liouville on a block of random conduction vectors."""
    import numpy as np
    import torch
    ctx.build_tau()
    rng = np.random.default_rng(0)
    psi = inst.psi
    A = rng.standard_normal((args.nvec, inst.n_occ, inst.n_pw))
    A -= (A @ psi.T) @ psi
    A[..., 1] = 0.0
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    for _ in range(args.warmup):
        ctx.apply(a, out)
    torch.cuda.synchronize()
    ctx.profile(-1)
    ctx.profile(1)
    l0 = binding.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.apply(a, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(0)
    prof, nl = ctx.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    regions = {k: {"ms": v["ms"] / v["calls"], "GBps": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                   "TFLOPs": v["flops"] / (v["ms"] * 1e-3) / 1e12}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    print(json.dumps({"mode": "apply_only", "config": args.config, "nvec": args.nvec,
                      "ms_per_apply": ms, "gpu_launches": nl - l0, "regions": regions}), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from synth import CONFIGS
    metric = "time_to_16_lowest_VEEs_1meV_vs_fp64_plain"
    probe = CONFIGS[args.config if not args.batch else "tiny"]()
    n_g = 2 * probe.n_half - 1
    # solver shape: the medium workload's block of 32 (subspace 128); the large one (96^3,
    # 1,024 orbitals, ~20k pairs) uses its block of 64 with a subspace of 96 to leave room
    # for its 71 GB of tau
    global BLOCK, MAX_SUB
    if args.config == "large":
        BLOCK, MAX_SUB = 64, 96
    pairs_desc = "~20k pairs" if args.config == "large" else "15% of pairs"
    cfg_desc = {"workload": f"{args.config}: L={probe.L:g} bohr, {probe.n_grid}^3 grid, N_G={n_g}, "
                            f"N_occ={probe.n_occ}, N_pdep={probe.n_pdep}, {pairs_desc}, {N_EIG} VEEs, "
                            f"Davidson block {BLOCK}, mixed FP32/FP64",
                "grid": probe.n_grid, "n_occ": probe.n_occ, "n_pdep": probe.n_pdep, "n_eig": N_EIG,
                "block": BLOCK,
                "l2": "inputs larger than L2 (tau and r-space workspaces exceed 129 MB)"}
    if args.config == "large":
        # one GPU cannot hold a second large context (e2e), the FP64 plain solve (142 GB of tau
        # plus an FP64 subspace) or, on the host, the FP64 oracle's tau (142 GB); the r-space
        # workspace is held to 48 GB (six trial vectors at a time) next to 108 GB of tau
        args.no_e2e = args.no_fp64 = args.no_cpu = args.no_batch_line = True
        os.environ.setdefault("BSE_WORKSPACE_GB", "48")

    if args.impl == "reference":
        if rank != 0:
            return
        inst = probe
        base = cpu_baseline_run(inst, N_APPLY_MEDIUM, steps=args.steps, warmup=args.warmup)
        v = base["value"]
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg_desc, "cpu_baseline": base,
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2409_15116_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2409_15116_gb300 import Context, PREC_MIXED, PREC_FP64, binding
    inst = probe if rank == 0 else CONFIGS[args.config](1000 + rank)
    stream = torch.cuda.current_stream()
    ctx = Context(inst, PREC_MIXED, stream=stream.cuda_stream)

    def step():
        ctx.build_tau()
        return ctx.davidson(N_EIG, BLOCK, MAX_SUB, max_it=200, res_tol=TOL_MIXED)

    if args.apply_only:
        return apply_only(args, inst, ctx, stream, binding)
    if args.lanczos:
        ctx.build_tau()
        ctx.lanczos(8, dirs=(0, 1, 2))                  # warm-up (tuning of the 3-vector width)
        torch.cuda.synchronize()
        ctx.profile(-1)
        ctx.profile(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a, b, n2 = ctx.lanczos(args.lanczos, dirs=(0, 1, 2))
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.profile(0)
        prof, _ = ctx.profile_read()
        om = np.linspace(0.0, 4.0, 2001)
        g = ctx.lanczos_spectrum(a[0], b[0], n2[0], om, 0.01)
        print(json.dumps({"mode": "lanczos", "config": args.config, "steps": args.lanczos, "n_pol": 3,
                          "s": e0.elapsed_time(e1) / 1e3, "ms_per_step": e0.elapsed_time(e1) / args.lanczos,
                          "spectrum_finite": bool(np.isfinite(g).all()),
                          "regions_ms": {k: v["ms"] for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}),
              flush=True)
        return
    if args.batch:
        return batch_mode(args, binding, Context, PREC_MIXED, PREC_FP64)

    for _ in range(args.warmup):
        om_mixed, st = step()
    torch.cuda.synchronize()
    ctx.profile(-1)
    ctx.profile(1)
    l0 = binding.launch_count()
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        om_mixed, st = step()
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = binding.launch_count() - l0
    ctx.profile(0)
    prof, _ = ctx.profile_read()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # roofline of the dominant region (CUDA events on the launching stream)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    per_kernel_launches = {"fft_inverse_a": 3, "fft_forward_r": 3}
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, d = dom
    nl = d["calls"] * per_kernel_launches.get(name, 1)
    t_launch = d["ms"] / nl * 1e-3
    bytes_launch = d["bytes"] / d["calls"] if name not in per_kernel_launches else d["bytes"] / d["calls"]
    achieved = bytes_launch / t_launch / 1e9
    # DRAM traffic per launch of the K1d kernel (model): its entry-major tau once (four slots
    # per entry of the row-block neighbour lists), a(r) and the result once, V_loc, V_H and
    # u_psi. The ncu capture of the op256 launch (32 vectors, 32^3 grid) read and wrote 4.311
    # GB where this model gives 4.331 GB, and of the 8-point, 8-vector tile with L2 prefetch
    # at 16 vectors 3.379 GB against 3.255 GB; the algorithmic bytes count tau once per pair.
    traffic = None
    if name == "k1d_combine":
        pr = ctx.pairs()
        n = inst.n_occ
        nbr = np.zeros((n, n), bool)
        nbr[pr[:, 0], pr[:, 1]] = True
        nbr[pr[:, 1], pr[:, 0]] = True
        n_ent = int(sum(np.any(nbr[b:b + 4], axis=0).sum() for b in range(0, n, 4)))
        n3 = inst.n_grid ** 3
        traffic = bytes_launch + (4.0 * n_ent - len(pr)) * n3 * 4.0
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": traffic,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    regions = {k: {"ms_per_step": v["ms"] / args.steps, "calls": v["calls"],
                   "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    # the sphere<->grid transforms of the timed steps against cuFFT on the same fields
    fftcmp = None
    if rank == 0 and "fft_inverse_a" in prof and "fft_forward_r" in prof:
        n_fields = sum(st_.n_apply for st_ in stats) * inst.n_occ
        fftcmp = cufft_comparison(inst.n_grid, inst.n_occ,
                                  prof["fft_inverse_a"]["ms"] * 1e3 / n_fields,
                                  prof["fft_forward_r"]["ms"] * 1e3 / n_fields)

    # end-to-end through the C ABI with host buffers (context creation uploads the inputs)
    e2e = None
    if rank == 0 and not args.no_e2e:
        h2d = sum(np.asarray(a).nbytes for a in (inst.miller, inst.psi, inst.eps, inst.v_loc,
                                                  inst.pdep, inst.lam))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = Context(inst, PREC_MIXED, stream=stream.cuda_stream)
        c2.build_tau()
        om2, _ = c2.davidson(N_EIG, BLOCK, MAX_SUB, max_it=200, res_tol=TOL_MIXED)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        c2.close()
        e2e = {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(om2.nbytes)}

    # FP64 plain path: accuracy gate and time-to-solution comparison
    fp64 = None
    max_err_mev = None
    if not args.no_fp64 and rank == 0:
        del ctx
        torch.cuda.empty_cache()
        c64 = Context(inst, PREC_FP64, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c64.build_tau()
        om64, st64 = c64.davidson(N_EIG, BLOCK, MAX_SUB, max_it=200, res_tol=TOL_FP64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        c64.close()
        max_err_mev = float(np.abs(om_mixed - om64).max() / MEV)
        fp64 = {"time_s": t64, "iterations": st64.iterations, "omega_ha": [float(x) for x in om64]}

    batch = None
    if rank == 0 and not args.no_batch_line and args.config == "medium":
        batch = batch_run(binding, Context, PREC_MIXED, PREC_FP64, 64, warmup=1, steps=1)

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline_run(inst, stats[-1].n_apply, steps=3)

    if rank == 0:
        line = {"metric": metric, "value": ms / 1e3, "unit": "s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": cfg_desc, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "valid_1meV": (max_err_mev is not None and max_err_mev <= 1.0) if not args.no_fp64 else None,
                "max_err_meV_vs_fp64": max_err_mev, "fp64_plain": fp64,
                "davidson": {"iterations": stats[-1].iterations, "n_apply": stats[-1].n_apply,
                             "ms_apply": stats[-1].ms_apply, "ms_total": stats[-1].ms_total},
                "omega_ha": [float(x) for x in om_mixed], "regions": regions, "batch": batch,
                "fft_vs_cufft": fftcmp}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
