#!/usr/bin/env python3
"""Benchmark of the separated Gaussian-sum operator apply (boxes/s and roofline fraction).

A step is one mra_apply of the whole hot path -- source norms, norm screen and
work list, sort on the destination key, the gather-apply kernel -- over the
resident input tree of the workload (default: BSH exp(-r)/r as 60 Gaussians,
8 Gaussians a~logU[1,1e4], adaptive k=10, 17,200 boxes).  Setup (projection,
fit, operator blocks) is outside the timed region.

Arms:
  default           the CUDA library through its C ABI (device-resident inputs);
                    also an end-to-end figure with host buffers (H2D + apply + D2H)
  --impl reference  the CPU oracle on this machine's cores, on a bounded seeded
                    sample of destination boxes, extrapolated by kept-term count

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica (the single-function apply does not shard) and value sums the ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# DRAM bytes (read + written) of one launch of the dominant kernel, from a one-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of this bench's own command, keyed by
# (workload, kernel).  An entry is removed whenever the kernel changes.
SPLIT_TRAFFIC = {("bsh_m60_adaptive_k10", "apply_src_kernel"): 68.46e6 + 687.48e6}

METRIC = "3D operator-apply boxes/s & % roofline, mixed vs FP64 GPU at 1e-6 rel L2"
def fixed_schedule(opts, text):
    """opts with the schedule fields given as 'field=value,...' (no tuning)."""
    from paper_1507_01888_gb300 import autotune, mra
    o = mra.copy_opts(opts)
    for item in text.split(","):
        f, v = item.split("=")
        if f.strip() not in ("split_kernel", "tile_variant", "join", "sums", "ahead"):
            raise ValueError(f"--schedule: unknown field {f}")
        setattr(o, f.strip(), int(v))
    return o, {"choice": autotune.describe(o), "candidates": "fixed by --schedule"}


def split_dtype(pieces, opts=None, k=0):
    """What the split-precision apply of order k computes in (the label of its JSON line)."""
    from paper_1507_01888_gb300 import mra
    if opts is not None and opts.split_kernel != mra.SPLIT_DEST and k in (4, 6, 8, 10):
        sums = "compensated f32 (sum + Kahan correction)" if opts.sums == mra.SUMS_COMPENSATED else "plain f32"
        join = int(opts.join) if opts.join else (2 if k * k > 64 else 1)  # 0: 2 in one-source tiles only
        return (f"bf16x{pieces}-split MMAs with f32 accumulation in tensor memory (up to {join} Gaussian terms "
                f"per accumulation); each (source, displacement) sum over terms in {sums}, stored as f32; "
                f"per-destination sums of those in f32 pairs (error-free TwoSum, ~48 bits), formed into f64")
    return (f"bf16x{pieces}-split MMAs with f32 accumulation; Gaussian-term and per-destination sums in "
            f"compensated f32 (sum + Kahan correction), formed into f64 at the end")


_FP64 = {}


def fp64_peak(dev_index=0):
    """FP64 rate of this GPU, measured by the library's probe (mra_measure_fp64_peak: a DFMA loop
    and an FP64 MMA loop over the whole device, ~2 s, before any timed region), with the clocks
    sampled while it ran.  The FP64 apply kernel issues DFMA, so its roofline peak is the DFMA rate."""
    if "v" not in _FP64:
        from paper_1507_01888_gb300 import mra
        clk = clocks_start(None)
        dfma, dmma = mra.measure_fp64_peak(2.0)
        clocks = clocks_stop(clk, dev_index)
        _FP64["v"] = {"dfma_tflops": dfma, "dmma_tflops": dmma, "clocks": clocks}
    return _FP64["v"]


def fp64_peak_source(dev_index=0):
    f = fp64_peak(dev_index)
    return (f"measured DFMA loop (mra_measure_fp64_peak; DMMA {f['dmma_tflops']:.3f} TFLOP/s), "
            f"SM clock median {f['clocks'].get('sm_mhz')} MHz, reasons {f['clocks'].get('reasons')}")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="bsh_m60_adaptive_k10", choices=sorted(W.WORKLOADS))
    p.add_argument("--precision", choices=["auto", "fp64", "split"], default="auto")
    p.add_argument("--pieces", type=int, default=3)
    p.add_argument("--schedule", default=None,
                   help="fixed split schedule instead of the autotuner, e.g. 'split_kernel=0,join=4,sums=0,ahead=2' "
                        "(the fields of mra_apply_opts; used to profile the schedule a tuned run chose)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU seconds of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--clocks-csv", default=None, help="also write the nvidia-smi samples here")
    p.add_argument("--learned-quantile", type=float, default=1.0,
                   help="learned-screen margin: this quantile of the held-out residuals (1 = largest)")
    p.add_argument("--dist-backend", default="nccl", choices=["nccl", "gloo"],
                   help="torch.distributed backend for N > 1 (gloo: host-side exchange, for tests)")
    p.add_argument("--partition", action="store_true",
                   help="N > 1, one function: each rank computes a destination key range (owner "
                        "computes) after an all-gather of the input parts (strong scaling) instead "
                        "of running a replica")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


L2_NOTE = "a 256 MB buffer is written before every timed step (device memory on the GPU arm, host memory on the oracle arm)"


def workload_config(w):
    """The workload's identifying parameters, printed as `config` by every arm (run results go to `run`)."""
    return {"workload": w.name, "k": w.k, "M": w.M, "kernel": "bsh" if w.kernel == W.BSH else "poisson",
            "mu": w.mu, "thresh": w.thresh, "tau": w.tau, "functions": len(w.funcs),
            "tree": "adaptive" if w.uniform_level < 0 else f"uniform level {w.uniform_level}",
            "stencil": "shells<=%d" % w.max_disp if w.stencil == 0 else "27-point", "l2": L2_NOTE}


def host_flush(buf):
    """Write a 256 MB host buffer (the oracle arm's counterpart of the GPU arm's L2 flush)."""
    buf.fill(np.random.default_rng().integers(1, 1 << 30))


def oracle_fit(w):
    import oracle as O
    r_lo, r_hi = O.kernel_range(w.kernel, w.mu, w.L, w.fit_eps)
    return O.fit_search(w.mu if w.kernel == W.BSH else 0.0, w.M, r_lo, r_hi)


def _candidate_dests(keys):
    """Input boxes and their 26 neighbours inside the cell: a superset of the destination set."""
    n = (keys >> np.uint64(57)).astype(np.int64)
    x = ((keys >> np.uint64(38)) & np.uint64(0x7FFFF)).astype(np.int64)
    y = ((keys >> np.uint64(19)) & np.uint64(0x7FFFF)).astype(np.int64)
    z = (keys & np.uint64(0x7FFFF)).astype(np.int64)
    out = []
    nb = np.left_shift(1, n)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                a, b, c = x + dx, y + dy, z + dz
                ok = (a >= 0) & (a < nb) & (b >= 0) & (b < nb) & (c >= 0) & (c < nb)
                out.append((n[ok].astype(np.uint64) << np.uint64(57)) | (a[ok].astype(np.uint64) << np.uint64(38))
                           | (b[ok].astype(np.uint64) << np.uint64(19)) | c[ok].astype(np.uint64))
    return np.unique(np.concatenate(out))


def cpu_prepare(w):
    """The oracle's projection and fit of the workload, and the time of its per-apply set-up
    (blocks, norms, screen, destination set), measured once."""
    import oracle as O
    keys, coeffs, _ = O.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level,
                                max_level=w.max_level, uniform_level=w.uniform_level)
    _, _, _, c, t = oracle_fit(w)
    never = np.array([np.uint64(0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
    t0 = time.perf_counter()
    O.apply(keys, coeffs, c, t, w.L, sample_keys=never, stencil=w.stencil, max_disp=w.max_disp, tau=w.tau)
    return keys, coeffs, c, t, time.perf_counter() - t0


def cpu_baseline(w, target_s=12.0, seed=12345, prepared=None):
    """The oracle, as it stands, on a seeded sample of destination boxes sized for about
    target_s seconds of work; whole-job time is extrapolated by the sample's share of kept
    terms (the oracle's own whole-job term count).  Returns a dict."""
    import oracle as O
    keys, coeffs, c, t, t_setup = prepared if prepared is not None else cpu_prepare(w)
    cores = os.cpu_count() or 1
    kw = dict(stencil=w.stencil, max_disp=w.max_disp, tau=w.tau)
    cand = _candidate_dests(keys) if w.stencil == 1 or w.max_disp <= 1 else keys
    rng = np.random.default_rng(seed)
    n_try = min(64, len(cand))
    r = None
    for _ in range(6):
        sample = np.sort(rng.choice(cand, n_try, replace=False))
        t0 = time.perf_counter()
        r = O.apply(keys, coeffs, c, t, w.L, sample_keys=sample, **kw)
        t_sample = max(time.perf_counter() - t0 - t_setup, 1e-6)
        if t_sample >= 0.5 * target_s or n_try >= len(cand):
            break
        n_try = int(min(len(cand), max(2 * n_try, n_try * target_s / max(t_sample, 1e-3))))
    return {"n_in": len(keys), "sample_dest": len(r.keys), "sample_terms": r.terms, "t_sample": t_sample,
            "t_setup": t_setup, "cores": cores, "terms_total": r.terms_total, "dest_total": r.dest_total}


def clocks_start(path=None):
    try:
        f = open(path, "w") if path else None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return p, f
    except Exception:
        return None, None


def clocks_stop(handle, gpu_index):
    p, f = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out = ""
    rows = []
    for line in out.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        rows.append(parts)
        if f:
            f.write(line + "\n")
    if f:
        f.close()
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    load = sorted(sm)[len(sm) // 2:] if sm else []
    return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def run_reference(args, rank, world):
    """The oracle as it stands on this machine's cores.  Every step is one whole oracle job when
    a job takes at most about 15 s (the headline workload: ~4.4 s on 16 cores), else a seeded
    sample of destination boxes with the job time extrapolated by kept terms (said in `sample`)."""
    if rank != 0:
        return
    w = W.WORKLOADS[args.workload]()
    buf = np.empty(256 * 1024 * 1024 // 8)
    if "post" in w.extra or "solver" in w.extra:  # whole steps of the oracle, no sampling
        runs = []
        for i in range(args.warmup + args.steps):
            host_flush(buf)
            runs.append(oracle_post_step(w) if "post" in w.extra else oracle_solver_step(w))
        runs = runs[args.warmup:]
        value = statistics.mean(r["value"] for r in runs)
        line = {"metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": workload_config(w), "run": {"parallelism": f"{os.cpu_count()} host cores"},
                "cpu_baseline": dict(runs[-1], value=value),
                "e2e": {"value": value, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import oracle as O
    prepared = cpu_prepare(w)  # the oracle's projection and fit, once
    keys, coeffs, c, t, t_setup = prepared
    probe = cpu_baseline(w, 2.0, seed=999, prepared=prepared)
    t_est = probe["t_sample"] * probe["terms_total"] / max(probe["sample_terms"], 1) + t_setup
    whole = t_est <= 15.0
    kw = dict(stencil=w.stencil, max_disp=w.max_disp, tau=w.tau)
    times, info = [], None
    for i in range(args.warmup + args.steps):
        host_flush(buf)
        if whole:
            t0 = time.perf_counter()
            r = O.apply(keys, coeffs, c, t, w.L, **kw)
            dt = time.perf_counter() - t0
            info = {"terms": r.terms, "dest": len(r.keys)}
        else:
            cb = cpu_baseline(w, args.cpu_seconds / max(args.steps + args.warmup, 1) * 2, seed=1000 + i,
                              prepared=prepared)
            dt = cb["t_sample"] * cb["terms_total"] / max(cb["sample_terms"], 1)
            info = cb
        if i >= args.warmup:
            times.append(dt)
    t_job = statistics.mean(times)
    value = len(keys) / t_job
    cores = os.cpu_count() or 1
    if whole:
        sample = (f"the whole job every step: {len(keys)} source boxes, {info['terms']} kept terms, "
                  f"{info['dest']} destination boxes (the oracle's own block generation and screen included, "
                  f"{t_setup:.2f} s of each step)")
    else:
        sample = (f"{info['sample_dest']} seeded destination boxes per step ({info['sample_terms']} of "
                  f"{info['terms_total']} kept terms); job time extrapolated by kept terms")
    line = {"metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_job * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(w),
            "run": {"n_boxes": len(keys), "parallelism": f"{cores} host cores (OpenMP over destinations)"},
            "cpu_baseline": {"value": value, "unit": "boxes/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_over_ranks(n_local: int, ms_local: float, world: int, device=None):
    """(units summed over ranks, time maximised over ranks): value = units / time for the job."""
    if world <= 1:
        return n_local, ms_local
    import torch
    import torch.distributed as dist
    n = torch.tensor([float(n_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return int(round(n.item())), float(t.item())


def ns_terms(N: int, n0: int, D: int, M: int):
    """Kept terms of each apply of the non-standard form without a screen: (level, order factor,
    terms) with order factor 1 for the k-basis applies and 2 for the 2k-basis applies."""
    def pairs(n, d):  # in-cell (box, l) pairs of a whole level with |l|_inf <= d
        nb = 1 << n
        per_dim = sum(min(nb - 1, x + d) - max(0, x - d) + 1 for x in range(nb))
        return per_dim ** 3
    out = [(n0, 1, pairs(n0, (1 << n0) - 1) * M)]
    for n in range(n0, N):
        dn = min(D, (1 << n) - 1)
        out += [(n, 2, pairs(n, dn) * M), (n, 1, pairs(n, dn) * M)]
    return out


def run_ns(args, w, rank, world):
    """The non-standard form apply (mra_apply_ns on a uniform tree, mra_apply_ns_tree on an adaptive
    one); same JSON line."""
    import torch
    from paper_1507_01888_gb300 import mra, autotune
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n0, D = w.extra["ns"]["n0"], w.max_disp
    adaptive = w.uniform_level < 0
    # orders 2k above 16 are applied in FP64 only
    prec = mra.PREC_FP64 if args.precision == "fp64" or 2 * w.k > 16 else mra.PREC_SPLIT_BF16
    tree = mra.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level,
                       uniform_level=w.uniform_level)
    keys_h0 = tree.host()[0]
    N = int((keys_h0 >> np.uint64(57)).max())
    op = mra.Operator(w.kernel, w.M, w.k, w.L, 0, N, max_disp=max(2 * D + 1, (1 << n0) - 1), mu=w.mu,
                      fit_eps=w.fit_eps)
    ns_op = mra.NSOperator(op, max_disp=D)
    opts = mra.make_opts(precision=prec, pieces=args.pieces, stencil=mra.STENCIL_SHELLS, max_disp=D)

    def make(o):
        if adaptive:
            return mra.NSTreeApplier(op, ns_op, n0, o, out_cap=8 * tree.n, device=dev)
        return mra.NSApplier(op, ns_op, tree, n0, o)
    tuning = {}
    if prec == mra.PREC_SPLIT_BF16 and args.schedule:
        opts, tuning = fixed_schedule(opts, args.schedule)
    elif prec == mra.PREC_SPLIT_BF16:
        opts, table = autotune.tune(op, tree, opts, make_applier=make)
        tuning = {"choice": autotune.describe(opts), "candidates": table}
    ap = make(opts)
    ap(tree)
    torch.cuda.synchronize()
    accuracy = {}
    if prec != mra.PREC_FP64:
        ref = make(mra.make_opts(stencil=mra.STENCIL_SHELLS, max_disp=D))
        cmp = mra.compare(ap(tree), ref(tree))
        accuracy = {"rel_l2_vs_fp64_gpu": cmp["rel_l2"], "max_box_rel_vs_fp64_gpu": cmp["max_box_rel"],
                    "per_level_rel_l2_vs_fp64_gpu": {str(x["level"]): x["rel_l2"] for x in cmp["levels"]},
                    "fp64_gpu_apply_ms": ref.stats.kernel_ms,
                    "speedup_vs_fp64_gpu_kernel": ref.stats.kernel_ms / max(ap.stats.kernel_ms, 1e-9)}
        del ref
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        ap(tree, stream)
    torch.cuda.synchronize()
    clk = clocks_start(args.clocks_csv)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kms = []
    launches0 = mra.launch_count()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        ap(tree, stream)
        ev[i][1].record(stream)
        kms.append(ap.stats.kernel_ms)
    torch.cuda.synchronize()
    launches = mra.launch_count() - launches0
    clocks = clocks_stop(clk, 0)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    n_all, ms = reduce_over_ranks(tree.n, ms, world, dev)
    value = n_all / (ms / 1e3)
    # end to end: host coefficients in, host result out, through the same call
    keys_h, coeffs_h = tree.host()
    keys_pin = torch.from_numpy(keys_h.view(np.int64).copy()).pin_memory()
    coeffs_pin = torch.from_numpy(coeffs_h.copy()).pin_memory()
    dev_tree = mra.Tree(torch.empty_like(keys_pin, device=dev), torch.empty_like(coeffs_pin, device=dev),
                        tree.n, w.k, w.L)
    out_pin = torch.empty((ap.out.n,) + tuple(coeffs_pin.shape[1:]), dtype=torch.float64).pin_memory()
    e_ms = []
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dev_tree.keys.copy_(keys_pin, non_blocking=True)
        dev_tree.coeffs.copy_(coeffs_pin, non_blocking=True)
        out = ap(dev_tree, stream)
        out_pin.copy_(out.coeffs[:out.n], non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    _, e2e_ms = reduce_over_ranks(tree.n, statistics.mean(e_ms), world, dev)
    k = w.k
    if adaptive:  # no screen: every level's 2k and k applies keep the same terms; the coarsest is T^{n0}
        tc = ns_terms(n0, n0, D, w.M)[0][2]
        t2 = (ap.stats.terms_kept - tc) // 2
        terms = [(n0, 1, tc), (-1, 2, t2), (-1, 1, t2)]
    else:
        terms = ns_terms(N, n0, D, w.M)
    flops = sum(t * (6 * (f * k) ** 4 + (f * k) ** 3) for _, f, t in terms)
    assert abs(flops - ap.stats.algo_flops) <= 1e-9 * flops, "term count differs from the library's"
    kms_mean = statistics.mean(kms)
    achieved = flops / (kms_mean / 1e3) / 1e12
    pk, pk_kind = peaks()
    if prec == mra.PREC_FP64:
        p64 = fp64_peak()["dfma_tflops"]
        roof = {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s",
                "frac": achieved / p64, "traffic": None, "kernel": "apply_f64_kernel (all levels)",
                "peak_source": fp64_peak_source(), "kernel_ms": kms_mean,
                "flops": "algorithmic (6k'^4+k'^3 per term, k' = k or 2k)"}
        dtype = "f64"
    else:
        peak = pk.get("bf16_tflops", 1856.3)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": ("apply_src_kernel (order k) and apply_split_kernel (order 2k), all levels"
                                            if k in (4, 6, 8, 10) and opts.split_kernel != mra.SPLIT_DEST
                                            else "apply_split_kernel (all levels)"),
                "peak_source": f"bf16 dense burst, {pk_kind}",
                "kernel_ms": kms_mean, "flops": "algorithmic (6k'^4+k'^3 per term, k' = k or 2k)"}
        dtype = (f"order {k}: {split_dtype(args.pieces, opts, k)}; order {2 * k}: "
                 f"{split_dtype(args.pieces, opts, 2 * k)}")
    line = {"metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": workload_config(w), "run": {"n_boxes": n_all, "result_leaves": ap.out.n, "k": k, "M": w.M,
                       "form": "non-standard" + (", adaptive tree" if adaptive else ", uniform tree"),
                       "levels": f"{n0}..{N}", "max_disp_per_level": D, "terms": sum(t for _, _, t in terms),
                       "terms_reported": ap.stats.terms_kept,
                       "precision": "fp64" if prec == mra.PREC_FP64 else "split",
                       "l2": "flushed by a 256 MB write before every step", "tuning": tuning,
                       "parallelism": "single GPU" if world == 1 else f"replicas x{world}"},
            "roofline": roof, "clocks": clocks,
            "gpu_launches": launches,
            "e2e": {"value": n_all / (e2e_ms / 1e3), "unit": "boxes/s", "h2d_bytes_per_step": keys_pin.numel() * 8
                    + coeffs_pin.numel() * 8, "d2h_bytes_per_step": out_pin.numel() * 8},
            "accuracy": accuracy}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _timed(args, step, dev):
    """W untimed steps, then K steps each after an L2 flush, CUDA events on the current stream.
    Returns (mean ms per step, clocks, kernel launches of the library inside the timed region)."""
    import torch
    from paper_1507_01888_gb300 import mra
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    clk = clocks_start(args.clocks_csv)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = mra.launch_count()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = mra.launch_count() - launches0
    clocks = clocks_stop(clk, 0)
    return statistics.mean(a.elapsed_time(b) for a, b in ev), clocks, launches


def run_post(args, w, rank, world):
    """Sum-down and truncation of the leaf-level apply's multi-level result: a step is
    mra_reconstruct followed by mra_truncate, timed as whole calls (their per-level kernels,
    CUB sorts and scans and host synchronisations).  Units: input boxes of the sum-down."""
    import torch
    from paper_1507_01888_gb300 import mra
    import oracle as O
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    th = w.extra["post"]["truncate_thresh"]
    tree = mra.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level)
    lv = (tree.host()[0] >> np.uint64(57)).astype(int)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, int(lv.min()), int(lv.max()), max_disp=w.max_disp, mu=w.mu,
                      fit_eps=w.fit_eps)
    multi, _ = mra.apply(op, tree, mra.make_opts(screen=mra.SCREEN_NORM, tau=w.tau, stencil=w.stencil,
                                                 max_disp=w.max_disp))
    k3 = w.k ** 3
    res = {}

    def step(src=multi):
        leaves = mra.reconstruct(src, out_cap=4 * src.n)
        tr, e2 = mra.truncate(leaves, th, out_cap=leaves.n)
        res.update(leaves=leaves, tr=tr, e2=e2)
        return tr

    ms, clocks, launches = _timed(args, step, dev)
    n_in, n_leaves, n_tr = multi.n, res["leaves"].n, res["tr"].n
    n_all, ms = reduce_over_ranks(n_in, ms, world, dev)
    box_bytes = k3 * 8 + 8
    algo_bytes = box_bytes * (n_in + 2 * n_leaves + n_tr)
    pk, pk_kind = peaks()
    achieved = algo_bytes / (ms / 1e3) / 1e9
    # end to end: host multi-level tree in, host truncated tree out
    mk, mc = multi.host()
    keys_pin = torch.from_numpy(mk.view(np.int64).copy()).pin_memory()
    coeffs_pin = torch.from_numpy(mc.copy()).pin_memory()
    dev_tree = mra.Tree(torch.empty_like(keys_pin, device=dev), torch.empty_like(coeffs_pin, device=dev),
                        n_in, w.k, w.L)
    out_k = torch.empty(n_tr, dtype=torch.int64).pin_memory()
    out_c = torch.empty((n_tr, w.k, w.k, w.k), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    e_ms = []
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dev_tree.keys.copy_(keys_pin, non_blocking=True)
        dev_tree.coeffs.copy_(coeffs_pin, non_blocking=True)
        tr = step(dev_tree)
        out_k.copy_(tr.keys[:n_tr], non_blocking=True)
        out_c.copy_(tr.coeffs[:n_tr], non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    _, e2e_ms = reduce_over_ranks(n_in, statistics.mean(e_ms), world, dev)
    line = {"metric": METRIC, "value": n_all / (ms / 1e3), "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w), "run": {"n_boxes": n_all, "k": w.k, "input": "leaf-level FP64 apply result of "
                       "the BSH M=60 k=10 workload (boxes on several levels)", "result_leaves": n_leaves,
                       "truncated_leaves": n_tr, "truncate_thresh": th, "l2_change": res["e2"] ** 0.5,
                       "l2": "flushed by a 256 MB write before every step",
                       "parallelism": "single GPU" if world == 1 else f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": None,
                         "kernel": "mra_reconstruct + mra_truncate, whole calls",
                         "peak_source": f"HBM copy, {pk_kind}",
                         "bytes": "algorithmic: (k^3 + 1) x 8 B per box read or written: input, leaves written "
                                  "and read back, truncated leaves"},
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": n_all / (e2e_ms / 1e3), "unit": "boxes/s",
                    "h2d_bytes_per_step": keys_pin.numel() * 8 + coeffs_pin.numel() * 8,
                    "d2h_bytes_per_step": out_k.numel() * 8 + out_c.numel() * 8}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_post_step(w)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_partitioned(args, w, rank, world, local):
    """One function over N ranks by destination key ranges (owner computes).  Each rank holds
    its key range of the input tree; the ranges are cut by work (the kept terms per source box of
    each level, from one untimed apply).  A step is one halo exchange (partition.HaloPlan: an
    all-to-all in which each rank receives exactly the boxes other ranks own in its halo) and
    the rank's apply on its halo with its destination range.  value = the function's boxes / the
    slowest rank's step time (strong scaling: the total work is fixed)."""
    import torch
    import torch.distributed as dist
    from paper_1507_01888_gb300 import mra, partition as PT
    dev = torch.device("cuda", local)
    prec = mra.PREC_FP64 if args.precision == "fp64" else mra.PREC_SPLIT_BF16
    tree = mra.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level,
                       uniform_level=w.uniform_level)
    keys_h, coeffs_h = tree.host()
    lv = (keys_h >> np.uint64(57)).astype(int)
    op = mra.Operator(w.kernel, w.M, w.k, w.L, int(lv.min()), int(lv.max()), max_disp=w.max_disp, mu=w.mu,
                      fit_eps=w.fit_eps)
    screen = mra.SCREEN_NORM if w.tau > 0 else mra.SCREEN_NONE
    base = dict(precision=prec, pieces=args.pieces, screen=screen, tau=w.tau, stencil=w.stencil,
                max_disp=w.max_disp, tile_variant=2 if prec == mra.PREC_SPLIT_BF16 and 4 <= w.k <= 10 else 0)
    _, st_all = mra.apply(op, tree, mra.make_opts(**base))  # per-level work, for the ranges
    lev = st_all["levels"]
    weights = PT.level_weights(keys_h, [lev.get(n, {}).get("sources", 0) for n in range(20)],
                               [lev.get(n, {}).get("terms_kept", 0) for n in range(20)])
    ranges = PT.split_ranges(keys_h, world, weights)
    lo, hi = ranges[rank]
    D = 1 if w.stencil == 1 else w.max_disp
    plan = PT.HaloPlan(keys_h, ranges, rank, D)
    local_coeffs = torch.from_numpy(coeffs_h[plan.own].copy()).to(dev)
    opts = mra.make_opts(**base, dest_range=(lo, hi))
    sub = mra.Tree(torch.from_numpy(plan.halo_keys.view(np.int64).copy()).to(dev),
                   torch.empty((plan.n_halo, w.k, w.k, w.k), dtype=torch.float64, device=dev), plan.n_halo, w.k, w.L)
    ap = mra.Applier(op, sub, opts)
    stream = torch.cuda.current_stream()
    del tree

    def step():
        plan.exchange(local_coeffs, out=sub.coeffs)
        ap(sub, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(args.clocks_csv)
    launches0 = mra.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kms = []
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        kms.append(ap.stats.kernel_ms)
    torch.cuda.synchronize()
    launches = mra.launch_count() - launches0
    dist.barrier()
    clocks = clocks_stop(clk, local)
    ms_local = statistics.mean(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    terms = torch.tensor([float(ap.stats.terms_kept)], dtype=torch.float64, device=dev)
    dist.all_reduce(terms, op=dist.ReduceOp.SUM)
    kmax = torch.tensor([statistics.mean(kms)], dtype=torch.float64, device=dev)
    dist.all_reduce(kmax, op=dist.ReduceOp.MAX)
    pk, pk_kind = peaks()
    k = w.k
    achieved = terms.item() * (6 * k ** 4 + k ** 3) / (kmax.item() / 1e3) / 1e12
    peak = pk.get("bf16_tflops", 1856.3) * world if prec == mra.PREC_SPLIT_BF16 else \
        fp64_peak(local)["dfma_tflops"] * world
    line = {"metric": METRIC, "value": len(keys_h) / (ms / 1e3), "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if prec == mra.PREC_FP64 else split_dtype(args.pieces, opts, k),
            "data": "synthetic",
            "config": workload_config(w), "run": {"n_boxes": len(keys_h), "k": k, "M": w.M,
                       "parallelism": f"{world} ranks, destination key ranges cut by work (owner computes), "
                                      f"{args.dist_backend} all-to-all of each rank's halo every step",
                       "halo_boxes_this_rank": plan.n_halo, "received_boxes_this_rank": plan.n_received,
                       "own_boxes_this_rank": int(plan.own.sum())},
            "roofline": {"bound": "tensor" if prec == mra.PREC_SPLIT_BF16 else "alu", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "apply kernel, slowest rank", "peak_source": f"{world} x per-GPU peak, {pk_kind}"},
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": None, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                    "note": "not measured in the partitioned mode (inputs are exchanged between devices)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def oracle_post_step(w):
    """The oracle's own multi-level result of the same workload (untimed), then its sum-down and
    truncation, timed as one whole step."""
    import oracle as O
    ok, oc, _ = O.project(w.funcs[0], w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level)
    _, _, _, c, t = oracle_fit(w)
    r = O.apply(ok, oc, c, t, w.L, stencil=w.stencil, max_disp=w.max_disp, tau=w.tau)
    t0 = time.perf_counter()
    lk, lc = O.reconstruct(r.keys, r.coeffs, w.k)
    O.truncate(lk, lc, w.k, w.extra["post"]["truncate_thresh"])
    t_cpu = time.perf_counter() - t0
    return {"value": len(r.keys) / t_cpu, "unit": "boxes/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"the whole job: {len(r.keys)} input boxes, {t_cpu:.2f} s"}


def run_solver(args, w, rank, world):
    """The bound-state Helmholtz fixed-point solve for Z = 1: converged first (untimed), then a
    step is one whole iteration (product, non-standard apply, truncation, inner products, energy
    update) at the converged state.  Units: leaves of V psi entering the non-standard apply."""
    import math
    import torch
    from paper_1507_01888_gb300 import mra, solvers
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg = w.extra["solver"]
    prec = mra.PREC_FP64 if args.precision == "fp64" else mra.PREC_SPLIT_BF16
    t0 = time.perf_counter()
    V, vfit = solvers.project_potential(cfg["Z"], w.k, w.L, w.thresh, M=cfg["M_potential"])
    psi = solvers.gaussian_start(cfg["Z"], w.k, w.L, w.thresh)
    E, hist = cfg["E0"], []
    cache = {}
    for _ in range(40):
        E, psi, dE = solvers.bsh_step(V, psi, E, w.thresh, w.M, w.fit_eps, prec, cache=cache)
        hist.append(E)
        if abs(dE) < 1e-3 * w.thresh:
            break
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    info = {}
    state = {"E": E}

    def step(p=psi):
        E1, new, _ = solvers.bsh_step(V, p, state["E"], w.thresh, w.M, w.fit_eps, prec, info=info, cache=cache)
        return new

    ms, clocks, launches = _timed(args, step, dev)
    st = info["apply_stats"]
    n_all, ms = reduce_over_ranks(info["n_vpsi"], ms, world, dev)
    # the non-standard apply inside a step, alone, for the roofline of its tensor-core kernel
    kms = st["kernel_ms"]
    achieved = st["algo_flops"] / (kms / 1e3) / 1e12
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops_sustained", 1688.5) if prec != mra.PREC_FP64 else fp64_peak()["dfma_tflops"]
    # end to end: psi from the host, the new psi back to the host
    pk_h, pc_h = psi.host()
    keys_pin = torch.from_numpy(pk_h.view(np.int64).copy()).pin_memory()
    coeffs_pin = torch.from_numpy(pc_h.copy()).pin_memory()
    dev_psi = mra.Tree(torch.empty_like(keys_pin, device=dev), torch.empty_like(coeffs_pin, device=dev),
                       psi.n, w.k, w.L)
    stream = torch.cuda.current_stream()
    e_ms, d2h = [], 0
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dev_psi.keys.copy_(keys_pin, non_blocking=True)
        dev_psi.coeffs.copy_(coeffs_pin, non_blocking=True)
        new = step(dev_psi)
        ok_ = torch.empty(new.n, dtype=torch.int64).pin_memory()
        oc_ = torch.empty((new.n, w.k, w.k, w.k), dtype=torch.float64).pin_memory()
        ok_.copy_(new.keys[:new.n], non_blocking=True)
        oc_.copy_(new.coeffs[:new.n], non_blocking=True)
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
        d2h = ok_.numel() * 8 + oc_.numel() * 8
    _, e2e_ms = reduce_over_ranks(info["n_vpsi"], statistics.mean(e_ms), world, dev)
    line = {"metric": METRIC, "value": n_all / (ms / 1e3), "unit": "boxes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == mra.PREC_FP64 else "bf16x3-split apply, f64 elsewhere", "data": "synthetic",
            "config": workload_config(w), "run": {"n_boxes": n_all, "k": w.k, "L": w.L, "thresh": w.thresh,
                       "Z": cfg["Z"], "psi_leaves": info["n_psi"], "apply_result_leaves": info["n_result"],
                       "bsh_terms": w.M, "potential_terms": cfg["M_potential"], "potential_fit_err": vfit,
                       "iterations_to_converge": len(hist), "solve_s": t_solve, "energy": E,
                       "energy_error": E + 0.5 * cfg["Z"] ** 2, "terms_kept": st["terms_kept"],
                       "precision": "fp64" if prec == mra.PREC_FP64 else "split",
                       "l2": "flushed by a 256 MB write before every step",
                       "parallelism": "single GPU" if world == 1 else f"replicas x{world}"},
            "roofline": {"bound": "alu" if prec == mra.PREC_FP64 else "tensor", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": "apply kernels of the non-standard apply (all levels)",
                         "peak_source": (fp64_peak_source() if prec == mra.PREC_FP64 else
                                         f"bf16 dense sustained, {pk_kind}"), "kernel_ms": kms,
                         "flops": "algorithmic (6k'^4+k'^3 per kept term, k' = k or 2k)",
                         "share_of_step": kms / ms},
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": n_all / (e2e_ms / 1e3), "unit": "boxes/s",
                    "h2d_bytes_per_step": keys_pin.numel() * 8 + coeffs_pin.numel() * 8,
                    "d2h_bytes_per_step": d2h}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_solver_step(w)
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_solver_step(w):
    """One iteration of the solve composed from the oracle's functions (product, non-standard
    apply with every term, truncation, inner products) on the oracle's own projections of -Z/r
    and the Gaussian start; the whole step is timed."""
    import math
    import oracle as O
    cfg = w.extra["solver"]
    Mv = cfg["M_potential"]
    _, _, _, c, t = O.fit_search(0.0, Mv, 1e-4, 2 * w.L)
    g = {"coef": -cfg["Z"] * c, "expnt": t, "cx": np.zeros(Mv), "cy": np.zeros(Mv), "cz": np.zeros(Mv)}
    Vk, Vc, _ = O.project(g, w.k, w.L, thresh=w.thresh, init_level=2, max_level=19)
    a = cfg["Z"] ** 2
    gp = {"coef": np.array([(2 * a / math.pi) ** 0.75]), "expnt": np.array([a]), "cx": np.zeros(1),
          "cy": np.zeros(1), "cz": np.zeros(1)}
    pk, pc, _ = O.project(gp, w.k, w.L, thresh=w.thresh, init_level=2, max_level=19)
    t0 = time.perf_counter()
    vk, vc = O.multiply(Vk, Vc, pk, pc, w.k, w.L)
    E = cfg["E0"]
    mu = math.sqrt(-2 * E)
    r_lo, r_hi = O.kernel_range(O.BSH, mu, w.L, w.fit_eps)
    _, _, _, cb, tb = O.fit_search(mu, w.M, r_lo, r_hi)
    rk, rc = O.apply_ns_tree(vk, vc, w.k, w.L, 1, cb, tb, w.max_disp)
    rc = rc * (-1.0 / (2.0 * math.pi))
    nk, nc, _ = O.truncate(rk, rc, w.k, w.thresh)
    O.inner(vk, vc, pk, pc, w.k)
    O.inner(vk, vc, nk, nc, w.k)
    O.inner(nk, nc, nk, nc, w.k)
    t_cpu = time.perf_counter() - t0
    return {"value": len(vk) / t_cpu, "unit": "boxes/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"one whole iteration from the Gaussian start ({len(vk)} leaves of V psi), {t_cpu:.1f} s"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    extra = W.WORKLOADS[args.workload]().extra
    if "ns" in extra:
        return run_ns(args, W.WORKLOADS[args.workload](), rank, world)
    if "post" in extra:
        return run_post(args, W.WORKLOADS[args.workload](), rank, world)
    if "solver" in extra:
        return run_solver(args, W.WORKLOADS[args.workload](), rank, world)

    import torch
    from paper_1507_01888_gb300 import mra

    local = local % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)
    dev = torch.device("cuda", local)
    w = W.shard(W.WORKLOADS[args.workload](), rank, world)
    if args.partition and world > 1 and len(w.funcs) == 1:
        return run_partitioned(args, w, rank, world, local)
    precision = args.precision
    if precision == "auto":
        precision = "split"
    prec = mra.PREC_SPLIT_BF16 if precision == "split" else mra.PREC_FP64

    # ---------------- setup (untimed): projection, operator, buffers, tile-width tuning
    trees = [mra.project(f, w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level,
                         uniform_level=w.uniform_level) for f in w.funcs]
    batched = len(trees) > 1
    if batched:
        tree, offsets = mra.concat_trees(trees)
    else:
        tree, offsets = trees[0], [0, trees[0].n]
    keys_h, coeffs_h = tree.host()
    levels = (keys_h >> np.uint64(57)).astype(int)
    train_trees = [mra.project(f, w.k, w.L, thresh=w.thresh, init_level=w.init_level, max_level=w.max_level,
                               uniform_level=w.uniform_level) for f in w.extra.get("train_funcs", [])]
    lev_lo, lev_hi = int(levels.min()), int(levels.max())
    for t in train_trees:
        tl = (t.host()[0] >> np.uint64(57)).astype(int)
        lev_lo, lev_hi = min(lev_lo, int(tl.min())), max(lev_hi, int(tl.max()))
    op = mra.Operator(w.kernel, w.M, w.k, w.L, lev_lo, lev_hi, max_disp=w.max_disp, mu=w.mu, fit_eps=w.fit_eps)
    screen = mra.SCREEN_NORM if w.tau > 0 else mra.SCREEN_NONE
    opts = mra.make_opts(precision=prec, pieces=args.pieces, screen=screen, tau=w.tau, stencil=w.stencil,
                         max_disp=w.max_disp)
    learned_cfg = None
    if train_trees:  # learned screen: train the network on terms logged from the training functions
        from paper_1507_01888_gb300 import learned
        model, linfo = learned.train_screen(op, train_trees, opts, terms_per_tree=20000, steps=2000,
                                            batch=1024, lr=3e-3, seed=0, quantile=args.learned_quantile)
        opts = mra.make_opts(precision=prec, pieces=args.pieces, screen=mra.SCREEN_LEARNED, tau=w.tau,
                             stencil=w.stencil, max_disp=w.max_disp, mlp=model, delta=linfo["delta"],
                             delta_level=linfo["delta_level"])
        learned_cfg = {"training_functions": len(train_trees), "logged_terms": linfo["n_train"] + linfo["n_val"],
                       "final_loss": linfo["final_loss"], "delta": linfo["delta"], "quantile": args.learned_quantile,
                       "delta_level": {str(n): d for n, d in enumerate(linfo["delta_level"]) if d != float("inf")},
                       "held_out_terms_per_level": {str(n): c for n, c in linfo["val_per_level"].items()}}
        del train_trees
    tuning = {}
    if prec == mra.PREC_SPLIT_BF16 and args.schedule:
        opts, tuning = fixed_schedule(opts, args.schedule)
    elif prec == mra.PREC_SPLIT_BF16:
        from paper_1507_01888_gb300 import autotune

        def batched_applier(o):
            return mra.BatchedApplier(op, tree, offsets, o)
        opts, table = autotune.tune(op, tree, opts, make_applier=batched_applier if batched else None)
        tuning = {"choice": autotune.describe(opts), "candidates": table}

    def make_applier(o):
        if batched:
            ba = mra.BatchedApplier(op, tree, offsets, o)
            return ba
        return mra.Applier(op, tree, o)

    ap = make_applier(opts)

    def run(a, t):
        return a(t)[0] if batched else a(t)

    run(ap, tree)
    torch.cuda.synchronize()
    st0 = ap.stats.as_dict()
    k = w.k
    flops_per_term = 6 * k ** 4 + k ** 3
    # accuracy of the timed path against the FP64 GPU apply (same screen)
    accuracy = {}
    if prec != mra.PREC_FP64:
        ref_ap = make_applier(mra.make_opts(precision=mra.PREC_FP64, screen=screen, tau=w.tau,
                                            stencil=w.stencil, max_disp=w.max_disp))
        if batched:  # keys are sorted within each function only: compare function by function
            ref_out, ref_offs = ref_ap(tree)
            _, offs_out = ap(tree)
            d2 = r2 = mx = 0.0
            lev = {}
            for f in range(len(trees)):
                def sl(t, o):
                    return mra.Tree(t.keys[o[f]:o[f + 1]], t.coeffs[o[f]:o[f + 1]], o[f + 1] - o[f], t.k, t.L)
                if offs_out[f + 1] == offs_out[f] and ref_offs[f + 1] == ref_offs[f]:
                    continue
                c = mra.compare(sl(ap.out, offs_out), sl(ref_out, ref_offs))
                d2 += c["diff_norm"] ** 2
                r2 += c["ref_norm"] ** 2
                mx = max(mx, c["max_box_rel"])
                for x in c["levels"]:
                    a_ = lev.setdefault(x["level"], [0.0, 0.0, 0])
                    a_[0] += x["diff_norm"] ** 2
                    a_[1] += x["ref_norm"] ** 2
                    a_[2] += x["ref_boxes"]
            cmp = {"rel_l2": (d2 / r2) ** 0.5 if r2 > 0 else 0.0, "max_box_rel": mx,
                   "levels": [{"level": n, "rel_l2": (v[0] / v[1]) ** 0.5 if v[1] > 0 else v[0] ** 0.5,
                               "ref_boxes": v[2]} for n, v in sorted(lev.items())]}
        else:
            ref_out = run(ref_ap, tree)
            cmp = mra.compare(ap.out, ref_out)
        accuracy = {"rel_l2_vs_fp64_gpu": cmp["rel_l2"], "max_box_rel_vs_fp64_gpu": cmp["max_box_rel"],
                    "per_level_rel_l2_vs_fp64_gpu": {str(x["level"]): x["rel_l2"] for x in cmp["levels"]},
                    "fp64_gpu_apply_ms": ref_ap.stats.kernel_ms,
                    "speedup_vs_fp64_gpu_kernel": ref_ap.stats.kernel_ms / max(ap.stats.kernel_ms, 1e-9)}
        del ref_out, ref_ap

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    graph = None
    if batched or (prec == mra.PREC_SPLIT_BF16 and not learned_cfg):
        # the whole apply recorded once as a CUDA graph, one launch per step (no host
        # synchronisation between its kernels); the plain apply above gave the same result
        graph = mra.ApplyGraph(op, tree, opts, offsets=offsets if batched else None, stream=stream)
        if not batched:  # a replay is the plain apply, bit for bit
            g_out = graph.launch(stream)
            graph.status(stream)
            assert g_out.n == ap.out.n and torch.equal(g_out.keys[:g_out.n], ap.out.keys[:ap.out.n]) and \
                torch.equal(g_out.coeffs[:g_out.n], ap.out.coeffs[:ap.out.n]), "graph replay differs from the apply"

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            ap(tree, stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(args.clocks_csv)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms, main_ms = [], []
    launches0 = mra.launch_count()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        if graph is None:
            kernel_ms.append(ap.stats.kernel_ms)
            main_ms.append(ap.stats.main_kernel_ms)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = mra.launch_count() - launches0
    if graph is not None:
        graph.status(stream)  # every replay kept the recorded sizes
        for _ in range(3):  # the apply kernel's own time, from plain applies of the same input
            ap(tree, stream)
            kernel_ms.append(ap.stats.kernel_ms)
            main_ms.append(ap.stats.main_kernel_ms)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = clocks_stop(clk, local)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    n_in = tree.n
    n_all, ms = reduce_over_ranks(n_in, statistics.mean(step_ms), world, dev)
    value = n_all / (ms / 1e3)

    # ---------------- end to end through the public API with host buffers
    keys_pin = torch.from_numpy(keys_h.view(np.int64).copy()).pin_memory()
    coeffs_pin = torch.from_numpy(coeffs_h.copy()).pin_memory()
    n_out = ap.out.n
    out_keys_pin = torch.empty(n_out, dtype=torch.int64).pin_memory()
    out_coeffs_pin = torch.empty((n_out, k, k, k), dtype=torch.float64).pin_memory()

    def e2e_step():
        if batched:  # the graph reads the tree's own buffers
            tree.keys[:n_in].copy_(keys_pin, non_blocking=True)
            tree.coeffs[:n_in].copy_(coeffs_pin, non_blocking=True)
            out = graph.launch(stream)
        else:  # one C-ABI call on host buffers: copies in, apply, copies out
            n_got, _ = mra.apply_host(op, keys_pin, coeffs_pin, opts, out_keys_pin, out_coeffs_pin, stream)
            assert n_got == n_out
            return
        out_keys_pin.copy_(out.keys[:n_out], non_blocking=True)
        out_coeffs_pin.copy_(out.coeffs[:n_out], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e_ms.append(a.elapsed_time(b))
    if graph is not None:
        graph.status(stream)
    _, e2e_ms = reduce_over_ranks(n_in, statistics.mean(e_ms), world, dev)
    e2e_val = n_all / (e2e_ms / 1e3)
    h2d = keys_pin.numel() * 8 + coeffs_pin.numel() * 8
    d2h = out_keys_pin.numel() * 8 + out_coeffs_pin.numel() * 8

    # ---------------- roofline of the dominant kernel (the apply kernel)
    pk, pk_kind = peaks()
    kms = statistics.mean(main_ms)  # the dominant kernel alone
    apply_ms = statistics.mean(kernel_ms)  # with the kernels around it
    terms = st0["terms_kept"]
    achieved_tflops = terms * flops_per_term / (kms / 1e3) / 1e12
    if prec == mra.PREC_FP64:
        p64 = fp64_peak(local)["dfma_tflops"]
        roof = {"bound": "alu", "achieved": achieved_tflops, "peak": p64, "unit": "TFLOP/s",
                "frac": achieved_tflops / p64, "traffic": None,
                "kernel": "apply_f64_kernel", "peak_source": fp64_peak_source(local),
                "kernel_ms": kms}
        dtype = "f64"
    else:
        peak = pk.get("bf16_tflops", 1856.3)
        roof = {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak,
                "traffic": SPLIT_TRAFFIC.get((w.name, mra.KERNEL_NAMES[st0["kernel"]])) if not batched else None,
                "kernel": mra.KERNEL_NAMES[st0["kernel"]],
                "apply_ms": apply_ms,
                "apply_ms_covers": ("the kernel with its work-list (sort, tiles) and per-destination "
                                    "summation kernels" if st0["kernel"] == mra.KERNEL_SPLIT_SRC else
                                    "the kernel alone"),
                "peak_source": f"bf16 dense burst, {pk_kind}", "kernel_ms": kms,
                "flops": "algorithmic (6k^4+k^3 per kept term)"}
        if st0["kernel"] == mra.KERNEL_SPLIT_SRC and st0.get("mma_passes", 0) > 0:
            # each pass issues M=128, K=16 MMAs over 16 (P(P+1)/2) columns in stages 1 and 2 and 48
            # (P(P+1)/2) in stage 3 (three l_z): the tensor core's own work, padding included
            cols = 80 * args.pieces * (args.pieces + 1) // 2
            issued = st0["mma_passes"] * 2 * 128 * 16 * cols / (kms / 1e3) / 1e12
            roof["issued"] = {"tflops": issued, "frac": issued / peak, "passes": st0["mma_passes"],
                              "terms_per_pass": terms / st0["mma_passes"],
                              "note": "BF16 flops the MMAs issue (k padded to 16, the six piece products, "
                                      "windows of three l_z); context only, not the algorithmic rate"}
        if (st0["kernel"] == mra.KERNEL_SPLIT_DEST and int(opts.tile_variant) == 2 and k * k <= 128
                and 128 // (k * k) == 1 and args.pieces == 3):
            # one slot per 128-row tile: each kept term issues 3 + 3 + 5 MMAs of M=128, K=16 with
            # N = 48, 32, 16 | 48, 32, 16 | 32, 16, 16, 16, 16 -- the tensor core's own work
            issued = terms * 2 * 128 * 16 * (96 + 96 + 96) / (kms / 1e3) / 1e12
            roof["issued"] = {"tflops": issued, "frac": issued / peak,
                              "note": "BF16 flops the MMAs issue (padding to 128x16x16 tiles and the six "
                                      "piece products included); context only, not the algorithmic rate"}
        dtype = split_dtype(args.pieces, opts, k)

    line = {"metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": workload_config(w), "run": {"n_boxes": n_all, "k": k, "M": w.M,
                       "kernel": "bsh" if w.kernel == W.BSH else "poisson", "mu": w.mu, "tau": w.tau,
                       "stencil": "shells<=%d" % w.max_disp if w.stencil == 0 else "27-point",
                       "terms_kept": terms, "pairs": st0["pairs"], "n_out": st0["n_out"],
                       "per_level": {str(n): [c["sources"], c["terms_kept"]] for n, c in st0["levels"].items()},
                       "precision": precision, "l2": "flushed by a 256 MB write before every step",
                       "functions": len(trees), "tuning": tuning,
                       **({"launch": f"one CUDA graph per step ({graph.kernels_per_launch} library kernels "
                                     "recorded: norms, screen, sorts, apply)"} if graph is not None else {}),
                       **({"learned_screen": dict(learned_cfg, terms_skipped=st0["terms_learned_skipped"],
                                                  skipped_bound=st0["learned_skipped_bound"])}
                          if learned_cfg else {}),
                       "parallelism": ("single GPU" if world == 1 else
                                       f"{world} ranks, own functions each" if "rank_funcs" in w.extra
                                       else f"replicas x{world}")},
            "roofline": roof, "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": "boxes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "accuracy": accuracy, "wall_s_timed": t_wall}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not batched:
        cb = cpu_baseline(w, args.cpu_seconds)
        t_job = cb["t_sample"] * cb["terms_total"] / max(cb["sample_terms"], 1)
        line["cpu_baseline"] = {"value": cb["n_in"] / t_job, "unit": "boxes/s", "cores": cb["cores"],
                                "kind": "oracle",
                                "sample": f"{cb['sample_dest']} seeded destination boxes of {cb['dest_total']} "
                                          f"({cb['sample_terms']} of {cb['terms_total']} kept terms, "
                                          f"{cb['t_sample']:.1f} s); job time extrapolated by kept terms"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
