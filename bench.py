#!/usr/bin/env python3
"""Benchmark: interaction pairs screened per second at >= 95% planted recall.

Workload (default, ``gwas_large``): the SNP-shaped binary problem n = 4000,
p = 1,000,000 (about 5e11 pairs) with 10 planted pairs of target strength
U[0.15, 0.5] (realised after the generator's feasibility scaling: 0.12 ..
0.37) and 10 main effects.  kappa = 0.28, so the 4 planted pairs with
strength >= 0.28 are the targets; M = 23 from the gamma0 = 0.55 rule of
Section 5.2 (M = round(log p / log(1/0.55))), and L is the least number of
runs that finds the weakest target with probability >= 0.95 (eq. L_choice).
One step is one complete search (all L runs: keys, survivor filter,
grouping, verification, union) with its own seed; "pairs screened" is
p(p-1)/2 per search.  The recall gate reports, per target, how often the
timed searches found it against its own eta(M, L).

Timing: inputs are resident in HBM before the timed region; each step is
bracketed by CUDA events on the library's stream, and a 256 MiB buffer is
written between steps to flush L2 (outside the timed window).  The e2e
figure repeats the step through the public host-pointer API: pinned host
X/Y -> xyz_create (copy + pack) -> xyz_search -> results to host ->
xyz_destroy.  The roofline denominators are measured in the same run by the
library's probe (xyz_probe_peaks): integer ALU-pipe and popcount rates at
the clock of the moment.

Extra keys of the default line: the operating point chosen by the
library's autotuner (M by measured cost, same recall target), the point of
eq. bestM (the paper's plug-in rule), the exhaustive GPU screen of all
pairs, the oracle on all host cores (cpu_baseline), and the two patterns
(``batch``: 256 responses on one X plus 64 uneven instances; ``serve``: a
Poisson stream over 32 resident datasets), each against the plain
one-search-per-call path.

--impl reference times the CPU oracle (plain C) on all host cores on a
bounded sample of runs of the same workload and operating point.  With
--gpus N > 1 (under torchrun) one search's runs are split over the ranks by
run range (xyz_search_range) and merged on rank 0 (strong scaling);
--scaling weak gives every rank its own searches instead.  --pattern
batch|serve|scaling|continuous runs one pattern alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "interaction pairs screened/s at ≥95% planted recall; p50/p99 search latency"
UNIT = "pairs/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------- workload

def make_workload(name: str):
    from paper_1610_05108_gb300 import synth
    if name == "gwas_large":
        d = synth.config_gwas_large(1)
        kappa = 0.28
        label = ("gwas n=4000 p=1000000 (AR(0.6) blocks of 20, MAF U[0.05,0.5], 10 planted pairs "
                 "U[0.15,0.5] + 10 main effects)")
    elif name == "gwas_mid":
        from paper_1610_05108_gb300 import synth as _s
        r = _s.rng_for(1, "plant")
        d = _s.gwas(4000, 300000, 1, targets=tuple(float(t) for t in r.uniform(0.15, 0.5, size=10)))
        kappa = 0.28
        label = ("gwas n=4000 p=300000 (AR(0.6) blocks of 20, MAF U[0.05,0.5], 10 planted pairs "
                 "U[0.15,0.5] + 10 main effects): a smaller case of the class-split filter")
    elif name == "gwas":
        d = synth.config_gwas(1)
        kappa = 0.3
        label = "gwas n=2000 p=100000 (AR(0.6) blocks of 20, MAF U[0.05,0.5], 5 planted pairs + 10 main effects)"
    elif name == "small":
        d = synth.config_small(1)
        kappa = 0.5
        label = "iid n=200 p=2000, Y = X_0 o X_1 flipped w.p. 0.1"
    else:
        raise SystemExit(f"unknown workload {name}")
    return d, kappa, label


# ------------------------------------------------------------- planning
# The same arithmetic as the library's host planner (xyz_M_for_gamma0,
# xyz_runs_for_recall, xyz_eta), written out here so that the reference arm
# plans without the library; the GPU arm checks the two agree.

def m_for_gamma0(p: int, gamma0: float = 0.55) -> int:
    m = math.log(p) / math.log(1.0 / gamma0)
    return max(1, min(64, int(math.floor(m + 0.5))))


def _hit(beta: float, L: float) -> float:
    return 1.0 if beta >= 1.0 else -math.expm1(L * math.log1p(-beta))


def runs_for_recall(beta: float, eta: float) -> int:
    if beta >= 1.0:
        return 1
    L = max(1, int(math.ceil(math.log1p(-eta) / math.log1p(-beta))))
    while _hit(beta, L) < eta:
        L += 1
    while L > 1 and _hit(beta, L - 1) >= eta:
        L -= 1
    return L


def plan(d, kappa: float):
    """M by the gamma0 = 0.55 rule, L for 95% recall of the weakest target
    (the planted pairs with strength >= kappa), eta of every target."""
    M = m_for_gamma0(d.p)
    targets = [(tuple(pr), s) for pr, s in zip(d.planted, d.strengths) if s >= kappa]
    g_min = (1.0 + min(s for _, s in targets)) / 2.0
    L = runs_for_recall(g_min ** M, 0.95)
    eta = [_hit(((1.0 + s) / 2.0) ** M, L) for _, s in targets]
    return M, L, targets, eta


# --------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- peaks

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return dict(FALLBACK_PEAKS)


def load_traffic():
    """ncu DRAM bytes per launch recorded under profiles/ (null when the
    kernel source changed since the capture)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    try:
        rec = json.load(open(path))
    except Exception:
        return {}
    out = {}
    for key, v in rec.items():
        src = os.path.join(ROOT, v.get("source", ""))
        if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == v.get("sha"):
            out[key] = v
    return out


# Algorithmic integer work of the survivor filter per column and run: the
# 32 x 32 bit transpose that forms the M-bit keys (304 ALU-pipe operations per
# 32 columns: 64 byte permutes for the 16- and 8-bit rounds, 5 operations for
# each of the 48 masked swaps of the 4-, 2- and 1-bit rounds), 6 to insert
# the key into a Bloom filter word (hash, word index, two bit positions, OR)
# and 8 to test kx ^ c (xor, hash, word, bits, compare).  The denominator is
# the measured integer ALU-pipe rate (lop3.b32), which also runs the shifts
# and byte permutes.
FILTER_OPS_PER_COLUMN = 304 / 32 + 6 + 8


# ----------------------------------------------------------- GPU arm

def _device_ctx(d, dev, stream, torch, xyz):
    with torch.cuda.stream(stream):
        dX = torch.from_numpy(np.ascontiguousarray(d.X.T)).to(dev)     # (p, n) rows = columns of X
        dY = torch.from_numpy(d.Y).to(dev)
    stream.synchronize()
    ctx = xyz.Context.from_device(dX.data_ptr(), dY.data_ptr(), d.n, d.p, stream.cuda_stream)
    stream.synchronize()
    del dX, dY
    return ctx


def _timed_searches(ctx, stream, flush, torch, L, M, kappa, seeds, hits):
    """Searches with the given seeds, each bracketed by CUDA events on the
    library's stream, L2 flushed before each (outside the events)."""
    ms, found, stats = [], [], []
    for s in seeds:
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ctx.search(L, M, kappa, s)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        found.append(hits(res))
        stats.append(ctx.stats())
    return ms, found, stats


def gpu_arm(args):
    import torch
    from paper_1610_05108_gb300 import build as _build
    from paper_1610_05108_gb300 import xyz

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        if rank == 0:
            _build.build()
        dist.barrier()
    else:
        _build.build()
    xyz.load()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    sharded = world > 1 and args.scaling == "strong"

    t0 = time.perf_counter()
    d, kappa, label = make_workload(args.workload)
    log(f"[bench] rank {rank}: data made in {time.perf_counter() - t0:.1f} s")
    stream = torch.cuda.Stream(device=dev)
    ctx = _device_ctx(d, dev, stream, torch, xyz)
    M, L, targets, eta = plan(d, kappa)
    assert M == xyz.M_for_gamma0(d.p, 0.55)
    assert L == xyz.runs_for_recall(((1 + min(s for _, s in targets)) / 2) ** M, 0.95)
    if args.M:
        M = args.M
        L = runs_for_recall(((1 + min(s for _, s in targets)) / 2) ** M, 0.95)
        eta = [_hit(((1.0 + s) / 2.0) ** M, L) for _, s in targets]
    if args.L:
        L = args.L
    log(f"[bench] rank {rank}: n={d.n} p={d.p} M={M} L={L} kappa={kappa} targets={targets} eta={eta}")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    pairs_per_search = d.p * (d.p - 1) // 2
    target_list = [pr for pr, _ in targets]

    def hits(res):
        got = set(zip(res["j"].tolist(), res["k"].tolist())) if len(res) else set()
        return [int(t in got) for t in target_list]

    peaks_probe = xyz.probe_peaks()
    seed_base = 1_000_003 * (rank + 1) if not sharded else 1_000_003
    from paper_1610_05108_gb300 import shard

    def one_search(seed):
        if not sharded:
            return ctx.search(L, M, kappa, seed)
        l0, l1 = shard.run_ranges(L, world)[rank]
        mine = ctx.search_range(l0, l1, M, kappa, seed) if l1 > l0 else None
        objs = [None] * world
        torch.distributed.all_gather_object(objs, shard._as_triples(mine))
        merged = shard.merge_pairs(objs)
        out = np.zeros(len(merged), dtype=xyz.PAIR_DTYPE)
        if len(merged):
            out["j"], out["k"], out["agree"] = merged[:, 0], merged[:, 1], merged[:, 2]
        return out

    for w in range(args.warmup):
        one_search(seed_base + 10_000 + w)
    ctx.set_timing(True)
    sampler = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms, found, stats = [], [], []
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)                       # L2 flush, outside the timed window
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t_host = time.perf_counter()
        res = one_search(seed_base + s)
        e1.record(stream)
        e1.synchronize()
        el = e0.elapsed_time(e1) if not sharded else (time.perf_counter() - t_host) * 1e3
        if world > 1:
            t = torch.tensor([el], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            el = float(t.item())
        step_ms.append(el)
        found.append(hits(res))
        stats.append(ctx.stats())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    searches = args.steps * (world if (world > 1 and not sharded) else 1)
    value = pairs_per_search * searches / (total_ms / 1e3)

    # per-stage device time and the dominant kernel's roofline
    stages = ["keys", "sort", "join", "verify", "dedup"]
    ms_stage = {st: sum(x[f"ms_{st}"] for x in stats) for st in stages}
    launches_stage = {st: sum(x[f"launches_{st}"] for x in stats) for st in stages}
    cand = sum(x["candidates"] for x in stats)
    runs = sum(x["runs"] for x in stats)
    chunks = sum(x["chunks"] for x in stats)
    surv = sum(x["survivors"] for x in stats)
    big = d.p > 262144
    kname = "filter_big_kernel" if big else "filter_kernel"
    filt_s = ms_stage["keys"] / 1e3
    alu_peak = peaks_probe["alu_ops_per_s"]
    achieved = runs * d.p * FILTER_OPS_PER_COLUMN / filt_s if filt_s > 0 else 0.0
    traffic = load_traffic().get(f"{kname}:{args.workload}")
    roofline = {
        "bound": "alu", "kernel": kname,
        "achieved": round(achieved / 1e12, 3), "peak": round(alu_peak / 1e12, 3), "unit": "TOPS (int32)",
        "frac": round(achieved / alu_peak, 4),
        "peak_source": (f"measured in this run: lop3.b32 chains on {peaks_probe['sms']} SMs at "
                        f"{peaks_probe['sm_mhz']:.0f} MHz (xyz_probe_peaks)"),
        "work_per_unit": f"{FILTER_OPS_PER_COLUMN:.1f} integer ALU-pipe ops per column per run "
                         "(key transpose 9.5, Bloom insert 6, Bloom test 8)",
        "traffic": traffic.get("bytes_per_launch") if traffic else None,
        "traffic_units": traffic.get("units_per_launch") if traffic else None,
        "traffic_note": traffic.get("note") if traffic else "no ncu capture of the current kernel source",
        "launches": launches_stage["keys"], "launch_groups": chunks,
        "stage_ms": {k: round(v, 3) for k, v in ms_stage.items()},
        "stage_share": {k: round(v / max(1e-9, sum(ms_stage.values())), 4) for k, v in ms_stage.items()},
    }
    # verification: term (iv) of Section 2.3.  Its algorithmic work: every
    # distinct column of a bucket read once (4W bytes) and W popcounts per
    # candidate; the slower of the two at the measured peaks bounds it.
    W = (d.n + 31) // 32
    ver_s = ms_stage["verify"] / 1e3
    members = sum(x["bucket_members"] for x in stats)
    hbm = float(load_peaks()["hbm_gbs"]) * 1e9
    # packed columns that fit in L2 (half of its 126 MB, say) are not read
    # from HBM after the first touch: then only the popcounts bound it
    Wp = (W + 3) // 4 * 4
    l2_resident = d.p * 4 * Wp <= 64 * 2**20
    t_bytes = 0.0 if l2_resident else members * 4 * W / hbm
    t_popc = cand * W / peaks_probe["popc_ops_per_s"]
    vb = "hbm" if t_bytes >= t_popc else "popc"
    verify_roofline = {
        "bound": vb, "kernel": "verify_kernel",
        "achieved": round((members * 4 * W / ver_s / 1e9) if vb == "hbm" else (cand * W / ver_s / 1e12), 3)
        if ver_s > 0 else 0.0,
        "peak": round(hbm / 1e9, 1) if vb == "hbm" else round(peaks_probe["popc_ops_per_s"] / 1e12, 3),
        "unit": "GB/s" if vb == "hbm" else "Tpopc/s",
        "frac": round(max(t_bytes, t_popc) / ver_s, 4) if ver_s > 0 else 0.0,
        "work_per_unit": f"{4 * W} bytes per distinct bucket column (columns of spilled runs not counted; "
                         f"none when the packed columns fit in L2) and {W} popcounts per candidate",
        "packed_columns_l2_resident": l2_resident,
        "traffic": (load_traffic().get(f"verify_kernel:{args.workload}") or {}).get("bytes_per_launch"),
        "traffic_units": (load_traffic().get(f"verify_kernel:{args.workload}") or {}).get("units_per_launch"),
        "bytes_alg": members * 4 * W, "popc_alg": cand * W, "t_hbm_ms": round(t_bytes * 1e3, 3),
        "t_popc_ms": round(t_popc * 1e3, 3),
        "peak_source": f"HBM: MEASURED_PEAKS.json hbm_gbs ({load_peaks().get('source')}); popc: measured in "
                       "this run (xyz_probe_peaks)"}

    fr = np.asarray(found, dtype=np.float64)          # steps x targets
    recall = float(fr.mean()) if fr.size else 0.0
    gpu_launches = sum(x["gpu_launches"] for x in stats)
    lat = sorted(step_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": label, "n": d.n, "p": d.p, "M": M, "L": L, "kappa": kappa,
                   "M_rule": "gamma0 = 0.55 (Section 5.2): M = round(log p / log(1/0.55))",
                   "L_rule": "eq. L_choice: least L finding the weakest target with probability >= 0.95",
                   "planted_strengths": [round(s, 4) for s in d.strengths],
                   "targets": [list(pr) for pr in target_list],
                   "l2": "256 MiB buffer written between steps (L2 flush), outside the timed window",
                   "parallelism": (f"one search's runs split over {world} GPUs by run range, merged on the host"
                                   if sharded else f"independent searches per GPU x{world}")},
        "recall": {"measured": round(recall, 4), "expected_min_eta": round(min(eta), 4), "steps": args.steps,
                   "per_target": [{"pair": list(pr), "strength": round(s, 4), "eta": round(e, 4),
                                   "found_rate": round(float(fr[:, i].mean()), 4) if fr.size else 0.0}
                                  for i, ((pr, s), e) in enumerate(zip(targets, eta))]},
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                       "p99": round(float(np.percentile(lat, 99)), 3), "n": len(lat)},
        "roofline": roofline,
        "verify_roofline": verify_roofline,
        "peaks_measured": {k: (round(v / 1e12, 3) if k.endswith("per_s") else v) for k, v in peaks_probe.items()},
        "search_stats": {"attempts": [int(x["attempts"]) for x in stats],
                         "filter_kept_per_run": round(sum(x["filter_kept"] for x in stats) / max(1, runs), 1),
                         "candidates_per_run": round(cand / max(1, runs), 1),
                         "bucket_members_per_run": round(members / max(1, runs), 1),
                         "spilled_per_search": round(surv / max(1, len(stats)), 1)},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }

    if rank == 0 and not args.no_extra:
        out["autotuned"] = autotuned_leg(args, ctx, stream, flush, d, kappa, M, targets, xyz, torch, hits)
        out["paper_bestM"] = bestM_leg(args, ctx, stream, flush, d, kappa, targets, xyz, torch, hits)
        out["exhaustive"] = exhaustive_leg(ctx, stream, d, kappa, pairs_per_search, total_ms / args.steps,
                                           set(target_list), torch)
    ctx.close()
    del flush
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(args, d, kappa, M, L, xyz, torch)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_leg(d, kappa, M, L, args.cpu_seconds)
    if rank == 0 and not args.no_patterns:
        torch.cuda.empty_cache()
        out["batch"] = batch_summary(args, xyz, torch)
        torch.cuda.empty_cache()
        out["serve"] = serve_summary(args, xyz, torch)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def autotuned_leg(args, ctx, stream, flush, d, kappa, M_rule, targets, xyz, torch, hits):
    """The operating point chosen by the library's autotuners (xyz_autotune_M
    over M_rule - 3 .. M_rule + 3 at 95% recall of the weakest target, then
    xyz_autotune_tiles for the launch shapes at that M), timed like the main
    line."""
    g_min = (1.0 + min(s_ for _, s_ in targets)) / 2.0
    t0 = time.perf_counter()
    M, L, pred, table = ctx.autotune_M(kappa, g_min, 0.95, max(1, M_rule - 3), min(31, M_rule + 3), seed=77)
    tiles, tiles_ms = ctx.autotune_tiles(M, kappa, seed=78, trial_runs=min(L, 4096))
    tune_s = time.perf_counter() - t0
    ctx.search(L, M, kappa, 5_999_999)              # warm-up at the chosen point
    ms, found, _ = _timed_searches(ctx, stream, flush, torch, L, M, kappa,
                                   [6_000_000 + s for s in range(args.extra_steps)], hits)
    t = float(np.mean(ms))
    ctx.set_tiles(0, 0, 0)                          # the main line's shapes again
    return {"M": M, "L": L, "tiles": tiles, "tiles_trial_ms": round(tiles_ms, 3),
            "ms_per_step": round(t, 3), "tuner_ms": round(pred, 3),
            "value": d.p * (d.p - 1) // 2 / (t / 1e3), "unit": UNIT, "steps": len(ms),
            "recall_measured": round(float(np.mean(found)), 4),
            "eta_min": round(xyz.eta(g_min, M, L), 4), "tuning_s": round(tune_s, 3),
            "table": [[int(r[0]), int(r[1]), round(float(r[2]), 3)] for r in table],
            "note": "M and launch shapes by this implementation's measured cost; same recall target"}


def bestM_leg(args, ctx, stream, flush, d, kappa, targets, xyz, torch, hits):
    """M by eq. bestM (the plug-in estimate of sum gamma_jk^M from 10^6
    sampled pairs, gamma = (1 + kappa)/2), L for the same recall target."""
    _, _, agree = ctx.sample_agree(10**6, 0x5EED)
    M, _ = xyz.best_M(d.n, d.p, (1.0 + kappa) / 2.0, agree)
    g_min = (1.0 + min(s_ for _, s_ in targets)) / 2.0
    L = xyz.runs_for_recall(g_min ** M, 0.95)
    steps = max(1, min(args.extra_steps, 2))
    ms, found, _ = _timed_searches(ctx, stream, flush, torch, L, M, kappa,
                                   [5_000_000 + s for s in range(steps)], hits)
    t = float(np.mean(ms))
    return {"M": M, "L": L, "ms_per_step": round(t, 3), "value": d.p * (d.p - 1) // 2 / (t / 1e3),
            "unit": UNIT, "steps": steps, "recall_measured": round(float(np.mean(found)), 4),
            "eta_min": round(xyz.eta(g_min, M, L), 4),
            "note": "the paper's cost model (eq. bestM), written for its CPU implementation"}


def exhaustive_leg(ctx, stream, d, kappa, pairs_per_search, ms_search, target_set, torch):
    """The exhaustive GPU screen of all pairs on the same data (recall 1 by
    construction), timed once beside the search."""
    if d.p <= 300000:
        ctx.brute_force(kappa)                     # warm-up (the large screen runs once)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = ctx.brute_force(kappa)
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1)
    got = {(int(a), int(b)) for a, b in zip(res["j"], res["k"])}
    return {"ms": round(t, 3), "value": pairs_per_search / (t / 1e3), "unit": UNIT,
            "pairs_found": len(res), "targets_found": sum(1 for x in target_set if x in got),
            "search_speedup": round(t / ms_search, 2),
            "kernel": "brute_kernel: 128 x 128 pair tiles, popcount over packed columns"}


def e2e_leg(args, d, kappa, M, L, xyz, torch):
    """Same search through the host-pointer API, copies inside the timing."""
    Xh = torch.from_numpy(np.ascontiguousarray(d.X.T)).pin_memory()
    Yh = torch.from_numpy(d.Y).pin_memory()
    Xv = Xh.numpy().T          # column-major view of the pinned buffer
    Yv = Yh.numpy()
    times, d2h, split = [], [], []
    steps = max(1, min(args.steps, args.e2e_steps))
    for s in range(steps + 1):
        t0 = time.perf_counter()
        c = xyz.Context.from_host(Xv, Yv)
        t1 = time.perf_counter()
        res = c.search(L, M, kappa, 7_000_000 + s)
        t2 = time.perf_counter()
        c.close()
        t3 = time.perf_counter()
        if s > 0:                       # first call warms the allocator
            times.append(t3 - t0)
            split.append((t1 - t0, t2 - t1, t3 - t2))
            d2h.append(len(res) * 16 + 16)
    t = float(np.mean(times))
    sp = np.mean(np.asarray(split), axis=0) * 1e3
    return {"value": d.p * (d.p - 1) // 2 / t, "unit": UNIT,
            "h2d_bytes_per_step": int(d.n * d.p + d.n), "d2h_bytes_per_step": int(np.mean(d2h)),
            "ms_per_step": round(t * 1e3, 3), "steps": steps,
            "split_ms": {"create": round(float(sp[0]), 3), "search": round(float(sp[1]), 3),
                         "destroy": round(float(sp[2]), 3)},
            "path": "pinned host X,Y -> xyz_create (H2D + pack) -> xyz_search -> pairs to host -> xyz_destroy"}


# --------------------------------------------------------- CPU oracle leg

def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_runs(d, kappa, M, seed, l_start, seconds, cores):
    """The oracle as it stands (plain C, one run per call) on ``cores`` host
    threads (the calls release the interpreter lock), each thread taking the
    next run from a shared counter, until ``seconds`` have passed; returns
    (runs done, elapsed seconds)."""
    import threading

    import oracle
    oracle.build()
    lock = threading.Lock()
    nxt = [l_start]
    done = [0]
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                if time.perf_counter() - t0 >= seconds:
                    return
                r = nxt[0]
                nxt[0] += 1
            oracle.xyz_range(d.X, d.Y, r, r + 1, M, kappa, seed)
            with lock:
                done[0] += 1

    th = [threading.Thread(target=worker) for _ in range(cores)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    return done[0], time.perf_counter() - t0


def cpu_leg(d, kappa, M, L, seconds):
    """The oracle, unchanged, on all host cores for a bounded time, scaled
    linearly to the L runs of one search (runs are i.i.d.)."""
    cores = _host_cores()
    runs, el = oracle_runs(d, kappa, M, 4242, 0, seconds, cores)
    per_search = el / max(1, runs) * L
    return {"value": d.p * (d.p - 1) // 2 / per_search, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{runs} of the {L} runs (seed 4242, same M, kappa) on {cores} threads in {el:.1f} s, "
                      f"scaled to one search"}


def reference_arm(args):
    """The oracle on all host cores at the GPU arm's workload, operating
    point, metric and unit: each step a bounded sample of runs, scaled to one
    search.  Under torchrun only rank 0 runs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    d, kappa, label = make_workload(args.workload)
    M, L, targets, eta = plan(d, kappa)
    if args.L:
        L = args.L
    cores = _host_cores()
    per_step, runs_step = [], []
    l_next = 0
    for w in range(args.warmup + args.steps):
        runs, el = oracle_runs(d, kappa, M, 4242, l_next, args.ref_seconds, cores)
        l_next += runs
        if w >= args.warmup:
            per_step.append(el)
            runs_step.append(runs)
    sample_s = float(np.sum(per_step))
    sample_runs = int(np.sum(runs_step))
    t_search = sample_s / max(1, sample_runs) * L
    value = d.p * (d.p - 1) // 2 / t_search
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_s / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
           "data": "synthetic",
           "config": {"workload": label, "n": d.n, "p": d.p, "M": M, "L": L, "kappa": kappa},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step: runs of the search for {args.ref_seconds:g} s on {cores} "
                                      f"threads; {sample_runs} runs in {sample_s:.1f} s over the timed steps"},
           "extrapolated_ms_per_search": round(t_search * 1e3, 1),
           "note": "ms_per_step is the measured sample time of a step; one whole search of L runs would take "
                   "extrapolated_ms_per_search (runs are i.i.d., so time scales linearly in L)",
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------- batch pattern

def batch_summary(args, xyz, torch):
    """Config 4: one SNP-shaped X (n = 2000, p = 200000) with B responses
    (3 planted pairs each, kappa = 0.4, M by eq. bestM, L for 95% recall of
    the weakest target) screened once by the batched search and once as B
    plain searches; plus uneven instances launched as one CUDA graph against
    one search after another."""
    from paper_1610_05108_gb300 import synth
    n, p, B = 2000, 200000, args.batch_responses
    t0 = time.perf_counter()
    X, _ = synth.gwas_X(n, p, synth.rng_for(21, "X"))
    Ys, planted, real = synth.extra_responses(X, B, 22, pairs_per_y=3, target_range=(0.45, 0.55),
                                                balance=True)
    log(f"[bench] batch: data made in {time.perf_counter() - t0:.1f} s")
    kappa = 0.4
    targets = [[pr for pr, s_ in zip(planted[b], real[b]) if s_ >= kappa] for b in range(B)]
    g_min = (1 + min(s_ for b in range(B) for s_ in real[b] if s_ >= kappa)) / 2
    seed = 77
    ctx = xyz.create(X, Ys[0])
    _, _, agree = ctx.sample_agree(10**6, 0x5EED)             # plug-in M of eq. bestM
    M, _ = xyz.best_M(n, p, (1 + kappa) / 2, agree)
    L = xyz.runs_for_recall(g_min ** M, 0.95)
    ctx.search_batch(Ys, L, M, kappa, seed + 1)                 # warm-up: sizes the workspace for B
    ctx.search(L, M, kappa, seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = ctx.search_batch(Ys, L, M, kappa, seed)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    plain = []
    for b in range(B):
        ctx.set_y(Ys[b])
        plain.append(ctx.search(L, M, kappa, seed))
    t_plain = time.perf_counter() - t0
    ctx.close()
    del X
    inst = instances_leg(args, xyz, torch) if args.batch_instances > 0 else None
    same = all(np.array_equal(a, b) for a, b in zip(got, plain))
    found = sum(1 for b in range(B) for pr in targets[b]
                if any((int(j), int(k)) == tuple(pr) for j, k in zip(got[b]["j"], got[b]["k"])))
    found_plain = sum(1 for b in range(B) for pr in targets[b]
                      if any((int(j), int(k)) == tuple(pr) for j, k in zip(plain[b]["j"], plain[b]["k"])))
    ntarget = sum(len(t) for t in targets)
    pairs = B * p * (p - 1) / 2
    return {"value": pairs / t_batch, "unit": UNIT, "ms_per_response": round(t_batch / B * 1e3, 3),
            "plain": {"value": pairs / t_plain, "ms_per_response": round(t_plain / B * 1e3, 3),
                      "recall": round(found_plain / max(1, ntarget), 4),
                      "path": "xyz_set_y + xyz_search per response"},
            "speedup_vs_plain": round(t_plain / t_batch, 3), "identical_to_plain": bool(same),
            "recall": {"found": found, "targets": ntarget, "measured": round(found / max(1, ntarget), 4),
                       "expected_min_eta": round(xyz.eta(g_min, M, L), 4)},
            "instances": inst,
            "config": {"workload": f"one SNP-shaped X n={n} p={p} with {B} responses x 3 planted pairs "
                                   f"(strength U[0.45,0.55] before scaling, balanced Y)",
                       "n": n, "p": p, "B": B, "M": M, "L": L, "kappa": kappa,
                       "timing": "host wall clock around the whole call, results on the host"}}


def instances_leg(args, xyz, torch):
    """Independent instances of log-uniform n in [500, 8000] and p in
    [1e4, 5e5] (i.i.d. X made on the device from a seeded generator, one
    planted pair of strength 0.8 each, M from gamma0 = 0.55, L for 95%
    recall): one search after another against all of them launched as one
    CUDA graph (xyz_search_many)."""
    from paper_1610_05108_gb300 import synth
    sizes = synth.instance_sizes(args.batch_instances, 44)
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    ctxs, L, M, kap, seeds, pairs = [], [], [], [], [], 0
    for i, (n, p) in enumerate(sizes):
        g.manual_seed(45_000 + i)
        dX = (torch.randint(0, 2, (p, n), generator=g, device=dev, dtype=torch.int8) * 2 - 1).to(torch.int8)
        dY = (dX[0] * dX[1]).to(torch.int8)
        flips = torch.randperm(n, generator=g, device=dev)[: n // 10]
        dY[flips] = -dY[flips]
        torch.cuda.synchronize()
        ctxs.append(xyz.Context.from_device(dX.data_ptr(), dY.data_ptr(), n, p, 0))
        torch.cuda.synchronize()
        del dX, dY
        m = xyz.M_for_gamma0(p, 0.55)
        M.append(m)
        L.append(xyz.runs_for_recall(0.9 ** m, 0.95))
        kap.append(0.6)
        seeds.append(1000 + i)
        pairs += p * (p - 1) // 2
    torch.cuda.empty_cache()
    for c, l_, m_, k_, s_ in zip(ctxs, L, M, kap, seeds):       # warm-up
        c.search(l_, m_, k_, s_)
    xyz.search_many(ctxs, L, M, kap, seeds)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alone = [c.search(l_, m_, k_, s_) for c, l_, m_, k_, s_ in zip(ctxs, L, M, kap, seeds)]
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    many = xyz.search_many(ctxs, L, M, kap, seeds)
    t_many = time.perf_counter() - t0
    for c in ctxs:
        c.set_fused_filter(False)
    xyz.search_many(ctxs, L, M, kap, seeds)           # warm-up of the unfused graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    unfused = xyz.search_many(ctxs, L, M, kap, seeds)
    t_unfused = time.perf_counter() - t0
    found = sum(int((0, 1) in set(zip(r["j"].tolist(), r["k"].tolist()))) for r in many)
    for c in ctxs:
        c.close()
    return {"count": len(sizes), "sizes": [list(x) for x in sizes], "M": M, "L": L,
            "sequential_s": round(t_seq, 4), "graph_s": round(t_many, 4),
            "graph_unfused_s": round(t_unfused, 4),
            "speedup": round(t_seq / t_many, 3), "value_graph": pairs / t_many,
            "value_sequential": pairs / t_seq, "unit": UNIT,
            "graph": "filters of one-group searches fused into one persistent launch per key class "
                     "(graph_unfused_s: each filter its own launch)",
            "identical": all(np.array_equal(a, b) for a, b in zip(alone, many))
                         and all(np.array_equal(a, b) for a, b in zip(alone, unfused)),
            "planted_found": found}


def batch_arm(args):
    import torch
    from paper_1610_05108_gb300 import build as _build
    from paper_1610_05108_gb300 import xyz
    _build.build()
    xyz.load()
    out = {"metric": METRIC, "pattern": "batch", "n_gpus": 1, "higher_is_better": True, "dtype": "u32",
           "data": "synthetic"}
    out.update(batch_summary(args, xyz, torch))
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------- serve pattern

def serve_summary(args, xyz, torch):
    """Config 5: a Poisson stream (200 requests/s) of searches with L in
    [20, 200] and kappa in [0.2, 0.6] over resident SNP-shaped datasets of
    log-uniform n in [500, 8000] and p in [1e4, 5e5] (a pool of 32), each
    request with its own response (one planted pair of gamma in {0.7, 0.8,
    0.9}) and M from the gamma0 = 0.55 rule; p50/p99 latency of the paced
    stream, throughput of the same requests submitted at once, and the plain
    path (one search after another)."""
    import threading

    from paper_1610_05108_gb300 import synth
    D, R = args.serve_datasets, 8
    sizes = synth.instance_sizes(D, 31)
    t0 = time.perf_counter()
    data = []
    for i, (n, p) in enumerate(sizes):
        X, f = synth.gwas_X(n, p, synth.rng_for(300 + i, "X"))
        Ys, pairs, real = synth.single_pair_responses(X, f, R, 400 + i)
        data.append((X, Ys, pairs, real))
    reqs = synth.serve_requests(args.serve_requests, args.serve_rate, 32, D, R)
    for q in reqs:
        n, p = sizes[q["dataset"]]
        q["M"] = xyz.M_for_gamma0(p, 0.55)
    log(f"[bench] serve: {D} datasets made in {time.perf_counter() - t0:.1f} s")

    # plain: the same searches one after another, one context per dataset
    ctxs = [xyz.create(X, Ys[0]) for X, Ys, _, _ in data]
    for i, c in enumerate(ctxs):                               # warm-up
        c.search(200, xyz.M_for_gamma0(sizes[i][1], 0.55), 0.2, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for q in reqs:
        c = ctxs[q["dataset"]]
        c.set_y(data[q["dataset"]][1][q["response"]])
        plain.append(c.search(q["L"], q["M"], q["kappa"], q["seed"]))
    t_plain = time.perf_counter() - t0
    for c in ctxs:
        c.close()

    def run_server(paced: bool):
        srv = xyz.Server(workers=args.serve_workers, hbm_budget_bytes=120 << 30,
                         slice_runs=args.serve_slice)
        ds = [srv.add_dataset(X, Ys[0]) for X, Ys, _, _ in data]
        for i in range(D):          # grow each worker's workspace before timing
            for r in [srv.submit(ds[i], 64, xyz.M_for_gamma0(sizes[i][1], 0.55), 0.2, 3)
                      for _ in range(args.serve_workers)]:
                srv.wait(r)
        ids = [None] * len(reqs)
        start = time.perf_counter()

        def producer():
            for i, q in enumerate(reqs):
                if paced:
                    dt = start + q["t"] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                ids[i] = srv.submit(ds[q["dataset"]], q["L"], q["M"], q["kappa"], q["seed"],
                                    Y=data[q["dataset"]][1][q["response"]])

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        res, lat = [], []
        for i in range(len(reqs)):
            r, l_ = srv.wait(ids[i])
            res.append(r)
            lat.append(l_)
        el = time.perf_counter() - start
        st = srv.stats()
        srv.close()
        return res, np.asarray(lat), el, st

    served, lat, el, st = run_server(True)
    sat, lat_sat, el_sat, _ = run_server(False)
    same = all(np.array_equal(a, b) for a, b in zip(served, plain)) and \
        all(np.array_equal(a, b) for a, b in zip(sat, plain))
    pairs_total = sum(sizes[q["dataset"]][1] * (sizes[q["dataset"]][1] - 1) / 2 for q in reqs)
    found = found_plain = targets = 0
    eta = []
    for q, r, rp in zip(reqs, served, plain):
        X, Ys, pairs, real = data[q["dataset"]]
        s_ = real[q["response"]]
        if s_ >= q["kappa"]:
            targets += 1
            pr = pairs[q["response"]]
            found += int(any((int(j), int(k)) == pr for j, k in zip(r["j"], r["k"])))
            found_plain += int(any((int(j), int(k)) == pr for j, k in zip(rp["j"], rp["k"])))
            eta.append(xyz.eta((1 + s_) / 2, q["M"], q["L"]))
    return {"value": pairs_total / el, "unit": UNIT,
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                           "p99": round(float(np.percentile(lat, 99)), 3), "n": len(lat)},
            "elapsed_s": round(el, 3), "arrivals_span_s": round(reqs[-1]["t"], 3),
            "saturated": {"value": pairs_total / el_sat, "elapsed_s": round(el_sat, 3),
                          "p50_ms": round(float(np.percentile(lat_sat, 50)), 3),
                          "p99_ms": round(float(np.percentile(lat_sat, 99)), 3),
                          "note": "all requests submitted at once"},
            "plain": {"value": pairs_total / t_plain, "elapsed_s": round(t_plain, 3),
                      "recall": round(found_plain / max(1, targets), 4),
                      "path": "one xyz_search per request, one after another"},
            "speedup_saturated_vs_plain": round(t_plain / el_sat, 3),
            "identical_to_plain": bool(same),
            "recall": {"found": found, "targets": targets, "measured": round(found / max(1, targets), 4),
                       "expected": round(float(np.mean(eta)) if eta else 0.0, 4)},
            "server": {"workers": args.serve_workers, "slice_runs": args.serve_slice,
                       "budget_bytes": 120 << 30, "device_bytes": st["device_bytes"]},
            "config": {"workload": f"Poisson {args.serve_rate:g} req/s, {len(reqs)} requests over {D} "
                                   "resident SNP-shaped datasets, n in [500,8000], p in [1e4,5e5] "
                                   "log-uniform, L in [20,200], kappa in [0.2,0.6]",
                       "datasets": [list(x) for x in sizes]}}


def serve_arm(args):
    import torch
    from paper_1610_05108_gb300 import build as _build
    from paper_1610_05108_gb300 import xyz
    _build.build()
    xyz.load()
    out = {"metric": METRIC, "pattern": "serve", "n_gpus": 1, "higher_is_better": True, "dtype": "u32",
           "data": "synthetic"}
    out.update(serve_summary(args, xyz, torch))
    print(json.dumps(out), flush=True)


# -------------------------------------------------------- scaling pattern

def scaling_arm(args):
    """Section 5.2: time for xyz to discover the one strong pair (0, 1) of
    strength gamma in {0.7, 0.8, 0.9} on i.i.d. +-1 data, against p, with M
    from gamma0 = p^(-1/M) ~ 0.55; the exhaustive GPU screen timed beside it.
    Theory (Theorem on minimal subsampling): time ~ n p^(1 + log gamma / log
    gamma0)."""
    import torch
    from paper_1610_05108_gb300 import build as _build
    from paper_1610_05108_gb300 import xyz
    _build.build()
    xyz.load()
    n = args.scaling_n
    ps = [int(v) for v in args.scaling_p.split(",")]
    gammas = (0.7, 0.8, 0.9)
    reps = args.scaling_reps
    rows = []
    rng = np.random.default_rng(1610)
    for p in ps:
        X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
        M = xyz.M_for_gamma0(p, 0.55)
        for g in gammas:
            Y = (X[:, 0] * X[:, 1]).astype(np.int8)
            flips = rng.choice(n, size=int(round((1 - g) * n)), replace=False)
            Y[flips] = -Y[flips]
            a12 = int(np.sum(Y == X[:, 0] * X[:, 1]))
            kappa = (2.0 * a12 - n) / n - 1e-9
            with xyz.create(X, Y) as ctx:
                expect = 1.0 / (a12 / n) ** M                  # mean runs to discovery
                step = max(1, int(expect / 4))
                ctx.search_range(0, step, M, kappa, 1)          # warm-up
                times, runs = [], []
                for r in range(reps):
                    seed = 1000 + r
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    l0 = 0
                    while True:
                        res = ctx.search_range(l0, l0 + step, M, kappa, seed)
                        l0 += step
                        if any(int(j) == 0 and int(k) == 1 for j, k in zip(res["j"], res["k"])):
                            break
                        if l0 > 200 * expect:
                            break
                    times.append(time.perf_counter() - t0)
                    runs.append(l0)
                ctx.brute_force(kappa)                          # warm-up
                t0 = time.perf_counter()
                bf = ctx.brute_force(kappa)
                t_bf = time.perf_counter() - t0
            found_bf = [(int(j), int(k)) for j, k in zip(bf["j"], bf["k"])] == [(0, 1)]
            rows.append({"p": p, "gamma": round(a12 / n, 4), "M": M, "runs_mean": float(np.mean(runs)),
                         "runs_expected": round(expect, 1), "xyz_ms": round(1e3 * float(np.mean(times)), 3),
                         "brute_ms": round(1e3 * t_bf, 3), "brute_found_only_pair": found_bf})
            log(f"[bench] scaling p={p} gamma={g} M={M} xyz {rows[-1]['xyz_ms']} ms brute {rows[-1]['brute_ms']} ms")
    fit = {}
    for g in gammas:
        rr = [r for r in rows if abs(r["gamma"] - g) < 0.01]
        big = [r for r in rr if r["p"] >= 10000]
        if len(big) >= 2:
            slope = float(np.polyfit(np.log([r["p"] for r in big]), np.log([r["xyz_ms"] for r in big]), 1)[0])
            work = float(np.polyfit(np.log([r["p"] for r in rr]),
                                    np.log([r["runs_mean"] * r["p"] for r in rr]), 1)[0])
            fit[str(g)] = {"time_slope_p_ge_1e4": round(slope, 3),
                           "work_slope": round(work, 3),
                           "theory": round(1 + np.log(g) / np.log(0.55), 3),
                           "note": "work = runs to discovery x p column keys; the time slope is "
                                   "flattened by the fixed cost of a call at small p"}
    out = {"metric": METRIC, "pattern": "scaling", "unit": "ms", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": f"iid +-1 X, n={n}, one planted pair (0,1) of gamma in {{0.7,0.8,0.9}}, "
                                  "M from gamma0=0.55, time to discovery (runs in slices of a quarter of "
                                  "the expected count) vs the exhaustive GPU screen",
                      "reps": reps},
           "rows": rows, "fit": fit}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------- continuous pattern

def realx_rows(args, xyz, torch):
    """Section 3.2's model on real X: X_ij ~ U(-1, 1), Y = X_a X_b + eps; the
    unbiased and the sign transforms, M from gamma0 = 0.55, L for 95% recall
    of the planted pair at its transformed strength (computed from the data)."""
    n, p = 2000, 20000
    rng = np.random.default_rng(33)
    X = rng.uniform(-1, 1, size=(n, p)).astype(np.float32, order="F")
    a, b = 77, 12345
    Y = X[:, a].astype(np.float64) * X[:, b] + rng.normal(0, 0.1, size=n)
    nu = np.abs(X).max(axis=1).astype(np.float64)
    Xs = X / nu[:, None].astype(np.float32)
    Yp = Y * nu * nu
    g_unb = 0.5 + float(np.sum(Yp * Xs[:, a].astype(np.float64) * Xs[:, b])) / (2 * np.abs(Yp).sum())
    g_sgn = 0.5 + float(np.sum(Y * np.sign(X[:, a]) * np.sign(X[:, b]))) / (2 * np.abs(Y).sum())
    M = xyz.M_for_gamma0(p, 0.55)
    rows = []
    for name, g, make in (("unbiased", g_unb, lambda: xyz.Context.from_real_unbiased(X, Y)),
                          ("sign", g_sgn, lambda: xyz.Context.from_real_sign(X))):
        L = xyz.runs_for_recall(g ** M, 0.95)
        kappa = 2 * (g - 0.05) - 1
        with make() as ctx:
            if name == "sign":
                ctx.set_y_real(Y)
            ctx.search(L, M, kappa, 1)
            ms, found = [], 0
            reps = max(args.steps, 40)
            for st in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = ctx.search(L, M, kappa, 200 + st)
                ms.append((time.perf_counter() - t0) * 1e3)
                found += int((a, b) in set(zip(res["j"].tolist(), res["k"].tolist())))
        rows.append({"transform": name, "gamma_g": round(float(g), 4), "M": M, "L": L,
                     "kappa": round(float(kappa), 4), "ms_per_search": round(float(np.mean(ms)), 3),
                     "value": p * (p - 1) / 2 / (float(np.mean(ms)) / 1e3),
                     "recall": round(found / reps, 3), "searches": reps})
        log(f"[bench] real X {rows[-1]}")
    return {"workload": f"X_ij ~ U(-1,1), n={n}, p={p}, Y = X_a X_b + N(0, 0.01)", "rows": rows}



def continuous_arm(args):
    """Section 3.1's model Y_i = X_ia X_ib + eps_i, eps ~ N(0, sigma^2), on
    i.i.d. +-1 X (n = 2000, p = 100000): weighted rows and strengths, M from
    gamma0 = 0.55, L for 95% recall of the planted pair from its weighted
    strength in closed form; the same shape with the binary response
    sgn(Y) timed beside it."""
    import torch
    from scipy.stats import norm
    from paper_1610_05108_gb300 import build as _build
    from paper_1610_05108_gb300 import xyz
    _build.build()
    xyz.load()
    n, p = 2000, 100000
    rng = np.random.default_rng(31)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    a, b = 123, 45678
    M = xyz.M_for_gamma0(p, 0.55)
    rows = []
    ctx = xyz.create(X, np.ones(n, np.int8))
    for s2 in (0.5, 1.0, 2.0):
        sd = float(np.sqrt(s2))
        Y = X[:, a].astype(np.float64) * X[:, b] + rng.normal(0, sd, size=n)
        g = (norm.cdf(1 / sd) + sd * norm.pdf(1 / sd)) / (2 * norm.cdf(1 / sd) - 1 + 2 * sd * norm.pdf(1 / sd))
        L = xyz.runs_for_recall(g ** M, 0.95)
        kappa = 2 * (g - 0.1) - 1                  # well below the pair, far above the bulk
        res_t = {}
        for mode in ("real", "sign"):
            if mode == "real":
                ctx.set_y_real(Y)
            else:
                ctx.set_y(np.where(Y < 0, -1, 1).astype(np.int8))
            ctx.search(L, M, kappa, 1)             # warm-up
            ms, found = [], 0
            reps = max(args.steps, 40)             # recall needs a few dozen searches
            for st in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = ctx.search(L, M, kappa, 100 + st)
                ms.append((time.perf_counter() - t0) * 1e3)
                found += int((a, b) in set(zip(res["j"].tolist(), res["k"].tolist())))
            res_t[mode] = {"ms_per_search": round(float(np.mean(ms)), 3),
                           "value": p * (p - 1) / 2 / (float(np.mean(ms)) / 1e3),
                           "recall": round(found / reps, 3), "searches": reps}
        rows.append({"sigma2": s2, "gamma_weighted": round(float(g), 4), "M": M, "L": L,
                     "kappa": round(kappa, 4), "real": res_t["real"], "sign_only": res_t["sign"]})
        log(f"[bench] continuous sigma2={s2} L={L} real {res_t['real']} sign {res_t['sign']}")
    ctx.close()
    realx = realx_rows(args, xyz, torch)
    out = {"metric": METRIC, "pattern": "continuous", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
           "real_x": realx,
           "dtype": "u32 keys, int64 fixed-point weights",
           "config": {"workload": f"iid +-1 X n={n} p={p}, Y = X_a X_b + N(0, sigma^2), weighted rows "
                                  "(Section 3.1); 'sign_only' is the binary search on sgn(Y) with the same L",
                      "steps": args.steps, "timing": "host wall clock per search, results on the host"},
           "rows": rows}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="gwas_large")
    ap.add_argument("--scaling", choices=["strong", "weak"], default="strong",
                    help="with --gpus N > 1: split one search's runs over the ranks (strong) or give every "
                         "rank its own searches (weak)")
    ap.add_argument("--L", type=int, default=0, help="override the number of runs")
    ap.add_argument("--M", type=int, default=0, help="override M (L then follows the recall rule)")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed searches of the autotuned and bestM legs")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=2.0, help="oracle time per step of --impl reference")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the autotuned, bestM and exhaustive legs")
    ap.add_argument("--no-patterns", action="store_true", help="skip the batch and serve keys")
    ap.add_argument("--pattern", choices=["search", "batch", "serve", "scaling", "continuous"],
                    default="search")
    ap.add_argument("--batch-responses", type=int, default=256)
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--serve-datasets", type=int, default=32)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-slice", type=int, default=128)
    ap.add_argument("--scaling-n", type=int, default=1000)
    ap.add_argument("--scaling-p", default="1000,3000,10000,30000,100000,250000")
    ap.add_argument("--scaling-reps", type=int, default=5)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gb300":
        log("[bench] warm-up raised to 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.pattern == "batch":
        batch_arm(args)
    elif args.pattern == "serve":
        serve_arm(args)
    elif args.pattern == "scaling":
        scaling_arm(args)
    elif args.pattern == "continuous":
        continuous_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
