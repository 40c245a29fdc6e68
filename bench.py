#!/usr/bin/env python
"""Throughput of the semiring SpGEMM C = A (+).(x) B on one GB300.

One step = the whole path (flops + binning, symbolic, scan, numeric with
in-row sort) for every product of the workload:

  rmat18 (default): R-MAT scale 18, edgefactor 16, a=0.57 b=c=0.19 d=0.05,
          symmetrised, duplicates removed, vertices permuted; C = A.A over
          (+,x) fp64 U(0,1), (min,+) uint32 U{1..255} and (or,and) bool.
  er16k:  ER n=16384 with exactly 8 distinct columns per row, (+,x) int64
          U{1..10}; C = A.A.

Inputs are seeded synthetic matrices resident in HBM; outputs go to
pre-reserved device buffers; validation is off inside the timed loop.  L2
is flushed (a 512 MB device write) before every timed step.  Each rank of a
multi-GPU launch runs an independent replica (weak scaling).

`--impl reference` times the CPU oracle on the host cores instead, on a
bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "semiring SpGEMM flops/s & nnz(C)/s on 1 GB300, learned/batched vs plain two-phase"
UNIT = "products/s"
VAL_BYTES = {"plus_times_i64": 8, "plus_times_f64": 8, "min_plus_u32": 4, "or_and_bool": 1,
             "sel2nd_min_i32": 4}
DTYPE_NAME = {"plus_times_i64": "int64", "plus_times_f64": "f64", "min_plus_u32": "u32",
              "or_and_bool": "u8", "sel2nd_min_i32": "i32"}


def workload(name: str):
    from paper_2106_14402_gb300 import gen
    if name == "rmat18":
        desc = ("R-MAT s18 ef16 (0.57/0.19/0.19/0.05) symmetrised+dedup+permuted; C=A.A over "
                "(+,x) f64, (min,+) u32, (or,and) bool")
        return desc, gen.rmat_square(18, 16, cfg=2)
    if name == "rmat16":
        desc = ("R-MAT s16 ef16 (0.57/0.19/0.19/0.05) symmetrised+dedup+permuted; C=A.A over (+,x) f64 "
                "(small profiling case)")
        return desc, gen.rmat_square(16, 16, cfg=2, semirings=("plus_times_f64",))
    if name == "er16k":
        desc = "ER n=16384, 8 distinct cols/row, (+,x) int64 U{1..10}; C=A.A"
        return desc, gen.er_square()
    if name == "blockclust":
        desc = ("block-clustered n=131072, clusters of 256, density 0.5, ~1 inter-cluster edge per "
                "vertex; C=A.A over (+,x) f64 (high-compression profiling case)")
        return desc, gen.high_compression()
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks of the process group (x itself without one):
    a multi-GPU step takes as long as its slowest rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each process units_per_rank
    units in `seconds` (the max over ranks): weak scaling."""
    return world * units_per_rank / seconds


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")
# the sources the fp64 numeric phase's kernels are built from: the measured
# traffic holds only while these are unchanged since the capture
NUMERIC_SOURCES = ("paper_2106_14402_gb300/csrc/k_numeric.cu", "paper_2106_14402_gb300/csrc/cb_common.cuh")


def sources_digest(paths=NUMERIC_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def fp64_traffic_per_product():
    """(DRAM bytes per product of the fp64 numeric phase, source note) from
    profiles/traffic.json, or (None, why) when absent or captured from other
    kernel sources."""
    try:
        with open(TRAFFIC_JSON) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None, "no traffic capture"
    if t.get("sources_digest") != sources_digest():
        return None, "kernel sources changed since the traffic capture"
    return float(t["fp64_numeric_bytes_per_product"]), t.get("capture", "")


# value bytes of A, B and C under the heterogeneous semiring
HETERO_VAL_BYTES = {"maxw_label": (4, 4, 8)}


def compulsory_bytes(sr, A, B, nnz_c, m):
    """bytes(A) + bytes(B rows touched, once) + bytes(C): row_ptr 8 B/row, col 4 B, val by type."""
    va, vb, vc = HETERO_VAL_BYTES.get(sr, (VAL_BYTES.get(sr),) * 3)
    a = 8 * (A.nrows + 1) + A.nnz * (4 + va)
    touched = np.unique(A.col)
    blen = np.diff(B.row_ptr)[touched]
    b = 8 * (touched.size + 1) + int(blen.sum()) * (4 + vb)
    c = 8 * (m + 1) + nnz_c * (4 + vc)
    return int(a + b + c)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        med = statistics.median(sm) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded row sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample_rate(problems, target_s: float = 12.0, seed: int = 0, keep=None):
    """Time the oracle on a seeded row sample of each product, sized to ~target_s in total.

    Returns (products/s, nnz/s, cores, description, seconds); with `keep` (a
    dict) the sampled rows and the oracle's output go to keep[semiring]."""
    import oracle
    cores = oracle.max_threads()
    rng = np.random.default_rng(seed)
    samples = []
    for sr, A, B in problems:
        flops, _ = oracle.row_stats(A, B)
        perm = rng.permutation(A.nrows)
        samples.append((sr, A, B, flops, perm))
    # calibrate on 0.2% of rows
    probe_prod, probe_t = 0, 0.0
    for sr, A, B, flops, perm in samples:
        rows = np.sort(perm[: max(1, A.nrows // 500)])
        t0 = time.perf_counter()
        oracle.spgemm(sr, A, B, rows=rows)
        probe_t += time.perf_counter() - t0
        probe_prod += int(flops[rows].sum())
    rate = probe_prod / max(probe_t, 1e-6)
    total_prod = sum(int(f.sum()) for _, _, _, f, _ in samples)
    frac = min(1.0, target_s * rate / max(total_prod, 1))
    prod, nnz, t = 0, 0, 0.0
    for sr, A, B, flops, perm in samples:
        rows = np.sort(perm[: max(1, int(A.nrows * frac))])
        t0 = time.perf_counter()
        res = oracle.spgemm(sr, A, B, rows=rows)
        t += time.perf_counter() - t0
        rp = res[0]
        if keep is not None:
            keep[sr] = (rows, res)
        prod += int(flops[rows].sum())
        nnz += int(rp[-1])
    desc = (f"seeded {frac * 100:.2f}% row sample of every product "
            f"({prod:.3e} products, {nnz:.3e} nnz(C)), oracle std::map Gustavson, OpenMP")
    return prod / t, nnz / t, cores, desc, t


def sampled_parity(dprob, kept):
    """The timed steps' last outputs on the oracle's sampled rows: exact
    equality for the integer, bool and min semirings; for (+,x) fp64 the
    largest |c - c_ref| / sum|a b| over the sampled entries (bound 1e-12)."""
    out = {}
    for sr, A, B, dA, dB, C, nnz in dprob:
        if sr not in kept:
            continue
        rows, (w_rp, w_col, w_val, w_abs) = kept[sr]
        g_rp = C.row_ptr[:A.nrows + 1].cpu().numpy()
        idx = np.concatenate([np.arange(g_rp[r], g_rp[r + 1]) for r in rows]) if len(rows) else \
            np.zeros(0, np.int64)
        torch = __import__("torch")
        it = torch.as_tensor(idx, device=C.col.device)
        g_col = C.col[it].cpu().numpy()
        if C.val.dtype == torch.uint32:  # no indexing kernels for uint32: go through int32
            g_val = C.val.view(torch.int32)[it].cpu().numpy().view(np.uint32)
        else:
            g_val = C.val[it].cpu().numpy()
        same = bool(np.array_equal(np.diff(g_rp)[rows], np.diff(w_rp)) and np.array_equal(g_col, w_col))
        rec = {"rows": int(len(rows)), "entries": int(idx.size), "pattern_equal": same}
        if sr == "plus_times_f64":
            ratio = np.abs(g_val - w_val) / np.where(w_abs > 0, w_abs, 1.0) if same else np.array([np.inf])
            rec["max_err_ratio"] = float(ratio.max()) if ratio.size else 0.0
            rec["bound"] = 1e-12
        else:
            rec["values_equal"] = bool(same and np.array_equal(g_val, w_val))
        out[sr] = rec
    return out


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    desc, problems = workload(args.workload)
    steps = []
    for _ in range(args.warmup):
        oracle_sample_rate(problems, target_s=2.0)
    for _ in range(args.steps):
        steps.append(oracle_sample_rate(problems, target_s=args.ref_seconds))
    rate = statistics.median(s[0] for s in steps)
    nnz_rate = statistics.median(s[1] for s in steps)
    cores, sample = steps[0][2], steps[0][3]
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.median(s[4] for s in steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": ",".join(DTYPE_NAME[sr] for sr, _, _ in problems), "data": "synthetic",
           "config": {"workload": desc, "sample": sample}, "nnz_per_s": nnz_rate,
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main_gpu(args):
    import torch

    from paper_2106_14402_gb300 import cb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cb.load()
    desc, problems = workload(args.workload)
    dev = torch.device("cuda", local)

    # device-resident inputs, pre-reserved outputs sized by one untimed call
    dprob = []
    for sr, A, B in problems:
        dA = cb.DeviceCSR.from_host(A, sr, dev)
        dB = dA if B is A else cb.DeviceCSR.from_host(B, sr, dev)
        C = cb.spgemm(sr, dA, dB, validate=True)
        nnz = C.nnz
        del C
        out = cb.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device=dev),
                           torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
                           torch.empty(max(nnz, 1), dtype=cb.SEMIRING[sr][1], device=dev))
        dprob.append((sr, A, B, dA, dB, out, nnz))
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = cb.context()

    def step(collect):
        launches = 0
        for sr, A, B, dA, dB, out, nnz in dprob:
            cb.spgemm(sr, dA, dB, validate=False, out=out, timing=True, ctx=ctx)
            st = ctx.stats()
            launches += st["kernels"]
            if collect is not None:
                collect.setdefault(sr, []).append(st)
        return launches

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    stats: dict = {}
    times = []
    launches = 0
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        launches += step(stats)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms_step = max_over_ranks(sum(times) / len(times), dist, dev)
    if dist:
        dist.barrier()

    products = sum(st[0]["flops"] for st in stats.values())
    nnz_c = sum(st[0]["nnz"] for st in stats.values())
    value = whole_job_rate(products, world, ms_step * 1e-3)
    nnz_rate = whole_job_rate(nnz_c, world, ms_step * 1e-3)

    # per-semiring breakdown and the numeric-phase roofline
    per_sr = {}
    num_bytes = 0
    num_ms = 0.0
    phase_tot = {"ms_stats": 0.0, "ms_symbolic": 0.0, "ms_scan": 0.0, "ms_numeric": 0.0}
    for sr, A, B, dA, dB, out, nnz in dprob:
        sts = stats[sr]
        ph = {k: statistics.median(s[k] for s in sts) for k in phase_tot}
        for k in phase_tot:
            phase_tot[k] += ph[k]
        cbytes = compulsory_bytes(sr, A, B, nnz, A.nrows)
        num_bytes += cbytes
        num_ms += ph["ms_numeric"]
        per_sr[sr] = {"products": sts[0]["flops"], "nnz_c": sts[0]["nnz"],
                      "heavy_rows": sts[0]["heavy_rows"], "heavy_units": sts[0]["heavy_units"],
                      "compulsory_bytes": cbytes, **{k: round(v, 4) for k, v in ph.items()}}
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            peak = float(json.load(f)["hbm_gbs"])
        peak_src = "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    achieved = num_bytes / (num_ms * 1e-3) / 1e9 if num_ms > 0 else 0.0
    all_sr = {"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
              "algorithmic_bytes_per_step": num_bytes, "ms_per_step_in_kernel": round(num_ms, 4)}
    if "plus_times_f64" in per_sr:
        # the dominant kernel: the numeric phase of the (+,x) fp64 product
        f = per_sr["plus_times_f64"]
        a64 = f["compulsory_bytes"] / (f["ms_numeric"] * 1e-3) / 1e9 if f["ms_numeric"] > 0 else 0.0
        tpp, tsrc = fp64_traffic_per_product()
        roofline = {"bound": "hbm", "achieved": round(a64, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(a64 / peak, 4),
                    "traffic": round(tpp * f["products"]) if tpp else None,
                    "kernel": "numeric phase of the (+,x) f64 product (k_num_rank<2> + k_num_hash<2,...>), "
                              "per SpGEMM",
                    "algorithmic_bytes": f["compulsory_bytes"], "ms_in_kernel": f["ms_numeric"],
                    "traffic_source": ("ncu DRAM bytes per product of the same kernels (profiles/traffic.json: "
                                       + tsrc + ") x this product's products") if tpp else tsrc,
                    "peak_source": peak_src, "all_semirings": all_sr}
    else:
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None,
                    "kernel": "numeric phase (hash tiers + rank windows of heavy rows, or the one-launch "
                              "kernel), per SpGEMM",
                    "peak_source": peak_src, **all_sr}

    # the end-to-end figure first, on the same resident inputs, before the legs
    # fill device and pinned host memory
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, cb, ctx, dprob, dev, world, dist, products)
        torch.cuda.empty_cache()

    legs = {}
    if not args.no_legs:
        legs = run_legs(args, cb, ctx, dprob, flush, ms_step, products, dev, peak, peak_src)
        legs["one_launch_er16k"] = run_one_launch(args, cb, ctx, flush, dev, peak, peak_src)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        kept = {}
        r, nr, cores, sample, _ = oracle_sample_rate(problems, target_s=args.ref_seconds, keep=kept)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        parity = sampled_parity(dprob, kept)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": ",".join(DTYPE_NAME[sr] for sr, *_ in dprob), "data": "synthetic",
                "config": {"workload": desc, "sizing": "exact (plain two-phase)",
                           "l2": "flushed by a 512 MB device write before every timed step",
                           "products_per_step": products, "nnz_c_per_step": nnz_c,
                           "validation": "off in the timed loop",
                           "parallelism": f"replicas x{world}"},
                "nnz_per_s": nnz_rate, "per_semiring": per_sr, "phase_ms_per_step":
                    {k: round(v, 4) for k, v in phase_tot.items()},
                "roofline": roofline, "cpu_baseline": cpu, "parity_sample": parity, "e2e": e2e,
                **legs,
                "gpu_launches": launches, "clocks": clocks, "wall_s_timed": round(wall, 3)}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def load_sizer(cb):
    """The trained predictor checkpoint, or a quickly trained stand-in when absent."""
    from paper_2106_14402_gb300 import sizer
    if os.path.exists(sizer.CHECKPOINT):
        model, meta = sizer.load()
        return model, {"source": "checkpoint", "train_rows": meta.get("rows"),
                       "train_matrices": meta.get("matrices")}
    feats, labels = zip(*(sizer.product_rows(sizer.gen.training_family(i))
                          for i in list(range(660, 667)) + list(range(667, 700, 4))))
    model, _ = sizer.train(__import__("torch").cat(feats), __import__("torch").cat(labels),
                           epochs=20, batch=4096, lr=3e-3)
    return model, {"source": "trained at start on 16 family matrices"}


def timed(fn, steps, flush):
    import torch
    times = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return sum(times) / len(times)


def run_legs(args, cb, ctx, dprob, flush, plain_ms, products, dev, peak, peak_src):
    """Learned sizing and column batching on the same workload, timed like the main loop."""
    model, src = load_sizer(cb)
    out = {}

    def learned_step():
        st = []
        for sr, A, B, dA, dB, o, nnz in dprob:
            cb.spgemm(sr, dA, dB, validate=False, out=o, sizing="learned", mlp=model, ctx=ctx)
            st.append(ctx.stats())
        return st

    for _ in range(max(1, args.warmup)):
        st = learned_step()
    ms = timed(learned_step, args.steps, flush)
    out["learned"] = {"value": products / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                      "vs_plain_two_phase": plain_ms / ms,
                      "overflow_rows": [x["overflow_rows"] for x in st], "sizer": src,
                      "margin": 0.25}
    # column batching of the 8-byte-value product under a budget of ~1/4 of its output
    sr, A, B, dA, dB, o, nnz = next((p for p in dprob if VAL_BYTES[p[0]] == 8), dprob[0])
    per = 4 + VAL_BYTES[sr]
    budget = 8 * (A.nrows + 1) + (nnz // 4 + 1) * per
    res = {"semiring": sr, "budget_bytes": budget, "output_bytes": 8 * (A.nrows + 1) + nnz * per}
    prods = None
    for mode in ("exact", "learned"):
        info = {}

        def run():
            st = cb.spgemm_column_batches(sr, dA, dB, budget, lambda *a: False, validate=False,
                                          sizing=mode, mlp=model if mode == "learned" else None,
                                          ctx=ctx)
            info.update(st)

        run()
        ms = timed(run, max(1, min(args.steps, 3)), flush)
        prods = info["flops"]
        res[mode] = {"ms": ms, "batches": info["batches"], "products_per_s": prods / (ms * 1e-3)}
    res["learned_vs_exact"] = res["exact"]["ms"] / res["learned"]["ms"]
    out["column_batched"] = res
    out["spmspv"] = run_spmspv_leg(args, cb, ctx, flush, dev, dprob, peak, peak_src)
    out["merge"] = run_merge_leg(args, cb, ctx, flush, dev, peak, peak_src)
    out["high_compression"] = run_high_compression(args, cb, ctx, flush, model, dev, peak, peak_src)
    out["heterogeneous"] = run_hetero_leg(args, cb, ctx, flush, dev, peak, peak_src)
    if not args.no_multi:
        out["multi_spgemm"] = run_multi(args, cb, ctx, model)
    if not args.no_full:
        out["memory_constrained"] = run_full_configs(args, cb, ctx, flush, model, dev, peak, peak_src)
    return out


def run_one_launch(args, cb, ctx, flush, dev, peak, peak_src):
    """ER n=16384, 8 distinct columns per row, C = A.A over (+,x) int64:
    the one-launch kernel for small rows (cb_spgemm_fused) timed alone, next
    to the same product on the two-phase path and through cb_spgemm_ex's
    automatic branch (flop count + host sync + the one launch)."""
    import torch
    from paper_2106_14402_gb300 import gen
    (sr, A, _), = gen.er_square()
    dA = cb.DeviceCSR.from_host(A, sr, dev)
    lanes, flops = cb.fused_lanes(dA, dA, ctx=ctx)
    dt = cb.SEMIRING[sr][1]
    out = cb.DeviceCSR(A.nrows, A.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device=dev),
                       torch.empty(flops, dtype=torch.int32, device=dev),
                       torch.empty(flops, dtype=dt, device=dev))
    status = torch.zeros(1, dtype=torch.int32, device=dev)

    def fused():
        cb.spgemm_fused(sr, dA, dA, out, status, lanes=lanes, ctx=ctx)

    steps = max(args.steps, 20)
    for _ in range(max(args.warmup, 3)):
        fused()
    torch.cuda.synchronize()
    assert int(status.item()) == 0, "one-launch SpGEMM reported an error"
    ms = timed(fused, steps, flush)
    nnz = int(out.row_ptr[-1].item())
    two = lambda: cb.spgemm(sr, dA, dA, validate=False, out=out, fused=False, ctx=ctx)  # noqa: E731
    auto = lambda: cb.spgemm(sr, dA, dA, validate=False, out=out, ctx=ctx)  # noqa: E731
    for f in (two, auto):
        f()
    ms_two = timed(two, steps, flush)
    ms_auto = timed(auto, steps, flush)
    nbytes = compulsory_bytes(sr, A, A, nnz, A.nrows)
    achieved = nbytes / (ms * 1e-3) / 1e9

    # warm: inputs and output L2-resident, 100 launches per CUDA graph replay
    gctx = cb.Context(torch.cuda.Stream(device=dev))
    with torch.cuda.stream(gctx.stream):
        fused_g = lambda: cb.spgemm_fused(sr, dA, dA, out, status, lanes=lanes, ctx=gctx)  # noqa: E731
        fused_g()
        gctx.stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        per_graph = 100
        with torch.cuda.graph(graph, stream=gctx.stream):
            for _ in range(per_graph):
                fused_g()
        graph.replay()
        gctx.stream.synchronize()
        reps = 10
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(gctx.stream)
        for _ in range(reps):
            graph.replay()
        e1.record(gctx.stream)
        e1.synchronize()
        ms_warm = e0.elapsed_time(e1) / (reps * per_graph)
    assert int(status.item()) == 0, "one-launch SpGEMM reported an error in graph replay"
    achieved_warm = nbytes / (ms_warm * 1e-3) / 1e9
    return {"workload": "ER n=16384, 8 distinct cols/row, (+,x) int64 U{1..10}; C=A.A",
            "lanes": lanes, "products": flops, "nnz_c": nnz,
            "us_per_call": round(ms * 1e3, 3), "products_per_s": flops / (ms * 1e-3),
            "nnz_per_s": nnz / (ms * 1e-3),
            "two_phase_us": round(ms_two * 1e3, 3), "auto_branch_us": round(ms_auto * 1e3, 3),
            "one_launch_vs_two_phase": ms_two / ms,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "k_fused (one launch, 8 lanes per row)",
                         "peak_source": peak_src, "algorithmic_bytes": nbytes,
                         "note": "bytes = A + B rows touched + C; B is A here, so A's "
                                 "bytes are counted twice"},
            "warm_graph": {"us_per_call": round(ms_warm * 1e3, 3), "launches": reps * per_graph,
                           "achieved_gbs": round(achieved_warm, 1),
                           "frac": round(achieved_warm / peak, 4),
                           "l2": "inputs and output L2-resident (no flush), 100 launches per "
                                 "CUDA graph replay"},
            "l2": "flushed before every timed call", "steps": steps}


def run_full_configs(args, cb, ctx, flush, model, dev, peak, peak_src):
    """The two memory-constrained workloads, formed in column batches under a
    24 GB output budget with exact and with learned sizing (batch count and
    per-batch sizing), plus the sizing step alone on the held-out product."""
    import torch
    from paper_2106_14402_gb300 import gen, sizer
    budget = 24 * 10**9
    out = {}
    for name, make in (("rmat21_fp64_colbatch", gen.rmat_column_batched),
                       ("rmat20_ef32_sel2nd_held_out", gen.rmat_held_out)):
        (sr, A, B), = make()
        dA = cb.DeviceCSR.from_host(A, sr, dev)
        dB = dA if B is A else cb.DeviceCSR.from_host(B, sr, dev)
        res = {"semiring": sr, "nrows": A.nrows, "nnz_a": A.nnz, "budget_bytes": budget}
        for mode in ("exact", "learned"):
            info = {}

            def run():
                info.update(cb.spgemm_column_batches(
                    sr, dA, dB, budget, lambda *a: False, validate=False, sizing=mode,
                    mlp=model if mode == "learned" else None, ctx=ctx))

            run()
            ms = timed(run, max(1, min(args.steps, 2)), flush)
            b = info["batches"]
            v = VAL_BYTES[sr]
            a_bytes = 8 * (A.nrows + 1) + A.nnz * (4 + v)
            b_bytes = 8 * (B.nrows + 1) + B.nnz * (4 + v)
            c_bytes = 8 * (A.nrows + 1) * b + info["nnz_total"] * (4 + v)
            nbytes = b * a_bytes + b_bytes + c_bytes
            res[mode] = {"ms": ms, "batches": b, "products": info["flops"], "nnz_c": info["nnz_total"],
                         "products_per_s": info["flops"] / (ms * 1e-3),
                         "nnz_per_s": info["nnz_total"] / (ms * 1e-3),
                         "roofline_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                         "algorithmic_bytes": nbytes}
        res["learned_vs_exact"] = res["exact"]["ms"] / res["learned"]["ms"]
        res["peak_gbs"] = peak
        res["peak_source"] = peak_src
        if name.startswith("rmat20"):
            def sizing_learned():
                model.predict(cb.row_features(dA, dB, ctx=ctx), B.ncols, ctx=ctx)

            def sizing_exact():
                cb.row_nnz(dA, dB, ctx=ctx)

            sizing_learned()
            sizing_exact()
            ms_l = timed(sizing_learned, 3, flush)
            ms_e = timed(sizing_exact, 3, flush)
            feat = cb.row_features(dA, dB, ctx=ctx)
            lab = cb.row_nnz(dA, dB, ctx=ctx)
            keep = lab > 0
            res["sizing_step"] = {"features_plus_mlp_ms": ms_l, "exact_symbolic_ms": ms_e,
                                  "speedup": ms_e / ms_l,
                                  "prediction": sizer.evaluate(model, feat[keep], lab[keep], B.ncols)}
        out[name] = res
        del dA, dB
        torch.cuda.empty_cache()
    return out


def run_high_compression(args, cb, ctx, flush, model, dev, peak, peak_src):
    """A high-compression product (block-clustered matrix, compression ratio
    ~36, shaped like the paper's protein-similarity networks): plain exact
    path with the default tier bounds and with autotuned ones, and learned
    per-row sizing."""
    import torch
    from paper_2106_14402_gb300 import gen
    (sr, A, _), = gen.high_compression()
    dA = cb.DeviceCSR.from_host(A, sr, dev)
    C = cb.spgemm(sr, dA, dA, validate=False, ctx=ctx)
    nnz = C.nnz
    del C
    out = cb.DeviceCSR(A.nrows, A.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device=dev),
                       torch.empty(nnz, dtype=torch.int32, device=dev),
                       torch.empty(nnz, dtype=cb.SEMIRING[sr][1], device=dev))
    steps = max(1, min(args.steps, 3))
    res = {"workload": "block-clustered n=131072, clusters of 256, density 0.5, ~1 inter-cluster edge "
                       "per vertex, symmetrised+permuted; C=A.A over (+,x) f64",
           "nnz_a": A.nnz, "nnz_c": nnz}
    saved = ctx.get_tune()
    info = {}

    def plain():
        cb.spgemm(sr, dA, dA, validate=False, out=out, ctx=ctx, timing=True)
        info.update(ctx.stats())

    def learned():
        cb.spgemm(sr, dA, dA, validate=False, out=out, ctx=ctx, sizing="learned", mlp=model)

    plain()
    ms = timed(plain, steps, flush)
    prods = info["flops"]
    res["products"] = prods
    res["compression_ratio"] = prods / max(nnz, 1)
    nbytes = compulsory_bytes(sr, A, A, nnz, A.nrows)
    res["default"] = {"ms": ms, "products_per_s": prods / (ms * 1e-3), "nnz_per_s": nnz / (ms * 1e-3),
                      "ms_symbolic": info["ms_symbolic"], "ms_numeric": info["ms_numeric"],
                      "roofline_frac_numeric": round(nbytes / (info["ms_numeric"] * 1e-3) / 1e9 / peak, 4)}
    best, _ = cb.autotune(sr, dA, dA, ctx=ctx)
    plain()
    ms_t = timed(plain, steps, flush)
    res["autotuned"] = {"bounds": best, "ms": ms_t, "products_per_s": prods / (ms_t * 1e-3),
                        "vs_default": ms / ms_t}
    learned()
    ms_l = timed(learned, steps, flush)
    res["learned"] = {"ms": ms_l, "vs_autotuned_plain": ms_t / ms_l}
    ctx.set_tune(**saved)
    res["peak_gbs"] = peak
    res["peak_source"] = peak_src
    return res


def run_hetero_leg(args, cb, ctx, flush, dev, peak, peak_src):
    """The heterogeneous semiring (three value types) on the R-MAT s18 ef16
    matrix: A float32 weights, B int32 labels, C (weight, label) records,
    plain two-phase path into a pre-reserved C."""
    import torch
    from paper_2106_14402_gb300 import gen
    (sr, A, B), = gen.rmat_square(18, 16, semirings=("maxw_label",))
    dA = cb.DeviceCSR.from_host(A, sr, dev, operand="A")
    dB = cb.DeviceCSR.from_host(B, sr, dev, operand="B")
    C = cb.spgemm(sr, dA, dB, validate=True, ctx=ctx)
    nnz = C.nnz
    del C
    out = cb.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int64, device=dev),
                       torch.empty(nnz, dtype=torch.int32, device=dev),
                       torch.empty(nnz, dtype=cb.SEMIRING[sr][1], device=dev))
    info = {}

    def plain():
        cb.spgemm(sr, dA, dB, validate=False, out=out, ctx=ctx, timing=True)
        info.update(ctx.stats())

    plain()
    ms = timed(plain, max(1, min(args.steps, 3)), flush)
    prods = info["flops"]
    nbytes = compulsory_bytes(sr, A, B, nnz, A.nrows)
    res = {"workload": "R-MAT s18 ef16 (same matrix as the headline), C = A.B with A float32 weights "
                       "U[0,1), B int32 labels U[0,2^30), C (weight, label) records; (+) = heaviest "
                       "weight (IEEE totalOrder), smaller label on ties",
           "ms": ms, "products": prods, "nnz_c": nnz, "products_per_s": prods / (ms * 1e-3),
           "nnz_per_s": nnz / (ms * 1e-3), "ms_symbolic": info["ms_symbolic"],
           "ms_numeric": info["ms_numeric"], "algorithmic_bytes": nbytes,
           "roofline_frac_numeric": round(nbytes / (info["ms_numeric"] * 1e-3) / 1e9 / peak, 4),
           "peak_gbs": peak, "peak_source": peak_src}
    del out, dA, dB
    torch.cuda.empty_cache()
    return res


def _inner_blocks(A, k):
    """The k (column block of A, row block of A) pairs of a split of the inner dimension."""
    cuts = np.linspace(0, A.ncols, k + 1).astype(np.int64)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.row_ptr))
    out = []
    from paper_2106_14402_gb300 import gen
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        keep = (A.col >= lo) & (A.col < hi)
        rp = np.zeros(A.nrows + 1, np.int64)
        np.add.at(rp, rows[keep] + 1, 1)
        L = gen.CSR(A.nrows, A.ncols, np.cumsum(rp), A.col[keep], A.val[keep])
        lens = np.diff(A.row_ptr).copy()
        lens[:lo] = 0
        lens[hi:] = 0
        rp2 = np.zeros(A.nrows + 1, np.int64)
        rp2[1:] = np.cumsum(lens)
        s0, e0 = A.row_ptr[lo], A.row_ptr[hi]
        R = gen.CSR(A.nrows, A.ncols, rp2, A.col[s0:e0], A.val[s0:e0])
        out.append((L, R))
    return out


def run_merge_leg(args, cb, ctx, flush, dev, peak, peak_src):
    """The merge of k partial results (Sec. 3.2): R-MAT s16 ef16 (+,x) f64,
    the inner dimension split into k = 8 blocks as in a SUMMA stage; the 8
    partial products are formed first (untimed), then merged (timed)."""
    import torch
    from paper_2106_14402_gb300 import gen
    (sr, A, _), = gen.rmat_square(16, 16, cfg=2, semirings=("plus_times_f64",))
    k = 8
    parts = []
    for L, R in _inner_blocks(A, k):
        parts.append(cb.spgemm(sr, cb.DeviceCSR.from_host(L, sr, dev), cb.DeviceCSR.from_host(R, sr, dev),
                               validate=False, ctx=ctx))
    torch.cuda.synchronize()
    nnz_parts = sum(p.nnz for p in parts)
    info = {}

    def run():
        C = cb.merge(sr, parts, validate=False, ctx=ctx)
        info["nnz"] = C.nnz
        info["kernels"] = ctx.stats()["kernels"]

    run()
    ms = timed(run, max(1, min(args.steps, 3)), flush)
    v = VAL_BYTES[sr]
    nbytes = k * 8 * (A.nrows + 1) + nnz_parts * (4 + v) + 8 * (A.nrows + 1) + info["nnz"] * (4 + v)
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "R-MAT s16 ef16 (+,x) f64, inner dimension in 8 blocks; merge of the 8 partial "
                        "products", "k": k, "nnz_parts": nnz_parts, "nnz_c": info["nnz"], "ms": ms,
            "entries_in_per_s": nnz_parts / (ms * 1e-3), "kernels": info["kernels"],
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "algorithmic_bytes": nbytes,
                         "peak_source": peak_src}}


def run_spmspv_leg(args, cb, ctx, flush, dev, dprob, peak, peak_src):
    """SpMSpV y^T = x^T A (Sec. 4.3) on the workload's R-MAT matrix: random
    frontiers of 1K, 16K and 128K vertices, (or,and) and (min,+), with the
    dense accumulator and in the bucket form; next to the same product as a
    one-row SpGEMM."""
    import torch
    from paper_2106_14402_gb300 import gen
    out = {"workload": "R-MAT s18 ef16 (the step's matrix); x = seeded random distinct vertices",
           "legs": []}
    for sr, A, B, dA, dB, o, nnz in dprob:
        if sr not in ("or_and_bool", "min_plus_u32"):
            continue
        rng = np.random.default_rng(7)
        v = VAL_BYTES[sr]
        for f in (1 << 10, 1 << 14, 1 << 17):
            idx = np.sort(rng.choice(A.nrows, f, replace=False)).astype(np.int32)
            val = gen.random_values(sr, f, 8)
            xi = torch.from_numpy(idx).to(dev)
            xv = torch.from_numpy(val.view(np.int32) if val.dtype == np.uint32 else val).to(dev)
            if cb.SEMIRING[sr][1] == torch.uint32:
                xv = xv.view(torch.uint32)
            res = {}

            def run():
                yi, _ = cb.spmspv(sr, dA, xi, xv, validate=False, ctx=ctx)
                res["nnz"] = yi.numel()

            run()
            ms = timed(run, max(3, args.steps), flush)
            X = cb.DeviceCSR(1, A.nrows, torch.tensor([0, f], dtype=torch.int64, device=dev), xi, xv)

            def as_spgemm():
                cb.spgemm(sr, X, dA, validate=False, ctx=ctx)

            as_spgemm()
            ms_g = timed(as_spgemm, max(3, args.steps), flush)

            def bucket():
                cb.spmspv(sr, dA, xi, xv, validate=False, ctx=ctx, bucket=True)

            bucket()
            ms_b = timed(bucket, max(3, args.steps), flush)
            lens = np.diff(A.row_ptr)[idx]
            prods = int(lens.sum())
            nbytes = f * (4 + v) + 16 * f + prods * (4 + v) + res["nnz"] * (4 + v)
            out["legs"].append({"semiring": sr, "nnz_x": f, "products": prods, "nnz_y": res["nnz"],
                                "us": round(ms * 1e3, 2), "products_per_s": prods / (ms * 1e-3),
                                "roofline_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                                "one_row_spgemm_us": round(ms_g * 1e3, 2),
                                "vs_one_row_spgemm": ms_g / ms,
                                "bucket_form_us": round(ms_b * 1e3, 2)})
    out["peak_gbs"] = peak
    out["peak_source"] = peak_src
    return out


def run_multi(args, cb, ctx, model):
    """4096 independent ER products (n log-uniform in [256, 65536], degree 4..64;
    half (min,+) u32, half (+,x) fp64), generated on the device: batched calls
    with waves under a 24 GB output budget in every mode, against one call per
    product, and against the two-phase path (no work-queue kernel) under each
    semiring's own autotuned bounds.  Outputs are consumed (dropped) as they are
    produced.  Each figure is the median of `reps` timed calls after one
    untimed call (host wall clock around a synchronised call, inputs
    resident)."""
    import time

    import torch

    from paper_2106_14402_gb300 import gen_device
    count = args.multi_count
    plan, As, Bs = gen_device.batched_workload(count)
    srs = [p["semiring"] for p in plan]
    torch.cuda.synchronize()
    budget = 24 << 30
    reps = 5
    res = {"products": count, "budget_bytes": budget, "reps": reps,
           "workload": "ER n log-U[256,65536], deg U{4..64}; half (min,+) u32 [1,1000], half (+,x) f64 U(-1,1)",
           "timing": "median of %d host wall-clock timed calls (synchronised), after one untimed call; "
                     "inputs resident" % reps}

    def median_time(fn):
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    def batched(mode, sizing="exact", fused=True, lo=0, hi=None):
        hi = count if hi is None else hi
        info = {}

        def run():
            info.update(cb.spgemm_batched(srs[lo:hi], As[lo:hi], Bs[lo:hi],
                                          (lambda *a: None) if mode == "graph" else (lambda *a: False),
                                          budget_bytes=budget, validate=False, sizing=sizing,
                                          mlp=model if sizing == "learned" else None, ctx=ctx,
                                          mode=mode, fused=fused))
            torch.cuda.synchronize()
        sec = median_time(run)
        return sec, info

    for key, mode, sizing in (("batched_graph", "graph", "exact"), ("batched_sync_free", "sync_free", "exact"),
                              ("batched_exact", "host", "exact"), ("batched_learned", "host", "learned")):
        sec, info = batched(mode, sizing)
        res[key] = {"seconds": sec, "waves": info["batches"], "products_per_s": info["flops"] / sec,
                    "nnz_per_s": info["nnz"] / sec}
    flops = info["flops"]
    res["batched_graph"]["note"] = ("one CUDA graph per semiring group; capture, instantiation and launch "
                                    "inside the timed call (batched_sync_free: the same launch sequence "
                                    "without the capture)")

    def plain():
        for sr, A, B in zip(srs, As, Bs):
            C = cb.spgemm(sr, A, B, validate=False, ctx=ctx)
            del C
        torch.cuda.synchronize()

    sec = median_time(plain)
    res["plain_per_product"] = {"seconds": sec, "products_per_s": flops / sec}
    # the two-phase path (hash tiers and rank windows, no work-queue kernel) in
    # graph mode, each semiring group under its own autotuned bounds
    half = count // 2
    two = 0.0
    tuned = {}
    for lo, hi in ((0, half), (half, count)):
        sr = srs[lo]
        i = max(range(lo, hi), key=lambda k: plan[k]["n"] * plan[k]["deg"] ** 2)
        tuned[sr], _ = cb.autotune(sr, As[i], Bs[i], ctx=ctx)
        ctx.set_tune(**tuned[sr])
        sec_g, _ = batched("graph", fused=False, lo=lo, hi=hi)
        two += sec_g
    ctx.set_tune()
    res["two_phase_graph"] = {"seconds": two, "products_per_s": flops / two, "tune": tuned}
    for key in ("batched_graph", "batched_sync_free", "batched_exact", "batched_learned"):
        res[key]["vs_plain_per_product"] = res["plain_per_product"]["seconds"] / res[key]["seconds"]
        res[key]["vs_two_phase_graph"] = two / res[key]["seconds"]
    del As, Bs
    torch.cuda.empty_cache()
    return res


def run_e2e(args, cb, ctx, dprob, dev, world, dist, products):
    """Same metric through the public call with host buffers: per step the
    inputs are copied from pinned host memory, C is computed, and all of C is
    read back into pinned host memory (a reused 2 GiB staging area), inside
    the timed region.  The read-back of one product runs on a copy stream
    while the next product computes (two output buffers alternate; the next
    step's first product included), so a step costs about the larger of the
    compute and the device-to-host traffic rather than their sum."""
    import torch
    hosts = []
    for sr, A, B, dA, dB, out, nnz in dprob:
        hA = [t.cpu().pin_memory() for t in (dA.row_ptr, dA.col, dA.val)]
        hB = None if dB is dA else [t.cpu().pin_memory() for t in (dB.row_ptr, dB.col, dB.val)]
        hosts.append((hA, hB))
    max_nnz = max(p[6] for p in dprob)
    max_rows = max(p[1].nrows for p in dprob)
    vmax = max(VAL_BYTES[p[0]] for p in dprob)
    # C is read back through a pinned staging area of 2 x 1 GiB, reused chunk by
    # chunk (every byte of C crosses to the host; the host keeps 2 GiB per rank)
    chunk = 1 << 30
    stage = [torch.empty(chunk, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    nstage = [0]

    def to_host(src_bytes):
        n = src_bytes.numel()
        for o in range(0, n, chunk):
            k = min(chunk, n - o)
            stage[nstage[0] & 1][:k].copy_(src_bytes[o:o + k], non_blocking=True)
            nstage[0] += 1
    # two device output buffers (raw bytes for the values, viewed per semiring)
    bufs = [(torch.empty(max_rows + 1, dtype=torch.int64, device=dev),
             torch.empty(max(max_nnz, 1), dtype=torch.int32, device=dev),
             torch.empty(max(max_nnz, 1) * vmax, dtype=torch.uint8, device=dev)) for _ in range(2)]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    for e in copied:
        e.record(ctx.stream)
    cstream = torch.cuda.Stream(device=dev)
    moved = {"h2d": 0, "d2h": 0}
    turn = [0]

    def one(count):
        for (sr, A, B, dA, dB, out, nnz), (hA, hB) in zip(dprob, hosts):
            pairs = list(zip((dA.row_ptr, dA.col, dA.val), hA))
            if hB is not None:
                pairs += list(zip((dB.row_ptr, dB.col, dB.val), hB))
            with torch.cuda.stream(ctx.stream):
                for dst, src in pairs:
                    dst.copy_(src, non_blocking=True)
                    if count:
                        moved["h2d"] += src.numel() * src.element_size()
            b = turn[0]
            turn[0] ^= 1
            rp, col, raw = bufs[b]
            ctx.stream.wait_event(copied[b])       # its previous read-back is done
            dt = cb.SEMIRING[sr][1]
            vals = raw.view(torch.int32).view(torch.uint32) if dt == torch.uint32 else raw.view(dt)
            o = cb.DeviceCSR(A.nrows, B.ncols, rp, col, vals)
            C = cb.spgemm(sr, dA, dB, validate=False, out=o, ctx=ctx)
            n = C.nnz
            ready = torch.cuda.Event()
            ready.record(ctx.stream)
            cstream.wait_event(ready)
            nb = n * VAL_BYTES[sr]
            with torch.cuda.stream(cstream):
                to_host(rp[: C.nrows + 1].view(torch.uint8))
                to_host(col[:n].view(torch.uint8))
                to_host(raw[:nb])
            copied[b].record(cstream)
            if count:
                moved["d2h"] += (C.nrows + 1) * 8 + n * 4 + nb

    one(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        one(True)      # a step's last read-backs overlap the next step's first product
    torch.cuda.synchronize()
    el = max_over_ranks((time.perf_counter() - t0) / steps, dist, dev)
    return {"value": whole_job_rate(products, world, el), "unit": UNIT,
            "h2d_bytes_per_step": moved["h2d"] // steps, "d2h_bytes_per_step": moved["d2h"] // steps,
            "ms_per_step": el * 1e3, "steps": steps,
            "timing": "host wall clock around all steps, synchronised at the end; the read-back "
                      "of a product overlaps the next product's compute, across steps too (copy "
                      "stream, two output buffers)"}

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="rmat18", choices=("rmat18", "rmat16", "er16k", "blockclust"))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-legs", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-full", action="store_true", help="skip the memory-constrained R-MAT workloads")
    ap.add_argument("--multi-count", type=int, default=4096)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--multi-only", action="store_true",
                    help="time only the batched leg (--multi-count products) and print its record")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.multi_only:
        import torch

        from paper_2106_14402_gb300 import cb
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        cb.load()
        model, _ = load_sizer(cb)
        print(json.dumps({"multi_spgemm": run_multi(args, cb, cb.context(), model)}), flush=True)
        return 0
    return main_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
