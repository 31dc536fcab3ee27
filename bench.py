"""SpMM benchmark: GFLOP/s (2 nnz n / t) and HBM-roofline fraction on one GB300.

Default workload: the 1M x 1M power-law CSR matrix (row lengths with density
exponent 2, mean about 16, capped at 100,000, 1% empty rows) times row-major
float32 B of widths n = 8, 32, 64, 128.  One step = C = A B for every width,
each through the C ABI with the algorithm chosen by the GB300 selector (the
Section 5.4 mean-row-length rule recalibrated, plus a longest-row guard); the
JSON line also reports the Section 5.4 rule's own pick and each family's
times (``--alg`` overrides).  After the headline, the growth forms are
measured: 16-bit storage (2M x 2M, n = 128), a GCN layer's forward and
backward (500k nodes, n = 256, with the transpose on its own) and a
2048-matrix batch in graph-captured persistent launches.  All inputs are
synthetic and seeded (gen/).

Timing: inputs resident in HBM; L2 is flushed (a write of twice its size)
before every step, outside the events; each call is bracketed by CUDA events on
the launching stream.  ``e2e`` times the same step through
``spmm_csr_host_multi`` (host buffers; H2D of A once and of every B, D2H of
every C and the final stream synchronisation inside the timed region; one
``spmm_csr_host_async`` or synchronous ``spmm_csr_host`` call per width
beside it) next to the host link's own copy rates.  ``--impl reference`` times the FP64 CPU oracle on
a bounded row sample.  ``--sweep aspect|density|spmv|tiling|selector`` runs one
of the parameter sweeps instead (a JSON line per point), and ``--ingest-ncu``
turns the recorded ncu traffic capture into the JSON the roofline reads.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
ALG_NAME = {1: "row_split", 2: "merge", 5: "hybrid"}  # spmm_alg_t codes of the families
FALLBACK_HBM_GBS = 6800.0


# ----------------------------------------------------------------------------- args / env

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="power_law", choices=["power_law", "plain"])
    p.add_argument("--n", type=int, nargs="*", default=None, help="dense widths (default 8 32 64 128)")
    p.add_argument("--alg", default="auto_gb300", choices=["auto_gb300", "auto", "row_split", "merge", "hybrid"])
    p.add_argument("--no-extras", action="store_true", help="skip e2e, cpu_baseline and per-algorithm breakdown "
                   "(the growth forms are controlled by --forms)")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--tuning", default=None, help='JSON spmm_tuning_t fields, e.g. {"column_slabs": 2}')
    p.add_argument("--forms", default="precision,backward,batched",
                   help="comma list of growth forms measured after the headline (empty: none)")
    p.add_argument("--batched-count", type=int, default=2048, help="matrices in the batched form")
    p.add_argument("--ingest-ncu", default=None, metavar="CSV",
                   help="instead of the benchmark: turn the ncu CSV of the traffic capture (the command recorded in "
                        "profiles/merge_kernel_power_law_1M_dram.json, with --print-units base) into that JSON")
    p.add_argument("--sweep", default=None, choices=["aspect", "density", "spmv", "tiling", "selector", "gather"],
                   help="instead of the benchmark: the aspect-ratio sweep (dense-as-CSR m x k with m*k = 2^24, "
                        "n = 64), the density sweep against dense GEMM (100k x 100k, n = 64) or SpMV (n = 1) on "
                        "five matrices against cuSPARSE through torch, the A/B tiling against both families "
                        "with B larger than L2, both selectors over row-length families (selector), or the "
                        "gather-only probe over B sizes 16 MB - 1 GB and row widths 32-512 B (gather); "
                        "JSON line per point")
    return p.parse_args()


def max_over_ranks(value: float) -> float:
    """The largest value over all ranks of the process group (the value itself
    when no group of size > 1 is initialised).  Replicas are timed separately and
    the job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput of `world` replicas that each did flops_per_rank in ms."""
    return world * flops_per_rank / (ms * 1e-3) / 1e9


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------------------- workload

def make_workload(name, ns):
    if name == "plain":
        a, B64 = gen.workload_plain()
        ns = ns or [64]
        Bs = {n: (B64 if n == 64 else gen.normal_matrix(a.k, n, gen.SEED_BASE + 1)) for n in ns}
        label = "plain_4096x4096_16nnz"
    else:
        a = gen.workload_power_law()
        ns = ns or [8, 32, 64, 128]
        Bs = {n: gen.normal_matrix(a.k, n, gen.SEED_BASE + 2, stream=2 + n) for n in ns}
        label = "power_law_1Mx1M_mean16_cap1e5"
    return label, a, ns, Bs


def compulsory_bytes(m, nnz, k, n, s_v=4, s_b=4, s_c=4):
    """row_ptr + col_ind + vals + B (each row once) + C: the bytes any SpMM must move."""
    return (m + 1) * 4 + nnz * (4 + s_v) + k * n * s_b + m * n * s_c


# Sampled GPU results kept on the host by the headline and the forms, checked against the FP64
# oracle by the cpu_baseline leg at the end of the run (the one place besides --impl reference where
# bench.py runs the oracle).  Each entry: (rows, row_ptr, col_ind, vals, B, C_rows, what it is).
SAMPLES = {}


def sample_rows(m, count, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(m, size=min(m, count), replace=False))


def row_nonzeros(rows, row_ptr):
    """Positions of the nonzeros of `rows` (in row order)."""
    rows = np.asarray(rows, dtype=np.int64)
    parts = [np.arange(row_ptr[r], row_ptr[r + 1], dtype=np.int64) for r in rows]
    return np.concatenate(parts) if parts else np.zeros(0, np.int64)


def subproblem(rows, row_ptr, col_ind, vals, B):
    """The rows `rows` of A as a CSR of their own, with the columns they touch renumbered
    0..u-1 and B reduced to those u rows: the product of the pieces is C[rows]."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = (row_ptr[rows + 1] - row_ptr[rows]).astype(np.int64)
    rp = np.zeros(len(rows) + 1, dtype=np.int32)
    np.cumsum(lens, out=rp[1:])
    idx = row_nonzeros(rows, row_ptr)
    cols = col_ind[idx]
    uniq, ci = np.unique(cols, return_inverse=True)
    return rp, ci.astype(np.int32), np.ascontiguousarray(vals[idx]), np.ascontiguousarray(B[uniq])


GATHER_JSON = os.path.join(ROOT, "profiles", "gather_ceiling_sweep.jsonl")
TRAFFIC_SOURCES = ["paper_1803_08601_gb300/csrc/kernels.cuh", "paper_1803_08601_gb300/csrc/common.cuh"]
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "merge_kernel_power_law_1M_dram.json")
TRAFFIC_COMMAND = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,lts__t_sector_hit_rate.pct,"
                   "gpu__time_duration.sum --print-units base --clock-control none -k regex:merge_kernel -s 12 -c 4 "
                   "--csv --log-file <CSV> python bench.py --alg merge --steps 1 --warmup 3 --no-extras --forms= "
                   "--no-clocks")


def sources_sha256(paths):
    import hashlib

    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def load_capture(kernel, label):
    """The committed ncu capture of the dominant kernel on this workload, or (None, why)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_power_law_1M_dram.json")
    if label != "power_law_1Mx1M_mean16_cap1e5" or not os.path.exists(path):
        return None, "no capture for this kernel and workload"
    with open(path) as f:
        cap = json.load(f)
    if sources_sha256(cap["sources"]) != cap["sources_sha256"]:
        return None, "kernel sources changed since the ncu capture"
    return cap, os.path.basename(path)


def measured_traffic(kernel, label, ns):
    """DRAM bytes (read + write) of the dominant kernel summed over the step's widths, from the
    committed ncu capture in profiles/, or None when the kernel sources changed since."""
    cap, note = load_capture(kernel, label)
    if cap is None:
        return None, note
    if not all(str(n) in cap["per_n"] for n in ns):
        return None, "capture lacks some widths"
    t = sum(cap["per_n"][str(n)]["dram_read_bytes"] + cap["per_n"][str(n)]["dram_write_bytes"] for n in ns)
    return t, ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch per width, summed over the "
               f"step's widths {ns} (profiles/{note}); same units as achieved x duration")


def gather_aware(kernel, label, m, nnz, k, ns, mean_call, peak, l2_bytes, s_b=4):
    """The gather-aware bound: A + C + nnz n s_B (1 - h), h the L2 hit rate of the B gathers.
    h is the capture's lts__t_sector_hit_rate (all L2 sectors of the launch, dominated by the
    gathers) while the capture is current, else the uniform-column model min(1, L2 / |B|)."""
    cap, note = load_capture(kernel, label)
    per_n, total_bytes, total_ms = {}, 0.0, 0.0
    for n in ns:
        if cap is not None and str(n) in cap["per_n"]:
            h, src = cap["per_n"][str(n)]["l2_sector_hit_pct"] / 100.0, f"ncu lts__t_sector_hit_rate ({note})"
        else:
            h, src = min(1.0, l2_bytes / float(k * n * s_b)), "model min(1, L2 / |B|)"
        b = (m + 1) * 4 + nnz * 8 + m * n * 4 + nnz * n * s_b * (1.0 - h)
        t_min = b / (peak * 1e9) * 1e3
        per_n[str(n)] = {"h": h, "h_source": src, "bytes": b, "t_min_ms": t_min, "frac": t_min / mean_call[n]}
        total_bytes += b
        total_ms += mean_call[n]
    return {"formula": "(m+1)*4 + nnz*8 + m*n*4 + nnz*n*4*(1-h) per call", "bytes": total_bytes,
            "frac": total_bytes / (peak * 1e9) * 1e3 / total_ms, "per_n": per_n}


def gather_ceiling(b_bytes, row_bytes):
    """Measured gather ceiling (TB/s of gathered bytes) for uniformly random rows of row_bytes
    bytes from a B of b_bytes bytes: the committed --sweep gather data, interpolated in log B
    between the measured sizes (clamped at both ends).  None without the data or the width."""
    if not os.path.exists(GATHER_JSON):
        return None
    pts = sorted((r["b_mb"] * (1 << 20), r["gathered_tb_s"]) for r in map(json.loads, open(GATHER_JSON))
                 if r["row_bytes"] == row_bytes)
    if not pts:
        return None
    if b_bytes <= pts[0][0]:
        return pts[0][1]
    for (b0, t0), (b1, t1) in zip(pts, pts[1:]):
        if b_bytes <= b1:
            w = (np.log(b_bytes) - np.log(b0)) / (np.log(b1) - np.log(b0))
            return float(t0 + w * (t1 - t0))
    return pts[-1][1]


def gather_bound(m, nnz, k, ns, mean_call, slabs_of, s_b=4):
    """Second roofline: the time the nonzeros' B-row gathers take at the measured gather ceiling
    (bench.py --sweep gather) for the row width and B (slab) size each call gathers from."""
    per_n, t_sum, ms_sum = {}, 0.0, 0.0
    for n in ns:
        slabs = slabs_of(n)
        row_bytes = n * s_b // slabs
        ceil = gather_ceiling(k * row_bytes, row_bytes)
        if ceil is None:
            return None
        t = nnz * n * s_b / (ceil * 1e12) * 1e3
        per_n[str(n)] = {"row_bytes": row_bytes, "b_slab_bytes": k * row_bytes, "ceiling_tb_s": ceil,
                         "t_gather_ms": t, "frac": t / mean_call[n]}
        t_sum += t
        ms_sum += mean_call[n]
    return {"source": "profiles/gather_ceiling_sweep.jsonl (bench.py --sweep gather)",
            "formula": "nnz*n*4 / ceiling(row bytes, B slab bytes) per call", "frac": t_sum / ms_sum,
            "per_n": per_n}


def ingest_ncu(csv_path, out_path=TRAFFIC_JSON):
    """Write the traffic JSON from the ncu CSV of TRAFFIC_COMMAND: the four merge_kernel launches
    of the timed step, in the step's width order 8, 32, 64, 128."""
    import csv

    launches = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(line for line in f if line.startswith('"'))]
    head = rows[0]
    col = {name: head.index(name) for name in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    for r in rows[1:]:
        d = launches.setdefault(int(r[col["ID"]]), {"kernel": r[col["Kernel Name"]]})
        d[r[col["Metric Name"]]] = (float(r[col["Metric Value"]].replace(",", "")), r[col["Metric Unit"]])
    ids = sorted(launches)
    if len(ids) != 4:
        raise SystemExit(f"expected 4 captured launches, found {len(ids)}")
    per_n = {}
    for n, i in zip((8, 32, 64, 128), ids):
        d = launches[i]
        assert d["dram__bytes_read.sum"][1] == "byte" and d["gpu__time_duration.sum"][1] == "ns", d
        per_n[str(n)] = {"dram_read_bytes": int(d["dram__bytes_read.sum"][0]),
                         "dram_write_bytes": int(d["dram__bytes_write.sum"][0]),
                         "duration_ns": int(d["gpu__time_duration.sum"][0]),
                         "l2_sector_hit_pct": round(d["lts__t_sector_hit_rate.pct"][0], 2),
                         "kernel": d["kernel"]}
    out = {"kernel": "merge_kernel (float32, 16-byte vectors; W = n/4 lanes per row, or n/8 with two slabs)",
           "workload": "power_law_1Mx1M_mean16_cap1e5", "command": TRAFFIC_COMMAND,
           "sources": TRAFFIC_SOURCES, "sources_sha256": sources_sha256(TRAFFIC_SOURCES), "per_n": per_n}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))
    return 0


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, enabled=True):
        self.enabled = enabled
        self.proc = None
        self.lines = []

    def __enter__(self):
        if self.enabled:
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                              "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.reader = threading.Thread(target=self._read, daemon=True)
                self.reader.start()
            except (FileNotFoundError, OSError):
                self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, gpu_index=None):
        rows = []
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                idx, sm, smax = int(parts[0]), float(parts[1]), float(parts[2])
            except ValueError:
                continue
            if gpu_index is not None and idx != gpu_index:
                continue
            rows.append((sm, smax, parts[5:9]))
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, x in enumerate(r) if x.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------- oracle timing

def time_oracle_sample(a, ns, Bs, target_s=12.0, seed=0):
    """FP64 oracle on a bounded, seeded sample of rows of the same workload.
    Returns (GFLOP/s, seconds, rows sampled, threads)."""
    import oracle

    rng = np.random.default_rng(seed)
    lens = a.row_lengths()
    rows = np.sort(rng.choice(a.m, size=min(a.m, 20_000), replace=False))
    t0 = time.perf_counter()
    for n in ns:
        oracle.spmm_rows(rows, a.row_ptr, a.col_ind, a.vals, Bs[n])
    t_probe = time.perf_counter() - t0
    scale = max(1.0, target_s / max(t_probe, 1e-3))
    rows = np.sort(rng.choice(a.m, size=int(min(a.m, len(rows) * scale)), replace=False))
    flops, passes = 0.0, 0
    t0 = time.perf_counter()
    while True:  # whole passes over the sample until about target_s of CPU work
        for n in ns:
            oracle.spmm_rows(rows, a.row_ptr, a.col_ind, a.vals, Bs[n])
        flops += sum(2.0 * float(lens[rows].sum()) * n for n in ns)
        passes += 1
        if time.perf_counter() - t0 >= target_s:
            break
    t = time.perf_counter() - t0
    return flops / t / 1e9, t, len(rows), oracle.num_threads(), passes


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    label, a, ns, Bs = make_workload(args.workload, args.n)
    import oracle

    vals = []
    rng = np.random.default_rng(1)
    lens = a.row_lengths()
    per_step_rows = None
    for step in range(args.warmup + args.steps):
        if per_step_rows is None:
            rows = np.sort(rng.choice(a.m, size=min(a.m, 20_000), replace=False))
        else:
            rows = np.sort(rng.choice(a.m, size=per_step_rows, replace=False))
        t0 = time.perf_counter()
        for n in ns:
            oracle.spmm_rows(rows, a.row_ptr, a.col_ind, a.vals, Bs[n])
        t = time.perf_counter() - t0
        if per_step_rows is None:  # size later steps to about 8 s each
            per_step_rows = int(min(a.m, len(rows) * max(1.0, 8.0 / max(t, 1e-3))))
        if step >= args.warmup:
            vals.append(sum(2.0 * float(lens[rows].sum()) * n for n in ns) / t / 1e9)
    v = float(statistics.mean(vals))
    line = {"impl": "reference", "metric": "SpMM GFLOP/s (2*nnz*n/t)", "value": v, "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (gen/, seeded)",
            "config": {"workload": label, "m": a.m, "k": a.k, "nnz": a.nnz, "n": ns},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step_rows} random rows of the {label} matrix per step, all n"},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ingest_ncu:
        return ingest_ncu(args.ingest_ncu)
    if args.sweep:
        return run_sweep(args)
    import torch

    import paper_1803_08601_gb300 as pkg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    pkg.build()
    pkg.load()
    label, a, ns, Bs = make_workload(args.workload, args.n)
    m, k, nnz = a.m, a.k, a.nnz
    stream = torch.cuda.current_stream()
    d_rp = torch.from_numpy(a.row_ptr).to(dev)
    d_ci = torch.from_numpy(a.col_ind).to(dev)
    d_v = torch.from_numpy(a.vals).to(dev)
    d_B = {n: torch.from_numpy(Bs[n]).to(dev) for n in ns}
    d_C = {n: torch.empty((m, n), dtype=torch.float32, device=dev) for n in ns}
    max_row = pkg.max_row_length(d_rp)  # measured once; passed to the GB300 selector as a hint
    paper_pick = {n: pkg.spmm_select_alg(m, nnz, 0.0) for n in ns}
    gb300_pick = {n: pkg.spmm_select_alg_gb300(m, nnz, max_row, n, pkg.F32) for n in ns}
    alg_of = {n: {"auto": paper_pick[n], "auto_gb300": gb300_pick[n]}.get(args.alg, pkg.alg_code(args.alg)) for n in ns}
    tuning_ws = json.loads(args.tuning) if args.tuning else None
    ws_bytes = max(pkg.workspace_size(m, k, n, nnz, al, tuning=tuning_ws)
                   for n in ns for al in (pkg.ALG_MERGE, pkg.ALG_ROW_SPLIT_HYBRID))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(2 * l2 // 4 + 1024, dtype=torch.float32, device=dev)

    tuning = dict(json.loads(args.tuning)) if args.tuning else {}
    tuning.setdefault("max_row_len", max_row)

    def one(n, alg):
        pkg.spmm(d_rp, d_ci, d_v, d_B[n], alg=alg, out=d_C[n], nnz=nnz, workspace=ws, tuning=tuning)

    def step(events=None):
        for i, n in enumerate(ns):
            if events is not None:
                events[i][0].record(stream)
            one(n, args.alg)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    per_call = {n: [] for n in ns}
    launches0 = pkg.spmm_launch_count()
    with ClockSampler(enabled=not args.no_clocks) as clk:
        barrier()
        for _ in range(args.steps):
            flush.zero_()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in ns]
            step(ev)
            torch.cuda.synchronize()
            for i, n in enumerate(ns):
                per_call[n].append(ev[i][0].elapsed_time(ev[i][1]))
        barrier()
    launches = pkg.spmm_launch_count() - launches0
    step_ms = [sum(per_call[n][s] for n in ns) for s in range(args.steps)]
    local_ms = float(statistics.mean(step_ms))
    ms = max_over_ranks(local_ms)
    flops_step = sum(2.0 * nnz * n for n in ns)
    value = whole_job_gflops(flops_step, world, ms)

    peak, peak_src = peaks()
    # dominant kernel: the (alg, n) call with the largest share of the step; roofline of its family
    comp = {n: compulsory_bytes(m, nnz, k, n) for n in ns}
    mean_call = {n: float(statistics.mean(per_call[n])) for n in ns}
    dom_alg = {pkg.ALG_ROW_SPLIT: "rowsplit_kernel", pkg.ALG_MERGE: "merge_kernel",
               pkg.ALG_ROW_SPLIT_HYBRID: "rowsplit_hybrid_kernel"}
    fam = max({alg_of[n] for n in ns}, key=lambda al: sum(mean_call[n] for n in ns if alg_of[n] == al))
    fam_ns = [n for n in ns if alg_of[n] == fam]
    achieved = sum(comp[n] for n in fam_ns) / (sum(mean_call[n] for n in fam_ns) * 1e-3) / 1e9
    traffic, traffic_note = measured_traffic(dom_alg[fam], label, fam_ns)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note, "kernel": dom_alg[fam], "peak_source": peak_src,
                "algorithmic_bytes": "compulsory: (m+1)*4 + nnz*8 + k*n*4 + m*n*4 per call, summed over n",
                "per_n": {str(n): {"ms": mean_call[n], "gb_s": comp[n] / (mean_call[n] * 1e-3) / 1e9,
                                   "gflops": 2.0 * nnz * n / (mean_call[n] * 1e-3) / 1e9,
                                   "alg": ALG_NAME[alg_of[n]]} for n in ns},
                "gather_aware": gather_aware(dom_alg[fam], label, m, nnz, k, fam_ns, mean_call, peak, l2),
                "gather_bound": gather_bound(m, nnz, k, ns, mean_call,
                                             lambda n: pkg.default_column_slabs(alg_of[n], k, n, pkg.F32)),
                "l2_bytes": l2}

    line = {"metric": "SpMM GFLOP/s (2*nnz*n/t)", "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (gen/, seed 1805): power-law CSR, N(0,1) B",
            "config": {"workload": label, "m": m, "k": k, "nnz": nnz, "max_row": max_row, "n": ns, "alg": args.alg,
                       "tuning": tuning,
                       "replicas": world, "l2_flush": "2x L2 write before every step", "parallelism": "replicas"},
            "roofline": roofline, "gpu_launches": int(launches),
            "ms_per_step_median": float(statistics.median(step_ms)),
            "step_ms_stats": {"median": float(statistics.median(step_ms)), "mean": float(statistics.mean(step_ms)),
                              "min": float(min(step_ms)), "max": float(max(step_ms)), "steps": len(step_ms)}}
    cs = clk.summary()
    if cs:
        line["clocks"] = cs

    line["selector"] = {"paper_section_5_4": {str(n): ALG_NAME[paper_pick[n]] for n in ns},
                        "gb300": {str(n): ALG_NAME[gb300_pick[n]] for n in ns}}
    head_rows = sample_rows(m, 4096, 51)
    head_C = {n: d_C[n][torch.from_numpy(head_rows).to(dev)].cpu().numpy() for n in ns}
    if rank == 0 and not args.no_extras:
        line["breakdown"] = breakdown(pkg, torch, one, ns, nnz, comp, args.steps, flush, stream)
        line["e2e"] = e2e(pkg, torch, a, ns, Bs, args, tuning)
    forms = [f for f in args.forms.split(",") if f]
    if rank == 0 and (forms or not args.no_extras):
        del d_B, d_C, ws
        torch.cuda.empty_cache()
    if rank == 0 and forms:
        line["forms"] = {}
        for form in forms:
            line["forms"][form] = FORMS[form](pkg, torch, flush, stream, args.steps, args)
            torch.cuda.empty_cache()
    if rank == 0 and not args.no_extras:
        line["plain"] = plain_latency(pkg, torch, flush, stream, args.steps)
        if world == 1:
            oracle_leg(line, a, ns, Bs, label, head_rows, head_C)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def breakdown(pkg, torch, one, ns, nnz, comp, steps, flush, stream):
    """GFLOP/s and compulsory GB/s of each algorithm family at every n (same timing rules)."""
    out = {}
    for alg in ("row_split", "merge", "hybrid"):
        out[alg] = {}
        for n in ns:
            for _ in range(2):
                one(n, alg)
            ts = []
            for _ in range(max(3, steps // 2)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one(n, alg)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            t = statistics.median(ts)
            out[alg][str(n)] = {"ms": t, "gflops": 2.0 * nnz * n / (t * 1e-3) / 1e9,
                                "gb_s": comp[n] / (t * 1e-3) / 1e9}
    return out


def e2e(pkg, torch, a, ns, Bs, args, tuning):
    """The step through the host-buffer entries: pinned host A, B in; host C out; copies timed.
    The step is one spmm_csr_host_multi call (A goes up once for the step's four products) and
    one synchronisation of the stream.  Beside it: the same step as one spmm_csr_host_async call
    per width (A goes up with each), and as synchronous spmm_csr_host calls."""
    rp = torch.from_numpy(a.row_ptr).pin_memory()
    ci = torch.from_numpy(a.col_ind).pin_memory()
    v = torch.from_numpy(a.vals).pin_memory()
    hB = {n: torch.from_numpy(Bs[n]).pin_memory() for n in ns}
    hC = {n: torch.empty((a.m, n), dtype=torch.float32).pin_memory() for n in ns}
    a_bytes = (a.m + 1) * 4 + a.nnz * 8
    h2d = a_bytes + sum(a.k * n * 4 for n in ns)
    h2d_per_width = sum(a_bytes + a.k * n * 4 for n in ns)
    d2h = sum(a.m * n * 4 for n in ns)
    stream = torch.cuda.current_stream()
    reps = max(5, min(args.steps, 10))
    Bl, Cl = [hB[n] for n in ns], [hC[n] for n in ns]

    def step(mode):
        if mode == "multi":
            pkg.spmm_host_multi(rp, ci, v, Bl, Cl, alg=args.alg, tuning=tuning)
        else:
            for n in ns:
                pkg.spmm_host(rp, ci, v, hB[n], hC[n], alg=args.alg, tuning=tuning, wait=mode == "sync")
        stream.synchronize()

    def timed(mode):
        for _ in range(max(args.warmup, 3)):  # warm-up steps (the staging pool grows to its steady size)
            step(mode)
        steps_s = []
        gc.disable()  # a collection of Python objects inside a step is not the library's time
        try:
            for _ in range(reps):  # each step is timed on its own, the median reported
                t0 = time.perf_counter()
                step(mode)
                steps_s.append(time.perf_counter() - t0)
        finally:
            gc.enable()
        return steps_s

    sync_s = timed("sync")
    async_s = timed("async")
    steps_s = timed("multi")
    t = statistics.median(steps_s)
    flops = sum(2.0 * a.nnz * n for n in ns)
    link = host_link(torch)

    def bound(up, down):  # the copies alone at the measured one-way and duplex rates
        return max(up / (link["h2d_gbs"] * 1e9), down / (link["d2h_gbs"] * 1e9),
                   (up + down) / (link["duplex_gbs"] * 1e9)) * 1e3

    bound_ms = bound(h2d, d2h)
    t_async = statistics.median(async_s)
    return {"value": flops / t / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": t * 1e3, "step_ms": {"median": t * 1e3, "min": min(steps_s) * 1e3,
                                                "max": max(steps_s) * 1e3, "steps": reps,
                                                "all": [round(x * 1e3, 3) for x in steps_s]},
            "api": "spmm_csr_host_multi",
            "per_width_calls": {"api": "spmm_csr_host_async", "h2d_bytes_per_step": h2d_per_width,
                                "ms_per_step": t_async * 1e3, "min": min(async_s) * 1e3, "max": max(async_s) * 1e3,
                                "value": flops / t_async / 1e9,
                                "frac_of_link_bound": bound(h2d_per_width, d2h) / (t_async * 1e3)},
            "sync_calls": {"api": "spmm_csr_host", "ms_per_step": statistics.median(sync_s) * 1e3,
                           "min": min(sync_s) * 1e3, "max": max(sync_s) * 1e3,
                           "value": flops / statistics.median(sync_s) / 1e9},
            "link": link, "link_bound_ms": bound_ms, "frac_of_link_bound": bound_ms / (t * 1e3)}


def host_link(torch, nbytes=256 << 20, reps=5):
    """Pinned host <-> device copy bandwidth (GB/s): one direction at a time and both at once.
    The e2e step cannot beat (h2d + d2h bytes) / duplex bandwidth."""
    dev = torch.device("cuda")
    n = nbytes // 4
    h_up, h_down = torch.empty(n).pin_memory(), torch.empty(n).pin_memory()
    d_up, d_down = torch.empty(n, device=dev), torch.empty(n, device=dev)
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()

    def rate(fn, moved):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return moved * reps / (time.perf_counter() - t0) / 1e9

    def duplex():
        with torch.cuda.stream(s_up):
            d_up.copy_(h_up, non_blocking=True)
        with torch.cuda.stream(s_down):
            h_down.copy_(d_down, non_blocking=True)

    out = {"h2d_gbs": rate(lambda: d_up.copy_(h_up, non_blocking=True), nbytes),
           "d2h_gbs": rate(lambda: h_down.copy_(d_down, non_blocking=True), nbytes),
           "duplex_gbs": rate(duplex, 2 * nbytes), "copy_bytes": nbytes}
    del h_up, h_down, d_up, d_down
    return out



# ----------------------------------------------------------------------------- growth forms

def _time(torch, fn, flush, stream, reps):
    """Median device time (ms) of fn() over reps runs, L2 flushed before each."""
    for _ in range(2):
        fn()
    ts = []
    for _ in range(max(3, reps)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(statistics.median(ts))


def _norm_diff(torch, C, C_ref, D):
    """max |C - C_ref| / D on the device (D = |A||B| from the library; where D == 0 both must be 0)."""
    diff = (C.float() - C_ref.float()).abs()
    nz = D > 0
    bad_zero = bool((diff[~nz] > 0).any().item()) if (~nz).any() else False
    return float("inf") if bad_zero else float((diff[nz] / D[nz]).max().item())


def form_precision(pkg, torch, flush, stream, steps, args):
    """2M x 2M, 32 nonzeros per row, n = 128: 16-bit storage vs the float32 plain kernel."""
    a, Bf = gen.workload_precision()
    dev = torch.device("cuda")
    rp, ci = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col_ind).to(dev)
    v32, B32 = torch.from_numpy(a.vals).to(dev), torch.from_numpy(Bf).to(dev)
    nnz, n = a.nnz, Bf.shape[1]
    lmax = pkg.max_row_length(rp)
    tun = {"max_row_len": lmax}
    flops = 2.0 * nnz * n
    out = {"workload": "uniform 2Mx2M, 32/row, n=128", "nnz": nnz}
    C32 = pkg.spmm(rp, ci, v32, B32, alg="auto_gb300", nnz=nnz, tuning=tun)
    D = pkg.spmm(rp, ci, v32.abs(), B32.abs(), alg="auto_gb300", nnz=nnz, tuning=tun)
    t32 = _time(torch, lambda: pkg.spmm(rp, ci, v32, B32, alg="auto_gb300", out=C32, nnz=nnz, tuning=tun),
                flush, stream, steps)
    out["f32_plain"] = {"ms": t32, "gflops": flops / t32 / 1e6}
    # sampled rows for the oracle leg: the original float32 sub-problem, and per variant the same
    # sub-problem with vals and B rounded as the variant stores them
    rows = sample_rows(a.m, 4096, 31)
    rows_d = torch.from_numpy(rows).to(dev)
    sub = subproblem(rows, a.row_ptr, a.col_ind, a.vals, Bf)
    SAMPLES["precision/f32_plain"] = dict(sub=sub, sub_rounded=None, C=C32[rows_d].float().cpu().numpy(),
                                          floor=0.0, tol_rounded=None)
    variants = {"bf16_vals_bf16_B_bf16_C": (torch.bfloat16, torch.bfloat16, torch.bfloat16),
                "bf16_vals_bf16_B_f32_C": (torch.bfloat16, torch.bfloat16, torch.float32),
                "bf16_vals_f16_B_f32_C": (torch.bfloat16, torch.float16, torch.float32),
                "f16_vals_f16_B_f16_C": (torch.float16, torch.float16, torch.float16)}
    for name, (tv, tb, tc) in variants.items():
        v16, B16 = v32.to(tv), B32.to(tb)
        C = pkg.spmm(rp, ci, v16, B16, alg="auto_gb300", out_dtype=tc, nnz=nnz, tuning=tun)
        t = _time(torch, lambda: pkg.spmm(rp, ci, v16, B16, alg="auto_gb300", out=C, nnz=nnz, tuning=tun),
                  flush, stream, steps)
        out[name] = {"ms": t, "gflops": flops / t / 1e6, "speedup_vs_f32": t32 / t,
                     "max_norm_diff_vs_f32_path": _norm_diff(torch, C, C32, D)}
        rnd = lambda x, dt: torch.from_numpy(x).to(dt).double().numpy()
        sub_r = (sub[0], sub[1], rnd(sub[2], tv), rnd(sub[3], tb))
        tc_name = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}[tc]
        SAMPLES["precision/" + name] = dict(
            sub=sub, sub_rounded=sub_r, C=C[rows_d].float().cpu().numpy(),
            floor=2.0 ** -25 if tc_name == "f16" else 0.0,
            tol_rounded={"f32": 1e-5, "bf16": 2.0 ** -8, "f16": 2.0 ** -10}[tc_name])
        del v16, B16, C
    return out


def form_backward(pkg, torch, flush, stream, steps, args):
    """GCN layer (500k nodes, mean degree ~20, n = 256): forward, dX = A^T dY, dvals = SDDMM."""
    a, X = gen.workload_gcn()
    dev = torch.device("cuda")
    rp, ci = torch.from_numpy(a.row_ptr).to(dev), torch.from_numpy(a.col_ind).to(dev)
    v, dX_in = torch.from_numpy(a.vals).to(dev), torch.from_numpy(X).to(dev)
    dY_h = gen.normal_matrix(a.m, X.shape[1], gen.SEED_BASE + 4, stream=7)
    dY = torch.from_numpy(dY_h).to(dev)
    A = pkg.CSRMatrix(rp, ci, (a.m, a.k))
    nnz, n = a.nnz, X.shape[1]
    flops = 2.0 * nnz * n
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    A.transpose_pattern()
    torch.cuda.synchronize()
    t_transpose = (time.perf_counter() - t0) * 1e3
    rpt, cit, perm, lmax_t = A.transpose_pattern()
    vt = pkg.gather_values(perm, v)
    Y = A.spmm(v, dX_in)
    dX = pkg.spmm(rpt, cit, vt, dY, alg="auto_gb300", nnz=nnz, tuning={"max_row_len": lmax_t})
    dv = pkg.sddmm(rp, ci, dY, dX_in)
    t_fwd = _time(torch, lambda: A.spmm(v, dX_in, out=Y), flush, stream, steps)
    t_dx = _time(torch, lambda: (pkg.gather_values(perm, v, out=vt),
                                 pkg.spmm(rpt, cit, vt, dY, alg="auto_gb300", out=dX, nnz=nnz,
                                          tuning={"max_row_len": lmax_t})), flush, stream, steps)
    t_sd = _time(torch, lambda: pkg.sddmm(rp, ci, dY, dX_in, out=dv), flush, stream, steps)
    # the transpose on its own (a pattern that changes every step would pay it every step): outputs and
    # workspace preallocated, device time
    rpt2, cit2, perm2 = torch.empty_like(rpt), torch.empty_like(cit), torch.empty_like(perm)
    ws_t = torch.empty(pkg.spmm_csr_transpose_workspace_size(a.m, a.k, nnz), dtype=torch.uint8, device=dev)
    t_tr = _time(torch, lambda: pkg._check(pkg.spmm_csr_transpose(
        a.m, a.k, nnz, rp.data_ptr(), ci.data_ptr(), rpt2.data_ptr(), cit2.data_ptr(), perm2.data_ptr(), ws_t.data_ptr(),
        ws_t.numel(), stream.cuda_stream), "spmm_csr_transpose"), flush, stream, steps)
    assert torch.equal(rpt2, rpt) and torch.equal(cit2, cit) and torch.equal(perm2, perm)
    # sampled outputs for the oracle leg: rows of Y, rows of dX (= columns of A), dvals of sampled rows
    rows = sample_rows(a.m, 2048, 41)
    cols = sample_rows(a.k, 2048, 42)
    idx = row_nonzeros(rows, a.row_ptr)
    SAMPLES["backward"] = dict(a=a, X=X, dY=dY_h, rows=rows, cols=cols, idx=idx,
                               Y=Y[torch.from_numpy(rows).to(dev)].cpu().numpy(),
                               dX=dX[torch.from_numpy(cols).to(dev)].cpu().numpy(),
                               dv=dv[torch.from_numpy(idx).to(dev)].cpu().numpy())
    step = t_fwd + t_dx + t_sd
    return {"workload": "Chung-Lu GCN 500k, n=256", "nnz": nnz, "mean_degree": a.info["mean_degree"],
            "max_degree": a.info["max_degree"], "transpose_first_call_ms": t_transpose,
            "transpose": {"ms": t_tr, "note": "stable radix sort by column, device time with preallocated "
                                               "outputs; the first call above also allocates and measures the "
                                               "longest row of A^T"},
            "forward": {"ms": t_fwd, "gflops": flops / t_fwd / 1e6},
            "dX_AT_dY": {"ms": t_dx, "gflops": flops / t_dx / 1e6, "includes": "vals gather + SpMM on A^T"},
            "dvals_sddmm": {"ms": t_sd, "gflops": flops / t_sd / 1e6},
            "fwd_bwd_step_ms": step,
            "vs_f32_plain_forward": {
                "note": "the plain float32 forward SpMM A X on this shape (GB300 selector) is the unit",
                "dX_over_forward": t_dx / t_fwd, "sddmm_over_forward": t_sd / t_fwd,
                "step_over_three_forwards": step / (3.0 * t_fwd)}}


def form_batched(pkg, torch, flush, stream, steps, args):
    """2048 CSR matrices of uneven sizes in one persistent graph-captured launch vs a loop of launches."""
    s = gen.workload_batched(count=args.batched_count)
    dev = torch.device("cuda")
    rps, cis, vs, Bs, Cs = [], [], [], [], []
    g = torch.Generator(device=dev).manual_seed(gen.SEED_BASE + 5)
    for i, (a, n) in enumerate(zip(s.mats, s.ns)):
        rps.append(torch.from_numpy(a.row_ptr).to(dev))
        cis.append(torch.from_numpy(a.col_ind).to(dev))
        vs.append(torch.from_numpy(a.vals).to(dev))
        Bs.append(torch.randn(a.k, n, device=dev, generator=g))
        Cs.append(torch.empty((a.m, n), device=dev))
    flops = sum(2.0 * a.nnz * n for a, n in zip(s.mats, s.ns))
    out = {"workload": f"{args.batched_count} matrices, m log-uniform [64, 65536], Poisson rows lambda U[4,64], "
                       "n in {32,64,128}",
           "total_nnz": s.info["total_nnz"], "total_rows": s.info["total_rows"]}
    for pol_name, pol in (("model", pkg.BATCHED_MODEL), ("autotune", pkg.BATCHED_AUTOTUNE)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = pkg.BatchedPlan(rps, cis, vs, Bs, Cs, policy=pol)
        torch.cuda.synchronize()
        t_plan = (time.perf_counter() - t0) * 1e3
        plan.capture_graph()
        algs, items, tiles = plan.query()
        t_graph = _time(torch, plan.launch_graph, flush, stream, steps)
        t_loop = _time(torch, plan.run_unfused, flush, stream, max(3, steps // 3))
        out[pol_name] = {"plan_ms": t_plan, "work_items": items, "merge_tiles": tiles,
                         "merge_matrices": int(sum(1 for x in algs if x == pkg.ALG_MERGE)),
                         "graph": {"ms": t_graph, "gflops": flops / t_graph / 1e6},
                         "loop_of_launches": {"ms": t_loop, "gflops": flops / t_loop / 1e6},
                         "speedup_vs_loop": t_loop / t_graph}
        plan.close()
    return out


def plain_latency(pkg, torch, flush, stream, steps):
    """The plain 4096 x 4096 product (16 nonzeros per row, n = 64, float32): one call with the L2
    flushed before it, one call warm, and a CUDA graph replaying 100 calls (per call)."""
    a, B = gen.workload_plain()
    dev = torch.device("cuda")
    rp, ci, v = (torch.from_numpy(x).to(dev) for x in (a.row_ptr, a.col_ind, a.vals))
    Bd = torch.from_numpy(B).to(dev)
    n = B.shape[1]
    C = torch.empty((a.m, n), device=dev)
    lmax = pkg.max_row_length(rp)
    tun = {"max_row_len": lmax}
    alg = pkg.spmm_select_alg_gb300(a.m, a.nnz, lmax, n, pkg.F32)
    ws_b = max(pkg.workspace_size(a.m, a.k, n, a.nnz, al) for al in (pkg.ALG_MERGE, pkg.ALG_ROW_SPLIT_HYBRID))
    ws = torch.empty(max(ws_b, 256), dtype=torch.uint8, device=dev)

    def call():
        pkg.spmm(rp, ci, v, Bd, alg=alg, out=C, nnz=a.nnz, tuning=tun, workspace=ws)

    reps = max(steps, 20)
    t_flushed = _time(torch, call, flush, stream, reps)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        call()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(100):
            call()
    g.replay()
    torch.cuda.synchronize()
    def replays(flushed):
        tg = []
        for _ in range(5):
            if flushed:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            tg.append(e0.elapsed_time(e1) / 100.0)
        return float(statistics.median(tg))

    t_graph = replays(True)
    t_warm = replays(False)
    del g
    SAMPLES["plain"] = dict(a=a, B=B, C=C.cpu().numpy())
    flops = 2.0 * a.nnz * n
    comp = compulsory_bytes(a.m, a.nnz, a.k, n)
    return {"workload": "plain 4096x4096, 16 nonzeros per row, n=64", "nnz": a.nnz, "alg": ALG_NAME[alg],
            "compulsory_bytes": comp,
            "l2_flushed_call": {"ms": t_flushed, "gflops": flops / t_flushed / 1e6,
                                "note": "one call, CUDA events, the L2 flush before it keeps the GPU busy "
                                        "while the call is enqueued"},
            "graph_100_calls_after_flush": {"ms_per_call": t_graph, "gflops": flops / t_graph / 1e6,
                                            "note": "L2 flushed before each replay of 100 back-to-back calls"},
            "graph_100_calls_warm": {"ms_per_call": t_warm, "gflops": flops / t_warm / 1e6,
                                     "note": "replays back to back, inputs resident in L2"}}


def oracle_leg(line, a, ns, Bs, label, head_rows, head_C):
    """The cpu_baseline leg: the FP64 oracle timed on a bounded sample of the headline workload, and
    the sampled GPU results of the headline and the forms checked against it (normalised error
    max |C - C_ref| / (|A||B|); the 16-bit forms against the oracle on the original float32 inputs
    and on the inputs rounded as stored)."""
    import oracle

    g, t, nrows, thr, passes = time_oracle_sample(a, ns, Bs)
    line["cpu_baseline"] = {"value": g, "unit": "GFLOP/s", "cores": thr, "kind": "oracle",
                            "sample": f"{passes} pass(es) over {nrows} seeded random rows of the {label} "
                                      f"matrix, all n, {t:.1f} s"}
    errs = {}
    for n in ns:
        ref = oracle.spmm_rows(head_rows, a.row_ptr, a.col_ind, a.vals, Bs[n])
        D = oracle.abs_bound_rows(head_rows, a.row_ptr, a.col_ind, a.vals, Bs[n])
        errs[str(n)] = oracle.normalized_error(head_C[n], ref, D)
    line["oracle_check"] = {"rows_sampled": int(len(head_rows)), "max_norm_error": errs, "bound": 1e-5}
    forms = line.get("forms", {})
    if "precision" in forms:
        for key, smp in SAMPLES.items():
            if not key.startswith("precision/"):
                continue
            rp, ci, v, Bsub = smp["sub"]
            e_o = oracle.normalized_error(smp["C"], oracle.spmm(rp, ci, v, Bsub), oracle.abs_bound(rp, ci, v, Bsub),
                                          abs_floor=smp["floor"])
            entry = {"vs_original_f32_inputs": e_o, "bound_original": 1e-2 if smp["sub_rounded"] else 1e-5,
                     "rows_sampled": int(len(rp) - 1)}
            if smp["sub_rounded"] is not None:
                rp, ci, v, Bsub = smp["sub_rounded"]
                entry["vs_rounded_inputs"] = oracle.normalized_error(
                    smp["C"], oracle.spmm(rp, ci, v, Bsub), oracle.abs_bound(rp, ci, v, Bsub), abs_floor=smp["floor"])
                entry["bound_rounded"] = smp["tol_rounded"]
            forms["precision"].setdefault(key.split("/", 1)[1], {})["oracle_error"] = entry
    if "backward" in forms and "backward" in SAMPLES:
        smp = SAMPLES["backward"]
        A, X, dY = smp["a"], smp["X"], smp["dY"]
        rp, ci, v, Xs = subproblem(smp["rows"], A.row_ptr, A.col_ind, A.vals, X)
        e_y = oracle.normalized_error(smp["Y"], oracle.spmm(rp, ci, v, Xs), oracle.abs_bound(rp, ci, v, Xs))
        rpt, cit, perm = oracle.csr_transpose(A.row_ptr, A.col_ind, A.k)
        rq, cq, vq, dYs = subproblem(smp["cols"], rpt, cit, A.vals[perm], dY)
        e_dx = oracle.normalized_error(smp["dX"], oracle.spmm(rq, cq, vq, dYs), oracle.abs_bound(rq, cq, vq, dYs))
        dYr = dY[smp["rows"]]
        e_dv = oracle.normalized_error(smp["dv"], oracle.sddmm(rp, ci, dYr, Xs), oracle.sddmm_abs_bound(rp, ci, dYr, Xs))
        forms["backward"]["oracle_error"] = {"forward_rows": e_y, "dX_rows": e_dx, "dvals_of_rows": e_dv,
                                             "rows_sampled": int(len(smp["rows"])), "bound": 1e-5}
    if "plain" in line and "plain" in SAMPLES:
        smp = SAMPLES["plain"]
        pa, B = smp["a"], smp["B"]
        ref = oracle.spmm(pa.row_ptr, pa.col_ind, pa.vals, B)
        line["plain"]["oracle_error"] = oracle.normalized_error(
            smp["C"], ref, oracle.abs_bound(pa.row_ptr, pa.col_ind, pa.vals, B))
        threads = oracle.num_threads()
        oracle.set_threads(1)
        try:
            reps, t0 = 0, time.perf_counter()
            while reps < 3 or time.perf_counter() - t0 < 1.0:
                oracle.spmm(pa.row_ptr, pa.col_ind, pa.vals, B)
                reps += 1
            t1 = (time.perf_counter() - t0) / reps
        finally:
            oracle.set_threads(threads)
        line["plain"]["oracle_one_thread"] = {"ms": t1 * 1e3, "gflops": 2.0 * pa.nnz * B.shape[1] / t1 / 1e9}


FORMS = {"precision": form_precision, "backward": form_backward, "batched": form_batched}


# ----------------------------------------------------------------------------- sweeps

def run_sweep(args):
    """Parameter sweeps of the two families (one JSON line per point; not the benchmark)."""
    import torch

    import paper_1803_08601_gb300 as pkg

    pkg.build()
    pkg.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size // 4 + 1024, device=dev)
    reps = max(3, min(args.steps, 5))
    n = args.n[0] if args.n else 64  # width of the aspect-ratio and density sweeps
    name = ALG_NAME
    if args.sweep == "gather":
        return run_gather_sweep(pkg, torch, dev, flush, stream, reps)
    if args.sweep == "aspect":
        # dense matrices stored as CSR, from 2 rows of 2^23 nonzeros to 2^23 rows of 2 (the paper's Fig. 1 / Fig. 4)
        total = 1 << 24
        for lg in range(1, 24):
            m, k = 1 << lg, total >> lg
            rp = torch.arange(0, total + 1, k, dtype=torch.int32, device=dev)
            ci = torch.arange(k, dtype=torch.int32, device=dev).repeat(m)
            v = torch.rand(total, device=dev, generator=torch.Generator(device=dev).manual_seed(lg)) * 2 - 1
            B = torch.randn(k, n, device=dev, generator=torch.Generator(device=dev).manual_seed(100 + lg))
            C = torch.empty(m, n, device=dev)
            ws = torch.empty(max(pkg.workspace_size(m, k, n, total, "merge"),
                                 pkg.workspace_size(m, k, n, total, "hybrid")), dtype=torch.uint8, device=dev)
            row = {"sweep": "aspect", "m": m, "k": k, "nnz": total, "n": n,
                   "paper_pick": name[pkg.spmm_select_alg(m, total, 0.0)],
                   "gb300_pick": name[pkg.spmm_select_alg_gb300(m, total, k, n, pkg.F32)]}
            for alg in ("row_split", "merge", "hybrid"):
                r = reps if (alg == "merge" or k <= (1 << 16)) else 1  # very long rows: one timed run
                t = _time(torch, lambda: pkg.spmm(rp, ci, v, B, alg=alg, out=C, nnz=total, workspace=ws),
                          flush, stream, r)
                row[alg] = {"ms": t, "gflops": 2.0 * total * n / t / 1e6}
            print(json.dumps(row), flush=True)
            del rp, ci, v, B, C, ws
            torch.cuda.empty_cache()
    elif args.sweep == "spmv":
        run_spmv_sweep(pkg, torch, dev, flush, stream, reps)
    elif args.sweep == "selector":
        run_selector_sweep(pkg, torch, dev, flush, stream, reps)
    elif args.sweep == "tiling":
        # dense rows and a B beyond L2: where staging B panels in shared memory should pay most
        for m, k, per_row, nn in ((10_000, 1_000_000, 50_000, 64), (20_000, 1_000_000, 10_000, 64),
                                  (4_000, 2_000_000, 100_000, 64), (10_000, 1_000_000, 50_000, 128)):
            a = gen.uniform_rows(m, k, per_row, gen.SEED_BASE + 90)
            rp, ci, v = (torch.from_numpy(x).to(dev) for x in (a.row_ptr, a.col_ind, a.vals))
            del a
            B = torch.randn(k, nn, device=dev, generator=torch.Generator(device=dev).manual_seed(91))
            C = torch.empty(m, nn, device=dev)
            nnz = m * per_row
            ws = torch.empty(max(256, pkg.workspace_size(m, k, nn, nnz, "merge")), dtype=torch.uint8, device=dev)
            row = {"sweep": "tiling", "m": m, "k": k, "per_row": per_row, "nnz": nnz, "n": nn,
                   "b_bytes": k * nn * 4, "l2_bytes": torch.cuda.get_device_properties(dev).L2_cache_size,
                   "tiled_reuse": pkg.spmm_tiled_reuse(m, k, nnz, nn, pkg.F32)}
            ref = None
            for alg in ("row_split", "merge", "tiled"):
                t = _time(torch, lambda: pkg.spmm(rp, ci, v, B, alg=alg, out=C, nnz=nnz, workspace=ws), flush, stream,
                          3)
                if ref is None:
                    ref = C.clone()
                row[alg] = {"ms": t, "gflops": 2.0 * nnz * nn / t / 1e6, "max_abs_diff_vs_row_split":
                            float((C - ref).abs().max())}
            print(json.dumps(row), flush=True)
            del rp, ci, v, B, C, ws
            torch.cuda.empty_cache()
    else:
        # fixed fraction of nonzeros per row of a 100k x 100k matrix vs dense GEMM (the paper's Fig. 7)
        mk = 100_000
        B = torch.randn(mk, n, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
        # up to 21 %: nnz = 2.1e9 keeps every index below 2^31
        for frac in (0.0001, 0.001, 0.005, 0.01, 0.02, 0.05, 0.1, 0.12, 0.15, 0.18, 0.21):
            per_row = max(1, int(round(frac * mk)))
            a = gen.uniform_rows(mk, mk, per_row, gen.SEED_BASE + 70)
            rp, ci, v = (torch.from_numpy(x).to(dev) for x in (a.row_ptr, a.col_ind, a.vals))
            del a
            C = torch.empty(mk, n, device=dev)
            lmax = per_row
            tun = {"max_row_len": lmax}
            row = {"sweep": "density", "m": mk, "k": mk, "per_row": per_row, "density": per_row / mk,
                   "nnz": per_row * mk, "n": n, "gb300_pick": name[pkg.spmm_select_alg_gb300(mk, per_row * mk, lmax, n, pkg.F32)]}
            t = _time(torch, lambda: pkg.spmm(rp, ci, v, B, alg="auto_gb300", out=C, nnz=per_row * mk, tuning=tun),
                      flush, stream, reps)
            row["spmm"] = {"ms": t, "gflops": 2.0 * per_row * mk * n / t / 1e6}
            ref = C.clone()
            for alg in ("row_split", "tiled"):
                t = _time(torch, lambda: pkg.spmm(rp, ci, v, B, alg=alg, out=C, nnz=per_row * mk, tuning=tun),
                          flush, stream, reps)
                row[alg] = {"ms": t, "gflops": 2.0 * per_row * mk * n / t / 1e6,
                            "max_abs_diff_vs_spmm": float((C - ref).abs().max())}
            row["tiled_reuse"] = pkg.spmm_tiled_reuse(mk, mk, per_row * mk, n, pkg.F32)
            dense = torch.zeros(mk, mk, device=dev)
            dense.view(-1)[(torch.repeat_interleave(torch.arange(mk, device=dev), per_row) * mk + ci.long())] = v
            for tf32 in (False, True):
                torch.backends.cuda.matmul.allow_tf32 = tf32
                t = _time(torch, lambda: torch.matmul(dense, B, out=C), flush, stream, reps)
                row["gemm_tf32" if tf32 else "gemm_fp32"] = {"ms": t, "dense_tflops": 2.0 * mk * mk * n / t / 1e9}
            torch.backends.cuda.matmul.allow_tf32 = False
            print(json.dumps(row), flush=True)
            del rp, ci, v, C, dense
            torch.cuda.empty_cache()
    return 0


def run_gather_sweep(pkg, torch, dev, flush, stream, reps):
    """The gather-only probe (spmm_gather_probe): 2^24 rows of B read at uniformly random row
    indices, lane groups of row_bytes / 16 lanes, eight rows in flight per lane, over every SM;
    B from 16 MB to 1 GB, rows of 32-512 bytes.  Gathered TB/s and gathers per second per point
    (L2 flushed before each run, median of the runs)."""
    count = 1 << 24
    g = torch.Generator(device=dev).manual_seed(93)
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    for mb in (16, 32, 48, 64, 80, 96, 128, 192, 256, 512, 1024):
        buf = torch.empty(mb << 20, dtype=torch.uint8, device=dev)
        buf.fill_(1)
        for rb in (32, 64, 128, 256, 512):
            rows = (mb << 20) // rb
            idx = torch.randint(rows, (count,), generator=g, device=dev, dtype=torch.int32)
            t = _time(torch, lambda: pkg.gather_probe(buf, idx, rb, out), flush, stream, reps)
            print(json.dumps({"sweep": "gather", "b_mb": mb, "row_bytes": rb, "gathers": count, "ms": t,
                              "gathered_tb_s": count * rb / t / 1e9, "g_gathers_per_s": count / t / 1e6,
                              "l2_bytes": l2}), flush=True)
            del idx
        del buf
        torch.cuda.empty_cache()
    return 0


def run_selector_sweep(pkg, torch, dev, flush, stream, reps):
    """Row split, merge and the hybrid row split on 1M x 1M matrices of three row-length families
    (every row the same length, Poisson lengths, power-law lengths with density exponent 2 capped
    at 10^5) and mean lengths 2-64, at n = 8, 32, 64, 128; each point records the three times, the
    Section 5.4 rule's pick, the GB300 selector's pick and each pick's time relative to the fastest
    of the three (1 = right)."""
    name = ALG_NAME
    m = k = 1_000_000
    Bs = {n: torch.randn(k, n, device=dev, generator=torch.Generator(device=dev).manual_seed(300 + n))
          for n in (8, 32, 64, 128)}
    rng = np.random.default_rng(gen.SEED_BASE + 95)
    families = {"uniform": (2, 4, 6, 8, 12, 16, 32, 64), "poisson": (2, 4, 6, 8, 12, 16, 32, 64),
                "power_law": (12, 16, 32, 64)}  # exponent 2 with minimum 1 and the cap keeps the mean >= ~12
    for family, means in families.items():
        for d in means:
            if family == "uniform":
                lens = np.full(m, d, dtype=np.int64)
            elif family == "poisson":
                lens = rng.poisson(d, m).astype(np.int64)
            else:
                lens, _ = gen.power_law_lengths(m, k, gen.SEED_BASE + 96 + d, mean=float(d))
            a = gen.csr_from_lengths(np.minimum(lens, k), k, gen.SEED_BASE + 97 + d)
            rp, ci, v = (torch.from_numpy(x).to(dev) for x in (a.row_ptr, a.col_ind, a.vals))
            nnz, lmax = a.nnz, int(np.diff(a.row_ptr).max()) if m else 0
            del a
            for n, B in Bs.items():
                C = torch.empty(m, n, device=dev)
                ws = torch.empty(max(256, pkg.workspace_size(m, k, n, nnz, "merge"),
                                     pkg.workspace_size(m, k, n, nnz, "hybrid")), dtype=torch.uint8, device=dev)
                t = {}
                for alg in ("row_split", "merge", "hybrid"):
                    r = 1 if (alg == "row_split" and lmax > 20_000) else reps
                    t[alg] = _time(torch, lambda: pkg.spmm(rp, ci, v, B, alg=alg, out=C, nnz=nnz, workspace=ws), flush,
                                   stream, r)
                best = min(t.values())
                paper = name[pkg.spmm_select_alg(m, nnz, 0.0)]
                gb300 = name[pkg.spmm_select_alg_gb300(m, nnz, lmax, n, pkg.F32)]
                print(json.dumps({"sweep": "selector", "family": family, "mean_row": nnz / m, "max_row": lmax,
                                  "n": n, "nnz": nnz, "row_split_ms": t["row_split"], "merge_ms": t["merge"],
                                  "hybrid_ms": t["hybrid"],
                                  "paper_pick": paper, "paper_regret": t[paper] / best,
                                  "gb300_pick": gb300, "gb300_regret": t[gb300] / best}), flush=True)
                del C, ws
            del rp, ci, v
            torch.cuda.empty_cache()


def run_spmv_sweep(pkg, torch, dev, flush, stream, reps):
    """y = A x (n = 1): both families, both selectors, and cuSPARSE's CSR SpMV through torch as a
    library reference, on the compulsory-bytes roofline (m+1)*4 + nnz*8 + k*4 + m*4."""
    peak, peak_src = peaks()
    mats = [("power_law_1Mx1M_mean16_cap1e5", lambda: gen.workload_power_law()),
            ("uniform_1Mx1M_16", lambda: gen.uniform_rows(1_000_000, 1_000_000, 16, gen.SEED_BASE + 80)),
            ("uniform_4Mx4M_4", lambda: gen.uniform_rows(4_000_000, 4_000_000, 4, gen.SEED_BASE + 81)),
            ("uniform_2Mx2M_32", lambda: gen.uniform_rows(2_000_000, 2_000_000, 32, gen.SEED_BASE + 82)),
            ("uniform_250kx250k_64", lambda: gen.uniform_rows(250_000, 250_000, 64, gen.SEED_BASE + 83))]
    name = ALG_NAME
    for label, make in mats:
        a = make()
        m, k, nnz = a.m, a.k, a.nnz
        rp, ci, v = (torch.from_numpy(x).to(dev) for x in (a.row_ptr, a.col_ind, a.vals))
        lmax = int(np.diff(a.row_ptr).max()) if m else 0
        del a
        x = torch.randn(k, 1, device=dev, generator=torch.Generator(device=dev).manual_seed(9))
        y = torch.empty(m, 1, device=dev)
        ws = torch.empty(max(256, pkg.workspace_size(m, k, 1, nnz, "merge")), dtype=torch.uint8, device=dev)
        comp = (m + 1) * 4 + nnz * 8 + k * 4 + m * 4
        row = {"sweep": "spmv", "matrix": label, "m": m, "k": k, "nnz": nnz, "max_row": lmax,
               "compulsory_bytes": comp, "peak_gbs": peak, "peak_source": peak_src,
               "paper_pick": name[pkg.spmm_select_alg(m, nnz, 0.0)],
               "gb300_pick": name[pkg.spmm_select_alg_gb300(m, nnz, lmax, 1, pkg.F32)]}
        tun = {"max_row_len": lmax}
        ref = None
        for alg in ("row_split", "merge", "auto", "auto_gb300"):
            r = reps if not (alg in ("row_split", "auto") and lmax > 10_000) else 1
            t = _time(torch, lambda: pkg.spmm(rp, ci, v, x, alg=alg, out=y, nnz=nnz, workspace=ws, tuning=tun),
                      flush, stream, r)
            if ref is None:
                ref = y.clone()
            row[alg] = {"ms": t, "gb_s": comp / t / 1e6, "frac": comp / t / 1e6 / peak,
                        "gflops": 2.0 * nnz / t / 1e6, "max_abs_diff_vs_row_split": float((y - ref).abs().max())}
        # the same nnz random 4-byte reads of x with no reduction: the gather-request ceiling
        xf = x.view(-1)
        g = torch.empty(nnz, device=dev)
        t = _time(torch, lambda: torch.index_select(xf, 0, ci, out=g), flush, stream, reps)
        row["gather_only_index_select"] = {"ms": t, "g_gathers_per_s": nnz / t / 1e6}
        del g
        try:
            A = torch.sparse_csr_tensor(rp, ci, v, size=(m, k))
            xv = x.view(-1)
            t = _time(torch, lambda: torch.mv(A, xv), flush, stream, reps)
            row["cusparse_via_torch"] = {"ms": t, "gb_s": comp / t / 1e6, "frac": comp / t / 1e6 / peak,
                                         "max_abs_diff_vs_row_split": float((torch.mv(A, xv) - ref.view(-1)).abs().max())}
        except Exception as e:  # library reference only; the sweep stands without it
            row["cusparse_via_torch"] = {"unavailable": str(e).splitlines()[0][:200]}
        print(json.dumps(row), flush=True)
        del rp, ci, v, x, y, ws
        torch.cuda.empty_cache()


if __name__ == "__main__":
    sys.exit(main())
