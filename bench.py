"""Benchmark: pair interactions/s of the batched G-Charm hot path on GB300.

Workload (one "step"): N-body at scale -- 1,048,576 Plummer-sphere particles
(float4 xyzm, FP32), softening 0.01, buckets <= 32, opening angle 0.7.  Each
step drifts every particle by N(0, 1e-3) per axis (positions pre-generated
and resident in HBM before timing), uploads them in place into the pool,
rebuilds the octree and interaction lists on the GPU, and runs one batched
flush: chare-table residency, sorted pack, persistent interaction kernel,
FP64 per-id scatter.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun with N > 1, every rank runs an independent replica problem
(its own seed) on its own GPU; there is no data-path collective.  Rank 0
prints one JSON line.
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

from paper_2008_05712_gb300 import inputs  # noqa: E402

N_PART = 1 << 20
THETA = (7, 10)
BUCKET = 32
EPS2 = float(np.float32(1e-4))
METRIC = "pair interactions/sec, batched vs per-task launch on 1 GB300; p50/p99 task latency"
WORKLOAD = ("nbody_plummer_1M: 1,048,576 Plummer particles, theta=0.7, buckets<=32, "
            "eps=0.01, drift N(0,1e-3) + rebuild + batched flush per step")
# FP32 flops of one gravity interaction in the plain formula (no compensation):
# 3 sub, 3 FMA for r^2 + eps^2, 3 mul, 3 FMA accumulate, 1 add for phi.
FLOPS_PER_INTERACTION = 19
SM_COUNT = 152
FP32_LANES = 128
# Algorithmic bytes of the pack per list entry: 4 B slot, 16 B value gathered
# from the pool, 16 B staging write, 4 B permutation write.
PACK_BYTES_PER_ENTRY = 40
# DRAM bytes (read + write) per unit of work from ncu captures of the current
# kernels (None until captured again after a kernel change):
# k_gravity per interaction, the pack kernels per list entry.
# profiles/k_gravity_nbody262k.md: 502.6 MB for 2.949e8 interactions (262,144-particle
# step, k_gravity<128, 32>, the tuned tile shape) -- taken before the kernel
# gained its targets-per-lane parameter, so not reported for the current one
GRAVITY_DRAM_BYTES_PER_INTERACTION = None
# profiles/k_pack_mid_nbody262k.md: 629.6 MB for 3.07e7 entries (262,144-particle step,
# the chunked block sort)
PACK_DRAM_BYTES_PER_ENTRY = 629.6e6 / 3.07e7
# Algorithmic bytes of the per-id accumulation: a row's 32-byte compensated
# partial and its 4-byte id read, the id's FP64 total (32 B) read and written;
# the per-cell MD form derives ids from the task structure (no id read).
SCATTER_BYTES_PER_ROW = 32 + 4 + 32 + 32
MD_SCATTER_BYTES_PER_ROW = 32
MD_SCATTER_BYTES_PER_ID = 32 + 32
# FP32 instructions of one LJ candidate pair: about 6 when rejected (the
# displacement, |r|^2, the compare) and 40 when inside the cutoff (plus the
# force, the energy and the compensated sums)
LJ_INSTR_REJECTED = 6
LJ_INSTR_INSIDE = 40


# Uneven batch and serving workload: a two-Plummer merger of 4,194,304
# particles (3:1 mass, separation 10); 200,000 gravity tasks, target counts
# log-uniform on 8..1024 (contiguous Morton-order runs), source lists
# log-uniform on 16..16384 (runs of <= 32 Morton-consecutive ids); staging
# budget 2 GiB, so one batch of all tasks runs in waves.
C4_N = (3 << 20, 1 << 20)
C4_TASKS = 200_000
C4_T_RANGE = (8, 1024)
C4_S_RANGE = (16, 16384)
C4_BUDGET = 2 << 30
C4_WORKLOAD = ("uneven_200k: 200,000 gravity tasks over a 4,194,304-particle two-Plummer "
               "merger, nT ~ logU[8,1024], nS ~ logU[16,16384], staging budget 2 GiB")
# Interaction schedules chosen by the autotuner on this GPU, per workload
# (written on the first run, then reused).
TUNE_CACHE = os.path.join(ROOT, "paper_2008_05712_gb300", "tuning.json")
# serving: aggregate Poisson rates of 16 producers (tasks/s); every rate runs
# under each combining policy for SERVE_WARMUP_S + SERVE_SECONDS of arrivals
# (latency statistics from the arrivals after the warm-up; the 200k tasks
# replayed cyclically), with at most SERVE_DRAIN_S after the schedule for the
# queue an overloaded policy leaves behind
SERVE_RATES = (1e4, 1e5, 1e6)
SERVE_SECONDS = 10.0
SERVE_WARMUP_S = 1.0
SERVE_DRAIN_S = 2.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp32_peak_tflops(sm_mhz):
    return SM_COUNT * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts once the first sample is in
        t0 = time.time()
        while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                   samples=len(rows))
        return out


def replica_seed(rank):
    """Seed of rank `rank`'s replica problem (independent problems per rank)."""
    return inputs.SEED_BASE + 2 + 1000 * rank


def reduce_over_ranks(seconds, count, device):
    """Whole-job figures over the ranks of the default process group: the
    slowest rank's time (max) and the units all ranks processed (sum)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(count)], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), int(c.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(x, n_tasks, seed, budget_s=None, keep=None):
    """Oracle (plain FP64 C, one thread) on a seeded sample of this step's
    tasks: tree build, interaction-list walk and gravity of the sampled
    buckets.  Returns (interactions, seconds of per-task work, n_tasks); with
    keep a dict, also stores the sampled buckets and their FP64 rows there."""
    from oracle import oracle as O
    tr = O.Tree(x, bucket_max=BUCKET)
    g = inputs.rng(seed)
    pick = np.sort(g.choice(tr.n_buckets, size=min(n_tasks, tr.n_buckets), replace=False))
    t0 = time.perf_counter()
    off, ids = tr.lists(THETA[0], THETA[1], buckets=pick)
    to, tg = tr.bucket_targets(pick)
    tab = np.concatenate([x, tr.node_table()])
    rows = O.gravity_batch(tab, to, tg, off, ids, EPS2)
    dt = time.perf_counter() - t0
    inter = int(np.sum(np.diff(to.astype(np.int64)) * np.diff(off.astype(np.int64))))
    if keep is not None:
        keep.update(buckets=pick, tgt_off=to, tgt=tg, rows=rows, n_buckets=tr.n_buckets)
    return inter, dt, len(pick)


def error_stats(got_rows, ref_rows, off):
    """Per-result relative L2 force errors e_r (first 3 components of each
    task's rows): max, p99, median and the number of results."""
    errs = []
    for t in range(len(off) - 1):
        a, b = int(off[t]), int(off[t + 1])
        if b == a:
            continue
        ref = ref_rows[a:b, :3]
        nr = np.linalg.norm(ref)
        d = np.linalg.norm(got_rows[a:b, :3] - ref)
        errs.append(d / nr if nr > 1e-30 else (0.0 if d == 0 else np.inf))
    e = np.array(errs)
    return {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
            "median": float(np.median(e)), "results": int(e.shape[0]), "tolerance": 1e-5}


def _oracle_worker(x, buckets, barrier):
    from oracle import oracle as O
    tr = O.Tree(x, bucket_max=BUCKET)
    tab = np.concatenate([x, tr.node_table()])
    barrier.wait()
    t0 = time.time()
    off, ids = tr.lists(THETA[0], THETA[1], buckets=buckets)
    to, tg = tr.bucket_targets(buckets)
    O.gravity_batch(tab, to, tg, off, ids, EPS2)
    t1 = time.time()
    inter = int(np.sum(np.diff(to.astype(np.int64)) * np.diff(off.astype(np.int64))))
    return inter, t0, t1


def oracle_all_cores(x, workers):
    """The oracle as it stands, one process per host core (spawned), each
    on an interleaved share of every bucket of the step: tree build untimed,
    walk + FP64 gravity timed from a common start.  Returns (interactions,
    seconds, buckets)."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    tr = O.Tree(x, bucket_max=BUCKET)
    nb = tr.n_buckets
    del tr
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(workers)
        with ctx.Pool(workers) as pool:
            res = pool.starmap(_oracle_worker,
                               [(x, np.arange(w, nb, workers), barrier) for w in range(workers)])
    inter = sum(r[0] for r in res)
    dt = max(r[2] for r in res) - min(r[1] for r in res)
    return inter, dt, nb


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    x = inputs.plummer(N_PART, inputs.SEED_BASE + 2)
    per_step = 600
    for k in range(args.warmup):
        oracle_sample(x, 50, 100 + k)
    tot_i, tot_t = 0, 0.0
    for k in range(args.steps):
        i, t, _ = oracle_sample(x, per_step, 1000 + k)
        tot_i += i
        tot_t += t
    v = tot_i / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "interactions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{per_step} seeded-random buckets per step"},
        "cpu_baseline": {"value": v, "unit": "interactions/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} random buckets of the 1M-particle step per "
                                   "step (walk + FP64 gravity; tree build untimed)"},
        "e2e": {"value": v, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


MD_WORKLOAD = ("lj_fcc_1M: 1,048,576 Lennard-Jones atoms, jittered FCC at density 0.8442, "
               "cutoff 2.5 sigma, 42^3 periodic cells, 1,037,232 cell-pair tasks")
RC2 = 6.25


def md_rooflines(md, fp32_tflops, hbm_gbs, hbm_basis):
    """LJ interaction against the FP32 pipe (instructions per candidate pair)
    and the per-cell accumulation of the MD step against HBM."""
    cand, inside = md["candidate_pairs_per_step"], md["pairs_in_cutoff"]
    instr = LJ_INSTR_REJECTED * (cand - inside) + LJ_INSTR_INSIDE * inside
    ms_lj, ms_sc = md["stage_ms_avg"]["interact"], md["stage_ms_avg"]["scatter"]
    lj = {"kernel": "k_lj (interaction)", "bound": "alu",
          "achieved": instr / (ms_lj / 1e3) / 1e12, "peak": fp32_tflops / 2,
          "unit": "T FP32 lane-instructions/s",
          "peak_basis": "measured paired-FP32 FMA probe (gc_fp32_peak), one lane-instruction "
                        "per FMA",
          "work_per_unit": f"{LJ_INSTR_REJECTED} instructions per rejected candidate, "
                           f"{LJ_INSTR_INSIDE} per pair inside the cutoff",
          "units_per_launch": cand, "ms_per_launch": ms_lj, "traffic": None}
    lj["frac"] = lj["achieved"] / lj["peak"]
    rows, ids = md["rows_per_step"], md["atoms"]
    by = MD_SCATTER_BYTES_PER_ROW * rows + MD_SCATTER_BYTES_PER_ID * ids
    sc = {"kernel": "k_reduce_md (per-cell accumulation)", "bound": "hbm",
          "achieved": by / (ms_sc / 1e3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
          "peak_basis": hbm_basis,
          "work_per_unit": f"{MD_SCATTER_BYTES_PER_ROW} B per row, "
                           f"{MD_SCATTER_BYTES_PER_ID} B per atom (FP64 total read and written)",
          "units_per_launch": rows, "ms_per_launch": ms_sc, "traffic": None}
    sc["frac"] = sc["achieved"] / sc["peak"]
    return {"lj": lj, "scatter": sc}


def md_section(gcharm, torch, seed, stream, reps=5, with_oracle=True, cells=64, ncell=42):
    """The MD workload (Section 4.2 on the 3-D FCC system): task build from
    device-resident cell indices and one batched flush per step, timed with
    events; candidate pairs per second; parity on a seeded task sample.
    cells / ncell: FCC unit cells and MD cells per axis (64 / 42: 1,048,576
    atoms; smaller systems serve profiling)."""
    sysm = inputs.fcc_lj(cells, seed, ncell=ncell)
    label = MD_WORKLOAD if (cells, ncell) == (64, 42) else (
        f"lj_fcc: {sysm.n:,} Lennard-Jones atoms, jittered FCC at density 0.8442, cutoff "
        f"2.5 sigma, {ncell}^3 periodic cells, {14 * ncell ** 3:,} cell-pair tasks")
    n, m = sysm.n, sysm.ncell
    pool = gcharm.Pool(id_capacity=n, pool_capacity=n, eps2=EPS2, lj_rc2=RC2,
                       md_edge=sysm.edge, stream=stream.cuda_stream)
    pool.upload(np.arange(n, dtype=np.uint32), sysm.u)
    cell = torch.from_numpy(sysm.cell.astype(np.int32)).cuda()

    def step():
        pool.reset_totals()
        pool.build_md(cell, m)
        pool.flush()

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    s0 = pool.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    pool.join(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s1 = pool.stats()
    pairs = (s1["interactions"] - s0["interactions"]) / reps
    nb = s1["timed_batches"] - s0["timed_batches"]
    stage = {k: (s1["stage_ms_sum"][k] - s0["stage_ms_sum"][k]) / max(nb, 1)
             for k in s1["stage_ms_sum"]}
    out = {"workload": label, "atoms": n, "rows_per_step": int(pool.result_rows()),
           "ms_per_step": ms, "candidate_pairs_per_step": int(pairs),
           "value": pairs / (ms / 1e3), "unit": "candidate pairs/s",
           "pairs_in_cutoff": s1["lj_pairs_in_cutoff"], "stage_ms_avg": stage,
           "tasks_per_step": int((s1["tasks"] - s0["tasks"]) / reps)}
    if with_oracle:
        from oracle import oracle as O
        start, atoms = O.md_cells(sysm.cell, m ** 3)
        ta, tb, td, ts = O.md_tasks(m)
        cnt = (start[1:] - start[:-1]).astype(np.int64)
        roff = np.concatenate([[0], np.cumsum(cnt[ta] + np.where(ts != 0, 0, cnt[tb]))])
        rows = pool.values()
        pick = np.sort(inputs.rng(seed + 1).choice(len(ta), 2000, replace=False))
        got, ref, off = [], [], [0]
        t0 = time.perf_counter()
        cand = 0
        for k in pick:
            A = atoms[start[ta[k]]:start[ta[k] + 1]]
            B = atoms[start[tb[k]]:start[tb[k] + 1]]
            fa, fb = O.lj(sysm.u, A, None if ts[k] else B, bool(ts[k]), td[k], sysm.E,
                          rc2_grid=int(RC2 * (1 << 42)))
            r = fa if ts[k] else np.concatenate([fa, fb])
            cand += len(A) * (len(A) - 1) // 2 if ts[k] else len(A) * len(B)
            ref.append(r)
            got.append(rows[roff[k]:roff[k + 1]])
            off.append(off[-1] + len(r))
        dt = time.perf_counter() - t0
        out["parity_on_sample"] = error_stats(np.concatenate(got), np.concatenate(ref),
                                              np.array(off))
        out["cpu_baseline"] = {"value": cand / dt, "unit": "candidate pairs/s", "cores": 1,
                               "kind": "oracle",
                               "sample": "2000 seeded-random cell-pair tasks of the step "
                                         "(FP64 LJ, one thread; includes Python call overhead "
                                         "per task)"}
    pool.close()
    return out


C1_WORKLOAD = ("plummer_4096: 4,096 Plummer particles, theta=0.7, buckets<=32, eps=0.01, "
               "every bucket's task in one batch")


def c1_section(gcharm, torch, seed, stream, reps=200, with_oracle=True):
    """The small case: one batch of every bucket of a 4096-particle tree, as
    a step (tree build and flush), as the flush of the built tasks alone,
    with one interaction launch per task, and replayed as a CUDA graph."""
    n = 4096
    x = inputs.plummer(n, seed)
    pool = gcharm.Pool(id_capacity=4 * n, pool_capacity=4 * n, eps2=EPS2,
                       stream=stream.cuda_stream)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    xd = torch.from_numpy(x).cuda()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        pool.join(stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    def step():
        pool.build_nbody(xd, BUCKET, *THETA)
        pool.flush()

    for _ in range(5):
        step()
    s0 = pool.stats()
    ms_step = timed(step, reps)
    s1 = pool.stats()
    inter = (s1["interactions"] - s0["interactions"]) / reps
    tasks = int((s1["tasks"] - s0["tasks"]) / reps)
    nbt = s1["timed_batches"] - s0["timed_batches"]
    flush_ms = (s1["stage_ms_sum"]["total"] - s0["stage_ms_sum"]["total"]) / max(nbt, 1)
    inter_ms = (s1["stage_ms_sum"]["interact"] - s0["stage_ms_sum"]["interact"]) / max(nbt, 1)
    out = {"workload": C1_WORKLOAD, "tasks": tasks, "interactions": int(inter),
           "step": {"ms": ms_step, "value": inter / (ms_step / 1e3), "unit": "interactions/s",
                    "note": "tree build, walk and one batched flush per step"},
           "batched_flush": {"ms": flush_ms, "value": inter / (flush_ms / 1e3),
                             "interaction_ms": inter_ms,
                             "interaction_value": inter / (inter_ms / 1e3),
                             "unit": "interactions/s"}}
    # one interaction launch per task (the uncombined form of Section 3.1)
    per = []
    for _ in range(5):
        pool.build_nbody(xd, BUCKET, *THETA)
        pool.flush_per_task()
        torch.cuda.synchronize()
        per.append(pool.timings())
    per_flush = statistics.median(t["total"] for t in per)
    per_inter = statistics.median(t["interact"] for t in per)
    out["per_task_launch"] = {"ms": per_flush, "value": inter / (per_flush / 1e3),
                              "interaction_ms": per_inter,
                              "interaction_value": inter / (per_inter / 1e3),
                              "unit": "interactions/s",
                              "speedup_batched_flush": per_flush / flush_ms,
                              "speedup_interaction": per_inter / inter_ms}
    # the batch captured once and replayed as a CUDA graph
    pool.build_nbody(xd, BUCKET, *THETA)
    graph = gcharm.Graph(pool)
    graph.launch()
    graph.wait()
    ms_graph = timed(graph.launch, reps)
    graph.wait()
    if with_oracle:
        from oracle import oracle as O
        tr = O.Tree(x)
        tab = np.concatenate([x, tr.node_table()])
        to, tg = tr.bucket_targets()
        lo, li = tr.lists(*THETA)
        ref = O.gravity_batch(tab, to, tg, lo, li, EPS2)
        out["parity_on_graph_rows"] = error_stats(gcharm.value(graph.results()), ref, to)
    graph.close()
    out["graph_replay"] = {"ms": ms_graph, "value": inter / (ms_graph / 1e3),
                           "unit": "interactions/s",
                           "note": "same tasks and chare table each replay (no tree build)"}
    pool.close()
    return out


EWALD_WORKLOAD = ("ewald_1M: Ewald corrections of 1,048,576 particles uniform in a periodic "
                  "unit cube, one task per tree bucket (targets = the bucket, source = the "
                  "root monopole), alpha = 2/L, images |n_i| <= 2, |h|^2 <= 10")


def ewald_section(gcharm, torch, seed, stream, reps=5, with_oracle=True):
    """Periodic-gravity corrections (the tree code's Ewald step) as a batch
    of GC_EWALD tasks over the buckets of a 1M-particle tree."""
    n = 1 << 20
    g = inputs.rng(seed)
    x = np.empty((n, 4), np.float32)
    x[:, :3] = g.uniform(0.0, 1.0, size=(n, 3))
    x[:, 3] = 1.0 / n
    pool = gcharm.Pool(id_capacity=2 * n + 1024, pool_capacity=2 * n + 1024, eps2=EPS2,
                       stream=stream.cuda_stream, ewald_box=1.0)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    info = pool.build_nbody(x, BUCKET, *THETA)
    pool.flush()
    counts = pool.nbody_bucket_counts(info["n_buckets"]).astype(np.int64)
    sid = pool.nbody_sorted_ids(n)
    nb = counts.shape[0]
    to = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    so = np.arange(nb + 1, dtype=np.uint64)
    sr = np.full(nb, n, np.uint32)                     # node id n + 0: the root
    dk = torch.full((nb,), 3, dtype=torch.int32, device="cuda")
    dto = torch.from_numpy(to.view(np.int64)).cuda()
    dso = torch.from_numpy(so.view(np.int64)).cuda()
    dtg = torch.from_numpy(sid.view(np.int32)).cuda()
    dsr = torch.from_numpy(sr.view(np.int32)).cuda()
    torch.cuda.synchronize()

    def step():
        pool.submit_csr_device(dk, dto, dtg, dso, dsr, n, nb)
        pool.flush()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    s0 = pool.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        step()
    pool.join(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s1 = pool.stats()
    nbt = s1["timed_batches"] - s0["timed_batches"]
    stage = {k: (s1["stage_ms_sum"][k] - s0["stage_ms_sum"][k]) / max(nbt, 1)
             for k in s1["stage_ms_sum"]}
    out = {"workload": EWALD_WORKLOAD, "tasks": nb, "pairs_per_batch": n,
           "ms_per_batch": ms, "value": n / (ms / 1e3), "unit": "target-source pairs/s",
           "stage_ms_avg": stage}
    if with_oracle:
        from oracle import oracle as O
        rows = pool.values()
        pick = np.sort(inputs.rng(seed + 1).choice(nb, 200, replace=False))
        tab = np.concatenate([x, np.zeros((1, 4), np.float32)])
        got, ref, off = [], [], [0]
        tab[n] = pool.nbody_node_values(info["n_nodes"])[0]   # the root's (COM, mass)
        for b in pick:
            tg = sid[to[b]:to[b + 1]]
            ref.append(O.ewald(tab, tg, [n], 1.0))
            got.append(rows[to[b]:to[b + 1]])
            off.append(off[-1] + len(tg))
        out["parity_on_sample"] = error_stats(np.concatenate(got), np.concatenate(ref),
                                              np.array(off))
    pool.close()
    return out


def uneven_setup(gcharm, torch, seed, stream):
    """Pool, merger and the 200k uneven tasks (host arrays)."""
    x = inputs.merger(*C4_N, seed)
    n = x.shape[0]
    pool = gcharm.Pool(id_capacity=2 * n + 1024, pool_capacity=2 * n + 1024, eps2=EPS2,
                       staging_budget_bytes=C4_BUDGET, stream=stream.cuda_stream)
    pool.upload(np.arange(n, dtype=np.uint32), x)
    # Morton order of the merger from the library's own tree build (the
    # built N-body step is flushed: it doubles as a warm-up)
    pool.build_nbody(x, BUCKET, *THETA)
    pool.flush()
    order = pool.nbody_sorted_ids(n)
    to, tg, so, sr = inputs.uneven_tasks(n, C4_TASKS, seed + 1, C4_T_RANGE, C4_S_RANGE,
                                         order=order)
    return x, pool, to, tg, so, sr


def uneven_plain(gcharm, torch, seed, stream, batches=2):
    """The uneven batch alone, flushed `batches` times from device-resident
    task arrays (no tuning, no graph, no serving): the profiling form."""
    x, pool, to, tg, so, sr = uneven_setup(gcharm, torch, seed, stream)
    dev = [torch.from_numpy(a.view(t)).cuda() for a, t in
           [(np.zeros(C4_TASKS, np.uint32), np.int32), (to, np.int64), (tg, np.int32),
            (so, np.int64), (sr, np.int32)]]
    torch.cuda.synchronize()
    out = {"workload": C4_WORKLOAD, "batches": []}
    for _ in range(batches):
        pool.submit_csr_device(*dev, tg.shape[0], sr.shape[0])
        pool.flush()
        stream.synchronize()
        out["batches"].append(pool.timings())
    pool.close()
    return out


def uneven_and_serving(gcharm, torch, seed, stream, batch_reps=3, with_oracle=True,
                       serve_seconds=SERVE_SECONDS, serve_warmup=SERVE_WARMUP_S):
    """The 200k-task uneven batch (device-resident task arrays, timed with
    events) and the serving loop at three arrival rates (host task arrays,
    host clock, latency from each task's scheduled arrival)."""
    x, pool, to, tg, so, sr = uneven_setup(gcharm, torch, seed, stream)
    n = x.shape[0]
    kinds = np.zeros(C4_TASKS, np.uint32)
    nt = (to[1:] - to[:-1]).astype(np.float64)
    ns = (so[1:] - so[:-1]).astype(np.float64)
    inter = float((nt * ns).sum())

    # one batch of all tasks, task arrays resident in HBM
    dk = torch.from_numpy(kinds.view(np.int32)).cuda()
    dto = torch.from_numpy(to.view(np.int64)).cuda()
    dso = torch.from_numpy(so.view(np.int64)).cuda()
    dtg = torch.from_numpy(tg.view(np.int32)).cuda()
    dsr = torch.from_numpy(sr.view(np.int32)).cuda()
    torch.cuda.synchronize()

    def batch():
        pool.submit_csr_device(dk, dto, dtg, dso, dsr, tg.shape[0], sr.shape[0])
        pool.flush()

    # autotune the interaction schedule on the first 40,000 tasks (one wave)
    m = 40_000
    pool.submit_csr(kinds[:m], to[:m + 1], tg[:int(to[m])], so[:m + 1], sr[:int(so[m])])
    pool.flush()
    tuning, tune_ms = pool.autotune(reps=2, cache=TUNE_CACHE, key="uneven_200k")
    batch()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    i0 = pool.stats()["interactions"]
    e0.record(stream)
    for _ in range(batch_reps):
        batch()
    pool.join(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / batch_reps
    st = pool.stats()
    uneven = {"workload": C4_WORKLOAD, "tasks": C4_TASKS,
              "interactions": int((st["interactions"] - i0) / batch_reps),
              "list_entries": int(tg.shape[0] + sr.shape[0]),
              "ms_per_batch": ms, "value": inter / (ms / 1e3), "unit": "interactions/s",
              "waves": st["last_waves"], "stage_ms_last_batch": pool.timings(),
              "reps": batch_reps,
              "tuning": {"wu_max_targets": tuning["wu_max_targets"],
                         "schedule": "lpt" if tuning["schedule"] else "fifo",
                         "tile_pairs": tuning["tile_pairs"],
                         "comp_block": tuning["comp_block"],
                         "targets_per_lane": tuning["targets_per_lane"],
                         "autotune_ms": tune_ms or tuning.get("times_ms")}}
    if with_oracle:
        # parity on 300 seeded tasks of the batch against the FP64 oracle
        from oracle import oracle as O
        rows = pool.results()
        pick = np.sort(inputs.rng(seed + 7).choice(C4_TASKS, 300, replace=False))
        nt_i = (to[1:] - to[:-1]).astype(np.int64)
        ns_i = (so[1:] - so[:-1]).astype(np.int64)
        sto = np.concatenate([[0], np.cumsum(nt_i[pick])]).astype(np.uint64)
        sso = np.concatenate([[0], np.cumsum(ns_i[pick])]).astype(np.uint64)
        stg = np.concatenate([tg[to[t]:to[t + 1]] for t in pick])
        ssr = np.concatenate([sr[so[t]:so[t + 1]] for t in pick])
        ref = O.gravity_batch(x, sto, stg, sso, ssr, EPS2)
        got = np.concatenate([gcharm.value(rows[to[t]:to[t + 1]]) for t in pick])
        uneven["parity_on_sample"] = error_stats(got, ref, sto)

    # the persistent + graph form: the batch captured once, then replayed
    pool.submit_csr_device(dk, dto, dtg, dso, dsr, tg.shape[0], sr.shape[0])
    graph = gcharm.Graph(pool)
    graph.launch()
    graph.wait()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(batch_reps):
        graph.launch()
    pool.join(stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    gms = e0.elapsed_time(e1) / batch_reps
    graph.wait()
    uneven["graph_replay"] = {"ms_per_batch": gms, "value": inter / (gms / 1e3),
                              "unit": "interactions/s", "reps": batch_reps,
                              "note": "same tasks and chare table each replay; values read "
                                      "from the pool at replay time"}
    graph.close()
    del dk, dto, dso, dtg, dsr

    # serving: open-loop Poisson arrivals (16 producers merged), every rate
    # under every combining policy
    serving = {"workload": C4_WORKLOAD + "; tasks arrive as open-loop Poisson streams of "
                                         "16 producers, the 200k tasks replayed cyclically",
               "latency": "host CLOCK_MONOTONIC, scheduled arrival -> completion observed; "
                          f"statistics over the arrivals after a {serve_warmup:g} s warm-up",
               "seconds_per_run": serve_seconds, "warmup_s": serve_warmup,
               "drain_limit_s": SERVE_DRAIN_S, "runs": []}
    policies = [
        (gcharm.GC_COMBINE_GREEDY, "greedy (continuous batching)"),
        (gcharm.GC_COMBINE_ADAPTIVE, "adaptive, running max of the arrival gaps (Section 3.1)"),
        (gcharm.GC_COMBINE_ADAPTIVE_WINDOW, "adaptive, running max over the last 1024 gaps"),
        (gcharm.GC_COMBINE_STATIC, "static, every 100 arrivals (Section 4.3)"),
        (gcharm.GC_COMBINE_PER_TASK, "per task (no combining)"),
    ]
    for k, rate in enumerate(SERVE_RATES):
        m = int(rate * (serve_warmup + serve_seconds))
        arr = inputs.poisson_arrivals(m, rate, seed + 10 + k)
        for policy, name in policies:
            rep, lat, _ = pool.serve(arr, kinds, to, tg, so, sr, policy=policy,
                                     task_set=C4_TASKS, warmup_ns=int(serve_warmup * 1e9),
                                     drain_ns=int(SERVE_DRAIN_S * 1e9))
            served = m - rep["unserved"]
            lat_ok = rep["measured"] > 0     # else no arrival after the warm-up was served
            serving["runs"].append({
                "rate_tasks_per_s": rate, "policy": name, "arrivals": m,
                "measured": rep["measured"], "unserved": rep["unserved"],
                "served_tasks_per_s": served / rep["wall_s"],
                "p50_us": rep["lat_p50_us"] if lat_ok else None,
                "p99_us": rep["lat_p99_us"] if lat_ok else None,
                "max_us": rep["lat_max_us"] if lat_ok else None,
                "mean_us": rep["lat_mean_us"] if lat_ok else None,
                "interactions_per_s": rep["interactions_per_s"], "wall_s": rep["wall_s"],
                "batches": rep["batches"], "mean_batch": rep["mean_batch"],
                "max_size": rep["max_size"], "busy_s": rep["busy_s"],
                "host_s": {"submit": rep["submit_s"], "flush": rep["flush_s"],
                           "retire": rep["retire_s"]},
                "pinned_bytes": rep["pinned_bytes"]})
    pool.close()
    return uneven, serving


def run_section(args):
    """One workload alone on one GPU: the form the profiles capture."""
    import torch

    from paper_2008_05712_gb300 import gcharm

    gcharm.load()
    stream = torch.cuda.Stream()
    if args.section == "md":
        out = md_section(gcharm, torch, inputs.SEED_BASE + 3, stream, with_oracle=False,
                         cells=args.md_cells, ncell=args.md_ncell)
    else:
        out = uneven_plain(gcharm, torch, inputs.SEED_BASE + 4, stream)
    print(json.dumps({"section": args.section, **out}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-task", action="store_true")
    ap.add_argument("--n", type=int, default=N_PART)
    ap.add_argument("--no-md", action="store_true", help="skip the MD measurement")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the uneven-batch and serving measurements")
    ap.add_argument("--section", choices=["md", "uneven"],
                    help="run one workload alone and print its figures (profiling form)")
    ap.add_argument("--md-cells", type=int, default=64, help="FCC unit cells per axis")
    ap.add_argument("--md-ncell", type=int, default=42, help="MD cells per axis")
    ap.add_argument("--serve-seconds", type=float, default=SERVE_SECONDS,
                    help="measured seconds of arrivals per serving run")
    ap.add_argument("--serve-warmup", type=float, default=SERVE_WARMUP_S,
                    help="warm-up seconds of arrivals per serving run")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.section:
        run_section(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2008_05712_gb300 import gcharm

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gcharm.load()
    n = args.n
    K, W = args.steps, max(args.warmup, 3)
    seed = replica_seed(rank)

    # pre-generate all steps' positions (a drift walk), resident in HBM
    xs = [inputs.plummer(n, seed)]
    for k in range(K + W + 1):
        xs.append(inputs.drift(xs[-1], seed + 1 + k))
    X = torch.from_numpy(np.stack(xs[1:])).cuda()        # (K+W+1, n, 4)
    ids_np = np.arange(n, dtype=np.uint32)
    ids_d = torch.from_numpy(ids_np).cuda()
    stream = torch.cuda.Stream()
    id_cap = 2 * n + 1024
    pool = gcharm.Pool(id_capacity=id_cap, pool_capacity=id_cap, eps2=EPS2,
                       stream=stream.cuda_stream)
    pool.upload(ids_np, xs[0])
    torch.cuda.synchronize()

    def step(k):
        pool.upload_device(ids_d, X[k])
        pool.reset_totals()
        pool.build_nbody(X[k], BUCKET, *THETA)
        pool.flush()

    step(0)
    cold_misses = pool.stats()["last_misses"]     # first flush: every id fetched
    tuning, tune_ms = pool.autotune(reps=2, cache=TUNE_CACHE, key="nbody_plummer_1M"
                                    if n == N_PART else f"nbody_plummer_{n}")
    for k in range(1, W):
        step(k)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    s0 = pool.stats()
    nb0 = pool.nbody_stats()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(W, W + K):
        step(k)
    pool.join(stream.cuda_stream)          # the last batch may run on the other context
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    s1 = pool.stats()
    nb1 = pool.nbody_stats()
    interactions = s1["interactions"] - s0["interactions"]
    launches = s1["kernel_launches"] - s0["kernel_launches"]
    prims = s1["primitive_calls"] - s0["primitive_calls"]
    if ws > 1:
        ms, interactions_all = reduce_over_ranks(ms, interactions, "cuda")
    else:
        interactions_all = interactions
    value = interactions_all / (ms / 1e3)
    hits, uniq = s1["last_hits"], s1["last_unique"]

    # rooflines: per-stage device times of the timed flushes (CUDA events on
    # the flush streams, summed by the library), algorithmic work per step
    nb = s1["timed_batches"] - s0["timed_batches"]
    stage = {k: (s1["stage_ms_sum"][k] - s0["stage_ms_sum"][k]) / max(nb, 1)
             for k in s1["stage_ms_sum"]}
    per_step_int = interactions / K
    per_step_entries = (s1["entries"] - s0["entries"]) / K
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    fp32_measured = gcharm.fp32_peak()
    grav = {"kernel": "k_gravity (interaction)", "bound": "alu",
            "achieved": FLOPS_PER_INTERACTION * per_step_int / (stage["interact"] / 1e3) / 1e12,
            "peak": fp32_measured, "unit": "TFLOP/s",
            "peak_basis": "measured: paired-FP32 FMA probe (gc_fp32_peak); clock-derived "
                          f"{fp32_peak_tflops(sm_max):.1f} TFLOP/s = {SM_COUNT} SMs x "
                          f"{FP32_LANES} lanes x 2 x {sm_max:.0f} MHz",
            "work_per_unit": f"{FLOPS_PER_INTERACTION} flop per interaction",
            "units_per_launch": per_step_int, "ms_per_launch": stage["interact"],
            "traffic": (GRAVITY_DRAM_BYTES_PER_INTERACTION * per_step_int
                        if GRAVITY_DRAM_BYTES_PER_INTERACTION else None)}
    grav["frac"] = grav["achieved"] / grav["peak"]
    pack = {"kernel": "pack (k_pack_small, k_pack_mid<1024>, k_pack_mid<2048>, k_pack_large)",
            "bound": "hbm",
            "achieved": PACK_BYTES_PER_ENTRY * per_step_entries / (stage["pack"] / 1e3) / 1e9,
            "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s",
            "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                          if "hbm_gbs" in pk else "fallback 6800 GB/s",
            "work_per_unit": f"{PACK_BYTES_PER_ENTRY} B per list entry",
            "units_per_launch": per_step_entries, "ms_per_launch": stage["pack"],
            "traffic": (PACK_DRAM_BYTES_PER_ENTRY * per_step_entries
                        if PACK_DRAM_BYTES_PER_ENTRY else None)}
    pack["frac"] = pack["achieved"] / pack["peak"]
    scatter = {"kernel": "k_reduce_unique (scatter: one row per particle, no sort)",
               "bound": "hbm",
               "achieved": SCATTER_BYTES_PER_ROW * n / (stage["scatter"] / 1e3) / 1e9,
               "peak": pack["peak"], "unit": "GB/s", "peak_basis": pack["peak_basis"],
               "work_per_unit": f"{SCATTER_BYTES_PER_ROW} B per row (32 B partial, 4 B id, "
                                "32 B FP64 total read and written)",
               "units_per_launch": n, "ms_per_launch": stage["scatter"], "traffic": None}
    scatter["frac"] = scatter["achieved"] / scatter["peak"]
    dominant = pack if stage["pack"] >= stage["interact"] else grav

    # reuse ablation (Section 3.2, Fig. 3) on the last timed batch
    ablation = pool.reuse_ablation(reps=3)
    ablation["cold_reuse_fetch_bytes"] = cold_misses * 16
    ablation["note"] = ("kernel times: packed staging (this engine) vs sources read through "
                        "their pool slots in list order / sorted by slot; transfer: redundant "
                        "host-packed staging vs the misses the chare table fetched (first "
                        "step: every id; later steps: none)")

    # end-to-end through the C ABI with host buffers (pinned), copies timed
    pinned = torch.empty((K, n, 4), dtype=torch.float32, pin_memory=True)
    pinned.copy_(X[W:W + K].cpu())
    hx = pinned.numpy()
    ids_pin_t = torch.from_numpy(ids_np).pin_memory()
    tot_pin_t = torch.empty((2, n, 4), dtype=torch.float64, pin_memory=True)
    ids_pin, tot_pin = ids_pin_t.numpy(), tot_pin_t.numpy()
    torch.cuda.synchronize()
    # every step copies its inputs in and reads its totals out; the copies
    # are queued on the pool's two copy streams (pinned buffers, two
    # alternating result buffers) and the host waits once, at the end
    t0 = time.perf_counter()
    for k in range(K):
        pool.upload_async(ids_pin, hx[k])        # ids + values H2D
        pool.reset_totals()
        pool.build_nbody_resident(n, BUCKET, *THETA)   # tree from the pool's values
        pool.flush()
        pool.totals_async(ids_pin, tot_pin[k % 2])     # ids H2D, totals D2H
    pool.join(stream.cuda_stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    last_ok = bool(np.array_equal(tot_pin[(K - 1) % 2], pool.totals(ids_np))) if K else True
    e2e = {"value": interactions / K * K / e2e_s if K else 0.0, "unit": "interactions/s",
           "h2d_bytes_per_step": int(n * (4 + 16 + 4)),
           "d2h_bytes_per_step": int(tot_pin[0].nbytes),
           "copies": "queued each step (gc_pool_upload_async, gc_read_totals_async) on "
                     "the pool's host-to-device and device-to-host copy streams, in "
                     "order with its device work by events; one host wait at the end",
           "last_totals_equal_sync_read": last_ok}
    if ws > 1:
        e2e_max, _ = reduce_over_ranks(e2e_s, 0, "cuda")
        e2e["value"] = interactions_all / e2e_max

    # the same step with one interaction launch per task (no combining)
    per_task = None
    if not args.no_per_task:
        step_k = W + K
        pool.upload_device(ids_d, X[step_k])
        pool.reset_totals()
        pool.build_nbody(X[step_k], BUCKET, *THETA)
        i0 = pool.stats()["interactions"]
        pool.flush_per_task()
        torch.cuda.synchronize()
        tp = pool.timings()
        pn = pool.stats()["interactions"] - i0
        pool.upload_device(ids_d, X[step_k])
        pool.reset_totals()
        pool.build_nbody(X[step_k], BUCKET, *THETA)
        pool.flush()
        torch.cuda.synchronize()
        tb = pool.timings()
        per_task = {
            "interact_ms_per_task_launch": tp["interact"],
            "interact_ms_batched": tb["interact"],
            "interactions": pn,
            "value_per_task_launch": pn / (tp["interact"] / 1e3),
            "value_batched": pn / (tb["interact"] / 1e3),
            "speedup_interaction_stage": tp["interact"] / tb["interact"],
            "flush_ms_per_task_launch": tp["total"],
            "flush_ms_batched": tb["total"],
            "speedup_flush": tp["total"] / tb["total"],
        }

    # tree stage: the timed steps (Morton order seeded by the previous
    # step's), then the same drift steps with every build sorted from
    # scratch and seeded again, each measured step preceded by its
    # predecessor so that the seeded build starts from a one-step-old order
    nbt = max(nb1["timed_builds"] - nb0["timed_builds"], 1)
    tree = {"timed_steps": {
        "order": "seeded",
        "order_ms": (nb1["order_ms_sum"] - nb0["order_ms_sum"]) / nbt,
        "tree_ms": (nb1["tree_ms_sum"] - nb0["tree_ms_sum"]) / nbt,
        "seeded_builds": nb1["seeded_builds"] - nb0["seeded_builds"], "builds": nbt}}
    J = min(K, 8)
    for mode, name in ((gcharm.GC_ORDER_FULL, "full"), (gcharm.GC_ORDER_SEEDED, "seeded")):
        pool.set_order(mode)
        om, tm, rs = [], [], []
        for k in range(W, W + J):
            step(k - 1)
            step(k)
            st = pool.nbody_stats()
            om.append(st["last_order_ms"])
            tm.append(st["last_tree_ms"])
            rs.append(st["last_resorted"] / n)
        tree[name] = {"order_ms": float(np.median(om)), "tree_ms": float(np.median(tm)),
                      "resorted_frac": float(np.median(rs)), "steps": J}
    pool.set_order(gcharm.GC_ORDER_SEEDED)
    tree["note"] = ("order_ms: bounding box to sorted Morton order; tree_ms: the whole build "
                    "(order, nodes, monopoles, buckets, list walk, tasks), CUDA events on the "
                    "build stream including the build's own host read-backs; medians over "
                    f"{J} drift steps")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        keep = {}
        ci, ct, cn = oracle_sample(xs[W], 60000, 77, keep=keep)
        cpu = {"value": ci / ct, "unit": "interactions/s", "cores": 1, "kind": "oracle",
               "sample": f"{cn} seeded-random buckets of the first timed step "
                         f"({ci} interactions): oracle walk + FP64 gravity, one thread; "
                         "tree build untimed"}
        # parity of the same sample: the step on these positions through the
        # engine, rows of the sampled buckets against the oracle's FP64 rows
        pool.upload(ids_np, xs[W])
        pool.reset_totals()
        pool.build_nbody(xs[W], BUCKET, *THETA)
        pool.flush()
        counts = pool.nbody_bucket_counts(keep["n_buckets"])
        boff = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
        rows_gpu = pool.values()
        got = np.concatenate([rows_gpu[boff[b]:boff[b + 1]] for b in keep["buckets"]])
        cpu["parity_on_sample"] = error_stats(got, keep["rows"], keep["tgt_off"])
        cores = os.cpu_count() or 1
        if cores > 1:
            ai, at, an = oracle_all_cores(xs[W], cores)
            cpu["all_cores"] = {"value": ai / at, "unit": "interactions/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"all {an} buckets of the first timed step "
                                          f"({ai} interactions), one spawned process per "
                                          "core on interleaved buckets; tree build untimed"}

    md = None
    if rank == 0 and not args.no_md:
        md = md_section(gcharm, torch, inputs.SEED_BASE + 3, stream,
                        with_oracle=not args.no_cpu_baseline)
        md["rooflines"] = md_rooflines(md, fp32_measured, pack["peak"], pack["peak_basis"])
    c1 = None
    if rank == 0:
        c1 = c1_section(gcharm, torch, inputs.SEED_BASE + 1, stream,
                        with_oracle=not args.no_cpu_baseline)
    ewald = None
    if rank == 0 and not args.no_md:
        ewald = ewald_section(gcharm, torch, inputs.SEED_BASE + 8, stream,
                              with_oracle=not args.no_cpu_baseline)
    uneven = serving = None
    if rank == 0 and not args.no_serve:
        pool.close()
        del X
        torch.cuda.empty_cache()
        uneven, serving = uneven_and_serving(gcharm, torch, inputs.SEED_BASE + 4, stream,
                                             with_oracle=not args.no_cpu_baseline,
                                             serve_seconds=args.serve_seconds,
                                             serve_warmup=args.serve_warmup)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": ws,
            "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": n, "tasks_per_step": None,
                       "l2": "inputs larger than L2 (staging ~4 GB per step)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": dominant,
            "rooflines": {"interaction": grav, "pack": pack, "scatter": scatter},
            "stage_ms_avg": stage,
            "tree": tree,
            "tuning": {"wu_max_targets": tuning["wu_max_targets"],
                       "schedule": "lpt" if tuning["schedule"] else "fifo",
                       "tile_pairs": tuning["tile_pairs"],
                       "comp_block": tuning["comp_block"],
                       "targets_per_lane": tuning["targets_per_lane"],
                       "autotune_ms": tune_ms or tuning.get("times_ms"),
                       "cache": os.path.relpath(TUNE_CACHE, ROOT)},
            "reuse": {"last_hits": hits, "last_unique": uniq},
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "primitive_calls": prims,
            "per_task_launch": per_task,
            "reuse_ablation": ablation,
            "md": md,
            "c1_small": c1,
            "ewald": ewald,
            "uneven_batch": uneven,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        line["config"]["tasks_per_step"] = int(s1["tasks"] - s0["tasks"]) // max(K, 1)
        line["config"]["interactions_per_step"] = int(interactions) // max(K, 1)
        line["config"]["list_entries_per_step"] = int(s1["entries"] - s0["entries"]) // max(K, 1)
        print(json.dumps(line), flush=True)
    if pool.h:
        pool.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
