#!/usr/bin/env python3
"""Benchmark of the fused DPF EvalAll + dpXOR server path (IM-PIR §3, Algorithm 1) on one GB300.

Workload (default): the 8 GiB uneven batch workload: N = 2^25 records x 256 B (8 GiB,
uniform random bytes), 1024 queries split into batches of uniform random size 1..512 whose
keys mix domain sizes 2^23, 2^24 and 2^25 (each against the DB prefix it covers). One step
answers all 1024 queries (one server's keys), batch after batch, each batch one persistent
fused launch. The DB (8 GiB) is larger than L2 (129 MB), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `value` is device-timed queries/s with keys already in HBM; `e2e`
is the same metric through the synchronous C-ABI call with host buffers (key upload and
answer download inside the timed region). Under torchrun each rank answers its own copy of
the workload (independent batches: weak scaling, no data-path collective).
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

WORKLOADS = ("uneven8g", "batched4g", "batched256m", "single")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=WORKLOADS, default="uneven8g")
    p.add_argument("--queries", type=int, default=None, help="query count of the batched256m workload (default 64)")
    p.add_argument("--record-bytes", type=int, default=None,
                   help="record size of the batched4g workload (a power of two; N = 4 GiB / record size)")
    p.add_argument("--db-log2", type=int, default=None,
                   help="database of 2^k bytes for the uneven8g / batched4g workloads (same batches; small "
                        "profiling cases)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the one-query-per-launch comparison")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--config", default=None,
                   help="fixed launch shape lane_bits,queries_per_warp,warps_per_cta (skips autotuning)")
    p.add_argument("--cpu-sample", type=int, default=6,
                   help="queries in the oracle's timed sample (the workload's domain sizes in turn)")
    p.add_argument("--no-serving", action="store_true", help="skip the serving sweep (three resident DBs)")
    p.add_argument("--no-streamed", action="store_true", help="skip the host-streamed database measurement")
    p.add_argument("--no-shards", action="store_true", help="skip the row-shard measurement")
    p.add_argument("--serving-requests", type=int, default=2000, help="requests per arrival rate")
    p.add_argument("--calibrate-only", action="store_true",
                   help="time the AES engines alone (calibration kernel, both PRFs) and exit")
    return p.parse_args()


def make_workload(name, queries=None, record_bytes=None, db_log2=None):
    """The named workload; db_log2 shrinks the uneven or 4 GiB workload's database to 2^db_log2
    bytes with the same batches (profiling captures of a small case)."""
    from paper_2509_06514_gb300 import workloads as W
    if name == "batched256m" and queries:
        return W.batched_256mib(n_queries=queries)
    if name == "batched4g" and (record_bytes or db_log2):
        return W.batched_4gib(record_bytes=record_bytes or 1024, db_bytes=1 << (db_log2 or 32))
    if name == "uneven8g" and db_log2:
        return W.uneven_8gib(log2n=db_log2 - 8)
    return {"uneven8g": W.uneven_8gib, "batched4g": W.batched_4gib, "batched256m": W.batched_256mib,
            "single": W.single_query}[name]()


# ---------------------------------------------------------------- distributed plumbing

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks during the timed region

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = max((num(r[2]) or 0) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0) for r in rows)}


# ---------------------------------------------------------------- algorithmic work

def aes_blocks(m: int) -> int:
    """AES-128 encryptions of one full-domain evaluation: 2 (2^m - 1) (one per tree edge)."""
    return 2 * ((1 << m) - 1)


def kernel_source_hash() -> str:
    """sha256 of the fused kernel's device code (a traffic capture is valid only for it): the
    sources with comments removed and whitespace collapsed, so that editing a comment keeps it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("fused.cuh", "bounds.cuh", "impir_internal.h", "fused_q1.cu", "fused_q2.cu", "fused_q4.cu", "fused_q8.cu",
              "fused_q16.cu", "setup.cu"):
        with open(os.path.join(ROOT, "paper_2509_06514_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def captured_traffic(cfg: dict, batches: list):
    """DRAM bytes per fused launch of this step, from the committed ncu capture of the same
    batches on a smaller database (1 GiB; the full-size workload is too large to capture with
    more than the launch-time metric): each batch's measured DRAM bytes per byte of the DB prefix
    its queries cover, times that prefix here, averaged over the step's launches. Valid only for
    the kernel source and launch shape the capture was taken with; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "fused_kernel_traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    if t.get("kernel_source_sha256") != kernel_source_hash() or t.get("launch") != cfg:
        return None
    per = t.get("per_batch", [])
    if [b["queries"] for b in per] != [bt["n"] for bt in batches]:
        return None
    total = 0.0
    for b, bt in zip(per, batches):
        ratio = (b["dram_read_bytes"] + b["dram_write_bytes"]) / b["db_prefix_bytes"]
        total += ratio * bt["prefix_bytes"]
    return total / len(per)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Shared-memory table lookups the fused kernel's keyed T-table engine executes per tree
# expansion (two AES blocks, both children of a node): an internal node pair costs 345 (key
# schedule 40, round 1 of both children 17, rounds 2-9 256, final rounds 32), a pair at the
# leaf level 288 (key schedule 36, round 1 17, rounds 2-8 224, column 0 of round 9 8, the
# three S-box lookups the selection bits need 3). A domain of 2^m leaves has 2^(m-1) leaf-level
# pairs and 2^(m-1) - 1 internal ones: 158.25 lookups per AES block on average.
LOOKUPS_INTERNAL_PAIR = 345
LOOKUPS_LEAF_PAIR = 288
# the additive answer's leaf-level pair: the low 32 bits of both leaves (key schedule 36, round 1
# 17, rounds 2-9 256, column 0 of round 10 and its round-key word 12)
LOOKUPS_LEAF_PAIR_ADD = 321
SMEM_LOOKUPS_PER_CLK_PER_SM = 32   # one 32-bit word per bank per clock, 32 banks


def lookups_per_query(m: int, leaf_pair: int = LOOKUPS_LEAF_PAIR) -> int:
    half = 1 << (m - 1)
    return leaf_pair * half + LOOKUPS_INTERNAL_PAIR * (half - 1)


def smem_peak_gaes(sms: int, mhz: float, lookups_per_block: float) -> float:
    """AES blocks per second the shared-memory port allows at the kernel's lookups per block."""
    return sms * mhz * 1e6 * SMEM_LOOKUPS_PER_CLK_PER_SM / lookups_per_block / 1e9


def alu_counts():
    """ALU-pipe instruction counts measured by ncu (committed summary, see profiles/): thread
    instructions per AES block of the isolated keyed engine and the ALU pipe's peak lanes per
    SM per clock; None when the summary is absent."""
    try:
        with open(os.path.join(ROOT, "profiles", "alu_pipe_counts.json")) as f:
            return json.load(f)
    except OSError:
        return None


# ---------------------------------------------------------------- reference arm: the CPU oracle

def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2509_06514_gb300 import workloads
    oracle.build()
    w = make_workload(args.workload, args.queries, args.record_bytes, args.db_log2)
    cores = os.cpu_count() or 1
    # one query per step, the workload's domain sizes taken in turn (so that a short run costs
    # what the workload's mix costs), records regenerated once
    db = workloads.make_db(w.n_records, w.record_bytes, w.db_seed)
    by_m = {}
    for b in w.batches:
        for m, a, s in zip(b.ms, b.alphas, b.seeds):
            by_m.setdefault(m, []).append((m, a, s))
    order = sorted(by_m)
    qs = [q for row in zip(*(by_m[m] for m in order)) for q in row]
    times = []
    for i in range(args.warmup + args.steps):
        m, a, s = qs[i % len(qs)]
        k0, _ = oracle.gen(a, m, oracle.PRF_KEYED, s)
        t0 = time.perf_counter()
        oracle.answer(k0, db, w.n_records, w.record_bytes, threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    v = args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": "PIR queries/s (DPF eval+dpXOR) at 8 GiB DB", "value": v,
        "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded uniform random records)",
        "config": {"workload": w.name, "step": "one query of the workload per step (bounded sample)"},
        "cpu_baseline": {"value": v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} queries of the workload, one per step, domain sizes in turn "
                                   f"(m = {[qs[i % len(qs)][0] for i in range(args.warmup, args.warmup + args.steps)]}), "
                                   f"threaded oracle"},
        "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- serving sweep

def run_serving(args, impir, workloads):
    """Three resident DBs, Poisson arrivals at each rate, uniform DB and target; continuous
    batching by the library's server. Returns per-rate throughput and p50/p99 latency."""
    import threading
    dbs = []
    for i, (n, b) in enumerate(workloads.SERVING_DBS):
        db = workloads.make_db(n, b, seed=900 + i)
        dbs.append((impir.impir_db_load(db, n, b), db, n, b))
    server = impir.impir_server_create(max_batch=256, streams=4, max_record_bytes=512,
                                       accumulator_budget=4 * 256 * 512)
    points = []
    try:
        sweep = [(r, False) for r in workloads.SERVING_LOW_RATES + workloads.SERVING_RATES] + [(20_000, True)]
        for rate, with_updates in sweep:
            n_req = args.serving_requests if rate >= 5000 else max(100, int(rate * 0.4))
            arr = workloads.poisson_arrivals(rate, n_req, dbs=workloads.SERVING_DBS)
            keys = []
            for i in range(len(arr.t)):
                d = int(arr.db[i])
                m = dbs[d][2].bit_length() - 1
                keys.append(impir.dpf_gen(int(arr.alpha[i]), m, impir.IMPIR_PRF_AES_KEYED, arr.seeds[i])[0])
            done = {}
            before = impir.impir_server_stats(server)
            t_sub = [0.0] * len(keys)

            def client():
                t0 = time.perf_counter()
                for i, k in enumerate(keys):
                    due = float(arr.t[i])
                    while True:
                        left = due - (time.perf_counter() - t0)
                        if left <= 0:
                            break
                        if left > 2e-4:
                            time.sleep(left - 1e-4)
                    t_sub[i] = time.perf_counter()
                    impir.impir_server_submit(server, dbs[int(arr.db[i])][0], k, i)

            th = threading.Thread(target=client)
            upd = {"count": 0, "bytes": 0}

            def updater():
                # bulk updates of 16 MiB into the largest DB while requests are served
                urng = np.random.default_rng(rate)
                h, _, n, b = dbs[-1]
                rec = urng.integers(0, 256, ((16 << 20) // b, b), dtype=np.uint8)
                for _ in range(8):
                    time.sleep(float(arr.t[-1]) / 9)
                    impir.impir_server_update(server, h, int(urng.integers(0, n - rec.shape[0])), rec)
                    upd["count"] += 1
                    upd["bytes"] += rec.nbytes

            tu = threading.Thread(target=updater) if with_updates else None
            t_start = time.perf_counter()
            th.start()
            if tu:
                tu.start()
            while len(done) < len(keys):
                r = impir.impir_server_take(server, 2_000_000)
                if r is None:
                    break
                done[r["tag"]] = (r, time.perf_counter())
            th.join()
            if tu:
                tu.join()
            t_end = max(t for _, t in done.values())
            after = impir.impir_server_stats(server)
            lat = np.array([r["latency_ns"] for r, _ in done.values()]) / 1e6
            bad = checked = 0
            # with updates interleaved the answers span several DB versions (the version
            # check is the updates test's job); without, compare a sample with answers alone
            for i in range(0, len(keys), max(1, len(keys) // 24)) if not with_updates else ():
                checked += 1
                h, _, _, b = dbs[int(arr.db[i])]
                bad += int(done[i][0]["answer"] != impir.impir_answer(h, keys[i], 1, b)[0].tobytes())
            points.append({
                "offered_req_s": rate, "requests": len(keys), "completed": len(done),
                "bulk_updates": upd if with_updates else None,
                "submit_rate_req_s": len(keys) / max(1e-9, t_sub[-1] - t_sub[0]),
                "queries_per_s": len(done) / (t_end - t_start),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_batch": (after["queries"] - before["queries"]) / max(1, after["batches"] - before["batches"]),
                "max_inflight_batches": after["max_inflight_batches"],
                "sampled_vs_alone": {"checked": checked, "mismatches": bad},
            })
    finally:
        impir.impir_server_destroy(server)
        for h, *_ in dbs:
            impir.impir_db_free(h)
    return {"dbs": [f"2^{n.bit_length() - 1} x {b} B" for n, b in workloads.SERVING_DBS],
            "server": {"max_batch": 256, "streams": 4, "accumulator_budget": 4 * 256 * 512},
            "points": points}


# ---------------------------------------------------------------- AES engine calibration

def calibrate_engines(impir, iters: int = 2000):
    """The AES engines alone (no tree walk, no scan), each thread iterating node expansions
    (two AES blocks each) in registers: the fused kernel's T-table engine with one CTA of 512
    threads per SM, both PRFs, and the bitsliced engine (fixed-key PRF only) with 256 threads of
    16 seeds each per SM. G AES blocks per second of device time."""
    sms = impir.impir_device_sm_count()
    n = sms * 512
    seeds = np.random.default_rng(7).integers(0, 256, (n, 16), dtype=np.uint8)
    out = {}
    for prf, name in ((impir.IMPIR_PRF_AES_KEYED, "ttable_keyed"), (impir.IMPIR_PRF_AES_MMO, "ttable_mmo")):
        _, ms = impir.impir_aes_calibrate(prf, iters, seeds, 512)
        out[name] = {"gaes_per_s": 2 * iters * n / (ms / 1e3) / 1e9, "ms": ms, "blocks": 2 * iters * n}
    nb = sms * 256
    bseeds = np.random.default_rng(8).integers(0, 256, (nb * 16, 16), dtype=np.uint8)
    biters = max(1, iters // 16)
    _, ms = impir.impir_aes_calibrate_bitsliced(biters, bseeds, 256)
    out["bitsliced_mmo"] = {"gaes_per_s": 2 * biters * 16 * nb / (ms / 1e3) / 1e9, "ms": ms,
                            "blocks": 2 * biters * 16 * nb}
    return out


# ---------------------------------------------------------------- our arm

def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_2509_06514_gb300 as impir
    from paper_2509_06514_gb300 import build, workloads

    torch.cuda.set_device(local)
    # one rank builds (the ranks share the source tree and its object files); the others find
    # the library up to date after the barrier
    if rank == 0:
        build.build()
    barrier(world)
    build.build()
    if args.calibrate_only:
        print(json.dumps({"calibration": calibrate_engines(impir)}), flush=True)
        return
    w = make_workload(args.workload, args.queries, args.record_bytes, args.db_log2)
    N, B = w.n_records, w.record_bytes
    t_setup = time.perf_counter()
    db = workloads.make_db(N, B, w.db_seed)
    dbh = impir.impir_db_load(db, N, B)
    stride = impir.impir_db_info(dbh)["stride_bytes"]
    sms = impir.impir_device_sm_count()

    # keys of both servers for every query (client side, outside any timed region)
    batches = []
    for b in w.batches:
        k0s, k1s = [], []
        for m, a, s in zip(b.ms, b.alphas, b.seeds):
            k0, k1 = impir.dpf_gen(a, m, impir.IMPIR_PRF_AES_KEYED, s)
            k0s.append(k0)
            k1s.append(k1)
        n = len(k0s)
        blob0, offs = impir.pack_keys(k0s)
        blob1, _ = impir.pack_keys(k1s)
        wsb = impir.impir_workspace_bytes(n, stride)
        batches.append({
            "n": n, "ms": list(b.ms), "alphas": list(b.alphas), "blob0": blob0, "blob1": blob1,
            "prefix_bytes": max(min(N, 1 << m) for m in b.ms) * stride,
            "d_keys0": torch.from_numpy(np.frombuffer(blob0, np.uint8).copy()).cuda(),
            "d_keys1": torch.from_numpy(np.frombuffer(blob1, np.uint8).copy()).cuda(),
            "d_off": torch.from_numpy(offs.view(np.int32).copy()).cuda(),
            "d_out": torch.zeros((n, B), dtype=torch.uint8, device="cuda"),
            "d_ws": torch.empty(wsb, dtype=torch.uint8, device="cuda"), "wsb": wsb,
        })
    nq = sum(bt["n"] for bt in batches)
    stream = torch.cuda.Stream()

    def run_step(server=0):
        for bt in batches:
            impir.impir_answer_async(dbh, bt["d_keys%d" % server], bt["d_off"], bt["n"], bt["d_out"], bt["d_ws"],
                                     bt["wsb"], stream)

    # autotune on the largest batch (outside the timed region)
    tuned = None
    if args.config:
        lb, qpw, wpc = (int(x) for x in args.config.split(","))
        impir.impir_set_config(dbh, lb, qpw, wpc, 0)
    elif not args.no_tune:
        big = max(batches, key=lambda bt: bt["n"])
        tuned = impir.impir_autotune(dbh, big["d_keys0"], big["d_off"], big["n"], big["d_out"], big["d_ws"],
                                     big["wsb"], stream).as_dict()
    cfg = impir.impir_get_config(dbh, max(bt["n"] for bt in batches)).as_dict()

    # parity on the GPU answers of this run: both servers, reconstruction of every query
    run_step(1)
    stream.synchronize()
    ans1 = [bt["d_out"].cpu().numpy().copy() for bt in batches]
    run_step(0)
    stream.synchronize()
    ans0 = [bt["d_out"].cpu().numpy().copy() for bt in batches]
    bad = 0
    for bt, a0, a1 in zip(batches, ans0, ans1):
        for i, (m, a) in enumerate(zip(bt["ms"], bt["alphas"])):
            want = db[a] if a < N else np.zeros(B, np.uint8)
            bad += int(not np.array_equal(a0[i] ^ a1[i], want))
    setup_s = time.perf_counter() - t_setup

    for _ in range(args.warmup):
        run_step()
    stream.synchronize()

    # ---- device-timed region: keys resident in HBM ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    impir.impir_timing_enable(True)
    with Clocks(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            run_step()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier(world)
    fused_ms, fused_launches, all_launches = impir.impir_timing_read()
    impir.impir_timing_enable(False)
    ms = max_over_ranks(world, e0.elapsed_time(e1))
    clocks = clk.summary()
    value = nq * args.steps * world / (ms / 1e3)

    # ---- the same step replayed from a captured CUDA graph (all 3 x batches launches) ----
    graph = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            run_step()
        with torch.cuda.stream(stream):          # replay() launches on the current stream
            g.replay()
            stream.synchronize()
            same = all(np.array_equal(bt["d_out"].cpu().numpy(), a) for bt, a in zip(batches, ans0))
            gs, ge = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gs.record(stream)
            for _ in range(args.steps):
                g.replay()
            ge.record(stream)
            ge.synchronize()
        torch.cuda.synchronize()
        graph = {"value": nq * args.steps / (gs.elapsed_time(ge) / 1e3), "unit": "queries/s",
                 "bit_identical": same}
        del g
    except Exception as e:  # capture needs the library's launches only; report why if it fails
        torch.cuda.synchronize()
        graph = {"error": str(e)[:200]}

    # ---- e2e: the synchronous C-ABI call with host buffers (H2D keys, D2H answers inside) ----
    h2d = sum(len(bt["blob0"]) + 4 * bt["n"] for bt in batches)
    d2h = nq * B
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for bt in batches:
            impir.impir_answer(dbh, bt["blob0"], bt["n"], B)
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": nq * args.steps * world / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    # ---- plain form: one query per launch on the same queries ----
    plain = None
    if not args.no_plain:
        impir.impir_set_config(dbh, cfg["lane_bits"], 1, cfg["warps_per_cta"], 1)
        pc = impir.impir_get_config(dbh, 1).as_dict()
        run_step()
        stream.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        run_step()
        p1.record(stream)
        p1.synchronize()
        pms = p0.elapsed_time(p1)
        same = all(np.array_equal(bt["d_out"].cpu().numpy(), a) for bt, a in zip(batches, ans0))
        plain = {"value": nq / (pms / 1e3), "unit": "queries/s", "config": pc, "bit_identical_to_batched": same}
        impir.impir_set_config(dbh, cfg["lane_bits"], cfg["queries_per_warp"], cfg["warps_per_cta"], 0)

    # ---- roofline of the dominant kernel (fused EvalAll + dpXOR) ----
    pk, pk_kind = peaks()
    mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    blocks_per_step = sum(aes_blocks(m) for bt in batches for m in bt["ms"])
    lookups_per_step = sum(lookups_per_query(m) for bt in batches for m in bt["ms"])
    lookups_per_block = lookups_per_step / blocks_per_step
    launch_ms = fused_ms / max(1, fused_launches)
    achieved = blocks_per_step * args.steps / (fused_ms / 1e3) / 1e9 if fused_ms else None
    peak = smem_peak_gaes(sms, mhz, lookups_per_block)
    scan_bytes = sum(min(N, 1 << m) * B for bt in batches for m in bt["ms"])
    # the integer-ALU form of the same bound: AES blocks x the engine's ALU-pipe instructions
    # per block (ncu, isolated engine, scaled from its internal-node pairs to the kernel's mix
    # of internal and leaf pairs by lookups) + one 32-bit mask-and-XOR per record word and query
    # of the scan, over the ALU pipe's lanes x SMs x clock
    alu = None
    ac = alu_counts()
    if ac and fused_ms:
        xor_ops = sum(min(N, 1 << m) * (stride // 4) for bt in batches for m in bt["ms"])
        per_block = ac["engine_alu_thread_inst_per_block"] * lookups_per_block / ac["engine_lookups_per_block"]
        ops = blocks_per_step * per_block + xor_ops
        alu_peak = sms * ac["alu_lanes_per_sm_per_clk"] * mhz * 1e6
        alu = {"bound": "alu", "achieved": ops * args.steps / (fused_ms / 1e3) / 1e12, "peak": alu_peak / 1e12,
               "unit": "T int-ops/s", "frac": ops * args.steps / alu_peak / (fused_ms / 1e3),
               "ops_per_step": ops, "aes_ops_per_block": per_block, "scan_xor_ops_per_step": xor_ops,
               "basis": f"{sms} SMs x {ac['alu_lanes_per_sm_per_clk']} ALU lanes/clk x {mhz:.0f} MHz; "
                        f"engine {ac['engine_alu_thread_inst_per_block']:.1f} ALU ops per block "
                        f"({ac['source']})"}

    # AES engines alone (no tree walk / scan): the ceiling the fused kernel approaches, and the
    # bitsliced alternative; the T-table engine's lookup rate shows how close it runs to the port
    cal = calibrate_engines(impir)
    engine_gaes = cal["ttable_keyed"]["gaes_per_s"]
    engine = {"gaes_per_s": engine_gaes,
              "lookups_per_clk_per_sm": engine_gaes * 1e9 * LOOKUPS_INTERNAL_PAIR / 2 / (sms * mhz * 1e6),
              "fused_over_engine": (achieved / engine_gaes) if achieved else None,
              "engines": {k: v["gaes_per_s"] for k, v in cal.items()},
              "note": "keyed T-table node expansions in registers, 172.5 table lookups per block (round 1 "
                      "shared); bitsliced engine: fixed-key PRF, 154-gate S-box circuit, no lookups"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        # the sample takes the workload's domain sizes in turn (first unused query of each),
        # so that its cost per query matches the workload's mix
        by_m = {}
        for bi, bt in enumerate(batches):
            for i, m in enumerate(bt["ms"]):
                by_m.setdefault(m, []).append((bi, i))
        order = sorted(by_m)
        qs = [by_m[order[j % len(order)]][j // len(order)] for j in range(args.cpu_sample)
              if j // len(order) < len(by_m[order[j % len(order)]])]
        t0 = time.perf_counter()
        agree = True
        for bi, i in qs:
            bt = batches[bi]
            o = sum(impir.impir_key_bytes(m) for m in bt["ms"][:i])
            key = bt["blob0"][o:o + impir.impir_key_bytes(bt["ms"][i])]
            r = oracle.answer(key, db, N, B, threads=cores)
            agree &= r == ans0[bi][i].tobytes()
        dt = time.perf_counter() - t0
        cpu = {"value": len(qs) / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(qs)} queries of the workload (m={[batches[b]['ms'][i] for b, i in qs]}), "
                         f"threaded oracle, {dt:.1f} s", "bit_identical_to_gpu": bool(agree)}

    # database streamed from host memory (the larger-than-HBM path): the largest batch against
    # the 8 GiB DB in the library's default 2 GiB chunks from pinned host memory, vs the same
    # batch resident
    streamed = None
    if rank == 0 and not args.no_streamed:
        big = max(batches, key=lambda bt: bt["n"])
        # a pinned (page-locked) host copy of the DB: copies then run at link speed
        pinned = torch.empty(N * B, dtype=torch.uint8, pin_memory=True)
        pinned.copy_(torch.from_numpy(db.reshape(-1)))
        tr = []
        for _ in range(3):
            t0 = time.perf_counter()
            res = impir.impir_answer(dbh, big["blob0"], big["n"], B)
            tr.append(time.perf_counter() - t0)
        t_res = statistics.median(tr)
        # the first call allocates the staging buffers (kept for later calls); the second is
        # the steady state of repeated calls
        t0 = time.perf_counter()
        got, scfg = impir.impir_answer_streamed(pinned.data_ptr(), N, B, big["blob0"], big["n"], 0)
        t_first = time.perf_counter() - t0
        warm = []
        for _ in range(3):  # call-to-call spread is a few per cent: report the median
            t0 = time.perf_counter()
            got2, _ = impir.impir_answer_streamed(pinned.data_ptr(), N, B, big["blob0"], big["n"], 0)
            warm.append(time.perf_counter() - t0)
        t_str = statistics.median(warm)
        dev_buf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
        dev_buf.copy_(pinned[: 1 << 30], non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(4):
            dev_buf.copy_(pinned[: 1 << 30], non_blocking=True)
        torch.cuda.synchronize()
        link = 4 * (1 << 30) / (time.perf_counter() - t0) / 1e9
        del dev_buf, pinned
        streamed = {"queries": big["n"], "db_bytes": N * B, "chunk_bytes": 2 << 30, "host_memory": "pinned",
                    "resident_queries_per_s": big["n"] / t_res, "streamed_queries_per_s": big["n"] / t_str,
                    "streamed_over_resident": t_res / t_str, "first_call_queries_per_s": big["n"] / t_first,
                    "warm_calls_queries_per_s": [big["n"] / t for t in warm],
                    "h2d_link_gb_per_s": link, "db_stream_gb_per_s": N * B / t_str / 1e9,
                    "bit_identical": bool(np.array_equal(got, res) and np.array_equal(got2, res)),
                    "launch": scfg}

    # additive (inner-product, Z_2^32) answer on 64 queries of the workload, vs the XOR answer
    additive = None
    if rank == 0:
        sub = [(bt, i) for bt in batches for i in range(bt["n"])][:64]
        k0s, k1s, al = [], [], []
        for bt, i in sub:
            o = sum(impir.impir_key_bytes(m) for m in bt["ms"][:i])
            kb = impir.impir_key_bytes(bt["ms"][i])
            k0s.append(bt["blob0"][o:o + kb])
            k1s.append(bt["blob1"][o:o + kb])
            al.append(bt["alphas"][i])
        b0, b1 = b"".join(k0s), b"".join(k1s)
        impir.impir_answer_add32(dbh, b0, len(sub), B)            # warm
        impir.impir_answer(dbh, b0, len(sub), B)
        ta, tx = [], []
        for _ in range(3):     # medians of three synchronous calls each
            t0 = time.perf_counter()
            a0 = impir.impir_answer_add32(dbh, b0, len(sub), B)
            ta.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            impir.impir_answer(dbh, b0, len(sub), B)
            tx.append(time.perf_counter() - t0)
        t_add, t_xor = statistics.median(ta), statistics.median(tx)
        a1 = impir.impir_answer_add32(dbh, b1, len(sub), B)
        s32 = (a0.view("<u4").astype(np.uint64) + a1.view("<u4").astype(np.uint64)) % (1 << 32)
        rec = s32.astype("<u4").view(np.uint8).reshape(len(sub), B)
        ok = sum(int(np.array_equal(rec[i], db[a])) for i, a in enumerate(al))
        add_blocks = sum(aes_blocks(bt["ms"][i]) for bt, i in sub)
        add_lookups = sum(lookups_per_query(bt["ms"][i], LOOKUPS_LEAF_PAIR_ADD) for bt, i in sub)
        add_peak = smem_peak_gaes(sms, mhz, add_lookups / add_blocks)
        additive = {"queries": len(sub), "add32_queries_per_s": len(sub) / t_add, "xor_queries_per_s": len(sub) / t_xor,
                    "reconstructed_ok": ok, "launch": impir.impir_get_config_add32(dbh, len(sub)).as_dict(),
                    # same AES work as the XOR answer (one block per tree edge), wall time of one call
                    "aes_gaes_per_s": add_blocks / t_add / 1e9,
                    "frac_of_peak": add_blocks / t_add / 1e9 / add_peak,
                    "peak_basis": f"{add_lookups / add_blocks:.2f} lookups per AES block (leaf-level pairs "
                                  f"{LOOKUPS_LEAF_PAIR_ADD})"}

    # the fixed-key PRF variant (Matyas-Meyer-Oseas with two fixed AES keys: no key schedule
    # per node, but no round shared between the two children) on the largest batch, against the
    # same batch with the keyed PRF; both answers reconstruct their records
    mmo = None
    if rank == 0:
        big = max(batches, key=lambda bt: bt["n"])
        wb = next(b for b in w.batches if len(b.ms) == big["n"])
        pairs = [impir.dpf_gen(a, m, impir.IMPIR_PRF_AES_MMO, sd) for m, a, sd in zip(wb.ms, wb.alphas, wb.seeds)]
        mblob0, _ = impir.pack_keys([p[0] for p in pairs])
        mblob1, _ = impir.pack_keys([p[1] for p in pairs])
        impir.impir_answer(dbh, mblob0, big["n"], B)
        tm, tk = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            m0 = impir.impir_answer(dbh, mblob0, big["n"], B)
            tm.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            impir.impir_answer(dbh, big["blob0"], big["n"], B)
            tk.append(time.perf_counter() - t0)
        m1 = impir.impir_answer(dbh, mblob1, big["n"], B)
        mmo = {"queries": big["n"], "mmo_queries_per_s": big["n"] / statistics.median(tm),
               "keyed_queries_per_s": big["n"] / statistics.median(tk),
               "mmo_over_keyed": statistics.median(tk) / statistics.median(tm),
               "reconstructed_ok": int(sum(np.array_equal(m0[i] ^ m1[i], db[a]) for i, a in enumerate(big["alphas"])))}

    # row shards (the multi-GPU split of one database, timed here on one GPU): the largest batch
    # answered on two row-shard handles of the DB, partial answers combined on the device, against
    # the whole DB; with one shard per GPU the step would take the slower shard plus the exchange
    row_shards = None
    if rank == 0 and not args.no_shards:
        from paper_2509_06514_gb300.sharding import combine, domain_weights, shard_rows
        big = max(batches, key=lambda bt: bt["n"])
        # split at half the batch's work (its domains cover DB prefixes), not half the rows
        blocks = shard_rows(N, 2, weights=domain_weights(N, big["ms"]))
        hs = [impir.impir_db_load_rows(db[lo:lo + n], n, B, lo, N) for lo, n in blocks]
        try:
            for hh in hs:
                impir.impir_set_config(hh, **{k: cfg[k] for k in ("lane_bits", "queries_per_warp", "warps_per_cta")})
            nb, d_keys, d_off, d_ws, wsb = big["n"], big["d_keys0"], big["d_off"], big["d_ws"], big["wsb"]
            parts = torch.zeros((2, nb, B), dtype=torch.uint8, device="cuda")
            whole = torch.zeros((nb, B), dtype=torch.uint8, device="cuda")
            st = torch.cuda.Stream()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            times = {"whole": [], "shard0": [], "shard1": [], "combine": []}
            with torch.cuda.stream(st):
                for rep in range(3):
                    ev[0].record(st)
                    impir.impir_answer_async(dbh, d_keys, d_off, nb, whole, d_ws, wsb, st)
                    ev[1].record(st)
                    impir.impir_answer_async(hs[0], d_keys, d_off, nb, parts[0], d_ws, wsb, st)
                    ev[2].record(st)
                    impir.impir_answer_async(hs[1], d_keys, d_off, nb, parts[1], d_ws, wsb, st)
                    ev[3].record(st)
                    out = combine(parts, 0, st)
                    ev[4].record(st)
                    st.synchronize()
                    for name, a, b in (("whole", 0, 1), ("shard0", 1, 2), ("shard1", 2, 3), ("combine", 3, 4)):
                        times[name].append(ev[a].elapsed_time(ev[b]))
            med = {k: statistics.median(v) for k, v in times.items()}
            row_shards = {"queries": nb, "shards": [{"row_lo": lo, "rows": n} for lo, n in blocks],
                          "ms": med, "bit_identical": bool(torch.equal(out, whole)),
                          "shards_sum_over_whole": (med["shard0"] + med["shard1"]) / med["whole"],
                          "two_gpu_projection_queries_per_s": nb / ((max(med["shard0"], med["shard1"]) + med["combine"]) / 1e3),
                          "note": "one GPU; the projection leaves out the all-gather of 2 x Q x B bytes"}
            del parts, whole
        finally:
            for hh in hs:
                impir.impir_db_free(hh)

    # latency of one query through the synchronous call (host key in, answer out) on the
    # single-query workload: N = 2^16 x 32 B (2 MiB), m = 16, both servers' keys
    single = None
    if rank == 0:
        sw = workloads.single_query()
        sdb = workloads.make_db(sw.n_records, sw.record_bytes, sw.db_seed)
        sh = impir.impir_db_load(sdb, sw.n_records, sw.record_bytes)
        try:
            b = sw.batches[0]
            k0, k1 = impir.dpf_gen(b.alphas[0], b.ms[0], 0, b.seeds[0])
            for _ in range(5):
                impir.impir_answer(sh, k0, 1, sw.record_bytes)
            lat = []
            for i in range(100):
                t0 = time.perf_counter()
                r = impir.impir_answer(sh, k0 if i % 2 == 0 else k1, 1, sw.record_bytes)
                lat.append(time.perf_counter() - t0)
            r0 = impir.impir_answer(sh, k0, 1, sw.record_bytes)
            r1 = impir.impir_answer(sh, k1, 1, sw.record_bytes)
            single = {"workload": sw.name, "median_us": statistics.median(lat) * 1e6,
                      "p99_us": sorted(lat)[98] * 1e6, "calls": len(lat),
                      "reconstructed": bool(np.array_equal(r0[0] ^ r1[0], sdb[b.alphas[0]]))}
        finally:
            impir.impir_db_free(sh)

    # bulk update bandwidth: 256 MiB of new records into the resident DB (synchronous call)
    upd_n = min((256 << 20) // B, N // 2)
    upd_rec = np.random.default_rng(11).integers(0, 256, (upd_n, B), dtype=np.uint8)
    t0 = time.perf_counter()
    impir.impir_db_update(dbh, N - upd_n, upd_rec)
    upd_s = time.perf_counter() - t0
    db_update = {"bytes": int(upd_rec.nbytes), "seconds": upd_s, "gb_per_s": upd_rec.nbytes / upd_s / 1e9,
                 "version": impir.impir_db_version(dbh)}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(args, impir, workloads)

    if rank == 0:
        traffic = captured_traffic(cfg, batches)
        out = {
            "metric": "PIR queries/s (DPF eval+dpXOR) at 8 GiB DB", "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded uniform random records; keys from the library's Gen)",
            "config": {"workload": w.name, "queries_per_step": nq, "batches": [bt["n"] for bt in batches],
                       "db_bytes": N * B, "record_bytes": B, "l2": "DB (8 GiB) larger than L2, no flush",
                       "prf": "AES-128 keyed by the node seed (paper's PRF)", "launch": cfg, "tuned": tuned},
            "e2e": e2e,
            "gpu_launches": all_launches,
            "clocks": clocks,
            "roofline": {"bound": "smem_port", "achieved": achieved, "peak": peak, "unit": "GAES/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic,
                         "peak_basis": f"{sms} SMs x {mhz:.0f} MHz x {SMEM_LOOKUPS_PER_CLK_PER_SM} table lookups/clk"
                                       f" / {lookups_per_block:.2f} lookups per AES block (the kernel's code: "
                                       f"{LOOKUPS_INTERNAL_PAIR} per internal node pair, {LOOKUPS_LEAF_PAIR} per "
                                       f"leaf-level pair)",
                         "kernel": "fused_kernel", "avg_launch_ms": launch_ms, "launches": fused_launches},
            "roofline_alu": alu,
            "scan": {"logical_gbs": scan_bytes * args.steps / (ms / 1e3) / 1e9,
                     # DRAM bytes of one fused launch (ncu capture) over its live duration
                     "physical_gbs": (traffic / (launch_ms / 1e3) / 1e9) if traffic and launch_ms else None,
                     "hbm_peak_gbs": pk.get("hbm_gbs"), "peak_kind": pk_kind},
            "aes_blocks_per_s": blocks_per_step * args.steps / (ms / 1e3),
            "aes_engine": engine,
            "one_query_per_launch": plain,
            "graph_replay": graph,
            "parity": {"reconstructed_ok": nq - bad, "queries": nq},
            "cpu_baseline": cpu,
            "serving": serving,
            "db_update": db_update,
            "single_query_latency": single,
            "row_shards": row_shards,
            "mmo_prf": mmo,
            "streamed": streamed,
            "additive": additive,
            "setup_s": setup_s,
        }
        print(json.dumps(out), flush=True)
    impir.impir_db_free(dbh)


if __name__ == "__main__":
    main()
