#!/usr/bin/env python3
"""Benchmark of the ZipPIR online server Response on GB300.

One step = one online Response for the workload's batch: the LWE answer
ans = D.q mod 2^32 over the whole database and the Paillier-side compression
t = (b' + H'.cko) mod m, both through the C ABI. Default workload: a 1 GiB
database (32768 x 32768 bytes uniform mod 256), one query, n = 1024, a 2048-bit
modulus. value = database bytes scanned per second (GB/s, 1 GB = 1e9 B) with
inputs resident in HBM, timed over K replays of one zp_respond captured in a CUDA
graph (inputs in place); the same step composed eagerly from its three calls gives
the per-kernel stages and the roofline (reported as "eager"). e2e = the same metric
through zp_respond_host with host buffers (query and offsets copied in, compressed
answer copied out, each step). The default line also carries "answer_alone" (the
single-query answer on every SM, against the HBM roofline) and "batched": 64 queries of
64 clients on the same database (graph-replayed zp_respond, its own e2e, and the answer
GEMM against the tensor-core roofline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 1gib|tiny|256mib|batch64|256mib_b64|8gib|8gib_b8|8gib_b32|8gib_b128|
                              serve|client_hint|lwe_compress]

--impl reference times the oracle (the plain CPU implementation) on a bounded
sample of the same workload on the host cores.
Under torchrun (N > 1) every rank runs its own replica of the workload on its own
GPU (the Response does not need any exchange between GPUs), value = all ranks'
bytes / the slowest rank's time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "online GB/s of DB scanned (1 query and batched) vs HBM/int8 roofline; p99 ms"

WORKLOADS = {
    # name: (R, C, n, B, description)
    "1gib": (32768, 32768, 1024, 1,
             "1 GiB database 32768x32768 u8 uniform mod 256, 1 query, n=1024, 2048-bit Paillier "
             "modulus: GEMV answer + compression"),
    "256mib": (16384, 16384, 1024, 1,
               "256 MiB database 16384x16384 u8 uniform mod 256, 1 query, n=1024, 2048-bit modulus"),
    "tiny": (1024, 1024, 1024, 1,
             "1 MiB database 1024x1024, 1 query, n=1024, 2048-bit modulus"),
    "batch64": (32768, 32768, 1024, 64,
                "1 GiB database 32768x32768, 64 queries of 64 clients, n=1024, 2048-bit moduli"),
    "256mib_b64": (16384, 16384, 1024, 64,
                   "256 MiB database 16384x16384, 64 queries of 64 clients, n=1024, 2048-bit moduli"),
    "8gib": (65536, 131072, 1024, 1,
             "8 GiB database 65536x131072, 1 query, n=1024, 2048-bit modulus"),
    "8gib_b8": (65536, 131072, 1024, 8, "8 GiB database 65536x131072, 8 queries"),
    "8gib_b32": (65536, 131072, 1024, 32, "8 GiB database 65536x131072, 32 queries"),
    "8gib_b128": (65536, 131072, 1024, 128, "8 GiB database 65536x131072, 128 queries"),
}
KEY_BITS = 2048
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of k_gemv<16, 6> (the GEMV
# beside the compression products), 1 GiB workload, mean of two captured launches
GEMV_TRAFFIC = {("1gib", True): 1075723136}
L = KEY_BITS // 32


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (context beside the measured peak)


def load_peaks():
    """(HBM GB/s, bf16 TFLOP/s burst, kind): the driver's measured copy bandwidth and cuBLAS
    bf16 rate on this machine's GPUs, else the fallback figures of an earlier GB300 measurement."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), d.get("bf16_tflops"), "measured"
    return 6800.0, 1900.0, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in the background."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.mark = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def window(self, t0, t1):
        self.mark = (t0, t1)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        t0, t1 = self.mark if self.mark else (0, 1e18)
        rows = [s for (t, s) in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or \
            [s for (_, s) in self.samples]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [x.strip() for x in r.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def dist_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_total_local: float, steps: int, bytes_per_step_per_rank: int, world: int):
    """Whole-job throughput over the ranks: every rank runs its own replica; the job's time is
    the slowest rank's, and the value counts the bytes of all ranks (GB/s)."""
    ms_total = dist_max(ms_total_local, world)
    ms_step = ms_total / steps
    return ms_step, bytes_per_step_per_rank * world / (ms_step * 1e-3) / 1e9


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- CPU oracle baseline
_CPU_SAMPLES = {}


def cpu_baseline(R, C, n, B, target_s=12.0, packed_rows=8):
    """Times the oracle's online Response (matvec mod 2^32 + compression with Python
    ints) on a bounded sample of rows of the same workload; returns GB/s of database
    bytes scanned, threads used and a description of the sample."""
    import synth
    from oracle import lwe, zippir
    from oracle.params import Params

    P = Params(n=n, key_bits=KEY_BITS)
    ell = P.ell
    rows = min(R, ell * packed_rows)  # whole packed rows
    key = (rows, C, n)
    if key not in _CPU_SAMPLES:  # the sample's inputs are built once (not timed)
        D = synth.database(rows, C, 101)
        q = synth.uniform_queries(1, C, 102)[0]
        # hint rows: uniform u32, statistically equal to -D.A for a uniform A (the hint
        # itself is offline work and not part of the timed online Response)
        Hn = synth.rng(103).integers(0, 2**32, size=(rows, n), dtype=np.uint64).astype(np.uint32)
        m = synth.random_odd_modulus(KEY_BITS, 104)
        _CPU_SAMPLES[key] = (D, q, Hn, m, synth.uniform_below(m, n, 105))
    D, q, Hn, m, cko = _CPU_SAMPLES[key]
    done_bytes, t_used, reps = 0, 0.0, 0
    t0 = time.perf_counter()
    while True:
        ans = lwe.matvec_mod_q(D, q)
        zippir.compress_rows(ans, Hn, cko, m, P)
        reps += 1
        done_bytes += rows * C
        t_used = time.perf_counter() - t0
        if t_used >= target_s or reps >= 2000:  # about target_s of CPU work
            break
    per_q = t_used / reps
    gbs = done_bytes / t_used / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d of %d rows (%d packed rows) x %d columns, 1 query, %d repetition(s), "
                      "%.2f s per repetition; numpy uint64 matvec + Python-int compression, "
                      "single thread" % (rows, R, rows // ell, C, reps, per_q),
            "seconds": t_used, "reps": reps, "rows": rows}


def cpu_matvec_all_cores(R, C, target_s=6.0):
    """The oracle's answer (numpy uint64 matvec mod 2^32) over a sample of the database's
    rows on every host core (row blocks in threads: numpy releases the GIL inside its
    integer products); the compression's Python integers stay single-threaded, so this is
    the answer alone. Returns GB/s of database bytes, the thread count and the sample."""
    from concurrent.futures import ThreadPoolExecutor
    import synth
    from oracle import lwe

    cores = max(1, len(os.sched_getaffinity(0)))
    rows = min(R, 64 * cores)
    D = synth.database(rows, C, 111)
    q = synth.uniform_queries(1, C, 112)[0]
    blocks = [(a, min(rows, a + 64)) for a in range(0, rows, 64)]
    done, reps = 0, 0
    with ThreadPoolExecutor(cores) as ex:
        t0 = time.perf_counter()
        while True:
            list(ex.map(lambda ab: lwe.matvec_mod_q(D[ab[0]:ab[1]], q), blocks))
            reps += 1
            done += rows * C
            dt = time.perf_counter() - t0
            if dt >= target_s or reps >= 1000:
                break
    return {"value": done / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "answer only (numpy uint64 matvec mod 2^32), %d of %d rows x %d columns in "
                      "blocks of 64 rows on %d threads, %d repetition(s)" % (rows, R, C, cores, reps)}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    R, C, n, B, desc = WORKLOADS[args.workload]
    vals, secs = [], []
    cb = None
    # each step is a bounded sample, sized so that all W + K steps take about 150 s
    budget = min(3.0, max(0.02, 150.0 / (args.warmup + args.steps)))
    packed = 8 if budget >= 0.5 else 1
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(R, C, n, B, target_s=budget, packed_rows=packed)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
            cb = r
    v = statistics.mean(vals)
    # ms_per_step: the measured wall time of one step (one bounded sample); the time the
    # oracle would take for the whole workload is an extrapolation, reported apart
    ms = statistics.mean(secs) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "step": "one bounded sample of the workload: %s" % cb["sample"],
            "extrapolated_full_workload_ms": R * C * B / (v * 1e9) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": desc, "R": R, "C": C, "n": n, "B": B, "key_bits": KEY_BITS},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"],
                             "value": v, "unit": "GB/s"},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, world, rank, local):
    import torch
    import paper_2603_09190_gb300 as zp
    from paper_2603_09190_gb300 import build as zb
    import synth

    if rank == 0:
        zb.build()
    dist_barrier(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R, C, n, B, desc = WORKLOADS[args.workload]
    ld = zp.db_pitch(C)

    ctx = zp.Context(local, n=n, key_bits=KEY_BITS)
    D = synth.device_database(R, C, 1 + rank, dev, ld=ld)
    A = synth.device_uniform_u32((C, n), 2 + rank, dev)
    db = zp.Database(ctx, D, R, C, ld)
    if B > 4:
        db.prepare_fp16()  # batched answers read the resident fp16 copy of D (2x its bytes)
    db.gen_hint(A)                                   # warm-up (allocations, attributes)
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record()
    db.gen_hint(A)
    h1.record()
    torch.cuda.synchronize()
    hint_ms = h0.elapsed_time(h1)
    del A
    moduli = [synth.random_odd_modulus(KEY_BITS, 1000 + b) for b in range(B)]
    clients = [ctx.register_client(m) for m in moduli]
    Q = synth.device_uniform_u32((B, C), 3 + rank, dev)
    # cko uniform below each client's m (limbs drawn on the host once)
    cko_h = np.stack([synth.ints_to_limbs(synth.uniform_below(moduli[b], n, 2000 + b), L)
                      for b in range(B)])
    CKO = torch.from_numpy(cko_h.view(np.int32)).to(dev)
    ans = torch.empty((B, R), dtype=torch.int32, device=dev)
    T = torch.empty((B, db.d1p, L), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    sp = stream.cuda_stream
    handles = [c.handle for c in clients]
    # thresholds and SM split measured on this database (zp_autotune)
    tuned = None if args.no_autotune else db.autotune()
    if args.overlap is not None:
        ctx.set_option("overlap_sms", args.overlap)
    overlap = B == 1 and zp.zp_get_overlap(ctx) > 0

    # One step = the same kernels zp_respond runs, composed here so that CUDA events
    # bracket the answer kernel on its own stream: for one query the compression
    # products run on `side` (a share of the SMs) while the GEMV runs on `stream`.
    def step(ev=None):
        if overlap:
            side.wait_stream(stream)
            if ev is not None:
                ev[3].record(side)
            zp.zp_compress_products(db.handle, CKO.data_ptr(), B, side.cuda_stream)
            if ev is not None:
                ev[4].record(side)
        if ev is not None:
            ev[0].record(stream)
        zp.zp_answer(db.handle, Q.data_ptr(), B, ans.data_ptr(), sp)
        if ev is not None:
            ev[1].record(stream)
        if overlap:
            stream.wait_stream(side)
        else:
            zp.zp_compress_products(db.handle, CKO.data_ptr(), B, sp)
        zp.zp_compress_finish(db.handle, handles, ans.data_ptr(), B, T.data_ptr(), sp)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ctx.device_status() != 0:
        raise RuntimeError("device status nonzero after warm-up")

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.kernel_launches()
    dist_barrier(world)
    torch.cuda.synchronize()
    tw0 = time.time()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    tw1 = time.time()
    dist_barrier(world)
    launches = ctx.kernel_launches() - launches0
    sampler.window(tw0, tw1)
    ms_step, value = aggregate(start.elapsed_time(end), args.steps, R * C * B, world)
    ans_ms = [e[0].elapsed_time(e[1]) for e in evs]
    cmp_ms = [e[1].elapsed_time(e[2]) for e in evs]
    prod_ms = [e[3].elapsed_time(e[4]) for e in evs] if overlap else []
    step_ms = [(e[3] if overlap else e[0]).elapsed_time(e[2]) for e in evs]
    db_bytes = R * C * B

    # ---- the composed step equals the library's zp_respond, bit for bit
    T_step = T.clone()
    ans2 = torch.empty_like(ans)
    T2 = torch.empty_like(T)
    zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans2.data_ptr(),
                  T2.data_ptr(), sp)
    torch.cuda.synchronize()
    if not (torch.equal(T2, T_step) and torch.equal(ans2, ans)):
        raise RuntimeError("composed step and zp_respond disagree")

    # ---- latency of one Response (zp_respond), warm and with L2 flushed before each call
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lat = {"warm": [], "cold": []}
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for kind in ("warm", "cold"):
        for _ in range(50):
            if kind == "cold":
                flush.fill_(1)
            e_a.record(stream)
            zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans2.data_ptr(),
                          T2.data_ptr(), sp)
            e_b.record(stream)
            torch.cuda.synchronize()
            lat[kind].append(e_a.elapsed_time(e_b) * 1e3)
    latency_us = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))}
                  for k, v in lat.items()}
    del flush

    # ---- the Response captured once in a CUDA graph and replayed (inputs in place): the
    # headline. W untimed replays, then exactly K timed ones between a barrier and a
    # synchronize on both sides; the eager composed loop above gives the per-kernel stages.
    l0 = ctx.kernel_launches()
    zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans2.data_ptr(), T2.data_ptr(), sp)
    torch.cuda.synchronize()
    launches_per_response = ctx.kernel_launches() - l0
    graph = None
    g_ms_total = None
    try:
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans2.data_ptr(),
                          T2.data_ptr(), gs.cuda_stream)      # sizes scratch before capture
        gs.synchronize()
        with torch.cuda.graph(g, stream=gs):
            zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans2.data_ptr(),
                          T2.data_ptr(), torch.cuda.current_stream().cuda_stream)
        T2.zero_()
        g.replay()
        torch.cuda.synchronize()
        same = bool(torch.equal(T2, T_step))
        if not same:
            raise RuntimeError("graph replay differs from the eager step")
        for _ in range(max(args.warmup, 3)):
            g.replay()
        torch.cuda.synchronize()
    except Exception as ex:  # noqa: BLE001 - reported in the line; the eager loop is the headline then
        graph = {"error": str(ex)[:200]}
        g = None
    # every rank takes the same branch (no rank waits at a barrier another one skips)
    if 1.0 - dist_max(0.0 if g is not None else 1.0, world) > 0.5:
        dist_barrier(world)
        torch.cuda.synchronize()
        tg0 = time.time()
        e_a.record(stream)
        for _ in range(args.steps):
            g.replay()
        e_b.record(stream)
        torch.cuda.synchronize()
        tg1 = time.time()
        dist_barrier(world)
        g_ms_total = e_a.elapsed_time(e_b)
        sampler.window(tg0, tg1)  # the clocks of the headline region
        graph = {"ms_per_step": g_ms_total / args.steps, "identical": True}

    # ---- batched answers against B single-query GEMV passes on the same database
    single = None
    if B > 1:
        q1 = torch.empty((1, R), dtype=torch.int32, device=dev)
        for _ in range(3):
            zp.zp_answer(db.handle, Q.data_ptr(), 1, q1.data_ptr(), sp)
        e_a.record(stream)
        for b in range(B):
            zp.zp_answer(db.handle, Q[b].data_ptr(), 1, q1.data_ptr(), sp)
        e_b.record(stream)
        torch.cuda.synchronize()
        single = e_a.elapsed_time(e_b)

    # ---- the single-query answer alone on the whole GPU (no compression products beside it)
    answer_alone = None
    if B == 1:
        ov = zp.zp_get_overlap(ctx)
        ctx.set_option("overlap_sms", 0)
        try:
            for _ in range(max(args.warmup, 3)):
                zp.zp_answer(db.handle, Q.data_ptr(), 1, ans2.data_ptr(), sp)
            reps = max(args.steps, 20)
            e_a.record(stream)
            for _ in range(reps):
                zp.zp_answer(db.handle, Q.data_ptr(), 1, ans2.data_ptr(), sp)
            e_b.record(stream)
            torch.cuda.synchronize()
        finally:
            ctx.set_option("overlap_sms", ov)
        if not torch.equal(ans2, ans):
            raise RuntimeError("answer on the whole GPU differs from the step's")
        a_ms = e_a.elapsed_time(e_b) / reps
        hbm_peak, _, peak_kind = load_peaks()
        gbs = (R * C + 4 * C + 4 * R) / (a_ms * 1e-3) / 1e9
        answer_alone = {"ms": a_ms, "launches": reps, "achieved_gb_s": gbs, "peak": hbm_peak,
                        "frac": gbs / hbm_peak, "frac_nominal": gbs / NOMINAL_HBM_GBS,
                        "peak_kind": peak_kind,
                        "kernel": "zp_answer alone (k_qplanes + k_gemv<8,12> on every SM)"}

    # ---- the batched half of the metric: 64 queries of 64 clients on the same database
    batched = None
    if args.workload == "1gib" and not args.no_batched:
        batched = measure_batched(args, zp, torch, ctx, db, dev, R, C, n, 64, stream, world)

    # ---- e2e through the host-buffer entry point
    hQ = torch.empty((B, C), dtype=torch.int32, pin_memory=True)
    hQ.copy_(Q.cpu())
    hC = torch.from_numpy(cko_h.view(np.int32)).pin_memory()
    hT = torch.empty((B, db.d1p, L), dtype=torch.int32, pin_memory=True)
    hQn, hCn, hTn = hQ.numpy().view(np.uint32), hC.numpy().view(np.uint32), hT.numpy().view(np.uint32)
    for _ in range(3):
        zp.zp_respond_host(db.handle, handles, hQn, hCn, B, hTn, None, sp)
    e2e_steps = max(3, min(args.steps, 200))
    dist_barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        zp.zp_respond_host(db.handle, handles, hQn, hCn, B, hTn, None, sp)
    torch.cuda.synchronize()
    e2e_s = dist_max((time.perf_counter() - t0) / e2e_steps, world)
    dist_barrier(world)
    sampler.stop()
    clocks = sampler.summary()
    status = ctx.device_status()
    if status != 0:
        raise RuntimeError("device status 0x%x after timing" % status)

    eager = {"ms_per_step": ms_step, "value": value, "gpu_launches": launches}
    if g_ms_total is not None:
        ms_step, value = aggregate(g_ms_total, args.steps, R * C * B, world)
        launches = launches_per_response * args.steps
        timing = "CUDA graph of zp_respond replayed K times (inputs in place)"
    else:
        timing = "eager composed step (zp_compress_products, zp_answer, zp_compress_finish)"
    if rank != 0:
        return 0
    hbm_peak, _, peak_kind = load_peaks()
    ans_avg = statistics.mean(ans_ms)
    # algorithmic bytes of one zp_answer (B = 1: query-plane prep + GEMV): D, q, ans
    alg_bytes = R * C + 4 * C * B + 4 * R * B
    achieved = alg_bytes / (ans_avg * 1e-3) / 1e9
    # DRAM bytes (read + write) of one launch of the GEMV in this configuration, from one
    # ncu capture of this workload (mean of two launches); None elsewhere
    traffic = GEMV_TRAFFIC.get((args.workload, overlap))
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "nominal_peak": NOMINAL_HBM_GBS, "traffic": traffic,
            "kernel": "zp_answer (k_qplanes + k_gemv)" if B == 1 else "zp_answer (batched)",
            "peak_kind": peak_kind}
    cb = None
    if world == 1 and not args.no_cpu:
        cb = cpu_baseline(R, C, n, B)
        cb["all_cores"] = cpu_matvec_all_cores(R, C)
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": desc, "R": R, "C": C, "n": n, "B": B, "key_bits": KEY_BITS,
                       "l2": "inputs larger than L2 (database %d MiB > 129 MB L2); no flush"
                             % (R * C >> 20),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "answer_operand": "fp16 copy of D" if B > 4 else "bytes of D",
                       "timing": timing},
            "eager": eager,
            "stages_ms": {"answer_avg": ans_avg,
                          "after_answer_avg": statistics.mean(cmp_ms),
                          "products_concurrent_avg": statistics.mean(prod_ms) if prod_ms else None,
                          "overlap_sms": zp.zp_get_overlap(ctx) if overlap else 0,
                          "step_p50": float(np.percentile(step_ms, 50)),
                          "step_p99": float(np.percentile(step_ms, 99))},
            "gib_s": value * 1e9 / 2**30,
            "latency_us": latency_us,
            "graph": graph,
            "autotuned": tuned,
            "batched_vs_single_gemv": None if single is None else
                {"single_query_gemv_x_B_ms": single, "batched_answers_ms": ans_avg,
                 "speedup": single / ans_avg},
            "hint_ms": hint_ms,
            "hint_tflops_fp16": 2.0 * R * C * 4 * n / (hint_ms * 1e-3) / 1e12,
            "roofline": roof,
            "e2e": {"value": db_bytes * world / e2e_s / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": 4 * B * C + 4 * B * n * L,
                    "d2h_bytes_per_step": 4 * B * db.d1p * L, "ms_per_step": e2e_s * 1e3},
            "gpu_launches": launches,
            "clocks": clocks,
            "answer_alone": answer_alone,
            "batched": batched,
            "cpu_baseline": cb}
    print(json.dumps(line))
    return 0


def measure_batched(args, zp, torch, ctx, db, dev, R, C, n, B, stream, world):
    """B queries of B clients (their own 2048-bit moduli) on the resident database: the
    answers from the fp16 copy of D on the tensor cores, the compression in the residue
    number system. Headline: K replays of one zp_respond captured in a CUDA graph (inputs in
    place), checked bit for bit against the eager call; the eager composed step (zp_answer,
    then zp_compress) brackets the answer GEMM with CUDA events for its tensor roofline;
    e2e through zp_respond_host (queries and offsets copied in, t copied out, every step)."""
    import synth
    sp = stream.cuda_stream
    db.prepare_fp16()
    moduli = [synth.random_odd_modulus(KEY_BITS, 5000 + b) for b in range(B)]
    clients = [ctx.register_client(m) for m in moduli]
    handles = [c.handle for c in clients]
    Q = synth.device_uniform_u32((B, C), 41, dev)
    cko_h = np.stack([synth.ints_to_limbs(synth.uniform_below(moduli[b], n, 6000 + b), L)
                      for b in range(B)])
    CKO = torch.from_numpy(cko_h.view(np.int32)).to(dev)
    ans = torch.empty((B, R), dtype=torch.int32, device=dev)
    T = torch.empty((B, db.d1p, L), dtype=torch.int32, device=dev)
    K, W = args.steps, max(args.warmup, 3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        zp.zp_answer(db.handle, Q.data_ptr(), B, ans.data_ptr(), sp)
        if ev is not None:
            ev[1].record(stream)
        zp.zp_compress(db.handle, handles, ans.data_ptr(), CKO.data_ptr(), B, T.data_ptr(), sp)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    for k in range(K):
        step(evs[k])
    torch.cuda.synchronize()
    ans_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    cmp_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    eager_ms = evs[0][0].elapsed_time(evs[-1][2]) / K
    T_ref, ans_ref = T.clone(), ans.clone()
    # the Response captured in a CUDA graph, replayed K times
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans.data_ptr(),
                      T.data_ptr(), gs.cuda_stream)
    gs.synchronize()
    with torch.cuda.graph(g, stream=gs):
        zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans.data_ptr(),
                      T.data_ptr(), torch.cuda.current_stream().cuda_stream)
    T.zero_()
    g.replay()
    torch.cuda.synchronize()
    if not (torch.equal(T, T_ref) and torch.equal(ans, ans_ref)):
        raise RuntimeError("batched graph replay differs from the eager step")
    for _ in range(W):
        g.replay()
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.kernel_launches()
    zp.zp_respond(db.handle, handles, Q.data_ptr(), CKO.data_ptr(), B, ans.data_ptr(),
                  T.data_ptr(), sp)
    torch.cuda.synchronize()
    per_resp = ctx.kernel_launches() - l0
    dist_barrier(world)
    torch.cuda.synchronize()
    e_a.record(stream)
    for _ in range(K):
        g.replay()
    e_b.record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    ms_step, value = aggregate(e_a.elapsed_time(e_b), K, R * C * B, world)
    # e2e: host buffers (pinned), copies inside the timed region
    hQ = torch.empty((B, C), dtype=torch.int32, pin_memory=True)
    hQ.copy_(Q.cpu())
    hC = torch.from_numpy(cko_h.view(np.int32)).pin_memory()
    hT = torch.empty((B, db.d1p, L), dtype=torch.int32, pin_memory=True)
    hQn, hCn, hTn = hQ.numpy().view(np.uint32), hC.numpy().view(np.uint32), hT.numpy().view(np.uint32)
    for _ in range(2):
        zp.zp_respond_host(db.handle, handles, hQn, hCn, B, hTn, None, sp)
    if not torch.equal(hT, T_ref.cpu()):
        raise RuntimeError("batched host-buffer Response differs from the device one")
    e2e_steps = max(3, min(K, 100))
    dist_barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        zp.zp_respond_host(db.handle, handles, hQn, hCn, B, hTn, None, sp)
    torch.cuda.synchronize()
    e2e_s = dist_max((time.perf_counter() - t0) / e2e_steps, world)
    dist_barrier(world)
    for c in clients:
        c.close()
    _, bf16_peak, peak_kind = load_peaks()
    flops = 2.0 * R * C * 4 * B          # executed: 4 byte planes of every query (fp16 MMAs)
    tfl = flops / (ans_ms * 1e-3) / 1e12
    return {"workload": "1 GiB database 32768x32768, %d queries of %d clients (own 2048-bit "
                        "moduli), n=1024: answers on the tensor cores from the fp16 copy of D, "
                        "compression in the residue number system" % (B, B),
            "B": B, "steps": K, "warmup": W, "ms_per_step": ms_step, "value": value, "unit": "GB/s",
            "gib_s": value * 1e9 / 2**30,
            "timing": "CUDA graph of zp_respond replayed K times (inputs in place)",
            "gpu_launches": per_resp * K,
            "eager": {"ms_per_step": eager_ms, "answer_ms": ans_ms, "compress_ms": cmp_ms},
            "roofline": {"bound": "tensor", "achieved": tfl, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": tfl / bf16_peak, "traffic": None,
                         "kernel": "zp_answer, B=%d (k_prep_q_rows + k_gemm_tc<ANS, 64, fp16 A>)" % B,
                         "peak_kind": peak_kind + " bf16 burst (kind::f16 with fp16 operands runs at "
                                                  "the bf16 rate)",
                         "executed_flops": flops, "algorithmic_macs": R * C * B,
                         "algorithmic_tmacs_s": R * C * B / (ans_ms * 1e-3) / 1e12},
            "e2e": {"value": R * C * B * world / e2e_s / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": 4 * B * C + 4 * B * n * L,
                    "d2h_bytes_per_step": 4 * B * db.d1p * L, "ms_per_step": e2e_s * 1e3}}


def run_serve(args, world, rank, local):
    """Serving workload: three resident databases, Poisson arrivals from many clients,
    row updates with idle-time hint regeneration; continuous batching (serve.Server)."""
    import threading
    import torch
    import paper_2603_09190_gb300 as zp
    from paper_2603_09190_gb300 import build as zb
    from paper_2603_09190_gb300.serve import Request, Server, ZipBackend
    import synth

    if rank == 0:
        zb.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1024
    ctx = zp.Context(local, n=n, key_bits=KEY_BITS)
    be = ZipBackend(ctx, max_batch=args.serve_batch, slots=args.serve_slots)
    shapes = {"db256m": (16384, 16384), "db1g": (32768, 32768), "db4g": (65536, 65536)}
    if args.serve_small:
        shapes = {"db256m": (4096, 4096), "db1g": (8192, 8192), "db4g": (16384, 16384)}
    for i, (name, (R, C)) in enumerate(shapes.items()):
        ld = zp.db_pitch(C)
        D = synth.device_database(R, C, 10 + i, dev, ld=ld)
        A = synth.device_uniform_u32((C, n), 20 + i, dev)
        db = zp.Database(ctx, D, R, C, ld)
        db.gen_hint(A)
        be.add_database(name, db, A)
    nclients = args.serve_clients
    moduli = [synth.random_odd_modulus(KEY_BITS, 3000 + k) for k in range(nclients)]
    for k, m in enumerate(moduli):
        be.add_client(k, m)
    g = synth.rng(77)
    qpool = {name: [g.integers(0, 2**32, size=C, dtype=np.uint64).astype(np.uint32) for _ in range(4)]
             for name, (R, C) in shapes.items()}
    kpool = [synth.ints_to_limbs(synth.uniform_below(moduli[k % nclients], n, 4000 + k), L)
             for k in range(8)]
    free = torch.cuda.mem_get_info(dev)[0]
    budget = int(free * 0.9) + sum(be.db_bytes(nm) for nm in shapes)
    results = []
    for rate in args.serve_rates:
        srv = Server(be, hbm_budget=budget, max_batch=args.serve_batch, slots=args.serve_slots)
        for name, (R, C) in shapes.items():
            srv.add_database(name, R, C)
        stop = threading.Event()
        names = list(shapes)

        def arrivals():
            rg = np.random.Generator(np.random.PCG64(int(rate)))
            t_next = time.perf_counter()
            rid = 0
            upd_next = time.perf_counter() + 0.1
            while not stop.is_set():
                now = time.perf_counter()
                if now >= upd_next:          # 1% of the rows per second, in 100 ms chunks
                    upd_next += 0.1
                    for name, (R, C) in shapes.items():
                        k = max(1, R // 1000)
                        rows = rg.choice(R, size=k, replace=False).astype(np.uint32)
                        new = torch.randint(0, 256, (k, C), dtype=torch.uint8, device=dev)
                        srv.update_rows(name, rows, new)
                if now < t_next:
                    time.sleep(min(t_next - now, 0.001))
                    continue
                name = names[int(rg.integers(0, 3))]
                cid = int(rg.integers(0, nclients))
                srv.submit(Request(rid, name, cid, qpool[name][rid % 4], kpool[cid % 8], t_next))
                rid += 1
                t_next += rg.exponential(1.0 / rate)

        th = threading.Thread(target=arrivals, daemon=True)
        t0 = time.perf_counter()
        th.start()
        while time.perf_counter() - t0 < args.serve_seconds:
            if srv.step() == 0:
                time.sleep(0.0001)
        stop.set()
        th.join()
        srv.run_until_idle(timeout=120)
        t1 = time.perf_counter()
        rep = srv.report(t0, t1)
        rep["offered_qps"] = rate
        results.append(rep)
    status = ctx.device_status()
    if rank == 0:
        best = max(results, key=lambda r: r["db_gb_s"])
        line = {"metric": METRIC, "value": best["db_gb_s"], "unit": "GB/s", "n_gpus": world,
                "steps": len(results), "warmup": 0, "ms_per_step": None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": "serving: resident databases %s, Poisson arrivals, %d "
                                       "clients with their own 2048-bit moduli, 1%% rows/s "
                                       "updated with idle-time hint regeneration, %d s per rate"
                                       % (",".join("%s %dx%d" % (k, *v) for k, v in shapes.items()),
                                          nclients, args.serve_seconds),
                           "max_batch": args.serve_batch, "slots_per_db": args.serve_slots},
                "rates": results, "device_status": status}
        print(json.dumps(line))
    return 0


def run_client_hint(args, world, rank, local):
    """Offline per-client hint k = PaillierMatMul(H', ck_r) for one client over a 1 GiB
    database (n = 1024), and the online combined response k (+) t for 1 and 64 queries."""
    import torch
    import paper_2603_09190_gb300 as zp
    from paper_2603_09190_gb300 import build as zb
    import synth

    if rank == 0:
        zb.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R = C = 32768
    n = 1024
    ctx = zp.Context(local, n=n, key_bits=KEY_BITS)
    ld = zp.db_pitch(C)
    D = synth.device_database(R, C, 1, dev, ld=ld)
    A = synth.device_uniform_u32((C, n), 2, dev)
    db = zp.Database(ctx, D, R, C, ld)
    db.gen_hint(A)
    del A
    m = synth.random_odd_modulus(KEY_BITS, 3)
    cl = ctx.register_client(m)
    g = synth.rng(9)
    m2 = m * m
    ckr = [int.from_bytes(g.bytes(2 * KEY_BITS // 8 + 16), "little") % m2 for _ in range(n)]
    CKR = torch.from_numpy(synth.ints_to_limbs(ckr, 2 * L).view(np.int32)).to(dev)
    K = torch.zeros((db.d1p, 2 * L), dtype=torch.int32, device=dev)
    db.client_hint(cl, CKR, out=K, packed_rows=[0])          # warm-up: one packed row
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.kernel_launches()
    e0.record()
    db.client_hint(cl, CKR, out=K)
    e1.record()
    torch.cuda.synchronize()
    k_ms = e0.elapsed_time(e1)
    comb = {}
    for B in (1, 64):
        T = synth.device_uniform_u32((B, db.d1p, L), 7, dev)
        KB = K[None].expand(B, -1, -1).contiguous()
        cls = [cl] * B
        for _ in range(max(args.warmup, 3)):
            db.combine(cls, KB, T)
        torch.cuda.synchronize()
        steps = max(args.steps // 100, 10)
        e0.record()
        for _ in range(steps):
            db.combine(cls, KB, T)
        e1.record()
        torch.cuda.synchronize()
        comb[B] = e0.elapsed_time(e1) / steps
    # client-side pieces: ChaCha20 keystream (1 GiB), ck_r from a seed, modexp and decryption
    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    ks = torch.empty(1 << 28, dtype=torch.int32, device=dev)
    ks_ms = ev_time(lambda: zp.prg_chacha20(bytes(32), bytes(12), 0, ks), 5)
    del ks
    ck16 = torch.empty((16384, 2 * L), dtype=torch.int32, device=dev)
    exp_ms = ev_time(lambda: cl.expand_ckr(bytes(range(32)), 16384, out=ck16), 5)
    lam = synth.random_odd_modulus(KEY_BITS, 5)   # 2048-bit exponents (timing: any value works)
    ct4 = ck16[:4096].contiguous()
    pw_ms = ev_time(lambda: cl.powm(ct4, lam), 2)
    dec_ms = ev_time(lambda: cl.decrypt(ct4, lam, lam), 2)
    client = {"chacha20_1gib_ms": ks_ms, "chacha20_gb_s": 2 ** 30 / (ks_ms * 1e-3) / 1e9,
              "expand_ckr_16384_ms": exp_ms, "powm_2048bit_exp_per_s": 4096 / (pw_ms * 1e-3),
              "decrypt_per_s": 4096 / (dec_ms * 1e-3)}
    status = ctx.device_status()
    if rank == 0:
        line = {"metric": METRIC, "value": R * C / (k_ms * 1e-3) / 1e9, "unit": "GB/s",
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": k_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": "per-client hint k = PaillierMatMul(H', ck_r) over a 1 GiB "
                                       "database 32768x32768, n=1024, 2048-bit modulus (offline; "
                                       "value = database bytes covered per second)",
                           "R": R, "C": C, "n": n, "d1p": db.d1p},
                "client_hint_s": k_ms / 1e3,
                "combine_ms": {"B1": comb[1], "B64": comb[64]},
                "client_side": client,
                "gpu_launches": ctx.kernel_launches() - launches0,
                "device_status": status}
        print(json.dumps(line))
    return 0


# Single-compression parameter sets of the evaluation (Sec. 5.1, table of single LWE
# ciphertext / RLWE coefficient compression): (kind, n or N, log2 q, the paper's time in ms
# on its CPU with a 3072-bit Paillier modulus -- context, not a target).
LC_SETS = [("lwe", 630, 64, 9.7), ("lwe", 742, 64, 11.0), ("lwe", 870, 64, 12.9), ("lwe", 1305, 11, 16.6),
           ("rlwe", 1024, 27, 7.2), ("rlwe", 2048, 54, 23.8), ("rlwe", 4096, 36, 33.8), ("rlwe", 8192, 43, 83.3)]


def run_lwe_compress(args, world, rank, local):
    """Standalone compression with a 3072-bit Paillier modulus: one ciphertext (latency) and
    256 ciphertexts (throughput) for every single-compression parameter set, RLWE
    coefficients after sample extraction, and batched compression of (630, 2^64)."""
    import torch
    import paper_2603_09190_gb300 as zp
    from paper_2603_09190_gb300 import build as zb
    import synth

    if rank == 0:
        zb.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bits = 3072
    m = synth.random_odd_modulus(bits, 11)
    comp = zp.LweCompressor(local, bits, m)
    g = synth.rng(12)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def u64(shape, lq):
        x = g.integers(0, 2 ** 63, size=shape, dtype=np.uint64) * np.uint64(2) + \
            g.integers(0, 2, size=shape, dtype=np.uint64)
        if lq < 64:
            x &= np.uint64((1 << lq) - 1)
        return torch.from_numpy(x.view(np.int64)).to(dev)

    def ck_of(n):  # uniform below 2^(64 L - 32) < m^2
        v = g.integers(0, 2 ** 32, size=(n, 2 * bits // 32), dtype=np.uint64).astype(np.uint32)
        v[:, -1] = 0
        return torch.from_numpy(v.view(np.int32)).to(dev)

    steps = max(args.steps // 200, 5)
    sets = []
    for kind, n, lq, paper_ms in LC_SETS:
        q = 1 << lq
        comp.set_key(ck_of(n), lq)
        if kind == "lwe":
            A1, B1 = u64((1, n), lq), u64((1,), lq)
            single = timed(lambda: comp.compress(A1, B1, q), steps)
        else:
            Ap, Bp = u64((n,), lq), u64((n,), lq)
            single = timed(lambda: comp.compress(*comp.rlwe_extract(Ap, Bp, q, [n // 2]), q), steps)
        A, B = u64((256, n), lq), u64((256,), lq)
        many = timed(lambda: comp.compress(A, B, q), 2)
        sets.append({"kind": kind, "n": n, "log2q": lq, "single_ms": single, "paper_single_ms": paper_ms,
                     "ct_per_s_256": 256 / many * 1e3})
    # batched (630, 2^64): gamma = q + n q^2, ell = largest with gamma^ell < m
    n, q = 630, 1 << 64
    gamma = q + n * q * q
    ell = 0
    while gamma ** (ell + 1) < m:
        ell += 1
    T = ((q - 1) * sum(gamma ** j for j in range(ell))).bit_length()
    comp.set_key(ck_of(n), T)
    batched = {}
    for groups in (1, 16):
        A, B = u64((groups * ell, n), 64), u64((groups * ell,), 64)
        ms = timed(lambda: comp.compress(A, B, q, ell=ell, gamma=gamma), 1)
        batched["groups%d" % groups] = {"cts": groups * ell, "ms": ms, "ct_per_s": groups * ell / ms * 1e3}
    cpu = None
    if not args.no_cpu:
        from oracle import lwecompress as olc
        from oracle import paillier as opl
        pk = opl.PublicKey(m)
        ck = [int.from_bytes(g.bytes(760), "little") for _ in range(630)]
        a = [int.from_bytes(g.bytes(8), "little") for _ in range(630)]
        t0 = time.perf_counter()
        olc.lwe_compress(pk, ck, a, 12345, 1 << 64)
        cpu = {"value": (time.perf_counter() - t0) * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": "one (630, 2^64) ciphertext, Python integers"}
    # roofline of the dominant kernel (k_lc_products): word multiply-accumulates of the
    # Montgomery products, 2 (2L)^2 per product, about n * 32 + 2 products per (630, 2^64)
    # ciphertext (the set bits of 64-bit exponents, the pairwise tree, the final factor),
    # against 152 SMs x 64 IMAD.WIDE lanes x 2.07 GHz; integer ALU-bound (ncu: ALU pipe 64 %)
    macs = sets[0]["ct_per_s_256"] * (630 * 32 + 2) * 2 * (2 * bits // 32) ** 2
    alu_peak = 152 * 64 * 2.07e9
    roof = {"bound": "alu", "achieved": macs, "peak": alu_peak, "unit": "word MAC/s",
            "frac": macs / alu_peak, "traffic": None, "kernel": "k_lc_products (+ pairwise tree)",
            "peak_kind": "derived: 152 SMs x 64 IMAD.WIDE lanes x 2.07 GHz"}
    if rank == 0:
        head = sets[0]
        line = {"metric": "single LWE ciphertext compression latency, (n, q) = (630, 2^64), 3072-bit Paillier",
                "value": head["single_ms"], "unit": "ms", "n_gpus": world, "steps": steps,
                "warmup": max(args.warmup, 3), "ms_per_step": head["single_ms"], "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": "standalone compression: single-compression parameter sets and batched "
                                       "(630, 2^64), 3072-bit modulus, inputs resident in HBM",
                           "key_bits": bits, "ell": ell, "T_folded": T},
                "sets": sets, "batched_630_64": batched, "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1gib", choices=sorted(WORKLOADS) + ["serve", "client_hint", "lwe_compress"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default thresholds and SM split")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-query measurement of the default workload")
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[50, 100, 200, 500, 1000, 2000])
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-slots", type=int, default=2,
                    help="batches of one database in flight at once (database views)")
    ap.add_argument("--serve-clients", type=int, default=1000)
    ap.add_argument("--serve-batch", type=int, default=64)
    ap.add_argument("--serve-small", action="store_true", help="smaller databases (smoke)")
    ap.add_argument("--overlap", type=int, default=None,
                    help="SMs for the compression products beside a single-query answer "
                         "(default: the library's)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if args.workload in ("serve", "client_hint", "lwe_compress"):
            args.workload = "1gib"
        return run_reference(args, world, rank)
    if args.workload == "serve":
        return run_serve(args, world, rank, local)
    if args.workload == "client_hint":
        return run_client_hint(args, world, rank, local)
    if args.workload == "lwe_compress":
        return run_lwe_compress(args, world, rank, local)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
