"""Benchmark: chunking throughput of RAM, AE and MAXP on a 4 GiB mixed stream.

One step = the whole hot path over one batch of input: the 4 GiB mixed
stream (seed 1; 1 MiB blocks of uniform / text-like / zero-run bytes) chunked
with RAM, AE and MAXP at mean chunk sizes 4, 8 and 16 KiB (min = mean/4,
max = 8*mean, windows from the calibrated table) -- 9 library calls, inputs
resident in HBM. value = bytes chunked / device time (GB/s, 1e9).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun), every rank chunks its own 4 GiB stream (seed 1 + rank):
independent replicas, no data-path collective (weak scaling).
The reference arm (--impl reference) times the CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GIB = 1 << 30
MIB = 1 << 20
STREAM_LEN = 4 * GIB
ALGS = ("ram", "ae", "maxp")
MEANS = (4096, 8192, 16384)
METRIC = "chunking GB/s per algo (RAM/AE/MAXP), % of HBM peak; batched GB/s; p50/p99 lat"
WORKLOAD = ("mixed stream 4 GiB (seed 1: 50% uniform, 30% Zipf-1.1 text over 64 symbols, 20% zero runs "
            "4-64 KiB, 1 MiB blocks); RAM, AE, MAXP x mean {4,8,16} KiB, min=mean/4, max=8*mean")


def wtable():
    with open(os.path.join(ROOT, "tests", "golden", "wtable.json")) as f:
        return json.load(f)


def configs(algs=ALGS, means=MEANS):
    t = wtable()["mixed_4g_seed1"]
    return [(alg, mean, t[alg][str(mean)]["w"], t[alg][str(mean)]["min"], t[alg][str(mean)]["max"])
            for alg in algs for mean in means]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SPEC_SOURCES = ("paper_2508_05797_gb300/csrc/chain.cu", "paper_2508_05797_gb300/csrc/chain_logic.cuh",
                "paper_2508_05797_gb300/csrc/warp_rules.cuh", "paper_2508_05797_gb300/csrc/cdc_device.cuh")
# machine-written record of the speculation kernel's DRAM traffic (written by
# `bench.py --write-traffic` from an ncu capture's CSV)
SPEC_TRAFFIC = os.path.join("profiles", "k_spec_traffic.json")


def sources_sha(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(path: str = None):
    """DRAM bytes per input byte of the speculation kernel from the capture
    record, if that record was taken on the current kernel sources."""
    p = path or os.path.join(ROOT, SPEC_TRAFFIC)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("source_sha256_16") != sources_sha(SPEC_SOURCES):
        return None
    try:
        return float(rec["dram_bytes_per_input_byte"])
    except (KeyError, TypeError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # one process per GPU over NCCL; gloo where there is no GPU (host-side tests)
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def write_traffic(csv_path: str, input_bytes: int, command: str, out_path: str = None):
    """Write SPEC_TRAFFIC from an ncu CSV (metrics dram__bytes_read.sum,
    dram__bytes_write.sum, gpu__time_duration.sum) of k_spec launches that
    each chunked `input_bytes` bytes: DRAM bytes per input byte per launch and
    their mean, with the hash of the kernel sources they were taken on."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    hdr = None
    per = {}
    for r in rows:
        if r and r[0] == "ID":
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        if "k_spec" not in d["Kernel Name"]:
            continue
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1, "us": 1e3, "ms": 1e6}
        v = float(d["Metric Value"].replace(",", "")) * scale.get(d["Metric Unit"], 1)
        per.setdefault(d["ID"], {"kernel": d["Kernel Name"]})[d["Metric Name"]] = v
    launches = []
    for k, d in sorted(per.items(), key=lambda x: int(x[0])):
        b = d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
        launches.append({"kernel": d["kernel"], "dram_bytes": int(b), "dram_bytes_per_input_byte": b / input_bytes,
                         "time_ns": d.get("gpu__time_duration.sum")})
    if not launches:
        raise SystemExit("no k_spec launches in %s" % csv_path)
    rec = {"kernel": "k_spec", "input_bytes_per_launch": input_bytes, "launches": launches,
           "dram_bytes_per_input_byte": sum(x["dram_bytes_per_input_byte"] for x in launches) / len(launches),
           "source_sha256_16": sources_sha(SPEC_SOURCES), "command": command,
           "note": "times under ncu are serialised and cold; only the byte counts are used"}
    with open(out_path or os.path.join(ROOT, SPEC_TRAFFIC), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm part)."""
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model Name", "Hardware"):
        for line in txt.splitlines():
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = {line.split(":", 1)[1].strip() for line in txt.splitlines()
             if line.startswith("CPU part") and ":" in line}
    impl = {line.split(":", 1)[1].strip() for line in txt.splitlines()
            if line.startswith("CPU implementer") and ":" in line}
    if parts:
        return "Arm implementer %s part %s" % (",".join(sorted(impl)), ",".join(sorted(parts)))
    return "unknown"


def cpu_baseline(sample_bytes: int = 128 * MIB):
    """The oracle on the host cores: each of the nine (algorithm, mean) jobs on
    one thread over the first sample_bytes of the stream (the chunk chain is
    sequential), then all nine at once (one thread each), and a sample of the
    batched files (log-normal sizes, seed 3) spread over every core."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    import synth
    cores = os.cpu_count() or 1
    data = synth.mixed_range(1, STREAM_LEN, 0, sample_bytes)
    cfg = configs()
    single = []
    t0 = time.perf_counter()
    for alg, mean, w, mn, mx in cfg:
        t1 = time.perf_counter()
        oracle.count(alg, data, w, mn, mx)
        single.append(sample_bytes / (time.perf_counter() - t1) / 1e9)
    dt_single = time.perf_counter() - t0
    # all nine jobs at once (the oracle's C loop releases the GIL)
    with ThreadPoolExecutor(min(len(cfg), cores)) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda c: oracle.count(c[0], data, c[2], c[3], c[4]), cfg))
        dt_par = time.perf_counter() - t0
    # files: log-normal sizes (median 64 KiB), RAM and MAXP at 8 KiB mean, over all cores
    sizes = synth.lognormal_sizes(3, 4000, 65536, 1.5, 1, 8 * MIB).astype(np.int64)
    off = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    arena = synth.mixed(3, int(off[-1]))
    t = wtable()["mixed_4g_seed1"]
    jobs = [(a, i) for a in ("maxp", "ram") for i in range(sizes.size)]

    def file_job(j):
        a, i = j
        e = t[a]["8192"]
        return oracle.count(a, arena[off[i]:off[i + 1]], e["w"], e["min"], e["max"])

    with ThreadPoolExecutor(cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(file_job, jobs))
        dt_files = time.perf_counter() - t0
    return {"value": round(len(cfg) * sample_bytes / dt_single / 1e9, 4), "unit": "GB/s", "cores": 1,
            "kind": "oracle",
            "sample": "first %d MiB of the 4 GiB mixed stream, each of the 9 (alg, mean) pairs on one thread" % (
                sample_bytes // MIB),
            "seconds": round(dt_single, 2), "per_job_GBps": [round(x, 4) for x in single],
            "host": {"hardware_concurrency": cores, "cpu_model": cpu_model()},
            "all_jobs_parallel": {"value": round(len(cfg) * sample_bytes / dt_par / 1e9, 4), "unit": "GB/s",
                                  "cores": min(len(cfg), cores), "seconds": round(dt_par, 2)},
            "files_all_cores": {"value": round(2 * int(off[-1]) / dt_files / 1e9, 4), "unit": "GB/s",
                                "cores": cores, "seconds": round(dt_files, 2),
                                "sample": "%d files (log-normal, median 64 KiB, seed 3, %.1f MB), MAXP and RAM at "
                                          "8 KiB mean" % (sizes.size, off[-1] / 1e6)}}


CDF_KIB = (1, 2, 4, 8, 16, 32, 64)


def size_cdf(bounds_list, bin_width: int = 1024, n_bins: int = 129):
    """Chunk-size distribution of one or more boundary lists (int64 CUDA
    tensors), counted on the device by cdc_size_histogram: the chunk count,
    the mean size and the CDF at 1..64 KiB (fraction of chunks smaller than
    each size), the paper's chunk-size CDF (Section 5.2) in a few points."""
    from paper_2508_05797_gb300 import size_histogram
    h = None
    total = 0
    for b in bounds_list:
        x = size_histogram(b, bin_width, n_bins)
        h = x if h is None else h + x
        total += int(b[-1].item()) if b.numel() else 0
    h = h.cpu().tolist()
    n = sum(h)
    cum, acc = [], 0
    for c in h:
        acc += c
        cum.append(acc)
    return {"chunks": n, "mean": round(total / max(n, 1), 1),
            "cdf_below_kib": {str(k): round(cum[k * 1024 // bin_width - 1] / max(n, 1), 4) for k in CDF_KIB}}


def batched_workload(dev, n_files: int = 100_000, warmup: int = 2, reps: int = 3):
    """The batched form against a per-file launch loop: files with log-normal
    sizes (median 64 KiB, sigma 1.5, clipped to 1 B .. 256 MiB, seed 3) of
    mixed content packed in one device arena, chunked with MAXP and RAM at
    8 KiB mean. The batched call is autotuned (cdc_autotune), captured in a
    CUDA graph and replayed; the loop calls cdc_chunk_async once per file.
    Both outputs are compared bit for bit."""
    import ctypes

    import numpy as np
    import torch

    import synth
    from paper_2508_05797_gb300 import Chunker
    from paper_2508_05797_gb300.cdc import Params, alg_id

    sizes = synth.lognormal_sizes(3, n_files, 65536, 1.5, 1, 256 * MIB).astype(np.int64)
    off = np.zeros(n_files + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    total = int(off[-1])
    host = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    synth.mixed(3, total, out=host.numpy())
    arena = host.to(dev)
    del host
    d_off = torch.from_numpy(off).to(dev)
    t = wtable()["mixed_4g_seed1"]
    res = {"workload": "%d files, log-normal sizes (median 64 KiB, sigma 1.5, 1 B..256 MiB, seed 3), mixed content, "
                       "%.2f GB in one device arena; 8 KiB mean" % (n_files, total / 1e9),
           "bytes": total}
    stream = torch.cuda.Stream(dev)
    for alg in ("maxp", "ram"):
        e = t[alg]["8192"]
        w, mn, mx = e["w"], e["min"], e["max"]
        ck = Chunker(dev.index)
        cap = total // mn + n_files + 1
        out = torch.empty(cap, dtype=torch.int64, device=dev)
        idx = torch.empty(n_files + 1, dtype=torch.int64, device=dev)
        seg, wc, tune_ms = ck.autotune(arena, alg, w, mn, mx, out=out, file_off=d_off, index=idx, stream=stream)
        ck.reserve(alg, w, mn, mx, total, n_files)
        with torch.cuda.stream(stream):
            ck.chunk_batch(arena, d_off, alg, w, mn, mx, out=out, index=idx, stream=stream, sync=False)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ck.chunk_batch(arena, d_off, alg, w, mn, mx, out=out, index=idx, stream=stream, sync=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):  # replay() launches on the current stream
            for _ in range(warmup):
                g.replay()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ck.sync_status(stream)
        batch_ms = e0.elapsed_time(e1) / reps
        index = idx.cpu().numpy()
        # per-file loop through the single-stream entry point
        out2 = torch.full((cap,), -1, dtype=torch.int64, device=dev)
        cnt = torch.zeros(n_files, dtype=torch.int64, device=dev)
        lib, h, prm, a = ck.lib, ck.h, Params(w, mn, mx), alg_id(alg)
        base, obase, cbase = arena.data_ptr(), out2.data_ptr(), cnt.data_ptr()
        sh = stream.cuda_stream
        fn = lib.cdc_chunk_async
        torch.cuda.synchronize()
        e0.record(stream)
        t0 = time.perf_counter()
        for f in range(n_files):
            st = fn(h, a, prm, base + int(off[f]), int(sizes[f]), obase + 8 * int(index[f]),
                    int(index[f + 1] - index[f]), cbase + 8 * f, sh)
            if st:
                raise RuntimeError("cdc_chunk_async failed on file %d: status %d" % (f, st))
        e1.record(stream)
        torch.cuda.synchronize()
        loop_wall = time.perf_counter() - t0
        loop_ms = e0.elapsed_time(e1)
        ck.sync_status(stream)
        same = bool(torch.equal(out2[:int(index[-1])], out[:int(index[-1])]) and
                    torch.equal(cnt, torch.from_numpy(np.diff(index)).to(dev)))
        res[alg] = {"batched_GBps": round(total / (batch_ms / 1e3) / 1e9, 1), "batched_ms": round(batch_ms, 3),
                    "loop_GBps": round(total / (loop_ms / 1e3) / 1e9, 2), "loop_ms": round(loop_ms, 1),
                    "loop_host_s": round(loop_wall, 2), "speedup": round(loop_ms / batch_ms, 1),
                    "bit_exact": same, "autotuned": {"segment": seg, "warp_chains": wc, "ms": round(tune_ms, 3)},
                    "boundaries": int(index[-1])}
        ck.close()
        del out, out2, idx, cnt, g
    # chunk-size distribution of every algorithm over all files (untimed)
    res["size_cdf"] = {}
    ck = Chunker(dev.index)
    for alg in ("ram", "ae", "ae_min", "maxp"):
        e = t["ae" if alg == "ae_min" else alg]["8192"]
        b, ix = ck.chunk_batch(arena, d_off, alg, e["w"], e["min"], e["max"])
        # boundaries are relative to each file's start: make them arena offsets
        b = b + torch.repeat_interleave(d_off[:-1], ix[1:] - ix[:-1])
        res["size_cdf"][alg] = size_cdf([b])
        del b, ix
    ck.close()
    del arena
    torch.cuda.empty_cache()
    return res


def serving_workload(host_stream, dev, n_req: int = 20000, rates=(0.1, 0.25, 0.5, 0.75, 0.9, 1.1), slots: int = 4,
                     budget: int = 40 << 30, max_batch: int = 0):
    """The serving loop: requests with log-normal sizes (median 64 KiB, sigma
    1.5, clipped to 4 KiB .. 64 MiB, seed 4) cut from the pinned host copy of
    the mixed stream, algorithm uniform over RAM / AE / MAXP at 8 KiB mean,
    through cdc_server_* (40 GiB device budget, continuous batching on `slots`
    streams). First all requests at once (saturation throughput, the median of
    three runs), then Poisson arrivals (seed 5) at fractions of that request
    rate; per rate the latency
    from arrival to boundaries in host memory (p50 / p99) and GB/s."""
    import numpy as np

    import synth
    from paper_2508_05797_gb300 import Server

    hnp = host_stream.numpy()
    sizes = synth.lognormal_sizes(4, n_req, 65536, 1.5, 4096, 64 * MIB).astype(np.int64)
    algs = synth.choice(4, n_req, 3)
    starts = (synth.lognormal_sizes(6, n_req, 1 << 30, 4.0, 0, hnp.size) % np.maximum(1, hnp.size - sizes)).astype(
        np.int64)
    t = wtable()["mixed_4g_seed1"]
    prm = [(a, t[a]["8192"]["w"], t[a]["8192"]["min"], t[a]["8192"]["max"]) for a in ALGS]
    outs = [np.zeros(int(sizes[i]) // prm[int(algs[i])][2] + 2, dtype=np.uint64) for i in range(n_req)]
    total = int(sizes.sum())

    # one server for every run (its device memory is allocated once)
    srv = Server(dev.index, budget, slots, max_batch)

    def run(arrivals):
        # arrival times start after the submission loop (about 20 us per request)
        t0 = srv.clock() + 50.0 + 0.03 * n_req
        for i in range(n_req):
            a, w, mn, mx = prm[int(algs[i])]
            srv.submit(hnp[int(starts[i]):int(starts[i]) + int(sizes[i])], a, w, mn, mx, outs[i], tag=i,
                       arrive_ms=t0 + float(arrivals[i]))
        res = []
        while len(res) < n_req:
            res.extend(srv.poll(4096, wait_ms=100))
        ok = all(r["status"] == 0 for r in res)
        arr = np.array([r["t_arrive_ms"] for r in res])
        done = np.array([r["t_done_ms"] for r in res])
        lat = done - arr
        span = (done.max() - arr.min()) / 1e3
        return {"GBps": round(total / span / 1e9, 2), "req_per_s": round(n_req / span, 1),
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "mean_batch": round(float(np.mean([r["batch_size"] for r in res])), 1), "all_ok": ok}

    # every request arrives at once; the first run (the device's first reads of
    # the host buffer) is a warm-up, and the few large batches make one run's
    # rate vary, so saturation is the median of the next three
    try:
        warm = run(np.zeros(n_req))
        sats = sorted((run(np.zeros(n_req)) for _ in range(3)), key=lambda r: r["req_per_s"])
        sat = dict(sats[1], runs_GBps=[r["GBps"] for r in sats], warmup_GBps=warm["GBps"])
        rate_runs = []
        for f in rates:
            rate = f * sat["req_per_s"]
            arrivals = synth.poisson_arrivals(5, n_req, rate / 1e3)  # ms
            r = run(arrivals)
            r["offered_req_per_s"] = round(rate, 1)
            r["offered_fraction"] = f
            rate_runs.append(r)
    finally:
        srv.close()
    out = {"workload": "%d requests, log-normal sizes (median 64 KiB, sigma 1.5, 4 KiB..64 MiB, seed 4), "
                       "%.2f GB from pinned host memory, RAM/AE/MAXP uniform at 8 KiB mean, %d GiB budget, %d slots, "
                       "batches up to %d requests" % (n_req, total / 1e9, budget >> 30, slots, max_batch or 4096),
           "saturation": sat, "rates": rate_runs}
    return out


def prims_workload(data, dev, n_q: int = 1 << 20, span: int = 8192, reps: int = 3):
    """The two processing patterns alone (cdc_ebs, cdc_rs): n_q ranges of
    `span` bytes at seeded offsets of the 4 GiB stream; Extreme Byte Search
    for the maximum and its first position, then a GEQ Range Scan for that
    maximum (so each scan stops at the maximum). GB/s of range bytes."""
    import numpy as np
    import torch

    import synth
    from paper_2508_05797_gb300 import ebs, rs

    n = data.numel()
    starts = (synth.lognormal_sizes(8, n_q, 1 << 30, 4.0, 0, n) % max(1, n - span)).astype(np.int64)
    r = torch.from_numpy(np.stack([starts, starts + span], axis=1)).to(dev)
    out = {"workload": "%d ranges of %d bytes at seeded offsets of the 4 GiB mixed stream" % (n_q, span)}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v, p = ebs(data, r, "max")
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        v, p = ebs(data, r, "max")
    e1.record()
    torch.cuda.synchronize()
    t_ebs = e0.elapsed_time(e1) / reps
    q = rs(data, r, v, "geq")
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        q = rs(data, r, v, "geq")
    e1.record()
    torch.cuda.synchronize()
    t_rs = e0.elapsed_time(e1) / reps
    scanned = int((q - r[:, 0] + 1).clamp(max=span).sum().item())
    out["ebs"] = {"ms": round(t_ebs, 3), "GBps": round(n_q * span / (t_ebs / 1e3) / 1e9, 1),
                  "queries_per_s": round(n_q / (t_ebs / 1e3), 0)}
    out["rs_geq"] = {"ms": round(t_rs, 3), "GBps_of_ranges": round(n_q * span / (t_rs / 1e3) / 1e9, 1),
                     "GBps_scanned": round(scanned / (t_rs / 1e3) / 1e9, 1),
                     "same_position": bool(torch.equal(q, p))}
    # byte shares of the two patterns in RAM and AE at 8 KiB mean (cdc_byte_shares
    # over the chunk boundaries of the whole stream)
    from paper_2508_05797_gb300 import byte_shares, chunk
    shares = {"paper_context": "Section 5.5 reports RAM 96.70 / 3.30 and MAXP 10.26 / 89.74 (EBS / RS %) on its "
                               "DEB dataset; these shares are on the synthetic mixed stream"}
    for alg in ("ram", "ae", "ae_min", "maxp"):
        e = wtable()["mixed_4g_seed1"]["ae" if alg == "ae_min" else alg]["8192"]
        b = chunk(data, alg, e["w"], e["min"], e["max"])
        byte_shares(data, b, alg, e["w"], e["min"], e["max"])
        torch.cuda.synchronize()
        e0.record()
        es, rb = byte_shares(data, b, alg, e["w"], e["min"], e["max"])
        e1.record()
        torch.cuda.synchronize()
        shares[alg] = {"ebs_pct": round(100.0 * es / max(1, es + rb), 2), "rs_pct": round(100.0 * rb / max(1, es + rb), 2),
                       "ebs_bytes": es, "rs_bytes": rb, "ms": round(e0.elapsed_time(e1), 3)}
    out["byte_shares_8k"] = shares
    # chunk-size distributions of the four algorithms on the whole stream
    out["size_cdf_8k"] = {}
    for alg in ("ram", "ae", "ae_min", "maxp"):
        e = wtable()["mixed_4g_seed1"]["ae" if alg == "ae_min" else alg]["8192"]
        out["size_cdf_8k"][alg] = size_cdf([chunk(data, alg, e["w"], e["min"], e["max"])])
    return out


def dedup_workload(dev, base_bytes: int = GIB, n_versions: int = 15, reps: int = 2):
    """Dedup-shaped versions: a uniform base (seed 2) and 15 versions, each
    0.1% of its predecessor's bytes edited (seeded insert / delete /
    overwrite runs of 1..512 bytes), chunked piece by piece (one call per
    version, device resident) with AE and RAM at 8 KiB mean; then GPU
    fingerprints and the unique-chunk ratio and space savings (Eq. 1)."""
    import torch

    import synth
    from paper_2508_05797_gb300 import Chunker, dedup_report

    vs = synth.versions(2, base_bytes, n_versions)
    dv = [torch.from_numpy(v).to(dev) for v in vs]
    total = sum(v.size for v in vs)
    del vs
    t = wtable()["uniform_16m_seed0"]
    res = {"workload": "uniform base of %d MiB (seed 2) + %d versions with 0.1%% edits, %.2f GB, one call per version"
                       % (base_bytes >> 20, n_versions, total / 1e9)}
    for alg in ("ae", "ram"):
        e = t[alg]["8192"]
        ck = Chunker(dev.index)
        outs = [torch.empty(d.numel() // e["min"] + 2, dtype=torch.int64, device=dev) for d in dv]
        cnts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in dv]
        for d, o, c in zip(dv, outs, cnts):  # warm-up: workspace sized
            ck.chunk_async(d, alg, e["w"], e["min"], e["max"], o, c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            for d, o, c in zip(dv, outs, cnts):
                ck.chunk_async(d, alg, e["w"], e["min"], e["max"], o, c)
        e1.record()
        torch.cuda.synchronize()
        ck.sync_status()
        ms = e0.elapsed_time(e1) / reps
        pieces = [(d, o[:int(c.item())]) for d, o, c in zip(dv, outs, cnts)]
        rep = dedup_report(pieces)
        res[alg] = {"GBps": round(total / (ms / 1e3) / 1e9, 1), "ms": round(ms, 2), "chunks": rep["chunks"],
                    "unique_chunks": rep["unique_chunks"], "unique_ratio": round(rep["unique_chunks"] / rep["chunks"], 5),
                    "savings_pct": round(100 * rep["savings"], 3), "mean_chunk": round(rep["mean_size"], 1),
                    "size_quantiles": rep["size_quantiles"]}
        res[alg]["size_cdf"] = size_cdf([b for _, b in pieces])
        ck.close()
        del outs, cnts, pieces
    # the other two algorithms' chunk-size distributions (untimed)
    for alg in ("ae_min", "maxp"):
        e = t["ae" if alg == "ae_min" else alg]["8192"]
        ck = Chunker(dev.index)
        res.setdefault("size_cdf_other", {})[alg] = size_cdf([ck.chunk(d, alg, e["w"], e["min"], e["max"]) for d in dv])
        ck.close()
    del dv
    torch.cuda.empty_cache()
    return res


def small_workload(dev, copies: int = 16, reps: int = 5):
    """Single 16 MiB buffers chunked with RAM, AE and MAXP at 8 KiB mean:
    uniform bytes (seed 0, windows calibrated on them) and the first 16 MiB of
    the mixed stream. A call this small is bound by the latency of its kernel
    sequence, not by HBM: 16 calls on 16 copies of the buffer (256 MiB, more
    than L2) are captured in one CUDA graph, replayed, and the time per call is
    the replay time / 16 (cold); `warm_*` repeats one copy 16 times (its bytes
    resident in L2)."""
    import torch

    import synth

    n = 16 * MIB
    res = {"workload": "16 MiB buffers, one call per buffer; %d calls on %d copies in one CUDA graph, "
                       "time per call = replay time / %d; `uniform`: uniform bytes (seed 0, windows calibrated on "
                       "them), `mixed_prefix`: the first 16 MiB of the 4 GiB mixed stream" % (copies, copies, copies)}
    res["uniform"] = _small_calls(dev, torch.from_numpy(synth.uniform(0, n)), wtable()["uniform_16m_seed0"],
                                  copies, reps)
    res["mixed_prefix"] = _small_calls(dev, torch.from_numpy(synth.mixed_range(1, STREAM_LEN, 0, n)),
                                       wtable()["mixed_4g_seed1"], copies, reps)
    torch.cuda.empty_cache()
    return res


def _small_calls(dev, host_buf, t, copies, reps):
    import torch

    from paper_2508_05797_gb300 import Chunker

    n = host_buf.numel()
    buf = host_buf.to(dev)
    ds = [buf.clone() for _ in range(copies)]
    del buf
    s = torch.cuda.Stream(dev)
    res = {}
    peak, _ = peaks()
    for alg in ALGS:
        e = t[alg]["8192"]
        w, mn, mx = e["w"], e["min"], e["max"]
        ck = Chunker(dev.index)
        ck.reserve(alg, w, mn, mx, n)
        outs = [torch.empty(n // mn + 1, dtype=torch.int64, device=dev) for _ in range(copies)]
        cnts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(copies)]

        def calls():
            for d, o, c in zip(ds, outs, cnts):
                ck.chunk_async(d, alg, w, mn, mx, o, c, stream=s)

        with torch.cuda.stream(s):
            calls()
        s.synchronize()
        ck.sync_status(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            calls()
        ts = []
        with torch.cuda.stream(s):
            for r in range(reps + 2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                g.replay()
                b.record(s)
                s.synchronize()
                if r >= 2:
                    ts.append(a.elapsed_time(b) / copies)
        ck.sync_status(s)
        counts = {int(c.item()) for c in cnts}
        if len(counts) != 1:
            raise RuntimeError("small workload: copies of one buffer gave different boundary counts")
        ms = statistics.median(ts)
        # warm: the same buffer (and its summaries) 16 times, resident in L2
        gw = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gw, stream=s):
            for o, c in zip(outs, cnts):
                ck.chunk_async(ds[0], alg, w, mn, mx, o, c, stream=s)
        tw = []
        with torch.cuda.stream(s):
            for r in range(reps + 2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                gw.replay()
                b.record(s)
                s.synchronize()
                if r >= 2:
                    tw.append(a.elapsed_time(b) / copies)
        ck.sync_status(s)
        msw = statistics.median(tw)
        res[alg] = {"us_per_call": round(ms * 1e3, 1), "GBps": round(n / (ms / 1e3) / 1e9, 1),
                    "hbm_frac": round(n / (ms / 1e3) / 1e9 / peak, 4), "boundaries": counts.pop(), "w": w,
                    "launches_per_call": ck.last_launches(), "chain_stage": ck.last_stage(),
                    "warm_us_per_call": round(msw * 1e3, 1), "warm_GBps": round(n / (msw / 1e3) / 1e9, 1)}
        del g, gw
        ck.close()
    del ds
    return res


def stream_workload(data, dev, pieces_mib=(64, 256), reps: int = 2):
    """Resumable chunking (cdc_feed_*): the 4 GiB mixed stream handed over in
    device pieces of a fixed size, RAM and MAXP at 8 KiB mean; GB/s of stream
    bytes over the whole feed (piece copies into staging and one
    synchronisation per push included), against one call on the whole
    stream; `same` checks that the pushes concatenate to the one-call
    boundaries."""
    import torch

    from paper_2508_05797_gb300 import Chunker, Feed

    n = data.numel()
    t = wtable()["mixed_4g_seed1"]
    res = {"workload": "the %d MiB mixed stream pushed in fixed-size device pieces" % (n >> 20)}
    ck = Chunker(dev.index)
    for alg in ("ram", "maxp"):
        e = t[alg]["8192"]
        w, mn, mx = e["w"], e["min"], e["max"]
        whole = ck.chunk(data, alg, w, mn, mx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        whole = ck.chunk(data, alg, w, mn, mx)
        e1.record()
        torch.cuda.synchronize()
        r = {"one_call_GBps": round(n / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)}
        f = Feed(ck, alg, w, mn, mx)
        for pm in pieces_mib:
            piece = pm * MIB
            best, same = None, True
            for rep in range(reps + 1):  # the first pass sizes the staging buffers
                f.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                got = []
                for pos in range(0, n, piece):
                    got.append(f.push(data[pos:pos + piece], final=pos + piece >= n))
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if rep:
                    best = dt if best is None else min(best, dt)
                same = same and bool(torch.equal(torch.cat(got), whole))
            r["piece_%dMiB" % pm] = {"GBps": round(n / best / 1e9, 1), "pushes": (n + piece - 1) // piece,
                                     "same": same}
        f.close()
        res[alg] = r
    ck.close()
    torch.cuda.empty_cache()
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    import synth
    sample = args.ref_sample_mib * MIB
    data = synth.mixed_range(1, STREAM_LEN, 0, sample)
    cfg = configs()

    def step():
        for alg, mean, w, mn, mx in cfg:
            oracle.count(alg, data, w, mn, mx)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    gbs = 9 * sample * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "sample_bytes_per_step": 9 * sample},
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first %d MiB of the 4 GiB mixed stream per (alg, mean) pair, one thread"
                                       % args.ref_sample_mib},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--batched-files", type=int, default=100_000)
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-prims", action="store_true", help="skip the EBS / RS measurement")
    ap.add_argument("--no-dedup", action="store_true", help="skip the dedup-shaped versions measurement")
    ap.add_argument("--no-stream", action="store_true", help="skip the resumable-feed measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 16 MiB single-buffer (latency) measurement")
    ap.add_argument("--streams", type=int, default=3, help="streams the nine calls of a step are spread over")
    ap.add_argument("--ref-sample-mib", type=int, default=32, help="reference arm: bytes per (alg, mean) pair")
    ap.add_argument("--serving-requests", type=int, default=20_000)
    ap.add_argument("--algs", default=",".join(ALGS), help="subset of ram,ae,maxp (profiling cases)")
    ap.add_argument("--means", default=",".join(map(str, MEANS)), help="subset of 4096,8192,16384")
    ap.add_argument("--len-mib", type=int, default=STREAM_LEN // MIB,
                    help="stream length (a prefix of the 4 GiB stream; profiling cases)")
    ap.add_argument("--pipeline", type=int, default=0,
                    help="chain stage: 0 automatic, 1 speculative segments, 2 candidate graph (profiling cases)")
    ap.add_argument("--write-traffic", metavar="CSV",
                    help="write the k_spec DRAM-traffic record from an ncu CSV of a --len-mib run and exit")
    ap.add_argument("--traffic-command", default="", help="the ncu command that made the CSV (recorded)")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(args.write_traffic, args.len_mib * MIB, args.traffic_command)
        return 0
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import synth
    from paper_2508_05797_gb300 import Chunker
    from paper_2508_05797_gb300.cdc import OPT_PROFILE

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seed = 1 + rank
    n = args.len_mib * MIB
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    synth.mixed_range(seed, STREAM_LEN, 0, n, out=host.numpy())
    data = host.to(dev, non_blocking=False)
    cfg = configs(tuple(args.algs.split(",")), tuple(int(x) for x in args.means.split(",")))
    ncfg = len(cfg)
    handles, outs, counts = [], [], []
    from paper_2508_05797_gb300.cdc import OPT_PIPELINE
    for alg, mean, w, mn, mx in cfg:
        ck = Chunker(local)
        ck.set_option(OPT_PIPELINE, args.pipeline)
        ck.reserve(alg, w, mn, mx, n)
        handles.append(ck)
        outs.append(torch.empty(n // mn + 1, dtype=torch.int64, device=dev))
        counts.append(torch.zeros(1, dtype=torch.int64, device=dev))
    stream = torch.cuda.current_stream(dev)
    # the nine calls are independent (one handle each): spread them over a few
    # streams so that one call's latency-bound kernels overlap another's
    nstreams = max(1, args.streams)
    side = [torch.cuda.Stream(dev) for _ in range(nstreams)]
    fork = [torch.cuda.Event() for _ in range(nstreams)]
    join = [torch.cuda.Event() for _ in range(nstreams)]

    def step():
        if nstreams == 1:
            for (alg, mean, w, mn, mx), ck, o, c in zip(cfg, handles, outs, counts):
                ck.chunk_async(data, alg, w, mn, mx, o, c, stream=stream)
            return
        for i in range(nstreams):
            fork[i].record(stream)
            side[i].wait_event(fork[i])
        for k, ((alg, mean, w, mn, mx), ck, o, c) in enumerate(zip(cfg, handles, outs, counts)):
            ck.chunk_async(data, alg, w, mn, mx, o, c, stream=side[k % nstreams])
        for i in range(nstreams):
            join[i].record(side[i])
            stream.wait_event(join[i])

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    for ck in handles:
        ck.sync_status(stream)
        ck.set_option(OPT_PROFILE, 1)
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    ms = allreduce_max(ms, world)
    for ck in handles:
        ck.sync_status(stream)
    per_cfg = []
    launches = 0
    spec_ms_total, spec_calls = 0.0, 0
    for (alg, mean, w, mn, mx), ck, c in zip(cfg, handles, counts):
        calls, sms, cms, pms, l = ck.profile_collect()
        ck.set_option(OPT_PROFILE, 0)
        launches += l
        spec_ms_total += pms
        spec_calls += calls
        per_cfg.append({"alg": alg, "mean": mean, "w": w, "calls": calls, "summary_ms": sms / max(calls, 1),
                        "chain_ms": cms / max(calls, 1), "spec_ms": pms / max(calls, 1),
                        "boundaries": int(c.item())})
    total_bytes = ncfg * n * args.steps * world
    gbs = total_bytes / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    # each call alone on one stream (after the timed region): per-algorithm
    # throughput and the speculation kernel's own launch time, free of the
    # overlap between the step's three streams
    iso = []
    for (alg, mean, w, mn, mx), ck, o, c in zip(cfg, handles, outs, counts):
        ck.set_option(OPT_PROFILE, 1)
        for _ in range(2):
            ck.chunk_async(data, alg, w, mn, mx, o, c, stream=stream)
        torch.cuda.synchronize()
        calls, sms, cms, pms, _ = ck.profile_collect()
        ck.set_option(OPT_PROFILE, 0)
        ck.sync_status(stream)
        iso.append({"alg": alg, "summary_ms": sms / max(calls, 1), "chain_ms": cms / max(calls, 1),
                    "spec_ms": pms / max(calls, 1)})
    per_alg = {}
    for alg in ALGS:
        rows = [r for r in iso if r["alg"] == alg]
        t = sum(r["summary_ms"] + r["chain_ms"] for r in rows)
        if not rows:
            continue
        per_alg[alg] = {"GBps": round(len(rows) * n / (t / 1e3) / 1e9, 1),
                        "hbm_frac": round(len(rows) * n / (t / 1e3) / 1e9 / peak, 4),
                        "summary_ms": [round(r["summary_ms"], 4) for r in rows],
                        "chain_ms": [round(r["chain_ms"], 4) for r in rows],
                        "spec_ms": [round(r["spec_ms"], 4) for r in rows]}
    # roofline of the dominant kernel, k_spec (the speculation kernel of the
    # chain stage): algorithmic bytes = the input bytes one launch chunks
    # (the chain stage's one pass over the stream); its launch times from the
    # calls alone on one stream (no other call's kernels on the GPU during a
    # launch), and from the timed region for comparison (three streams overlap
    # there). k_spec is bound by the latency of dependent chain steps, not by
    # DRAM (its own DRAM traffic, `traffic`, is under 0.1 byte per input
    # byte); the block-summary kernel is the one that streams every byte.
    spec_avg_ms = spec_ms_total / max(1, spec_calls)
    achieved_tr = n / (spec_avg_ms / 1e3) / 1e9
    iso_spec_ms = sum(r["spec_ms"] for r in iso) / max(1, len(iso))
    iso_achieved = n / (iso_spec_ms / 1e3) / 1e9
    iso_sum_ms = sum(r["summary_ms"] for r in iso) / max(1, len(iso))
    sum_achieved = n / (iso_sum_ms / 1e3) / 1e9
    # the two summary kernels apart: RAM/AE (maxima) and MAXP (targets)
    sum_kernels = {}
    for kn, algs in (("k_summary_max", ("ram", "ae")), ("k_summary_maxp", ("maxp",))):
        rows = [r["summary_ms"] for r in iso if r["alg"] in algs and r["summary_ms"] > 0]
        if rows:
            kms = sum(rows) / len(rows)
            sum_kernels[kn] = {"achieved": round(n / (kms / 1e3) / 1e9, 1),
                               "frac": round(n / (kms / 1e3) / 1e9 / peak, 4), "avg_launch_ms": round(kms, 4)}
    # which chain stage the calls took (the automatic policy: the candidate
    # graph up to 512 MiB, 768 MiB for AE; speculation beyond)
    stages = sorted({ck.last_stage() for ck in handles})
    graph = stages == [2]
    dpb = profile_traffic() if stages == [1] else None
    kname = ("k_gcand + k_glocal (chain stage: candidates, F and pointer jumping of the candidate graph)" if graph
             else "k_spec (chain stage: speculative chains), the largest share of the step's device time"
             if stages == [1] else "k_spec or k_gcand + k_glocal (chain stage; the calls took both stages)")
    roofline = {"bound": "hbm", "achieved": round(iso_achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(iso_achieved / peak, 4), "traffic": int(dpb * n) if dpb is not None else None,
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "kernel": kname, "chain_stage": "graph" if graph else "speculation" if stages == [1] else "both",
                "algorithmic_bytes_per_launch": n, "avg_launch_ms": round(iso_spec_ms, 4),
                "launch_times": "each call alone on one stream, CUDA events around the kernel",
                "limited_by": "latency of dependent chain steps (its DRAM traffic is `traffic`)",
                "timed_region": {"achieved": round(achieved_tr, 1), "frac": round(achieved_tr / peak, 4),
                                 "avg_launch_ms": round(spec_avg_ms, 4),
                                 "note": "the step's nine calls overlap on %d streams" % nstreams},
                "summary_kernel": {"kernel": "k_summary_max / k_summary_maxp (block summaries: reads every byte)",
                                   "achieved": round(sum_achieved, 1), "frac": round(sum_achieved / peak, 4),
                                   "avg_launch_ms": round(iso_sum_ms, 4), "per_kernel": sum_kernels}}
    line = {"metric": METRIC, "value": round(gbs, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD if ncfg == 9 and n == STREAM_LEN else
                       "%s; subset algs=%s means=%s, first %d MiB" % (WORKLOAD, args.algs, args.means, args.len_mib),
                       "bytes_per_step": ncfg * n,
                       "l2": "inputs larger than L2 (4 GiB per call, 129 MB L2)",
                       "streams": nstreams,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "hbm_frac": round(gbs / world / peak, 4), "per_alg": per_alg,
            "per_alg_timing": "each call alone on one stream, after the timed region", "roofline": roofline,
            "gpu_launches": int(launches), "clocks": clocks}
    # end to end through the host entry point (pinned host memory in, host boundaries out)
    if not args.no_e2e:
        outs_h = [np.empty(n // mn + 1, dtype=np.uint64) for (_, _, _, mn, _) in cfg]
        hnp = host.numpy()
        d2h = 0
        # the same nine calls from one host thread per stream (a handle is used
        # by one thread), so one call's copies overlap another call's kernels
        from concurrent.futures import ThreadPoolExecutor

        def lane(j, steps):
            got = 0
            for _ in range(steps):
                for k in range(j, ncfg, nstreams):
                    alg, mean, w, mn, mx = cfg[k]
                    b = handles[k].chunk_host(hnp, alg, w, mn, mx, out=outs_h[k], stream=side[j])
                    got += b.size * 8
            return got

        with ThreadPoolExecutor(nstreams) as ex:  # untimed: sizes each handle's staging buffers
            list(ex.map(lambda j: lane(j, 1), range(nstreams)))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        with ThreadPoolExecutor(nstreams) as ex:
            d2h = sum(ex.map(lambda j: lane(j, e2e_steps), range(nstreams))) // e2e_steps
        torch.cuda.synchronize()
        dt = allreduce_max(time.perf_counter() - t0, world)
        line["e2e"] = {"value": round(ncfg * n * e2e_steps * world / dt / 1e9, 2), "unit": "GB/s",
                       "h2d_bytes_per_step": ncfg * n, "d2h_bytes_per_step": int(d2h),
                       "steps": e2e_steps, "host_threads": nstreams,
                       "path": "cdc_chunk_host (pinned host bytes in, host boundaries out), one thread and "
                               "stream per group of calls"}
    if rank == 0 and not args.no_small:
        line["small"] = small_workload(dev)
    if rank == 0 and not args.no_stream:
        line["stream"] = stream_workload(data, dev)
    if rank == 0 and not args.no_dedup:
        line["dedup"] = dedup_workload(dev)
    if rank == 0 and not args.no_prims:
        line["prims"] = prims_workload(data, dev)
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_workload(host, dev, n_req=args.serving_requests)
        # the same with batches capped at 256 requests: lower saturation, shorter tails
        line["serving_capped"] = serving_workload(host, dev, n_req=args.serving_requests, max_batch=256)
    if rank == 0 and not args.no_batched:
        for ck in handles:
            ck.close()
        handles = []
        del data
        torch.cuda.empty_cache()
        line["batched"] = batched_workload(dev, n_files=args.batched_files)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    for ck in handles:
        ck.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
