"""Benchmark of the FPTC batch decoder on one GB300 (or N, one process per GPU).

One step = one decode of the whole batch: SymLen index + fused Huffman decode,
dequantization, inverse DCT and window reassembly of every stream, with the
compressed streams already in GPU memory (the paper's timed region, Sec. 5.1).

Workload (default): 10,000 synthetic signals with log-uniform lengths in
[4096, 4194304] samples, 2,500 per domain (EEG-like, seismic, power-grid,
meteorological), Table 1 parameters, encoded on the host by the library's own
encoder with tables trained on disjoint seeds.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

--impl reference times the FP64 CPU oracle decoder on the host cores on a
bounded sample of the same workload (the reference arm of this build).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import siggen  # noqa: E402

METRIC = "decoded GB/s (float32 out)"
UNIT = "GB/s"
PARAMS = dict(N=32, E=16, B1=2, B2=16, mu=50.0, alpha1=0.004, lmax=12, percentile=99.9)
L2_BYTES = 129 * 2 ** 20


def workload(name: str, rank: int = 0) -> siggen.Workload:
    """The named workload; rank r > 0 gets a copy of the same shape with other seeds
    (weak scaling: every rank decodes a batch of its own)."""
    if name == "mixed":
        wl = siggen.mixed_10000_logu()
    elif name == "eeg2048":
        wl = siggen.eeg_2048x1m()
    elif name == "seismic":
        wl = siggen.seismic_16384x4096()
    elif name == "power":
        wl = siggen.power_1024x65536()
    elif name == "eeg1":
        wl = siggen.eeg_1x65536()
    elif name == "mixed_small":
        wl = siggen.mixed_10000_logu(n=400, lo=4096, hi=262144)
    elif name == "mixed_medium":
        wl = siggen.mixed_10000_logu(n=2000, lo=4096, hi=524288)
    else:
        raise SystemExit(f"unknown workload {name}")
    if rank:  # weak scaling: every rank decodes its own batch of the same shape, other seeds
        wl.seeds = np.array([siggen.splitmix64(int(s) + 0x9E3779B97F4A7C15 * rank & (2 ** 64 - 1))
                             for s in wl.seeds], dtype=np.uint64)
    return wl


def workload_config(wl: siggen.Workload) -> dict:
    """The workload as both arms report it (the same keys and values in each)."""
    n = int(wl.n_samples)
    return {"workload": wl.name, "n_streams": int(wl.n_streams), "n_samples": n, "out_bytes": 4 * n,
            "params": PARAMS, "domains": "eeg,seismic,power,met",
            "l2": (f"no flush: the output alone is {4 * n / 2 ** 30:.1f} GiB >> L2 129 MB" if 4 * n > 8 * L2_BYTES
                   else f"output {4 * n / 2 ** 20:.0f} MiB, not far above the 129 MB L2: not a roofline size")}


def subset_batch(batch, idx):
    """The streams idx of a batch, words packed again from 0 and outputs packed at 128 bytes."""
    from paper_2605_01086_gb300 import codec
    segs = batch.segments[np.asarray(idx, dtype=np.int64)]
    nw = segs["n_words"].astype(np.uint64)
    woff = np.zeros(len(segs), np.uint64)
    if len(segs) > 1:
        woff[1:] = np.cumsum(nw[:-1])
    words = np.concatenate([batch.words[int(a):int(a) + int(b)] for a, b in zip(segs["word_offset"], nw)]) \
        if len(segs) else np.zeros(0, np.uint64)
    symlen = np.concatenate([batch.symlen[int(a):int(a) + int(b)] for a, b in zip(segs["word_offset"], nw)]) \
        if len(segs) else np.zeros(0, np.uint8)
    lengths = segs["n_samples"].astype(np.uint64)
    out = codec.segments_array(woff, nw, lengths, codec.packed_out_offsets(lengths), segs["domain"])
    return codec.Batch(words, symlen, out, batch.domains)


def train_tables():
    from paper_2605_01086_gb300 import codec
    doms = []
    for d in range(4):
        ts = siggen.training_set(d)
        flat, offs = siggen.signals(ts.domains, ts.seeds, ts.lengths)
        p = PARAMS
        doms.append(codec.train_domain(flat, offs, ts.lengths, p["N"], p["E"], p["B1"], p["B2"], p["mu"],
                                       p["alpha1"], p["lmax"], p["percentile"]))
    return doms


def encode(wl: siggen.Workload, doms, chunk_samples: int = 1 << 29, keep=None):
    """Generate + encode in chunks of about chunk_samples samples (bounded host memory);
    keep(first, last, flat, offsets), if given, receives each chunk's signals."""
    from paper_2605_01086_gb300 import codec
    parts = []
    i = 0
    n = wl.n_streams
    while i < n:
        j = i
        acc = 0
        while j < n and (acc < chunk_samples or j == i):
            acc += int(wl.lengths[j])
            j += 1
        sub = wl.subset(np.arange(i, j))
        flat, offs = siggen.signals(sub.domains, sub.seeds, sub.lengths)
        parts.append(codec.encode_batch(doms, flat, offs, sub.lengths, sub.domains.astype(np.uint32)))
        if keep is not None:
            keep(i, j, flat, offs)
        del flat
        i = j
    words = np.concatenate([p.words for p in parts])
    symlen = np.concatenate([p.symlen for p in parts])
    nw = np.concatenate([p.segments["n_words"] for p in parts])
    woff = np.zeros(n, np.uint64)
    woff[1:] = np.cumsum(nw[:-1])
    segs = codec.segments_array(woff, nw, wl.lengths, codec.packed_out_offsets(wl.lengths), wl.domains)
    return codec.Batch(words, symlen, segs, doms)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {1: ["decode.cu"], 2: ["decode_fixed.cu"],
                  3: ["decode_warp.cu", "warp_tile.cuh", "symlen_chunks.cuh", "device_util.cuh"],
                  4: ["decode_tc.cu", "tc_ops.cuh", "warp_tile.cuh", "symlen_chunks.cuh", "device_util.cuh"],
                  5: ["backward_warp.cu", "dct32.cuh", "warp_tile.cuh", "symlen_chunks.cuh", "device_util.cuh"]}


def _kernel_source_hash(kind: int):
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES.get(kind, ["decode.cu"]):
        with open(os.path.join(ROOT, "paper_2605_01086_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kind: int, n_samples: int):
    """DRAM bytes per launch from the committed ncu summary (profiles/dram_traffic.txt:
    'kind sha1 bytes_per_sample'), scaled to this launch; None if the kernel changed since.
    Kinds: 1-4 the decode kernels (fptc_kernel), 5 the warp-tile adjoint."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    h = _kernel_source_hash(kind)
    for line in open(p):
        f = line.split("#", 1)[0].split()
        if len(f) == 3 and int(f[0]) == kind and f[1] == h:
            return float(f[2]) * n_samples
    return None


def oracle_sample_time(batch, idx, n_threads):
    """Times the FP64 CPU oracle decoder on the streams idx (OpenMP over streams)."""
    import oracle
    ods = [oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(d.scale), d.lmax, d.code_len)
           for d in batch.domains]
    segs = batch.segments
    ob = oracle.EncodedBatch(batch.words, batch.symlen, segs["word_offset"].copy(), segs["n_words"].copy(),
                             segs["n_samples"].copy(), segs["domain"].astype(np.int32), ods)
    t = time.perf_counter()
    oracle.decode_many(ob, idx, n_threads=n_threads)
    return time.perf_counter() - t


def cpu_sample(batch, target_s: float, seed: int = 0):
    """A bounded random sample of streams sized for about target_s seconds of oracle time."""
    n_threads = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(batch.segments))
    S = batch.segments["n_samples"].astype(np.float64)
    # calibrate on ~1/200 of the samples
    k = 1
    while k < len(order) and S[order[:k]].sum() < S.sum() / 200:
        k += 1
    t = oracle_sample_time(batch, order[:k], n_threads)
    rate = S[order[:k]].sum() / max(t, 1e-6)  # samples / s
    want = rate * target_s
    m = int(np.searchsorted(np.cumsum(S[order]), want)) + 1
    return order[:min(m, len(order))], n_threads


def oracle_encode(wl: siggen.Workload, idx, odoms):
    """Generates the streams idx of a workload and encodes them with the oracle's encoder."""
    import oracle
    sub = wl.subset(np.asarray(idx))
    flat, offs = siggen.signals(sub.domains, sub.seeds, sub.lengths)
    return oracle.encode_many(flat, offs, sub.lengths, sub.domains, odoms)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle (its own trainer, encoder and decoder;
    nothing of the library) on the host cores, a bounded random sample of the
    workload's streams per step."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args.workload)
    p = PARAMS
    odoms = [oracle.trained_domain(d, p["N"], p["E"], p["B1"], p["B2"], p["mu"], p["alpha1"], p["lmax"],
                                   p["percentile"]) for d in range(4)]
    n_threads = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    order = rng.permutation(wl.n_streams)
    S = wl.lengths.astype(np.float64)
    # calibrate the oracle's decode rate on ~1/400 of the samples, then size the sample
    k = 1
    while k < len(order) and S[order[:k]].sum() < S.sum() / 400:
        k += 1
    cal = oracle_encode(wl, order[:k], odoms)
    t = time.perf_counter()
    oracle.decode_many(cal, n_threads=n_threads)
    rate = S[order[:k]].sum() / max(time.perf_counter() - t, 1e-6)
    m = int(np.searchsorted(np.cumsum(S[order]), rate * args.ref_seconds)) + 1
    idx = np.sort(order[:min(m, len(order))])
    ob = oracle_encode(wl, idx, odoms)
    samples = int(ob.lengths.sum())

    def step(sel=None):
        t0 = time.perf_counter()
        oracle.decode_many(ob, sel, n_threads=n_threads)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step(np.arange(max(1, len(idx) // 8)))
    ts = [step() for _ in range(args.steps)]
    ms = 1000 * statistics.mean(ts)
    value = 4.0 * samples / (ms / 1000) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                             "sample": f"{len(idx)} random streams of the {wl.n_streams}, {samples} samples per "
                                       "step, encoded by the oracle's own encoder with its own trained tables; "
                                       "FP64 bit-serial decode, OpenMP over streams"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(fn, steps, stream, torch):
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run(args):
    import torch

    from paper_2605_01086_gb300 import STAGE_DECODE, STAGE_INDEX, STAGE_LOSSLESS, STAGE_LOSSY, Plan

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    t_setup = time.perf_counter()
    # weak scaling: every rank decodes a batch of the workload's shape of its own;
    # strong scaling: the one batch, cut by LPT on each stream's bytes (4 S + 9 n_words)
    wl = workload(args.workload, rank if args.scaling == "weak" else 0)
    doms = train_tables()
    # the original signals at the decoder's output layout, for the GPU encoder's line
    x_orig = None
    keep = None
    if not args.no_encode and rank == 0 and not (world > 1 and args.scaling == "strong"):
        from paper_2605_01086_gb300 import codec as _codec
        x_off = _codec.packed_out_offsets(wl.lengths)
        x_orig = torch.zeros(int(x_off[-1] + wl.lengths[-1]) if wl.n_streams else 1, dtype=torch.float32,
                             device=dev)

        def keep(i, j, flat, offs):
            base = int(x_off[i])
            span = np.zeros(int(x_off[j - 1] + wl.lengths[j - 1]) - base, np.float32)
            for t in range(i, j):
                o, n = int(x_off[t]) - base, int(wl.lengths[t])
                span[o:o + n] = flat[int(offs[t - i]):int(offs[t - i]) + n]
            x_orig[base:base + span.size].copy_(torch.from_numpy(span))
    batch = encode(wl, doms, keep=keep)
    mine = np.arange(wl.n_streams)  # workload index of each stream of this rank's batch
    if world > 1 and args.scaling == "strong":
        from paper_2605_01086_gb300.shard import decode_cost, shard_streams
        mine = shard_streams(decode_cost(batch.segments["n_samples"], batch.segments["n_words"]), world, rank)
        batch = subset_batch(batch, mine)
    t_encode = time.perf_counter() - t_setup
    n_samples = batch.n_samples
    out_bytes = 4 * n_samples
    in_bytes = 9 * int(batch.segments["n_words"].sum())
    job_out_bytes = out_bytes  # summed over ranks below
    if dist:
        t = torch.tensor([float(out_bytes)], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        job_out_bytes = int(t.item())

    t0 = time.perf_counter()
    plan = Plan(doms, batch.segments, device=local, kernel=args.kernel or "auto", threads=args.threads,
                idct=args.idct)
    if args.kernel:
        args.no_autotune = True
    t_plan = time.perf_counter() - t0
    w, s = plan.to_device(batch.words, batch.symlen)
    out = plan.empty_out().zero_()
    stream = torch.cuda.Stream(dev)
    tuned, tuned_ms = None, None
    with torch.cuda.stream(stream):
        if not args.no_autotune:
            tuned, tuned_ms = plan.autotune(w, s, out, trials=3, stream=stream)
        plan.decode(w, s, out=out, stream=stream)
    torch.cuda.synchronize()
    if plan.device_status()[0] != 0:
        raise SystemExit("device reported a corrupt stream")

    # one step = the index graph then the decode graph (each one CUDA graph of
    # that stage's launches), with events around each on the launching stream:
    # the dominant kernel's duration is measured inside the timed region itself
    g_idx, g_dec = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_idx, stream=stream):
        plan.decode_stages(w, s, out, STAGE_INDEX, stream=stream)
    with torch.cuda.graph(g_dec, stream=stream):
        plan.decode_stages(w, s, out, STAGE_DECODE, stream=stream)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            g_idx.replay()
            g_dec.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        start.record(stream)
        for a, b, c in evs:
            a.record(stream)
            g_idx.replay()
            b.record(stream)
            g_dec.replay()
            c.record(stream)
        end.record(stream)
    torch.cuda.synchronize()
    total_ms = start.elapsed_time(end)
    trials = [a.elapsed_time(c) for a, b, c in evs]
    idx_ms = [a.elapsed_time(b) for a, b, c in evs]
    dec_ms = [b.elapsed_time(c) for a, b, c in evs]
    clk = clocks.stop()
    if dist:
        dist.barrier()
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = job_out_bytes / (ms_per_step / 1e3) / 1e9
    rank_value = out_bytes / (ms_per_step / 1e3) / 1e9  # this rank's own batch
    if plan.device_status()[0] != 0:
        raise SystemExit("device reported a corrupt stream")

    # accuracy: PRD of a few streams against their original signals
    idx = np.random.default_rng(1).choice(len(mine), size=min(8, len(mine)), replace=False)
    num = den = 0.0
    for i in idx:
        j = int(mine[i])
        x = siggen.signal(int(wl.domains[j]), int(wl.seeds[j]), int(wl.lengths[j])).astype(np.float64)
        xh = plan.segment_view(out, int(i)).double().cpu().numpy()
        num += float(np.sum((x - xh) ** 2))
        den += float(np.sum(x ** 2))
    prd = 100.0 * (num / den) ** 0.5

    peak, peak_kind = measured_peaks()
    dec_avg = statistics.mean(dec_ms)
    kernel_names = {1: "k_decode (generic)", 2: "k_decode_fixed (block tile)", 3: "k_decode_warp (warp tile)",
                    4: "k_decode_tc (tensor core, %s)" % args.idct}
    kname = kernel_names.get(plan.info["kernel"], "?")
    traffic = args.traffic if args.traffic is not None else measured_traffic(plan.info["kernel"], n_samples)
    achieved = (out_bytes + in_bytes) / (dec_avg / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind, "traffic": traffic, "kernel": kname,
                "algorithmic_bytes_per_launch": out_bytes + in_bytes, "launch_ms": dec_avg,
                "index_ms": statistics.mean(idx_ms), "nominal_frac": achieved / 7900.0}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": args.scaling,
            "vs_baseline": None, "dtype": "f32" if args.idct == "fp32" else "f32 (%s products)" % args.idct,
            "data": "synthetic",
            "config": workload_config(wl),
            "run": {"streams_on_rank0": int(len(mine)), "samples_on_rank0": int(n_samples),
                    "compressed_bytes_rank0": in_bytes, "schedule": "persistent, CUDA graph", "tuning": tuned,
                    "sharding": ("LPT on 4 S + 9 n_words of the one batch" if args.scaling == "strong" and world > 1
                                 else "one batch of the workload's shape per rank" if world > 1 else "one GPU"),
                    "setup_s": {"generate_encode": round(t_encode, 1), "plan": round(t_plan, 3)}},
            "trials_ms": {"median": statistics.median(trials), "mean": statistics.mean(trials), "min": min(trials),
                          "max": max(trials), "n": len(trials)},
            "roofline": roofline, "gpu_launches": args.steps * plan.launches_per_decode, "clocks": clk,
            "prd_percent_sample": prd}

    # tensor-core forms of the inverse transform on the same streams: throughput
    # (index + decode per step, and the decode kernel alone against the roofline)
    # and relative L2 distance to the FP32 output (the FP64 comparison is in the tests)
    if not args.no_forms and rank == 0:
        forms = {}
        ref = out.clone()
        for idct in ("tf32x3", "bf16x3", "tf32"):
            fplan = Plan(doms, batch.segments, device=local, idct=idct)
            out3 = torch.zeros_like(out)
            with torch.cuda.stream(stream):
                fplan.autotune(w, s, out3, trials=2, stream=stream)
                fplan.decode(w, s, out=out3, stream=stream)
                fms = time_steps(lambda: fplan.decode(w, s, out=out3, stream=stream), 5, stream, torch)
                kms = time_steps(lambda: fplan.decode_stages(w, s, out3, STAGE_DECODE, stream=stream), 5, stream,
                                 torch)
            torch.cuda.synchronize()
            rel = float(torch.linalg.vector_norm((out3 - ref).double()) / torch.linalg.vector_norm(ref.double()))
            ka = (out_bytes + in_bytes) / (statistics.median(kms) / 1e3) / 1e9
            forms[idct] = {"value": out_bytes / (statistics.median(fms) / 1e3) / 1e9, "unit": UNIT,
                           "ms_per_step": statistics.median(fms), "rel_l2_vs_fp32": rel,
                           "threads": fplan.info["threads"],
                           "roofline": {"bound": "hbm", "achieved": ka, "peak": peak, "unit": "GB/s",
                                        "frac": ka / peak, "launch_ms": statistics.median(kms),
                                        "traffic": measured_traffic(4, n_samples) if fplan.info["kernel"] == 4
                                        else None,
                                        "kernel": "k_decode_tc (tcgen05)"}}
            fplan.close()
            del out3
        line["forms"] = forms
        del ref

    # differentiable form: forward keeping the levels, then the hand-written
    # adjoint (dL/dA_z with an FP64 reduction, and dL/dC for every coefficient)
    # for dL/dx = x_hat - x0 with x0 = 0 (the decoded samples themselves)
    if not args.no_forms and rank == 0:
        n_lev = plan.info["n_levels_total"]
        lv = torch.empty(max(1, n_lev), dtype=torch.uint8, device=dev)
        gco = torch.empty(max(1, n_lev), dtype=torch.float32, device=dev)
        sc = torch.tensor([[float(x) for x in d.scale] for d in doms], dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            plan.decode(w, s, out=out, levels=lv, scale=sc, stream=stream)
            fw = time_steps(lambda: plan.decode(w, s, out=out, levels=lv, scale=sc, stream=stream), 5, stream,
                            torch)
            plan.backward(out, levels=lv, scale=sc, grad_coeffs=gco, stream=stream)
            bw = time_steps(lambda: plan.backward(out, levels=lv, scale=sc, grad_coeffs=gco, stream=stream), 5,
                            stream, torch)
        torch.cuda.synchronize()
        gsc, _ = plan.backward(out, levels=lv, scale=sc, grad_coeffs=gco, stream=stream)
        torch.cuda.synchronize()
        fwd_ms, bwd_ms = statistics.median(fw), statistics.median(bw)
        # adjoint bytes: dL/dx read (4 B / sample), levels read (1 B / coefficient), dL/dC written (4 B / coefficient)
        b_bytes = 4 * n_samples + 5 * n_lev
        line["differentiable"] = {
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "value": out_bytes / ((fwd_ms + bwd_ms) / 1e3) / 1e9, "unit": UNIT,
            "grad_scale_finite": bool(torch.isfinite(gsc).all()),
            "roofline": {"bound": "hbm", "achieved": b_bytes / (bwd_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": b_bytes / (bwd_ms / 1e3) / 1e9 / peak, "algorithmic_bytes_per_launch": b_bytes,
                         "traffic": measured_traffic(5, n_samples) if plan.info["kernel"] in (3, 4) else None,
                         "kernel": "k_backward_warp (adjoint)"}}
        del lv, gco, sc

    # the GPU encoder (Eq. 1, zone quantizer, Alg. 1) on the original signals, whose words
    # must equal the host encoder's (those the decoder read) bit for bit; and on the decoded
    # batch (re-encoding: every level-127/129 bin then sits on the deadzone edge)
    if x_orig is not None:
        from paper_2605_01086_gb300 import Encoder
        enc = Encoder(doms, wl.lengths, wl.domains, device=local, in_offsets=batch.segments["out_offset"])
        ew, es, enw = enc.buffers()
        elv = torch.empty(max(1, enc.n_levels), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            enc.encode(x_orig, ew, es, enw, levels=elv, stream=stream)
            ems = time_steps(lambda: enc.encode(x_orig, ew, es, enw, levels=elv, stream=stream), 5, stream, torch)
            pms = time_steps(lambda: enc.pack(elv, ew, es, enw, stream=stream), 5, stream, torch)
        torch.cuda.synchronize()
        est = enc.status()[0]
        # words against the host encoder's: the same counts, then every word and symbol count
        nw_host = torch.from_numpy(batch.segments["n_words"].astype(np.int64)).to(dev)
        same_counts = bool(torch.equal(enw[:wl.n_streams], nw_host))
        same_words = False
        if same_counts:
            shift = torch.from_numpy((enc.room_offsets.astype(np.int64) -
                                      batch.segments["word_offset"].astype(np.int64))).to(dev)
            idx = torch.repeat_interleave(shift, nw_host) + torch.arange(int(nw_host.sum()), device=dev)
            same_words = bool(torch.equal(ew[idx], w[:idx.numel()])) and bool(torch.equal(es[idx], s[:idx.numel()]))
            del idx, shift
        n_enc_words = int(enw[:wl.n_streams].sum())
        # algorithmic bytes: samples read (4 B), levels written and read back by the
        # packing's reference and packing passes (3 x 1 B per level), words and symbol counts written (9 B)
        n_lev = int(enc.n_levels)
        enc_bytes = 4 * n_samples + 3 * n_lev + 9 * n_enc_words
        e_ms = statistics.median(ems)
        # re-encoding the decoded batch
        lvd = torch.empty_like(elv)  # the original streams' levels, same layout (caller order, packed)
        with torch.cuda.stream(stream):
            plan.decode(w, s, out=out, levels=lvd, stream=stream)
            enc.encode(out, ew, es, enw, levels=elv, stream=stream)
            rms = time_steps(lambda: enc.encode(out, ew, es, enw, levels=elv, stream=stream), 3, stream, torch)
        torch.cuda.synchronize()
        same = float((lvd[:enc.n_levels] == elv[:enc.n_levels]).double().mean())
        del lvd
        line["gpu_encode"] = {"value": 4.0 * n_samples / (e_ms / 1e3) / 1e9,
                              "unit": "GB/s of float32 input", "ms_per_step": e_ms,
                              "pack_ms": statistics.median(pms), "levels_ms": e_ms - statistics.median(pms),
                              "compressed_bytes": 9 * n_enc_words, "status": est,
                              "input": "the original signals",
                              "words_equal_to_host_encoder": same_words, "word_counts_equal": same_counts,
                              "roofline": {"bound": "hbm", "achieved": enc_bytes / (e_ms / 1e3) / 1e9, "peak": peak,
                                           "unit": "GB/s", "frac": enc_bytes / (e_ms / 1e3) / 1e9 / peak,
                                           "algorithmic_bytes_per_step": enc_bytes},
                              "reencode": {"ms_per_step": statistics.median(rms),
                                           "value": 4.0 * n_samples / (statistics.median(rms) / 1e3) / 1e9,
                                           "input": "the decoded batch",
                                           "levels_equal_to_decoded_fraction": same},
                              "arithmetic": "FP32 butterfly with per-bin error bounds, compensated FP32 where a bin "
                                            "is near a level boundary, FP64 where that cannot settle it (levels "
                                            "equal to the FP64 encoder's)"}
        enc.close()
        del ew, es, enw, elv, x_orig

    # the paper's three-kernel GPU design on the same streams (global per-word offsets and
    # level array, one thread per output sample), for comparison with the fused kernels
    if not args.no_plain and rank == 0:
        tplan = Plan(doms, batch.segments, device=local, schedule="three_kernel")
        out4 = torch.zeros_like(out)
        with torch.cuda.stream(stream):
            tplan.decode(w, s, out=out4, stream=stream)
            tms = time_steps(lambda: tplan.decode(w, s, out=out4, stream=stream), 3, stream, torch)
            tix = time_steps(lambda: tplan.decode_stages(w, s, out4, STAGE_INDEX, stream=stream), 3, stream, torch)
            tdc = time_steps(lambda: tplan.decode_stages(w, s, out4, STAGE_DECODE, stream=stream), 3, stream, torch)
            # the paper's runtime breakdown (Sec. 6, Fig. 13): its lossless and lossy kernels timed apart
            tll = time_steps(lambda: tplan.decode_stages(w, s, out4, STAGE_LOSSLESS, stream=stream), 3, stream, torch)
            tly = time_steps(lambda: tplan.decode_stages(w, s, out4, STAGE_LOSSY, stream=stream), 3, stream, torch)
        torch.cuda.synchronize()
        rel = float(torch.linalg.vector_norm((out4 - out).double()) / torch.linalg.vector_norm(out.double()))
        tv = out_bytes / (statistics.median(tms) / 1e3) / 1e9
        ll, ly, ix = statistics.median(tll), statistics.median(tly), statistics.median(tix)
        line["three_kernel"] = {"value": tv, "unit": UNIT, "ms_per_step": statistics.median(tms),
                                "index_ms": ix, "decode_ms": statistics.median(tdc),
                                "lossless_ms": ll, "lossy_ms": ly,
                                "share": {"index": ix / (ix + ll + ly), "lossless": ll / (ix + ll + ly),
                                          "lossy": ly / (ix + ll + ly)},
                                "launches_per_step": tplan.launches_per_decode, "rel_l2_vs_fused": rel,
                                "fused_over_three_kernel": rank_value / tv}
        tplan.close()
        del out4

    # plain baseline: one set of launches per stream, same streams, same output
    if not args.no_plain and rank == 0:
        pplan = Plan(doms, batch.segments, device=local, schedule="per_segment")
        out2 = torch.zeros_like(out)
        with torch.cuda.stream(stream):
            pplan.decode(w, s, out=out2, stream=stream)
            pms = time_steps(lambda: pplan.decode(w, s, out=out2, stream=stream), 3, stream, torch)
        torch.cuda.synchronize()
        same = bool(torch.equal(out, out2))
        pv = out_bytes / (statistics.mean(pms) / 1e3) / 1e9
        line["plain"] = {"value": pv, "unit": UNIT, "ms_per_step": statistics.mean(pms),
                         "launches_per_step": pplan.launches_per_decode, "identical_output": same,
                         "batched_over_plain": rank_value / pv}
        pplan.close()
        del out2

    # end to end through the C ABI with host buffers: H2D of the compressed
    # batch + decode + D2H of every sample, inside the timed region
    if not args.no_e2e:
        h_w = torch.from_numpy(batch.words.view(np.int64)).pin_memory()
        h_s = torch.from_numpy(batch.symlen).pin_memory()
        h_o = torch.empty(out.numel(), dtype=torch.float32).pin_memory()
        plan.decode_host(h_w, h_s, h_o, w, s, out, stream=stream)  # warm-up
        e2e = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            plan.decode_host(h_w, h_s, h_o, w, s, out, stream=stream)
            e2e.append(time.perf_counter() - t)
        e_s = statistics.mean(e2e)
        if dist:
            tt = torch.tensor([e_s], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_s = float(tt.item())
        line["e2e"] = {"value": job_out_bytes / e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                       "d2h_bytes_per_step": 4 * plan.info["out_extent"], "steps": args.e2e_steps,
                       "api": "fptc_decode_host (pinned host buffers)"}
        del h_w, h_s, h_o

    if rank == 0 and not args.no_cpu:
        idxs, n_threads = cpu_sample(batch, target_s=args.cpu_seconds)
        t = oracle_sample_time(batch, idxs, n_threads)
        smp = int(batch.segments["n_samples"][idxs].sum())
        line["cpu_baseline"] = {"value": 4.0 * smp / t / 1e9, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                                "sample": f"{len(idxs)} random streams of the workload, {smp} samples, "
                                          f"{t:.1f} s, FP64 bit-serial decode, OpenMP over streams"}
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


SWEEP_SHAPES = [(16, 8), (32, 8), (32, 16), (32, 32), (64, 16), (64, 32), (128, 32), (128, 64),
                (24, 12), (48, 24), (100, 50)]  # the last three: N not a power of two


def run_sweep(args):
    """Throughput over the window size N and kept bins E (Table 1 ranges; the paper's Fig. 14
    trend): 512 EEG-like signals of 65,536 samples per shape, tables trained per shape, encoded
    once and decoded as `--sweep-copies` copies of the batch (each copy its own words and output,
    4.3 GB of output per shape at 32 copies: far beyond L2, so every row is a fraction of the HBM
    roofline), index + decode per step on the plan's default kernel; for E >= 32 also the
    tensor-core forms of the transform."""
    import torch

    from paper_2605_01086_gb300 import Plan, codec

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = siggen.eeg_2048x1m()
    n, S, R = 512, 65536, max(1, args.sweep_copies)
    seeds = wl.seeds[:n]
    doms_d = np.zeros(n, np.int32)
    lengths = np.full(n, S, np.uint64)
    flat, offs = siggen.signals(doms_d, seeds, lengths)
    ts = siggen.training_set(0)
    tflat, toffs = siggen.signals(ts.domains, ts.seeds, ts.lengths)
    peak, peak_kind = measured_peaks()
    rows = []
    stream = torch.cuda.Stream(dev)
    for N, E in SWEEP_SHAPES:
        d = codec.train_domain(tflat, toffs, ts.lengths, N, E, min(2, E), E, 50.0, 0.004, 12, 99.9)
        b = codec.encode_batch([d], flat, offs, lengths, np.zeros(n, np.uint32))
        sg = b.segments
        n_w = int(b.words.size)
        out_one = int(np.max(sg["out_offset"] + sg["n_samples"]))
        out_one = (out_one + 31) // 32 * 32
        segs = np.concatenate([codec.segments_array(sg["word_offset"] + np.uint64(r * n_w), sg["n_words"],
                                                    sg["n_samples"], sg["out_offset"] + np.uint64(r * out_one),
                                                    sg["domain"]) for r in range(R)])
        w1 = torch.from_numpy(np.ascontiguousarray(b.words, np.uint64).view(np.int64)).to(dev)
        s1 = torch.from_numpy(np.ascontiguousarray(b.symlen, np.uint8)).to(dev)
        w, s = w1.repeat(R), s1.repeat(R)  # copy r of the streams at words r * n_w
        del w1, s1
        out_b = 4 * n * S * R
        alg = out_b + 9 * int(sg["n_words"].sum()) * R
        ref = None
        # the FP32 transform, and for E >= 32 the tensor-core forms
        pow2 = N & (N - 1) == 0
        forms = ["fp32"] + (["tf32x3", "bf16x3", "tf32"] if E >= 32 and pow2 else []) + ([] if pow2 else ["generic"])
        for idct in forms:
            try:
                plan = (Plan([d], segs, device=0, kernel="generic") if idct == "generic"
                        else Plan([d], segs, device=0, idct=idct))
            except Exception:  # a shape the tensor-core kernel does not serve
                continue
            out = plan.empty_out()
            with torch.cuda.stream(stream):
                plan.decode(w, s, out=out, stream=stream)
                for _ in range(args.warmup):
                    plan.decode(w, s, out=out, stream=stream)
                ms = time_steps(lambda: plan.decode(w, s, out=out, stream=stream), args.steps, stream, torch)
            torch.cuda.synchronize()
            x = flat.astype(np.float64)
            xh = out[:n * S].double().cpu().numpy()
            prd = 100.0 * float(np.sqrt(np.sum((x - xh) ** 2) / np.sum(x ** 2)))
            same = bool(torch.equal(out[:out_one], out[(R - 1) * out_one:R * out_one]))
            if ref is None:
                ref = out[:out_one].clone()
                rel = 0.0
            else:
                rel = float(torch.linalg.vector_norm((out[:out_one] - ref).double()) /
                            torch.linalg.vector_norm(ref.double()))
            med = statistics.median(ms)
            rows.append({"N": N, "E": E, "idct": idct, "kernel": plan.info["kernel"], "threads": plan.info["threads"],
                         "ms": med, "GBps": out_b / (med / 1e3) / 1e9,
                         "roofline_frac": alg / (med / 1e3) / 1e9 / peak,
                         "compression_ratio": 4 * n * S / (9.0 * int(sg["n_words"].sum())), "prd_percent": prd,
                         "rel_l2_vs_fp32": rel, "copies_identical": same})
            plan.close()
            del out
        del w, s, ref
    print(json.dumps({"sweep": f"N x E, {R} copies of 512 EEG-like signals x 65536 samples "
                               f"({4 * n * S * R / 1e9:.1f} GB out per shape), index + decode per step",
                      "unit": UNIT, "peak": peak, "peak_kind": peak_kind, "rows": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fptc", choices=["fptc", "reference"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: a batch of the workload's shape per rank (weak), or the one batch cut across "
                         "ranks by LPT on each stream's bytes (strong)")
    ap.add_argument("--workload", default="mixed")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per decode launch, if measured")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-encode", action="store_true", help="skip the GPU encoder line")
    ap.add_argument("--kernel", default=None, help="fix the decode kernel (no autotuning): warp_tile, block_tile, generic")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--sweep", action="store_true", help="throughput over window size N and kept bins E instead")
    ap.add_argument("--sweep-copies", type=int, default=32, help="copies of the sweep's batch decoded per step")
    ap.add_argument("--idct", default="fp32", choices=["fp32", "tf32", "bf16x3", "tf32x3"],
                    help="inverse-transform form of the timed plan (tensor-core forms use the tcgen05 kernel)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
