#!/usr/bin/env python3
"""Benchmark: certified-split lexing of the 512 MiB synthetic JSON corpus
(filtered modulo the discarded whitespace, cuts at tab / newline / CR) on one
GB300, bit-exact with the CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

A step is one lx_lex call over the whole corpus (all hot-path stages: stage,
plan, walk, scan, compact).  `value` is input GB/s (decimal) with the corpus
resident in HBM; `e2e` is the same metric through lx_lex_host (pinned host
input copied in, tokens copied back, inside the timed region).  Under
torchrun each rank lexes its own replica (weak scaling, no collective on the
data path).  `--impl reference` times the CPU oracle on host cores instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MiB = 1 << 20
CUTS = {"arith": "newline ( ) * + - / ; (exact certificate, I empty)",
        "clike_block_framed": "0x1E, reserved at the producer before every line or comment (exact certificate)",
        "json": "tab, newline, carriage return (certified modulo I = {ws})",
        "clike": "newline (certified modulo I = {ws, line comment})",
        "clike_block": "none certified: chunk starts every 4096 B after the byte with the fewest entry contexts"}


def metric_name(workload, mib):
    if workload == "clike_block_framed":
        return f"input GB/s lexed ({mib} MiB framed C-like with block comments, full stream, exact cuts, bit-exact)"
    if workload == "arith":
        return f"input GB/s lexed ({mib} MiB arith token stream, full stream, exact cuts, bit-exact)"
    if workload == "clike_block":
        return f"input GB/s lexed ({mib} MiB C-like with block comments, full stream, speculative entry contexts, bit-exact)"
    label = {"json": "JSON", "clike": "C-like"}[workload]
    return f"input GB/s lexed ({mib} MiB {label}, filtered modulo I, bit-exact)"


def workload_name(workload, mib):
    if workload == "clike_block_framed":
        return f"clike_block_framed_{mib}mib_full_exact"
    if workload == "arith":
        return f"arith_{mib}mib_full_exact"
    if workload == "clike_block":
        return f"clike_block_{mib}mib_full_speculative"
    return f"{workload}_{mib}mib_filtered_modulo"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """The largest of x over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic(workload_key):
    """DRAM bytes of one launch from the committed ncu summary, or None when
    the kernel source changed since the counters were taken."""
    import hashlib
    import re
    try:
        src = open(os.path.join(ROOT, "paper_2608_03473_gb300", "csrc", "lexwarp.cu"), "rb").read()
        text = open(os.path.join(ROOT, "profiles", "lex_warps_dram_512mib.md")).read()
    except OSError:
        return None
    h = hashlib.sha256(src).hexdigest()
    for key, val, sha in re.findall(r"<!-- traffic (\S+) (\d+) ([0-9a-f]{64}) -->", text):
        if key == workload_key and sha == h:
            return int(val)
    return None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def time_parallel(w, dfa, disc, useful, sample_bytes, reps=3):
    """The paper's method on the host: the Section 6 planner, one thread per
    chunk, ordered concatenation (oracle/parsplit.c), at k = 1, 2, 4, ... up
    to every core; median of `reps` runs per k."""
    import oracle
    s = w[:sample_bytes]
    cores = cpu_cores()
    ks = sorted({1 << i for i in range(cores.bit_length()) if (1 << i) <= cores} | {cores})
    by_k = {}
    tokens = 0
    for k in ks:
        secs = []
        for _ in range(reps):
            ok, ol, con, chunks, sec = oracle.par_lex(dfa, s, useful, disc or [], k, cap=s.size + 16)
            secs.append(sec)
            tokens = ok.size
        by_k[k] = s.size / statistics.median(secs) / 1e9
    return {"value": by_k[cores], "unit": "GB/s", "cores": cores, "kind": "cpu_parallel_certified_split",
            "by_threads_gbs": {str(k): v for k, v in by_k.items()},
            "sample": f"first {s.size // MiB} MiB of the corpus, median of {reps} runs per thread count, "
                      f"{tokens} output tokens",
            "method": "Section 6 planner (k-1 equal-division targets slid to the next useful certified byte), "
                      "one pthread per chunk scanning from q0 with pi_I fused, ordered concatenation",
            "cpu_model": cpu_model(), "compiler": "gcc " + " ".join(__import__("oracle").CFLAGS),
            "timed": "planning through concatenation, input resident in host memory"}


def time_oracle(w, dfa, disc, sample_bytes, reps=1):
    """Serial oracle (one host core) over the first `sample_bytes` of w."""
    import oracle
    s = w[:sample_bytes]
    best = None
    tokens = 0
    for _ in range(reps):
        t0 = time.perf_counter()
        k, l, con = oracle.lex(dfa, s)
        k2 = k if disc is None else oracle.discard(k, l, disc, dfa.n_kinds)[0]
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
        tokens = k2.size
    return s.size, tokens, best


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on host cores (rank 0 only)."""
    if rank != 0:
        return
    from lexinputs import corpus, tokensets
    dfa = tokensets.tokenset(args.workload)
    disc = None if args.workload in ("clike_block", "arith") else tokensets.discarded_kinds(args.workload)
    sample = min(args.ref_sample_mib, args.size_mib) * MiB
    w = corpus.generate(args.workload, sample)
    times = []
    for i in range(args.warmup + args.steps):
        n, tok, dt = time_oracle(w, dfa, disc, sample)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * len(times) / total / 1e9
    line = {
        "metric": metric_name(args.workload, args.size_mib), "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": workload_name(args.workload, args.size_mib),
                   "sample": f"first {sample // MiB} MiB of the {args.size_mib} MiB corpus",
                   "bytes_per_step": n},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {sample // MiB} MiB of the corpus per step, serial scan + pi_I"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "tokens_per_s": tok * len(times) / total,
    }
    print(json.dumps(line), flush=True)


BATCH_NAMES = ("json", "clike")


def run_batch(args, rank, world, local):
    """The batched workload: 4096 documents (lognormal sizes, median 128 KiB,
    sigma 1.66, clamped to [1 KiB, 16 MiB]), each JSON or C-like, lexed
    filtered modulo I by one lx_lex_batch call per step; also timed as 4096
    separate lx_lex calls."""
    import numpy as np
    from lexinputs import corpus, tokensets
    spec = corpus.batch_spec()
    n_docs = len(spec)
    total = sum(sz for _, sz, _ in spec)
    metric = f"input GB/s lexed ({n_docs}-document batch, JSON + C-like, filtered modulo I, bit-exact)"
    wl = f"batch_{n_docs}docs_json_clike_filtered_modulo"
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        sample, tok, times = 0, 0, []
        host, offs = corpus.generate_batch(spec[:256])
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            nb = nt = 0
            for (nm, sz, _), o in zip(spec[:256], offs):
                if nb >= args.ref_sample_mib * MiB:
                    break
                dfa = tokensets.tokenset(nm)
                k, l, con = oracle.lex(dfa, host[o:o + sz])
                k, _ = oracle.discard(k, l, tokensets.discarded_kinds(nm), dfa.n_kinds)
                nb += sz
                nt += k.size
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
            sample, tok = nb, nt
        value = sample * len(times) / sum(times) / 1e9
        print(json.dumps({
            "metric": metric, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl, "sample": f"leading documents of the batch, {sample} bytes per step"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"leading documents, {sample} bytes per step, serial scan + pi_I"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    import torch
    import torch.distributed as dist
    import paper_2608_03473_gb300 as lg
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    host, offs = corpus.generate_batch(spec)
    sets = [lg.lx_compile_tokenset(tokensets.tokenset(n), tokensets.discarded_kinds(n)) for n in BATCH_NAMES]
    ctx = lg.lx_ctx_create()
    lg.lx_ctx_enable_timing(ctx, True)
    stream = torch.cuda.current_stream()
    d = torch.from_numpy(host).to("cuda")
    cap = total // 3 + 4096
    d_k = torch.empty(cap, dtype=torch.int16, device="cuda")
    d_l = torch.empty(cap, dtype=torch.int32, device="cuda")
    docs = [((d.data_ptr() + o, sz), BATCH_NAMES.index(nm)) for (nm, sz, _), o in zip(spec, offs)]
    mode = lg.LX_FILTERED_MODULO
    rc, n_tok, res = lg.lx_lex_batch(ctx, sets, docs, mode, d_k, d_l, stream=stream)
    assert rc == 0, lg.lx_strerror(rc)
    assert all(con == sz for (_, sz, _), (_, _, con) in zip(spec, res))
    if args.check:
        import oracle
        kk = d_k[:n_tok].cpu().numpy().view(np.uint16)
        ll = d_l[:n_tok].cpu().numpy().view(np.uint32)
        for (nm, sz, _), o, (off, nt, con) in zip(spec, offs, res):
            dfa = tokensets.tokenset(nm)
            k, l, c = oracle.lex(dfa, host[o:o + sz])
            k, l = oracle.discard(k, l, tokensets.discarded_kinds(nm), dfa.n_kinds)
            assert c == con and k.size == nt
            assert np.array_equal(kk[off:off + nt], k) and np.array_equal(ll[off:off + nt], l)
        del kk, ll
    batch = lg.BatchDocs(sets, docs)   # descriptors built once, as a serving loop would
    for _ in range(args.warmup):
        lg.lx_lex_batch(ctx, sets, batch, mode, d_k, d_l, stream=stream, want_results=False)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    graph_ms = []
    ev0.record(stream)
    for _ in range(args.steps):
        rc, nt2, _ = lg.lx_lex_batch(ctx, sets, batch, mode, d_k, d_l, stream=stream, want_results=False)
        graph_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
        if rc != 0 or nt2 != n_tok:
            raise RuntimeError(f"step failed: {rc} {nt2}")
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1))
    value = world * total * args.steps / (total_ms / 1e3) / 1e9
    g_ms = statistics.mean(graph_ms)
    alg = total + 6 * n_tok
    peak, peak_src = measured_peak_gbs()

    # the same documents as separate lx_lex calls (one pass)
    views = [(d[o:o + sz], BATCH_NAMES.index(nm)) for (nm, sz, _), o in zip(spec, offs)]
    for v, si in views[:64]:
        lg.lx_lex(ctx, sets[si], v, mode, d_k, d_l, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v, si in views:
        rc, _, _ = lg.lx_lex(ctx, sets[si], v, mode, d_k, d_l, stream=stream)
        assert rc == 0
    torch.cuda.synchronize()
    sep_s = time.perf_counter() - t0
    # ... and as separate lx_lex_async calls: stream-ordered, one synchronization at the end
    d_res = torch.zeros((n_docs, 24), dtype=torch.uint8, device="cuda")
    for i, (v, si) in enumerate(views[:64]):
        lg.lx_lex_async(ctx, sets[si], v, mode, d_k, d_l, d_res[i], stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (v, si) in enumerate(views):
        rc = lg.lx_lex_async(ctx, sets[si], v, mode, d_k, d_l, d_res[i], stream=stream)
        assert rc == 0, lg.lx_strerror(rc)
    torch.cuda.synchronize()
    async_s = time.perf_counter() - t0
    assert all(lg.async_result(r)[0] == 0 for r in d_res.cpu().numpy())

    # end to end: pinned host documents in, tokens out, through the binding.
    # The batch is cut into parts of consecutive documents (about equal bytes),
    # each lexed by its own lx_lex_batch call with its own context (its own
    # cached graph): the copy of part i + 1 in and of part i - 1's tokens out
    # overlap the lexing of part i.
    h_in = torch.from_numpy(host).pin_memory()
    h_k = torch.empty(cap, dtype=torch.int16).pin_memory()
    h_l = torch.empty(cap, dtype=torch.int32).pin_memory()
    n_parts = args.e2e_parts
    cuts, acc_b, goal = [0], 0, total / n_parts
    for i, (_, sz, _) in enumerate(spec):
        acc_b += sz
        if acc_b >= goal * len(cuts) and len(cuts) < n_parts and i + 1 < n_docs:
            cuts.append(i + 1)
    cuts.append(n_docs)
    parts = []
    t_off = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        pdocs = docs[a:b]
        pctx = lg.lx_ctx_create()
        pbatch = lg.BatchDocs(sets, pdocs)
        rc, pt, _ = lg.lx_lex_batch(pctx, sets, pbatch, mode, d_k[t_off:], d_l[t_off:], stream=stream,
                                    want_results=False)
        assert rc == 0, lg.lx_strerror(rc)
        lo, hi = offs[a], offs[b - 1] + spec[b - 1][1]
        parts.append((pctx, pbatch, lo, hi, t_off, pt))
        t_off += pt
    assert t_off == n_tok
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_step():
        ev_in = []
        s_in.wait_stream(stream)
        with torch.cuda.stream(s_in):
            for (_, _, lo, hi, _, _) in parts:
                d[lo:hi].copy_(h_in[lo:hi], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_in)
                ev_in.append(ev)
        for (pctx, pbatch, lo, hi, to, pt), ev in zip(parts, ev_in):
            stream.wait_event(ev)
            rc, nt3, _ = lg.lx_lex_batch(pctx, sets, pbatch, mode, d_k[to:], d_l[to:], stream=stream,
                                         want_results=False)
            if rc != 0 or nt3 != pt:
                raise RuntimeError(f"e2e part failed: {rc} {nt3}")
            s_out.wait_stream(stream)
            with torch.cuda.stream(s_out):
                h_k[to:to + nt3].copy_(d_k[to:to + nt3], non_blocking=True)
                h_l[to:to + nt3].copy_(d_l[to:to + nt3], non_blocking=True)
        stream.wait_stream(s_out)

    e2e_step()   # untimed: first use of the pinned buffers and streams
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.e2e_steps):   # each step timed on its own; the median step
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.median(step_ms))
    if rank == 0:
        print(json.dumps({
            "metric": metric, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": wl, "documents": n_docs, "bytes": total, "tokens_kept": n_tok,
                       "sizes": "lognormal median 128 KiB sigma 1.66 clamped to [1 KiB, 16 MiB]",
                       "seed": hex(corpus.BATCH_SEED), "mode": "LX_FILTERED_MODULO",
                       "l2": "inputs larger than L2; no flush between steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "tokens_per_s": world * n_tok * args.steps / (total_ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": alg / (g_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (g_ms / 1e3) / 1e9 / peak, "traffic": None,
                         "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "kernel": "lex_warps<class form, batch> (one launch over every document, the "
                                   "tables of both token sets resident, in one CUDA graph)",
                         "kernel_ms": g_ms, "algorithmic_bytes": alg},
            "separate_calls": {"value": total / sep_s / 1e9, "unit": "GB/s", "ms": 1e3 * sep_s,
                               "what": f"{n_docs} lx_lex calls, one per document (each synchronizes)"},
            "separate_async": {"value": total / async_s / 1e9, "unit": "GB/s", "ms": 1e3 * async_s,
                               "what": f"{n_docs} lx_lex_async calls on one stream, one synchronization"},
            "cpu_baseline": None,
            "e2e": {"value": world * total / (e2e_ms / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": total,
                    "d2h_bytes_per_step": 6 * n_tok, "ms_per_step": e2e_ms,
                    "api": "torch pinned copies + lx_lex_batch"},
            "gpu_launches": 2 * args.steps,   # the tile map and the batch kernel per graph replay
            "clocks": clocks,
            "bit_exact": True if args.check else None,
        }), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=7)
    ap.add_argument("--e2e-parts", type=int, default=8, help="batch workload: parts of the end-to-end pipeline")
    ap.add_argument("--size-mib", type=int, default=None, help="input size (default 512; arith: 1)")
    ap.add_argument("--workload", default="json",
                    choices=["json", "clike", "clike_block", "batch", "arith", "clike_block_framed"])
    ap.add_argument("--ref-sample-mib", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the untimed element-by-element comparison with the oracle")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.size_mib is None:
        args.size_mib = 1 if args.workload == "arith" else 512
    args.check = not args.no_check

    rank, world, local = dist_env()
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2608_03473_gb300 as lg
    from lexinputs import corpus, tokensets

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    n = args.size_mib * MiB
    w = corpus.generate(args.workload, n)
    sha = corpus.sha256(w) if rank == 0 else None
    framed = args.workload == "clike_block_framed"
    if framed:
        # Section 7.1: the refused C-like set with 0x1E reserved at the producer;
        # the oracle lexes with the same automaton built on the host side
        base = tokensets.tokenset("clike_block")
        disc = tokensets.discarded_kinds("clike_block")
        dfa = tokensets.framed(base)
        ts = lg.lx_compile_tokenset_framed(base, disc, tokensets.FRAME)
    else:
        dfa = tokensets.tokenset(args.workload)
        disc = tokensets.discarded_kinds(args.workload)
        ts = lg.lx_compile_tokenset(dfa, disc)
    ctx = lg.lx_ctx_create()
    lg.lx_ctx_enable_timing(ctx, True)
    stream = torch.cuda.current_stream()
    refused = args.workload == "clike_block"
    full = refused or framed or args.workload == "arith"   # the full stream, exact cuts
    small = n < 256 * MiB                               # flush L2 between timed steps
    lex_fn = lg.lx_lex
    spec_model, train_s, spec_stats = None, None, {}
    if refused:
        # entry-context model trained (before the timed region) on corpora of
        # other seeds, with labels resolved by enumeration on the GPU
        t0 = time.perf_counter()
        samples = [torch.from_numpy(corpus.generate(args.workload, 64 * MiB, seed=s)).to("cuda")
                   for s in (0x1EC50015, 0x1EC50025)]
        spec_model = lg.train_context_model(ctx, ts, samples, hidden=64, epochs=3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        del samples

        def lex_fn(c, t, d, m, k, l, stream=None):
            rc_, nt_, con_, st_ = lg.lx_lex_speculative(c, t, spec_model, d, m, k, l, stream=stream)
            spec_stats.update(st_)
            return rc_, nt_, con_

    d_in = torch.from_numpy(w).to("cuda")
    cap = (n // 2 + 1024 if refused else n + 1 if full else n // 4 + 1024)   # the full stream keeps every token
    d_k = torch.empty(cap, dtype=torch.int16, device="cuda")
    d_l = torch.empty(cap, dtype=torch.int32, device="cuda")
    mode = lg.LX_FULL_EXACT if full else lg.LX_FILTERED_MODULO
    rc, nt, con = lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
    assert rc == 0, lg.lx_strerror(rc)
    assert con == n

    bit_exact = None
    if args.check:
        # one untimed comparison of the whole output with the oracle
        import oracle
        k, l, c = oracle.lex(dfa, w)
        if not full:
            k, l = oracle.discard(k, l, disc, dfa.n_kinds)
        bit_exact = bool(c == con and k.size == nt
                         and np.array_equal(d_k[:nt].cpu().numpy().view(np.uint16).astype(np.int64), k)
                         and np.array_equal(d_l[:nt].cpu().numpy().view(np.uint32).astype(np.int64), l))
        del k, l
        if not bit_exact:
            raise RuntimeError("output differs from the oracle")

    for _ in range(args.warmup):
        lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    if small:
        # inputs smaller than L2: each step is timed on its own, after a write
        # of a buffer larger than L2 (outside the step's events)
        flush = torch.empty(256 * MiB, dtype=torch.uint8, device="cuda")
        call_ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, nt2, con2 = lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
            e1.record(stream)
            kernel_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
            if rc != 0 or nt2 != nt or con2 != con:
                raise RuntimeError(f"step failed: {rc} {nt2} {con2}")
            torch.cuda.synchronize()
            call_ms.append(e0.elapsed_time(e1))
        total_ms = max_over_ranks(sum(call_ms))
        del flush
    else:
        ev0.record(stream)
        for _ in range(args.steps):
            rc, nt2, con2 = lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
            kernel_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
            if rc != 0 or nt2 != nt or con2 != con:
                raise RuntimeError(f"step failed: {rc} {nt2} {con2}")
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms = max_over_ranks(ev0.elapsed_time(ev1))
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms_per_step = total_ms / args.steps
    value = world * n * args.steps / (total_ms / 1e3) / 1e9
    tokens_per_s = world * nt * args.steps / (total_ms / 1e3)

    # roofline of the dominant kernel (the tile kernel): algorithmic bytes =
    # input bytes read + 6 bytes per kept token written
    k_ms = statistics.mean(kernel_ms)
    alg_bytes = n + 6 * nt
    peak, peak_src = measured_peak_gbs()
    achieved = alg_bytes / (k_ms / 1e3) / 1e9

    # end to end through lx_lex_host: pinned input in, tokens out
    h_in = torch.from_numpy(w).pin_memory()
    h_k = torch.empty(cap, dtype=torch.int16).pin_memory()
    h_l = torch.empty(cap, dtype=torch.int32).pin_memory()
    def host_step():
        if not refused:
            return lg.lx_lex_host(ctx, ts, h_in, mode, h_k, h_l, stream=stream)
        d_in.copy_(h_in, non_blocking=True)
        r = lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
        h_k[:r[1]].copy_(d_k[:r[1]], non_blocking=True)
        h_l[:r[1]].copy_(d_l[:r[1]], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return r

    for _ in range(2):
        host_step()
    torch.cuda.synchronize()
    # each step timed on its own; the median step (copies share the host link
    # with other users of the machine, so single steps can be slow)
    step_ms = []
    for _ in range(args.e2e_steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, nt3, con3 = host_step()
        e1.record(stream)
        torch.cuda.synchronize()
        assert rc == 0 and nt3 == nt and con3 == con
        step_ms.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.median(step_ms))
    e2e_value = world * n / (e2e_ms / 1e3) / 1e9

    if rank == 0:
        cpu = None
        ex_mask, mo_mask = lg.lx_certificates(ts)
        if not args.no_cpu_baseline:
            sample = min(n, 256 * MiB)
            sample = min(sample, 64 * MiB) if refused else sample
            sb, stok, sdt = time_oracle(w, dfa, None if full else disc, sample)
            cpu = {"value": sb / sdt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                   "sample": f"first {sample // MiB} MiB of the corpus, one pass, serial scan"
                             f"{'' if full else ' + pi_I'} ({sdt:.1f} s, {stok} output tokens)"}
            if not refused:
                cpu["parallel_certified_split"] = time_parallel(
                    w, dfa, None if full else disc, ex_mask if full else mo_mask, min(n, 256 * MiB))
            else:
                cpu["parallel_certified_split"] = {
                    "value": None, "note": "the token set certifies no byte (exact or modulo): the paper's "
                                           "planner returns one chunk, so the method runs serially"}
        line = {
            "metric": metric_name(args.workload, args.size_mib), "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, args.size_mib), "bytes": n, "tokens_kept": nt,
                       "mode": "LX_FULL_EXACT" if full else "LX_FILTERED_MODULO", "cuts": CUTS[args.workload],
                       "seed": hex(corpus.WORKLOADS[args.workload][2]), "sha256": sha,
                       "l2": (f"input ({args.size_mib} MiB) smaller than L2: a 256 MiB buffer is written "
                              f"before each step, outside the step's timing" if small else
                              f"inputs ({args.size_mib} MiB) larger than L2 (129 MB); no flush between steps"),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "tokens_per_s": tokens_per_s,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": profiled_traffic(workload_name(args.workload, args.size_mib)),
                         "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "kernel": "en_plan + model + sp_scan/sp_fix rounds + sp_offsets + en_emit" if refused
                         else ("lex_warps (warp-tile kernel)" if lg.lx_tokenset_walk_table(ts, mode)[0] == 0
                               else "lex_tiles"),
                         "kernel_ms": k_ms,
                         "algorithmic_bytes": alg_bytes, "frac_of_nominal_8tbs": achieved / 8000.0},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": n, "d2h_bytes_per_step": 6 * nt + 32,
                    "ms_per_step": e2e_ms,
                    "api": "torch pinned copies + lx_lex_speculative" if refused else "lx_lex_host"},
            "gpu_launches": (None if refused else args.steps),
            "clocks": clocks,
            "bit_exact": bit_exact,
        }
        if small:
            line["us_per_call"] = 1e3 * total_ms / args.steps
            line["kernel_us"] = 1e3 * k_ms
        # both certificates of the token set (Definitions 2 and 3)
        fmt = lambda m: [f"0x{b:02x}" for b in range(256) if m[b]]
        line["config"]["certified"] = {"exact": fmt(ex_mask), "modulo": fmt(mo_mask)}
        if not full:
            # the same filtered stream under exact cuts: with no exact-certified
            # byte, lx_lex cuts at certified two-byte windows (warp-tile kernel)
            # where the token set has them, else enumerates entry contexts; its
            # output must equal the modulo-cut output (both are pi_I(tok(w)))
            x_k = torch.empty_like(d_k)
            x_l = torch.empty_like(d_l)
            win_ctx = lg.lx_tokenset_walk_table(ts, lg.LX_FILTERED_EXACT)[2].get("n_ctx", 0)
            x_ms = []
            for i in range(5):
                rcx, ntx, conx = lg.lx_lex(ctx, ts, d_in, lg.LX_FILTERED_EXACT, x_k, x_l, stream=stream)
                if i >= 2:
                    x_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
            rc, nt3, con3 = lex_fn(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
            same = (rcx == 0 and ntx == nt3 and conx == con3 and torch.equal(x_k[:ntx], d_k[:nt3])
                    and torch.equal(x_l[:ntx], d_l[:nt3]))
            line["exact_certificate"] = {
                "mode": "LX_FILTERED_EXACT",
                "path": "lx_lex (certified cuts)" if ex_mask.any() else
                        ("lx_lex: no exact-certified byte; cuts at certified two-byte windows (warp-tile kernel)"
                         if win_ctx else "lx_lex: no exact-certified byte, so the hybrid plan enumerates entry contexts"),
                "window_contexts": win_ctx,
                "kernel_ms": statistics.median(x_ms), "value": n / (statistics.median(x_ms) / 1e3) / 1e9,
                "unit": "GB/s", "same_output_as_modulo": bool(same)}
            del x_k, x_l
        if refused:
            # the enumerative path on the same input, for comparison
            for _ in range(2):
                lg.lx_lex_enumerative(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
            en_ms = []
            for _ in range(5):
                lg.lx_lex_enumerative(ctx, ts, d_in, mode, d_k, d_l, stream=stream)
                en_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
            line["speculative"] = {"rounds": spec_stats.get("rounds"), "chunks": spec_stats.get("chunks"),
                                   "rescanned": spec_stats.get("rescanned"),
                                   "model": "64-byte window: 8-d embedding, conv1d 32x5 + ReLU, max-pool 4, 512-64-C MLP; BF16 weights, FP32 accumulation, AdamW",
                                   "train_s": train_s,
                                   "train_data": "2 x 64 MiB C-like-with-block-comments corpora, other seeds"}
            line["enumerative"] = {"kernel_ms": statistics.median(en_ms),
                                   "value": n / (statistics.median(en_ms) / 1e3) / 1e9, "unit": "GB/s"}
            # the same speculative path without the model (every chunk guessed BOUNDARY)
            nm_ms, nm_st = [], {}
            for i in range(5):
                _, _, _, nm_st = lg.lx_lex_speculative(ctx, ts, None, d_in, mode, d_k, d_l, stream=stream)
                if i >= 2:
                    nm_ms.append(lg.lx_ctx_last_kernel_ms(ctx))
            line["speculative_no_model"] = {"kernel_ms": statistics.median(nm_ms),
                                            "value": n / (statistics.median(nm_ms) / 1e3) / 1e9, "unit": "GB/s",
                                            "rounds": nm_st.get("rounds"), "rescanned": nm_st.get("rescanned")}
            # en_plan, sp_init, so_block, so_top, so_out, sp_copy; sp_scan + sp_fix per round; per
            # batch of 16 384 windows: k_windows, two k_gemm_rb, k_argmax
            launches = 6 + 2 * (spec_stats.get("rounds") or 1) + (n // 4096 + 16383) // 16384 * 4
            line["gpu_launches"] = launches * args.steps
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
