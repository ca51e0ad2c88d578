"""Benchmark of the single-stream exact-sequence fills on one GB300.

A step is the single-stream workload: for each engine (xoshiro256++,
PCG64-DXSM, Philox4x32-10) and each sampler (ziggurat normal, ziggurat
exponential, bounded uint64 in [0, m) for m in {6, 1e9+7, 2^63+1}) one fresh
fill of n = 2^28 variates from seed 2024, word 0 -- 15 fills, 4.03e9
variates.  Outputs (2 GiB per fill) are far larger than L2, so no flush is
needed between timed fills.

Prints one JSON line (metric variates/s).  --impl reference times the serial
CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FILL = 1 << 28
SEED = 2024
ENGINES = ["xoshiro256pp", "pcg64dxsm", "philox4x32_10"]
SAMPLERS = [("normal", ()), ("exp", ()), ("bounded", (6,)), ("bounded", (1_000_000_007,)),
            ("bounded", (2 ** 63 + 1,))]
METRIC = "variates/s (single-stream exact-sequence fills, 3 engines x {normal, exp, bounded m in {6, 1e9+7, 2^63+1}})"
WORKLOAD = "single-stream fills: engines {xoshiro256++, PCG64-DXSM, Philox4x32-10}, seed 2024, n=2^28 each of normal, exp, bounded m=6, 1e9+7, 2^63+1"


# DRAM bytes (read + write) per launch of the fill kernel at n = 2^28, from
# one ncu capture at n = 2^26 scaled by outputs (profiles/*_n2e26.md), by fill
# key.  Only kernels whose current version was captured are listed.
TRAFFIC = {
    "philox4x32_10/bounded:9223372036854775809": 4 * 1580355904,
}


# Integer operations per 64-bit word of each engine, counted as 32-bit
# operations of its definition (each 32 x 32 partial product's low and high
# halves, adds with carry, shifts (a funnel shift is one), two-input xors):
#   xoshiro256++  output: two 64-bit adds and a rotate (6); update: a 64-bit
#                 shift, five 64-bit xors and a rotate (14)              -> 20
#   PCG64-DXSM    LCG step: 128 x 64-bit multiply mod 2^128 (12 products,
#                 ~10 carry adds) and the 128-bit increment (4); DXSM
#                 output: or, two xor-shifts and two 64-bit multiplies  -> 42
#   Philox4x32-10 per 128-bit block: the counter increment (4) and ten
#                 rounds of two 32 x 32 -> 64 products (4) and four xors;
#                 the round keys depend on the key alone, so every block
#                 of a fill shares them                                 -> 42 per word
# With the issue rate of this GPU (4 schedulers x 32 lanes per SM and clock)
# these give the derived integer peak that the measured engine-only rates
# (rp_engine_fold) are compared with.
ENGINE_OPS = {"xoshiro256pp": 20, "pcg64dxsm": 42, "philox4x32_10": 42}

# FP64 flops per gradient (DADD + DMUL + 2 DFMA, thread level, predicated on)
# counted by ncu on n = 2^24 samples of the same workloads
# (profiles/k_gamma_grad_n2e24.md, profiles/k_beta_grad_a2_b5_n2e24.md); the
# kernels are bound by the FP64 pipe: 2 DFMA per SM per clock.
GRAD_FLOPS = {"gamma(2.5)": 252.5, "gamma(30.0)": 371.9, "beta(2.0, 5.0)": 442.3}
FP64_FLOPS_PER_SM_CLK = 4
ISSUE_LANES_PER_SM = 128


def words_per_output(dist, params):
    """Expected engine words per output: ziggurat geometry (normal 1.0235,
    exponential 1.036) and Lemire's acceptance 1 - (2^64 mod m)/2^64."""
    if dist == "normal":
        return 1.0235
    if dist == "exp":
        return 1.036
    m = params[0]
    return 1.0 / (1.0 - ((2**64) % m) / 2.0**64)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def wait_first(self, timeout=3.0):
        """Block until nvidia-smi has produced its first sample."""
        t0 = time.time()
        while self.proc is not None and not self.rows and time.time() - t0 < timeout:
            time.sleep(0.02)

    def mark(self, t_begin, t_end):
        """Host time window of the timed region (samples outside it are dropped)."""
        self.window = (t_begin, t_end)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        win = getattr(self, "window", None)
        rows = [r for t, r in self.rows if win is None or win[0] <= t <= win[1] + 0.25]
        if not rows:
            rows = [r for _, r in self.rows]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _key(engine, dist, params):
    return f"{engine}/{dist}{'' if not params else ':' + str(params[0])}"


def _dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)   # before the process group, so that NCCL binds this rank's GPU
        dist.init_process_group("nccl")
    return world, rank, local


def run_gpu(args):
    import torch

    import paper_2605_05099_gb300 as rp

    world, rank, local = _dist_init()
    torch.cuda.set_device(local)
    rp.lib()
    stream = torch.cuda.current_stream()
    # ranks fill independent spawn-key streams (weak scaling, no collective on the data path)
    from paper_2605_05099_gb300 import shard
    spawn = shard.rank_spawn_key(rank, world)
    out_f = torch.empty(N_FILL, dtype=torch.float64, device="cuda")
    out_u = torch.empty(N_FILL, dtype=torch.uint64, device="cuda")

    def one_fill(engine, dist, params, buf=None):
        of = out_f if buf is None else buf.view(torch.float64)
        ou = out_u if buf is None else buf.view(torch.uint64)
        if dist == "normal":
            return rp.rp_fill_normal(engine, SEED, spawn, 0, of, stream)
        if dist == "exp":
            return rp.rp_fill_exp(engine, SEED, spawn, 0, of, stream)
        return rp.rp_fill_bounded(engine, SEED, spawn, 0, params[0], ou, stream)

    fills = [(e, d, p) for e in ENGINES for d, p in SAMPLERS]
    if args.only:
        fills = [f for f in fills if _key(*f) == args.only]
        if not fills:
            raise SystemExit(f"--only {args.only}: no such fill; keys are "
                             + ", ".join(_key(e, d, p) for e in ENGINES for d, p in SAMPLERS))
    per_fill_ms = {_key(e, d, p): 0.0 for e, d, p in fills}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in fills]

    def step(record):
        for i, (e, d, p) in enumerate(fills):
            if record:
                ev[i][0].record(stream)
            one_fill(e, d, p)
            if record:
                ev[i][1].record(stream)

    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    launches0 = rp.rp_kernel_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    h_begin = time.time()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
        for i, key in enumerate(per_fill_ms):
            ev[i][1].synchronize()
            per_fill_ms[key] += ev[i][0].elapsed_time(ev[i][1])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(h_begin, time.time())
    launches = rp.rp_kernel_launches() - launches0
    ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    ms, variates = shard.reduce_timing(ms, len(fills) * N_FILL * args.steps, device="cuda")
    value = variates / (ms / 1e3)

    # ---- roofline of each fill: the slower of the HBM write time (8 B per
    # output at the copy rate of MEASURED_PEAKS.json) and the engine time
    # (words per output at the engine-only rate measured here with
    # rp_engine_fold); the line reports the dominant fill (largest time)
    peaks, peak_kind = _peaks()
    ceil = measure_ceilings(rp, stream, out_u, [e for e, _, _ in fills])
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    issue_peak = sms * ISSUE_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6   # thread ops/s
    hbm = peaks["hbm_gbs"] * 1e9
    flat, best = {}, None
    for (e, d, p), key in zip(fills, per_fill_ms):
        t = per_fill_ms[key] / args.steps / 1e3
        words = N_FILL * words_per_output(d, p)
        t_hbm, t_w, t_eng = 8.0 * N_FILL / hbm, 8.0 * N_FILL / (ceil["write_gbs"] * 1e9), words / ceil[e]
        flat[f"ms:{key}"] = round(t * 1e3, 4)
        flat[f"frac:{key}"] = round(max(t_hbm, t_eng) / t, 4)
        flat[f"frac_vs_write_only:{key}"] = round(max(t_w, t_eng) / t, 4)
        if best is None or t > best[0]:
            best = (t, key, t_hbm, t_eng, words, e)
    t, key, t_hbm, t_eng, words, e = best
    if t_eng > t_hbm:
        roof = {"bound": "alu", "kernel": key, "achieved": round(words / t / 1e9, 2), "peak": round(ceil[e] / 1e9, 2),
                "unit": "Gwords/s (engine words)", "frac": round(t_eng / t, 4),
                "peak_source": "measured: engine-only kernel (rp_engine_fold) of this engine, this run"}
    else:
        roof = {"bound": "hbm", "kernel": key, "achieved": round(8.0 * N_FILL / t / 1e9, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(t_hbm / t, 4), "peak_source": peak_kind + " (MEASURED_PEAKS.json copy rate)"}
    roof.update({"traffic": TRAFFIC.get(key) if N_FILL == 1 << 28 else None,
                 "hbm_time_ms": round(t_hbm * 1e3, 4), "engine_time_ms": round(t_eng * 1e3, 4),
                 "write_only_gbs": round(ceil["write_gbs"], 1),
                 "frac_vs_write_only": round(max(8.0 * N_FILL / (ceil["write_gbs"] * 1e9), t_eng) / t, 4),
                 "issue_peak_tops": round(issue_peak / 1e12, 2)})
    for eng in sorted(set(x for x, _, _ in fills)):
        roof[f"engine_gwords_per_s:{eng}"] = round(ceil[eng] / 1e9, 2)
        roof[f"engine_issue_frac:{eng}"] = round(ceil[eng] * ENGINE_OPS[eng] / issue_peak, 3)
    roof.update(flat)

    # ---- end to end through the C ABI with host buffers: rp_fill_to_host
    # fills a device staging slot and copies it to pinned host memory inside
    # the library (its copy stream overlaps the next fill); the positions are
    # pinned words written by the stream.  Timed from the first call to the
    # device synchronisation after the last copy.
    e2e = None
    if rank == 0 or world > 1:
        e_steps = max(1, args.steps)
        hbuf = [torch.empty(N_FILL, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        hpos = torch.zeros(e_steps * len(fills), dtype=torch.int64, pin_memory=True)
        codes = {"normal": 3, "exp": 4, "bounded": 2}
        # the link's own rate, the ceiling of this leg (8 bytes per variate
        # cross it): plain 2 GiB device-to-host copies into the same pinned
        # buffers, one step's worth back to back, before and after the leg
        dsrc = torch.zeros(N_FILL, dtype=torch.int64, device="cuda")

        def link_gbs():
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            for j in range(len(fills)):
                hbuf[j % 2].copy_(dsrc, non_blocking=True)
            c1.record()
            c1.synchronize()
            return len(fills) * N_FILL * 8 / (c0.elapsed_time(c1) * 1e-3) / 1e9
        link = link_gbs()
        # untimed: one step of the same calls puts the staging slots and every
        # fill's tables in place
        wpos = torch.zeros(len(fills), dtype=torch.int64, pin_memory=True)
        for j, (e, d, p) in enumerate(fills):
            rp.rp_fill_to_host(e, SEED, spawn, wpos[j:j + 1], codes[d], hbuf[j % 2], m=p[0] if p else 0,
                               cuda_stream=stream)
        torch.cuda.synchronize()
        rp.rp_async_status(None)
        h0 = time.perf_counter()
        i = 0
        for _ in range(e_steps):
            for e, d, p in fills:
                rp.rp_fill_to_host(e, SEED, spawn, hpos[i:i + 1], codes[d], hbuf[i % 2], m=p[0] if p else 0,
                                   cuda_stream=stream)
                i += 1
        torch.cuda.synchronize()
        esec = time.perf_counter() - h0
        rp.rp_async_status(None)
        link_after = link_gbs()
        del dsrc
        e2e = {"value": len(fills) * N_FILL * e_steps / esec, "unit": "variates/s",
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": len(fills) * N_FILL * 8,
               "api": "rp_fill_to_host (C ABI, host buffers; copies inside the library)",
               "d2h_copy_gbs": round(link, 1), "d2h_copy_gbs_after": round(link_after, 1),
               "frac_of_d2h_copy": round(len(fills) * N_FILL * e_steps * 8 / esec / 1e9 / link, 3)}
        del hbuf

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample)
    extras = None
    # the other workloads are single-GPU: only a one-GPU run times them (a
    # multi-GPU run would hold every GPU while rank 0 ran them)
    if world == 1 and not args.no_extras and not args.only and args.log2n == 28:
        del out_f, out_u
        torch.cuda.empty_cache()
        extras = run_extras(rp, stream)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "variates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64/f64",
                "data": "synthetic (seeded engine streams; no dataset)",
                "config": {"workload": WORKLOAD, "n_per_fill": N_FILL, "fills_per_step": len(fills),
                           "l2": "outputs (2 GiB per fill) exceed L2; no flush needed",
                           "parallelism": f"independent streams x{world}",
                           **({"profiling_subset": args.only or f"n=2^{args.log2n}"}
                              if (args.only or args.log2n != 28) else {})},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "extras": extras,
                "clocks": clk}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def measure_ceilings(rp, stream, buf_u, engines):
    """The two measured ceilings of the fills, timed with CUDA events after
    three untimed runs (median of five): the engine-only rate of each
    engine, words/s of rp_engine_fold over N_FILL words (generation as in a
    fill, nothing stored), and the write-only HBM rate, GB/s of filling the
    2 GiB output buffer (torch fill_ of a pattern and zero_, the faster)."""
    import torch
    out = {}
    fold = torch.zeros(1, dtype=torch.uint64, device="cuda")

    def med(f):
        for _ in range(3):
            f()
        ts = sorted(_ev_ms(stream, f) for _ in range(5))
        return ts[2]
    for e in engines:
        if e not in out:
            out[e] = N_FILL / (med(lambda: rp.rp_engine_fold(e, SEED, rp.NO_STREAM, 0, N_FILL, fold, stream)) / 1e3)
    buf = buf_u.view(torch.float64)
    with torch.cuda.stream(stream):
        ms = min(med(lambda: buf.fill_(1.5)), med(lambda: buf.zero_()))
    out["write_gbs"] = 8.0 * N_FILL / (ms / 1e3) / 1e9
    return out


def _ev_ms(stream, fn, reps=1):
    """Device time of fn() on `stream` (CUDA events), min over reps."""
    import torch
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return best


def run_extras(rp, stream):
    """The other workloads, each timed after one untimed run: config 1 (2^20
    words then 2^20 uniforms, xoshiro seed 12345), gamma/beta at n = 2^26
    with their pathwise gradients (xoshiro seed 7, upstream g ~ N(0,1)), the
    derived distributions at n = 2^26, the paper's Philox4x64-10 fills at
    n = 2^28, the batched substream workload (4096 requests, autotuned graph plan, against
    per-request launches) and the multivariate normal (d = 64, 512; n = 2^20)."""
    import numpy as np
    import torch

    from paper_2605_05099_gb300 import inputs
    ex = {}
    # config 1
    w = torch.empty(1 << 20, dtype=torch.uint64, device="cuda")
    u = torch.empty(1 << 20, dtype=torch.float64, device="cuda")

    def c1(cs=stream):
        p = rp.rp_fill_u64("xoshiro256pp", 12345, rp.NO_STREAM, 0, w, cs)
        rp.rp_fill_uniform("xoshiro256pp", 12345, rp.NO_STREAM, p, u, cs)
    c1()
    # one-word fills do not wait for their kernels: 100 back-to-back pairs of
    # calls between the events (host launch rate included) ...
    ms = _ev_ms(stream, lambda: [c1() for _ in range(100)], reps=3) / 100
    # ... and the same 100 pairs captured once into a CUDA graph and replayed
    # (device time alone); the replayed outputs are checked against the calls'
    ref_w, ref_u = w.clone(), u.clone()
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        c1(cap)                                   # tables and jump tables in place on this stream
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap, capture_error_mode="relaxed"):
        for _ in range(100):
            c1(cap)
    w.zero_()
    u.zero_()
    ms_g = _ev_ms(stream, graph.replay, reps=3) / 100
    torch.cuda.synchronize()
    same = bool(torch.equal(w.view(torch.int64), ref_w.view(torch.int64)) and torch.equal(u, ref_u))
    ex["config1_words_then_uniforms"] = {"variates_per_s": 2 * (1 << 20) / (ms_g / 1e3), "ms": ms_g,
                                         "form": "CUDA graph of 100 fill pairs, replayed", "replays": 100,
                                         "replay_outputs_identical": same,
                                         "variates_per_s_calls": 2 * (1 << 20) / (ms / 1e3), "ms_calls": ms}
    del graph, w, u, ref_w, ref_u
    # gamma / beta forward and gradients (config 3)
    n = 1 << 26
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.tensor(inputs.upstream_grads(n), device="cuda")
    dz = torch.empty_like(z)
    fwd, grads = {}, {}
    for a_ in (0.3, 1.0, 2.5, 30.0):
        f = lambda: rp.rp_fill_gamma("xoshiro256pp", 7, rp.NO_STREAM, 0, a_, z, stream)
        f()
        ms = _ev_ms(stream, f)
        fwd[f"gamma({a_})"] = n / (ms / 1e3)
        bg = lambda: rp.rp_gamma_grad(z, a_, g, dz, stream)
        bg()
        grads[f"gamma({a_})"] = n / (_ev_ms(stream, bg) / 1e3)
    dz2 = torch.empty_like(z)
    for ab in ((0.5, 0.5), (2.0, 5.0)):
        f = lambda: rp.rp_fill_beta("xoshiro256pp", 7, rp.NO_STREAM, 0, ab[0], ab[1], z, stream)
        f()
        fwd[f"beta{ab}"] = n / (_ev_ms(stream, f) / 1e3)
        bg = lambda: rp.rp_beta_grad(z, ab[0], ab[1], g, dz, dz2, stream)
        bg()
        grads[f"beta{ab}"] = n / (_ev_ms(stream, bg) / 1e3)
    zx, zy = torch.empty_like(z), torch.empty_like(z)
    for ab in ((2.0, 5.0),):
        rp.rp_fill_beta_xy("xoshiro256pp", 7, rp.NO_STREAM, 0, ab[0], ab[1], z, zx, zy, stream)
        bg = lambda: rp.rp_beta_grad_composed(zx, zy, ab[0], ab[1], g, dz, dz2, stream)
        bg()
        grads[f"beta_composed{ab}"] = n / (_ev_ms(stream, bg) / 1e3)
    del zx, zy
    ex["gamma_beta_fill"] = {"unit": "variates/s", "n": n, **{k: round(v) for k, v in fwd.items()}}
    props = torch.cuda.get_device_properties(0)
    fp64_peak = props.multi_processor_count * FP64_FLOPS_PER_SM_CLK * 2.07e9
    ex["gamma_beta_grads"] = {"unit": "grads/s (per-sample dz/dtheta and the reduced sum)", "n": n,
                              **{k: round(v) for k, v in grads.items()},
                              "fp64_roofline": {k: {"flops_per_grad": f, "achieved_tflops": grads[k] * f / 1e12,
                                                    "peak_tflops": fp64_peak / 1e12,
                                                    "frac": grads[k] * f / fp64_peak}
                                                for k, f in GRAD_FLOPS.items() if k in grads},
                              "fp64_peak": "SMs x 2 DFMA x 2 flops x 2070 MHz (derived, not measured)"}
    # derived distributions (Table "continuous"), fused output transforms of
    # the base fills; xoshiro seed 7, n = 2^26
    dv = {}
    for name, par in (("unif", (-2.0, 3.0)), ("normal_ms", (1.5, 2.0)), ("lognormal", (0.3, 0.7)),
                      ("exp_scale", (2.5,)), ("gamma_scale", (2.5, 0.5)), ("chi2", (5.0,)), ("gumbel", (1.0, 2.0)),
                      ("pareto", (2.0, 3.0)), ("weibull", (1.7, 2.0)), ("gpd", (0.5, 1.5, 0.3)), ("f", (5.0, 7.0)),
                      ("skew_normal", (1.0, 2.0, 4.0)), ("t", (3.0,))):
        f = lambda: rp.rp_fill_derived("xoshiro256pp", 7, rp.NO_STREAM, 0, name, par, z, stream)
        f()
        dv[f"{name}{par}"] = round(n / (_ev_ms(stream, f) / 1e3))
    ex["derived_fill"] = {"unit": "variates/s", "n": n, **dv}
    del z, g, dz, dz2
    torch.cuda.empty_cache()
    # the paper's own Philox (4x64-10) and xoshiro256**, with the paper's
    # default 52-bit uniform, n = 2^28
    n28 = 1 << 28
    of = torch.empty(n28, dtype=torch.float64, device="cuda")
    for eng in ("philox4x64_10", "xoshiro256ss"):
        ph = {}
        for key, f in (("uniform52", lambda: rp.rp_fill_uniform52(eng, SEED, rp.NO_STREAM, 0, of, stream)),
                       ("normal", lambda: rp.rp_fill_normal(eng, SEED, rp.NO_STREAM, 0, of, stream)),
                       ("exp", lambda: rp.rp_fill_exp(eng, SEED, rp.NO_STREAM, 0, of, stream)),
                       ("bounded:6", lambda: rp.rp_fill_bounded(eng, SEED, rp.NO_STREAM, 0, 6, of.view(torch.uint64), stream)),
                       ("bounded:9223372036854775809",
                        lambda: rp.rp_fill_bounded(eng, SEED, rp.NO_STREAM, 0, 2 ** 63 + 1, of.view(torch.uint64), stream))):
            f()
            ms = _ev_ms(stream, f)
            ph[key] = {"ms": round(ms, 4), "variates_per_s": round(n28 / (ms / 1e3))}
        ex[f"{eng}_fills"] = {"n": n28, **ph}
    del of
    torch.cuda.empty_cache()
    # float variants (suffix f), n = 2^28 floats (1 GiB), 4 B per output
    ff = torch.empty(n28, dtype=torch.float32, device="cuda")
    fl = {}
    peaks, _ = _peaks()
    for eng in ENGINES:
        for key, fn in (("uniformf", rp.rp_fill_uniformf), ("normalf", rp.rp_fill_normalf), ("expf", rp.rp_fill_expf)):
            f = lambda: fn(eng, SEED, rp.NO_STREAM, 0, ff, stream)
            f()
            ms = _ev_ms(stream, f, reps=3)
            fl[f"{eng}/{key}"] = {"ms": round(ms, 4), "variates_per_s": round(n28 / (ms / 1e3)),
                                  "write_gbs": round(4.0 * n28 / (ms / 1e3) / 1e9, 1),
                                  "frac_hbm_copy_peak": round(4.0 * n28 / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 3)}
    ex["float_fills"] = {"n": n28, **fl}
    del ff
    torch.cuda.empty_cache()
    # batched substreams (config 4)
    reqs = inputs.batch_workload()
    tot = sum(r["n"] for r in reqs)
    outs = [torch.empty(r["n"], dtype=torch.float64, device="cuda") for r in reqs]
    arr = rp.make_requests([dict(r, out=o) for r, o in zip(reqs, outs)])
    b = {}
    for eng in ("xoshiro256pp", "philox4x32_10"):
        plan = rp.BatchPlan(arr, eng, 99, autotune=True, cuda_stream=stream)
        info = plan.info()
        ms = _ev_ms(stream, lambda: plan.run(stream), reps=2)
        plan.close()
        words = [rp.rp_substream_state(eng, 99, r["stream"]) for r in reqs]

        def per_request():
            for r, o, wd in zip(reqs, outs, words):
                rp.rp_fill_state(eng, wd, 0, r["dist"], o, r["p0"], r["p1"], r["m"], stream)
        ms_pr = _ev_ms(stream, per_request)
        b[eng] = {"variates_per_s": tot / (ms / 1e3), "ms": ms, "per_request_ms": ms_pr,
                  "speedup_vs_per_request": ms_pr / ms, "schedule": info["schedule"], "items": info["items"]}
    ex["batch_substreams"] = {"requests": len(reqs), "variates": tot, **b}
    del outs, arr
    torch.cuda.empty_cache()
    # multivariate normal (config 5)
    m = {}
    n = 1 << 20
    for d in (64, 512):
        mu_h, L_h = inputs.mvn_inputs(d)
        mu, L = torch.tensor(mu_h, device="cuda"), torch.tensor(L_h, device="cuda")
        Z = torch.empty((n, d), dtype=torch.float64, device="cuda")
        X = torch.empty_like(Z)
        G = torch.tensor(np.random.default_rng(3).standard_normal((n, d)), device="cuda")
        gmu = torch.empty(d, dtype=torch.float64, device="cuda")
        gL = torch.empty((d, d), dtype=torch.float64, device="cuda")
        f = lambda: rp.rp_mvn("xoshiro256pp", 3, 1, 0, mu, L, Z, X, stream)
        f()
        ms_f = _ev_ms(stream, f)
        bg = lambda: rp.rp_mvn_grads(G, Z, gmu, gL, stream)
        bg()
        ms_b = _ev_ms(stream, bg)
        fl = 2.0 * n * d * (d + 1) / 2  # triangular L: d (d + 1) / 2 multiply-adds per sample
        m[f"d={d}"] = {"samples_per_s_fwd": n / (ms_f / 1e3), "ms_fwd": ms_f, "ms_bwd": ms_b,
                       "fwd_fp64_tflops_incl_fill": fl / (ms_f / 1e3) / 1e12,
                       "bwd_fp64_tflops": fl / (ms_b / 1e3) / 1e12}
        del Z, X, G
        torch.cuda.empty_cache()
    ex["mvn"] = {"n": n, **m}
    return ex


def run_profile(args):
    """One workload alone, for ncu (--profile KIND; not a bench line):
    gamma:ALPHA, beta:A:B, grad:ALPHA (gamma gradient), bgrad:A:B (beta
    gradient), normalf|expf|uniformf[:ENGINE] (float fills), mvn:D (forward and
    backward, n = 2^20) or batch:ENGINE (4096 requests; --log2n scales the
    request sizes' upper end).  Runs --warmup untimed and --steps timed
    repetitions and prints their mean time."""
    import numpy as np
    import torch

    import paper_2605_05099_gb300 as rp
    from paper_2605_05099_gb300 import inputs
    stream = torch.cuda.current_stream()
    kind, _, rest = args.profile.partition(":")
    vals = [x for x in rest.split(":") if x]
    if kind in ("gamma", "beta", "grad", "bgrad"):
        n = 1 << args.log2n
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        if kind == "bgrad":
            ab = (float(vals[0]), float(vals[1]))
            rp.rp_fill_beta("xoshiro256pp", 7, rp.NO_STREAM, 0, ab[0], ab[1], z, stream)
            g = torch.tensor(inputs.upstream_grads(n), device="cuda")
            dz, dz2 = torch.empty_like(z), torch.empty_like(z)
            f = lambda: rp.rp_beta_grad(z, ab[0], ab[1], g, dz, dz2, stream)
        elif kind == "beta":
            f = lambda: rp.rp_fill_beta("xoshiro256pp", 7, rp.NO_STREAM, 0, float(vals[0]), float(vals[1]), z, stream)
        else:
            a_ = float(vals[0])
            rp.rp_fill_gamma("xoshiro256pp", 7, rp.NO_STREAM, 0, a_, z, stream)
            if kind == "gamma":
                f = lambda: rp.rp_fill_gamma("xoshiro256pp", 7, rp.NO_STREAM, 0, a_, z, stream)
            else:
                g = torch.tensor(inputs.upstream_grads(n), device="cuda")
                dz = torch.empty_like(z)
                f = lambda: rp.rp_gamma_grad(z, a_, g, dz, stream)
    elif kind in ("normalf", "expf", "uniformf"):
        n = 1 << args.log2n
        ff = torch.empty(n, dtype=torch.float32, device="cuda")
        fn = {"normalf": rp.rp_fill_normalf, "expf": rp.rp_fill_expf, "uniformf": rp.rp_fill_uniformf}[kind]
        eng = vals[0] if vals else "xoshiro256pp"
        f = lambda: fn(eng, SEED, rp.NO_STREAM, 0, ff, stream)
    elif kind == "mvn":
        d, n = int(vals[0]), 1 << 20
        mu_h, L_h = inputs.mvn_inputs(d)
        mu, L = torch.tensor(mu_h, device="cuda"), torch.tensor(L_h, device="cuda")
        Z = torch.empty((n, d), dtype=torch.float64, device="cuda")
        X = torch.empty_like(Z)
        G = torch.tensor(np.random.default_rng(3).standard_normal((n, d)), device="cuda")
        gmu = torch.empty(d, dtype=torch.float64, device="cuda")
        gL = torch.empty((d, d), dtype=torch.float64, device="cuda")

        def f():
            rp.rp_mvn("xoshiro256pp", 3, 1, 0, mu, L, Z, X, stream)
            rp.rp_mvn_grads(G, Z, gmu, gL, stream)
    elif kind == "batch":
        hi = 1e7 if args.log2n >= 28 else 10.0 ** (7 - (28 - args.log2n) / 2)
        reqs = inputs.batch_workload(hi=hi)
        outs = [torch.empty(r["n"], dtype=torch.float64, device="cuda") for r in reqs]
        arr = rp.make_requests([dict(r, out=o) for r, o in zip(reqs, outs)])
        plan = rp.BatchPlan(arr, vals[0] if vals else "xoshiro256pp", 99, autotune=False, cuda_stream=stream)
        f = lambda: plan.run(stream)
    else:
        raise SystemExit(f"--profile {args.profile}: unknown workload")
    for _ in range(args.warmup):
        f()
    ms = _ev_ms(stream, lambda: [f() for _ in range(args.steps)]) / max(args.steps, 1)
    print(json.dumps({"profile": args.profile, "log2n": args.log2n, "ms": ms, "not_a_bench_line": True}))


def cpu_baseline(sample):
    """The serial C oracle as it stands, one host core, on a bounded sample of
    the same workload: `sample` variates of each of the 15 fills."""
    import oracle
    t = 0.0
    for e in ENGINES:
        for d, p in SAMPLERS:
            g = oracle.gen(e, SEED)
            t0 = time.perf_counter()
            oracle.fill(g, d, sample, *p)
            t += time.perf_counter() - t0
    total = sample * len(ENGINES) * len(SAMPLERS)
    return {"value": total / t, "unit": "variates/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample} variates of each of the 15 fills (first {sample} of each stream)",
            "seconds": round(t, 3)}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.lib()
    for _ in range(args.warmup):
        cpu_baseline(max(1024, args.cpu_sample // 16))
    t0 = time.perf_counter()
    res = None
    for _ in range(args.steps):
        res = cpu_baseline(args.cpu_sample)
    dt = time.perf_counter() - t0
    total = args.cpu_sample * len(ENGINES) * len(SAMPLERS) * args.steps
    v = total / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "variates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64/f64",
            "data": "synthetic (seeded engine streams; no dataset)",
            "config": {"workload": WORKLOAD, "n_per_fill": N_FILL, "fills_per_step": 15,
                       "sample_per_fill": args.cpu_sample},
            "cpu_baseline": {"value": v, "unit": "variates/s", "cores": 1, "kind": "oracle",
                             "sample": res["sample"] if res else ""},
            "e2e": {"value": v, "unit": "variates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="oracle variates per fill (default 2^24 for the baseline leg, 2^21 per reference step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads (batch, gamma, MVN)")
    ap.add_argument("--only", default=None,
                    help="profiling: run only this fill (e.g. xoshiro256pp/normal); not a bench line")
    ap.add_argument("--log2n", type=int, default=28, help="profiling: n = 2^log2n per fill (bench: 28)")
    ap.add_argument("--profile", default=None, help="profiling: run one other workload alone (see run_profile)")
    args = ap.parse_args()
    global N_FILL
    N_FILL = 1 << args.log2n
    if args.cpu_sample is None:
        args.cpu_sample = (1 << 21) if args.impl == "reference" else (1 << 26)
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
