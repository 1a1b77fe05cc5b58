"""Benchmark of the tropical-algebra hot path on GB300.

One step = one pass of the hot path over the n = 8192 workload:
  * tropical matrix product M = N = K = 8192: int32 (uniform [0, 10^6]) in
    min-plus and max-plus, FP32 (uniform [0, 1)) in min-plus and max-plus;
  * APSP by repeated squaring of one random directed graph, n = 8192, edge
    probability 0.01, int32 weights uniform [1, 1000], 13 squarings with
    early exit (the library picks the exact path from the weight bound).
Metric: tropical Gop/s = (add-min/max terms computed) / time, where a
product is M*N*K terms and APSP counts n^3 per squaring actually computed.

Other keys: the roofline of the dominant kernel (the int32 min-plus product,
ALU-bound; peak = SMs x 128 lanes x SM clock), the CPU oracle timed on a
bounded sample (`cpu_baseline`), the end-to-end number through the public
API with host buffers (`e2e`), SM clocks sampled during the timed region,
and the number of library kernels launched in it.

`--impl reference` times the CPU oracle (the plain triple loop of
oracle/btas_oracle.c) on a bounded row sample of the same products.

Under torchrun (N > 1) every rank runs the same step on its own GPU
(replicas: the workload is independent per GPU); value = total terms of all
ranks / max time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tropical Gop/s & % ALU peak (n=8192); batched APSP graphs/s; serve p50/p99 ms"
N = 8192
LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="btas", choices=["btas", "reference"])
    p.add_argument("--n", type=int, default=N)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fw8192", action="store_true",
                   help="leave the one-off oracle Floyd-Warshall at n = 8192 out of cpu_baseline")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-graphs", type=int, default=512)
    p.add_argument("--batched-profile", action="store_true",
                   help="also run one profiled launch and report cycles per task kind")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the small-config timings (n = 256 solve, n = 4096 packed vs int32, Table II sizes)")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the autotuner (kernels then come from the built-in defaults)")
    p.add_argument("--probe-mix", type=int, default=None,
                   help="with --only probe: run this one mix (btas_measure_issue_rate_ex) and nothing else")
    p.add_argument("--probe-ctas", type=int, default=1, help="with --probe-mix: CTAs per SM (1 or 2)")
    p.add_argument("--paths-dtype", choices=["i32", "f32"], default="i32",
                   help="with --only paths: int32 or binary32 weights")
    p.add_argument("--mid-whi", type=int, default=100,
                   help="with --only mid: largest edge weight (10^6 keeps the squarings on int32)")
    p.add_argument("--fw-int32", action="store_true",
                   help="with --only fw: keep phase 3 on the int32 kernel (no packed phase 3)")
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-rates", default="100,300,1000,3000,5000")
    p.add_argument("--only", default=None,
                   choices=["kernels", "batched", "serve", "next", "tune", "configs", "probe", "mid", "paths", "fw"],
                   help="profiling aids: run one part alone and print its JSON (not a bench line)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(units_per_rank, seconds_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum(units_per_rank) / max(seconds_per_rank)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        load = [s for s in sm if s >= 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---------------------------------------------------------------- inputs
def make_inputs(n):
    import numpy as np
    import gen
    s = gen.BASE_SEED
    Ai = gen.uniform_int(s, 21, (n, n), 0, 10 ** 6)
    Bi = gen.uniform_int(s, 22, (n, n), 0, 10 ** 6)
    Af = gen.uniform_f32(s, 23, (n, n))
    Bf = gen.uniform_f32(s, 24, (n, n))
    W = gen.random_graph(s, 2, n, 0.01, 1, 1000)
    return {"Ai": Ai, "Bi": Bi, "Af": Af, "Bf": Bf, "W": W,
            "BiT": np.ascontiguousarray(Bi.T), "BfT": np.ascontiguousarray(Bf.T)}


# ------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(inp, budget_s=15.0, threads=None):
    """Oracle triple loop on a bounded row sample of the four products;
    returns (Gop/s, threads, sample description)."""
    import oracle
    n = inp["Ai"].shape[0]
    threads = threads or os.cpu_count() or 1
    oracle.set_threads(threads)
    try:
        rows = max(1, threads)
        t0 = time.perf_counter()
        oracle.tgemm(0, inp["Ai"][:rows], inp["Bi"])
        dt = time.perf_counter() - t0
        per_row = dt / rows
        R = int(max(rows, min(n, budget_s / 4 / per_row)))
        R = max(threads, (R // threads) * threads)
        total = 0.0
        t0 = time.perf_counter()
        for sr, A, B in ((0, "Ai", "Bi"), (1, "Ai", "Bi"), (0, "Af", "Bf"), (1, "Af", "Bf")):
            oracle.tgemm(sr, inp[A][:R], inp[B])
            total += float(R) * n * n
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return total / dt / 1e9, threads, f"{R} rows x {n} x {n} of each of the 4 products ({total:.3g} terms, {dt:.1f} s)"


def oracle_single_thread_gops(n=1024):
    """The oracle's int32 min-plus product at n^3 on ONE host thread (the
    paper's single-thread CPU methodology), in Gop/s."""
    import gen
    import oracle
    A = gen.uniform_int(gen.BASE_SEED, 91, (n, n), 0, 10 ** 6)
    B = gen.uniform_int(gen.BASE_SEED, 92, (n, n), 0, 10 ** 6)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.tgemm(0, A, B)
    return round(float(n) ** 3 / (time.perf_counter() - t0) / 1e9, 3)


def oracle_fw_n256_us():
    """The oracle's Floyd-Warshall (one thread) on the n = 256 graph of the
    config timings, in microseconds: the CPU side of that comparison."""
    import gen
    import oracle
    W = gen.random_graph(gen.BASE_SEED, 1, 256, 0.1, 1, 100)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.floyd_warshall(W)
    return round((time.perf_counter() - t0) * 1e6, 1)


def cpu_model():
    """Host CPU model string (Linux /proc/cpuinfo), for the cpu_baseline key."""
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model Name", "CPU part"):
        for line in txt.splitlines():
            if line.split(":")[0].strip() == key:
                v = line.split(":", 1)[1].strip()
                return v if key != "CPU part" else f"Arm CPU part {v} ({txt.count('processor')} cores listed)"
    return "unknown"


def oracle_apsp_timings(threads, fw_n8192=True):
    """The oracle on the APSP configurations, timed once each with `threads`
    host threads: Floyd-Warshall (Algorithm 2, rows of one pivot in
    parallel) on the n = 256 graph (p = 0.1, w in [1, 100]), the n = 4096
    graph (p = 0.05, w in [1, 7]) and, unless disabled, the n = 8192 graph
    of the step (p = 0.01, w in [1, 1000]); APSP by repeated squaring on the
    n = 256 graph."""
    import gen
    import oracle
    s = gen.BASE_SEED
    out = {"threads": threads}
    oracle.set_threads(threads)
    try:
        W1 = gen.random_graph(s, 1, 256, 0.1, 1, 100)
        t0 = time.perf_counter()
        oracle.floyd_warshall(W1)
        out["fw_n256_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        t0 = time.perf_counter()
        oracle.apsp_squaring(W1)
        out["squaring_n256_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
        W3 = gen.random_graph(s, 3, 4096, 0.05, 1, 7)
        t0 = time.perf_counter()
        oracle.floyd_warshall(W3)
        dt = time.perf_counter() - t0
        out["fw_n4096_s"] = round(dt, 2)
        out["fw_n4096_grelax_s"] = round(4096.0 ** 3 / dt / 1e9, 2)
        if fw_n8192:
            W2 = gen.random_graph(s, 2, 8192, 0.01, 1, 1000)
            t0 = time.perf_counter()
            oracle.floyd_warshall(W2)
            dt = time.perf_counter() - t0
            out["fw_n8192_s"] = round(dt, 2)
            out["fw_n8192_grelax_s"] = round(8192.0 ** 3 / dt / 1e9, 2)
    finally:
        oracle.set_threads(1)
    return out


PROBE_MIXES = ((0, "int32_dpx"), (4, "int32_iadd_min3"), (5, "int32_imad_min3"), (6, "int32_split_imad5_dpx3"),
               (1, "fp32_f32x2_min3"), (7, "fp32_2fadd_min3"), (2, "u16x2_dpx"), (3, "ffma_reference"),
               (8, "ffma_imm_operand"))
PROBE_DIAG_MIXES = ((9, "fp32_2fadd_imm_min3"), (10, "int32_iadd_imm_min3"),
                    (11, "int32_dpx_imm"), (12, "int32_3pipe_dpx3_imad3_fadd2"), (13, "dpx3_f32x2_5"),
                    (14, "int32_imad_imm_min3"), (15, "int32_dpx_a_rotated"))


def issue_probe(btas, full=False):
    """Measured issue ceilings of the inner-loop instruction mixes, in
    tropical terms per clock per SM (btas_measure_issue_rate).  With `full`,
    also the diagnostic mixes, each at 1 and 2 CTAs per SM."""
    probe = {}
    mixes = PROBE_MIXES + (PROBE_DIAG_MIXES if full else ())
    for ctas in ((1, 2) if full else (1,)):
        for mix, name in mixes:
            key = name if ctas == 1 else f"{name}@2cta"
            try:
                probe[key] = round(btas.measure_issue_rate(mix, ctas), 1)
            except Exception as exc:  # diagnostic only
                probe[key] = f"unavailable: {exc}"
    return probe


def workload_config(n, world):
    """The `config` of a bench line (both arms)."""
    S = max(0, (n - 2).bit_length()) if n > 2 else 0
    return {"workload": f"tropical product {n}^3 (int32 [0,1e6] and f32 [0,1), min-plus and max-plus) + "
                        f"int32 APSP n={n} p=0.01 w[1,1000] ({S} squarings, early exit)",
            "n": n, "b_operand": "supplied transposed (BTAS_GEMM_TRANS_B)",
            "l2": (f"inputs ({n * n * 4 >> 20} MiB per matrix) larger than L2 (129 MB)" if n * n * 4 > 129e6
                   else f"inputs ({n * n * 4 >> 20} MiB per matrix) fit in L2 (129 MB): not an L2-cold number"),
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import gen
    n = args.n
    inp = {"Ai": gen.uniform_int(gen.BASE_SEED, 21, (n, n), 0, 10 ** 6),
           "Bi": gen.uniform_int(gen.BASE_SEED, 22, (n, n), 0, 10 ** 6),
           "Af": gen.uniform_f32(gen.BASE_SEED, 23, (n, n)), "Bf": gen.uniform_f32(gen.BASE_SEED, 24, (n, n))}
    total_steps = args.steps + args.warmup
    budget = max(2.0, min(20.0, 150.0 / max(total_steps, 1)))
    rates = []
    sample = ""
    threads = os.cpu_count() or 1
    step_s = []
    for i in range(total_steps):
        t0 = time.perf_counter()
        rate, threads, sample = cpu_oracle_rate(inp, budget_s=budget, threads=threads)
        if i >= args.warmup:
            rates.append(rate)
            step_s.append(time.perf_counter() - t0)
    value = statistics.median(rates)
    line = {"metric": METRIC, "value": round(value, 3), "unit": "Gop/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.median(step_s) * 1e3, 1) if step_s else None,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic", "impl": "reference",
            "config": workload_config(n, args.gpus),
            "cpu_baseline": {"value": round(value, 3), "unit": "Gop/s", "cores": threads, "kind": "oracle",
                             "sample": sample + "; the APSP squarings are the same int32 min-plus products, "
                                       "so the product rate stands for the whole step"},
            "e2e": {"value": round(value, 3), "unit": "Gop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU arm
def autotune(btas, combos):
    """Run the library's autotuner once per (semiring, dtype, m, n, k); the
    library then uses the winners for those size buckets.  Untimed set-up."""
    names = {btas.I32: "i32", btas.F32: "f32", btas.U16: "u16"}
    out = {}
    t0 = time.perf_counter()
    for sr, dt, m, n, k in combos:
        r = btas.tune_gemm(sr, dt, m, n, k)
        key = f"{names[dt]}_{'min' if sr == btas.MINPLUS else 'max'}_{m}x{n}x{k}"
        out[key] = {"variant": r["variant"], "ns": r["ns"], "cfg": r["cfg"], "tile": [r["tile_m"], r["tile_n"]],
                    "group_m": r["group_m"], "candidates": r["candidates"],
                    "top_s": round(r["terms_per_second"] / 1e12, 2)}
    return out, round(time.perf_counter() - t0, 1)


def run_btas(args):
    import numpy as np
    import torch
    import paper_1701_04733_gb300 as btas

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n
    inp = make_inputs(n)
    dev = {k: torch.from_numpy(v).cuda() for k, v in inp.items()}
    Ci = torch.empty((n, n), dtype=torch.int32, device="cuda")
    Cf = torch.empty((n, n), dtype=torch.float32, device="cuda")
    D = torch.empty((n, n), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    n3 = float(n) ** 3
    tuned, tune_s = ({}, 0.0)
    if not args.no_tune:
        tuned, tune_s = autotune(btas, [(sr, dt, n, n, n) for dt in (btas.I32, btas.F32) for sr in (0, 1)] +
                                 [(0, btas.U16, n, n, n)])

    # APSP: squarings actually computed (early exit) for this fixed graph
    _, info = btas.apsp(dev["W"], out=D, info=True)
    S = btas.btas_apsp_squarings(n)
    computed = min(S, info["squarings"] + 1)
    units_per_step = 4 * n3 + computed * n3
    ev = {}

    def step(record=False):
        def rec(name):
            if record:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                ev.setdefault(name, []).append(e)
        rec("i32min0")
        btas.gemm(dev["Ai"], dev["BiT"], btas.MINPLUS, out=Ci, trans_b=True)
        rec("i32min1")
        btas.gemm(dev["Ai"], dev["BiT"], btas.MAXPLUS, out=Ci, trans_b=True)
        rec("f32min0")
        btas.gemm(dev["Af"], dev["BfT"], btas.MINPLUS, out=Cf, trans_b=True)
        rec("f32min1")
        btas.gemm(dev["Af"], dev["BfT"], btas.MAXPLUS, out=Cf, trans_b=True)
        rec("apsp0")
        btas.apsp(dev["W"], out=D)
        rec("apsp1")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = btas.btas_kernel_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        torch.cuda.synchronize()
    launches = btas.btas_kernel_launches() - launches0
    seconds = t0.elapsed_time(t1) / 1e3
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([seconds], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        seconds = float(tt.item())
        dist.barrier()
    value = aggregate([units_per_step * args.steps] * world, [seconds]) / 1e9

    def dur(a, b):
        return statistics.mean(x.elapsed_time(y) for x, y in zip(ev[a], ev[b])) / 1e3

    t_i32min = dur("i32min0", "i32min1")
    t_i32max = dur("i32min1", "f32min0")
    t_f32min = dur("f32min0", "f32min1")
    t_f32max = dur("f32min1", "apsp0")
    t_apsp = dur("apsp0", "apsp1")
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or peaks().get("sm_max_mhz") or 2070.0
    peak_tops = sms * LANES_PER_SM * max_mhz * 1e6 / 1e12

    def roof(name, terms, secs):
        achieved = terms / secs / 1e12
        r = {"bound": "alu", "kernel": name, "achieved": round(achieved, 3), "peak": round(peak_tops, 3),
             "unit": "Top/s", "frac": round(achieved / peak_tops, 4),
             "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes x {max_mhz:.0f} MHz (max SM clock), "
                           "one tropical term per lane per clock",
             "frac_at_median_clock": (round(achieved / (sms * LANES_PER_SM * clocks['sm_mhz'] * 1e-6), 4)
                                      if clocks.get("sm_mhz") else None)}
        return r
    traffic = {}
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f)
    kern = {"tgemm_nt int32 min/max-plus 8192^3": (2 * n3, t_i32min + t_i32max),
            "tgemm_nt fp32 min/max-plus 8192^3": (2 * n3, t_f32min + t_f32max),
            f"APSP squarings n=8192 ({info['path']})": (computed * n3, t_apsp)}
    dom = max(kern, key=lambda k: kern[k][1])
    roofline = roof(dom, *kern[dom])
    roofline["traffic"] = traffic.get(dom)
    roofline["share_of_step"] = round(kern[dom][1] / (seconds / args.steps), 3)
    roof_i32 = roof("tgemm_nt int32 min-plus 8192^3", n3, t_i32min)
    roof_i32["traffic"] = traffic.get("tgemm_nt int32 min-plus 8192^3")
    # measured issue ceilings of the instruction mixes (terms / clock / SM)
    probe = issue_probe(btas)
    int_best = max((v for k, v in probe.items() if k.startswith("int32") and isinstance(v, float)), default=None)
    if int_best:
        ceil = int_best * sms * max_mhz * 1e6 / 1e12
        roof_i32["measured_issue_ceiling_tops"] = round(ceil, 3)
        roof_i32["measured_issue_ceiling_basis"] = "best int32 instruction mix of the probe"
        roof_i32["frac_of_measured_ceiling"] = round(n3 / t_i32min / 1e12 / ceil, 4)
    # fp32: the same lane-clock peak, and the survey's two-instruction count
    # (FADD + FMNMX per term: half the lane-clock peak in terms); the kernel
    # itself issues one instruction per term (add.f32x2 + 3-input min per
    # two terms)
    roof_f32 = roof("tgemm_nt fp32 min-plus 8192^3", n3, t_f32min)
    roof_f32["traffic"] = traffic.get("tgemm_nt fp32 min-plus 8192^3")
    roof_f32["frac_two_instruction_basis"] = round(2 * n3 / t_f32min / 1e12 / peak_tops, 4)
    if isinstance(probe.get("fp32_f32x2_min3"), float):
        ceil_f = probe["fp32_f32x2_min3"] * sms * max_mhz * 1e6 / 1e12
        roof_f32["measured_issue_ceiling_tops"] = round(ceil_f, 3)
        roof_f32["frac_of_measured_ceiling"] = round(n3 / t_f32min / 1e12 / ceil_f, 4)
    if isinstance(probe.get("ffma_reference"), float) and isinstance(probe.get("ffma_imm_operand"), float):
        # the same FFMA stream with one register operand replaced by an
        # immediate: the speed-up shows the register-operand read limit
        roof_i32["limiter"] = ("register-operand reads, about 2 warp-wide 32-bit operands per scheduler per "
                               "clock: FFMA with 3 register operands "
                               f"{probe['ffma_reference']} vs 2 register operands {probe['ffma_imm_operand']} "
                               "terms/clk/SM; a product term reads >= 3 registers (A, B, accumulator)")

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Gop/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(seconds / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32", "data": "synthetic",
        "config": {**workload_config(n, world), "apsp_path": info["path"], "apsp_squarings_computed": computed,
                   "apsp_bound": info["bound"]},
        "parts_ms": {"i32_minplus": round(t_i32min * 1e3, 3), "i32_maxplus": round(t_i32max * 1e3, 3),
                     "f32_minplus": round(t_f32min * 1e3, 3), "f32_maxplus": round(t_f32max * 1e3, 3),
                     "apsp": round(t_apsp * 1e3, 3)},
        "parts_gops": {"i32_minplus": round(n3 / t_i32min / 1e9, 1), "i32_maxplus": round(n3 / t_i32max / 1e9, 1),
                       "f32_minplus": round(n3 / t_f32min / 1e9, 1), "f32_maxplus": round(n3 / t_f32max / 1e9, 1),
                       "apsp": round(computed * n3 / t_apsp / 1e9, 1)},
        "roofline": roofline,
        "roofline_int32_minplus": roof_i32,
        "roofline_fp32_minplus": roof_f32,
        "issue_probe_terms_per_clk_per_sm": probe,
        "clocks": clocks,
        "gpu_launches": launches,
        "autotune": {"choices": tuned, "tuning_s": tune_s} if tuned else "off (built-in defaults)",
    }

    # the same APSP held to int32 on every squaring (no packed representation):
    # the rate that does not depend on this graph's small distances
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D32 = torch.empty_like(D)
    _, info32 = btas.apsp(dev["W"], out=D32, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32, info=True)
    e0.record(stream)
    btas.apsp(dev["W"], out=D32, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32)
    e1.record(stream)
    torch.cuda.synchronize()
    t32 = e0.elapsed_time(e1) / 1e3
    sq32 = min(S, info32["squarings"] + 1)
    line["apsp_int32_only"] = {"ms": round(t32 * 1e3, 3), "squarings_computed": sq32,
                               "gops": round(sq32 * n3 / t32 / 1e9, 1), "identical_to_step_result":
                               bool(torch.equal(D32, D))}
    del D32
    if not args.no_e2e:
        line["e2e"] = e2e(args, inp, btas, torch, units_per_step)
    if not args.no_configs:
        line["config_timings"] = config_timings(args, btas, torch)
    if not args.no_batched:
        del dev, Ci, Cf, D
        torch.cuda.empty_cache()
        line["batched"] = batched(args, btas, torch)
    if not args.no_serve:
        torch.cuda.empty_cache()
        line["serve"] = serve(args, btas, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, sample = cpu_oracle_rate(inp)
        line["cpu_baseline"] = {"value": round(rate, 3), "unit": "Gop/s", "cores": threads, "kind": "oracle",
                                "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                                "fw_n256_us_1_thread": oracle_fw_n256_us(),
                                "int32_product_1024_gops_1_thread": oracle_single_thread_gops(),
                                "apsp_all_threads": oracle_apsp_timings(threads, fw_n8192=not args.no_fw8192)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def batched(args, btas, torch):
    """Batched workload: G random graphs, n uniform in [32, 1024], p = 0.1,
    int32 w in [1, 100] (APSP), plus G FP32 max-plus products of the same
    sizes, U[0, 1).  One persistent graph-captured launch vs one library call
    (and its launches) per problem, same results."""
    import numpy as np
    import gen
    G = args.batched_graphs
    sizes = gen.graph_sizes(gen.BASE_SEED, 40, G, 32, 1024)
    Ws, Ds, Ls, As, Bs, Cs, Cl = [], [], [], [], [], [], []
    for i, n in enumerate(sizes):
        n = int(n)
        W = torch.from_numpy(gen.random_graph(gen.BASE_SEED, 1000 + i, n, 0.1, 1, 100)).cuda()
        Ws.append(W)
        Ds.append(torch.empty_like(W))
        Ls.append(torch.empty_like(W))
        As.append(torch.from_numpy(gen.uniform_f32(gen.BASE_SEED, 3000 + i, (n, n))).cuda())
        Bs.append(torch.from_numpy(gen.uniform_f32(gen.BASE_SEED, 5000 + i, (n, n))).cuda())
        Cs.append(torch.empty_like(As[-1]))
        Cl.append(torch.empty_like(As[-1]))
    stream = torch.cuda.current_stream()

    def make_batch():
        bb = btas.Batch()
        for W, D in zip(Ws, Ds):
            bb.add_apsp(W, D)
        for A, B_, C in zip(As, Bs, Cs):
            bb.add_gemm(A, B_, C, btas.MAXPLUS)
        return bb

    # output tile per instance from the batched launch's autotuner (timed
    # against the untuned 128 x 128 plan of the same batch)
    t_untuned, tiles, tile_tune_s = None, None, 0.0
    if not args.no_tune:
        btas.btas_batch_tune_clear()
        b0 = make_batch()
        b0.launch()
        b0.wait()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_untuned = None
        for _ in range(3):
            e0.record(stream)
            b0.launch()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            t_untuned = t if t_untuned is None else min(t_untuned, t)
        b0.close()
        t_tt = time.perf_counter()
        table = btas.batch_tune(1024)
        tile_tune_s = round(time.perf_counter() - t_tt, 2)
        tiles = {kind: {"buckets_on_64x64": [f"{lo}-{hi}" for lo, hi, tl, _, _ in rows if tl == 64],
                        "ms_128_vs_64": {f"{lo}-{hi}": [m1, m2] for lo, hi, _, m1, m2 in rows[::8]}}
                 for kind, rows in table.items()}
    b = make_batch()
    n64 = sum(1 for n in sizes if btas.btas_batch_tile(0, int(n)) == 64) if tiles else 0
    selected = b.select_tiles() if tiles else None

    def run_batch():
        b.launch()

    # two single-call modes: adaptive precision (u16x2 where exact; reads a
    # flag back after every squaring) and int32 kernels with the device-side
    # early exit (no host round trips); the baseline is the faster one
    def loop_with(flags):
        def run():
            for W, D in zip(Ws, Ls):
                btas.apsp(W, out=D, flags=flags)
            for A, B_, C in zip(As, Bs, Cl):
                btas.gemm(A, B_, btas.MAXPLUS, out=C)
        return run

    # the one-call-per-problem baseline runs the autotuner's kernels: one
    # tuning run per size bucket (largest size of the bucket) and kernel family
    tuned = 0
    if not args.no_tune:
        by_bucket = {}
        for n in sizes:
            bkt = int(n - 1).bit_length()
            by_bucket[bkt] = max(by_bucket.get(bkt, 0), int(n))
        combos = [(sr, dt, n, n, n) for n in sorted(by_bucket.values())
                  for sr, dt in ((0, btas.U16), (0, btas.I32), (1, btas.F32))]
        tuned = len(autotune(btas, combos)[0])

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return best

    t_batch = timed(run_batch)
    b.wait()
    modes = {"adaptive": btas.APSP_EARLY_EXIT, "int32_device_exit": btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32}
    loop_t, loop_l, same = {}, {}, True
    for name, flags in modes.items():
        l0 = btas.btas_kernel_launches()
        loop_t[name] = timed(loop_with(flags))
        loop_l[name] = (btas.btas_kernel_launches() - l0) // 4
        same = same and all(torch.equal(x, y) for x, y in zip(Ds, Ls)) and \
            all(torch.equal(x, y) for x, y in zip(Cs, Cl))
        for L in Ls:
            L.fill_(-1)
    best = min(loop_t, key=loop_t.get)
    t_loop, loop_launches = loop_t[best], loop_l[best]
    gemm_terms = float(sum(int(n) ** 3 for n in sizes))
    tasks = b.tasks
    b.close()
    prof = None
    if args.batched_profile:
        pb = btas.Batch(profile=True)
        for W, D in zip(Ws, Ls):
            pb.add_apsp(W, D)
        for A, B_, C in zip(As, Bs, Cl):
            pb.add_gemm(A, B_, C, btas.MAXPLUS)
        pb.launch()
        pb.wait()
        raw = pb.profile()
        pb.close()
        total = sum(v["cycles"] for k, v in raw.items() if k != "wait") or 1
        mhz = peaks().get("sm_max_mhz") or 2070.0
        prof = {k: {"tasks": v["tasks"], "share_of_task_cycles": round(v["cycles"] / total, 4),
                    "us_per_task": round(v["cycles"] / max(v["tasks"], 1) / mhz, 2)}
                for k, v in raw.items() if v["tasks"]}
    return {"workload": f"{G} APSP graphs n~U[32,1024] p=0.1 w[1,100] int32 + {G} fp32 max-plus products same sizes",
            "batch_ms": round(t_batch * 1e3, 3), "loop_ms": round(t_loop * 1e3, 3),
            "graphs_per_s": round(G / t_batch, 1), "loop_graphs_per_s": round(G / t_loop, 1),
            "speedup_vs_one_launch_per_problem": round(t_loop / t_batch, 3),
            "batch_launches": 1, "loop_launches": int(loop_launches), "tasks": tasks,
            "gemm_terms": gemm_terms, "identical_results": bool(same),
            "loop_kernels": f"autotuned ({tuned} size-bucket entries)" if tuned else "built-in defaults",
            "batch_ms_untuned_128x128": round(t_untuned * 1e3, 3) if t_untuned else None,
            "task_tiles": {"tuning_s": tile_tune_s, "graphs_on_64x64_by_table": n64,
                           "selected_plan": selected[0], "plan_ms": selected[1], "table": tiles} if tiles else
            "off (128 x 128 for every instance)",
            "profile": prof,
            "loop_apsp_mode": best, "loop_ms_by_mode": {k: round(v * 1e3, 3) for k, v in loop_t.items()}}


def serve(args, btas, torch):
    """Serving workload: Poisson arrivals of mixed requests -- 50 % APSP
    (int32, p = 0.1, w in [1, 100]) and 50 % single tropical products (n x n x n,
    min/max-plus 50/50, int32/fp32 50/50) -- with n log-uniform in [64, 4096],
    host buffers, admitted under a 40 GB device-memory budget.  For every
    arrival rate: p50/p99 latency (scheduled arrival -> result in host memory)
    and completed requests/s, for the continuous-batching server and for plain
    serial execution (one request at a time through the single calls).

    Every in-flight server request writes its own pinned output buffer: each
    template keeps a pool of buffers that are reused in completion order
    (when the pool of a template is exhausted the producer waits for that
    template's oldest request, and that wait counts in the latency, which is
    always measured from the scheduled arrival).  After each rate the last
    result held by every buffer is compared bit for bit with the single-call
    result of its template."""
    import collections
    import threading
    import numpy as np
    import gen
    T = 32
    sizes = gen.loguniform_sizes(gen.BASE_SEED, 60, T, 64, 4096)
    kinds = gen.uniform_int(gen.BASE_SEED, 61, (T,), 0, 1)
    srs = gen.uniform_int(gen.BASE_SEED, 62, (T,), 0, 1)
    dts = gen.uniform_int(gen.BASE_SEED, 63, (T,), 0, 1)
    R = args.serve_requests
    pick = gen.uniform_int(gen.BASE_SEED, 64, (R,), 0, T - 1)
    u = gen.uniform_unit_f64(gen.BASE_SEED, 65, np.arange(R, dtype=np.uint64))
    gaps = -np.log1p(-u)  # exponential(1)
    counts = np.bincount(pick, minlength=T)
    tmpl, expect, pools = [], [], []
    out_bytes = [int(sizes[i]) ** 2 * 4 for i in range(T)]
    demand = sum(out_bytes[i] * counts[i] for i in range(T))
    # pinned bytes of all output pools together: every request its own buffer
    # when a quarter of the host's available memory holds them, else a share
    mem_avail = 0
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    mem_avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    pool_cap = int(min(demand, max(6 << 30, mem_avail // 4)))
    t_pool = time.perf_counter()
    for i in range(T):
        n = int(sizes[i])
        odt = torch.int32 if (kinds[i] == 0 or dts[i] == 0) else torch.float32
        if kinds[i] == 0:
            W = torch.from_numpy(gen.random_graph(gen.BASE_SEED, 6000 + i, n, 0.1, 1, 100)).pin_memory()
            tmpl.append(("apsp", n, W))
            expect.append(btas.apsp(W.cuda()).cpu())
        else:
            if dts[i] == 0:
                A = gen.uniform_int(gen.BASE_SEED, 7000 + i, (n, n), 0, 10 ** 6)
                B = gen.uniform_int(gen.BASE_SEED, 8000 + i, (n, n), 0, 10 ** 6)
            else:
                A = gen.uniform_f32(gen.BASE_SEED, 7000 + i, (n, n))
                B = gen.uniform_f32(gen.BASE_SEED, 8000 + i, (n, n))
            tmpl.append(("gemm", n, torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(),
                         int(srs[i])))
            expect.append(btas.gemm(tmpl[-1][2].cuda(), tmpl[-1][3].cuda(), tmpl[-1][4]).cpu())
        share = out_bytes[i] * counts[i] / max(demand, 1)
        k = int(max(2, min(counts[i], pool_cap * share // out_bytes[i]))) if counts[i] else 1
        pools.append([torch.empty((n, n), dtype=odt).pin_memory() for _ in range(k)])
    torch.cuda.synchronize()
    t_pool = time.perf_counter() - t_pool

    def pct(lat):
        lat = np.sort(np.asarray(lat))
        return float(np.percentile(lat, 50) * 1e3), float(np.percentile(lat, 99) * 1e3)

    def top_share(lat, reqs):
        """Kind and size of the slowest 1 % of the requests."""
        order = np.argsort(np.asarray(lat))[::-1][:max(1, len(lat) // 100)]
        kinds_top = collections.Counter(tmpl[pick[r]][0] for r in order)
        return {"apsp": kinds_top.get("apsp", 0), "gemm": kinds_top.get("gemm", 0),
                "median_n": int(np.median([tmpl[pick[r]][1] for r in order]))}

    out = {"workload": "Poisson arrivals; 50% APSP int32 (p=0.1, w[1,100]) / 50% tropical product "
                       "(min/max 50/50, int32/fp32 50/50); n log-uniform [64,4096]; host buffers; 40 GB budget",
           "requests_per_rate": R, "templates": T,
           "latency": "scheduled Poisson arrival -> result in pinned host memory",
           "output_buffers": f"one per in-flight request: {sum(len(p) for p in pools)} pinned buffers "
                             f"({sum(len(pools[t]) * out_bytes[t] for t in range(T)) / 1e9:.1f} GB of {demand / 1e9:.1f} GB "
                             f"for one per request; host MemAvailable {mem_avail / 1e9:.0f} GB) in per-template pools "
                             f"reused in completion order; set-up {t_pool:.1f} s",
           "rates": []}
    checked = mismatched = 0
    # one long-lived server for every rate, as a deployment runs it
    srv = btas.Server(40 << 30)
    for rate in [float(x) for x in args.serve_rates.split(",")]:
        arrivals = np.cumsum(gaps / rate)
        # continuous-batching server
        steps0 = srv.stats()["steps"]
        tickets = [None] * R
        lag = np.zeros(R)
        holder = [collections.deque() for _ in range(T)]   # (ticket, buffer index) in submission order
        free = [collections.deque(range(len(pools[t]))) for t in range(T)]
        last = [[None] * len(pools[t]) for t in range(T)]  # last request written to each buffer

        def producer():
            start = time.perf_counter()
            for i in range(R):
                while time.perf_counter() - start < arrivals[i]:
                    time.sleep(max(0.0, min(1e-4, arrivals[i] - (time.perf_counter() - start))))
                t = int(pick[i])
                if not free[t]:
                    tk, b = holder[t][0]
                    while srv.poll(tk)["state"] < 2:  # wait for the template's oldest request
                        time.sleep(5e-5)
                    holder[t].popleft()
                    free[t].append(b)
                elif holder[t] and srv.poll(holder[t][0][0])["state"] >= 2:
                    free[t].append(holder[t].popleft()[1])
                b = free[t].popleft()
                tp = tmpl[t]
                lag[i] = time.perf_counter() - start - arrivals[i]
                if tp[0] == "apsp":
                    tickets[i] = srv.submit_apsp(tp[2], pools[t][b])
                else:
                    tickets[i] = srv.submit_gemm(tp[2], tp[3], pools[t][b], tp[4])
                holder[t].append((tickets[i], b))
                last[t][b] = i
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        srv.wait_all(600)
        polls = [srv.poll(tk) for tk in tickets]
        stats = srv.stats()
        stats["steps"] -= steps0
        lat = [p["t_done"] - p["t_submit"] + lag[i] for i, p in enumerate(polls)]
        service = collections.defaultdict(list)  # admission -> done, per template
        for i, p in enumerate(polls):
            service[int(pick[i])].append(p["t_done"] - p["t_admit"])
        failed = sum(1 for p in polls if p["state"] != 2)
        span = max(p["t_done"] for p in polls) - min(p["t_submit"] - lag[i] for i, p in enumerate(polls))
        p50, p99 = pct(lat)
        for t in range(T):
            for b, r in enumerate(last[t]):
                if r is None:
                    continue
                checked += 1
                got, ref = pools[t][b], expect[t]
                if got.dtype == torch.float32:
                    got, ref = got.view(torch.int32), ref.view(torch.int32)
                mismatched += 0 if torch.equal(got, ref) else 1
        # serial plain execution of the same arrival sequence
        slat = []
        sservice = collections.defaultdict(list)
        start = time.perf_counter()
        for i in range(R):
            now = time.perf_counter() - start
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            t_begin = time.perf_counter()
            t = int(pick[i])
            tp = tmpl[t]
            if tp[0] == "apsp":
                d = btas.apsp(tp[2].cuda(non_blocking=True))
                pools[t][0].copy_(d)
            else:
                c = btas.gemm(tp[2].cuda(non_blocking=True), tp[3].cuda(non_blocking=True), tp[4])
                pools[t][0].copy_(c)
            torch.cuda.synchronize()
            slat.append(time.perf_counter() - start - arrivals[i])
            sservice[t].append(time.perf_counter() - t_begin)
        sspan = time.perf_counter() - start
        s50, s99 = pct(slat)
        out["rates"].append({"rate_req_s": rate, "p50_ms": round(p50, 3), "p99_ms": round(p99, 3),
                             "throughput_req_s": round(R / span, 1), "steps": stats["steps"], "failed": failed,
                             "slowest_1pct": top_share(lat, R),
                             "serial_p50_ms": round(s50, 3), "serial_p99_ms": round(s99, 3),
                             "serial_throughput_req_s": round(R / sspan, 1),
                             "serial_slowest_1pct": top_share(slat, R),
                             "large_template_service_ms": {
                                 f"{tmpl[t][0]} n={tmpl[t][1]}": [round(float(np.median(service[t])) * 1e3, 2),
                                                                  round(float(np.median(sservice[t])) * 1e3, 2)]
                                 for t in sorted(service, key=lambda t: -tmpl[t][1])[:6]}})
    srv.close()
    out["results_checked"] = checked
    out["results_mismatched"] = mismatched
    return out


def e2e(args, inp, btas, torch, units_per_step):
    """Same step through the public API with pinned host buffers: every step
    copies its inputs host -> device and its results device -> host.  The
    copies run on two copy streams (one per direction) and overlap the
    compute: each product waits only for its own operands, each result is
    read back as soon as its kernel is done, and the next step's inputs are
    uploaded while the current step computes (device input and result
    buffers are double-buffered, with events guarding their reuse)."""
    n = inp["Ai"].shape[0]
    h = {k: torch.from_numpy(v).pin_memory() for k, v in inp.items() if k in ("Ai", "BiT", "Af", "BfT", "W")}
    names = ("i32_min", "i32_max", "f32_min", "f32_max", "apsp")
    outs = {k: torch.empty((n, n), dtype=torch.float32 if k.startswith("f32") else torch.int32).pin_memory()
            for k in names}
    d = [{k: torch.empty_like(v, device="cuda") for k, v in h.items()} for _ in range(2)]
    dres = [{k: torch.empty_like(outs[k], device="cuda") for k in names} for _ in range(2)]
    comp = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    bi = sum(v.numel() * 4 for v in h.values())
    bo = sum(v.numel() * 4 for v in outs.values())
    ready = [{}, {}]
    inputs_free = [None, None]   # comp: the last kernel that read the set's inputs
    results_read = [None, None]  # down: the last read-back of the set's results

    def upload(b):
        with torch.cuda.stream(up):
            if inputs_free[b] is not None:
                up.wait_event(inputs_free[b])
            for group in (("Ai", "BiT"), ("Af", "BfT"), ("W",)):
                for k in group:
                    d[b][k].copy_(h[k], non_blocking=True)
                ready[b][group[0]] = torch.cuda.Event()
                ready[b][group[0]].record(up)

    def run(b, next_b):
        if results_read[b] is not None:
            comp.wait_event(results_read[b])
        db, rb = d[b], dres[b]
        jobs = (("i32_min", "Ai", lambda o: btas.gemm(db["Ai"], db["BiT"], btas.MINPLUS, out=o, trans_b=True)),
                ("i32_max", "Ai", lambda o: btas.gemm(db["Ai"], db["BiT"], btas.MAXPLUS, out=o, trans_b=True)),
                ("f32_min", "Af", lambda o: btas.gemm(db["Af"], db["BfT"], btas.MINPLUS, out=o, trans_b=True)),
                ("f32_max", "Af", lambda o: btas.gemm(db["Af"], db["BfT"], btas.MAXPLUS, out=o, trans_b=True)),
                ("apsp", "W", lambda o: btas.apsp(db["W"], out=o)))
        for name, dep, fn in jobs:
            if name == "apsp" and next_b is not None:
                upload(next_b)  # before the APSP call, which waits on the host between squarings
            comp.wait_event(ready[b][dep])
            fn(rb[name])
            done = torch.cuda.Event()
            done.record(comp)
            down.wait_event(done)
            with torch.cuda.stream(down):
                outs[name].copy_(rb[name], non_blocking=True)
        inputs_free[b] = torch.cuda.Event()
        inputs_free[b].record(comp)
        results_read[b] = torch.cuda.Event()
        results_read[b].record(down)

    def steps_run(k):
        upload(0)
        for i in range(k):
            run(i % 2, (i + 1) % 2 if i + 1 < k else None)
        torch.cuda.synchronize()

    steps_run(1)
    steps = max(1, args.steps)  # the same step count as the device-timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps_run(steps)
    dt = time.perf_counter() - t0
    return {"value": round(units_per_step * steps / dt / 1e9, 2), "unit": "Gop/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "steps": steps, "timing": "host wall clock around all steps, "
            "from the first upload to the last read-back",
            "overlap": "H2D and D2H on their own streams, overlapping the compute; the next step's inputs "
                       "upload during the current step (double-buffered device buffers)"}


PAPER_TABLE2_MS = {4: (0.008, 0.001062), 16: (0.078, 0.001163999), 32: (0.543, 0.002068), 64: (4.034, 0.0011743),
                   128: (31.066, 0.004833)}  # Table II: (1-thread CPU FW, Fermi GPU FW), context only


def config_timings(args, btas, torch):
    """The smaller configurations as timings: one APSP solve at n = 256
    (p = 0.1, w in [1, 100]); the n = 4096 graph with w in [1, 7] on the
    packed kernel vs the int32 kernel (same bits); mid sizes n = 192 ... 4096
    (p = 0.05) on the cooperative kernel (the default there), the same with
    its edge-list shortcuts off, and the tiled path; and the Floyd-Warshall
    sizes of the paper's Table II (4 ... 128 vertices), blocked FW and
    squaring, with the paper's own numbers beside them as context."""
    import gen
    s = gen.BASE_SEED

    def lat(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return round(statistics.median(ts), 1)

    out = {}
    W1h = gen.random_graph(s, 1, 256, 0.1, 1, 100)
    W1 = torch.from_numpy(W1h).cuda()
    D1 = torch.empty_like(W1)
    c1 = {"us_per_solve_adaptive": lat(lambda: btas.apsp(W1, out=D1)),
          "us_per_solve_int32_device_exit": lat(
              lambda: btas.apsp(W1, out=D1, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32)),
          "us_per_solve_noalloc": lat(lambda: btas.btas_apsp_noalloc(256, W1.data_ptr(), D1.data_ptr(),
                                                                     torch.cuda.current_stream().cuda_stream))}
    out["n256_p0.1_w1-100"] = c1
    W3 = torch.from_numpy(gen.random_graph(s, 3, 4096, 0.05, 1, 7)).cuda()
    D3a, D3b = torch.empty_like(W3), torch.empty_like(W3)
    t_u16 = lat(lambda: btas.apsp(W3, out=D3a, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_U16), reps=3)
    t_i32 = lat(lambda: btas.apsp(W3, out=D3b, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32), reps=3)
    out["n4096_p0.05_w1-7"] = {"packed_u16x2_ms": round(t_u16 / 1e3, 3), "int32_ms": round(t_i32 / 1e3, 3),
                               "speedup": round(t_i32 / t_u16, 3), "identical": bool(torch.equal(D3a, D3b))}
    mid = []
    for n in (192, 256, 512, 1024, 1536, 2048, 3072, 4096):
        W = torch.from_numpy(gen.random_graph(s, 300 + n, n, 0.05, 1, 100)).cuda()
        D = torch.empty_like(W)
        row = {"n": n, "cooperative_us": lat(lambda: btas.apsp(W, out=D), reps=5)}
        if n >= 512:  # the edge lists' shortcuts off: first squaring dense, confirming squaring computed
            os.environ.update(BTAS_MID_NO_SPARSE="1", BTAS_MID_NO_CERT="1", BTAS_APSP_MID_MAX_N="4096")
            try:
                row["cooperative_no_shortcuts_us"] = lat(lambda: btas.apsp(W, out=D), reps=5)
            finally:
                for k in ("BTAS_MID_NO_SPARSE", "BTAS_MID_NO_CERT", "BTAS_APSP_MID_MAX_N"):
                    del os.environ[k]
        os.environ["BTAS_APSP_NO_MID"] = "1"
        try:
            row["tiled_adaptive_us"] = lat(lambda: btas.apsp(W, out=D), reps=5)
            if n <= 1024:
                row["tiled_int32_device_exit_us"] = lat(
                    lambda: btas.apsp(W, out=D, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32), reps=5)
        finally:
            del os.environ["BTAS_APSP_NO_MID"]
        mid.append(row)
    out["mid_sizes_p0.05_w1-100"] = mid
    t2 = []
    for n, (cpu_ms, gpu_ms) in PAPER_TABLE2_MS.items():
        W = torch.from_numpy(gen.random_graph(s, 200 + n, n, 0.5, 1, 100)).cuda()
        D = torch.empty_like(W)
        t2.append({"n": n, "blocked_fw_us": lat(lambda: btas.apsp_fw(W, out=D)),
                   "squaring_us": lat(lambda: btas.apsp(W, out=D)),
                   "paper_cpu_fw_us": round(cpu_ms * 1e3, 3), "paper_gpu_fw_us": round(gpu_ms * 1e3, 3)})
    out["paper_table2_sizes"] = t2
    return out


def next_rows(args, btas, torch):
    """The follow-on routines at the n = 8192 graph: tropical gemv (HBM
    roofline), Bellman-Ford SSSP by repeated vector-matrix products, blocked
    Floyd-Warshall vs squaring, APSP with next-hop matrix, FP32 closure."""
    import gen
    n = args.n
    s = gen.BASE_SEED
    W = torch.from_numpy(gen.random_graph(s, 2, n, 0.01, 1, 1000)).cuda()
    A = torch.from_numpy(gen.uniform_int(s, 21, (n, n), 0, 10 ** 6)).cuda()
    x = torch.from_numpy(gen.uniform_int(s, 27, (n,), 0, 10 ** 6)).cuda()
    hbm = peaks().get("hbm_gbs") or 6800.0

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return best
    out = {"n": n, "hbm_peak_gbs_measured": hbm}
    y = torch.empty(n, dtype=torch.int32, device="cuda")

    def back_to_back(fn, calls=20):
        # one event pair around `calls` launches: the per-call launch latency
        # overlaps the previous call's kernel, as in a loop of products
        def run():
            for _ in range(calls):
                fn()
        return timed(run, reps=3) / calls

    for trans in (False, True):
        t = back_to_back(lambda: btas.gemv(A, x, 0, trans=trans, out=y))
        gbs = (n * n * 4 + 2 * n * 4) / t / 1e9
        out[f"gemv_{'trans' if trans else 'rows'}"] = {"ms": round(t * 1e3, 4), "GB_s": round(gbs, 1),
                                                        "frac_of_hbm": round(gbs / hbm, 3)}
    d, info = btas.sssp(W, 0, info=True)
    t = timed(lambda: btas.sssp(W, 0))
    out["sssp"] = {"ms": round(t * 1e3, 3), "products": info["iterations"] + 1,
                   "GB_s_per_product": round((info["iterations"] + 1) * n * n * 4 / t / 1e9, 1)}
    t_fw = timed(lambda: btas.apsp_fw(W), reps=2)
    t_sq = timed(lambda: btas.apsp(W), reps=2)
    t_i32 = timed(lambda: btas.apsp(W, flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32), reps=2)
    out["apsp_blocked_fw"] = {"ms": round(t_fw * 1e3, 3), "terms_tops": round(float(n) ** 3 / t_fw / 1e12, 2)}
    out["apsp_squaring_auto_ms"] = round(t_sq * 1e3, 3)
    out["apsp_squaring_int32_ms"] = round(t_i32 * 1e3, 3)
    np_ = min(n, 4096)
    Wp = W[:np_, :np_].contiguous()
    t_p = timed(lambda: btas.apsp_paths(Wp), reps=1)
    sq_p = btas.apsp_paths(Wp, info=True)[2]["squarings"]
    terms_p = min(btas.btas_apsp_squarings(np_), sq_p + 1) * float(np_) ** 3
    out["apsp_paths"] = {"n": np_, "ms": round(t_p * 1e3, 3), "squarings_computed": int(terms_p / float(np_) ** 3),
                         "terms_tops": round(terms_p / t_p / 1e12, 2)}
    # the same solve on the argmin kernel (group records, no keys), and on
    # binary32 weights (the same integer weights, so the same distances)
    os.environ["BTAS_PATHS_NO_KEYED"] = "1"
    try:
        t_pa = timed(lambda: btas.apsp_paths(Wp), reps=1)
        sq_pa = btas.apsp_paths(Wp, info=True)[2]["squarings"]
    finally:
        os.environ.pop("BTAS_PATHS_NO_KEYED", None)
    terms_pa = min(btas.btas_apsp_squarings(np_), sq_pa + 1) * float(np_) ** 3
    out["apsp_paths_argmin_int32"] = {"n": np_, "ms": round(t_pa * 1e3, 3),
                                      "squarings_computed": int(terms_pa / float(np_) ** 3),
                                      "terms_tops": round(terms_pa / t_pa / 1e12, 2)}
    Wf = torch.where(W[:np_, :np_] == btas.INF_I32, torch.tensor(float("inf"), device="cuda"),
                     W[:np_, :np_].float()).contiguous()
    t_pf = timed(lambda: btas.apsp_paths(Wf), reps=1)
    sq_pf = btas.apsp_paths(Wf, info=True)[2]["squarings"]
    terms_pf = min(btas.btas_apsp_squarings(np_), sq_pf + 1) * float(np_) ** 3
    out["apsp_paths_fp32"] = {"n": np_, "ms": round(t_pf * 1e3, 3),
                              "squarings_computed": int(terms_pf / float(np_) ** 3),
                              "terms_tops": round(terms_pf / t_pf / 1e12, 2)}
    t_c = timed(lambda: btas.closure(Wf, "min"), reps=1)
    sq_c = btas.closure(Wf, "min", info=True)[1]["squarings"]
    terms_c = min(btas.btas_apsp_squarings(np_) + 1, sq_c + 1) * float(np_) ** 3
    out["closure_fp32_minplus"] = {"n": np_, "ms": round(t_c * 1e3, 3), "squarings_computed": int(terms_c / float(np_) ** 3),
                                   "terms_tops": round(terms_c / t_c / 1e12, 2)}
    # exact packed int32 products (BTAS_GEMM_PACKED): small-range operands
    # (values in [-4000, 4000]) on the packed kernel vs the int32 kernel
    del Wp, Wf
    Ap = torch.from_numpy(gen.uniform_int(s, 28, (n, n), -4000, 4000)).cuda()
    Bp = torch.from_numpy(gen.uniform_int(s, 29, (n, n), -4000, 4000)).cuda()
    Cp = torch.empty_like(Ap)
    Cq = torch.empty_like(Ap)
    for sr, name in ((0, "min"), (1, "max")):
        c0 = btas.btas_packed_products()
        t_pk = timed(lambda: btas.gemm(Ap, Bp, sr, out=Cp, packed=True), reps=2)
        took = btas.btas_packed_products() - c0
        t_32 = timed(lambda: btas.gemm(Ap, Bp, sr, out=Cq), reps=2)
        out[f"gemm_i32_packed_{name}"] = {
            "ms": round(t_pk * 1e3, 3), "tops": round(float(n) ** 3 / t_pk / 1e12, 2),
            "int32_kernel_ms": round(t_32 * 1e3, 3), "speedup": round(t_32 / t_pk, 3),
            "packed_path_taken": took == 3, "identical": bool(torch.equal(Cp, Cq))}
    return out


def run_only(args):
    """One part alone, for profiling: `kernels` runs one product of each
    kernel family at size --n (B supplied transposed; the packed 16-bit
    product on values < 2^14); `batched` / `serve` run those workloads."""
    import torch
    import paper_1701_04733_gb300 as btas
    torch.cuda.set_device(dist_env()[2])
    if args.only == "kernels":
        import gen
        n = args.n
        s = gen.BASE_SEED
        Ai = torch.from_numpy(gen.uniform_int(s, 21, (n, n), 0, 10 ** 6)).cuda()
        BiT = torch.from_numpy(gen.uniform_int(s, 22, (n, n), 0, 10 ** 6)).cuda()
        Af = torch.from_numpy(gen.uniform_f32(s, 23, (n, n))).cuda()
        BfT = torch.from_numpy(gen.uniform_f32(s, 24, (n, n))).cuda()
        A16 = torch.from_numpy(gen.uniform_int(s, 25, (n, n), 0, 1 << 14).astype("int16")).cuda()
        B16 = torch.from_numpy(gen.uniform_int(s, 26, (n, n), 0, 1 << 14).astype("int16")).cuda()
        Ci, Cf, C16 = torch.empty_like(Ai), torch.empty_like(Af), torch.empty_like(A16)
        t = {}
        for name, fn in (("i32_min", lambda: btas.gemm(Ai, BiT, 0, out=Ci, trans_b=True)),
                         ("i32_max", lambda: btas.gemm(Ai, BiT, 1, out=Ci, trans_b=True)),
                         ("f32_min", lambda: btas.gemm(Af, BfT, 0, out=Cf, trans_b=True)),
                         ("f32_max", lambda: btas.gemm(Af, BfT, 1, out=Cf, trans_b=True)),
                         ("u16_min", lambda: btas.gemm(A16, B16, 0, out=C16))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t[name] = round(e0.elapsed_time(e1), 3)
        print(json.dumps({"only": "kernels", "n": n, "ms": t}))
    elif args.only == "batched":
        print(json.dumps({"only": "batched", **batched(args, btas, torch)}))
    elif args.only == "tune":
        n = args.n
        combos = [(sr, dt, n, n, n) for dt in (btas.I32, btas.F32) for sr in (0, 1)] + [(0, btas.U16, n, n, n)]
        choices, secs = autotune(btas, combos)
        print(json.dumps({"only": "tune", "n": n, "tuning_s": secs, "choices": choices}))
    elif args.only == "next":
        print(json.dumps({"only": "next", **next_rows(args, btas, torch)}))
    elif args.only == "probe":
        if args.probe_mix is not None:
            r = btas.measure_issue_rate(args.probe_mix, args.probe_ctas)
            print(json.dumps({"only": "probe", "mix": args.probe_mix, "ctas_per_sm": args.probe_ctas,
                              "terms_per_clk_per_sm": round(r, 1)}))
        else:
            print(json.dumps({"only": "probe", "terms_per_clk_per_sm": issue_probe(btas, full=True)}))
    elif args.only == "configs":
        print(json.dumps({"only": "configs", **config_timings(args, btas, torch)}))
    elif args.only == "mid":
        # one mid-size solve (p = 0.05, w in [1, 100], or [1, --mid-whi]) at --n, five calls
        import gen
        n = args.n
        W = torch.from_numpy(gen.random_graph(gen.BASE_SEED, 300 + n, n, 0.05, 1, args.mid_whi)).cuda()
        D = torch.empty_like(W)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = btas.apsp(W, out=D, info=True)
            e1.record()
            torch.cuda.synchronize()
            ts.append(round(e0.elapsed_time(e1) * 1e3, 1))
        print(json.dumps({"only": "mid", "n": n, "us_per_call": ts, "squarings_changing": info["squarings"],
                          "path": info["path"]}))
    elif args.only == "fw":
        # blocked Floyd-Warshall at --n (p = 0.01, w in [1, 1000]): one warm-up
        # solve and three timed ones
        import gen
        n = args.n
        if args.fw_int32:
            os.environ["BTAS_FW_NO_U16"] = "1"
        W = torch.from_numpy(gen.random_graph(gen.BASE_SEED, 7, n, 0.01, 1, 1000)).cuda()
        D = btas.apsp_fw(W)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            btas.apsp_fw(W, out=D)
            e1.record()
            torch.cuda.synchronize()
            ts.append(round(e0.elapsed_time(e1), 3))
        print(json.dumps({"only": "fw", "n": n, "int32_phase3": bool(args.fw_int32), "ms": ts,
                          "terms_tops": round(float(n) ** 3 / min(ts) / 1e9, 2)}))
    elif args.only == "paths":
        # one next-hop solve at --n on the argmin kernel (no keyed squarings):
        # p = 0.01, int32 weights in [1, 1000] or binary32 U[0, 1) on the same edges
        import gen
        import numpy as np
        n = args.n
        Wi = gen.random_graph(1, 3, n, 0.01, 1, 1000)
        if args.paths_dtype == "f32":
            W = np.where(Wi == btas.INF_I32, np.float32(np.inf), gen.uniform_f32(2, 5, (n, n))).astype(np.float32)
            np.fill_diagonal(W, 0)
        else:
            W = Wi
        Wd = torch.from_numpy(W).cuda()
        os.environ["BTAS_PATHS_NO_KEYED"] = "1"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, info = btas.apsp_paths(Wd, info=True)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"only": "paths", "n": n, "dtype": args.paths_dtype, "ms": round(e0.elapsed_time(e1), 3),
                          "squarings_changing": info["squarings"]}))
    else:
        print(json.dumps({"only": "serve", **serve(args, btas, torch)}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_btas(args)


if __name__ == "__main__":
    sys.exit(main())
