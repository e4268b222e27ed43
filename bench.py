#!/usr/bin/env python
"""Benchmark of the GB300 FP64 hybrid symplectic step (GENGA, arXiv:1404.2324).

Workload: the 2048-planetesimal disk (0.5-4 AU, total mass 2 Earth masses, seed 2), 4th-order
(Yoshida) hybrid scheme with close encounters integrated by Bulirsch-Stoer and perfect merging,
dt = 6 days. One "step" is one full 4th-order hybrid step of all 2048 bodies through the C ABI
(genga_step -> one replay of the captured step graph).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints ONE JSON line. value: steps/s with the state resident in HBM, timed with CUDA events per
step on the launching stream, L2 flushed (256 MiB write) before every timed step and the stream
then held ~100 us by a fixed device spin, so that the start event and the step are already queued
when the device reaches them (host submission latency stays out of value, in e2e). e2e: the same
metric through the public API with host buffers: each step uploads the state from pinned host
memory (genga_set_state), steps, and reads it back (genga_get_state). roofline: the pairwise
kick kernel (dominant), FP64-ALU bound, against the derived FP64 peak and against the FP64
throughput measured in the same run (genga_fp64_probe); step_fp64: the kick flops over the whole
step's time. cpu_baseline: the CPU oracle on a bounded sample, single-threaded and built with
OpenMP on all host cores. Further legs: the batched many-systems mode, the test-particle mode,
the differentiable engine (adjoint/forward), config 1 (32 bodies, 2nd order) and the n1/n2 sweep
of Sect. 5 (energy error and time).
With --gpus N > 1 (torchrun) every rank runs an independent replica (the method does not shard
at this N); value counts the steps of all ranks over the slowest rank's time, and only the main
line runs (the batched, test-particle and adjoint legs are single-GPU measurements).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=2048 hybrid steps/s & FP64-peak fraction; batched sys-steps/s; adjoint/fwd"
UNIT = "steps/s"
N_BODIES = 2048
ORDER = 4
SEED = 2
FMA_LANES_PER_SM_CLK = 2  # FP64 FMA lanes per SM per clock on GB300 (measured: 1.9-2.0 at load clocks)
FLOPS_PER_PAIR = 20       # algorithmic flops per ordered pair of the kick (sqrt and division count 1)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "kick_disk2048_ncu.md")
KICK_SOURCES = [os.path.join(ROOT, "paper_1404_2324_gb300", "csrc", f) for f in ("kick.cu", "genga_dev.cuh")]


def workload_config():
    return {"workload": "disk2048: N=2048 planetesimals, 4th-order hybrid step, BS + merging, dt=6 d",
            "n_bodies": N_BODIES, "order": ORDER, "dt_days": 6.0, "seed": SEED,
            "l2": "flushed before every timed step (256 MiB write), then a ~100 us device-side hold so that the step is queued before its start event",
            "inputs": "synthetic disk, a U[0.5,4] AU, e~Rayleigh(0.01), i~Rayleigh(0.005), 2 Earth masses"}


def make_input():
    from paper_1404_2324_gb300 import ics
    d = ics.disk2048(SEED, n=N_BODIES, order=ORDER)
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    x = np.vstack([np.zeros(3), d["x"]])
    v = np.vstack([np.zeros(3), d["v"]])
    return d, m, R, x, v


HOLD_CYCLES = 200_000  # ~100 us at the SM clock


def flush_l2(flush):
    """Evicts L2 (a 256 MiB write), then holds the current stream ~100 us with a fixed-length device
    spin, so that the host has enqueued the start event and the timed work behind it before the
    device reaches them: the timed region then holds the device's work alone, not the host's
    submission latency (the end-to-end figure keeps that)."""
    import torch
    flush.zero_()
    torch.cuda._sleep(HOLD_CYCLES)


def kick_source_hash():
    h = hashlib.sha256()
    for p in KICK_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per kick launch from the committed ncu summary, if it was taken on these sources."""
    try:
        with open(PROFILE_SUMMARY) as f:
            txt = f.read()
    except OSError:
        return None
    mh = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    mt = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mt or mh.group(1) != kick_source_hash():
        return None
    return float(mt.group(1))


# ------------------------------------------------------------------------------------ oracle arm
def run_oracle(steps, warmup, omp=False):
    import oracle as O
    d, *_ = make_input()
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=ORDER)
    sim = O.Sim(p, d["m"], d["R"], d["x"], d["v"], omp=omp)
    sim.step(warmup)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    sim.close()
    return steps / dt, dt


def cpu_baseline_entry(steps, warmup, omp=False):
    rate, secs = run_oracle(steps, warmup)
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{steps} full steps of the same N=2048 4th-order disk after {warmup} warm-up steps, "
                     f"single-threaded C oracle ({secs:.1f} s)"}
    if omp:
        import oracle as O
        if O.lib_omp() is not None:
            r2, s2 = run_oracle(steps, warmup, omp=True)
            out["all_cores"] = {"value": r2, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"the same {steps} steps, the oracle built with OpenMP (its pair sums split "
                                          f"over bodies, results bit-identical), {os.cpu_count()} threads ({s2:.1f} s)"}
        else:
            out["all_cores"] = {"unavailable": "gcc without OpenMP on this host"}
    return out


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [s.strip() for s in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------ batched mode
BATCH_SYSTEMS = 8192
BATCH_SEED = 4


def run_batched(args):
    """Many-systems mode: 8192 systems of 4..64 bodies (incl. the star), 2nd order, graph launches of
    100 steps; compared with one system per launch (a main-mode context per system) on a sample."""
    import torch
    from paper_1404_2324_gb300 import genga, ics
    b = ics.batch(BATCH_SEED, n_sys=BATCH_SYSTEMS)
    n = int(b["offsets"][-1])
    spl = 100
    h = genga.genga_init_batch(b["offsets"], b["m0"], b["m"], b["R"], b["x"], b["v"], b["G"], b["dt"], 2, spl)
    stream = torch.cuda.Stream()  # a real stream: the legacy default stream would not order the graph
    torch.cuda.set_stream(stream)
    genga.genga_set_stream(h, stream)
    split, block, _ = genga.genga_batch_info(h)
    kps = genga.genga_launch_count(h)
    genga.genga_step(h, spl)  # warm-up launch
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = max(1, args.batch_launches)
    tot = 0.0
    for _ in range(launches):
        flush_l2(flush)
        ev0.record(stream)
        genga.genga_step(h, spl)
        ev1.record(stream)
        ev1.synchronize()
        tot += ev0.elapsed_time(ev1)
    code, cnt = genga.genga_status(h)
    sched = genga.genga_batch_schedule(h)
    # the other schedule on the same systems (continuing from the state reached), for comparison
    other = 1 - sched["persistent"]
    try:
        genga.genga_batch_set_schedule(h, other)
        genga.genga_step(h, spl)
        tot_o = 0.0
        for _ in range(launches):
            flush_l2(flush)
            ev0.record(stream)
            genga.genga_step(h, spl)
            ev1.record(stream)
            ev1.synchronize()
            tot_o += ev0.elapsed_time(ev1)
        other_value = BATCH_SYSTEMS * spl * launches / (tot_o * 1e-3)
    except RuntimeError:
        other_value = None
    genga.genga_free(h)
    value = BATCH_SYSTEMS * spl * launches / (tot * 1e-3)
    # one system per launch: a main-mode context per system, one step graph per system per step
    nsamp, ksteps = 64, 20
    ctxs = []
    for s in range(nsamp):
        o0, o1 = b["offsets"][s], b["offsets"][s + 1]
        m = np.concatenate([[b["m0"][s]], b["m"][o0:o1]])
        R = np.concatenate([[0.0], b["R"][o0:o1]])
        x = np.vstack([np.zeros(3), b["x"][o0:o1]])
        v = np.vstack([np.zeros(3), b["v"][o0:o1]])
        c = genga.genga_init(m, R, x, v, b["G"], b["dt"], 2)
        genga.genga_set_stream(c, stream)
        genga.genga_step(c, 1)
        ctxs.append(c)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(ksteps):
        for c in ctxs:
            genga.genga_step(c, 1)
    ev1.record(stream)
    ev1.synchronize()
    t_one = ev0.elapsed_time(ev1)
    for c in ctxs:
        genga.genga_free(c)
    one_value = nsamp * ksteps / (t_one * 1e-3)
    return {"metric": "batched system-steps/s", "value": value, "unit": "system-steps/s",
            "n_systems": BATCH_SYSTEMS, "bodies": n, "steps": spl * launches, "steps_per_launch": spl,
            "ms_per_launch": tot / launches, "gpu_launches": kps * launches,
            "autotuned": {"threads_per_body": split, "block": block,
                          "schedule": "persistent launch" if sched["persistent"] else "step graph",
                          "persistent_ctas": sched["ctas"], "trial_ms_per_step_graph": sched["ms_graph"],
                          "trial_ms_per_step_persistent": sched["ms_persistent"]},
            "other_schedule": {"schedule": "persistent launch" if other else "step graph", "value": other_value,
                               "unit": "system-steps/s",
                               "note": "the same systems continued on the schedule the autotuner did not pick"},
            "one_system_per_launch": {"value": one_value, "unit": "system-steps/s",
                                      "sample": f"{nsamp} systems x {ksteps} steps, one step graph per system"},
            "speedup_vs_one_per_launch": value / one_value, "status": code, "counters": cnt,
            "config": f"batch recipe seed {BATCH_SEED}: N_s ~ U{{4..64}} incl. star, m log-U[1e-7,1e-4], "
                      f"a U[0.1,5], e~Rayleigh(0.02), i~Rayleigh(0.01), 2nd order, dt 6 d; L2 flushed per launch; "
                      f"the library runs batches of 1024+ systems in parts of ~256 systems side by side"}


def batched_cpu_baseline(nsys=512, steps=100):
    import oracle as O
    from paper_1404_2324_gb300 import ics
    b = ics.batch(BATCH_SEED, n_sys=BATCH_SYSTEMS)
    off = b["offsets"]
    t0 = time.perf_counter()
    for s in range(nsys):
        sl = slice(off[s], off[s + 1])
        p = O.params(G=b["G"], m0=b["m0"][s], dt=b["dt"], order=2)
        sim = O.Sim(p, b["m"][sl], b["R"][sl], b["x"][sl], b["v"][sl])
        sim.step(steps)
        sim.close()
    dt = time.perf_counter() - t0
    return {"value": nsys * steps / dt, "unit": "system-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nsys} systems of the batch x {steps} steps ({dt:.1f} s)"}


# ------------------------------------------------------------------------------------ test-particle mode
TP_COUNT = 1 << 20
TP_SEED = 3
TP_STEPS = 200
TP_BYTES_PER_TP_STEP = 96  # algorithmic HBM traffic: read x, v (48 B) and write x, v (48 B) per particle
TP_PROFILE = os.path.join(ROOT, "profiles", "tp_pass_ncu.md")
TP_SOURCES = [os.path.join(ROOT, "paper_1404_2324_gb300", "csrc", f) for f in ("tp.cu", "genga_dev.cuh")]


def tp_profile_counts():
    """Per particle-step FP64 flops (thread level: DFMA = 2, DADD/DMUL = 1), FP64 warp instructions
    and DRAM bytes of the particle kernels, from the committed ncu summary, if it was taken from
    the current sources (else None)."""
    try:
        txt = open(TP_PROFILE).read()
    except OSError:
        return None
    h = hashlib.sha256()
    for f in TP_SOURCES:
        h.update(open(f, "rb").read())
    vals = {}
    for key in ("source_sha256", "fp64_flop_per_tp_step", "fp64_warp_inst_per_tp_step", "dram_bytes_per_tp_step"):
        m = re.search(key + r":\s*([0-9a-fA-F.eE+-]+)", txt)
        if not m:
            return None
        vals[key] = m.group(1)
    if vals.pop("source_sha256") != h.hexdigest():
        return None
    return {k: float(v) for k, v in vals.items()}


def run_tp(args, peaks):
    """Test-particle mode: 8 planets + 2^20 massless particles, 2nd order, dt 6 d. One step = one
    replay of the step graph (planets and particles). Each timed step follows an L2 flush."""
    import torch
    from paper_1404_2324_gb300 import genga, ics
    n_tp = max(1, getattr(args, "tp_count", TP_COUNT))
    d = ics.tp_disk(TP_SEED, n_tp=n_tp)
    m = np.concatenate([[d["m0"]], d["m"]])
    R = np.concatenate([[0.0], d["R"]])
    x = np.vstack([np.zeros(3), d["x"]])
    v = np.vstack([np.zeros(3), d["v"]])
    h = genga.genga_init_tp(m, R, x, v, d["G"], d["dt"], 2, d["x_tp"], d["v_tp"], d["R_tp"])
    stream = torch.cuda.Stream()  # a real stream: the legacy default stream would not order the graph
    torch.cuda.set_stream(stream)
    genga.genga_set_stream(h, stream)
    genga.genga_step(h, max(3, min(args.warmup, 20)))
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, args.tp_steps)
    tot = 0.0
    for _ in range(steps):
        flush_l2(flush)
        ev0.record(stream)
        genga.genga_step(h, 1)
        ev1.record(stream)
        ev1.synchronize()
        tot += ev0.elapsed_time(ev1)
    kps = genga.genga_launch_count(h)
    st = genga.genga_tp_status(h)
    code, _ = genga.genga_status(h)
    genga.genga_free(h)
    sec = tot * 1e-3 / steps
    rate = n_tp / sec
    gbs = TP_BYTES_PER_TP_STEP * rate / 1e9
    out = {"metric": "test-particle steps/s", "value": rate, "unit": "TP-steps/s", "n_tp": n_tp,
           "n_planets": len(d["m"]), "steps": steps, "ms_per_step": tot / steps, "gpu_launches": kps * steps,
           "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                   "bytes_per_tp_step": TP_BYTES_PER_TP_STEP, "peak_source": peaks["hbm_source"]},
           "status": code, "counters": st,
           "config": f"tp_disk seed {TP_SEED}: 8 planets m log-U[1e-7,1e-3], a 0.4-30 AU; 2^20 particles "
                     f"a U[0.3,5], e U[0,0.3], i U[0,0.2]; 2nd order, dt 6 d; L2 flushed per step"}
    if n_tp != TP_COUNT:
        out["config"] = out["config"].replace("2^20 particles", f"{n_tp} particles")
    prof = tp_profile_counts()
    if prof is not None:
        fl = prof["fp64_flop_per_tp_step"] * rate / 1e12
        # a warp FP64 instruction holds its sub-partition 64 cycles whatever its active lanes
        import torch
        props = torch.cuda.get_device_properties(0)
        warp_slots = props.multi_processor_count * 4 * peaks["sm_max_mhz"] * 1e6 / 64.0
        out["fp64"] = {"achieved": fl, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s", "frac": fl / peaks["fp64_tflops"],
                       "pipe_busy_frac": prof["fp64_warp_inst_per_tp_step"] * rate / warp_slots,
                       "dram_bytes_per_tp_step": prof["dram_bytes_per_tp_step"],
                       "source": "per particle-step counts from profiles/tp_pass_ncu.md (ncu, 2^18 particles)"}
    return out


def tp_cpu_baseline(n_tp=1 << 20, steps=6):
    import oracle as O
    from paper_1404_2324_gb300 import ics
    d = ics.tp_disk(TP_SEED, n_tp=n_tp)
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2)
    sim = O.TPSim(p, d["m"], d["R"], d["x"], d["v"], d["x_tp"], d["v_tp"], d["R_tp"])
    sim.step(1)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    sim.close()
    return {"value": n_tp * steps / dt, "unit": "TP-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"8 planets + {n_tp} particles of the same recipe x {steps} steps after one ({dt:.1f} s)"}


# ------------------------------------------------------------------------------------ adjoint
ADJ_SYSTEMS, ADJ_N, ADJ_STEPS, ADJ_CKPT, ADJ_SEED = 64, 256, 2000, 50, 5


def run_adjoint(args):
    """Differentiable engine: 64 disks of 256 planetesimals (2048-disk shapes), 2nd order, 2000 steps,
    a checkpoint every 50 steps. Forward = 2000 steps; backward = the gradient of a random linear
    functional of the final state with respect to the initial x, v and masses (segment recompute
    from the checkpoints + the VJPs). Reported: backward time / forward time, and the gradient's
    agreement with central differences (h = 1e-7 relative along a random direction) on a bounded
    sample (4 systems, 20 steps: over 2000 steps close passes make finite differences meaningless)."""
    import torch
    from paper_1404_2324_gb300 import ics
    from paper_1404_2324_gb300.adjoint import AdjointEngine
    d = ics.adj_disks(ADJ_SEED, n_sys=ADJ_SYSTEMS, n=ADJ_N)
    steps = max(1, args.adj_steps)

    def T(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    eng = AdjointEngine(d["m0"], d["G"], d["dt"], 2, ckpt_every=ADJ_CKPT)
    X, V, M = T(d["x"]), T(d["v"]), T(d["m"])
    rng = np.random.default_rng(1)
    ux, uv = T(rng.standard_normal(d["x"].shape)), T(rng.standard_normal(d["v"].shape))
    eng.forward(X, V, M, 20)  # warm-up
    eng.backward(ux, uv)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    eng.forward(X, V, M, steps)
    e1.record(stream)
    eng.backward(ux, uv)
    e2.record(stream)
    e2.synchronize()
    f_ms, b_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    status = eng.status()
    eng.close()
    # bounded central-difference check
    S, K = 4, 20
    e4 = AdjointEngine(d["m0"][:S], d["G"], d["dt"], 2, ckpt_every=ADJ_CKPT)
    x4, v4, m4 = d["x"][:S], d["v"][:S], d["m"][:S]
    u4x, u4v = rng.standard_normal(x4.shape), rng.standard_normal(v4.shape) * 50.0
    dx = rng.standard_normal(x4.shape) * np.linalg.norm(x4, axis=-1, keepdims=True)
    dv = rng.standard_normal(v4.shape) * np.linalg.norm(v4, axis=-1, keepdims=True)
    dm = rng.standard_normal(m4.shape) * m4
    e4.forward(T(x4), T(v4), T(m4), K)
    gx, gv, gm = (t.cpu().numpy() for t in e4.backward(T(u4x), T(u4v)))
    pred = (gx * dx).sum() + (gv * dv).sum() + (gm * dm).sum()

    def loss(h):
        xo, vo = e4.forward(T(x4 + h * dx), T(v4 + h * dv), T(m4 + h * dm), K)
        return (xo.cpu().numpy() * u4x).sum() + (vo.cpu().numpy() * u4v).sum()

    fd = (loss(1e-7) - loss(-1e-7)) / 2e-7
    e4.close()
    # the product's forward on the same systems: one main-mode context per disk (merging off, as in
    # the differentiable engine), all on their own streams at once, over a bounded sample of steps
    from paper_1404_2324_gb300 import genga
    ctxs, streams = [], []
    for b in range(ADJ_SYSTEMS):
        m = np.concatenate([[d["m0"][b]], d["m"][b]])
        R = np.zeros(ADJ_N + 1)
        x = np.vstack([np.zeros(3), d["x"][b]]); v = np.vstack([np.zeros(3), d["v"][b]])
        c = genga.genga_init(m, R, x, v, d["G"], d["dt"], 2)
        prm = genga.genga_default_params()
        prm.collisions = 0
        genga.genga_set_params(c, prm)
        st = torch.cuda.Stream()
        genga.genga_set_stream(c, st)
        genga.genga_step(c, 2)
        ctxs.append(c)
        streams.append(st)
    torch.cuda.synchronize()
    psteps = 100
    t0 = time.perf_counter()
    for c in ctxs:
        genga.genga_step(c, psteps)
    torch.cuda.synchronize()
    p_sec = time.perf_counter() - t0
    for c in ctxs:
        genga.genga_free(c)
    prod_ms = p_sec * 1e3 * steps / psteps  # the same work as the timed forward
    return {"metric": "adjoint/fwd", "value": b_ms / f_ms, "unit": "backward time / forward time",
            "higher_is_better": False, "forward_ms": f_ms, "backward_ms": b_ms, "steps": steps,
            "forward_system_steps_per_s": ADJ_SYSTEMS * steps / (f_ms * 1e-3),
            "vs_product_forward": {"value": b_ms / prod_ms, "product_forward_ms": prod_ms,
                                   "product_system_steps_per_s": ADJ_SYSTEMS * psteps / p_sec,
                                   "basis": f"backward time over the time genga_step takes for the same "
                                            f"{ADJ_SYSTEMS} disks x {steps} steps (one main-mode context per disk, "
                                            f"merging off, concurrent streams; timed over {psteps} steps, host clock)"},
            "grad_vs_central_fd": {"rel_err": abs(fd - pred) / abs(pred), "h_rel": 1e-7,
                                   "sample": f"{S} systems x {K} steps, one random direction"},
            "status": status,
            "config": f"adj_disks seed {ADJ_SEED}: {ADJ_SYSTEMS} disks x {ADJ_N} planetesimals (0.5-4 AU, "
                      f"2 Earth masses x {ADJ_N}/2048 each), 2nd order, dt 6 d, checkpoint every {ADJ_CKPT} "
                      f"steps, merging off; state resident in HBM (no L2 flush: each timed region is seconds long)"}


# ------------------------------------------------------------------------------------ config 1 and the n1/n2 sweep
def run_config1(args):
    """The plain 2nd-order step of 32 planetesimals (config 1 of the recipe, Sect. 4.1's energy runs):
    1000 steps timed as one stretch of graph replays (32 bodies: everything stays in L2)."""
    import torch
    from paper_1404_2324_gb300 import genga, ics
    d = ics.disk32(1)
    m = np.concatenate([[d["m0"]], d["m"]]); R = np.concatenate([[0.0], d["R"]])
    x = np.vstack([np.zeros(3), d["x"]]); v = np.vstack([np.zeros(3), d["v"]])
    ctx = genga.genga_init(m, R, x, v, d["G"], d["dt"], 2)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    genga.genga_set_stream(ctx, stream)
    genga.genga_step(ctx, 20)
    torch.cuda.synchronize()
    steps = 1000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    genga.genga_step(ctx, steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    kps = genga.genga_launch_count(ctx)
    genga.genga_free(ctx)
    import oracle as O
    p = O.params(G=d["G"], m0=d["m0"], dt=d["dt"], order=2)
    sim = O.Sim(p, d["m"], d["R"], d["x"], d["v"])
    t0 = time.perf_counter()
    sim.step(steps)
    osec = time.perf_counter() - t0
    sim.close()
    return {"metric": "config-1 steps/s", "value": steps / (ms * 1e-3), "unit": "steps/s", "steps": steps,
            "ms_per_step": ms / steps, "gpu_launches": kps * steps,
            "cpu_baseline": {"value": steps / osec, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"the same {steps} steps, single-threaded C oracle ({osec:.2f} s)"},
            "config": "disk32 seed 1: 32 planetesimals, m log-U[1e-8,1e-6], a U[0.5,1.5] AU, 2nd order, dt 6 d; "
                      "no L2 flush (the 32-body state is a few KB)"}


def run_sweep(args):
    """The paper's Sect. 5 experiment: cumulative energy error and execution time against the
    critical-radius parameters, n2 with n1 = 3 and n1 with n2 = 0, on a 32-body disk (2000 steps,
    2nd order); and the 2048-body disk at 4th order for growing n2, where the encounter groups merge
    into one large group (Sect. 5)."""
    import torch
    from paper_1404_2324_gb300 import genga, ics
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(d, order, n1, n2, steps, chunk):
        m = np.concatenate([[d["m0"]], d["m"]]); R = np.concatenate([[0.0], d["R"]])
        x = np.vstack([np.zeros(3), d["x"]]); v = np.vstack([np.zeros(3), d["v"]])
        ctx = genga.genga_init(m, R, x, v, d["G"], d["dt"], order)
        prm = genga.genga_default_params()
        prm.n1, prm.n2 = n1, n2
        genga.genga_set_params(ctx, prm)
        genga.genga_set_stream(ctx, stream)
        E0, U0 = genga.genga_energy(ctx)
        err, ms = 0.0, 0.0
        for _ in range(steps // chunk):
            e0.record(stream)
            genga.genga_step(ctx, chunk)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            E, U = genga.genga_energy(ctx)
            err = max(err, abs((E + U - E0 - U0) / E0))
        code, cnt = genga.genga_status(ctx)
        genga.genga_free(ctx)
        return {"n1": n1, "n2": n2, "energy_error": err, "ms": ms, "ms_per_step": ms / steps,
                "encounters_per_step": cnt["encounters"] / steps, "bs_steps_per_step": cnt["bs_steps"] / steps,
                "status": code}

    d32 = ics.disk32(1)
    small = [run(d32, 2, 3.0, n2, 2000, 100) for n2 in (0.0, 0.4, 0.7, 1.0, 1.5)]
    small += [run(d32, 2, n1, 0.0, 2000, 100) for n1 in (1.0, 7.0, 15.0, 30.0)]
    d2048 = ics.disk2048(SEED, n=N_BODIES, order=ORDER)
    large = [run(d2048, ORDER, 3.0, n2, 20, 10) for n2 in (0.4, 0.7, 1.0, 1.5)]
    return {"disk32": small, "disk2048": large,
            "config": "disk32 seed 1, 2nd order, dt 6 d, 2000 steps, energy sampled every 100 steps; "
                      f"disk2048 seed {SEED}, 4th order, 20 steps each; n1 = 3 where n2 varies, n2 = 0 where n1 varies"}


# ------------------------------------------------------------------------------------ ranks
def rank_max(x, world, device=None):
    """The largest x over all ranks (the slowest replica sets the job's time); x itself at N = 1."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units, timed by
    the slowest one."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world):
    import torch
    from paper_1404_2324_gb300 import genga

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    genga.lib()
    d, m, R, x, v = make_input()
    ctx = genga.genga_init(m, R, x, v, d["G"], d["dt"], ORDER)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    genga.genga_set_stream(ctx, stream)
    genga.genga_set_profiling(ctx, True)
    kernels_per_step = genga.genga_launch_count(ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    genga.genga_step(ctx, args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms, kick_ms, kick_launches = 0.0, 0.0, 0
    for _ in range(args.steps):
        flush_l2(flush)
        ev0.record(stream)
        genga.genga_step(ctx, 1)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        km, kn = genga.genga_kick_time(ctx)
        kick_ms += km
        kick_launches += kn
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    code, counters = genga.genga_status(ctx)
    t_max = rank_max(total_ms, world, "cuda")
    value = job_rate(args.steps, world, t_max * 1e-3)

    # end to end through the public API with host buffers (pinned)
    genga.genga_set_profiling(ctx, False)
    n = N_BODIES + 1
    hx = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hv = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    st = genga.genga_get_state(ctx, n)
    hx[:] = st["x"]
    hv[:] = st["v"]
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    genga.genga_step(ctx, 1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        genga.genga_set_state(ctx, hx, hv)
        genga.genga_step(ctx, 1)
        genga.lib().genga_get_state(ctx, hx.ctypes.data_as(genga._D), hv.ctypes.data_as(genga._D), None, None, None)
    t_e2e = rank_max(time.perf_counter() - t0, world, "cuda")
    e2e = {"value": job_rate(e2e_steps, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": int(hx.nbytes + hv.nbytes),
           "d2h_bytes_per_step": int(hx.nbytes + hv.nbytes), "steps": e2e_steps,
           "note": "genga_set_state + genga_step + genga_get_state per step; the step after set_state opens with the full pair kick"}
    genga.genga_free(ctx)

    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * FMA_LANES_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
    probe_tflops, probe_ms = genga.genga_fp64_probe(1 << 15)
    kick_avg_s = (kick_ms / max(kick_launches, 1)) * 1e-3
    algo_flops = FLOPS_PER_PAIR * N_BODIES * (N_BODIES - 1)
    achieved = algo_flops / kick_avg_s / 1e12
    traffic = committed_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": "k_kick (pairwise K-weighted kick + precheck)", "kick_avg_us": kick_avg_s * 1e6,
                "kick_launches": kick_launches,
                "peak_basis": f"FP64: {props.multi_processor_count} SMs x {FMA_LANES_PER_SM_CLK} FMA/clk x 2 flop x "
                              f"{sm_max:.0f} MHz (derived)",
                "peak_probe": probe_tflops, "frac_probe": achieved / probe_tflops,
                "peak_probe_basis": f"measured in this run: genga_fp64_probe, 8 independent FMA chains per thread, "
                                    f"4 x 256 threads per SM, {probe_ms:.1f} ms",
                "achieved_basis": f"{FLOPS_PER_PAIR} flop x N(N-1) ordered pairs per launch"}
    kicks_per_step = kick_launches / max(args.steps, 1)
    step_flops = kicks_per_step * algo_flops
    step_tflops = step_flops / (t_max / args.steps * 1e-3) / 1e12
    step_fp64 = {"achieved": step_tflops, "unit": "TFLOP/s", "frac": step_tflops / peak_tflops,
                 "frac_probe": step_tflops / probe_tflops,
                 "basis": f"{kicks_per_step:.0f} pairwise kicks x {FLOPS_PER_PAIR} flop x N(N-1) per step over the "
                          f"whole step's time (drift, encounters, BS and the small kernels included)"}
    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(), "roofline": roofline, "step_fp64": step_fp64, "e2e": e2e,
           "gpu_launches": kernels_per_step * args.steps, "kernels_per_step": kernels_per_step,
           "clocks": clocks, "status": code, "counters": counters}
    return res


def measured_peaks(res):
    """HBM copy bandwidth from the measured-peaks file (fallback 6.8 TB/s) and the derived FP64 peak
    of the main line's roofline."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm, src = float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        hbm, src = 6800.0, "fallback"
    sm = (res.get("clocks") or {}).get("sm_max_mhz") or 2070.0
    return {"hbm_gbs": hbm, "hbm_source": src, "fp64_tflops": res["roofline"]["peak"], "sm_max_mhz": sm}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--cpu-steps", type=int, default=40, help="oracle steps in the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-launches", type=int, default=5, help="timed 100-step launches of the batched mode")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--tp-steps", type=int, default=TP_STEPS, help="timed steps of the test-particle mode")
    ap.add_argument("--tp-count", type=int, default=TP_COUNT, help="particles of the test-particle leg (profiling: smaller)")
    ap.add_argument("--no-tp", action="store_true")
    ap.add_argument("--adj-steps", type=int, default=ADJ_STEPS, help="steps of the differentiable-engine leg")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-config1", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        ref_steps = min(args.steps, args.cpu_steps)
        ref_warm = min(args.warmup, 2)
        cb = cpu_baseline_entry(ref_steps, ref_warm)
        res = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 / cb["value"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": workload_config(), "impl": "reference", "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(res))
        return 0

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    if world == 1:  # the other modes are single-GPU measurements: with replicas only the main line runs
        if not args.no_batched:
            res["batched"] = run_batched(args)
        if not args.no_tp:
            res["test_particles"] = run_tp(args, measured_peaks(res))
        if not args.no_adjoint:
            res["adjoint"] = run_adjoint(args)
        if not args.no_config1:
            res["config1"] = run_config1(args)
        if not args.no_sweep:
            res["sweep"] = run_sweep(args)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            res["cpu_baseline"] = cpu_baseline_entry(args.cpu_steps, 2, omp=True)
            if "batched" in res:
                res["batched"]["cpu_baseline"] = batched_cpu_baseline()
            if "test_particles" in res:
                res["test_particles"]["cpu_baseline"] = tp_cpu_baseline()
        else:
            res["cpu_baseline"] = None
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
