#!/usr/bin/env python
"""Benchmark of the GB300 gate-bootstrapping path.

Metric: bootstrapped gates per second on one GB300 (exact: every output is
the bit-exact result of the plain definition), plus encrypted 16-bit ADD and
MUL latency percentiles.  A step is one evaluation of the 16-bit
parallel-prefix adder (§5 "Adder": 194 bootstrapped gates, 9 levels) on 256
encrypted operand pairs drawn uniformly from [0, 2^16): every level of all
256 additions is one pass of the whole hot path (linear combination +
modulus switch, blind rotation, sample extraction + key switching), i.e.
49,664 bootstraps per step.  MUL latency: the array multiplier on 64 pairs.
Inputs are synthetic and seeded (fresh encryptions under keys generated from
seed 20210103).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`value` uses device-resident inputs (device-side time of K steps, L2 flushed
between steps); `e2e` runs the same steps through the library's host-buffer
call (ce_unit_eval: the step's inputs copied from pinned host memory and its
results copied back inside the call, inside the timed region).  Latency:
one 16-bit ADD and one 16-bit MUL alone (graph replay, CUDA events, 20+
repeats), and a short serving run (16 clients with their own keys,
ADD/SUB/MUL/UDIV 40/30/20/10 at Poisson arrivals) for per-request p50/p99.
`--impl reference` times the plain CPU oracle (test infrastructure, used here
only as the reference arm) on a bounded sample of the same workload.
Under torchrun every rank evaluates its own batch (independent gates, no
data-path collective) and rank 0 prints one JSON line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SEED = 20210103
METRIC = "bootstrapped gates/s on 1 GB300 (exact)"
UNIT = "gates/s"
# Algorithmic work of one bootstrap in 32-bit integer operations of the
# two-prime transform method.  Per CMux step and per prime: 6 forward and 2
# inverse 1024-point transforms (512 * 10 butterflies each) and 12 * 1024
# pointwise multiply-accumulates.  A butterfly is 7 int32 operations (add,
# conditional subtract (2), offset subtract, Shoup product (3)); a
# multiply-accumulate is 2.5 (a 32x32->64 multiply-add per product, then one
# Montgomery reduction (2) and one add per pair of products).
BFLY_PER_CMUX = 2 * 8 * 512 * 10                               # 81,920
MAC_PER_CMUX = 2 * 12 * 1024                                   # 24,576
OPS_PER_GATE = 500 * (7 * BFLY_PER_CMUX + 2.5 * MAC_PER_CMUX)   # 317,440,000
# Integer issue peak from unit counts: SMs x 4 schedulers x 32 lanes x SM
# clock (multiply-adds and other integer operations issue to separate 64-lane
# pipes).  The SM count is read from the device and the clock is the median
# sampled during the timed region.
INT_LANES_PER_SM = 128


def int_peak_tops(sms: int, sm_mhz: float) -> float:
    return sms * INT_LANES_PER_SM * sm_mhz * 1e6 / 1e12


# The unit that binds the blind rotation on GB300 (ncu: the FMA-heavy pipe
# ~80 % busy, the ALU ~47 %, issue ~63 %) is the 16-lane integer multiply-add
# pipe, one per scheduler: a 32-bit multiply-add holds it 2 cycles per warp,
# its high-half and 64-bit forms 4.  The method's multiplies per thread (128
# per gate) and CMux step: 656 Shoup products of the transforms (one high-half
# and two low multiplies: 8 cycles), 32 key positions of six 64-bit products
# plus one Montgomery reduction (6 x 4 + 2 + 4 = 30 cycles) and 16
# reconstructions (a Shoup product and a 64-bit multiply-add: 12 cycles).
MULPIPE_WARP_CYCLES_PER_STEP = 656 * 8 + 32 * 30 + 16 * 12          # 6,400
MULPIPE_CYCLES_PER_GATE = 500 * 4 * MULPIPE_WARP_CYCLES_PER_STEP    # 12.8 M
# The same multiplies counted by kind, per thread and CMux step: 32-bit
# multiply-adds (two per Shoup product, one per Montgomery reduction), high
# halves (one per Shoup product), 64-bit products (key products, Montgomery
# reductions, reconstructions).
MUL_COUNTS_PER_THREAD_STEP = {"imad": 2 * 656 + 32 + 2 * 16, "imad_hi": 656 + 16,
                              "imad_wide": 6 * 32 + 32 + 16}


def mulpipe_peak(sms: int, sm_mhz: float) -> float:
    """Multiply-pipe warp-cycles per second of the GPU (4 pipes per SM)."""
    return sms * 4 * sm_mhz * 1e6


KERNEL_SOURCES = ["bootstrap_kernels.cu", "rns_ntt.cuh", "rns_arith.h"]
N_PAIRS = 256
# External-product forms compared on one gate batch (19 tiles of 128 gates:
# two whole tiles per CTA of the tensor-core kernel's stream-K schedule on 152
# SMs) and on a mid-size batch.
XP_GATES = 2432
XP_MID_GATES = 1216   # 10 gate tiles of 128: the mid-size batch of the tensor form
# Tensor (Toeplitz) form: per CMux step and gate, eight limb products of the
# [2048 x 6144] key block with the 6144 digits, 2 flops per multiply-add.
XP_FLOPS_PER_GATE = 500 * 2 * 2048 * 6144 * 8                  # 1.0066e11


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=256, help="ADD operand pairs per step")
    return ap.parse_args()


# ------------------------------------------------------------ distributed ---
def dist_setup(backend: str):
    """Rank/world from the torchrun environment (single process otherwise)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    return units_per_rank * steps * world / (max_ms / 1e3)


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.samples, self.stop = index, [], threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.th.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.th.join(timeout=10)

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------------ oracle ---
_ORACLE_KEYS = None


def oracle_sample(n_gates: int, threads: int):
    """Time the plain CPU oracle on n_gates gates of the same workload."""
    global _ORACLE_KEYS
    from oracle import oracle as O
    if _ORACLE_KEYS is None:
        _ORACLE_KEYS = O.keygen(O.GATE_PARAMS, SEED)
    keys = _ORACLE_KEYS
    rng = np.random.default_rng(SEED)
    bits = rng.integers(0, 2, (n_gates, 2))
    p = O.GATE_PARAMS
    ca = np.stack([O.encrypt(p, keys.s, int(b), 31, i) for i, b in enumerate(bits[:, 0])])
    cb = np.stack([O.encrypt(p, keys.s, int(b), 32, i) for i, b in enumerate(bits[:, 1])])
    ops = np.tile([1, 3], n_gates // 2 + 1)[:n_gates]
    t0 = time.perf_counter()
    O.gates(keys, ops, ca, cb, threads=threads)
    return n_gates / (time.perf_counter() - t0)


def cpu_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    cores = cpu_cores()
    per_step = cores  # one gate per core per step (~5 s of CPU work per core)
    for _ in range(args.warmup):
        oracle_sample(per_step, cores)
    vals, t_all = [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(oracle_sample(per_step, cores))
        t_all += time.perf_counter() - t0
    value = per_step * args.steps / t_all
    sample = f"{per_step} bootstrapped gates (AND/XOR of the adder's first level) per step, one per core"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_all / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded encryptions of uniform bits)",
            "config": {"workload": f"16-bit Kogge-Stone ADD on {args.pairs} encrypted operand "
                                   "pairs, level-batched (n=500 N=1024 l=3 Bg=2^10 t=8); the "
                                   "oracle times a sample of its gates",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our arm ---
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2101_03403_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, launches_per_step=None):
    """DRAM bytes per launch of the bench workload from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def encrypt_operands(ce, sk, a, b, seed):
    """[n][32][501]: bits of a then bits of b, each a fresh encryption."""
    n = len(a)
    out = np.zeros((n, 32, 501), np.uint32)
    for i in range(n):
        for j in range(16):
            out[i, j] = ce.ce_encrypt_bit(sk, int(a[i] >> j) & 1, seed, 32 * i + j)
            out[i, 16 + j] = ce.ce_encrypt_bit(sk, int(b[i] >> j) & 1, seed, 32 * i + 16 + j)
    return out


def decrypt_word(ce, sk, bits) -> int:
    return sum(ce.ce_decrypt_bit(sk, bits[j]) << j for j in range(16))


def run_ours(args, rank: int, world: int, local: int):
    import torch

    import paper_2101_03403_gb300 as ce
    from paper_2101_03403_gb300 import build as b
    b.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.pairs
    sk = ce.ce_secret_keygen(SEED)
    ck = ce.ce_cloud_keygen(sk, SEED)
    stream = torch.cuda.current_stream(dev)
    ctx = ce.ce_create(local, 0, stream)
    cid = ce.ce_client_admit(ctx, ck)
    tuned = ce.ce_autotune(ctx, cid)              # launch shapes measured on this device
    gates_per_add = ce.ce_unit_info("ADD")["n_bootstraps"]
    boots = n * gates_per_add

    rng = np.random.default_rng(SEED + rank)
    a = rng.integers(0, 1 << 16, n)
    bb = rng.integers(0, 1 << 16, n)
    host_in = encrypt_operands(ce, sk, a, bb, 31 + rank)
    d_in = torch.from_numpy(host_in.view(np.int32)).to(dev)
    d_out = torch.empty((n, 16, 501), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > 129 MB L2

    def step(profiled: bool):
        ce.ce_profile_enable(ctx, profiled)
        ce.ce_unit_eval_device(ctx, cid, "ADD", d_in, d_out, n, 0, stream)

    for _ in range(max(args.warmup, 3)):
        step(True)
    step(False)                                   # captures the graph
    ce.ce_synchronize(ctx)
    ce.ce_profile_read(ctx)

    out = d_out.cpu().numpy().view(np.uint32)     # correctness guard on the measured output
    for i in rng.choice(n, 16, replace=False):
        assert decrypt_word(ce, sk, out[i]) == (int(a[i]) + int(bb[i])) & 0xFFFF, "wrong sum"

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.zero_()                         # outside the per-step events
            starts[k].record(stream)
            step(True)                            # eager, per-kernel events on
            launches += ce.ce_last_launch_count(ctx)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
    ce.ce_synchronize(ctx)
    prof = ce.ce_profile_read(ctx)
    ce.ce_profile_enable(ctx, False)
    step_ms = [st.elapsed_time(en) for st, en in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = weak_scaling_value(boots, args.steps, world, total_ms)

    # the same steps replayed as the captured CUDA graph of the unit
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        step(False)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    graph_value = boots * args.steps / (g0.elapsed_time(g1) / 1e3)

    # end to end through the host-buffer call: pinned host inputs -> device ->
    # unit (captured graph) -> pinned host results, all inside ce_unit_eval
    pin_in = torch.from_numpy(host_in.view(np.int32)).pin_memory()
    pin_out = torch.empty((n, 16, 501), dtype=torch.int32).pin_memory()
    h_in, h_out = pin_in.numpy().view(np.uint32), pin_out.numpy().view(np.uint32)

    def e2e_step():
        ce.ce_unit_eval(ctx, cid, "ADD", h_in, h_out)

    e2e_step()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_val = boots * args.steps * world / e2e_s
    assert (h_out == d_out.cpu().numpy().view(np.uint32)).all(), "e2e output differs"

    # latency of one instruction alone: one operand pair, graph replay
    def alone_ms(unit, reps):
        x = rng.integers(0, 1 << 16, 2)
        d1 = torch.from_numpy(encrypt_operands(ce, sk, x[:1], x[1:], 91).view(np.int32)).to(dev)
        o1 = torch.empty((1, 16, 501), dtype=torch.int32, device=dev)
        ce.ce_unit_eval_device(ctx, cid, unit, d1, o1, 1, 0, stream)    # plan + capture
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ce.ce_unit_eval_device(ctx, cid, unit, d1, o1, 1, 0, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        want = {"ADD": (int(x[0]) + int(x[1])) & 0xFFFF, "MUL": (int(x[0]) * int(x[1])) & 0xFFFF,
                "ADD_MUX": (int(x[0]) + int(x[1])) & 0xFFFF,
                "MUL_TREE": (int(x[0]) * int(x[1])) & 0xFFFF}
        assert decrypt_word(ce, sk, o1.cpu().numpy().view(np.uint32)[0]) == want[unit]
        return ts

    add1_ms = alone_ms("ADD", 30)
    mul1_ms = alone_ms("MUL", 20)
    addmux1_ms = alone_ms("ADD_MUX", 30)   # the same adder, each span's carry one MUX
    multree1_ms = alone_ms("MUL_TREE", 20)  # the low half by column compression

    def batching_leg(pairs):
        """Level batching against one launch per gate (ce_set_level_batching):
        the same 16-bit ADDs eagerly both ways, outputs compared word for
        word."""
        x = rng.integers(0, 1 << 16, (2, pairs))
        d1 = torch.from_numpy(encrypt_operands(ce, sk, x[0], x[1], 93).view(np.int32)).to(dev)
        outs, res = {}, {}
        ce.ce_set_unit_graphs(ctx, False)
        try:
            for mode, reps in (("level_batched", 3), ("one_launch_per_gate", 2)):
                ce.ce_set_level_batching(ctx, mode == "level_batched")
                o1 = torch.empty((pairs, 16, 501), dtype=torch.int32, device=dev)
                ce.ce_unit_eval_device(ctx, cid, "ADD", d1, o1, pairs, 0, stream)  # warm-up
                torch.cuda.synchronize(dev)
                ts = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ce.ce_unit_eval_device(ctx, cid, "ADD", d1, o1, pairs, 0, stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    ts.append(e0.elapsed_time(e1))
                outs[mode] = o1.cpu()
                res[mode] = {"ms": statistics.median(ts), "launches": ce.ce_last_launch_count(ctx)}
        finally:
            ce.ce_set_level_batching(ctx, True)
            ce.ce_set_unit_graphs(ctx, True)
        assert torch.equal(outs["level_batched"], outs["one_launch_per_gate"]), "batching modes differ"
        boots = pairs * gates_per_add
        for v in res.values():
            v["gates_per_s"] = boots / (v["ms"] / 1e3)
        return {"unit": "ADD", "pairs": pairs, "bootstraps": boots, **res,
                "speedup": res["one_launch_per_gate"]["ms"] / res["level_batched"]["ms"],
                "identical_outputs": True}

    batching = batching_leg(2)

    # 16-bit MUL latency on 64 pairs (array multiplier)
    mul_n = 64
    ma, mb = rng.integers(0, 1 << 16, mul_n), rng.integers(0, 1 << 16, mul_n)
    d_min = torch.from_numpy(encrypt_operands(ce, sk, ma, mb, 77).view(np.int32)).to(dev)
    d_mout = torch.empty((mul_n, 16, 501), dtype=torch.int32, device=dev)
    ce.ce_unit_eval_device(ctx, cid, "MUL", d_min, d_mout, mul_n, 0, stream)
    torch.cuda.synchronize(dev)
    mul_ms = []
    for _ in range(max(3, args.steps)):
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        ce.ce_unit_eval_device(ctx, cid, "MUL", d_min, d_mout, mul_n, 0, stream)
        m1.record(stream)
        torch.cuda.synchronize(dev)
        mul_ms.append(m0.elapsed_time(m1))
    mo = d_mout.cpu().numpy().view(np.uint32)
    for i in range(4):
        assert decrypt_word(ce, sk, mo[i]) == (int(ma[i]) * int(mb[i])) & 0xFFFF, "wrong product"
    mul_boots = mul_n * ce.ce_unit_info("MUL")["n_bootstraps"]

    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak_tops = int_peak_tops(sms, sm_mhz)
    forms = external_product_forms(ce, ctx, cid, stream, dev, rng, d_min, d_mout, mul_n,
                                   peak_tops, mulpipe_peak(sms, sm_mhz)) if rank == 0 else None
    programs = serving = None
    if rank == 0:
        from paper_2101_03403_gb300 import serve_bench
        extra, _, _ = serve_bench.admit_clients(ce, ctx, 32, SEED + 1000, rng)
        programs = programs_leg(ce, ctx, extra, rng)
        for k, (cid, sk) in enumerate(extra[:16]):    # serving reads r0, r1, r3 (r3 nonzero)
            ce.ce_reg_write(ctx, cid, 3, np.stack(
                [ce.ce_encrypt_bit(sk, ((k + 1) >> j) & 1, 950 + k, j) for j in range(16)]))
        serving = serving_leg(ce, ctx, extra[:16])
        # the same requests with ADD / SUB / MUL on the low-latency circuits
        ce.ce_set_instruction_circuits(ctx, True)
        try:
            fast = serving_leg(ce, ctx, extra[:16])
        finally:
            ce.ce_set_instruction_circuits(ctx, False)
        serving["low_latency_circuits"] = {
            k: fast[k] for k in ("requests_per_s", "bootstraps_per_s", "latency_ms_p50",
                                 "latency_ms_p99", "latency_ms_p50_by_op", "latency_ms_p99_by_op",
                                 "saturated_requests_per_s", "saturated_bootstraps_per_s")}
        for cid, _ in extra:
            ce.ce_client_evict(ctx, cid)

    br_ms, br_launches = prof["blind_rotate"]
    achieved = boots * args.steps * OPS_PER_GATE / (br_ms / 1e3) / 1e12
    # the same bound from the pipe's measured rates on this GPU
    rates = ce.ce_probe_int_pipes(ctx)
    sm_cycles_per_gate = 128 * 500 * sum(n / rates[k] for k, n in MUL_COUNTS_PER_THREAD_STEP.items())
    measured_bound = sms * sm_mhz * 1e6 / sm_cycles_per_gate
    measured_gps = boots * args.steps / (br_ms / 1e3)
    mp_peak = mulpipe_peak(sms, sm_mhz)
    mp_achieved = boots * args.steps * MULPIPE_CYCLES_PER_GATE / (br_ms / 1e3)
    roof = {"kernel": "blind_rotate", "bound": "alu", "achieved": mp_achieved / 1e12,
            "peak": mp_peak / 1e12, "unit": "T multiply-pipe warp-cycles/s",
            "frac": mp_achieved / mp_peak,
            "traffic": recorded_traffic("blind_rotate", args.steps and br_launches / args.steps),
            "peak_note": f"derived: {sms} SMs x 4 integer multiply-add pipes (16 lanes) x "
                         f"{sm_mhz:.0f} MHz (median SM clock sampled in the timed region); "
                         f"work = {MULPIPE_CYCLES_PER_GATE / 1e6:.1f} M pipe warp-cycles per "
                         "bootstrap (Shoup products 8, 64-bit key products 4, Montgomery "
                         "reductions 6, reconstructions 12 cycles per warp); ncu: that pipe is "
                         "~80 % busy, the binding unit",
            "measured_pipe": {"lane_ops_per_clock_per_sm": rates,
                              "bound_gates_per_s": measured_bound,
                              "blind_rotation_gates_per_s": measured_gps,
                              "frac": measured_gps / measured_bound,
                              "note": "the method's multiplies per bootstrap at the rates "
                                      "ce_probe_int_pipes measures on this GPU"},
            "int32_issue": {"achieved": achieved, "peak": peak_tops, "unit": "Tops/s (int32)",
                            "frac": achieved / peak_tops,
                            "note": f"{sms} SMs x {INT_LANES_PER_SM} int32 lanes per clock; "
                                    "work = 7 ops per butterfly + 2.5 per multiply-accumulate"},
            "launches_per_step": br_launches / args.steps,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}

    def pct(xs, q):
        return float(np.percentile(np.array(xs), q))

    cpu = None
    if rank == 0 and world == 1:
        cores = cpu_cores()
        g = 2 * cores
        cpu = {"value": oracle_sample(g, cores), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{g} bootstrapped gates (AND/XOR of the adder's first level), "
                         "one gate per thread"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (seeded encryptions of uniform 16-bit operands)",
                "config": {"workload": f"16-bit Kogge-Stone ADD on {n} encrypted operand pairs, "
                                       "level-batched (n=500 N=1024 l=3 Bg=2^10 t=8)",
                           "bootstraps_per_step": boots, "levels": 9,
                           "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"independent batches x{world}",
                           "graph_replay_gates_per_s": graph_value,
                           "autotuned_gates_per_block": tuned},
                "level_batching": batching,
                "latency_ms": {"add16_alone_p50": pct(add1_ms, 50),
                               "add16_alone_p99": pct(add1_ms, 99),
                               "add16_alone_repeats": len(add1_ms),
                               "add16_mux_carry_alone_p50": pct(addmux1_ms, 50),
                               "add16_mux_carry_alone_p99": pct(addmux1_ms, 99),
                               "mul16_alone_p50": pct(mul1_ms, 50),
                               "mul16_tree_alone_p50": pct(multree1_ms, 50),
                               "mul16_tree_alone_p99": pct(multree1_ms, 99),
                               "mul16_alone_p99": pct(mul1_ms, 99),
                               "mul16_alone_repeats": len(mul1_ms),
                               "add16_batch256_step_p50": pct(step_ms, 50),
                               "mul16_batch64_p50": pct(mul_ms, 50),
                               "mul16_bootstraps": mul_boots},
                "serving": serving,
                "programs": programs,
                "e2e": {"value": e2e_val, "unit": UNIT,
                        "h2d_bytes_per_step": int(host_in.nbytes),
                        "d2h_bytes_per_step": int(n * 16 * 501 * 4)},
                "gpu_launches": launches, "roofline": roof, "clocks": clocks,
                "cpu_baseline": cpu, "external_product_forms": forms}
        print(json.dumps(line), flush=True)
    ctx.close()


def program_set(rng, n=32, lo=8, hi=64):
    """Register programs of seeded random length lo..hi over 8 registers:
    ADD, SUB, AND, ORR, LSL (register and immediate), CMP, and conditional-
    select loops (a cleartext trip count of 2..4 of CMP; CSEL)."""
    progs = []
    for _ in range(n):
        length = int(rng.integers(lo, hi + 1))
        prog = [("CMP", 0, 1, 2, 0, 0)]                  # flags defined before any CSEL
        while len(prog) < length:
            kind = str(rng.choice(["ADD", "SUB", "AND", "ORR", "LSL", "LSL_IMM", "CMP",
                                   "CSEL_LOOP"]))
            r = [int(x) for x in rng.integers(0, 8, 3)]
            if kind == "CSEL_LOOP":
                cond = int(rng.integers(14))
                for _ in range(int(rng.integers(2, 5))):
                    prog += [("CMP", 0, r[1], r[2], 0, 0), ("CSEL", r[0], r[1], r[2], 0, cond)]
            elif kind == "LSL_IMM":
                prog.append(("LSL_IMM", r[0], r[1], 0, int(rng.integers(16)), 0))
            else:
                prog.append((kind, r[0], r[1], r[2], 0, 0))
        progs.append(prog[:length])
    return progs


def programs_leg(ce, ctx, clients, rng):
    """32 register programs, one per client, advancing together: the eager
    tick loop against the planned program set replayed as a captured CUDA
    graph (identical ciphertexts checked), wall time with a device sync."""
    progs = program_set(rng, len(clients))
    init = [[int(x) for x in rng.integers(0, 1 << 16, 8)] for _ in clients]
    ids = [cid for cid, _ in clients]
    code = [[ce.insn(*i) for i in p] for p in progs]

    def load():
        for k, (cid, sk) in enumerate(clients):
            for r, v in enumerate(init[k]):
                ce.ce_reg_write(ctx, cid, r, np.stack(
                    [ce.ce_encrypt_bit(sk, (v >> j) & 1, 900 + k, 16 * r + j) for j in range(16)]))

    def run(graphs):
        load()
        ce.ce_set_unit_graphs(ctx, graphs)
        ce.ce_synchronize(ctx)
        t0 = time.perf_counter()
        ce.ce_exec_multi(ctx, ids, code)
        ce.ce_synchronize(ctx)
        ms = (time.perf_counter() - t0) * 1e3
        regs = [ce.ce_reg_read(ctx, cid, r) for cid in ids[:4] for r in range(8)]
        return ms, regs

    eager_ms, eager = run(False)
    first_ms, _ = run(True)                       # plans the set and captures its graph
    replay_ms, replay = run(True)
    ce.ce_set_unit_graphs(ctx, True)
    assert all((a == b).all() for a, b in zip(eager, replay)), "program graph replay differs"
    n_ins = sum(len(p) for p in progs)
    return {"programs": len(progs), "instructions": n_ins,
            "lengths_min_max": [min(map(len, progs)), max(map(len, progs))],
            "eager_ms": eager_ms, "graph_plan_and_first_run_ms": first_ms,
            "graph_replay_ms": replay_ms, "per_program_ms_eager": eager_ms / len(progs),
            "per_program_ms_graph": replay_ms / len(progs), "identical_outputs": True}


def serving_leg(ce, ctx, clients, requests: int = 256, load: float = 0.9):
    """Short serving run (the configs' request mix at Poisson arrivals, a
    fraction of the measured saturated rate): per-request p50/p99 latency and
    bootstraps/s.  Clients have their own seeded key sets."""
    from paper_2101_03403_gb300 import serve_bench
    res = serve_bench.serve(ce, ctx, len(clients), requests, [load], seed=SEED + 1000,
                            clients=clients)
    pt = res["points"][0]
    return {"clients": res["clients_admitted"], "requests": pt["requests"], "load": load,
            "mix": res["mix"], "requests_per_s": pt["requests_per_s"],
            "bootstraps_per_s": pt["bootstraps_per_s"],
            "latency_ms_p50": pt["latency_ms_p50"], "latency_ms_p99": pt["latency_ms_p99"],
            "latency_ms_p50_by_op": pt["latency_ms_p50_by_op"],
            "latency_ms_p99_by_op": pt["latency_ms_p99_by_op"],
            "saturated_requests_per_s": res["saturated"]["requests_per_s"],
            "saturated_bootstraps_per_s": res["saturated"]["bootstraps_per_s"]}


def external_product_forms(ce, ctx, cid, stream, dev, rng, d_min, d_mout, mul_n, peak_tops,
                           mp_peak):
    """The blind rotation's external products in both forms on one batch of
    XP_GATES seeded gates and on the MUL-64 unit: the two-prime transform on
    the CUDA cores (default) and the Toeplitz contraction on the tensor cores.
    Outputs must be identical; each form's dominant kernel is set against its
    roofline (integer issue rate; measured tensor rate, fp16 = bf16 rate)."""
    import torch
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peaks = json.load(f)
    n = XP_GATES

    def dev_ct(shape):
        x = rng.integers(0, 1 << 32, shape + (501,), dtype=np.uint64).astype(np.uint32)
        return torch.from_numpy(x.view(np.int32)).to(dev)

    a, b = dev_ct((n,)), dev_ct((n,))
    ops = torch.from_numpy(rng.integers(0, 10, n).astype(np.uint8)).to(dev)
    outs, mul_outs, res = {}, {}, {}

    def ev_ms(fn, reps):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return ts

    for form, name in ((0, "transform_cuda_cores"), (1, "toeplitz_tensor_cores")):
        ce.ce_set_external_product_form(ctx, form)
        o = torch.empty((n, 501), dtype=torch.int32, device=dev)

        def batch():
            ce.ce_gates_batch_device(ctx, cid, ops, a, b, o, n, stream)

        batch()                                   # the tensor form builds its key here
        ce.ce_synchronize(ctx)
        batch_ms = statistics.median(ev_ms(batch, 3))
        ce.ce_profile_enable(ctx, True)
        batch()
        ce.ce_synchronize(ctx)
        prof = ce.ce_profile_read(ctx)
        ce.ce_profile_enable(ctx, False)
        outs[form] = o.cpu()

        def mul():
            ce.ce_unit_eval_device(ctx, cid, "MUL", d_min, d_mout, mul_n, 0, stream)

        mul()
        torch.cuda.synchronize(dev)
        mul_ms = statistics.median(ev_ms(mul, 2))
        mul_outs[form] = d_mout.cpu()
        nm = XP_MID_GATES
        om = torch.empty((nm, 501), dtype=torch.int32, device=dev)

        def mid():
            ce.ce_gates_batch_device(ctx, cid, ops[:nm], a[:nm], b[:nm], om, nm, stream)

        mid()
        mid_ms = statistics.median(ev_ms(mid, 3))
        outs[(form, "mid")] = om.cpu()
        entry = {"gates_per_s": n / (batch_ms / 1e3), "batch_ms": batch_ms,
                 "mul16_batch64_ms": mul_ms,
                 "mid_batch": {"gates": nm, "gates_per_s": nm / (mid_ms / 1e3),
                               "of_large_batch_rate": (nm / mid_ms) / (n / batch_ms)}}
        if form == 0:
            ms = prof["blind_rotate"][0]
            ach = n * MULPIPE_CYCLES_PER_GATE / (ms / 1e3)
            entry["roofline"] = {"kernel": "blind_rotate", "bound": "alu", "achieved": ach / 1e12,
                                 "peak": mp_peak / 1e12, "unit": "T multiply-pipe warp-cycles/s",
                                 "frac": ach / mp_peak,
                                 "int32_issue_frac": n * OPS_PER_GATE / (ms / 1e3) / 1e12 /
                                 peak_tops}
        else:
            ms, cnt = prof["external_product_mma"]
            ach = n * XP_FLOPS_PER_GATE / (ms / 1e3) / 1e12
            peak = peaks["bf16_tflops"]
            entry["roofline"] = {"kernel": "tt_mma", "bound": "tensor", "achieved": ach,
                                 "peak": peak, "unit": "TFLOP/s (fp16)", "frac": ach / peak,
                                 "frac_of_sustained_peak": ach / peaks["bf16_tflops_sustained"],
                                 "peak_note": "measured bf16 GEMM, burst (each MMA launch is "
                                              "timed alone; fp16 runs at the bf16 rate)",
                                 "launches": cnt, "kernel_ms": ms,
                                 "blind_rotate_ms": prof["blind_rotate"][0]}
        res[name] = entry
    ce.ce_set_external_product_form(ctx, 0)
    assert torch.equal(outs[0], outs[1]), "external-product forms disagree"
    assert torch.equal(mul_outs[0], mul_outs[1]), "external-product forms disagree on MUL"
    assert torch.equal(outs[(0, "mid")], outs[(1, "mid")]), "forms disagree on the mid batch"
    assert torch.equal(outs[(0, "mid")], outs[0][:XP_MID_GATES]), "mid batch differs"
    res["identical_outputs"] = True
    res["gates"] = n
    return res


def main():
    args = parse()
    if args.impl == "reference":
        rank, world, _ = dist_setup("gloo")
        run_reference(args, rank, world)
    else:
        rank, world, local = dist_setup("nccl")
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
