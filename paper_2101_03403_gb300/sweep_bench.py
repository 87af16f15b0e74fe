"""Latency and throughput sweeps on one GPU (one JSON line):

  python -m paper_2101_03403_gb300.sweep_bench [--programs 32] [--reps 5]
  python -m paper_2101_03403_gb300.sweep_bench --xp-gates 2432
  python -m paper_2101_03403_gb300.sweep_bench --forms-sweep
  python -m paper_2101_03403_gb300.sweep_bench --width 32

* gate batches: bootstrapped gates/s and batch latency for batch sizes from
  one gate to 9728 (autotuned launch shape per size);
* functional units: latency p50/p99 of every 16-bit unit on 1 and on 256
  operand sets (captured-graph replay, as a serving loop would run them);
* register programs: 32 encrypted programs (one per client, lengths uniform
  in [8, 64], ADD/SUB/AND/ORR/LSL/LSL_IMM/CMP/CSEL/MOV/MOV_IMM) advancing
  together through ce_exec_multi, and the longest one alone.

With --width W (W != 16): only the functional units at width W, latency of
1 and of 16 operand sets (UDIV: 1).

With --forms-sweep: only the gate-batch sweep, once with the blind rotation's
external products in the transform form (CUDA cores, autotuned shape) and
once in the Toeplitz form (tensor cores).

With --xp-gates N: one batch of N gates with the blind rotation's external
products on the tensor cores (Toeplitz form), after one warm-up batch that
also builds the key form; nothing else runs, so a profiler skips the
admission (2 launches) and the warm-up batch (1005 launches for N >= 32).

Inputs are seeded uniform 501-word ciphertexts (the bootstrapping path is a
fixed function of any input, so timing does not need valid encryptions);
keys come from seed 20210103 + client.  Times are CUDA events on the
calling stream (units, gates) or host wall time around synchronous calls
(programs).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

SEED = 20210103
BATCHES = [1, 8, 38, 76, 152, 304, 608, 1216, 2432, 4864, 9728]


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q))


def tensor_form_batch(n):
    import torch

    import paper_2101_03403_gb300 as ce
    rng = np.random.default_rng(SEED)
    sk = ce.ce_secret_keygen(SEED)
    ctx = ce.ce_create(0)
    cid = ce.ce_client_admit(ctx, ce.ce_cloud_keygen(sk, SEED))
    st = torch.cuda.current_stream()

    def ct():
        x = rng.integers(0, 2 ** 32, (n, 501), dtype=np.uint64).astype(np.uint32)
        return torch.from_numpy(x.view(np.int32)).cuda()

    a, b = ct(), ct()
    ops = torch.from_numpy(rng.integers(0, 10, n).astype(np.uint8)).cuda()
    o = torch.empty((n, 501), dtype=torch.int32, device="cuda")
    ce.ce_set_external_product_form(ctx, 1)
    ms = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ce.ce_gates_batch_device(ctx, cid, ops, a, b, o, n, st)
        e1.record(st)
        ce.ce_synchronize(ctx)
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"form": "toeplitz_tensor_cores", "gates": n, "warmup_ms": ms[0],
                      "batch_ms": ms[1], "gates_per_s": n / ms[1] * 1e3,
                      "launches": ce.ce_last_launch_count(ctx)}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--programs", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--xp-gates", type=int, default=0)
    ap.add_argument("--forms-sweep", action="store_true")
    ap.add_argument("--width", type=int, default=16)
    args = ap.parse_args()
    if args.xp_gates:
        return tensor_form_batch(args.xp_gates)
    import torch

    import paper_2101_03403_gb300 as ce
    rng = np.random.default_rng(SEED)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    sk = ce.ce_secret_keygen(SEED)
    ctx = ce.ce_create(0)
    cid = ce.ce_client_admit(ctx, ce.ce_cloud_keygen(sk, SEED))
    ce.ce_autotune(ctx, cid)

    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ce.ce_synchronize(ctx)
        return ts

    def rand_ct(shape):
        return torch.from_numpy(rng.integers(0, 2 ** 32, shape + (501,), dtype=np.uint64)
                                .astype(np.uint32).view(np.int32)).to(dev)

    out = {"gpu": torch.cuda.get_device_name(0)}

    # gate batches
    def batch_sweep():
        sweep = []
        for n in BATCHES:
            a, b = rand_ct((n,)), rand_ct((n,))
            ops = torch.from_numpy(rng.integers(0, 10, n).astype(np.uint8)).to(dev)
            o = torch.empty((n, 501), dtype=torch.int32, device=dev)
            ts = ev_time(lambda: ce.ce_gates_batch_device(ctx, cid, ops, a, b, o, n, stream),
                         args.reps)
            ms = pct(ts, 50)
            sweep.append({"gates": n, "ms_p50": ms, "gates_per_s": n / ms * 1e3})
        return sweep

    if args.width != 16:
        units = {}
        for unit in ce.UNITS:
            info = ce.ce_unit_info(unit, 0, args.width)
            row = {"bootstraps_per_op": info["n_bootstraps"], "depth": info["depth"]}
            for n in ((1,) if unit == "UDIV" else (1, 16)):
                d_in = rand_ct((n, info["n_inputs"]))
                d_out = torch.empty((n, info["n_outputs"], 501), dtype=torch.int32, device=dev)
                ts = ev_time(lambda: ce.ce_unit_eval_device_width(ctx, cid, unit, args.width, d_in,
                                                                  d_out, n, 0, stream),
                             min(args.reps, 3))
                row[f"n{n}"] = {"p50_ms": pct(ts, 50), "p99_ms": pct(ts, 99),
                                "bootstraps_per_s": n * info["n_bootstraps"] / pct(ts, 50) * 1e3}
            units[unit] = row
        out[f"unit_latency_width{args.width}"] = units
        print(json.dumps(out), flush=True)
        ctx.close()
        return

    out["gate_batch_sweep"] = batch_sweep()
    if args.forms_sweep:
        ce.ce_set_external_product_form(ctx, 1)
        out["gate_batch_sweep_tensor_form"] = batch_sweep()
        ce.ce_set_external_product_form(ctx, 0)
        print(json.dumps(out), flush=True)
        ctx.close()
        return

    # functional units
    units = {}
    for unit in ce.UNITS:
        info = ce.ce_unit_info(unit)
        row = {"bootstraps_per_op": info["n_bootstraps"], "depth": info["depth"]}
        for n in (1, 256):
            d_in = rand_ct((n, info["n_inputs"]))
            d_out = torch.empty((n, info["n_outputs"], 501), dtype=torch.int32, device=dev)
            ts = ev_time(lambda: ce.ce_unit_eval_device(ctx, cid, unit, d_in, d_out, n, 0, stream),
                         args.reps)
            row[f"n{n}"] = {"p50_ms": pct(ts, 50), "p99_ms": pct(ts, 99),
                            "bootstraps_per_s": n * info["n_bootstraps"] / pct(ts, 50) * 1e3}
        units[unit] = row
    out["unit_latency"] = units

    # register programs, one client each
    ops = ["ADD", "SUB", "AND", "ORR", "LSL", "LSL_IMM", "CMP", "CSEL", "MOV", "MOV_IMM"]
    clients, progs = [], []
    for p in range(args.programs):
        c = ce.ce_client_admit(ctx, ce.ce_cloud_keygen(ce.ce_secret_keygen(SEED + 1 + p), SEED + 1 + p))
        clients.append(c)
        for r in range(8):
            ce.ce_reg_write(ctx, c, r, rng.integers(0, 2 ** 32, (16, 501), dtype=np.uint64)
                            .astype(np.uint32))
        length = int(rng.integers(8, 65))
        prog = [ce.insn("CMP", 0, 1, 2)]
        while len(prog) < length:
            op = ops[rng.integers(len(ops))]
            prog.append(ce.insn(op, int(rng.integers(8)), int(rng.integers(8)), int(rng.integers(8)),
                                int(rng.integers(256)), int(rng.integers(14))))
        progs.append(prog)
    ce.ce_exec_multi(ctx, clients[:1], progs[:1])  # warm-up (netlists, graphs, scratch)
    t0 = time.perf_counter()
    ce.ce_exec_multi(ctx, clients, progs)
    ce.ce_synchronize(ctx)
    wall = time.perf_counter() - t0
    longest = int(np.argmax([len(p) for p in progs]))
    t1 = time.perf_counter()
    ce.ce_exec(ctx, clients[longest], progs[longest])
    ce.ce_synchronize(ctx)
    alone = time.perf_counter() - t1
    out["programs"] = {"count": len(progs), "instructions": int(sum(len(p) for p in progs)),
                       "all_together_s": wall, "longest_instructions": len(progs[longest]),
                       "longest_alone_s": alone}
    print(json.dumps(out), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
