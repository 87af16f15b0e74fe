"""Runs one batch of bootstrapped gates through the device C-ABI call, for
profiling a single launch of each kernel (e.g. under Nsight Compute).

  python -m paper_2101_03403_gb300.profile_case --gates 608 [--reps 1] [--gpb 0] [--xp 1]
  python -m paper_2101_03403_gb300.profile_case --unit ADD --pairs 256

The second form runs one eager evaluation of a functional unit on encrypted
operand pairs (the benchmark's step for ADD with 256 pairs).  --xp 1 selects
the Toeplitz form of the external products on the tensor cores (its key is
built by an untimed first call); --ks selects the key-switch engine.

Keys come from seed 20210103; inputs are uniform 501-word ciphertexts (the
bootstrapping path is a fixed function of any input, so timing and
profiling do not need valid encryptions).
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gates", type=int, default=608)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--gpb", type=int, default=0, help="gates per block (0 = autotuned)")
    ap.add_argument("--mux", action="store_true")
    ap.add_argument("--unit", default=None, help="run a functional unit instead of gates")
    ap.add_argument("--pairs", type=int, default=256)
    ap.add_argument("--xp", type=int, default=0, help="external-product form (1: tensor cores)")
    ap.add_argument("--ks", type=int, default=0, help="key-switch engine (1 CUDA, 2 tensor)")
    args = ap.parse_args()
    import torch

    import paper_2101_03403_gb300 as ce
    sk = ce.ce_secret_keygen(20210103)
    ck = ce.ce_cloud_keygen(sk, 20210103)
    ctx = ce.ce_create(0)
    cid = ce.ce_client_admit(ctx, ck)
    ce.ce_set_blind_rotate_config(ctx, args.gpb, 0)
    ce.ce_set_external_product_form(ctx, args.xp)
    ce.ce_set_keyswitch_config(ctx, args.ks)
    if args.unit:
        rng = np.random.default_rng(2)
        info = ce.ce_unit_info(args.unit)
        n = args.pairs
        bits = rng.integers(0, 2, (n, info["n_inputs"]))
        inp = np.zeros((n, info["n_inputs"], 501), np.uint32)
        for i in range(n):
            for j in range(info["n_inputs"]):
                inp[i, j] = ce.ce_encrypt_bit(sk, int(bits[i, j]), 3, i * info["n_inputs"] + j)
        d_in = torch.from_numpy(inp.view(np.int32)).cuda()
        d_out = torch.empty((n, info["n_outputs"], 501), dtype=torch.int32, device="cuda")
        ce.ce_set_unit_graphs(ctx, False)
        for _ in range(args.reps):
            ce.ce_unit_eval_device(ctx, cid, args.unit, d_in, d_out, n, 0, torch.cuda.current_stream())
        ce.ce_synchronize(ctx)
        print(f"ran {args.reps} x {args.unit} on {n} pairs")
        ctx.close()
        return
    n = args.gates
    rng = np.random.default_rng(1)
    a = torch.from_numpy(rng.integers(0, 2 ** 32, (n, 501), dtype=np.uint64)
                         .astype(np.uint32).view(np.int32)).cuda()
    b = torch.roll(a, 1, 0).contiguous()
    c = torch.roll(a, 2, 0).contiguous()
    ops = torch.from_numpy(rng.integers(0, 10, n).astype(np.uint8)).cuda()
    out = torch.empty_like(a)
    s = torch.cuda.current_stream()
    if args.xp:   # builds the tensor form's key (kernels outside the profiled launches)
        ce.ce_gates_batch_device(ctx, cid, ops[:1], a[:1], b[:1], out[:1], 1, s)
        ce.ce_synchronize(ctx)
    for _ in range(args.reps):
        if args.mux:
            ce.ce_mux_batch_device(ctx, cid, a, b, c, out, n, s)
        else:
            ce.ce_gates_batch_device(ctx, cid, ops, a, b, out, n, s)
    ce.ce_synchronize(ctx)
    print(f"ran {args.reps} x {n} {'mux' if args.mux else 'gates'}")
    ctx.close()


if __name__ == "__main__":
    main()
