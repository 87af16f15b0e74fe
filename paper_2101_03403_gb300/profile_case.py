"""Runs one batch of bootstrapped gates through the device C-ABI call, for
profiling a single launch of each kernel (e.g. under Nsight Compute).

  python -m paper_2101_03403_gb300.profile_case --gates 608 [--reps 1] [--gpb 0]

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
    args = ap.parse_args()
    import torch

    import paper_2101_03403_gb300 as ce
    sk = ce.ce_secret_keygen(20210103)
    ck = ce.ce_cloud_keygen(sk, 20210103)
    ctx = ce.ce_create(0)
    cid = ce.ce_client_admit(ctx, ck)
    ce.ce_set_blind_rotate_config(ctx, args.gpb, 0)
    n = args.gates
    rng = np.random.default_rng(1)
    a = torch.from_numpy(rng.integers(0, 2 ** 32, (n, 501), dtype=np.uint64)
                         .astype(np.uint32).view(np.int32)).cuda()
    b = torch.roll(a, 1, 0).contiguous()
    c = torch.roll(a, 2, 0).contiguous()
    ops = torch.from_numpy(rng.integers(0, 10, n).astype(np.uint8)).cuda()
    out = torch.empty_like(a)
    s = torch.cuda.current_stream()
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
