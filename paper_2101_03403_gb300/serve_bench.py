"""Serving benchmark: many clients, each with its own keys, send encrypted
16-bit ADD/SUB/MUL/DIV instructions at Poisson arrivals; the server batches
them continuously.  Reports per-request latency percentiles, bootstraps/s,
and admissions refused by the HBM budget.

  python -m paper_2101_03403_gb300.serve_bench --clients 256 --requests 8192 \\
      --loads 0.5,0.9,1.2 [--budget-gb 0]

Capacity is first measured by submitting one request per client at once and
timing their completion; the offered loads are fractions of it.  Inputs are
synthetic and seeded (client keys from seed 20210103 + client index, register
values uniform 16-bit).
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np

MIX = [("ADD", 0.4), ("SUB", 0.3), ("MUL", 0.2), ("UDIV", 0.1)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--clients", type=int, default=256)
    ap.add_argument("--requests", type=int, default=8192, help="requests per load point")
    ap.add_argument("--loads", default="0.5,0.9,1.2")
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=20210103)
    args = ap.parse_args()
    import torch

    import paper_2101_03403_gb300 as ce
    torch.cuda.init()
    ctx = ce.ce_create(0, int(args.budget_gb * 2**30))
    rng = np.random.default_rng(args.seed)
    clients, refused = [], 0
    t0 = time.perf_counter()
    for k in range(args.clients):
        sk = ce.ce_secret_keygen(args.seed + k)
        ck = ce.ce_cloud_keygen(sk, args.seed + k)
        try:
            cid = ce.ce_client_admit(ctx, ck)
        except ce.CeError as e:
            if e.code == -3:
                refused += 1
                continue
            raise
        for r in range(4):
            v = int(rng.integers(0, 1 << 16))
            if r == 3:
                v = int(rng.integers(1, 1 << 16))      # divisor register nonzero
            bits = np.stack([ce.ce_encrypt_bit(sk, (v >> j) & 1, 7, 64 * k + 16 * r + j)
                             for j in range(16)])
            ce.ce_reg_write(ctx, cid, r, bits)
        clients.append((cid, sk))
    setup_s = time.perf_counter() - t0
    boots = {u: ce.ce_unit_info(u)["n_bootstraps"] for u, _ in MIX}
    ops, probs = zip(*MIX)

    def request(i):
        op = ops[rng.choice(len(ops), p=probs)]
        rm = 3 if op == "UDIV" else 1
        return op, ce.insn(op, 2, 0, rm)

    srv = ce.ce_server_create(ctx)

    def run(n, rate):
        """Submit n requests (Poisson at `rate` per second, or all at once)."""
        tickets, kinds = [], []
        start = time.perf_counter()
        tnext = start
        for i in range(n):
            cid, _ = clients[i % len(clients)]
            op, ins = request(i)
            if rate:
                tnext += rng.exponential(1.0 / rate)
                d = tnext - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            tickets.append(ce.ce_server_submit(srv, cid, ins))
            kinds.append(op)
        for t in tickets:
            ce.ce_server_wait(srv, t, 3600 * 10**9)
        wall = time.perf_counter() - start
        info = [ce.ce_server_poll(srv, t) for t in tickets]
        lat = np.array([(x["done_ns"] - x["submit_ns"]) / 1e6 for x in info])
        b = sum(boots[k] for k in kinds)
        return {"requests": n, "offered_rate_per_s": rate, "wall_s": wall,
                "bootstraps_per_s": b / wall, "requests_per_s": n / wall,
                "latency_ms_p50": float(np.percentile(lat, 50)),
                "latency_ms_p99": float(np.percentile(lat, 99)),
                "latency_ms_p50_by_op": {o: float(np.percentile(lat[np.array(kinds) == o], 50))
                                         for o in ops if (np.array(kinds) == o).any()}}

    sat = run(min(args.requests, 4 * len(clients)), 0)
    cap = sat["requests_per_s"]
    points = []
    for load in [float(x) for x in args.loads.split(",") if x]:
        points.append({"load": load, **run(args.requests, load * cap)})
    stats = ce.ce_server_stats(srv)
    ce.ce_server_destroy(srv)
    print(json.dumps({"clients_admitted": len(clients), "clients_refused": refused,
                      "client_device_bytes": ce.ce_client_footprint_bytes(),
                      "setup_s": setup_s, "saturated": sat, "points": points,
                      "server_ticks": stats["ticks"]}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
