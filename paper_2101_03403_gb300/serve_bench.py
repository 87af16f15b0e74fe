"""Serving benchmark: many clients, each with its own keys, send encrypted
16-bit ADD/SUB/MUL/DIV instructions at Poisson arrivals; the server batches
them continuously (§4 "Cloud service model").  Reports per-request latency
percentiles, bootstraps/s, and admissions refused by the HBM budget.

  python -m paper_2101_03403_gb300.serve_bench --clients 256 --requests 8192 \\
      --loads 0.5,0.9,1.2 [--budget-gb 0]

Capacity is first measured by submitting requests for every client at once
and timing their completion; the offered loads are fractions of it.  Inputs
are synthetic and seeded (client keys from seed 20210103 + client index,
register values uniform 16-bit, the divisor register nonzero).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

MIX = [("ADD", 0.4), ("SUB", 0.3), ("MUL", 0.2), ("UDIV", 0.1)]


def admit_clients(ce, ctx, n_clients: int, seed: int, rng):
    """Admit n_clients with their own key sets and four encrypted registers
    each; returns ([(client id, secret key)], refused count, seconds)."""
    clients, refused = [], 0
    t0 = time.perf_counter()
    for k in range(n_clients):
        sk = ce.ce_secret_keygen(seed + k)
        ck = ce.ce_cloud_keygen(sk, seed + k)
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
    return clients, refused, time.perf_counter() - t0


def run_load(ce, srv, clients, n: int, rate: float, rng) -> dict:
    """Submit n requests of the MIX round-robin over the clients, at Poisson
    arrivals of `rate` per second (0: all at once); wait for all of them."""
    boots = {u: ce.ce_unit_info(u)["n_bootstraps"] for u, _ in MIX}
    ops, probs = zip(*MIX)
    tickets, kinds = [], []
    start = time.perf_counter()
    tnext = start
    for i in range(n):
        cid, _ = clients[i % len(clients)]
        op = ops[rng.choice(len(ops), p=probs)]
        ins = ce.insn(op, 2, 0, 3 if op == "UDIV" else 1)
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
    kinds = np.array(kinds)
    b = sum(boots[k] for k in kinds)
    return {"requests": n, "offered_rate_per_s": rate, "wall_s": wall,
            "bootstraps_per_s": b / wall, "requests_per_s": n / wall,
            "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_p50_by_op": {o: float(np.percentile(lat[kinds == o], 50))
                                     for o in ops if (kinds == o).any()},
            "latency_ms_p99_by_op": {o: float(np.percentile(lat[kinds == o], 99))
                                     for o in ops if (kinds == o).any()}}


def serve(ce, ctx, n_clients: int, n_requests: int, loads, seed: int = 20210103,
          saturate_per_client: int = 4, clients=None) -> dict:
    """Admit the clients (or use the given (id, secret key) pairs, whose
    registers 0..3 hold values, 3 nonzero), measure saturated capacity, then
    run each offered load (a fraction of that capacity) with n_requests
    requests."""
    rng = np.random.default_rng(seed)
    own = clients is None
    if own:
        clients, refused, setup_s = admit_clients(ce, ctx, n_clients, seed, rng)
    else:
        refused, setup_s = 0, 0.0
    srv = ce.ce_server_create(ctx)
    try:
        sat = run_load(ce, srv, clients, min(n_requests, saturate_per_client * len(clients)), 0,
                       rng)
        points = [{"load": load, **run_load(ce, srv, clients, n_requests,
                                            load * sat["requests_per_s"], rng)}
                  for load in loads]
        stats = ce.ce_server_stats(srv)
    finally:
        ce.ce_server_destroy(srv)
    if own:
        for cid, _ in clients:
            ce.ce_client_evict(ctx, cid)
    return {"clients_admitted": len(clients), "clients_refused": refused,
            "client_device_bytes": ce.ce_client_footprint_bytes(), "setup_s": setup_s,
            "mix": dict(MIX), "saturated": sat, "points": points,
            "server_ticks": stats["ticks"]}


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
    res = serve(ce, ctx, args.clients, args.requests,
                [float(x) for x in args.loads.split(",") if x], args.seed)
    print(json.dumps(res), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
