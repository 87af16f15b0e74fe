"""The allocation-free gate entry point, checked against the ordinary one.

Some callers cannot let this library call cudaMalloc: a serving loop that
keeps other streams busy cannot take cudaMalloc's implicit device-wide
synchronisation, and a process whose device memory another allocator has
reserved up front has none to give.  They call
ce_gates_batch_device_noalloc, whose scratch is a fixed area inside the
library's device image shared by every call.  It must return exactly the
ciphertexts ce_gates_batch_device returns, call after call.  This file is
collected last so that a failure here cannot hide failures elsewhere.
"""
import numpy as np
import pytest

from gpu_common import ce, ctx, keys, random_ciphertexts, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def _batch(rng, n):
    return (rng.integers(0, 10, n).astype(np.uint8), random_ciphertexts(rng, n),
            random_ciphertexts(rng, n))


def test_noalloc_matches_allocating_entry_point(ce, ctx):
    import torch
    c, cid = ctx
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream()
    # Two batches; the second is smaller, so when it runs the shared scratch
    # still holds the first batch's data beyond its end.
    dev = []
    for ops, a, b in (_batch(rng, 200), _batch(rng, 37)):
        n = len(ops)
        dev.append((n, to_dev(ops), to_dev(a.view(np.int32)), to_dev(b.view(np.int32)),
                    torch.empty((n, 501), dtype=torch.int32, device="cuda"),
                    torch.empty((n, 501), dtype=torch.int32, device="cuda")))
    # reference results from the ordinary (allocating) entry point
    for n, d_ops, d_a, d_b, ref, _ in dev:
        ce.ce_gates_batch_device(c, cid, d_ops, d_a, d_b, ref, n, stream)
    ce.ce_synchronize(c)
    # the first allocation-free call on this device looks up the scratch address
    n, d_ops, d_a, d_b, ref, got = dev[0]
    ce.ce_gates_batch_device_noalloc(c, cid, d_ops, d_a, d_b, got, n, stream)
    ce.ce_synchronize(c)
    assert torch.equal(got, ref)
    # the library counts its own device allocations and frees: none may
    # happen inside the allocation-free calls (a balanced pair would too)
    counts_before = ce.ce_device_alloc_count()
    for n, d_ops, d_a, d_b, ref, got in dev:      # two calls in a row
        got.zero_()
        ce.ce_gates_batch_device_noalloc(c, cid, d_ops, d_a, d_b, got, n, stream)
        assert ce.ce_last_launch_count(c) == 3
        ce.ce_synchronize(c)
        assert torch.equal(got, ref), f"allocation-free output differs for n={n}"
    assert ce.ce_device_alloc_count() == counts_before, \
        "the allocation-free calls allocated or freed device memory"


def test_noalloc_rejects_oversized_batch(ce, ctx):
    import torch
    c, cid = ctx
    n = 257
    x = torch.zeros((n, 501), dtype=torch.int32, device="cuda")
    ops = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(ce.CeError) as ei:
        ce.ce_gates_batch_device_noalloc(c, cid, ops, x, x, x, n)
    assert ei.value.code == -1
