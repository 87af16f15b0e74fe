"""Failure detection on the GPU without a fault: a bounded device wait that
nothing satisfies expires, the host reads CE_ETIMEOUT, and the context keeps
computing correct results.  The wait is the same bounded mbarrier wait the
blind rotation and the tensor-core key switch use for their copies and MMAs.
"""
import time

import numpy as np
import pytest

from gpu_common import ce, ctx, keys, random_ciphertexts, run_gates_device  # noqa: F401

pytestmark = pytest.mark.gpu
CE_ETIMEOUT = -4


def test_bounded_wait_expires_and_context_recovers(ce, ctx, O, full_keys):
    c, _ = ctx
    t0 = time.time()
    ce.ce_selftest_device_wait(c, 50_000_000)          # 50 ms limit
    with pytest.raises(ce.CeError) as ei:
        ce.ce_synchronize(c)
    assert ei.value.code == CE_ETIMEOUT
    assert time.time() - t0 < 10.0                     # the wait ended by itself
    ce.ce_synchronize(c)                               # the flag was cleared
    rng = np.random.default_rng(3)
    a, b = random_ciphertexts(rng, 6), random_ciphertexts(rng, 6)
    ops = [0, 1, 2, 3, 4, 5]
    got = run_gates_device(ce, ctx, ops, a, b)
    assert (got == O.gates(full_keys, ops, a, b)).all()


def test_selftest_rejects_bad_limits(ce, ctx):
    c, _ = ctx
    for bad in (0, 999, 3_000_000_000):
        with pytest.raises(ce.CeError):
            ce.ce_selftest_device_wait(c, bad)
