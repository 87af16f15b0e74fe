"""Shared fixtures for the GPU tests (library context, keys, oracle)."""
import os

import numpy as np
import pytest

MASTER_SEED = 20210103


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ce():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2101_03403_gb300 import build
    build.build()
    import paper_2101_03403_gb300 as ce
    return ce


@pytest.fixture(scope="session")
def keys(ce, full_keys):
    """Library secret + cloud key (byte-identical to the oracle's, checked)."""
    sk = ce.ce_secret_keygen(MASTER_SEED)
    ck = ce.ce_cloud_keygen(sk, MASTER_SEED)
    assert (ck.bsk() == full_keys.bsk).all() and (ck.ksk() == full_keys.ksk).all()
    return sk, ck


@pytest.fixture(scope="session")
def ctx(ce, keys):
    import torch
    torch.cuda.init()
    c = ce.ce_create(0)
    cid = ce.ce_client_admit(c, keys[1])
    yield c, cid
    c.close()


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def run_gates_device(ce, ctx, ops, a, b):
    import torch
    c, cid = ctx
    n = len(ops)
    d_ops = to_dev(np.asarray(ops, np.uint8))
    d_a = to_dev(np.asarray(a, np.uint32).reshape(n, 501).view(np.int32))
    d_b = to_dev(np.asarray(b, np.uint32).reshape(n, 501).view(np.int32))
    d_out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
    ce.ce_gates_batch_device(c, cid, d_ops, d_a, d_b, d_out, n, torch.cuda.current_stream())
    ce.ce_synchronize(c)
    torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.uint32)


def random_ciphertexts(rng, n):
    """Uniform 501-word inputs: bootstrapping is a deterministic function of
    any input, so parity does not need valid encryptions."""
    return rng.integers(0, 2 ** 32, (n, 501), dtype=np.uint64).astype(np.uint32)


def encrypt_bits(ce, sk, bits, seed):
    return np.stack([ce.ce_encrypt_bit(sk, int(b), seed, i) for i, b in enumerate(bits)])
