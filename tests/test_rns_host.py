"""Host build of the blind rotation's two-prime transform against the oracle.

The transform header of the CUDA path (two primes below 2^28, Shoup
products, Montgomery key sums, Garner reconstruction) is compiled for the
host with every lazy bound checked, and one CMux step's external product
(six TRGSW rows: 3 gadget levels x 2 components, §3 "TFHE Library") is
compared bit for bit with the oracle's schoolbook negacyclic product,
including the largest exact sum the six rows can reach.  The harness runs
the 128-thread phases one thread after another in the kernel's barrier
order, so a wrong index map or a violated bound fails here without a GPU.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("rns") / "rns_host_check")
    subprocess.run([gxx, "-O2", "-std=c++17", os.path.join(HERE, "rns_host_check.cpp"), "-o", exe],
                   check=True)
    return exe


def run(exe, dig, key):
    data = np.ascontiguousarray(dig, np.int32).tobytes() + np.ascontiguousarray(key, np.uint32).tobytes()
    r = subprocess.run([exe], input=data, capture_output=True, check=True)
    out = np.frombuffer(r.stdout, np.uint32)
    return out[:2048].reshape(2, 1024), int(out[2048]), int(out[2049])


def expected(O, dig, key):
    exp = np.zeros((2, 1024), np.uint32)
    for o in range(2):
        acc = np.zeros(1024, np.uint64)
        for lvl in range(3):
            for c in range(2):
                acc += O.poly_mul(dig[lvl, c].astype(np.int64).astype(np.uint32), key[lvl, c, o])
        exp[o] = (acc & 0xFFFFFFFF).astype(np.uint32)
    return exp


@pytest.mark.parametrize("case", ["random", "max_positive", "max_negative", "mixed_extremes"])
def test_external_product_matches_oracle(O, harness, case):
    rng = np.random.default_rng({"random": 1, "max_positive": 2, "max_negative": 3,
                                 "mixed_extremes": 4}[case])
    if case == "random":
        dig = rng.integers(-512, 512, (3, 2, 1024))
        key = rng.integers(0, 2 ** 32, (3, 2, 2, 1024), dtype=np.uint64).astype(np.uint32)
    elif case == "max_positive":   # every term (-512)(-2^31) = +2^40: sum 6 * 1024 * 2^40
        dig = np.full((3, 2, 1024), -512)
        key = np.full((3, 2, 2, 1024), 0x80000000, np.uint32)
    elif case == "max_negative":   # every term 511 * (-2^31)
        dig = np.full((3, 2, 1024), 511)
        key = np.full((3, 2, 2, 1024), 0x80000000, np.uint32)
    else:
        dig = rng.choice([-512, 511, 0, -1, 1], (3, 2, 1024))
        key = rng.choice(np.array([0x80000000, 0x7FFFFFFF, 0, 1, 0xFFFFFFFF], np.uint32),
                         (3, 2, 2, 1024))
    got, bad_bounds, bad_direct = run(harness, dig, key)
    assert bad_bounds == 0, "a lazy bound of the transform arithmetic was exceeded"
    assert bad_direct == 0, "the forward transform differs from its definition"
    assert (got == expected(O, dig, key)).all()
