"""CPU-side checks of the C-ABI library: it loads, exports every declared
symbol, and its host key generation / encryption match the oracle's
independent implementation byte for byte."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2101_03403_gb300 import build
    build.build()
    import paper_2101_03403_gb300 as ce
    ce.lib()
    return ce


def test_exports_every_declared_symbol(L):
    names = L.header_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L.lib(), n)]
    assert not missing, missing


def test_secret_key_matches_oracle(L, O):
    sk = L.ce_secret_keygen(20210103)
    s, K = O.secret_keygen(O.GATE_PARAMS, 20210103)
    assert (sk.s == s).all() and (sk.K == K).all()


def test_cloud_key_matches_oracle_bytes(L, O, full_keys):
    sk = L.ce_secret_keygen(20210103)
    ck = L.ce_cloud_keygen(sk, 20210103)
    assert (ck.bsk() == full_keys.bsk).all()
    assert (ck.ksk() == full_keys.ksk).all()


def test_encrypt_decrypt_match_oracle(L, O, full_keys):
    sk = L.ce_secret_keygen(20210103)
    p = O.GATE_PARAMS
    for ctr in range(50):
        bit = ctr % 2
        c = L.ce_encrypt_bit(sk, bit, 99, ctr)
        assert (c == O.encrypt(p, full_keys.s, bit, 99, ctr)).all()
        assert L.ce_decrypt_bit(sk, c) == bit == O.decrypt(p, full_keys.s, c)


def test_bad_arguments_are_errors_not_crashes(L):
    import ctypes
    assert L.lib().ce_decrypt_bit(None, None) == -1
    with pytest.raises(L.CeError):
        L.ce_cloud_keygen(L.SecretKey(0, 0), 1)
    with pytest.raises(L.CeError):   # no GPU here or bad device: an error code, not an abort
        L.ce_create(device=9999)
