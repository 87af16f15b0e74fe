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
    # option setters: a null context is an error code
    for fn in ("ce_set_level_batching", "ce_set_instruction_circuits", "ce_set_unit_graphs",
               "ce_set_external_product_form", "ce_set_keyswitch_config"):
        assert getattr(L.lib(), fn)(None, 1) != 0, fn


def test_blind_rotation_launch_plan(L):
    """Launch planning of the blind rotation (host logic, no GPU): a batch
    whose gate groups leave the last round over the blocks part filled runs
    its whole rounds in the chosen shape and the rest as one more launch of
    one gate per block (up to one gate per block left) or, from four-gate
    groups, two (up to two per block); every gate lands in exactly one
    launch, the first launch is whole rounds, and the tail launch's blocks
    hold its gates."""
    for G in (1, 2, 3, 4):
        gsz = 1 if G == 3 else G
        for blocks in (1, 7, 152, 304):
            for n in list(range(0, 40)) + [151, 152, 153, 607, 608, 609, 700, 912, 913,
                                            2048, 3840, 5518, 7424, 7936, 8192]:
                p = L.ce_blind_rotate_plan(n, G, blocks)
                main, tail = p["main_jobs"], p["tail_jobs"]
                assert main + tail == n
                groups = -(-n // gsz)
                if tail == 0:
                    assert main == n
                    continue
                assert G in (2, 4) and groups > blocks
                assert main % (blocks * gsz) == 0 and main > 0
                if p["tail_shape"] == 3:
                    assert tail <= blocks and p["tail_blocks"] == tail
                else:
                    assert G == 4 and p["tail_shape"] == 2 and blocks < tail <= 2 * blocks
                    assert p["tail_blocks"] == -(-tail // 2)
    # the bench step's levels (16-bit ADD on 256 pairs, four-gate groups, 152 SMs)
    split = {n: L.ce_blind_rotate_plan(n, 4, 152) for n in (8192, 7936, 7680, 7424, 6656,
                                                           3584, 3840, 2304, 2048)}
    assert {n: (p["main_jobs"], p["tail_jobs"], p["tail_shape"]) for n, p in split.items()
            if p["tail_jobs"]} == {8192: (7904, 288, 2), 7936: (7904, 32, 3),
                                   7424: (7296, 128, 3), 3840: (3648, 192, 2),
                                   2048: (1824, 224, 2)}
    for bad in ((-1, 4, 152), (10, 0, 152), (10, 5, 152), (10, 4, 0)):
        with pytest.raises(Exception):
            L.ce_blind_rotate_plan(*bad)
