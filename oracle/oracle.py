"""Python access to the plain CPU oracle (oracle/tfhe_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.  The oracle computes TFHE gate bootstrapping (the binary gates of
the paper's §3, Table "TFHE API Benchmark") by plain schoolbook integer
arithmetic; see tfhe_oracle.h for the conventions.

The shared library is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "tfhe_oracle.c")]
_HDR = os.path.join(_HERE, "tfhe_oracle.h")

GATES = ["NAND", "AND", "OR", "XOR", "NOR", "XNOR", "ANDNY", "ANDYN", "ORNY", "ORYN"]
GATE_ID = {g: i for i, g in enumerate(GATES)}
TRUTH = {
    "NAND": lambda a, b: 1 - (a & b),
    "AND": lambda a, b: a & b,
    "OR": lambda a, b: a | b,
    "XOR": lambda a, b: a ^ b,
    "NOR": lambda a, b: 1 - (a | b),
    "XNOR": lambda a, b: 1 - (a ^ b),
    "ANDNY": lambda a, b: (1 - a) & b,
    "ANDYN": lambda a, b: a & (1 - b),
    "ORNY": lambda a, b: (1 - a) | b,
    "ORYN": lambda a, b: a | (1 - b),
}
MU = 1 << 29  # +1/8 on the torus


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("Bgbit", ctypes.c_int32), ("t", ctypes.c_int32), ("basebit", ctypes.c_int32),
                ("sigma_lwe", ctypes.c_double), ("sigma_bk", ctypes.c_double)]


@dataclass(frozen=True)
class Params:
    n: int = 500
    N: int = 1024
    l: int = 3
    Bgbit: int = 10
    t: int = 8
    basebit: int = 2
    sigma_lwe: float = 2.0 ** -15
    sigma_bk: float = 9e-9

    def c(self) -> _Params:
        return _Params(self.n, self.N, self.l, self.Bgbit, self.t, self.basebit,
                       self.sigma_lwe, self.sigma_bk)

    @property
    def bsk_words(self) -> int:
        return self.n * 2 * self.l * 2 * self.N

    @property
    def ksk_words(self) -> int:
        return self.N * self.t * (1 << self.basebit) * (self.n + 1)


GATE_PARAMS = Params()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp] + _SRC + ["-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        u32p = ctypes.c_void_p
        L.or_splitmix64_at.restype = ctypes.c_uint64
        L.or_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_uniform32.restype = ctypes.c_uint32
        L.or_uniform32.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.or_gauss32.restype = ctypes.c_uint32
        L.or_gauss32.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double]
        L.or_secret_keygen.argtypes = [P, ctypes.c_uint64, u32p, u32p]
        L.or_bsk_keygen.argtypes = [P, ctypes.c_uint64, u32p, u32p, u32p]
        L.or_ksk_keygen.argtypes = [P, ctypes.c_uint64, u32p, u32p, u32p]
        L.or_encrypt.argtypes = [P, u32p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u32p]
        L.or_phase.restype = ctypes.c_uint32
        L.or_phase.argtypes = [P, u32p, u32p]
        L.or_decrypt.restype = ctypes.c_int
        L.or_decrypt.argtypes = [P, u32p, u32p]
        L.or_poly_mul.argtypes = [ctypes.c_int32, u32p, u32p, u32p]
        L.or_decompose.argtypes = [P, ctypes.c_uint32, u32p]
        L.or_modswitch.restype = ctypes.c_uint32
        L.or_modswitch.argtypes = [ctypes.c_uint32, ctypes.c_int32]
        L.or_gate_lincomb.argtypes = [P, ctypes.c_int, u32p, u32p, u32p]
        L.or_blind_rotate.argtypes = [P, u32p, u32p, ctypes.c_uint32, ctypes.c_uint32, u32p]
        L.or_sample_extract.argtypes = [P, u32p, u32p]
        L.or_key_switch.argtypes = [P, u32p, u32p, u32p]
        L.or_bootstrap.argtypes = [P, u32p, u32p, u32p, u32p]
        L.or_gate.argtypes = [P, u32p, u32p, ctypes.c_int, u32p, u32p, u32p]
        L.or_mux.argtypes = [P, u32p, u32p, u32p, u32p, u32p, u32p]
        L.or_constant.argtypes = [P, ctypes.c_int, u32p]
        L.or_not.argtypes = [P, u32p, u32p]
        L.or_gates_threaded.argtypes = [P, u32p, u32p, u32p, u32p, u32p, u32p,
                                        ctypes.c_int64, ctypes.c_int32]
        L.or_muxes_threaded.argtypes = [P, u32p, u32p, u32p, u32p, u32p, u32p,
                                        ctypes.c_int64, ctypes.c_int32]
        _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- PRNG ---
def splitmix64_at(seed: int, k: int) -> int:
    return int(lib().or_splitmix64_at(seed, k))


def uniform32(seed: int, domain: int, i: int) -> int:
    return int(lib().or_uniform32(seed, domain, i))


def gauss32(seed: int, domain: int, i: int, sigma: float) -> int:
    return int(lib().or_gauss32(seed, domain, i, sigma))


# ---------------------------------------------------------------- keys ---
@dataclass
class Keys:
    params: Params
    s: np.ndarray      # [n] uint32 in {0,1}
    K: np.ndarray      # [N] uint32 in {0,1}
    bsk: np.ndarray    # [n][2l][2][N] uint32
    ksk: np.ndarray    # [N][t][2^basebit][n+1] uint32


def secret_keygen(p: Params, seed: int):
    s = np.zeros(p.n, np.uint32)
    K = np.zeros(p.N, np.uint32)
    lib().or_secret_keygen(ctypes.byref(p.c()), seed, _ptr(s), _ptr(K))
    return s, K


def keygen(p: Params, seed: int, cloud_seed: int | None = None) -> Keys:
    """Secret keys from `seed`; bootstrapping and key-switching keys from
    `cloud_seed` (defaults to `seed`)."""
    cs = seed if cloud_seed is None else cloud_seed
    s, K = secret_keygen(p, seed)
    bsk = np.zeros(p.bsk_words, np.uint32)
    ksk = np.zeros(p.ksk_words, np.uint32)
    lib().or_bsk_keygen(ctypes.byref(p.c()), cs, _ptr(s), _ptr(K), _ptr(bsk))
    lib().or_ksk_keygen(ctypes.byref(p.c()), cs, _ptr(s), _ptr(K), _ptr(ksk))
    return Keys(p, s, K, bsk.reshape(p.n, 2 * p.l, 2, p.N),
                ksk.reshape(p.N, p.t, 1 << p.basebit, p.n + 1))


# ------------------------------------------------------------ enc / dec ---
def encrypt(p: Params, s: np.ndarray, bit: int, seed: int, ctr: int) -> np.ndarray:
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_encrypt(ctypes.byref(p.c()), _ptr(_u32(s)), int(bit), seed, ctr, _ptr(out))
    return out


def phase(p: Params, s: np.ndarray, c: np.ndarray) -> int:
    return int(lib().or_phase(ctypes.byref(p.c()), _ptr(_u32(s)), _ptr(_u32(c))))


def decrypt(p: Params, s: np.ndarray, c: np.ndarray) -> int:
    return int(lib().or_decrypt(ctypes.byref(p.c()), _ptr(_u32(s)), _ptr(_u32(c))))


# --------------------------------------------------------- primitives ---
def poly_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a, b = _u32(a), _u32(b)
    out = np.zeros(len(a), np.uint32)
    lib().or_poly_mul(len(a), _ptr(a), _ptr(b), _ptr(out))
    return out


def decompose(p: Params, x: int) -> list[int]:
    d = np.zeros(p.l, np.int32)
    lib().or_decompose(ctypes.byref(p.c()), x & 0xFFFFFFFF, _ptr(d))
    return [int(v) for v in d]


def modswitch(x: int, N: int) -> int:
    return int(lib().or_modswitch(x & 0xFFFFFFFF, N))


def gate_lincomb(p: Params, op, c1, c2) -> np.ndarray:
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_gate_lincomb(ctypes.byref(p.c()), _op(op), _ptr(_u32(c1)), _ptr(_u32(c2)), _ptr(out))
    return out


def blind_rotate(p: Params, bsk: np.ndarray, abar, bbar: int, mu: int = MU) -> np.ndarray:
    acc = np.zeros(2 * p.N, np.uint32)
    lib().or_blind_rotate(ctypes.byref(p.c()), _ptr(_u32(bsk)), _ptr(_u32(abar)), bbar, mu,
                          _ptr(acc))
    return acc.reshape(2, p.N)


def sample_extract(p: Params, acc: np.ndarray) -> np.ndarray:
    big = np.zeros(p.N + 1, np.uint32)
    lib().or_sample_extract(ctypes.byref(p.c()), _ptr(_u32(acc)), _ptr(big))
    return big


def key_switch(p: Params, ksk: np.ndarray, big: np.ndarray) -> np.ndarray:
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_key_switch(ctypes.byref(p.c()), _ptr(_u32(ksk)), _ptr(_u32(big)), _ptr(out))
    return out


def bootstrap(keys: Keys, c: np.ndarray) -> np.ndarray:
    p = keys.params
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_bootstrap(ctypes.byref(p.c()), _ptr(keys.bsk), _ptr(keys.ksk), _ptr(_u32(c)), _ptr(out))
    return out


def _op(op) -> int:
    return GATE_ID[op] if isinstance(op, str) else int(op)


def gate(keys: Keys, op, c1, c2) -> np.ndarray:
    p = keys.params
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_gate(ctypes.byref(p.c()), _ptr(keys.bsk), _ptr(keys.ksk), _op(op),
                  _ptr(_u32(c1)), _ptr(_u32(c2)), _ptr(out))
    return out


def gates(keys: Keys, ops, c1, c2, threads: int | None = None) -> np.ndarray:
    """Many independent gates, spread over POSIX threads inside the C oracle."""
    p = keys.params
    ops = np.ascontiguousarray([_op(o) for o in ops], dtype=np.int32)
    c1 = _u32(c1).reshape(-1, p.n + 1)
    c2 = _u32(c2).reshape(-1, p.n + 1)
    out = np.zeros_like(c1)
    thr = threads or os.cpu_count() or 1
    lib().or_gates_threaded(ctypes.byref(p.c()), _ptr(keys.bsk), _ptr(keys.ksk), _ptr(ops),
                            _ptr(c1), _ptr(c2), _ptr(out), len(ops), thr)
    return out


def muxes(keys: Keys, a, b, c, threads: int | None = None) -> np.ndarray:
    """Many independent MUX gates (a ? b : c), spread over POSIX threads."""
    p = keys.params
    a = _u32(a).reshape(-1, p.n + 1)
    b = _u32(b).reshape(-1, p.n + 1)
    c = _u32(c).reshape(-1, p.n + 1)
    out = np.zeros_like(a)
    thr = threads or os.cpu_count() or 1
    lib().or_muxes_threaded(ctypes.byref(p.c()), _ptr(keys.bsk), _ptr(keys.ksk), _ptr(a), _ptr(b),
                            _ptr(c), _ptr(out), len(a), thr)
    return out


def mux(keys: Keys, a, b, c) -> np.ndarray:
    p = keys.params
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_mux(ctypes.byref(p.c()), _ptr(keys.bsk), _ptr(keys.ksk), _ptr(_u32(a)),
                 _ptr(_u32(b)), _ptr(_u32(c)), _ptr(out))
    return out


def constant(p: Params, bit: int) -> np.ndarray:
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_constant(ctypes.byref(p.c()), int(bit), _ptr(out))
    return out


def not_(p: Params, c) -> np.ndarray:
    out = np.zeros(p.n + 1, np.uint32)
    lib().or_not(ctypes.byref(p.c()), _ptr(_u32(c)), _ptr(out))
    return out
