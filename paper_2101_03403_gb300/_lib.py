"""ctypes binding of libcryptoemu.so (argument marshalling only).

Every function keeps the name of the C entry point it wraps (see
include/cryptoemu.h).  Host buffers are numpy arrays; device buffers are
torch CUDA tensors (or raw device addresses as ints); streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` ints, or None for the
context's stream.  All computation happens inside the library: if the shared
library is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

LWE_N = 500
LWE_WORDS = 501
RING_N = 1024
GATES = ["NAND", "AND", "OR", "XOR", "NOR", "XNOR", "ANDNY", "ANDYN", "ORNY", "ORYN"]
GATE_ID = {g: i for i, g in enumerate(GATES)}

STATUS = {0: "CE_OK", -1: "CE_EINVAL", -2: "CE_ENOMEM", -3: "CE_EADMIT", -4: "CE_ETIMEOUT",
          -5: "CE_ECUDA", -6: "CE_ENOTFOUND"}


class CeError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


_L = None


def lib() -> ctypes.CDLL:
    """Load the library (it must have been built: ``__graft_entry__.build()``)."""
    global _L
    if _L is not None:
        return _L
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(_build.LIB)
    vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "ce_secret_keygen": (i32, [u64, pp, ctypes.POINTER(sz)]),
        "ce_cloud_keygen": (i32, [vp, u64, pp, ctypes.POINTER(sz)]),
        "ce_free": (None, [vp]),
        "ce_encrypt_bit": (i32, [vp, i32, u64, u64, vp]),
        "ce_decrypt_bit": (i32, [vp, vp]),
        "ce_create": (i32, [pp, i32, u64, vp]),
        "ce_destroy": (None, [vp]),
        "ce_last_error": (ctypes.c_char_p, []),
        "ce_device_alloc_count": (None, [ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "ce_client_admit": (i32, [vp, vp, sz, ctypes.POINTER(i32)]),
        "ce_client_evict": (i32, [vp, i32]),
        "ce_client_footprint_bytes": (u64, []),
        "ce_gate": (i32, [vp, i32, i32, vp, vp, vp]),
        "ce_gates_batch": (i32, [vp, i32, vp, vp, vp, vp, sz]),
        "ce_gates_batch_device": (i32, [vp, i32, vp, vp, vp, vp, sz, vp]),
        "ce_gates_batch_device_noalloc": (i32, [vp, i32, vp, vp, vp, vp, sz, vp]),
        "ce_mux_batch_device": (i32, [vp, i32, vp, vp, vp, vp, sz, vp]),
        "ce_negacyclic_mul_device": (i32, [vp, vp, vp, vp, sz, vp]),
        "ce_set_blind_rotate_config": (i32, [vp, i32, i32]),
        "ce_set_level_batching": (i32, [vp, i32]),
        "ce_set_instruction_circuits": (i32, [vp, i32]),
        "ce_blind_rotate_plan": (i32, [i32, i32, i32, ctypes.POINTER(i32)]),
        "ce_set_keyswitch_config": (i32, [vp, i32]),
        "ce_set_external_product_form": (i32, [vp, i32]),
        "ce_selftest_device_wait": (i32, [vp, ctypes.c_uint64]),
        "ce_last_launch_count": (i32, [vp]),
        "ce_synchronize": (i32, [vp]),
        "ce_profile_enable": (i32, [vp, i32]),
        "ce_unit_info": (i32, [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ce_unit_netlist": (i32, [i32, i32, i32, vp, sz, ctypes.POINTER(sz)]),
        "ce_unit_eval_device": (i32, [vp, i32, i32, i32, vp, vp, sz, vp]),
        "ce_unit_eval_device_width": (i32, [vp, i32, i32, i32, i32, vp, vp, sz, vp]),
        "ce_unit_eval": (i32, [vp, i32, i32, i32, i32, vp, vp, sz]),
        "ce_set_unit_graphs": (i32, [vp, i32]),
        "ce_reg_write": (i32, [vp, i32, i32, vp]),
        "ce_reg_read": (i32, [vp, i32, i32, vp]),
        "ce_flags_read": (i32, [vp, i32, vp]),
        "ce_exec": (i32, [vp, i32, vp, sz, u64]),
        "ce_exec_multi": (i32, [vp, sz, vp, vp, vp, u64]),
        "ce_exec_branching": (i32, [vp, i32, vp, sz, vp, vp, u64, u64, ctypes.POINTER(u64)]),
        "ce_server_create": (i32, [vp, i32, pp]),
        "ce_server_submit": (i32, [vp, i32, vp, ctypes.POINTER(u64)]),
        "ce_server_poll": (i32, [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(u64),
                                 ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "ce_server_wait": (i32, [vp, u64, u64]),
        "ce_server_stats": (i32, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                  ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "ce_server_destroy": (None, [vp]),
        "ce_autotune": (i32, [vp, i32, vp, vp, i32, ctypes.POINTER(i32)]),
        "ce_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), i32]),
        "ce_trace_enable": (i32, [vp, i32, sz]),
        "ce_probe_int_pipes": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "ce_trace_read": (i32, [vp, vp, sz, ctypes.POINTER(sz), ctypes.POINTER(u64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _L = L
    return L


def header_functions() -> list[str]:
    """Names of the functions declared in include/cryptoemu.h."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "cryptoemu.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ce_[a-z0-9_]+)\s*\(", text)))


def _check(code: int, where: str):
    if code != 0:
        raise CeError(code, where, (lib().ce_last_error() or b"").decode())


def _addr(x) -> int | None:
    """Device address of a torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _host(a, dtype=np.uint32) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------- client ---
class SecretKey:
    def __init__(self, ptr: int, nbytes: int):
        self.ptr, self.nbytes = ptr, nbytes

    def words(self) -> np.ndarray:
        return np.ctypeslib.as_array((ctypes.c_uint32 * (self.nbytes // 4)).from_address(self.ptr))

    @property
    def s(self) -> np.ndarray:
        return self.words()[2:2 + LWE_N].copy()

    @property
    def K(self) -> np.ndarray:
        return self.words()[2 + LWE_N:2 + LWE_N + RING_N].copy()

    def __del__(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.ce_free(self.ptr)
            self.ptr = None


class CloudKey:
    def __init__(self, ptr: int, nbytes: int):
        self.ptr, self.nbytes = ptr, nbytes

    def words(self) -> np.ndarray:
        return np.ctypeslib.as_array((ctypes.c_uint32 * (self.nbytes // 4)).from_address(self.ptr))

    def bsk(self) -> np.ndarray:
        return self.words()[2:2 + 500 * 6 * 2 * 1024].reshape(500, 6, 2, 1024)

    def ksk(self) -> np.ndarray:
        off = 2 + 500 * 6 * 2 * 1024
        return self.words()[off:].reshape(1024, 8, 4, 501)

    def __del__(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.ce_free(self.ptr)
            self.ptr = None


def ce_secret_keygen(seed: int) -> SecretKey:
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    _check(lib().ce_secret_keygen(seed, ctypes.byref(p), ctypes.byref(n)), "ce_secret_keygen")
    return SecretKey(p.value, n.value)


def ce_cloud_keygen(secret: SecretKey, seed: int) -> CloudKey:
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    _check(lib().ce_cloud_keygen(secret.ptr, seed, ctypes.byref(p), ctypes.byref(n)),
           "ce_cloud_keygen")
    return CloudKey(p.value, n.value)


def ce_encrypt_bit(secret: SecretKey, bit: int, seed: int, ctr: int) -> np.ndarray:
    out = np.zeros(LWE_WORDS, np.uint32)
    _check(lib().ce_encrypt_bit(secret.ptr, int(bit), seed, ctr, out.ctypes.data),
           "ce_encrypt_bit")
    return out


def ce_decrypt_bit(secret: SecretKey, c) -> int:
    c = _host(c)
    r = lib().ce_decrypt_bit(secret.ptr, c.ctypes.data)
    if r < 0:
        _check(r, "ce_decrypt_bit")
    return r


# ------------------------------------------------------------ context ---
class Context:
    def __init__(self, ptr: int):
        self.ptr = ptr

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.ce_destroy(self.ptr)
        self.ptr = None


def ce_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None) -> Context:
    p = ctypes.c_void_p()
    _check(lib().ce_create(ctypes.byref(p), device, hbm_budget_bytes, _stream(stream)),
           "ce_create")
    return Context(p.value)


def ce_destroy(ctx: Context):
    ctx.close()


def ce_last_error() -> str:
    return (lib().ce_last_error() or b"").decode()


def ce_client_admit(ctx: Context, cloud: CloudKey) -> int:
    cid = ctypes.c_int()
    _check(lib().ce_client_admit(ctx.ptr, cloud.ptr, cloud.nbytes, ctypes.byref(cid)),
           "ce_client_admit")
    return cid.value


def ce_client_evict(ctx: Context, client: int):
    _check(lib().ce_client_evict(ctx.ptr, client), "ce_client_evict")


def ce_client_footprint_bytes() -> int:
    return int(lib().ce_client_footprint_bytes())


def _op(op) -> int:
    return GATE_ID[op] if isinstance(op, str) else int(op)


def ce_gate(ctx: Context, client: int, op, a, b) -> np.ndarray:
    a, b = _host(a), _host(b)
    out = np.zeros(LWE_WORDS, np.uint32)
    _check(lib().ce_gate(ctx.ptr, client, _op(op), a.ctypes.data, b.ctypes.data, out.ctypes.data),
           "ce_gate")
    return out


def ce_gates_batch(ctx: Context, client: int, ops, a, b, out=None) -> np.ndarray:
    ops = _host([_op(o) for o in ops] if not isinstance(ops, np.ndarray) else ops, np.uint8)
    a = _host(a).reshape(-1, LWE_WORDS)
    b = _host(b).reshape(-1, LWE_WORDS)
    n = len(ops)
    if out is None:
        out = np.empty((n, LWE_WORDS), np.uint32)
    _check(lib().ce_gates_batch(ctx.ptr, client, ops.ctypes.data, a.ctypes.data, b.ctypes.data,
                                out.ctypes.data, n), "ce_gates_batch")
    return out


def ce_gates_batch_device(ctx: Context, client: int, d_ops, d_a, d_b, d_out, n: int,
                          stream=None):
    _check(lib().ce_gates_batch_device(ctx.ptr, client, _addr(d_ops), _addr(d_a), _addr(d_b),
                                       _addr(d_out), n, _stream(stream)), "ce_gates_batch_device")


def ce_gates_batch_device_noalloc(ctx: Context, client: int, d_ops, d_a, d_b, d_out, n: int,
                                  stream=None):
    """ce_gates_batch_device without any device allocation (at most 256 gates;
    scratch is a fixed area of the library's device image shared by all calls)."""
    _check(lib().ce_gates_batch_device_noalloc(ctx.ptr, client, _addr(d_ops), _addr(d_a),
                                               _addr(d_b), _addr(d_out), n, _stream(stream)),
           "ce_gates_batch_device_noalloc")


def ce_mux_batch_device(ctx: Context, client: int, d_a, d_b, d_c, d_out, n: int, stream=None):
    _check(lib().ce_mux_batch_device(ctx.ptr, client, _addr(d_a), _addr(d_b), _addr(d_c),
                                     _addr(d_out), n, _stream(stream)), "ce_mux_batch_device")


def ce_negacyclic_mul_device(ctx: Context, d_d, d_k, d_out, n: int, stream=None):
    _check(lib().ce_negacyclic_mul_device(ctx.ptr, _addr(d_d), _addr(d_k), _addr(d_out), n,
                                          _stream(stream)), "ce_negacyclic_mul_device")


def ce_set_blind_rotate_config(ctx: Context, gates_per_block: int, blocks_per_sm: int = 0):
    _check(lib().ce_set_blind_rotate_config(ctx.ptr, gates_per_block, blocks_per_sm),
           "ce_set_blind_rotate_config")


def ce_blind_rotate_plan(n_jobs: int, gates_per_block: int, blocks: int) -> dict:
    """Launches of a blind rotation of n_jobs gates: {"main_jobs", "tail_jobs",
    "tail_shape", "tail_blocks"} (tail_jobs 0: one launch)."""
    out = (ctypes.c_int * 4)()
    _check(lib().ce_blind_rotate_plan(n_jobs, gates_per_block, blocks, out),
           "ce_blind_rotate_plan")
    return {"main_jobs": out[0], "tail_jobs": out[1], "tail_shape": out[2], "tail_blocks": out[3]}


def ce_set_instruction_circuits(ctx: Context, low_latency: bool):
    """False: ADD / SUB / MUL / UDIV instructions on the paper's circuits
    (default); True: on ADD_MUX / SUB_MUX / MUL_TREE / UDIV_MUX (same
    semantics, fewer levels)."""
    _check(lib().ce_set_instruction_circuits(ctx.ptr, 1 if low_latency else 0),
           "ce_set_instruction_circuits")


def ce_set_level_batching(ctx: Context, on: bool):
    """True: one batched launch per level step (default); False: one launch per
    gate and step (comparison mode, bit-identical results)."""
    _check(lib().ce_set_level_batching(ctx.ptr, 1 if on else 0), "ce_set_level_batching")


def ce_set_keyswitch_config(ctx: Context, engine: int):
    """0 automatic, 1 CUDA cores, 2 tensor cores (single-client launches)."""
    _check(lib().ce_set_keyswitch_config(ctx.ptr, engine), "ce_set_keyswitch_config")


def ce_set_external_product_form(ctx: Context, form: int):
    """0 transform form (CUDA cores), 1 Toeplitz form (tensor cores)."""
    _check(lib().ce_set_external_product_form(ctx.ptr, form), "ce_set_external_product_form")


def ce_selftest_device_wait(ctx: Context, limit_ns: int):
    """Launch a bounded device wait that must expire (ce_synchronize then
    raises CE_ETIMEOUT)."""
    _check(lib().ce_selftest_device_wait(ctx.ptr, limit_ns), "ce_selftest_device_wait")


def ce_device_alloc_count() -> tuple[int, int]:
    """(device allocations, device frees) the library has made in this process."""
    a, f = ctypes.c_uint64(), ctypes.c_uint64()
    lib().ce_device_alloc_count(ctypes.byref(a), ctypes.byref(f))
    return a.value, f.value


def ce_last_launch_count(ctx: Context) -> int:
    return int(lib().ce_last_launch_count(ctx.ptr))


def ce_synchronize(ctx: Context):
    _check(lib().ce_synchronize(ctx.ptr), "ce_synchronize")


# ce_trace_rec: op, neg[3], client, tick, index, pad, in[3][501], out[501]
TRACE_DTYPE = np.dtype([("op", "<i4"), ("neg", "<i4", 3), ("client", "<i4"), ("tick", "<u4"),
                        ("index", "<u4"), ("pad", "<u4"), ("inp", "<u4", (3, LWE_WORDS)),
                        ("out", "<u4", LWE_WORDS)])
assert TRACE_DTYPE.itemsize == 8048


def ce_probe_int_pipes(ctx: Context) -> dict:
    """Measured lane operations per clock per SM of the integer multiply-add
    pipe: 32-bit multiply-add, high-half multiply, 64-bit-result multiply-add."""
    out = (ctypes.c_double * 3)()
    _check(lib().ce_probe_int_pipes(ctx.ptr, out), "ce_probe_int_pipes")
    return {"imad": out[0], "imad_hi": out[1], "imad_wide": out[2]}


def ce_trace_enable(ctx: Context, per_tick: int, cap: int = 4096):
    """Record up to per_tick gates of every engine tick (0 stops tracing)."""
    _check(lib().ce_trace_enable(ctx.ptr, per_tick, cap), "ce_trace_enable")


def ce_trace_read(ctx: Context, cap: int = 4096):
    """(records as a TRACE_DTYPE array, records made since the last read)."""
    out = np.zeros(cap, TRACE_DTYPE)
    n, seen = ctypes.c_size_t(), ctypes.c_uint64()
    _check(lib().ce_trace_read(ctx.ptr, out.ctypes.data, cap, ctypes.byref(n), ctypes.byref(seen)),
           "ce_trace_read")
    return out[:n.value], int(seen.value)


KERNEL_KINDS = ["lincomb_modswitch", "blind_rotate", "extract_keyswitch", "external_product_mma"]


def ce_profile_enable(ctx: Context, on: bool = True):
    _check(lib().ce_profile_enable(ctx.ptr, int(on)), "ce_profile_enable")


def ce_profile_read(ctx: Context) -> dict:
    k = len(KERNEL_KINDS)
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_int * k)()
    _check(lib().ce_profile_read(ctx.ptr, ms, cnt, k), "ce_profile_read")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(KERNEL_KINDS)}


UNITS = ["ADD", "ADD_RIPPLE", "SUB", "AND", "ORR", "LSL", "MUL", "UDIV", "CMP", "CSEL", "LSR",
         "ASR", "EOR", "ORN", "ADDS", "SUBS", "SMULL", "UMULL", "ADD_MUX", "SUB_MUX",
         "MUL_TREE", "UDIV_MUX"]
UNIT_ID = {u: i for i, u in enumerate(UNITS)}


def _unit(u) -> int:
    return UNIT_ID[u] if isinstance(u, str) else int(u)


def ce_unit_info(unit, cond: int = 0, width: int = 16) -> dict:
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().ce_unit_info(_unit(unit), cond, width, *[ctypes.byref(x) for x in v]),
           "ce_unit_info")
    return dict(zip(["n_inputs", "n_outputs", "n_gates", "n_bootstraps", "depth"],
                    [x.value for x in v]))


def ce_unit_netlist(unit, cond: int = 0, width: int = 16) -> dict:
    """The library's netlist: gates as (op, a, b, c, out, level) with refs
    (wire, negated), ordered by level."""
    used = ctypes.c_size_t()
    _check(lib().ce_unit_netlist(_unit(unit), cond, width, None, 0, ctypes.byref(used)),
           "ce_unit_netlist")
    buf = np.zeros(used.value, np.int32)
    _check(lib().ce_unit_netlist(_unit(unit), cond, width, buf.ctypes.data, used.value,
                                 ctypes.byref(used)), "ce_unit_netlist")
    n_in, n_wires, depth, n_g, n_o = (int(x) for x in buf[:5])
    g = buf[5:5 + 9 * n_g].reshape(n_g, 9)
    gates = []
    for r in g:
        op = int(r[0])
        c = (int(r[5]), bool(r[6])) if op == 10 else (-1, False)
        gates.append((op, (int(r[1]), bool(r[2])), (int(r[3]), bool(r[4])), c, int(r[7]),
                      int(r[8])))
    o = buf[5 + 9 * n_g:].reshape(n_o, 2)
    return {"n_inputs": n_in, "n_wires": n_wires, "depth": depth, "gates": gates,
            "outputs": [(int(x), bool(y)) for x, y in o]}


OPCODES = ["ADD", "SUB", "AND", "ORR", "LSL", "LSL_IMM", "MUL", "UDIV", "CMP", "CSEL", "MOV",
           "MOV_IMM", "LSR", "ASR", "LSR_IMM", "ASR_IMM", "EOR", "ORN", "MVN", "AND_IMM", "ORR_IMM",
           "EOR_IMM", "BFC", "BFI", "RBIT", "REV", "ADDS", "SUBS", "SMULH", "UMULH", "BCOND",
           "B"]
OPCODE_ID = {o: i for i, o in enumerate(OPCODES)}
CONDS = ["EQ", "NE", "CS", "CC", "MI", "PL", "VS", "VC", "HI", "LS", "GE", "LT", "GT", "LE"]


class Insn(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint8), ("rd", ctypes.c_uint8), ("rn", ctypes.c_uint8),
                ("rm", ctypes.c_uint8), ("imm", ctypes.c_uint8), ("cond", ctypes.c_uint8)]


def insn(op, rd=0, rn=0, rm=0, imm=0, cond=0) -> Insn:
    op = OPCODE_ID[op] if isinstance(op, str) else int(op)
    cond = CONDS.index(cond) if isinstance(cond, str) else int(cond)
    return Insn(op, rd, rn, rm, imm, cond)


def ce_unit_eval_device(ctx: Context, client: int, unit, d_in, d_out, n: int, cond: int = 0,
                        stream=None):
    _check(lib().ce_unit_eval_device(ctx.ptr, client, _unit(unit), cond, _addr(d_in), _addr(d_out),
                                     n, _stream(stream)), "ce_unit_eval_device")


def ce_unit_eval_device_width(ctx: Context, client: int, unit, width: int, d_in, d_out, n: int,
                              cond: int = 0, stream=None):
    _check(lib().ce_unit_eval_device_width(ctx.ptr, client, _unit(unit), cond, width, _addr(d_in),
                                           _addr(d_out), n, _stream(stream)),
           "ce_unit_eval_device_width")


def ce_unit_eval(ctx: Context, client: int, unit, inp, out=None, cond: int = 0, width: int = 16):
    """Host buffers: inp [n][n_inputs][501] uint32 (numpy, e.g. a view of pinned
    memory), out [n][n_outputs][501] (allocated if None)."""
    inp = _host(inp)
    info = ce_unit_info(unit, cond, width)
    n = inp.size // (info["n_inputs"] * LWE_WORDS)
    if out is None:
        out = np.empty((n, info["n_outputs"], LWE_WORDS), np.uint32)
    _check(lib().ce_unit_eval(ctx.ptr, client, _unit(unit), cond, width, inp.ctypes.data,
                              out.ctypes.data, n), "ce_unit_eval")
    return out


def ce_set_unit_graphs(ctx: Context, on: bool):
    _check(lib().ce_set_unit_graphs(ctx.ptr, int(on)), "ce_set_unit_graphs")


def ce_reg_write(ctx: Context, client: int, reg: int, bits):
    bits = _host(bits).reshape(16, LWE_WORDS)
    _check(lib().ce_reg_write(ctx.ptr, client, reg, bits.ctypes.data), "ce_reg_write")


def ce_reg_read(ctx: Context, client: int, reg: int) -> np.ndarray:
    out = np.zeros((16, LWE_WORDS), np.uint32)
    _check(lib().ce_reg_read(ctx.ptr, client, reg, out.ctypes.data), "ce_reg_read")
    return out


def ce_flags_read(ctx: Context, client: int) -> np.ndarray:
    out = np.zeros((4, LWE_WORDS), np.uint32)
    _check(lib().ce_flags_read(ctx.ptr, client, out.ctypes.data), "ce_flags_read")
    return out


def _prog(prog):
    arr = (Insn * max(len(prog), 1))(*prog)
    return arr, len(prog)


def ce_exec(ctx: Context, client: int, prog, timeout_ns: int = 0):
    arr, n = _prog(prog)
    _check(lib().ce_exec(ctx.ptr, client, ctypes.addressof(arr), n, timeout_ns), "ce_exec")


def ce_exec_multi(ctx: Context, clients, progs, timeout_ns: int = 0):
    arrs = [_prog(p) for p in progs]
    cl = (ctypes.c_int * len(clients))(*clients)
    ptrs = (ctypes.c_void_p * len(progs))(*[ctypes.addressof(a) for a, _ in arrs])
    lens = (ctypes.c_size_t * len(progs))(*[n for _, n in arrs])
    _check(lib().ce_exec_multi(ctx.ptr, len(progs), cl, ptrs, lens, timeout_ns), "ce_exec_multi")


BRANCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint8,
                             ctypes.c_void_p)


def ce_exec_branching(ctx: Context, client: int, prog, decide, max_steps: int = 0,
                      timeout_ns: int = 0) -> int:
    """Run a program with branches; decide(client, cond, nzcv[4][501]) -> bool
    is the key owner's branch decision.  Returns the executed step count."""
    arr, n = _prog(prog)
    err = []

    def cb(_user, client_, cond, p):
        try:
            nz = np.ctypeslib.as_array((ctypes.c_uint32 * (4 * LWE_WORDS)).from_address(p))
            return 1 if decide(client_, int(cond), nz.reshape(4, LWE_WORDS).copy()) else 0
        except Exception as e:            # surfaced after the call
            err.append(e)
            return -1

    fn = BRANCH_FN(cb)
    steps = ctypes.c_uint64()
    code = lib().ce_exec_branching(ctx.ptr, client, ctypes.addressof(arr), n, fn, None, max_steps,
                                   timeout_ns, ctypes.byref(steps))
    if err:
        raise err[0]
    _check(code, "ce_exec_branching")
    return steps.value


class Server:
    def __init__(self, ptr: int):
        self.ptr = ptr

    def close(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.ce_server_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        self.close()


def ce_server_create(ctx: Context, max_inflight: int = 0) -> Server:
    p = ctypes.c_void_p()
    _check(lib().ce_server_create(ctx.ptr, max_inflight, ctypes.byref(p)), "ce_server_create")
    return Server(p.value)


def ce_server_submit(srv: Server, client: int, ins: Insn) -> int:
    t = ctypes.c_uint64()
    _check(lib().ce_server_submit(srv.ptr, client, ctypes.byref(ins), ctypes.byref(t)),
           "ce_server_submit")
    return t.value


def ce_server_poll(srv: Server, ticket: int) -> dict:
    d = ctypes.c_int()
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().ce_server_poll(srv.ptr, ticket, ctypes.byref(d), ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(c)), "ce_server_poll")
    return {"done": bool(d.value), "submit_ns": a.value, "start_ns": b.value, "done_ns": c.value}


def ce_server_wait(srv: Server, ticket: int, timeout_ns: int = 0):
    _check(lib().ce_server_wait(srv.ptr, ticket, timeout_ns), "ce_server_wait")


def ce_server_stats(srv: Server) -> dict:
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(lib().ce_server_stats(srv.ptr, *[ctypes.byref(x) for x in v]), "ce_server_stats")
    return dict(zip(["ticks", "bootstraps", "queued", "running"], [x.value for x in v]))


def ce_server_destroy(srv: Server):
    srv.close()


def ce_autotune(ctx: Context, client: int) -> dict:
    """Measure and install the fastest blind-rotation shape per batch size."""
    jobs = (ctypes.c_int * 32)()
    g = (ctypes.c_int * 32)()
    n = ctypes.c_int()
    _check(lib().ce_autotune(ctx.ptr, client, jobs, g, 32, ctypes.byref(n)), "ce_autotune")
    return {int(jobs[i]): int(g[i]) for i in range(n.value)}
