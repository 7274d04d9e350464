"""ctypes binding of ``liblec_es.so`` -- argument marshalling only.

Every function has the name of the C entry point it calls (``include/lec_es.h``)
and does no computation of its own: each step of exact simulation runs in the
library's front end and CUDA kernels.  PyTorch appears only to provide device
memory (the context arena) and the CUDA stream.

The library must be present: ``load()`` raises ``LecEsError`` if it is
missing or cannot be loaded; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblec_es.so")

# status codes (lec_es_status)
OK, EINVAL, ETOOBIG, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ECANCELLED, EDEVICE_WAIT, EJIT, ENOTFOUND = range(11)
EQUIVALENT, NONEQUIVALENT, UNDECIDED = 0, 1, 2
TIER_AUTO, TIER_INTERP, TIER_JIT, TIER_SPILL = 0, 1, 2, 3
ORDER_AUTO, ORDER_DFS, ORDER_VAR, ORDER_LEVEL, ORDER_GREEDY = 0, 1, 2, 3, 4
NO_CEX = (1 << 64) - 1

# every entry point declared in include/lec_es.h
EXPORTS = [
    "lec_es_create", "lec_es_destroy", "lec_es_strerror", "lec_es_compile", "lec_es_check",
    "lec_es_check_ex", "lec_es_prepare", "lec_es_run_async", "lec_es_plan_result", "lec_es_plan_info",
    "lec_es_plan_free", "lec_es_truth_tables", "lec_es_truth_tables_ex", "lec_es_batch", "lec_es_batch_prepare",
    "lec_es_batch_run_async", "lec_es_batch_results", "lec_es_batch_free", "lec_es_submit", "lec_es_poll",
    "lec_es_submit_many", "lec_es_wait", "lec_es_cancel", "lec_es_server_config", "lec_es_lop3_peak", "lec_es_jit_compile",
    "lec_es_check_noalloc", "lec_es_batch_info", "lec_es_signatures", "lec_es_match_pairs",
    "lec_es_codegen_version", "lec_es_cost_fit", "lec_es_cost_model", "lec_es_cost_predict", "lec_es_sweep",
]


class LecEsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _strerror(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


class lec_es_miter(ctypes.Structure):
    _fields_ = [("num_pis", ctypes.c_uint32), ("num_ands", ctypes.c_uint32),
                ("fanins", ctypes.POINTER(ctypes.c_uint32)), ("out_lit", ctypes.c_uint32)]


class lec_es_result(ctypes.Structure):
    _fields_ = [("verdict", ctypes.c_int), ("support_n", ctypes.c_uint32), ("cex", ctypes.c_uint64),
                ("support", ctypes.c_uint32 * 64), ("cone_ands", ctypes.c_uint32),
                ("num_slots", ctypes.c_uint32), ("tier", ctypes.c_uint32), ("order", ctypes.c_uint32),
                ("words_checked", ctypes.c_uint64), ("device_ms", ctypes.c_double),
                ("host_ms", ctypes.c_double), ("jit_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]

    @property
    def cex_or_none(self) -> Optional[int]:
        return None if self.cex == NO_CEX else int(self.cex)

    def support_list(self) -> List[int]:
        return [int(self.support[k]) for k in range(self.support_n)]


class lec_es_options(ctypes.Structure):
    _fields_ = [("word_begin", ctypes.c_uint64), ("word_end", ctypes.c_uint64), ("tier", ctypes.c_uint32),
                ("order", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("grid_blocks", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("tile_granularity", ctypes.c_uint32), ("stage_records", ctypes.c_uint32)]


class lec_es_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("max_pis", ctypes.c_uint32), ("timeout_s", ctypes.c_double),
                ("jit_cache_dir", ctypes.c_char_p)]


class lec_es_program_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("support", ctypes.c_uint32 * 64), ("cone_ands", ctypes.c_uint32),
                ("num_slots", ctypes.c_uint32), ("out_slot", ctypes.c_uint32), ("out_compl", ctypes.c_uint32),
                ("order", ctypes.c_uint32), ("num_records", ctypes.c_uint64), ("hash", ctypes.c_uint64),
                ("num_luts", ctypes.c_uint32), ("lut_live", ctypes.c_uint32), ("lop3_per_pass", ctypes.c_double),
                ("interp_step", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class lec_es_cost_coeffs(ctypes.Structure):
    _fields_ = [("a_ms", ctypes.c_double), ("c_ms", ctypes.c_double), ("alpha_ms", ctypes.c_double),
                ("samples", ctypes.c_uint64)]


class lec_es_cost(ctypes.Structure):
    _fields_ = [("interp_ms", ctypes.c_double), ("jit_ms", ctypes.c_double), ("jit_compile_ms", ctypes.c_double),
                ("paper_cpu_s", ctypes.c_double), ("gates", ctypes.c_uint32), ("n", ctypes.c_uint32),
                ("num_luts", ctypes.c_uint32), ("tier", ctypes.c_uint32), ("gpu_offload", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


class lec_es_sweep_options(ctypes.Structure):
    _fields_ = [("sim_words", ctypes.c_uint32), ("max_rounds", ctypes.c_uint32), ("max_leaves", ctypes.c_uint32),
                ("max_nodes", ctypes.c_uint32), ("final_max_pis", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class lec_es_sweep_result(ctypes.Structure):
    _fields_ = [("verdict", ctypes.c_int), ("rounds", ctypes.c_uint32), ("pairs_checked", ctypes.c_uint64),
                ("pairs_proven", ctypes.c_uint64), ("pairs_refuted", ctypes.c_uint64),
                ("pairs_skipped", ctypes.c_uint64), ("ands_initial", ctypes.c_uint32),
                ("ands_final", ctypes.c_uint32), ("final_support", ctypes.c_uint32), ("decided_by", ctypes.c_uint32),
                ("sim_ms", ctypes.c_double), ("es_ms", ctypes.c_double), ("host_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("rounds_reused", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


_lib: Optional[ctypes.CDLL] = None
_P = ctypes.c_void_p
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def load() -> ctypes.CDLL:
    """Load liblec_es.so (raises LecEsError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LecEsError(ECUDA, f"{LIB_PATH} is missing; run paper_2512_06627_b300.build")
    try:
        lib = ctypes.CDLL(LIB_PATH)
    except OSError as e:
        raise LecEsError(ECUDA, f"cannot load {LIB_PATH}: {e}") from e
    R = ctypes.POINTER(lec_es_result)
    M = ctypes.POINTER(lec_es_miter)
    O = ctypes.POINTER(lec_es_options)
    sig = {
        "lec_es_create": ([ctypes.POINTER(_P), ctypes.POINTER(lec_es_config)], ctypes.c_int),
        "lec_es_destroy": ([_P], None),
        "lec_es_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "lec_es_compile": ([M, ctypes.c_uint32, ctypes.POINTER(lec_es_program_info), _u64p, ctypes.c_uint64],
                           ctypes.c_int),
        "lec_es_check": ([_P, M, R], ctypes.c_int),
        "lec_es_check_ex": ([_P, M, O, R], ctypes.c_int),
        "lec_es_prepare": ([_P, M, O, ctypes.POINTER(_P)], ctypes.c_int),
        "lec_es_run_async": ([_P, _P, O], ctypes.c_int),
        "lec_es_plan_result": ([_P, _P, R], ctypes.c_int),
        "lec_es_plan_info": ([_P, ctypes.POINTER(lec_es_program_info)], ctypes.c_int),
        "lec_es_plan_free": ([_P, _P], None),
        "lec_es_truth_tables": ([_P, M, ctypes.c_uint64, ctypes.c_uint64, _u32p, _u64p], ctypes.c_int),
        "lec_es_batch": ([_P, M, ctypes.c_size_t, R], ctypes.c_int),
        "lec_es_batch_prepare": ([_P, M, ctypes.c_size_t, O, ctypes.POINTER(_P)], ctypes.c_int),
        "lec_es_batch_run_async": ([_P, _P], ctypes.c_int),
        "lec_es_batch_info": ([_P, ctypes.POINTER(lec_es_batch_layout)], ctypes.c_int),
        "lec_es_signatures": ([_P, ctypes.c_uint32, ctypes.c_uint32, _u32p, _u64p, ctypes.c_uint32, _u64p, _u64p],
                              ctypes.c_int),
        "lec_es_match_pairs": ([_P, ctypes.c_uint32, ctypes.c_uint32, _u32p, _u64p, ctypes.c_uint32,
                                ctypes.c_uint32, _u32p, ctypes.c_uint64, _u64p], ctypes.c_int),
        "lec_es_batch_results": ([_P, _P, R, ctypes.c_size_t], ctypes.c_int),
        "lec_es_batch_free": ([_P, _P], None),
        "lec_es_submit": ([_P, M, _u64p], ctypes.c_int),
        "lec_es_submit_many": ([_P, M, ctypes.c_size_t, _u64p], ctypes.c_int),
        "lec_es_poll": ([_P, ctypes.c_uint64, R], ctypes.c_int),
        "lec_es_wait": ([_P, ctypes.c_uint64, ctypes.c_double, R], ctypes.c_int),
        "lec_es_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
        "lec_es_server_config": ([_P, ctypes.c_size_t, ctypes.c_uint32], ctypes.c_int),
        "lec_es_truth_tables_ex": ([_P, M, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _u32p,
                                    ctypes.POINTER(ctypes.c_uint8), _u64p], ctypes.c_int),
        "lec_es_jit_compile": ([M, ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t, _u64p],
                               ctypes.c_int),
        "lec_es_check_noalloc": ([_P, ctypes.c_uint64, ctypes.POINTER(lec_es_program_info), ctypes.c_uint64,
                                  ctypes.c_uint64, _P, _P], ctypes.c_int),
        "lec_es_codegen_version": ([], ctypes.c_uint32),
        "lec_es_sweep": ([_P, M, ctypes.POINTER(lec_es_sweep_options), ctypes.POINTER(lec_es_sweep_result), _u64p,
                          _u32p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "lec_es_cost_fit": ([_u32p, _u32p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                             ctypes.POINTER(lec_es_cost_coeffs)], ctypes.c_int),
        "lec_es_cost_model": ([_P, ctypes.c_uint32, ctypes.POINTER(lec_es_cost_coeffs)], ctypes.c_int),
        "lec_es_cost_predict": ([_P, M, ctypes.c_uint32, ctypes.POINTER(lec_es_cost)], ctypes.c_int),
        "lec_es_lop3_peak": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _strerror(status: int) -> str:
    try:
        return load().lec_es_strerror(status).decode()
    except LecEsError:
        return f"status {status}"


def _ok(rc: int, what: str) -> None:
    if rc != OK:
        raise LecEsError(rc, what)


class Miter:
    """Keeps the fanin array alive for the duration of a call."""

    def __init__(self, num_pis: int, fanins, out_lit: int):
        self.fanins = np.ascontiguousarray(np.asarray(fanins, dtype=np.uint32).reshape(-1))
        self.c = lec_es_miter(num_pis, len(self.fanins) // 2,
                              self.fanins.ctypes.data_as(_u32p), out_lit)


def miter_of(aig, out_lit: Optional[int] = None) -> Miter:
    return Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0] if out_lit is None else out_lit)


FLAG_JIT_AND_FORM, FLAG_TEST_WAIT_TIMEOUT, FLAG_AUTOTUNE = 1, 2, 4


class lec_es_batch_layout(ctypes.Structure):
    _fields_ = [("miters", ctypes.c_uint32), ("jit_miters", ctypes.c_uint32), ("tile_miters", ctypes.c_uint32),
                ("fallback_miters", ctypes.c_uint32), ("tiles", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("stage_records", ctypes.c_uint32),
                ("tile_granularity", ctypes.c_uint32), ("grid_blocks", ctypes.c_uint32),
                ("prepare_ms", ctypes.c_double), ("jit_ms", ctypes.c_double), ("tune_ms", ctypes.c_double)]


def options(word_begin: int = 0, word_end: int = NO_CEX, tier: int = TIER_AUTO, order: int = ORDER_AUTO,
            block_threads: int = 0, grid_blocks: int = 0, flags: int = 0, tile_granularity: int = 0,
            stage_records: int = 0) -> lec_es_options:
    return lec_es_options(word_begin, word_end, tier, order, block_threads, grid_blocks, flags,
                          tile_granularity, stage_records)


# ---- entry points (same names as the C ABI) -------------------------------------

class Context:
    """A lec_es_ctx plus the torch arena tensor and stream it was given."""

    def __init__(self, handle, arena, stream):
        self.handle = handle
        self.arena = arena
        self.stream = stream

    def __del__(self):
        try:
            lec_es_destroy(self)
        except Exception:
            pass


def lec_es_create(device: int = 0, arena_bytes: int = 1 << 30, max_pis: int = 63, timeout_s: float = 0.0,
                  jit_cache_dir: Optional[str] = None, stream=None) -> Context:
    import torch
    lib = load()
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
    if stream is None:
        stream = torch.cuda.Stream(device=device)
    cfg = lec_es_config(device, ctypes.c_void_p(arena.data_ptr()), arena_bytes,
                        ctypes.c_void_p(stream.cuda_stream), max_pis, timeout_s,
                        jit_cache_dir.encode() if jit_cache_dir else None)
    h = _P()
    _ok(lib.lec_es_create(ctypes.byref(h), ctypes.byref(cfg)), "lec_es_create")
    return Context(h, arena, stream)


def lec_es_destroy(ctx: Context) -> None:
    if ctx.handle:
        load().lec_es_destroy(ctx.handle)
        ctx.handle = None


def lec_es_compile(m: Miter, order: int = ORDER_AUTO):
    """Host-only slot program: (info, records as (num_records,) uint64)."""
    lib = load()
    info = lec_es_program_info()
    _ok(lib.lec_es_compile(ctypes.byref(m.c), order, ctypes.byref(info), None, 0), "lec_es_compile")
    recs = np.zeros(max(1, info.num_records), dtype=np.uint64)
    _ok(lib.lec_es_compile(ctypes.byref(m.c), order, ctypes.byref(info), recs.ctypes.data_as(_u64p),
                           info.num_records), "lec_es_compile")
    return info, recs[: info.num_records]


def lec_es_check(ctx: Context, m: Miter) -> lec_es_result:
    r = lec_es_result()
    _ok(load().lec_es_check(ctx.handle, ctypes.byref(m.c), ctypes.byref(r)), "lec_es_check")
    return r


def lec_es_check_ex(ctx: Context, m: Miter, opt: lec_es_options) -> lec_es_result:
    r = lec_es_result()
    _ok(load().lec_es_check_ex(ctx.handle, ctypes.byref(m.c), ctypes.byref(opt), ctypes.byref(r)),
        "lec_es_check_ex")
    return r


def lec_es_prepare(ctx: Context, m: Miter, opt: Optional[lec_es_options] = None):
    p = _P()
    _ok(load().lec_es_prepare(ctx.handle, ctypes.byref(m.c), ctypes.byref(opt) if opt else None,
                              ctypes.byref(p)), "lec_es_prepare")
    return p


def lec_es_run_async(ctx: Context, plan, opt: Optional[lec_es_options] = None) -> None:
    _ok(load().lec_es_run_async(ctx.handle, plan, ctypes.byref(opt) if opt else None), "lec_es_run_async")


def lec_es_plan_result(ctx: Context, plan) -> lec_es_result:
    r = lec_es_result()
    _ok(load().lec_es_plan_result(ctx.handle, plan, ctypes.byref(r)), "lec_es_plan_result")
    return r


def lec_es_plan_info(plan) -> lec_es_program_info:
    info = lec_es_program_info()
    _ok(load().lec_es_plan_info(plan, ctypes.byref(info)), "lec_es_plan_info")
    return info


def lec_es_plan_free(ctx: Context, plan) -> None:
    load().lec_es_plan_free(ctx.handle, plan)


def lec_es_truth_tables(ctx: Context, m: Miter, word_begin: int, word_end: int):
    """(vars, (cone_ands, words) uint64 table) from the interpreter kernel."""
    info, _ = lec_es_compile(m)
    nw = word_end - word_begin
    vars_ = np.zeros(max(1, info.cone_ands), dtype=np.uint32)
    out = np.zeros((max(1, info.cone_ands), nw), dtype=np.uint64)
    _ok(load().lec_es_truth_tables(ctx.handle, ctypes.byref(m.c), word_begin, word_end,
                                   vars_.ctypes.data_as(_u32p), out.ctypes.data_as(_u64p)),
        "lec_es_truth_tables")
    return vars_[: info.cone_ands], out[: info.cone_ands]


def lec_es_truth_tables_ex(ctx: Context, m: Miter, word_begin: int, word_end: int, tier: int):
    """(vars, (cone_ands, words) uint64 table, row_valid bool array) from the
    given kernel tier (TIER_SPILL, TIER_INTERP or TIER_JIT)."""
    info, _ = lec_es_compile(m)
    nw = word_end - word_begin
    k = max(1, info.cone_ands)
    vars_ = np.zeros(k, dtype=np.uint32)
    valid = np.zeros(k, dtype=np.uint8)
    out = np.zeros((k, nw), dtype=np.uint64)
    _ok(load().lec_es_truth_tables_ex(ctx.handle, ctypes.byref(m.c), word_begin, word_end, tier,
                                      vars_.ctypes.data_as(_u32p), valid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      out.ctypes.data_as(_u64p)),
        "lec_es_truth_tables_ex")
    n = info.cone_ands
    return vars_[:n], out[:n], valid[:n].astype(bool)


def _miter_array(ms: Sequence[Miter]):
    arr = (lec_es_miter * len(ms))()
    for i, m in enumerate(ms):
        arr[i] = m.c
    return arr


def lec_es_batch(ctx: Context, ms: Sequence[Miter]) -> List[lec_es_result]:
    arr = _miter_array(ms)
    res = (lec_es_result * len(ms))()
    _ok(load().lec_es_batch(ctx.handle, arr, len(ms), res), "lec_es_batch")
    return list(res)


def lec_es_batch_prepare(ctx: Context, ms: Sequence[Miter], opt: Optional[lec_es_options] = None):
    arr = _miter_array(ms)
    b = _P()
    _ok(load().lec_es_batch_prepare(ctx.handle, arr, len(ms), ctypes.byref(opt) if opt else None,
                                    ctypes.byref(b)), "lec_es_batch_prepare")
    return b


def lec_es_batch_info(b) -> lec_es_batch_layout:
    info = lec_es_batch_layout()
    _ok(load().lec_es_batch_info(b, ctypes.byref(info)), "lec_es_batch_info")
    return info


def lec_es_batch_run_async(ctx: Context, b) -> None:
    _ok(load().lec_es_batch_run_async(ctx.handle, b), "lec_es_batch_run_async")


def lec_es_batch_results(ctx: Context, b, k: int) -> List[lec_es_result]:
    res = (lec_es_result * k)()
    _ok(load().lec_es_batch_results(ctx.handle, b, res, k), "lec_es_batch_results")
    return list(res)


def lec_es_batch_free(ctx: Context, b) -> None:
    load().lec_es_batch_free(ctx.handle, b)


def lec_es_server_config(ctx: Context, slot_budget_bytes: int, max_inflight: int) -> None:
    _ok(load().lec_es_server_config(ctx.handle, slot_budget_bytes, max_inflight), "lec_es_server_config")


def lec_es_submit(ctx: Context, m: Miter) -> int:
    t = ctypes.c_uint64()
    _ok(load().lec_es_submit(ctx.handle, ctypes.byref(m.c), ctypes.byref(t)), "lec_es_submit")
    return int(t.value)


def lec_es_submit_many(ctx: Context, ms: Sequence[Miter]) -> List[int]:
    """Submit many miters in one call; their tickets, in order."""
    k = len(ms)
    t = np.zeros(max(1, k), dtype=np.uint64)
    arr = _miter_array(ms)
    _ok(load().lec_es_submit_many(ctx.handle, arr, k, t.ctypes.data_as(_u64p)), "lec_es_submit_many")
    return [int(x) for x in t[:k]]


def lec_es_poll(ctx: Context, ticket: int) -> Optional[lec_es_result]:
    """The result once done, None while running (EBUSY)."""
    r = lec_es_result()
    rc = load().lec_es_poll(ctx.handle, ticket, ctypes.byref(r))
    if rc == EBUSY:
        return None
    _ok(rc, "lec_es_poll")
    return r


def lec_es_wait(ctx: Context, ticket: int, timeout_s: float = 600.0) -> lec_es_result:
    r = lec_es_result()
    _ok(load().lec_es_wait(ctx.handle, ticket, timeout_s, ctypes.byref(r)), "lec_es_wait")
    return r


def lec_es_cancel(ctx: Context, ticket: int) -> None:
    _ok(load().lec_es_cancel(ctx.handle, ticket), "lec_es_cancel")


def lec_es_jit_compile(m: Miter, cc_major: int = 10, cc_minor: int = 3):
    """Host-only NVRTC compile of the specialised kernel: (log, cubin bytes)."""
    buf = ctypes.create_string_buffer(1 << 16)
    n = ctypes.c_uint64()
    _ok(load().lec_es_jit_compile(ctypes.byref(m.c), cc_major, cc_minor, buf, len(buf), ctypes.byref(n)),
        "lec_es_jit_compile")
    return buf.value.decode(errors="replace"), int(n.value)


def lec_es_check_noalloc(d_records: int, records_capacity: int, info: lec_es_program_info, word_begin: int,
                         word_end: int, d_result: int, stream: int) -> None:
    """Enqueue the allocation-free check: device pointers and a stream handle
    are passed as integers; the call allocates nothing."""
    _ok(load().lec_es_check_noalloc(ctypes.c_void_p(d_records), records_capacity, ctypes.byref(info),
                                    word_begin, word_end, ctypes.c_void_p(d_result), ctypes.c_void_p(stream)),
        "lec_es_check_noalloc")


def lec_es_signatures(ctx: Context, num_pis: int, fanins, pi_words, want_sigs: bool = True):
    """(signatures (V, nwords) uint64 or None, hashes (V,) uint64) of every
    variable; pi_words is a (num_pis, nwords) uint64 array."""
    f = np.ascontiguousarray(np.asarray(fanins, dtype=np.uint32).reshape(-1))
    pw = np.ascontiguousarray(np.asarray(pi_words, dtype=np.uint64).reshape(num_pis, -1))
    nw = pw.shape[1] if num_pis else 1
    V = num_pis + len(f) // 2 + 1
    h = np.zeros(V, dtype=np.uint64)
    sg = np.zeros((V, nw), dtype=np.uint64) if want_sigs else None
    _ok(load().lec_es_signatures(ctx.handle, num_pis, len(f) // 2, f.ctypes.data_as(_u32p),
                                 pw.ctypes.data_as(_u64p), nw, sg.ctypes.data_as(_u64p) if want_sigs else None,
                                 h.ctypes.data_as(_u64p)), "lec_es_signatures")
    return sg, h


def lec_es_match_pairs(ctx: Context, num_pis: int, fanins, pi_words, max_support: int):
    """List of (representative var, member var) candidate pairs."""
    f = np.ascontiguousarray(np.asarray(fanins, dtype=np.uint32).reshape(-1))
    pw = np.ascontiguousarray(np.asarray(pi_words, dtype=np.uint64).reshape(num_pis, -1))
    n = ctypes.c_uint64()
    lib = load()
    args = (ctx.handle, num_pis, len(f) // 2, f.ctypes.data_as(_u32p), pw.ctypes.data_as(_u64p), pw.shape[1],
            max_support)
    _ok(lib.lec_es_match_pairs(*args, None, 0, ctypes.byref(n)), "lec_es_match_pairs")
    out = np.zeros(max(1, 2 * n.value), dtype=np.uint32)
    _ok(lib.lec_es_match_pairs(*args, out.ctypes.data_as(_u32p), n.value, ctypes.byref(n)), "lec_es_match_pairs")
    return [(int(out[2 * i]), int(out[2 * i + 1])) for i in range(n.value)]


def lec_es_lop3_peak(ctx: Context):
    """(LOP3 results / clk / SM, SM count, SM clock kHz, LOP3 / s)."""
    a, b, c, d = ctypes.c_double(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _ok(load().lec_es_lop3_peak(ctx.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                ctypes.byref(d)), "lec_es_lop3_peak")
    return a.value, b.value, c.value, d.value


def lec_es_codegen_version() -> int:
    """Version of the specialised-kernel code generator."""
    return int(load().lec_es_codegen_version())


TIER_COMPILE = 4  # lec_es_cost_model: the kernel-build model
TIER_KERNEL = 5   # lec_es_cost_model: the specialised kernel by its executed lop3


def lec_es_cost_fit(gates, n, ms) -> lec_es_cost_coeffs:
    """Fit t = a + c * gates + alpha * gates * 2^(n-23) (relative error, all >= 0)."""
    g = np.ascontiguousarray(np.asarray(gates, dtype=np.uint32))
    nn = np.ascontiguousarray(np.asarray(n, dtype=np.uint32))
    t = np.ascontiguousarray(np.asarray(ms, dtype=np.float64))
    out = lec_es_cost_coeffs()
    _ok(load().lec_es_cost_fit(g.ctypes.data_as(_u32p), nn.ctypes.data_as(_u32p),
                               t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t), ctypes.byref(out)),
        "lec_es_cost_fit")
    return out


def lec_es_cost_model(ctx: Optional[Context], tier: int) -> lec_es_cost_coeffs:
    out = lec_es_cost_coeffs()
    _ok(load().lec_es_cost_model(ctx.handle if ctx else None, tier, ctypes.byref(out)), "lec_es_cost_model")
    return out


def lec_es_cost_predict(ctx: Optional[Context], m: Miter, cpu_threads: int = 1) -> lec_es_cost:
    out = lec_es_cost()
    _ok(load().lec_es_cost_predict(ctx.handle if ctx else None, ctypes.byref(m.c), cpu_threads, ctypes.byref(out)),
        "lec_es_cost_predict")
    return out


def lec_es_sweep(ctx: Context, m: Miter, sim_words: int = 0, max_rounds: int = 0, max_leaves: int = 0,
                 max_nodes: int = 0, final_max_pis: int = 0, seed: int = 0, merges_cap: int = 0):
    """Sweep a miter: (result, cex as a list of PI values or None, merges as
    (member, representative, phase) triples of the input AIG)."""
    num_pis = int(m.c.num_pis)
    o = lec_es_sweep_options(sim_words, max_rounds, max_leaves, max_nodes, final_max_pis, 0, seed)
    r = lec_es_sweep_result()
    cex = np.zeros(max(1, (num_pis + 63) // 64), dtype=np.uint64)
    mg = np.zeros(max(1, 3 * merges_cap), dtype=np.uint32)
    n = ctypes.c_uint64()
    _ok(load().lec_es_sweep(ctx.handle, ctypes.byref(m.c), ctypes.byref(o), ctypes.byref(r), cex.ctypes.data_as(_u64p),
                            mg.ctypes.data_as(_u32p), merges_cap, ctypes.byref(n)), "lec_es_sweep")
    bits = None
    if r.verdict == NONEQUIVALENT:
        bits = [int((int(cex[k // 64]) >> (k % 64)) & 1) for k in range(num_pis)]
    trip = [(int(mg[3 * i]), int(mg[3 * i + 1]), int(mg[3 * i + 2])) for i in range(min(merges_cap, n.value))]
    return r, bits, trip
