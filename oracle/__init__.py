"""CPU oracle for exact simulation (ES) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never imports, links or runs it, and shares no code with it.

The oracle is the definition of ES written out in plain C (``es_oracle.c``):
enumerate every assignment of the miter output's PI support and check the
output (paper §2.2 "Exact Simulation"; miter semantics §2.1), one value per AIG
node, single thread.  Functions here are ctypes wrappers; the C file is built
with gcc on first use (``build()``).

Parity status of each function is pinned by ``tests/test_oracle_pins.py``
(brute force, integer closed forms, named identities, mutants confirmed by
evaluating both netlists directly, a closed-form counterexample).

``cpu_es_blocked`` (``cpu_es_blocked.c``, its own library) is not the oracle
but a CPU exact-simulation baseline in the paper's CPU setting (an
instruction stream over reference-counted value rows, 2^14 patterns per pass
and thread, all host threads); the benchmark times it beside the oracle, and
``tests/test_oracle_pins.py`` pins it to the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "es_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libes_oracle.so")
CPU_ES_SRC = os.path.join(HERE, "cpu_es_blocked.c")
CPU_ES_LIB = os.path.join(BUILD_DIR, "libcpu_es_blocked.so")

NONE = (1 << 64) - 1
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile es_oracle.c with gcc (plain -O2, no vectorisation flags), and
    the CPU-ES baseline (-O3, portable x86-64 code, pthreads)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    for src, lib, flags in ((SRC, LIB, ["-O2"]), (CPU_ES_SRC, CPU_ES_LIB, ["-O3", "-pthread"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc"] + flags + ["-std=c11", "-shared", "-fPIC", "-o", tmp, src])
            os.replace(tmp, lib)
    return LIB


def _load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_support.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                           _u32p, _u32p, _u32p]
            lib.oracle_check.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _u64p, _u64p, _u32p]
            lib.oracle_truth_tables.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                                ctypes.c_uint64, ctypes.c_uint64, _u32p, ctypes.c_uint32, _u64p]
            lib.oracle_eval_patterns.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, _u64p,
                                                 ctypes.c_uint64, _u32p, ctypes.c_uint32, _u64p]
            for f in (lib.oracle_support, lib.oracle_check, lib.oracle_truth_tables, lib.oracle_eval_patterns):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


_cpu_es: Optional[ctypes.CDLL] = None


def _load_cpu_es() -> ctypes.CDLL:
    global _cpu_es
    with _lock:
        if _cpu_es is None:
            build()
            lib = ctypes.CDLL(CPU_ES_LIB)
            lib.cpu_es_blocked.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           _u64p, _u32p]
            lib.cpu_es_blocked.restype = ctypes.c_int
            _cpu_es = lib
    return _cpu_es


def cpu_es_blocked(num_pis: int, fanins, out_lit: int, word_begin: int = 0, word_end: int = NONE,
                   block_words: int = 256, threads: Optional[int] = None) -> Tuple[Optional[int], int]:
    """CPU-ES baseline (not the oracle): lowest failing pattern over the word
    range or None, and n.  block_words = 256 is the paper's 2^14 patterns
    per pass; threads defaults to every host thread."""
    f = _arr32(fanins)
    first = ctypes.c_uint64()
    n = ctypes.c_uint32()
    t = threads or (os.cpu_count() or 1)
    _check(_load_cpu_es().cpu_es_blocked(num_pis, len(f) // 2, _p32(f), out_lit, word_begin, word_end,
                                         block_words, t, ctypes.byref(first), ctypes.byref(n)))
    return (None if first.value == NONE else int(first.value)), int(n.value)


def _arr32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32).reshape(-1))


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _check(rc: int) -> None:
    if rc != 0:
        raise ValueError(f"oracle error {rc}")


def support(num_pis: int, fanins, out_lit: int) -> Tuple[List[int], int]:
    """(sorted support PI indices, number of cone ANDs) of out_lit."""
    f = _arr32(fanins)
    sup = np.zeros(max(1, num_pis), dtype=np.uint32)
    n = ctypes.c_uint32()
    na = ctypes.c_uint32()
    _check(_load().oracle_support(num_pis, len(f) // 2, _p32(f), out_lit, _p32(sup),
                                  ctypes.byref(n), ctypes.byref(na)))
    return [int(x) for x in sup[: n.value]], int(na.value)


def num_words(n: int) -> int:
    return 1 if n <= 6 else 1 << (n - 6)


def check(num_pis: int, fanins, out_lit: int, word_begin: int = 0, word_end: int = NONE,
          count_all: bool = False) -> Tuple[Optional[int], int, int]:
    """ES of the miter output over a word range.

    Returns (lowest failing pattern or None, failing-pattern count (full
    count only when count_all), support size n)."""
    f = _arr32(fanins)
    first = ctypes.c_uint64()
    cnt = ctypes.c_uint64()
    n = ctypes.c_uint32()
    _check(_load().oracle_check(num_pis, len(f) // 2, _p32(f), out_lit, word_begin, word_end,
                                1 if count_all else 0, ctypes.byref(first), ctypes.byref(cnt),
                                ctypes.byref(n)))
    cex = None if first.value == NONE else int(first.value)
    return cex, int(cnt.value), int(n.value)


def check_parallel(num_pis: int, fanins, out_lit: int, threads: int, word_begin: int = 0,
                   word_end: Optional[int] = None) -> Tuple[Optional[int], int]:
    """The same oracle run unchanged on ``threads`` disjoint word ranges (ctypes
    releases the GIL during each call); the lowest failing pattern of the
    lowest range that fails is the answer.  Returns (cex or None, n)."""
    sup, _ = support(num_pis, fanins, out_lit)
    W = num_words(len(sup))
    end = W if word_end is None else min(word_end, W)
    span = max(1, (end - word_begin + threads - 1) // threads)
    res = [None] * threads

    def run(i: int) -> None:
        lo = word_begin + i * span
        hi = min(end, lo + span)
        if lo < hi:
            res[i] = check(num_pis, fanins, out_lit, lo, hi)[0]

    ts = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    found = [r for r in res if r is not None]
    return (min(found) if found else None), len(sup)


def truth_tables(num_pis: int, fanins, out_lit: int, vars_: Sequence[int], word_begin: int = 0,
                 word_end: Optional[int] = None) -> np.ndarray:
    """(len(vars_), words) uint64 truth tables of the given variables over the
    output cone's pattern space."""
    f = _arr32(fanins)
    sup, _ = support(num_pis, f, out_lit)
    W = num_words(len(sup))
    we = W if word_end is None else word_end
    v = _arr32(vars_)
    out = np.zeros((len(v), we - word_begin), dtype=np.uint64)
    _check(_load().oracle_truth_tables(num_pis, len(f) // 2, _p32(f), out_lit, word_begin, we,
                                       _p32(v), len(v), _p64(out)))
    return out


def eval_patterns(num_pis: int, fanins, patterns, lits: Sequence[int]) -> np.ndarray:
    """Values of ``lits`` at explicit patterns.  ``patterns`` is an (m,) uint64
    array; bit k = value of PI k (num_pis <= 64).  Returns a (len(lits), m)
    bool array."""
    f = _arr32(fanins)
    pats = np.asarray(patterns, dtype=np.uint64).reshape(-1)
    m = len(pats)
    nw = max(1, (m + 63) // 64)
    padded = np.zeros(nw * 64, dtype=np.uint64)
    padded[:m] = pats
    pw = np.zeros((num_pis, nw), dtype=np.uint64)
    for k in range(num_pis):
        bits = ((padded >> np.uint64(k)) & np.uint64(1)).astype(np.uint8).reshape(nw, 64)
        pw[k] = np.packbits(bits, axis=1, bitorder="little").view("<u8").reshape(nw)
    l = _arr32(lits)
    out = np.zeros((len(l), nw), dtype=np.uint64)
    _check(_load().oracle_eval_patterns(num_pis, len(f) // 2, _p32(f), _p64(pw), nw,
                                        _p32(l), len(l), _p64(out)))
    bits = np.unpackbits(out.view(np.uint8).reshape(len(l), nw * 8), axis=1, bitorder="little")
    return bits[:, :m].astype(bool)
