"""Per-node values of the kernels that carry the work, element by element
against the oracle's truth tables: the word interpreter (es_interp_w) on
every cone AND, and the specialised kernel (in its own layout, through its
dump variant) on every node its 3-input tables compute -- over full pattern
spaces and word ranges that start and end off any alignment."""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx
from tests.reference_eval import random_aig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lec_es_destroy(c)


def _cases():
    rng = np.random.default_rng(2024)
    cases = [C.config1_adders(), C.config1_adders(2), C.build_multiplier_pair(5, "dadda"),
             C.build_multiplier_pair(6, "wallace", planted_minterm=0xABC)]
    for n_pis in (1, 3, 5, 6, 7, 9, 12, 14):
        cases.append(random_aig(rng, n_pis, int(rng.integers(20, 160))))
    return cases


def _ranges(W):
    out = [(0, W)]
    if W >= 8:
        out += [(W // 3 + 1, W - 3), (1, 2), (W - 1, W)]
    return [(a, b) for a, b in out if a < b]


def _compare(ctx, aig, tier, ranges=None):
    out = aig.outputs[0]
    m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
    n = L.lec_es_compile(m)[0].n
    W = O.num_words(n)
    vm = np.uint64((1 << (1 << n)) - 1) if n < 6 else np.uint64((1 << 64) - 1)
    rows = 0
    for wb, we in (ranges or _ranges(W)):
        vars_, tt, valid = L.lec_es_truth_tables_ex(ctx, m, wb, we, tier)
        exp = O.truth_tables(aig.num_pis, aig.fanins, out, [int(v) for v in vars_], wb, we)
        assert np.array_equal(tt[valid] & vm, exp[valid] & vm), (tier, wb, we)
        if tier != L.TIER_JIT:
            assert valid.all()
        rows = max(rows, int(valid.sum()))
    return rows


@pytest.mark.parametrize("i", range(12))
def test_word_interpreter_every_node(ctx, i):
    _compare(ctx, _cases()[i], L.TIER_INTERP)


@pytest.mark.parametrize("i", range(12))
def test_specialised_kernel_every_table(ctx, i):
    aig = _cases()[i]
    rows = _compare(ctx, aig, L.TIER_JIT)
    info, _ = L.lec_es_compile(L.Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0]))
    assert rows == info.num_luts  # one row per table of the cover (a table's node is unique)


def test_chunk_interpreter_through_the_same_call(ctx):
    _compare(ctx, C.config1_adders(1), L.TIER_SPILL)


def test_specialised_kernel_12x12_ranges(ctx):
    """The 12x12 miter (24 PIs) in its default layout (one pass PI), over
    word ranges at the start, in the middle (unaligned) and at the end."""
    aig = C.config2_mult12(mutant_seed=2)
    W = 1 << 18
    _compare(ctx, aig, L.TIER_JIT, [(0, 2048), (100_001, 102_050), (W - 1500, W)])
    _compare(ctx, aig, L.TIER_INTERP, [(100_001, 101_000)])


@pytest.mark.parametrize("env", [{"LEC_ES_JIT_REP": "32", "LEC_ES_JIT_NEST": "1"},
                                 {"LEC_ES_JIT_REP": "32", "LEC_ES_JIT_NEST": "3", "LEC_ES_JIT_UNROLL": "4"},
                                 {"LEC_ES_JIT_REP": "16", "LEC_ES_JIT_NEST": "2", "LEC_ES_JIT_UNROLL": "0"},
                                 {"LEC_ES_JIT_REP": "32", "LEC_ES_JIT_NEST": "3", "LEC_ES_JIT_UNROLL": "2",
                                  "LEC_ES_JIT_HOIST": "8"},
                                 {"LEC_ES_JIT_REP": "8", "LEC_ES_JIT_NEST": "0"}])
def test_specialised_kernel_forced_layouts(env, monkeypatch):
    """Pass loops, nested and unrolled levels, tables hoisted to outer levels
    and values kept in shared memory (a small register budget): every
    table's value, wherever the layout computes it, equals the oracle's."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    c = make_ctx(arena_bytes=2 << 30)
    try:
        rng = np.random.default_rng(31)
        cases = [C.config1_adders(3), C.build_multiplier_pair(8, "dadda", planted_minterm=0x1357),
                 random_aig(rng, 17, 220)]
        for aig in cases:
            n = L.lec_es_compile(L.Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0]))[0].n
            W = O.num_words(n)
            _compare(c, aig, L.TIER_JIT, [(0, W), (W // 5 + 3, W - W // 7)])
    finally:
        L.lec_es_destroy(c)
