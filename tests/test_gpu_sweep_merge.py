"""The sweeping loop with ES as its engine (§2.3 flow, §3.2 local
sub-miters): verdicts against the oracle on miters it can enumerate, every
counterexample re-evaluated by the oracle, every proven merge re-checked by
the oracle (exhaustively on small inputs, on random patterns on 64-PI
graphs), and 64-PI multiplier miters that direct ES cannot enumerate."""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx, oracle_cex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(arena_bytes=1 << 30)
    yield c
    L.lec_es_destroy(c)


def _miter(aig):
    return L.Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0])


def _pattern(bits):
    return sum(b << k for k, b in enumerate(bits))


def _check_merges_exhaustive(aig, merges):
    """member == representative XOR phase on every input pattern."""
    P = aig.num_pis
    pats = np.arange(1 << P, dtype=np.uint64)
    lits = sorted({2 * v for t in merges for v in t[:2]})
    vals = dict(zip(lits, O.eval_patterns(P, aig.fanins, pats, lits)))
    for mem, rep, ph in merges:
        assert np.array_equal(vals[2 * mem], vals[2 * rep] ^ bool(ph)), (mem, rep, ph)


def _check_merges_sampled(aig, merges, n=4096, seed=3):
    rng = np.random.default_rng(seed)
    pats = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    lits = sorted({2 * v for t in merges for v in t[:2]})
    vals = dict(zip(lits, O.eval_patterns(aig.num_pis, aig.fanins, pats, lits)))
    for mem, rep, ph in merges:
        assert np.array_equal(vals[2 * mem], vals[2 * rep] ^ bool(ph)), (mem, rep, ph)


@pytest.mark.parametrize("make", [
    lambda: C.build_revised_pair(6), lambda: C.build_revised_pair(8, "booth"), lambda: C.config1_adders(),
    lambda: C.config2_mult12(), lambda: C.build_revised_pair(8, mutant_seed=2),
    lambda: C.config1_adders(1), lambda: C.config2_mult12(2)])
def test_verdicts_and_merges_match_the_oracle(ctx, make):
    aig = make()
    out = aig.outputs[0]
    want = oracle_cex(aig, out)
    r, cex, merges = L.lec_es_sweep(ctx, _miter(aig), merges_cap=1 << 20, seed=7)
    assert r.pairs_proven == len(merges)
    if want is None:
        assert r.verdict == L.EQUIVALENT
    else:
        assert r.verdict == L.NONEQUIVALENT
        got = O.eval_patterns(aig.num_pis, aig.fanins, [_pattern(cex)], [out])[0, 0]
        assert got, "the counterexample does not fail the miter"
        if r.decided_by == 2:  # decided by the output's own ES: the lowest one
            assert _pattern(cex) == want
    if merges and aig.num_pis <= 16:
        _check_merges_exhaustive(aig, merges)
    elif merges:
        _check_merges_sampled(aig, merges)


def test_revised_multiplier_32x32_is_proven(ctx):
    """64 PIs: the output cannot be enumerated; merging the re-synthesized
    copy into the original, pair by pair, collapses the miter to 0."""
    aig = C.build_revised_pair(32)
    r, cex, merges = L.lec_es_sweep(ctx, _miter(aig), merges_cap=1 << 20, seed=1)
    assert r.verdict == L.EQUIVALENT and r.decided_by == 0
    assert r.ands_final == 0 and r.pairs_proven > 0
    _check_merges_sampled(aig, merges[:: max(1, len(merges) // 2000)])


def test_revised_multiplier_32x32_mutant_is_refuted(ctx):
    aig = C.build_revised_pair(32, mutant_seed=4)
    r, cex, merges = L.lec_es_sweep(ctx, _miter(aig), merges_cap=1 << 20, seed=1)
    assert r.verdict == L.NONEQUIVALENT
    assert O.eval_patterns(aig.num_pis, aig.fanins, [_pattern(cex)], [aig.outputs[0]])[0, 0]
    if merges:
        _check_merges_sampled(aig, merges[:: max(1, len(merges) // 2000)])


def test_structurally_different_64_pi_miter_is_not_refuted(ctx):
    """Array against Booth: few internal equivalences, 64 PIs; the sweep
    must not claim a difference (it is equivalent) and says what it did."""
    aig = C.build_multiplier_pair(32)
    r, cex, merges = L.lec_es_sweep(ctx, _miter(aig), merges_cap=1 << 16, seed=2, max_rounds=8)
    assert r.verdict in (L.EQUIVALENT, L.UNDECIDED)
    if r.verdict == L.UNDECIDED:
        assert r.decided_by == 3 and r.final_support > 36
    if merges:
        _check_merges_sampled(aig, merges)
