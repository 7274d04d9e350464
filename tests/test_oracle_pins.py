"""Pins of the CPU oracle against facts fixed by the paper and by arithmetic.

Each test is chosen so that a plausible oracle mistake fails it: a wrong PI
mask or word-bit mapping breaks the integer closed forms and brute force; a
dropped complement or a wrong fanin breaks brute force on random graphs; a
wrong n<6 mask breaks the small-support cases; a wrong counterexample index
breaks the hand-derived fixtures and the closed-form counterexample
2^32 - 1 of the 16x16 mutant; a checker that always answers EQUIVALENT fails
every mutant test.  The evaluators in ``reference_eval`` are independent of
the oracle (per-assignment booleans, one numpy bool per pattern).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from tests.reference_eval import eval_one, eval_vectors, random_aig, to_int

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_force(aig, out_lit):
    """Per-assignment evaluation over the support (pattern bit k -> support PI k)."""
    sup, _ = O.support(aig.num_pis, aig.fanins, out_lit)
    n = len(sup)
    fails = []
    for p in range(1 << n):
        asg = 0
        for k, pi in enumerate(sup):
            if (p >> k) & 1:
                asg |= 1 << pi
        if eval_one(aig, asg, [out_lit])[0]:
            fails.append(p)
    return sup, fails


# --- hand-derived fixtures ----------------------------------------------------

@pytest.mark.parametrize("name", ["xor_forms_equiv.aag", "xor_vs_or_buggy.aag", "skip_pi_support.aag"])
def test_golden_fixtures(name):
    exp = json.load(open(os.path.join(GOLDEN, "expected.json")))[name]
    aig = C.read_aiger(open(os.path.join(GOLDEN, name), "rb").read())
    sup, _ = O.support(aig.num_pis, aig.fanins, aig.outputs[0])
    assert sup == exp["support"]
    cex, count, n = O.check(aig.num_pis, aig.fanins, aig.outputs[0], count_all=True)
    assert cex == exp["cex"]
    assert count == exp["fail_count"]
    assert (cex is None) == (exp["verdict"] == "EQUIVALENT")


# --- brute force on random graphs -----------------------------------------------

@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_random_graphs(seed):
    rng = np.random.default_rng(seed)
    num_pis = int(rng.integers(1, 11))
    aig = random_aig(rng, num_pis, int(rng.integers(1, 60)))
    out = aig.outputs[0]
    sup, fails = brute_force(aig, out)
    cex, count, n = O.check(aig.num_pis, aig.fanins, out, count_all=True)
    assert n == len(sup)
    assert count == len(fails)
    assert cex == (fails[0] if fails else None)
    cex0, _, _ = O.check(aig.num_pis, aig.fanins, out)  # first-failure mode
    assert cex0 == cex


@pytest.mark.parametrize("seed", range(12))
def test_truth_tables_every_node_bruteforce(seed):
    rng = np.random.default_rng(1000 + seed)
    num_pis = int(rng.integers(2, 10))
    aig = random_aig(rng, num_pis, 50)
    out = aig.outputs[0]
    sup, _ = O.support(aig.num_pis, aig.fanins, out)
    n = len(sup)
    # every variable of the cone: the constant, support PIs, cone ANDs
    base = aig.num_pis + 1
    cone = set()
    stack = [out >> 1]
    while stack:
        v = stack.pop()
        if v in cone:
            continue
        cone.add(v)
        if v >= base:
            stack += [int(aig.fanins[v - base, 0]) >> 1, int(aig.fanins[v - base, 1]) >> 1]
    vars_ = sorted(cone | {0})
    tt = O.truth_tables(aig.num_pis, aig.fanins, out, vars_)
    for p in range(1 << n):
        asg = sum(1 << pi for k, pi in enumerate(sup) if (p >> k) & 1)
        vals = eval_one(aig, asg, [2 * v for v in vars_])
        got = (tt[:, p >> 6] >> np.uint64(p & 63)) & np.uint64(1)
        assert [bool(x) for x in got] == vals, f"pattern {p}"


# --- small supports and constants (n < 6 masking) -------------------------------

def _aig(num_pis, ands, out):
    f = np.array(ands, dtype=np.uint32).reshape(-1, 2)
    return C.Aig(num_pis, f, [out])


def test_constant_outputs():
    a = _aig(3, [], 0)
    assert O.check(3, a.fanins, 0, count_all=True) == (None, 0, 0)
    # constant TRUE: one pattern (n = 0) and it fails
    assert O.check(3, a.fanins, 1, count_all=True) == (0, 1, 0)


def test_single_pi_outputs():
    a = _aig(5, [], 0)
    assert O.check(5, a.fanins, 2 * 4, count_all=True) == (1, 1, 1)       # PI 3
    assert O.check(5, a.fanins, 2 * 4 + 1, count_all=True) == (0, 1, 1)   # !PI 3


def test_and_of_k_pis_has_single_failing_pattern():
    for k in range(2, 9):
        g = C.AigBuilder(k + 2)
        out = g.and_tree([g.pi(i) for i in range(1, k + 1)])  # skips PI 0
        aig = g.finish([out])
        cex, count, n = O.check(aig.num_pis, aig.fanins, out, count_all=True)
        assert n == k and count == 1 and cex == (1 << k) - 1


def test_xor_parity_counts():
    for k in range(1, 9):
        g = C.AigBuilder(k)
        x = 0
        for i in range(k):
            x = g.XOR(x, g.pi(i))
        aig = g.finish([x])
        cex, count, n = O.check(aig.num_pis, aig.fanins, x, count_all=True)
        assert n == k and count == (1 << (k - 1)) and cex == 1


# --- integer closed forms (pin both generators and oracle) ---------------------

def test_adder_closed_form_all_patterns():
    m = C.config1_adders()
    out = m.outputs[0]
    P = np.arange(1 << 16, dtype=np.uint64)
    a, b = P & np.uint64(0xFF), P >> np.uint64(8)
    for side in ("A", "B"):
        lits = m.side_outputs[side]
        tt = O.truth_tables(m.num_pis, m.fanins, out, [l >> 1 for l in lits])
        bits = np.unpackbits(tt.view(np.uint8), axis=1, bitorder="little").astype(bool)
        bits ^= np.array([bool(l & 1) for l in lits])[:, None]
        assert np.array_equal(to_int(bits), a + b), side
        # and the independent evaluator agrees with the same closed form
        assert np.array_equal(to_int(eval_vectors(m, P, lits)), a + b)


def test_multiplier12_closed_form_all_patterns():
    m = C.config2_mult12()
    out = m.outputs[0]
    W = 1 << 18
    step = 1 << 14
    for side in ("A", "B"):
        lits = m.side_outputs[side]
        comp = np.array([bool(l & 1) for l in lits])[:, None]
        for w0 in range(0, W, step):
            tt = O.truth_tables(m.num_pis, m.fanins, out, [l >> 1 for l in lits], w0, w0 + step)
            bits = np.unpackbits(tt.view(np.uint8), axis=1, bitorder="little").astype(bool) ^ comp
            P = np.arange(64 * w0, 64 * (w0 + step), dtype=np.uint64)
            a, b = P & np.uint64(0xFFF), P >> np.uint64(12)
            assert np.array_equal(to_int(bits), a * b), (side, w0)


def test_multiplier16_closed_form_samples():
    m = C.config3_mult16()
    rng = np.random.default_rng(16)
    P = rng.integers(0, 1 << 32, size=1 << 16, dtype=np.uint64)
    P[:4] = [0, 0xFFFFFFFF, 0xFFFF, 0xFFFF0000]
    a, b = P & np.uint64(0xFFFF), P >> np.uint64(16)
    for side in ("A", "B"):
        bits = O.eval_patterns(m.num_pis, m.fanins, P, m.side_outputs[side])
        assert np.array_equal(to_int(bits), a * b), side


@pytest.mark.parametrize("w,tree", [(4, "wallace"), (5, "dadda"), (7, "wallace"), (8, "dadda")])
def test_small_multipliers_closed_form_and_equivalence(w, tree):
    m = C.build_multiplier_pair(w, tree=tree)
    P = np.arange(1 << (2 * w), dtype=np.uint64)
    a, b = P & np.uint64((1 << w) - 1), P >> np.uint64(w)
    for side in ("A", "B"):
        bits = O.eval_patterns(m.num_pis, m.fanins, P, m.side_outputs[side])
        assert np.array_equal(to_int(bits), a * b)
    assert O.check(m.num_pis, m.fanins, m.outputs[0], count_all=True)[:2] == (None, 0)


# --- identities named by the method ---------------------------------------------

def test_identity_rca_equals_kogge_stone():
    for w in (1, 2, 3, 5, 8, 11):
        m = C.build_adder_pair(w)
        assert O.check(m.num_pis, m.fanins, m.outputs[0], count_all=True)[:2] == (None, 0)


def test_identity_array_equals_booth_12():
    m = C.config2_mult12()
    cex, _, n = O.check(m.num_pis, m.fanins, m.outputs[0])
    assert n == 24 and cex is None


def test_identity_commutativity():
    for w in (6, 9):
        g = C.AigBuilder(2 * w)
        a = [g.pi(i) for i in range(w)]
        b = [g.pi(w + i) for i in range(w)]
        x = C.array_multiplier(g, a, b)
        g.new_scope()
        y = C.booth_multiplier(g, b, a, tree="dadda")  # b * a
        g.new_scope()
        out = C.miter_outputs(g, x, y)
        aig = g.finish([out])
        assert O.check(aig.num_pis, aig.fanins, out, count_all=True)[:2] == (None, 0)


# --- mutants: counterexample confirmed on both netlists directly ---------------

def _confirm_lowest(m, cex, w):
    """Both sides' integer outputs differ at cex and agree on every p < cex."""
    A, B = m.side_outputs["A"], m.side_outputs["B"]
    ra = eval_one(m, cex, A)
    rb = eval_one(m, cex, B)
    assert ra != rb
    if cex:
        P = np.arange(cex, dtype=np.uint64)
        assert np.array_equal(to_int(eval_vectors(m, P, A)), to_int(eval_vectors(m, P, B)))


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_adder_mutants(seed):
    m = C.config1_adders(mutant_seed=seed)
    cex, count, n = O.check(m.num_pis, m.fanins, m.outputs[0], count_all=True)
    assert cex is not None and n == 16
    _confirm_lowest(m, cex, 8)
    P = np.arange(1 << 16, dtype=np.uint64)
    diff = to_int(eval_vectors(m, P, m.side_outputs["A"])) != to_int(eval_vectors(m, P, m.side_outputs["B"]))
    assert int(diff.sum()) == count


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_multiplier12_mutants(seed):
    m = C.config2_mult12(mutant_seed=seed)
    cex, _, n = O.check(m.num_pis, m.fanins, m.outputs[0])
    assert cex is not None and n == 24
    _confirm_lowest(m, cex, 12)


def test_multiplier16_mutant_closed_form_cex():
    """The 16x16 mutant XORs AND(all 32 PIs) into the MSB, so its only failing
    pattern is a = b = 0xFFFF, i.e. p = 2^32 - 1 (closed form)."""
    m = C.config3_mult16(mutant=True)
    W = 1 << 26
    cex, count, n = O.check(m.num_pis, m.fanins, m.outputs[0], W - 64, W, count_all=True)
    assert n == 32 and cex == (1 << 32) - 1 and count == 1
    rng = np.random.default_rng(3)
    for w0 in rng.integers(0, W - 64, size=8):
        assert O.check(m.num_pis, m.fanins, m.outputs[0], int(w0), int(w0) + 32)[0] is None
    A, B = m.side_outputs["A"], m.side_outputs["B"]
    assert eval_one(m, (1 << 32) - 1, A) != eval_one(m, (1 << 32) - 1, B)
    assert eval_one(m, (1 << 32) - 2, A) == eval_one(m, (1 << 32) - 2, B)


def test_word_range_split_is_consistent():
    """A range split never changes the lowest counterexample."""
    m = C.config1_adders(mutant_seed=1)
    full = O.check(m.num_pis, m.fanins, m.outputs[0], count_all=True)
    parts = [O.check(m.num_pis, m.fanins, m.outputs[0], w, w + 100, count_all=True) for w in range(0, 1024, 100)]
    assert min(p[0] for p in parts if p[0] is not None) == full[0]
    assert sum(p[1] for p in parts) == full[1]
    assert O.check_parallel(m.num_pis, m.fanins, m.outputs[0], 4)[0] == full[0]


def test_oracle_rejects_bad_graphs():
    bad = _aig(2, [6, 2], 6)  # AND var 3 reads itself
    with pytest.raises(ValueError):
        O.check(2, bad.fanins, 6)
    ok = _aig(2, [2, 4], 6)
    with pytest.raises(ValueError):
        O.check(2, ok.fanins, 2 * 9)  # literal out of range


# --- planted minterms: one failing pattern by construction -----------------------

@pytest.mark.parametrize("w,p,bit", [(6, 0, None), (6, 0xABC, 3), (8, 0x8000, None), (8, 0x1234, 7),
                                     (8, 0xFFFF, 0), (8, 0x0400, 15)])
def test_planted_minterm_is_the_only_failing_pattern(w, p, bit):
    """XORing the minterm of p into one product bit of the Booth side makes p
    the only pattern where the sides differ: the oracle's lowest cex and
    failing count (1) match the independent per-pattern evaluation of both
    sides over the whole space."""
    m = C.build_multiplier_pair(w, tree="dadda", planted_minterm=p, planted_bit=bit)
    cex, count, n = O.check(m.num_pis, m.fanins, m.outputs[0], count_all=True)
    assert (cex, count, n) == (p, 1, 2 * w)
    P = np.arange(1 << (2 * w), dtype=np.uint64)
    diff = to_int(eval_vectors(m, P, m.side_outputs["A"])) != to_int(eval_vectors(m, P, m.side_outputs["B"]))
    assert np.flatnonzero(diff).tolist() == [p]


@pytest.mark.parametrize("p", [1 << 20, (1 << 28) + 0x5A5A, (1 << 31) + (1 << 26) + 77, 0x9E3779B9])
def test_planted_minterm_16x16_closed_form(p):
    """The 16x16 planted mutant fails at p and nowhere near it: the oracle on
    the 64 words around p's word finds p with count 1, seeded word ranges
    elsewhere pass, and both netlists evaluated directly differ at p only."""
    m = C.config3_mult16(minterm=p)
    w = p >> 6
    lo = max(0, w - 32)
    cex, count, n = O.check(m.num_pis, m.fanins, m.outputs[0], lo, lo + 64, count_all=True)
    assert (cex, count, n) == (p, 1, 32)
    rng = np.random.default_rng(p & 0xFFFF)
    for w0 in rng.integers(0, (1 << 26) - 32, size=6):
        if not (w0 <= w < w0 + 32):
            assert O.check(m.num_pis, m.fanins, m.outputs[0], int(w0), int(w0) + 32)[0] is None
    A, B = m.side_outputs["A"], m.side_outputs["B"]
    assert eval_one(m, p, A) != eval_one(m, p, B)
    for q in (p - 1, p + 1, p ^ (1 << 31)):
        assert eval_one(m, q, A) == eval_one(m, q, B)


def test_reference_pairs_find_the_equal_sum_bits():
    """The test-side pair reference (oracle evaluation at random patterns)
    pairs every sum bit of a ripple-carry adder with the same bit of a
    Kogge-Stone adder built in another hashing scope: equal functions have
    equal signatures, and the lower variable (the ripple-carry side) is the
    representative."""
    from tests.reference_pairs import pairs_from_oracle
    g = C.AigBuilder(16)
    a = [g.pi(i) for i in range(8)]
    b = [g.pi(8 + i) for i in range(8)]
    x = C.ripple_carry_adder(g, a, b)
    g.new_scope()
    y = C.kogge_stone_adder(g, a, b)
    aig = g.finish(x + y)
    pw = C.signature_words(aig, 4, 9)
    pairs = set(pairs_from_oracle(aig, pw, 16))
    for lx, ly in zip(x[1:], y[1:]):  # bit 0 is a single XOR (hashed the same way on both sides)
        if (lx >> 1) != (ly >> 1) and (lx & 1) == (ly & 1):
            assert (min(lx, ly) >> 1, max(lx, ly) >> 1) in pairs, (lx, ly)


# --- the CPU-ES baseline (reference counting, 2^14 patterns per pass) ------------

@pytest.mark.parametrize("seed", range(20))
def test_cpu_es_baseline_matches_oracle_random_graphs(seed):
    """The blocked, reference-counted CPU-ES baseline gives the oracle's
    lowest counterexample on random graphs (all supports 0..12, blocks that
    do not divide the words, one to several threads, word ranges)."""
    rng = np.random.default_rng(7000 + seed)
    aig = random_aig(rng, int(rng.integers(1, 13)), int(rng.integers(1, 120)))
    out = aig.outputs[0]
    n = O.support(aig.num_pis, aig.fanins, out)[0]
    W = O.num_words(len(n))
    for block, threads in ((256, 4), (3, 1), (1, 7)):
        assert O.cpu_es_blocked(aig.num_pis, aig.fanins, out, block_words=block, threads=threads)[0] == \
            O.check(aig.num_pis, aig.fanins, out)[0]
    wb, we = sorted(int(x) for x in rng.integers(0, W + 1, 2))
    assert O.cpu_es_blocked(aig.num_pis, aig.fanins, out, wb, we, 5, 3)[0] == \
        O.check(aig.num_pis, aig.fanins, out, wb, we)[0]


@pytest.mark.parametrize("seed", [None, 1, 2, 3])
def test_cpu_es_baseline_matches_oracle_12x12(seed):
    m = C.config2_mult12(mutant_seed=seed)
    out = m.outputs[0]
    if seed is None:  # the whole space would take the baseline seconds; a range of it
        assert O.cpu_es_blocked(m.num_pis, m.fanins, out, 1000, 9000)[0] is None
    else:
        assert O.cpu_es_blocked(m.num_pis, m.fanins, out)[0] == O.check(m.num_pis, m.fanins, out)[0]
    assert O.cpu_es_blocked(C.config1_adders().num_pis, C.config1_adders().fanins,
                            C.config1_adders().outputs[0]) == (None, 16)


# --- stored oracle values -------------------------------------------------------

def test_stored_node_pair_results_are_current():
    """The stored per-miter oracle results of the 4,096 node-pair batch
    (written by tests/golden/make_config4_oracle.py) belong to the graph the
    generator builds today, and a seeded sample of them (every
    non-equivalent one of small support, plus equivalent ones) re-checks."""
    from tests.golden.make_config4_oracle import OUT, fingerprint
    pb = C.config4_pairs()
    stored = json.load(open(OUT))
    assert stored["fingerprint"] == fingerprint(pb.aig)
    assert len(stored["cex"]) == len(pb.aig.outputs) == 4096
    a = pb.aig
    small = [i for i, s in enumerate(pb.support_sizes) if s <= 16]
    rng = np.random.default_rng(4)
    sample = [i for i in small if stored["cex"][i] is not None]
    sample += [int(i) for i in rng.choice(small, size=min(40, len(small)), replace=False)]
    assert any(stored["cex"][i] is not None for i in sample)
    for i in sorted(set(sample)):
        assert O.check(a.num_pis, a.fanins, a.outputs[i])[0] == stored["cex"][i], i


def test_stored_spread_results_are_current():
    """The stored oracle results of the 1,024-miter spread batch (written by
    tests/golden/make_spread_oracle.py) belong to the miters the generator
    builds today, and a seeded sample of the small ones (plus every
    non-equivalent one of up to 18 PIs) re-checks."""
    from tests.golden.make_spread_oracle import NUM, OUT, SEED, fingerprint
    trip = C.config4_spread(num=NUM, seed=SEED)
    stored = json.load(open(OUT))
    assert stored["fingerprint"] == fingerprint(trip)
    assert len(stored["cex"]) == len(trip) == NUM
    sup = [len(O.support(a.num_pis, a.fanins, o)[0]) for a, o, _ in trip]
    small = [i for i, s in enumerate(sup) if s <= 18]
    rng = np.random.default_rng(6)
    sample = [i for i in small if stored["cex"][i] is not None]
    sample += [int(i) for i in rng.choice(small, size=min(30, len(small)), replace=False)]
    assert any(stored["cex"][i] is not None for i in sample)
    for i in sorted(set(sample)):
        a, o, _ = trip[i]
        assert O.check(a.num_pis, a.fanins, o)[0] == stored["cex"][i], i
