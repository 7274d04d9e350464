"""GPU parity: the CUDA path against the CPU oracle, bit-exact.

Everything is integer and exact, so the bar is equality of the verdict, the
counterexample index and (for small cones) every node's truth table.  All
calls go through the C ABI (ctypes binding).
"""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.reference_eval import narrow_aig, random_aig

pytestmark = pytest.mark.gpu

TIERS = [L.TIER_INTERP, L.TIER_SPILL]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2512_06627_b300 import build
    build.build()
    c = L.lec_es_create(0, arena_bytes=4 << 30)
    yield c
    L.lec_es_destroy(c)


def _oracle(aig, out, wb=0, we=None):
    cex, _, n = O.check(aig.num_pis, aig.fanins, out, wb, O.NONE if we is None else we)
    return cex, n


def _gpu(ctx, aig, out, tier=L.TIER_AUTO, wb=0, we=L.NO_CEX, order=L.ORDER_AUTO, block=0):
    m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
    return L.lec_es_check_ex(ctx, m, L.options(wb, we, tier, order, block))


@pytest.mark.parametrize("tier", TIERS)
@pytest.mark.parametrize("seed", range(25))
def test_random_graphs(ctx, tier, seed):
    rng = np.random.default_rng(7000 + seed)
    aig = random_aig(rng, int(rng.integers(1, 14)), int(rng.integers(1, 120)))
    out = aig.outputs[0]
    cex, n = _oracle(aig, out)
    r = _gpu(ctx, aig, out, tier)
    assert r.support_n == n
    assert r.cex_or_none == cex
    assert r.verdict == (L.EQUIVALENT if cex is None else L.NONEQUIVALENT)


@pytest.mark.parametrize("n", range(0, 9))
def test_small_supports(ctx, n):
    """n < 6: masks of the single word; PI k >= 5 from the chunk index."""
    for neg in (0, 1):
        g = C.AigBuilder(10)
        lits = [g.pi(i + 1) for i in range(n)]
        x = g.and_tree(lits) if n else 0
        out = x ^ neg
        aig = g.finish([out])
        for tier in TIERS:
            r = _gpu(ctx, aig, out, tier)
            assert r.cex_or_none == _oracle(aig, out)[0], (n, neg, tier)


@pytest.mark.parametrize("tier", TIERS)
def test_config1_adders(ctx, tier):
    m = C.config1_adders()
    r = _gpu(ctx, m, m.outputs[0], tier)
    assert r.verdict == L.EQUIVALENT and r.cex == L.NO_CEX and r.support_n == 16
    for seed in (1, 2, 3, 4, 5):
        mm = C.config1_adders(mutant_seed=seed)
        r = _gpu(ctx, mm, mm.outputs[0], tier)
        assert r.cex_or_none == _oracle(mm, mm.outputs[0])[0]


@pytest.mark.parametrize("tier", TIERS)
def test_config2_mult12(ctx, tier):
    m = C.config2_mult12()
    r = _gpu(ctx, m, m.outputs[0], tier)
    assert r.verdict == L.EQUIVALENT and r.support_n == 24
    for seed in (1, 2, 3):
        mm = C.config2_mult12(mutant_seed=seed)
        r = _gpu(ctx, mm, mm.outputs[0], tier)
        assert r.verdict == L.NONEQUIVALENT
        assert r.cex_or_none == _oracle(mm, mm.outputs[0])[0]


@pytest.mark.parametrize("order", [L.ORDER_DFS, L.ORDER_VAR, L.ORDER_LEVEL])
@pytest.mark.parametrize("block", [32, 64, 128, 256])
def test_orders_and_blocks_agree(ctx, order, block):
    mm = C.config1_adders(mutant_seed=1)
    r = _gpu(ctx, mm, mm.outputs[0], L.TIER_INTERP, order=order, block=block)
    assert r.cex_or_none == _oracle(mm, mm.outputs[0])[0]


def test_word_ranges_ragged(ctx):
    """Sub-ranges that start and end mid-pass give the oracle's first failure
    in that range (and UNDECIDED when it passes)."""
    mm = C.config2_mult12(mutant_seed=1)
    out = mm.outputs[0]
    rng = np.random.default_rng(11)
    W = 1 << 18
    ranges = [(0, 1), (0, 129), (127, 300), (W - 77, W)] + [
        tuple(sorted(rng.integers(0, W, size=2))) for _ in range(10)]
    for wb, we in ranges:
        if wb == we:
            continue
        for tier in TIERS:
            r = _gpu(ctx, mm, out, tier, int(wb), int(we))
            cex, _ = _oracle(mm, out, int(wb), int(we))
            assert r.cex_or_none == cex, (wb, we, tier)
            if cex is None:
                assert r.verdict == L.UNDECIDED


@pytest.mark.parametrize("tier", TIERS)
def test_truth_tables_every_node(ctx, tier):
    """Per-node values of small cones equal the oracle's truth tables."""
    for aig in (C.config1_adders(), C.config1_adders(3), C.build_multiplier_pair(5, "dadda"),
                random_aig(np.random.default_rng(3), 4, 40)):
        out = aig.outputs[0]
        m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
        W = O.num_words(L.lec_es_compile(m)[0].n)
        for wb, we in ((0, W), (W // 3, W)):
            if wb >= we:
                continue
            vars_, tt = L.lec_es_truth_tables(ctx, m, wb, we)
            exp = O.truth_tables(aig.num_pis, aig.fanins, out, [int(v) for v in vars_], wb, we)
            n = L.lec_es_compile(m)[0].n
            vm = np.uint64((1 << (1 << n)) - 1) if n < 6 else np.uint64((1 << 64) - 1)
            assert np.array_equal(tt & vm, exp & vm)


def test_config3_full_enumeration(ctx):
    """16x16 array vs Booth/Dadda: all 2^32 patterns, EQUIVALENT; the mutant's
    only failing pattern is the closed-form 2^32 - 1."""
    m = C.config3_mult16()
    r = _gpu(ctx, m, m.outputs[0], L.TIER_INTERP)
    assert r.verdict == L.EQUIVALENT and r.support_n == 32
    mm = C.config3_mult16(mutant=True)
    r = _gpu(ctx, mm, mm.outputs[0], L.TIER_INTERP)
    assert r.verdict == L.NONEQUIVALENT and r.cex == (1 << 32) - 1


def test_config3_sampled_ranges_vs_oracle(ctx):
    mm = C.config3_mult16(mutant=True)
    out = mm.outputs[0]
    W = 1 << 26
    rng = np.random.default_rng(5)
    for wb in list(rng.integers(0, W - 40, size=6)) + [W - 40]:
        wb = int(wb)
        r = _gpu(ctx, mm, out, L.TIER_INTERP, wb, wb + 40)
        assert r.cex_or_none == _oracle(mm, out, wb, wb + 40)[0]


def test_lop3_peak_measures(ctx):
    per_clk, sms, khz, rate = L.lec_es_lop3_peak(ctx)
    assert sms >= 100 and 16 <= per_clk <= 300 and 500_000 < khz < 3_000_000


def test_bounded_wait_gives_up_and_context_survives(ctx):
    """Test hook: the interpreter waits for 16 bytes its record copy never
    delivers; the bounded wait must give up (about a second), the call must
    return EDEVICE_WAIT, and the context must keep working."""
    import time
    mm = C.config1_adders(mutant_seed=1)
    m = L.miter_of(mm)
    t0 = time.time()
    with pytest.raises(L.LecEsError) as e:
        L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_INTERP, grid_blocks=1,
                                            flags=L.FLAG_TEST_WAIT_TIMEOUT))
    assert e.value.status == L.EDEVICE_WAIT
    assert time.time() - t0 < 15
    r = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_INTERP))
    assert r.cex_or_none == _oracle(mm, mm.outputs[0])[0]


@pytest.mark.parametrize("seed,reach", [(0, 32), (1, 32), (2, 48), (3, 4)])
def test_step_programs_with_run_breaks(ctx, seed, reach):
    """Cones of 256 ANDs or more run four independent records per step on
    the interpreter; where an AND reads one of the three ANDs before it the
    slot program ends the run with a load (reach 32-48: a few dozen), and a
    cone that would need more than one per 16 ANDs keeps the forwarding
    program instead (reach 4).  Every node's value (single-miter
    interpreter, breaks kept) and the lowest counterexample (single miter;
    tile queue, breaks dropped and forwarding on; served) equal the
    oracle's, over the whole space and ragged ranges."""
    rng = np.random.default_rng(900 + seed)
    for _ in range(100):  # the first seeded graph whose output cone has 300+ ANDs
        aig = narrow_aig(rng, int(rng.integers(12, 15)), int(rng.integers(600, 2000)), float(reach))
        f = aig.flat_fanins()
        ms = [L.Miter(aig.num_pis, f, o) for o in aig.outputs]
        info, recs = L.lec_es_compile(ms[0])
        if info.cone_ands >= 300:
            break
    breaks = int(((recs >> np.uint64(56)) == 1).sum())
    assert info.cone_ands >= 300 and (breaks > 3 if reach >= 32 else breaks == 0)
    assert breaks * 16 <= info.cone_ands
    W = O.num_words(info.n)
    for wb, we in ((0, W), (W // 3 + 1, W - 3)):
        vars_, tt, valid = L.lec_es_truth_tables_ex(ctx, ms[0], wb, we, L.TIER_INTERP)
        exp = O.truth_tables(aig.num_pis, aig.fanins, aig.outputs[0], [int(v) for v in vars_], wb, we)
        assert valid.all() and np.array_equal(tt, exp), (wb, we)
    want = [_oracle(aig, o)[0] for o in aig.outputs]
    n1 = L.lec_es_compile(ms[1])[0].n
    assert want[1] is not None or want[2] is not None
    assert all(x is None or x >= 7 << (n1 - 3) for x in want[1:])
    single = [L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_INTERP)).cex_or_none for m in ms]
    assert single == want
    b = L.lec_es_batch_prepare(ctx, ms, L.options(tier=L.TIER_INTERP))
    L.lec_es_batch_run_async(ctx, b)
    got = [r.cex for r in L.lec_es_batch_results(ctx, b, len(ms))]
    L.lec_es_batch_free(ctx, b)
    assert got == [L.NO_CEX if x is None else x for x in want]
    W = O.num_words(n1)
    for o in aig.outputs[1:]:
        for wb, we in ((1, W - 1), (W // 2 + 3, W)):
            r = _gpu(ctx, aig, o, L.TIER_INTERP, wb, we)
            assert r.cex_or_none == _oracle(aig, o, wb, we)[0], (wb, we)
    t = [L.lec_es_submit(ctx, m) for m in ms]
    assert [L.lec_es_wait(ctx, x, 60.0).cex_or_none for x in t] == want


def test_wide_interpreter_blocks_vs_oracle(ctx):
    """Node-pair miters with 52..68 live slots are the ones whose
    single-miter interpreter run takes a 384-thread block (at 256 threads
    their slots leave room for one block per SM, at 384 for one 12-warp
    block).  Every such miter is checked whole against the stored oracle
    result, and a sample over partial word ranges against the oracle run on
    the same range."""
    import json
    from tests.golden.make_config4_oracle import OUT, fingerprint
    pb = C.config4_pairs()
    stored = json.load(open(OUT))
    assert stored["fingerprint"] == fingerprint(pb.aig)
    f = pb.aig.flat_fanins()
    picked = []
    for i, o in enumerate(pb.aig.outputs):
        m = L.Miter(pb.aig.num_pis, f, o)
        info = L.lec_es_compile(m)[0]
        if 52 <= info.num_slots <= 68 and info.n >= 16:
            picked.append((i, m, info))
    assert len(picked) >= 20
    for i, m, _ in picked:
        r = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_INTERP))
        assert r.cex_or_none == stored["cex"][i], i
    rng = np.random.default_rng(5)
    small = [x for x in picked if x[2].n <= 22]
    for i, m, info in small[:: max(1, len(small) // 8)]:
        W = 1 << (info.n - 6)
        wb = int(rng.integers(0, W // 2))
        we = int(rng.integers(wb + 1, W + 1))
        want, _ = _oracle(pb.aig, pb.aig.outputs[i], wb, we)
        r = L.lec_es_check_ex(ctx, m, L.options(wb, we, L.TIER_INTERP))
        assert r.cex_or_none == want, (i, wb, we)
