"""GPU parity of the specialised (run-time compiled, register-resident) tier."""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx, oracle_cex
from tests.reference_eval import random_aig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lec_es_destroy(c)


def jit(ctx, aig, out, wb=0, we=L.NO_CEX):
    r = L.lec_es_check_ex(ctx, L.Miter(aig.num_pis, aig.flat_fanins(), out), L.options(wb, we, L.TIER_JIT))
    assert r.tier == L.TIER_JIT
    return r


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs(ctx, seed):
    rng = np.random.default_rng(9100 + seed)
    aig = random_aig(rng, int(rng.integers(1, 14)), int(rng.integers(1, 120)))
    out = aig.outputs[0]
    assert jit(ctx, aig, out).cex_or_none == oracle_cex(aig, out)


def test_small_supports(ctx):
    for n in range(0, 9):
        g = C.AigBuilder(10)
        x = g.and_tree([g.pi(i + 1) for i in range(n)]) if n else 0
        for neg in (0, 1):
            aig = g.finish([x ^ neg])
            assert jit(ctx, aig, x ^ neg).cex_or_none == oracle_cex(aig, x ^ neg), (n, neg)


def test_configs_1_2(ctx):
    for aig in [C.config1_adders()] + [C.config1_adders(s) for s in (1, 2, 3)] + [C.config2_mult12()] + \
               [C.config2_mult12(s) for s in (1, 2, 3)]:
        out = aig.outputs[0]
        r = jit(ctx, aig, out)
        assert r.cex_or_none == oracle_cex(aig, out)


def test_word_ranges(ctx):
    mm = C.config2_mult12(mutant_seed=1)
    out = mm.outputs[0]
    rng = np.random.default_rng(12)
    for _ in range(8):
        wb, we = sorted(int(x) for x in rng.integers(0, 1 << 18, size=2))
        if wb == we:
            continue
        assert jit(ctx, mm, out, wb, we).cex_or_none == oracle_cex(mm, out, wb, we)


def test_config3_full_and_closed_form_cex(ctx):
    m = C.config3_mult16()
    r = jit(ctx, m, m.outputs[0])
    assert r.verdict == L.EQUIVALENT
    mm = C.config3_mult16(mutant=True)
    r = jit(ctx, mm, mm.outputs[0])
    assert r.verdict == L.NONEQUIVALENT and r.cex == (1 << 32) - 1


def test_auto_picks_jit_for_big_work(ctx):
    # with the kernel held (a cold check races the interpreter against the
    # build instead: test_cold_check_races_interpreter_against_kernel_build)
    m = C.config3_mult16()
    L.lec_es_check_ex(ctx, L.miter_of(m), L.options(tier=L.TIER_JIT))
    r = L.lec_es_check(ctx, L.miter_of(m))
    assert r.tier == L.TIER_JIT and r.verdict == L.EQUIVALENT


def test_disk_cache_roundtrip(tmp_path):
    aig = C.config2_mult12(mutant_seed=2)
    out = aig.outputs[0]
    for _ in range(2):
        c = make_ctx(arena_bytes=64 << 20, jit_cache_dir=str(tmp_path))
        r = L.lec_es_check_ex(c, L.miter_of(aig), L.options(tier=L.TIER_JIT))
        assert r.cex_or_none == oracle_cex(aig, out)
        L.lec_es_destroy(c)
    assert any(p.suffix == ".cubin" for p in tmp_path.iterdir())


def test_and_form_and_table_form_agree(ctx):
    for aig in (C.config2_mult12(1), C.config2_mult12(), C.config1_adders(2)):
        m = L.miter_of(aig)
        a = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT, flags=L.FLAG_JIT_AND_FORM))
        b = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT))
        assert a.cex == b.cex == (oracle_cex(aig, aig.outputs[0]) if oracle_cex(aig, aig.outputs[0]) is not None
                                  else L.NO_CEX)


def test_grid_sizes_and_grab_balance(ctx):
    """Tiny grids (a few warps grab everything) and the default grid agree."""
    mm = C.config2_mult12(mutant_seed=3)
    m = L.miter_of(mm)
    ref = oracle_cex(mm, mm.outputs[0])
    for grid in (1, 3, 0):
        r = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT, grid_blocks=grid))
        assert r.cex_or_none == ref
    eq = C.config2_mult12()
    r = L.lec_es_check_ex(ctx, L.miter_of(eq), L.options(tier=L.TIER_JIT, grid_blocks=2))
    assert r.verdict == L.EQUIVALENT


def test_cached_kernel_skips_table_cover():
    """A second check of a cone whose kernel this context holds reuses it (the
    cover is not rebuilt) and reports the kernel's table counts; a mutant
    (different program hash) is mapped and compiled afresh."""
    c = make_ctx(arena_bytes=64 << 20)
    try:
        aig = C.config2_mult12(mutant_seed=5)
        out = aig.outputs[0]
        want = oracle_cex(aig, out)
        info0, _ = L.lec_es_compile(L.miter_of(aig))
        opt = L.options(tier=L.TIER_JIT)
        plans = []
        for _ in range(3):
            p = L.lec_es_prepare(c, L.miter_of(aig), opt)
            L.lec_es_run_async(c, p)
            r = L.lec_es_plan_result(c, p)
            assert r.tier == L.TIER_JIT and r.cex_or_none == want
            i = L.lec_es_plan_info(p)
            assert (i.num_luts, i.lut_live, i.hash) == (info0.num_luts, info0.lut_live, info0.hash)
            plans.append(p)
        for p in plans:
            L.lec_es_plan_free(c, p)
        other = C.config2_mult12(mutant_seed=6)
        r = L.lec_es_check_ex(c, L.miter_of(other), opt)
        assert r.cex_or_none == oracle_cex(other, other.outputs[0])
        good = C.config2_mult12()
        r = L.lec_es_check(c, L.miter_of(good))
        assert r.verdict == L.EQUIVALENT
    finally:
        L.lec_es_destroy(c)


@pytest.mark.parametrize("rep,hoist,nest", [("4", "0", "2"), ("16", "64", "1"), ("32", "128", "2"), ("8", "16", "3"),
                                            ("16", "128", "0"), ("16", "0", "2"), ("32", "128", "3")])
def test_passes_per_grab_and_hoisted_tables_keep_results(rep, hoist, nest, monkeypatch):
    """Every grab shape, hoisting budget and pass-loop nesting gives the
    oracle's result, including word ranges that start and end off the grab
    alignment (nested passes do not run in chunk order)."""
    monkeypatch.setenv("LEC_ES_JIT_REP", rep)
    monkeypatch.setenv("LEC_ES_JIT_HOIST", hoist)
    monkeypatch.setenv("LEC_ES_JIT_NEST", nest)
    c = make_ctx(arena_bytes=64 << 20)
    try:
        rng = np.random.default_rng(700 + int(rep) + int(hoist) + 1000 * int(nest))
        cases = [(C.config2_mult12(mutant_seed=1), None), (C.config2_mult12(), None)]
        for _ in range(4):
            a = random_aig(rng, int(rng.integers(10, 16)), int(rng.integers(40, 160)))
            cases.append((a, None))
        for aig, _ in cases:
            out = aig.outputs[0]
            m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
            r = L.lec_es_check_ex(c, m, L.options(tier=L.TIER_JIT))
            assert r.cex_or_none == oracle_cex(aig, out)
            W = 1 << max(0, r.support_n - 6)
            for wb, we in ((1, W), (W // 3 + 1, W - W // 5), (0, max(1, W // 7))):
                if wb < we:
                    g = L.lec_es_check_ex(c, m, L.options(wb, we, L.TIER_JIT))
                    assert g.cex_or_none == oracle_cex(aig, out, wb, we), (wb, we)
        mm = C.config3_mult16(mutant=True)
        r = L.lec_es_check_ex(c, L.miter_of(mm), L.options((1 << 26) - 37, 1 << 26, L.TIER_JIT))
        assert r.cex == (1 << 32) - 1
    finally:
        L.lec_es_destroy(c)


@pytest.mark.parametrize("rep,unroll", [("", "0"), ("", "4"), ("16", "2"), ("16", "4"), ("32", "4")])
def test_unrolled_pass_levels_keep_results(rep, unroll, monkeypatch):
    """Nested pass loops whose innermost levels are unrolled into copies with
    their PIs folded as constants (none, up to two or four copies): every
    verdict and lowest counterexample equals the oracle's, also over word
    ranges off the grab alignment."""
    if rep:
        monkeypatch.setenv("LEC_ES_JIT_REP", rep)
    monkeypatch.setenv("LEC_ES_JIT_UNROLL", unroll)
    c = make_ctx(arena_bytes=64 << 20)
    try:
        rng = np.random.default_rng(800 + int(unroll) + 7 * int(rep or 0))
        cases = [C.config2_mult12(), C.config2_mult12(mutant_seed=2)]
        for _ in range(3):
            cases.append(random_aig(rng, int(rng.integers(12, 17)), int(rng.integers(60, 200))))
        for aig in cases:
            out = aig.outputs[0]
            m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
            r = L.lec_es_check_ex(c, m, L.options(tier=L.TIER_JIT))
            assert r.tier == L.TIER_JIT
            assert r.cex_or_none == oracle_cex(aig, out)
            W = 1 << max(0, r.support_n - 6)
            for wb, we in ((W // 5 + 3, W - W // 7), (W // 2 - 1, W // 2 + 5)):
                wb, we = max(0, wb), min(W, we)
                if wb < we:
                    g = L.lec_es_check_ex(c, m, L.options(wb, we, L.TIER_JIT))
                    assert g.cex_or_none == oracle_cex(aig, out, wb, we), (wb, we)
        # planted 16x16 counterexamples (closed form) under the forced layout
        for p in ((1 << 31) | 0x2345, (1 << 28) | (1 << 26) | 7, 0x6A09E667):
            mm = C.config3_mult16(minterm=p)
            assert L.lec_es_check_ex(c, L.miter_of(mm), L.options(tier=L.TIER_JIT)).cex == p, hex(p)
    finally:
        L.lec_es_destroy(c)


def test_repeated_checks_see_a_changed_fanin_buffer(ctx):
    """Repeated checks of one fanin buffer reuse the cone's facts only while
    the buffer is byte-identical: after the buffer is overwritten in place
    with a mutant (same sizes and output), the result is the mutant's, as the
    oracle gives it."""
    good = C.config2_mult12()
    bad = C.config2_mult12(mutant_seed=1)
    assert good.num_ands == bad.num_ands and good.outputs == bad.outputs
    good_f = np.array(good.flat_fanins(), dtype=np.uint32).reshape(-1)  # private copies: the
    bad_f = np.array(bad.flat_fanins(), dtype=np.uint32).reshape(-1)    # buffer is written below
    m = L.Miter(good.num_pis, good_f.copy(), good.outputs[0])
    for _ in range(3):
        assert L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT)).verdict == L.EQUIVALENT
    m.fanins[:] = bad_f
    r = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT))
    assert r.cex_or_none == oracle_cex(bad, bad.outputs[0])
    m.fanins[:] = good_f
    assert L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT)).verdict == L.EQUIVALENT


def test_plan_info_reports_lop3_per_pass(ctx):
    """A specialised-kernel plan reports the lop3 its kernel executes per
    32-pattern chunk (at most one per table, fewer where tables run once per
    loop level or fold in unrolled copies); an interpreter plan reports 0."""
    m = L.miter_of(C.config2_mult12())
    p = L.lec_es_prepare(ctx, m, L.options(tier=L.TIER_JIT))
    try:
        info = L.lec_es_plan_info(p)
        assert 0 < info.lop3_per_pass <= info.num_luts
    finally:
        L.lec_es_plan_free(ctx, p)
    p = L.lec_es_prepare(ctx, m, L.options(tier=L.TIER_INTERP))
    try:
        assert L.lec_es_plan_info(p).lop3_per_pass == 0
    finally:
        L.lec_es_plan_free(ctx, p)


def test_searched_layouts_match_the_oracle(monkeypatch):
    """Cones of 1,000 tables or more get a layout chosen by dry runs of the
    generator (more pass PIs, nested and unrolled levels).  On 28-30-PI
    node-pair mutants (up to 2^24 words) that layout's lowest
    counterexample equals the oracle's over the full pattern space and over
    seeded word ranges; so does the simplest kernel form (one pass loop,
    nothing unrolled)."""
    import os
    pm = C.ProductBitMiters(seed=5)
    cases = [pm.miter(15, 22, mutant=True, mutant_seed=s) for s in (1, 2)]
    cases.append(pm.miter(14, 26, mutant=True, mutant_seed=3))
    rng = np.random.default_rng(77)
    threads = max(4, os.cpu_count() or 4)
    spans, want = [], []
    for aig, o in cases:
        info, _ = L.lec_es_compile(L.Miter(aig.num_pis, aig.flat_fanins(), o))
        W = 1 << (info.n - 6)
        rs = [(0, W)] + [tuple(sorted(int(x) for x in rng.integers(0, W, 2))) for _ in range(3)]
        spans.append(rs)
        want.append([O.check_parallel(aig.num_pis, aig.fanins, o, threads, wb, we)[0] for wb, we in rs])
    assert any(x is not None for w in want for x in w)

    def lowest(env):
        for k in ("LEC_ES_JIT_NEST", "LEC_ES_JIT_UNROLL"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        c = make_ctx(arena_bytes=64 << 20)
        try:
            out = []
            for (aig, o), ranges in zip(cases, spans):
                m = L.Miter(aig.num_pis, aig.flat_fanins(), o)
                got = []
                for wb, we in ranges:
                    r = L.lec_es_check_ex(c, m, L.options(wb, we, L.TIER_JIT))
                    assert r.tier == L.TIER_JIT
                    got.append(r.cex_or_none)
                out.append(got)
            return out
        finally:
            L.lec_es_destroy(c)

    assert lowest({}) == want
    assert lowest({"LEC_ES_JIT_NEST": "0", "LEC_ES_JIT_UNROLL": "0"}) == want


# Planted counterexamples of the 16x16 miter (the benchmark's cone plus one
# minterm): below the grab bits (lane and mask PIs), in the low and high
# grab bits, at each of the six least influential PIs b10..b15 (PIs 26..31:
# the pass PIs of its loop and unrolled levels), in pairs of them, and at
# seeded points of the whole space.
_PLANTED = ([37, (1 << 10) | 5, (1 << 14) | 0x3FF, (1 << 25) | 0xABCD]
            + [(1 << k) | 0x1234 for k in range(26, 32)]
            + [(1 << 31) | (1 << 30) | 99, (1 << 29) | (1 << 27) | (1 << 12), (1 << 30) | (1 << 26)]
            + [int(x) for x in np.random.default_rng(1616).integers(0, 1 << 32, 3)])


def test_planted_minterms_16x16_default_layout(ctx):
    """The 16x16 miter with one planted minterm fails at that pattern alone
    (closed form, pinned on the CPU).  The specialised kernel in the layout
    its search picks for the cone (the benchmark's layout: nested and
    unrolled pass levels, in-grab early exit) returns exactly that pattern
    wherever it sits, so does the default AUTO check (whichever tier it
    takes), and the oracle agrees on the 64 words around it."""
    for p in _PLANTED:
        mm = C.config3_mult16(minterm=p)
        out = mm.outputs[0]
        r = L.lec_es_check_ex(ctx, L.miter_of(mm), L.options(tier=L.TIER_JIT))
        assert r.tier == L.TIER_JIT, p
        assert r.verdict == L.NONEQUIVALENT and r.cex == p, (hex(p), hex(r.cex))
        assert L.lec_es_check(ctx, L.miter_of(mm)).cex == p
        lo = max(0, (p >> 6) - 32)
        assert oracle_cex(mm, out, lo, lo + 64) == p
        # a range that starts past p passes (UNDECIDED); one that ends at p's word misses it
        w = p >> 6
        if w + 1 < (1 << 26):
            g = L.lec_es_check_ex(ctx, L.miter_of(mm), L.options(w + 1, 1 << 26, L.TIER_JIT))
            assert g.cex_or_none is None and g.verdict == L.UNDECIDED
        if w > 0:
            g = L.lec_es_check_ex(ctx, L.miter_of(mm), L.options(0, w, L.TIER_JIT))
            assert g.cex_or_none is None
        g = L.lec_es_check_ex(ctx, L.miter_of(mm), L.options(w, w + 1, L.TIER_JIT))
        assert g.cex == p


def test_cold_check_races_interpreter_against_kernel_build():
    """A one-off AUTO check of a cone whose kernel the context does not hold
    starts on the interpreter (ascending word slices) while the kernel builds
    in the background.  Results are exact either way: the 16x16 miter is
    EQUIVALENT, and a planted 16x16 mutant and 30-PI node-pair mutants (where
    the build lands first and the kernel takes the rest of the range) give
    the closed-form or oracle counterexample.  Once built, the kernel serves
    the next check."""
    import os
    import time
    c = make_ctx(arena_bytes=256 << 20)
    try:
        m = L.miter_of(C.config3_mult16())
        r = L.lec_es_check(c, m)
        assert r.verdict == L.EQUIVALENT and r.tier in (L.TIER_INTERP, L.TIER_JIT)
        t0 = time.time()
        while time.time() - t0 < 120:  # the background build lands
            r = L.lec_es_check(c, m)
            if r.tier == L.TIER_JIT:
                break
            time.sleep(0.2)
        assert r.tier == L.TIER_JIT and r.verdict == L.EQUIVALENT
        p = (1 << 31) | 0x5EED
        mm = C.config3_mult16(minterm=p)
        assert L.lec_es_check(c, L.miter_of(mm)).cex == p
        pm = C.ProductBitMiters(seed=5)
        handed = 0
        for s in (4, 5, 6):
            aig, o = pm.miter(15, 22, mutant=True, mutant_seed=s)
            r = L.lec_es_check(c, L.Miter(aig.num_pis, aig.flat_fanins(), o))
            want = O.check_parallel(aig.num_pis, aig.fanins, o, max(4, os.cpu_count() or 4))[0]
            assert r.cex_or_none == want, s
            handed += r.tier == L.TIER_JIT
        aig, o = pm.miter(15, 22)
        r = L.lec_es_check(c, L.Miter(aig.num_pis, aig.flat_fanins(), o))
        assert r.verdict == L.EQUIVALENT
    finally:
        L.lec_es_destroy(c)


def _plant(aig, out, p):
    """aig with one more output: out XOR (the minterm of pattern p over out's
    support), so with out equivalent to 0 the only failing pattern is p."""
    from paper_2512_06627_b300.circuits import Aig
    sup, _ = O.support(aig.num_pis, aig.fanins, out)
    rows = [tuple(int(x) for x in r) for r in np.asarray(aig.fanins)]
    base = aig.num_pis + len(rows)

    def new_and(x, y):
        rows.append((x, y))
        return 2 * (aig.num_pis + len(rows))
    m = 1  # constant 1
    for k, pi in enumerate(sup):
        lit = 2 * (pi + 1) + (0 if (p >> k) & 1 else 1)
        m = lit if m == 1 else new_and(m, lit)
    x = new_and(new_and(out, m ^ 1) ^ 1, new_and(out ^ 1, m) ^ 1) ^ 1
    assert base < x // 2
    return Aig(aig.num_pis, np.array(rows, dtype=np.uint32), [x]), len(sup)


def test_grouped_passes_find_planted_minterms_in_ranges(ctx):
    """Specialised kernels of small-live cones run their passes in groups
    with one output check per group.  On equivalent 28-PI node-pair miters
    with one failing pattern planted (at low bits, in pass PIs, at the end of
    the space), the kernel returns exactly that pattern over the whole space
    and over ranges that start and end next to it (partial grabs), and
    nothing over a range that leaves it out -- the closed form, and the
    oracle's answer on the ranges."""
    import json
    from tests.golden.make_config4_oracle import OUT
    pb = C.config4_pairs()
    stored = json.load(open(OUT))["cex"]
    f = pb.aig.flat_fanins()
    picks = []
    for i, o in enumerate(pb.aig.outputs):
        if stored[i] is None and not pb.mutated[i]:
            info = L.lec_es_compile(L.Miter(pb.aig.num_pis, f, o))[0]
            if info.n == 28 and info.lut_live <= 80:
                picks.append(i)
    assert len(picks) >= 2
    for i in picks[:2]:
        for p in (12345, (1 << 20) + 7, (1 << 24) + 99, (3 << 25) + 5, (1 << 27) + (1 << 23) + 3, (1 << 28) - 1):
            aig, n = _plant(pb.aig, pb.aig.outputs[i], p)
            assert n == 28
            m = L.Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0])
            r = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_JIT))
            assert r.cex_or_none == p, (i, p)
            w = p // 64
            W = 1 << 22
            for wb, we in ((max(0, w - 3), min(W, w + 4)), (w, w + 1), (w + 1, W), (0, w)):
                if wb >= we:
                    continue
                g = L.lec_es_check_ex(ctx, m, L.options(wb, we, L.TIER_JIT))
                want = p if wb <= w < we else None
                assert g.cex_or_none == want, (i, p, wb, we)
            assert O.check(aig.num_pis, aig.fanins, aig.outputs[0], max(0, w - 3), w + 4)[0] == p


def _too_wide(n_pis, nterms, seed, planted=None):
    """An AND of `nterms` random 3-literal clauses whose tables keep too many
    values live for a specialised kernel (each clause meets a near and a far
    one); with 600 clauses over 30 PIs it is unsatisfiable.  planted: OR in
    the minterm of that pattern (its only failing pattern then)."""
    from paper_2512_06627_b300.circuits import Aig
    rng = np.random.default_rng(seed)
    rows = []

    def a(x, y):
        rows.append((x, y))
        return 2 * (n_pis + len(rows))
    terms = []
    for _ in range(nterms):
        lit = [2 * int(rng.integers(1, n_pis + 1)) + int(rng.integers(0, 2)) for _ in range(3)]
        terms.append(a(a(lit[0] ^ 1, lit[1] ^ 1), lit[2] ^ 1) ^ 1)
    acc = None
    for j in range(nterms):
        x = a(terms[j], terms[(j * 7 + nterms // 2) % nterms])
        acc = x if acc is None else a(acc, x)
    if planted is not None:
        m = None
        for k in range(n_pis):
            lit = 2 * (k + 1) + (0 if (planted >> k) & 1 else 1)
            m = lit if m is None else a(m, lit)
        acc = a(acc ^ 1, m ^ 1) ^ 1
    return Aig(n_pis, np.array(rows, dtype=np.uint32), [acc])


def test_cold_check_of_a_cone_too_wide_for_a_kernel():
    """A one-off AUTO check leaves the table cover to the background build;
    for a cone whose tables keep more values live than a kernel can hold
    that build gives up, and the interpreter's slices finish the check: the
    oracle's verdict, and the planted pattern of the variant with one."""
    import os
    c = make_ctx(arena_bytes=1 << 30)
    try:
        aig = _too_wide(30, 600, 3)
        m = L.Miter(aig.num_pis, aig.flat_fanins(), aig.outputs[0])
        info = L.lec_es_compile(m)[0]
        assert info.n == 30 and info.lut_live > 230
        want = O.check_parallel(aig.num_pis, aig.fanins, aig.outputs[0], max(4, os.cpu_count() or 4))[0]
        for _ in range(2):  # the second check finds the build given up, not a kernel
            r = L.lec_es_check(c, m)
            assert r.tier == L.TIER_INTERP and r.cex_or_none == want
        p = (1 << 29) + 123457
        mp = _too_wide(30, 600, 3, planted=p)
        r = L.lec_es_check(c, L.Miter(mp.num_pis, mp.flat_fanins(), mp.outputs[0]))
        assert want is None and r.cex_or_none == p
    finally:
        L.lec_es_destroy(c)


def test_19x19_planted_minterms_past_2_to_32_chunks(ctx):
    """A 19x19 multiplier miter has 38 PIs, so its 2^33 chunks of 32
    patterns are indexed past 2^32.  With one planted minterm the only
    counterexample is that pattern (closed form, pinned on the CPU for
    small widths); the specialised kernel returns it for minterms whose
    chunk index has bit 32 set and for the very last pattern (the whole
    space enumerated), and the oracle agrees on the 64 words around it."""
    for p in ((1 << 37) + (1 << 33) + 12345, (1 << 38) - 1):
        mm = C.build_multiplier_pair(19, tree="dadda", planted_minterm=p)
        r = jit(ctx, mm, mm.outputs[0])
        assert r.support_n == 38
        assert r.verdict == L.NONEQUIVALENT and r.cex == p, (hex(p), hex(r.cex))
        lo = max(0, (p >> 6) - 32)
        assert oracle_cex(mm, mm.outputs[0], lo, lo + 64) == p


def test_wide_live_sets_in_batch_server_and_auto(ctx):
    """Cones whose tables keep more values live than a static shared array
    holds run as specialised kernels with dynamic shared memory on every
    path: a 17x17 miter with one planted minterm (235 live tables) as a
    batch's own kernel and as a served request with the kernel held, and an
    18x18 one (about 250 live) through a default AUTO check, which starts on
    the interpreter and hands the rest of the range to the kernel when its
    build lands.  Each returns the planted pattern, the only
    counterexample."""
    p17 = (1 << 33) + 4321
    m17 = L.miter_of(C.build_multiplier_pair(17, tree="dadda", planted_minterm=p17))
    small = [L.miter_of(C.config1_adders(s)) for s in (None, 1, 2)]
    got = L.lec_es_batch(ctx, small + [m17])
    assert got[3].cex == p17 and got[3].tier == L.TIER_JIT
    assert [r.cex_or_none for r in got[:3]] == [L.lec_es_check(ctx, m).cex_or_none for m in small]
    r = L.lec_es_wait(ctx, L.lec_es_submit(ctx, m17), 600.0)
    assert r.cex == p17 and r.tier == L.TIER_JIT
    p18 = (1 << 35) + (1 << 20) + 99
    aig18 = C.build_multiplier_pair(18, tree="dadda", planted_minterm=p18)
    r = L.lec_es_check(ctx, L.miter_of(aig18))
    assert r.cex == p18 and r.support_n == 36
    lo = (p18 >> 6) - 32
    assert oracle_cex(aig18, aig18.outputs[0], lo, lo + 64) == p18
