"""Batched ES: one persistent launch over (miter, word-range) tiles gives,
for every miter, exactly the single-miter result (and the oracle's)."""
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


def test_mixed_batch_vs_oracle(ctx):
    aigs = [C.config1_adders(), C.config1_adders(1), C.config2_mult12(), C.config2_mult12(1),
            C.build_multiplier_pair(6, "dadda")]
    rng = np.random.default_rng(77)
    aigs += [random_aig(rng, int(rng.integers(1, 14)), int(rng.integers(1, 100))) for _ in range(40)]
    ms = [L.miter_of(a) for a in aigs]
    res = L.lec_es_batch(ctx, ms)
    for a, r in zip(aigs, res):
        assert r.cex_or_none == oracle_cex(a, a.outputs[0])
        assert r.verdict == (L.EQUIVALENT if r.cex_or_none is None else L.NONEQUIVALENT)


@pytest.fixture(scope="module")
def pairs():
    return C.config4_pairs()


def test_node_pairs_small_support_vs_oracle(ctx, pairs):
    f = pairs.aig.flat_fanins()
    sel = [i for i, s in enumerate(pairs.support_sizes) if s <= 18][:600]
    sel += [i for i, m in enumerate(pairs.mutated) if m and pairs.support_sizes[i] <= 22]
    sel = sorted(set(sel))
    ms = [L.Miter(pairs.aig.num_pis, f, pairs.aig.outputs[i]) for i in sel]
    res = L.lec_es_batch(ctx, ms)
    for i, r in zip(sel, res):
        assert r.cex_or_none == oracle_cex(pairs.aig, pairs.aig.outputs[i]), i


def test_full_4096_pairs_batch_equals_single(ctx, pairs):
    """All 4096 node-pair miters in one launch; each equals its own
    single-miter run (graph replayed twice)."""
    f = pairs.aig.flat_fanins()
    ms = [L.Miter(pairs.aig.num_pis, f, o) for o in pairs.aig.outputs]
    b = L.lec_es_batch_prepare(ctx, ms)
    outs = []
    for _ in range(2):
        L.lec_es_batch_run_async(ctx, b)
        outs.append([r.cex for r in L.lec_es_batch_results(ctx, b, len(ms))])
    L.lec_es_batch_free(ctx, b)
    assert outs[0] == outs[1]
    single = [L.lec_es_check(ctx, m).cex for m in ms]
    assert outs[0] == single
    nonequiv = sum(1 for x in single if x != L.NO_CEX)
    assert nonequiv >= sum(pairs.mutated) // 2
    # every miter against the oracle (its results stored by
    # tests/golden/make_config4_oracle.py; the fingerprint pins the inputs)
    import json
    from tests.golden.make_config4_oracle import OUT, fingerprint
    stored = json.load(open(OUT))
    assert stored["fingerprint"] == fingerprint(pairs.aig)
    assert outs[0] == [L.NO_CEX if x is None else x for x in stored["cex"]]


def test_layouts_and_autotune_give_identical_results(ctx, pairs, tmp_path):
    """Every tile layout (threads per pass, tiles per block slot, staging
    depth) and the autotuned one give the same result for every miter."""
    f = pairs.aig.flat_fanins()
    sel = list(range(0, 4096, 5))
    ms = [L.Miter(pairs.aig.num_pis, f, pairs.aig.outputs[i]) for i in sel]
    ref = None
    # blocks need not be powers of two; 512 threads do not fit this selection's
    # largest live set, so the library steps down by 32 to a block that fits
    for blk, gran, ring in [(256, 16, 256), (128, 4, 128), (64, 64, 1024), (256, 1, 2), (224, 16, 256),
                            (160, 4, 128), (96, 16, 256), (512, 16, 256)]:
        b = L.lec_es_batch_prepare(ctx, ms, L.options(tier=L.TIER_INTERP, block_threads=blk,
                                                       tile_granularity=gran, stage_records=ring))
        info = L.lec_es_batch_info(b)
        assert info.stage_records == ring and info.tile_granularity == gran
        if blk < 512:
            assert info.block_threads == blk
        else:
            assert 64 <= info.block_threads < 512 and info.block_threads % 32 == 0
        L.lec_es_batch_run_async(ctx, b)
        got = [r.cex for r in L.lec_es_batch_results(ctx, b, len(ms))]
        L.lec_es_batch_free(ctx, b)
        ref = got if ref is None else ref
        assert got == ref
    tuned = L.lec_es_create(0, arena_bytes=1 << 30, jit_cache_dir=str(tmp_path))
    b = L.lec_es_batch_prepare(tuned, ms, L.options(flags=L.FLAG_AUTOTUNE))
    info = L.lec_es_batch_info(b)
    assert info.block_threads % 32 == 0 and 64 <= info.block_threads <= 512
    assert info.tile_granularity in (4, 8, 16, 64)
    L.lec_es_batch_run_async(tuned, b)
    assert [r.cex for r in L.lec_es_batch_results(tuned, b, len(ms))] == ref
    L.lec_es_batch_free(tuned, b)
    assert (tmp_path / "batch_layouts.txt").exists()
    L.lec_es_destroy(tuned)


def test_every_mutated_pair_and_sampled_ranges_of_heavy_pairs_vs_oracle(ctx, pairs):
    """At the full batch size: every mutated node-pair miter (any support,
    up to 28 PIs) gets the oracle's lowest counterexample from the batch;
    for heavy equivalent miters (the ones on specialised kernels), random
    word ranges are checked by both the GPU and the oracle."""
    import numpy as np
    f = pairs.aig.flat_fanins()
    ms = [L.Miter(pairs.aig.num_pis, f, o) for o in pairs.aig.outputs]
    res = L.lec_es_batch(ctx, ms)
    for i, mut in enumerate(pairs.mutated):
        if mut:
            assert res[i].cex_or_none == oracle_cex(pairs.aig, pairs.aig.outputs[i]), i
    heavy = [i for i, r in enumerate(res) if r.tier == L.TIER_JIT and not pairs.mutated[i]]
    assert len(heavy) > 100
    rng = np.random.default_rng(21)
    for i in rng.choice(heavy, size=24, replace=False):
        W = 1 << max(0, pairs.support_sizes[i] - 6)
        wb = int(rng.integers(0, max(1, W - 1024)))
        we = min(W, wb + 1024)
        g = L.lec_es_check_ex(ctx, ms[i], L.options(wb, we, L.TIER_JIT))
        assert g.cex_or_none == oracle_cex(pairs.aig, pairs.aig.outputs[i], wb, we), (i, wb, we)


def test_spread_batch_equals_single_and_oracle():
    """The batched workload at its stated spread (10..28 PIs, node pairs up
    to whole four-multiplier miters): one prepared batch gives every miter's
    lec_es_check result, and the oracle's -- all 1,024 against the oracle's
    stored results (tests/golden/make_spread_oracle.py; the fingerprint pins
    the inputs), and live on every miter of up to 16 PIs, every mutant and a
    seeded sample of the rest."""
    import os
    from tests.gpu_common import make_ctx
    ctx = make_ctx()
    try:
        trip = C.config4_spread(num=1024, seed=9)
        flat = {}
        ms = []
        for aig, out, _ in trip:
            f = flat.setdefault(id(aig), aig.flat_fanins())
            ms.append(L.Miter(aig.num_pis, f, out))
        got = L.lec_es_batch(ctx, ms)
        one = [L.lec_es_check(ctx, m) for m in ms]
        assert [r.cex for r in got] == [r.cex for r in one]
        rng = np.random.default_rng(33)
        sample = set(int(x) for x in rng.choice(len(ms), size=10, replace=False))
        threads = max(4, os.cpu_count() or 4)
        checked = 0
        for i, ((aig, out, _), r) in enumerate(zip(trip, got)):
            if r.support_n <= 16 or r.cex_or_none is not None or i in sample:
                want = O.check_parallel(aig.num_pis, aig.fanins, out, threads)[0]
                assert r.cex_or_none == want, i
                checked += 1
        assert checked >= 20 and any(r.cex_or_none is not None for r in got)
        import json
        from tests.golden.make_spread_oracle import NUM, OUT, SEED, fingerprint
        assert (NUM, SEED) == (1024, 9)
        stored = json.load(open(OUT))
        assert stored["fingerprint"] == fingerprint(trip)
        assert [r.cex_or_none for r in got] == stored["cex"]
    finally:
        L.lec_es_destroy(ctx)
