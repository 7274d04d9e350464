"""The ES time model on the GPU: a context folds its own full, equivalent
single runs into the fit (and only those), its predictions for miters it has
not run are close to the measured device times, and an AUTO check takes the
tier the model predicts."""
import pytest

from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def _run(ctx, m, tier, runs=1, **kw):
    """Prepare once, run `runs` times, return the last result (a second run
    times the kernel without its module's first-launch cost)."""
    opt = L.options(tier=tier, **kw)
    p = L.lec_es_prepare(ctx, m, opt)
    try:
        for _ in range(runs):
            L.lec_es_run_async(ctx, p, opt)
            r = L.lec_es_plan_result(ctx, p)
        return r
    finally:
        L.lec_es_plan_free(ctx, p)


def test_model_learns_from_full_equivalent_runs_only():
    c = make_ctx(arena_bytes=256 << 20)
    try:
        pm = C.ProductBitMiters(seed=5)
        s0 = {t: L.lec_es_cost_model(c, t).samples for t in (L.TIER_INTERP, L.TIER_JIT)}
        assert s0 == {L.TIER_INTERP: 0, L.TIER_JIT: 0}
        aig, out = pm.miter(12, 17)
        m = L.Miter(aig.num_pis, aig.flat_fanins(), out)
        for tier in (L.TIER_INTERP, L.TIER_JIT):
            r = _run(c, m, tier)
            assert r.verdict == L.EQUIVALENT and r.tier == tier
            assert L.lec_es_cost_model(c, tier).samples == 1
        # a word range, a caller's grid and a counterexample add nothing
        _run(c, m, L.TIER_INTERP, word_begin=0, word_end=4)
        _run(c, m, L.TIER_JIT, grid_blocks=2)
        bad, bout = pm.miter(12, 17, mutant=True, mutant_seed=3)
        r = _run(c, L.Miter(bad.num_pis, bad.flat_fanins(), bout), L.TIER_INTERP)
        assert r.verdict == L.NONEQUIVALENT
        assert L.lec_es_cost_model(c, L.TIER_INTERP).samples == 1
        assert L.lec_es_cost_model(c, L.TIER_JIT).samples == 1
    finally:
        L.lec_es_destroy(c)


def test_predictions_track_measured_times():
    """Learn from a few product-bit miters, predict others (different widths
    and bits) within 40% on the interpreter, or 20 us for launch-sized runs;
    the model is the paper's form plus a launch and a one-pass term, fitted
    in relative error.  The specialised kernel's time follows the lop3 it
    executes per pass, not the gates (hoisting and folded pass PIs make the
    ratio vary from cone to cone), so once the context holds a cone's kernel
    its prediction uses that figure and lands within 30%; before, by gates,
    within a factor of two."""
    c = make_ctx(arena_bytes=512 << 20)
    try:
        pm = C.ProductBitMiters(seed=5)
        def miter(w, bit):
            aig, out = pm.miter(w, bit)
            return L.Miter(aig.num_pis, aig.flat_fanins(), out)
        for w, bit in ((10, 15), (12, 12), (14, 20)):
            for tier in (L.TIER_INTERP, L.TIER_JIT):
                _run(c, miter(w, bit), tier)
        held = [(13, 19), (14, 27), (15, 22)]  # 2^26..2^30 patterns; smaller runs are launch-dominated
        for w, bit in held:
            m = miter(w, bit)
            p = L.lec_es_cost_predict(c, m, 16)
            r = _run(c, m, L.TIER_INTERP, runs=2)
            assert r.verdict == L.EQUIVALENT
            assert p.interp_ms == pytest.approx(r.device_ms, rel=0.4, abs=0.02), (w, bit, p.interp_ms, r.device_ms)
            opt = L.options(tier=L.TIER_JIT)
            plan = L.lec_es_prepare(c, m, opt)
            try:
                held_pred = L.lec_es_cost_predict(c, m, 16)  # the context holds the kernel, no run of it yet
                times = []
                for _ in range(3):  # back to back; the least is the steady time (clocks ramped up)
                    L.lec_es_run_async(c, plan, opt)
                    r = L.lec_es_plan_result(c, plan)
                    assert r.verdict == L.EQUIVALENT
                    times.append(r.device_ms)
            finally:
                L.lec_es_plan_free(c, plan)
            t = min(times)
            assert 0.5 * t - 0.02 <= p.jit_ms <= 2.0 * t + 0.02, (w, bit, p.jit_ms, times)
            assert held_pred.jit_compile_ms == 0.0
            assert held_pred.jit_ms == pytest.approx(t, rel=0.3, abs=0.02), (w, bit, held_pred.jit_ms, times)
        assert L.lec_es_cost_model(c, L.TIER_KERNEL).samples > 0
    finally:
        L.lec_es_destroy(c)


def test_auto_takes_the_predicted_tier():
    c = make_ctx(arena_bytes=256 << 20)
    try:
        for aig in (C.config1_adders(), C.config2_mult12(), C.config3_mult16()):
            m = L.miter_of(aig)
            p = L.lec_es_cost_predict(c, m, 16)
            r = L.lec_es_check(c, m)
            # a cold cone starts on the interpreter; its kernel, built in the
            # background, may take over the rest of the range
            assert r.tier == p.tier or (p.tier == L.TIER_INTERP and r.tier == L.TIER_JIT)
            assert r.verdict == L.EQUIVALENT
        # after its kernel is built the 12x12 miter goes to the kernel
        m = L.miter_of(C.config2_mult12())
        _run(c, m, L.TIER_JIT)
        p = L.lec_es_cost_predict(c, m, 16)
        assert p.jit_compile_ms == 0.0 and p.tier == L.TIER_JIT
        assert L.lec_es_check(c, m).tier == L.TIER_JIT
    finally:
        L.lec_es_destroy(c)
