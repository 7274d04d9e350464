"""The ES time model of §3.2, refit per tier as t = a + c * gates + alpha *
gates * 2^(n - 23): the fit against plain weighted least squares (numpy) with
a brute-force non-negativity rule, exact recovery, input errors, and the
host-side prediction with built-in values (including the paper's one-core
CPU model and GPU-offload rule)."""
import itertools

import numpy as np
import pytest

from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L


def _features(g, n):
    g = np.asarray(g, dtype=np.float64)
    x = g * np.exp2(np.asarray(n, dtype=np.float64) - 23.0)
    return np.stack([np.ones_like(g), g, x], axis=1)


def _nonneg_lstsq(F, t):
    """Minimise sum ((F c - t) / t)^2 over c >= 0 by trying every subset of
    free coefficients with numpy's least squares (3 unknowns: 7 subsets)."""
    A = F / t[:, None]
    y = np.ones_like(t)
    best, best_e = None, np.inf
    for k in (3, 2, 1):
        for sel in itertools.combinations(range(3), k):
            sol, *_ = np.linalg.lstsq(A[:, sel], y, rcond=None)
            if np.any(sol < 0):
                continue
            c = np.zeros(3)
            c[list(sel)] = sol
            e = np.sum((A @ c - y) ** 2)
            if best is None or e < best_e - 1e-15 * max(1.0, best_e):
                best, best_e = c, e
    return best


def test_fit_recovers_exact_coefficients():
    rng = np.random.default_rng(1)
    g = rng.integers(5, 20000, size=40)
    n = rng.integers(8, 40, size=40)
    co = np.array([0.0125, 2.5e-6, 3.5e-6])
    t = _features(g, n) @ co
    f = L.lec_es_cost_fit(g, n, t)
    assert f.samples == 40
    assert [f.a_ms, f.c_ms, f.alpha_ms] == pytest.approx(list(co), rel=1e-8)


@pytest.mark.parametrize("seed", range(6))
def test_fit_equals_nonnegative_weighted_least_squares(seed):
    rng = np.random.default_rng(10 + seed)
    k = int(rng.integers(3, 60))
    g = rng.integers(5, 6000, size=k)
    n = rng.integers(4, 36, size=k)
    F = _features(g, n)
    truth = np.array([0.01, 3e-6, 5e-6]) * rng.uniform(0.0, 2.0, size=3)
    t = np.maximum(F @ truth, 1e-4) * rng.uniform(0.7, 1.4, size=k)
    want = _nonneg_lstsq(F, t)
    f = L.lec_es_cost_fit(g, n, t)
    got = np.array([f.a_ms, f.c_ms, f.alpha_ms])
    assert np.all(got >= 0)
    A = F / t[:, None]
    err = lambda c: np.sum((A @ c - 1.0) ** 2)
    # same minimiser (up to rounding), compared by the objective and the values
    assert err(got) == pytest.approx(err(want), rel=1e-9, abs=1e-12)
    assert got == pytest.approx(want, rel=1e-6, abs=1e-12)


def test_fit_pins_negative_coefficients_at_zero():
    """Times of one pass only (no n dependence) with the n term pulling
    negative: alpha must come out exactly 0 and a, c fit the rest."""
    g = np.array([100, 200, 400, 800, 1600, 3200])
    n = np.array([30, 24, 20, 16, 12, 8])
    t = 0.01 + 1e-5 * g
    t[0] *= 0.8  # the largest x is faster than the trend
    f = L.lec_es_cost_fit(g, n, t)
    want = _nonneg_lstsq(_features(g, n), t)
    assert f.alpha_ms == 0.0 and want[2] == 0.0
    assert [f.a_ms, f.c_ms] == pytest.approx(list(want[:2]), rel=1e-9)


def test_fit_rejects_bad_input():
    with pytest.raises(L.LecEsError):
        L.lec_es_cost_fit([], [], [])
    with pytest.raises(L.LecEsError):
        L.lec_es_cost_fit([10], [64], [1.0])
    with pytest.raises(L.LecEsError):
        L.lec_es_cost_fit([10, 20], [10, 12], [1.0, 0.0])


def test_builtin_model_and_prediction_without_a_context():
    for tier in (L.TIER_INTERP, L.TIER_JIT, L.TIER_SPILL, L.TIER_COMPILE, L.TIER_KERNEL):
        f = L.lec_es_cost_model(None, tier)
        assert f.a_ms > 0 and f.samples == 0
    for tier in (0, 6):
        with pytest.raises(L.LecEsError):
            L.lec_es_cost_model(None, tier)
    fi = L.lec_es_cost_model(None, L.TIER_INTERP)
    fj = L.lec_es_cost_model(None, L.TIER_JIT)
    fc = L.lec_es_cost_model(None, L.TIER_COMPILE)
    for aig, threads in ((C.config3_mult16(), 16), (C.config2_mult12(), 16), (C.config1_adders(), 16)):
        m = L.miter_of(aig)
        info, _ = L.lec_es_compile(m)
        p = L.lec_es_cost_predict(None, m, threads)
        assert (p.gates, p.n, p.num_luts) == (info.cone_ands, info.n, info.num_luts)
        g = info.cone_ands
        x = g * 2.0 ** (info.n - 23)
        assert p.interp_ms == pytest.approx(fi.a_ms + fi.c_ms * g + fi.alpha_ms * x, rel=1e-12)
        assert p.jit_ms == pytest.approx(fj.a_ms + fj.c_ms * g + fj.alpha_ms * x, rel=1e-12)
        assert p.jit_compile_ms == pytest.approx(fc.a_ms + fc.c_ms * info.num_luts, rel=1e-12)
        # the paper's one-core CPU model and GPU-offload rule (§3.2 footnote values)
        assert p.paper_cpu_s == pytest.approx(0.0003 * x, rel=1e-12)
        assert p.gpu_offload == int(0.0003 * x / threads > 0.1)
        want = L.TIER_JIT if p.jit_ms + p.jit_compile_ms < p.interp_ms else L.TIER_INTERP
        assert p.tier == want
    # 16x16: 759 s on one core by the paper's model -> offloaded; the adders are not
    big = L.lec_es_cost_predict(None, L.miter_of(C.config3_mult16()), 16)
    assert big.gpu_offload == 1 and big.tier == L.TIER_JIT
    small = L.lec_es_cost_predict(None, L.miter_of(C.config1_adders()), 16)
    assert small.gpu_offload == 0 and small.tier == L.TIER_INTERP
