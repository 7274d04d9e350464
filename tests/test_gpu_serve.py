"""Served ES: requests admitted while others run give the same result as
alone; cancellation, timeouts and a tight slot budget behave."""
import time

import numpy as np
import pytest

from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx, oracle_cex
from tests.reference_eval import random_aig

pytestmark = pytest.mark.gpu


def _mix():
    pm = C.ProductBitMiters(seed=5)
    items = []
    for w, bit, mut in [(8, 9, False), (8, 12, True), (9, 10, False), (10, 15, False), (10, 11, True),
                        (11, 12, False), (12, 20, False), (12, 13, True)]:
        aig, out = pm.miter(w, bit, mut)
        items.append((aig, out))
    for a in (C.config1_adders(), C.config1_adders(1), C.config2_mult12(2)):
        items.append((a, a.outputs[0]))
    rng = np.random.default_rng(4)
    for _ in range(12):
        a = random_aig(rng, int(rng.integers(1, 14)), int(rng.integers(1, 90)))
        items.append((a, a.outputs[0]))
    return items


def test_alone_equals_in_mix():
    ctx = make_ctx()
    items = _mix()
    ms = [L.Miter(a.num_pis, a.flat_fanins(), o) for a, o in items]
    alone = [L.lec_es_check(ctx, m).cex for m in ms]
    tickets = []
    for i, m in enumerate(ms):
        tickets.append(L.lec_es_submit(ctx, m))
        if i % 5 == 0:
            time.sleep(0.002)  # arrivals while earlier requests run
    mixed = [L.lec_es_wait(ctx, t, 120.0) for t in tickets]
    assert [r.cex for r in mixed] == alone
    for (a, o), r in zip(items[:11], mixed[:11]):
        assert r.cex_or_none == oracle_cex(a, o)
    assert all(r.latency_ms > 0 for r in mixed)
    L.lec_es_destroy(ctx)


def test_tight_budget_still_completes():
    ctx = make_ctx()
    L.lec_es_server_config(ctx, 1 << 20, 2)
    items = _mix()[:8]
    ms = [L.Miter(a.num_pis, a.flat_fanins(), o) for a, o in items]
    ts = [L.lec_es_submit(ctx, m) for m in ms]
    got = [L.lec_es_wait(ctx, t, 120.0).cex for t in ts]
    assert got == [L.lec_es_check(ctx, m).cex for m in ms]
    L.lec_es_destroy(ctx)


def test_cancel_timeout_and_unknown_ticket():
    ctx = make_ctx()
    big = C.config3_mult16()
    m = L.miter_of(big)
    t = L.lec_es_submit(ctx, m)
    with pytest.raises(L.LecEsError) as e:
        L.lec_es_wait(ctx, t, 0.001)
    assert e.value.status == L.ETIMEOUT
    L.lec_es_cancel(ctx, t)
    t0 = time.time()
    with pytest.raises(L.LecEsError) as e:
        L.lec_es_wait(ctx, t, 60.0)
    assert e.value.status == L.ECANCELLED
    assert time.time() - t0 < 30
    with pytest.raises(L.LecEsError) as e:
        L.lec_es_poll(ctx, 987654321)
    assert e.value.status == L.ENOTFOUND
    # a queued request can be cancelled before it runs, others still finish
    small = L.miter_of(C.config1_adders(1))
    t1 = L.lec_es_submit(ctx, small)
    r = L.lec_es_wait(ctx, t1, 60.0)
    assert r.cex_or_none == oracle_cex(C.config1_adders(1), C.config1_adders(1).outputs[0])
    L.lec_es_destroy(ctx)


def test_cancel_then_resubmit_resident_program():
    """Cancelling a running request zeroes its counterexample word on a
    control stream; the result slot it frees is reused at once by the next
    request.  With the small program already resident (no upload, no sync
    on admission), the next requests must still get their own verdicts:
    every equivalent request EQUIVALENT and every mutant the oracle's cex."""
    ctx = make_ctx()
    L.lec_es_server_config(ctx, 32 << 30, 2)  # two result slots: the freed one is reused at once
    good_a = C.config1_adders()
    bad_a = C.config1_adders(1)
    good, bad = L.miter_of(good_a), L.miter_of(bad_a)
    want_bad = oracle_cex(bad_a, bad_a.outputs[0])
    for m in (good, bad):  # make both programs resident on the server
        L.lec_es_wait(ctx, L.lec_es_submit(ctx, m), 60.0)
    pm = C.ProductBitMiters(seed=5)
    big_aig, big_out = pm.miter(18, 26)  # 2^36 patterns: still running when the cancel comes
    big = L.Miter(big_aig.num_pis, big_aig.flat_fanins(), big_out)
    cancelled = 0
    for i in range(40):
        t = L.lec_es_submit(ctx, big)
        time.sleep(0.0005 * (i % 4))
        L.lec_es_cancel(ctx, t)
        ts = [L.lec_es_submit(ctx, good if j % 2 == 0 else bad) for j in range(4)]
        try:
            assert L.lec_es_wait(ctx, t, 120.0).verdict == L.EQUIVALENT  # finished before the cancel landed
        except L.LecEsError as e:
            assert e.status == L.ECANCELLED
            cancelled += 1
        got = [L.lec_es_wait(ctx, x, 60.0) for x in ts]
        assert [r.verdict for r in got] == [L.EQUIVALENT, L.NONEQUIVALENT] * 2, i
        assert got[1].cex == want_bad and got[3].cex == want_bad
    assert cancelled >= 20
    L.lec_es_destroy(ctx)


def test_submit_copies_the_cone_before_returning():
    """lec_es_submit keeps its own copy of the miter's cone: overwriting the
    caller's fanin buffer right after submitting does not change the result,
    which equals the oracle's for the original miter.  Many small node-pair
    cones of one large shared graph, submitted at once, come back equal to
    one lec_es_check each."""
    ctx = make_ctx()
    try:
        good = C.config2_mult12()
        bad = C.config2_mult12(mutant_seed=1)
        f = np.array(good.flat_fanins(), dtype=np.uint32).reshape(-1)
        m = L.Miter(good.num_pis, f, good.outputs[0])
        t = L.lec_es_submit(ctx, m)
        m.fanins[:] = np.array(bad.flat_fanins(), dtype=np.uint32).reshape(-1)
        assert L.lec_es_wait(ctx, t, 120.0).verdict == L.EQUIVALENT
        t = L.lec_es_submit(ctx, m)  # now the mutant
        m.fanins[:] = np.array(good.flat_fanins(), dtype=np.uint32).reshape(-1)
        assert L.lec_es_wait(ctx, t, 120.0).cex_or_none == oracle_cex(bad, bad.outputs[0])
        pb = C.config4_pairs(num_pairs=512)
        fan = pb.aig.flat_fanins()
        ms = [L.Miter(pb.aig.num_pis, fan, o) for o in pb.aig.outputs]
        ts = [L.lec_es_submit(ctx, x) for x in ms]
        got = [L.lec_es_wait(ctx, x, 300.0) for x in ts]
        alone = [L.lec_es_check(ctx, x) for x in ms]
        assert [r.cex for r in got] == [r.cex for r in alone]
        many = [L.lec_es_wait(ctx, x, 300.0) for x in L.lec_es_submit_many(ctx, ms)]  # one call for all
        assert [r.cex for r in many] == [r.cex for r in alone]
        assert [list(r.support[: r.support_n]) for r in got] == [list(r.support[: r.support_n]) for r in alone]
        for j in range(0, 512, 37):
            o = pb.aig.outputs[j]
            assert got[j].cex_or_none == oracle_cex(pb.aig, o)
    finally:
        L.lec_es_destroy(ctx)
