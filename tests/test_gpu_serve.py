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
