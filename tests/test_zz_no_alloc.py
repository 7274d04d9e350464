"""The allocation-free entry point, for callers that cannot allocate device
memory (their framework's allocator owns it, or they may not allocate after
start-up).  Its output must equal the ordinary entry point's and the CPU
oracle's on the same miters and word ranges, exactly (all results are
integers), on two calls in a row: the calls share one fixed scratch array,
so the second call also checks that leftover contents do not leak into a
result.  The cases include a partial word range and a cone with more
records than shared memory holds at once (the records then stream through a
ring of stages).  This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.reference_eval import random_aig

pytestmark = pytest.mark.gpu


def _chain_aig(seed, num_pis=12, num_ands=30000, window=64, out_compl=0):
    """A deep random graph whose output cone holds every AND: AND i reads
    AND i-1 and a random node among the previous `window`, each edge
    complemented at random."""
    rng = np.random.default_rng(seed)
    f = np.zeros((num_ands, 2), dtype=np.uint32)
    for i in range(num_ands):
        v = num_pis + 1 + i
        a = v - 1
        b = int(rng.integers(max(1, v - window), v))
        f[i] = (2 * a + int(rng.integers(0, 2)), 2 * b + int(rng.integers(0, 2)))
    return C.Aig(num_pis, f, [2 * (num_pis + num_ands) + out_compl])


def _cases():
    rng = np.random.default_rng(2024)
    aigs = [C.config1_adders(1), C.config2_mult12(1), C.config2_mult12(), C.config1_adders(),
            random_aig(rng, 9, 70)]
    big = [_chain_aig(77), _chain_aig(77, out_compl=1)]  # cones of more than 28k records
    out = []
    for a in aigs + big:
        m = L.miter_of(a)
        info, _ = L.lec_es_compile(m)
        W = 1 if info.n <= 6 else 1 << (info.n - 6)
        out.append((a, m, 0, W))
    a = C.config2_mult12()
    out.append((a, L.miter_of(a), 12_345, 200_001))  # a partial range, off any alignment
    a = C.config2_mult12(2)
    out.append((a, L.miter_of(a), 7, 1 << 18))  # every miter's output is a.outputs[0]
    return out


def test_noalloc_matches_check_ex_and_oracle_twice():
    import torch
    from paper_2512_06627_b300 import build
    build.build()
    assert torch.cuda.is_available()
    ctx = L.lec_es_create(0, arena_bytes=256 << 20)
    stream = torch.cuda.current_stream()
    saw_ring = False
    try:
        for aig, m, wb, we in _cases():
            info, recs = L.lec_es_compile(m)
            saw_ring |= len(recs) > 28_000
            cap = (len(recs) + 1) & ~1
            host = np.zeros(max(2, cap), dtype=np.uint64)
            host[: len(recs)] = recs
            d_recs = torch.from_numpy(host.view(np.int64)).to("cuda")
            d_res = torch.zeros(4, dtype=torch.int64, device="cuda")
            ref = L.lec_es_check_ex(ctx, m, L.options(wb, we, tier=L.TIER_INTERP))
            want = O.check(aig.num_pis, aig.fanins, aig.outputs[0], wb, we)[0]
            assert ref.cex_or_none == want
            for _ in range(2):
                L.lec_es_check_noalloc(d_recs.data_ptr(), len(host), info, wb, we, d_res.data_ptr(),
                                       stream.cuda_stream)
                stream.synchronize()
                got = d_res.cpu().numpy().view(np.uint64)
                assert int(got[2]) == 0
                assert int(got[0]) == int(ref.cex)
                assert (None if int(got[0]) == L.NO_CEX else int(got[0])) == want
                if want is None and info.n >= 6:  # every pattern of the range evaluated
                    assert int(got[1]) == (we - wb) * 64
        assert saw_ring
    finally:
        L.lec_es_destroy(ctx)
