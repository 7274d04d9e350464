"""The allocation-free entry point, for callers that cannot allocate device
memory (their framework's allocator owns it, or they may not allocate after
start-up).  Its output must equal the ordinary entry point's on the same
miters, exactly (all results are integers), on two calls in a row: the
calls share one fixed scratch array, so the second call also checks that
leftover contents do not leak into a result.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.reference_eval import random_aig

pytestmark = pytest.mark.gpu


def _miters():
    rng = np.random.default_rng(2024)
    aigs = [C.config1_adders(1), C.config2_mult12(1), C.config2_mult12(), C.config1_adders(),
            random_aig(rng, 9, 70)]
    return [L.miter_of(a) for a in aigs]


def test_noalloc_matches_check_ex_twice():
    import torch
    from paper_2512_06627_b300 import build
    build.build()
    assert torch.cuda.is_available()
    ctx = L.lec_es_create(0, arena_bytes=256 << 20)
    stream = torch.cuda.current_stream()
    try:
        for m in _miters():
            info, recs = L.lec_es_compile(m)
            cap = (len(recs) + 1) & ~1
            host = np.zeros(max(2, cap), dtype=np.uint64)
            host[: len(recs)] = recs
            d_recs = torch.from_numpy(host.view(np.int64)).to("cuda")
            d_res = torch.zeros(4, dtype=torch.int64, device="cuda")
            W = 1 if info.n <= 6 else 1 << (info.n - 6)
            ref = L.lec_es_check_ex(ctx, m, L.options(tier=L.TIER_INTERP))
            for _ in range(2):
                L.lec_es_check_noalloc(d_recs.data_ptr(), len(host), info, 0, W, d_res.data_ptr(),
                                       stream.cuda_stream)
                stream.synchronize()
                got = d_res.cpu().numpy().view(np.uint64)
                assert int(got[2]) == 0
                assert int(got[0]) == int(ref.cex)
    finally:
        L.lec_es_destroy(ctx)
