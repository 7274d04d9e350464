"""Shared GPU-test helpers."""
import pytest

import oracle as O
from paper_2512_06627_b300 import lec_es as L


def make_ctx(arena_bytes=4 << 30, jit_cache_dir=None):
    import torch
    assert torch.cuda.is_available()
    from paper_2512_06627_b300 import build
    build.build()
    return L.lec_es_create(0, arena_bytes=arena_bytes, jit_cache_dir=jit_cache_dir)


def oracle_cex(aig, out, wb=0, we=None):
    return O.check(aig.num_pis, aig.fanins, out, wb, O.NONE if we is None else we)[0]
