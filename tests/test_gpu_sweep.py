"""Sweeping step (1) on the GPU: random-simulation signatures and candidate
pairs.  Signatures must equal the oracle's evaluation of every node at the
same patterns (bit-exact); the candidate pairs must equal the pairing
defined from the oracle's evaluation of every node at the same patterns
(tests/reference_pairs.py)."""
import numpy as np
import pytest

import oracle as O
from paper_2512_06627_b300 import circuits as C
from paper_2512_06627_b300 import lec_es as L
from tests.gpu_common import make_ctx
from tests.reference_eval import random_aig
from tests.reference_pairs import pairs_from_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    L.lec_es_destroy(c)


def _patterns(pi_words):
    """Explicit patterns (bit k = PI k) of the words: pattern 64j+b takes bit b of word j."""
    npi, nw = pi_words.shape
    pats = np.zeros(nw * 64, dtype=np.uint64)
    for k in range(npi):
        bits = np.unpackbits(pi_words[k].view(np.uint8), bitorder="little").astype(np.uint64)
        pats |= bits << np.uint64(k)
    return pats


@pytest.mark.parametrize("seed", range(4))
def test_signatures_match_oracle_random_graphs(ctx, seed):
    rng = np.random.default_rng(300 + seed)
    aig = random_aig(rng, int(rng.integers(2, 40)), int(rng.integers(1, 300)))
    nw = int(rng.integers(1, 70))
    pw = rng.integers(0, 2**63, size=(aig.num_pis, nw), dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=(aig.num_pis, nw), dtype=np.uint64)
    sig, h = L.lec_es_signatures(ctx, aig.num_pis, aig.flat_fanins(), pw)
    V = aig.max_var + 1
    bits = O.eval_patterns(aig.num_pis, aig.fanins, _patterns(pw), [2 * v for v in range(V)])
    exp = np.packbits(bits.reshape(V, nw, 64), axis=2, bitorder="little").view("<u8").reshape(V, nw)
    assert np.array_equal(sig, exp)
    # equal signatures, equal hashes
    for v in range(V):
        for u in range(v):
            if np.array_equal(sig[u], sig[v]):
                assert h[u] == h[v]


def test_signatures_32x32_pair_graph_sampled(ctx):
    base = C.build_golden_revised_multipliers(32)
    pw = C.signature_words(base, 64, 4)
    sig, h = L.lec_es_signatures(ctx, base.num_pis, base.flat_fanins(), pw)
    rng = np.random.default_rng(9)
    vs = sorted(set(rng.integers(base.num_pis + 1, base.max_var + 1, size=400).tolist()))
    bits = O.eval_patterns(base.num_pis, base.fanins, _patterns(pw)[:1024], [2 * v for v in vs])
    got = np.unpackbits(sig[vs][:, :16].copy().view(np.uint8), axis=1, bitorder="little").astype(bool)
    assert np.array_equal(got, bits)


def test_pairs_equal_oracle_pairing(ctx):
    """The GPU matcher's pairs on the 32x32 four-multiplier graph equal the
    pairs defined from the oracle's own evaluation of every node at the same
    random patterns (tests/reference_pairs.py)."""
    base = C.build_golden_revised_multipliers(32)
    pw = C.signature_words(base, 64, 4)
    gpu = L.lec_es_match_pairs(ctx, base.num_pis, base.flat_fanins(), pw, 28)
    ref = pairs_from_oracle(base, pw, 28)
    assert gpu == ref and len(gpu) == 4238


@pytest.mark.parametrize("seed", range(3))
def test_pairs_equal_oracle_pairing_random_graphs(ctx, seed):
    rng = np.random.default_rng(500 + seed)
    aig = random_aig(rng, int(rng.integers(4, 20)), int(rng.integers(50, 400)))
    pw = rng.integers(0, 2**63, size=(aig.num_pis, 3), dtype=np.uint64)
    for ms in (4, 8, 64):
        gpu = L.lec_es_match_pairs(ctx, aig.num_pis, aig.flat_fanins(), pw, ms)
        assert gpu == pairs_from_oracle(aig, pw, ms), ms
