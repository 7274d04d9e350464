"""Test-side reference for sweeping step (1)'s candidate pairs, computed
from the oracle (tests only).

Node pairs by their definition: every AND variable's signature is its value
at the random patterns (the oracle's ``eval_patterns``); AND variables with
identical, non-constant signatures form a class; each member is paired with
the class's lowest variable; a pair is kept if the union of the two PI
supports has at most ``max_support`` PIs (supports here are plain sets
grown through the fanins in variable order, since the oracle's ``support``
stops at 63 PIs and these graphs have 64).
"""
import numpy as np

import oracle as O


def words_to_patterns(pi_words):
    """Explicit patterns (bit k = PI k): pattern 64j+b takes bit b of word j."""
    npi, nw = pi_words.shape
    pats = np.zeros(nw * 64, dtype=np.uint64)
    for k in range(npi):
        bits = np.unpackbits(np.ascontiguousarray(pi_words[k]).view(np.uint8), bitorder="little")
        pats |= bits.astype(np.uint64) << np.uint64(k)
    return pats


def pairs_from_oracle(aig, pi_words, max_support, chunk=4096):
    pats = words_to_patterns(pi_words)
    first = aig.num_pis + 1
    V = aig.max_var + 1
    classes = {}
    for v0 in range(first, V, chunk):
        vs = list(range(v0, min(V, v0 + chunk)))
        bits = O.eval_patterns(aig.num_pis, aig.fanins, pats, [2 * v for v in vs])
        packed = np.packbits(bits, axis=1)
        for v, row in zip(vs, packed):
            if not row.any() or (row == 0xFF).all():
                continue
            classes.setdefault(row.tobytes(), []).append(v)
    sup = [frozenset()] * V
    for k in range(aig.num_pis):
        sup[k + 1] = frozenset([k])
    for i in range(aig.num_ands):
        l0, l1 = int(aig.fanins[i, 0]), int(aig.fanins[i, 1])
        sup[first + i] = sup[l0 >> 1] | sup[l1 >> 1]

    def support(v):
        return sup[v]

    pairs = []
    for members in classes.values():
        rep = members[0]
        for v in members[1:]:
            if len(support(rep) | support(v)) <= max_support:
                pairs.append((rep, v))
    pairs.sort()
    return pairs
