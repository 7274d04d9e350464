"""Independent evaluators used to pin the oracle (tests only).

Neither bit-packs patterns nor shares code with the oracle: ``eval_one``
walks the graph with Python booleans for one assignment, ``eval_vectors``
keeps one numpy bool per pattern.  Both evaluate every AND of the graph in
variable order (AIGER's topological order).
"""
import numpy as np


def eval_one(aig, assignment, lits):
    """Values of ``lits`` under one assignment (bit k of ``assignment`` = PI k)."""
    val = [False] * (aig.max_var + 1)
    for k in range(aig.num_pis):
        val[k + 1] = bool((assignment >> k) & 1)
    base = aig.num_pis + 1
    for i in range(aig.num_ands):
        l0, l1 = int(aig.fanins[i, 0]), int(aig.fanins[i, 1])
        x = val[l0 >> 1] != bool(l0 & 1)
        y = val[l1 >> 1] != bool(l1 & 1)
        val[base + i] = x and y
    return [val[l >> 1] != bool(l & 1) for l in lits]


def eval_vectors(aig, patterns, lits):
    """(len(lits), len(patterns)) bool array; bit k of pattern = PI k."""
    pats = np.asarray(patterns, dtype=np.uint64)
    val = np.zeros((aig.max_var + 1, len(pats)), dtype=bool)
    for k in range(aig.num_pis):
        val[k + 1] = ((pats >> np.uint64(k)) & np.uint64(1)).astype(bool)
    base = aig.num_pis + 1
    f = aig.fanins
    for i in range(aig.num_ands):
        l0, l1 = int(f[i, 0]), int(f[i, 1])
        x = val[l0 >> 1] ^ bool(l0 & 1)
        y = val[l1 >> 1] ^ bool(l1 & 1)
        val[base + i] = x & y
    return np.stack([val[l >> 1] ^ bool(l & 1) for l in lits])


def to_int(bits):
    """Stack of output bit vectors (LSB first) -> Python-int-safe uint64 values."""
    v = np.zeros(bits.shape[1], dtype=np.uint64)
    for j in range(bits.shape[0]):
        v |= bits[j].astype(np.uint64) << np.uint64(j)
    return v


def random_aig(rng, num_pis, num_ands, p_const=0.03):
    """Random AIG with complemented edges and occasional constant fanins."""
    from paper_2512_06627_b300.circuits import Aig
    f = np.zeros((num_ands, 2), dtype=np.uint32)
    for i in range(num_ands):
        v = num_pis + 1 + i
        for e in range(2):
            if rng.random() < p_const:
                f[i, e] = rng.integers(0, 2)
            else:
                u = int(rng.integers(1, v))
                f[i, e] = 2 * u + int(rng.integers(0, 2))
    out = 2 * (num_pis + num_ands) + int(rng.integers(0, 2))
    return Aig(num_pis, f, [out])


def narrow_aig(rng, num_pis, num_ands, reach):
    """A deep, narrow random AIG (fanins mostly among the `reach` previous
    variables): its slot program, at 256 ANDs or more, needs many run-break
    loads.  Three outputs: the last AND x, and x and not-x each ANDed with
    the three highest PIs (failing patterns only in the top eighth of the
    space; at least one of the two fails)."""
    from paper_2512_06627_b300.circuits import Aig
    rows = []

    def new_and(a, b):
        rows.append((a, b))
        return 2 * (num_pis + len(rows))

    def recent():
        top = num_pis + len(rows)
        if rng.random() < 0.15 or top == num_pis:
            return 2 * int(rng.integers(1, num_pis + 1)) + int(rng.integers(0, 2))
        return 2 * max(1, top + 1 - int(rng.geometric(1.0 / reach))) + int(rng.integers(0, 2))

    while len(rows) < num_ands:  # ANDs, and XORs (three ANDs) so values stay balanced
        a, b = recent(), recent()
        if rng.random() < 0.5:
            new_and(a, b)
        else:
            new_and(new_and(a, b ^ 1) ^ 1, new_and(a ^ 1, b) ^ 1)
    last = 2 * (num_pis + len(rows))
    outs = [last]
    for start in (last, last ^ 1):
        prev = start
        for j in range(3):
            prev = new_and(prev, 2 * (num_pis - j))
        outs.append(prev)
    return Aig(num_pis, np.array(rows, dtype=np.uint32), outs)
