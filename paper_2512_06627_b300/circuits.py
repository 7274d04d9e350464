"""Seeded input generators for exact simulation: datapath AIGs, miters and mutants.

This module builds the *inputs* of the exact-simulation (ES) engine and nothing
else.  It holds none of the engine's arithmetic: it does not extract cones for
the checker, assign value slots, or enumerate input patterns.  Both the CPU
oracle (``oracle/``) and the CUDA path receive the arrays produced here.

Representation (AIGER conventions, "Combinational Equivalence Checking", §2.1
of the paper: latch-free And-Inverter Graphs):

* variable 0 is constant FALSE; variables ``1..num_pis`` are primary inputs;
  AND variables follow in topological order (each fanin variable is smaller
  than the AND's own variable);
* a literal is ``2*var + complement``.

Generators (inputs of the paper's multiplier/adder miter workloads, Table 1):
ripple-carry and Kogge-Stone adders, array multiplier (AND partial products,
ripple-carry rows), unsigned radix-4 Booth multiplier with Wallace or Dadda
reduction and a Kogge-Stone final adder.  The miter follows §2.1: corresponding
outputs are XORed pairwise and the XORs ORed into one output, which is
identically zero iff the two circuits are equivalent.

The random simulator below exists only to *select* inputs: node pairs with equal
64-word signatures (step (1) of the sweeping flow, §2.3) and to redraw a
seeded single-edge inversion that random patterns cannot observe.  It is not
used to decide any result.
"""
from __future__ import annotations

import dataclasses
import struct
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------
# AIG container and builder
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Aig:
    """A combinational AIG.  ``fanins`` is a (num_ands, 2) uint32 array."""

    num_pis: int
    fanins: np.ndarray
    outputs: List[int]
    # optional bookkeeping: AND-variable ranges that belong to each side
    side_ranges: Dict[str, Tuple[int, int]] = dataclasses.field(default_factory=dict)
    side_outputs: Dict[str, List[int]] = dataclasses.field(default_factory=dict)

    @property
    def num_ands(self) -> int:
        return int(self.fanins.shape[0])

    @property
    def max_var(self) -> int:
        return self.num_pis + self.num_ands

    def flat_fanins(self) -> np.ndarray:
        """Contiguous uint32 array of 2*num_ands literals (C-ABI layout)."""
        return np.ascontiguousarray(self.fanins.reshape(-1), dtype=np.uint32)


class AigBuilder:
    """Incremental AIG construction with constant folding and scoped hashing.

    Structural hashing (strash) merges identical AND(a, b) nodes.  ``new_scope``
    starts a fresh hash table, so two sides built in different scopes share
    only their primary inputs (the "no structural hashing across the two
    sides" setting of the 16x16 workload).
    """

    def __init__(self, num_pis: int, strash: bool = True, style: str = "plain"):
        assert style in ("plain", "alt")
        self.style = style
        self.num_pis = num_pis
        self.f0: List[int] = []
        self.f1: List[int] = []
        self.use_strash = strash
        self.table: Dict[Tuple[int, int], int] = {}

    # literals -----------------------------------------------------------
    def pi(self, k: int) -> int:
        assert 0 <= k < self.num_pis
        return 2 * (k + 1)

    def new_scope(self) -> None:
        self.table = {}

    @property
    def next_var(self) -> int:
        return self.num_pis + 1 + len(self.f0)

    # gates --------------------------------------------------------------
    def AND(self, a: int, b: int) -> int:
        if a > b:
            a, b = b, a
        if a == 0:
            return 0
        if a == 1:
            return b
        if a == b:
            return a
        if (a ^ 1) == b:
            return 0
        key = (a, b)
        if self.use_strash:
            hit = self.table.get(key)
            if hit is not None:
                return hit
        lit = 2 * self.next_var
        self.f0.append(a)
        self.f1.append(b)
        if self.use_strash:
            self.table[key] = lit
        return lit

    def OR(self, a: int, b: int) -> int:
        return self.AND(a ^ 1, b ^ 1) ^ 1

    def XOR(self, a: int, b: int) -> int:
        if self.style == "alt":
            # (a | b) & ~(a & b): the same function, a different three-AND form
            return self.AND(self.OR(a, b), self.AND(a, b) ^ 1)
        # (a & ~b) | (~a & b), three ANDs
        return self.OR(self.AND(a, b ^ 1), self.AND(a ^ 1, b))

    def full_adder(self, a: int, b: int, c: int) -> Tuple[int, int]:
        t = self.XOR(a, b)
        s = self.XOR(t, c)
        if self.style == "alt":
            co = self.OR(self.OR(self.AND(a, b), self.AND(a, c)), self.AND(b, c))
        else:
            co = self.OR(self.AND(a, b), self.AND(c, t))
        return s, co

    def half_adder(self, a: int, b: int) -> Tuple[int, int]:
        return self.XOR(a, b), self.AND(a, b)

    def or_tree(self, lits: Sequence[int]) -> int:
        lits = list(lits)
        if not lits:
            return 0
        while len(lits) > 1:
            nxt = [self.OR(lits[i], lits[i + 1]) for i in range(0, len(lits) - 1, 2)]
            if len(lits) % 2:
                nxt.append(lits[-1])
            lits = nxt
        return lits[0]

    def and_tree(self, lits: Sequence[int]) -> int:
        lits = list(lits)
        if not lits:
            return 1
        while len(lits) > 1:
            nxt = [self.AND(lits[i], lits[i + 1]) for i in range(0, len(lits) - 1, 2)]
            if len(lits) % 2:
                nxt.append(lits[-1])
            lits = nxt
        return lits[0]

    def finish(self, outputs: Sequence[int], **extra) -> Aig:
        f = np.zeros((len(self.f0), 2), dtype=np.uint32)
        if self.f0:
            f[:, 0] = self.f0
            f[:, 1] = self.f1
        return Aig(self.num_pis, f, list(outputs), **extra)


# ----------------------------------------------------------------------------
# Adders
# ----------------------------------------------------------------------------

def ripple_carry_adder(g: AigBuilder, x: Sequence[int], y: Sequence[int], cin: int = 0) -> List[int]:
    """w-bit ripple-carry adder; returns w+1 sum bits (carry-out last)."""
    assert len(x) == len(y)
    c = cin
    out = []
    for xi, yi in zip(x, y):
        s, c = g.full_adder(xi, yi, c)
        out.append(s)
    out.append(c)
    return out


def kogge_stone_adder(g: AigBuilder, x: Sequence[int], y: Sequence[int]) -> List[int]:
    """w-bit Kogge-Stone parallel-prefix adder; returns w+1 sum bits."""
    w = len(x)
    assert len(y) == w and w >= 1
    gen = [g.AND(a, b) for a, b in zip(x, y)]
    prop = [g.XOR(a, b) for a, b in zip(x, y)]
    G, P = list(gen), list(prop)
    d = 1
    while d < w:
        nG, nP = list(G), list(P)
        for i in range(d, w):
            nG[i] = g.OR(G[i], g.AND(P[i], G[i - d]))
            if i >= 2 * d:  # group propagate is only needed while spans grow
                nP[i] = g.AND(P[i], P[i - d])
        G, P = nG, nP
        d *= 2
    s = [prop[0]] + [g.XOR(prop[i], G[i - 1]) for i in range(1, w)]
    return s + [G[w - 1]]


# ----------------------------------------------------------------------------
# Multipliers
# ----------------------------------------------------------------------------

def array_multiplier(g: AigBuilder, a: Sequence[int], b: Sequence[int]) -> List[int]:
    """Unsigned w x w array multiplier: AND partial products, one ripple-carry
    row per multiplier bit.  Returns the 2w product bits (LSB first)."""
    w = len(a)
    assert len(b) == w
    acc = [g.AND(a[j], b[0]) for j in range(w)]
    for i in range(1, w):
        row = [g.AND(a[j], b[i]) for j in range(w)]
        hi = acc[i:]
        hi = hi + [0] * (w - len(hi))
        acc = acc[:i] + ripple_carry_adder(g, hi, row)
    return acc[: 2 * w]


def booth_partial_products(g: AigBuilder, a: Sequence[int], b: Sequence[int]) -> List[List[int]]:
    """Unsigned radix-4 Booth recoding.  Returns bit columns (weight 2^j) whose
    sum is a*b modulo 2^(2w).

    Digit i looks at (b[2i+1], b[2i], b[2i-1]) with b[-1] = b[k>=w] = 0; there
    are w//2+1 digits so the top digit is never negative.  For a digit d with
    magnitude M = |d|*a (w+1 bits) and sign bit s, the partial product is
    X + s - s*2^(w+1) where X = M xor s (bitwise).  Rewriting -s*2^(w+1) as
    (not s)*2^(w+1) - 2^(w+1) moves every sign into one bit per row plus one
    constant  -sum_i 2^(w+1+2i)  added into the columns.
    """
    w = len(a)
    W = 2 * w
    cols: List[List[int]] = [[] for _ in range(W)]

    def bb(k: int) -> int:
        return b[k] if 0 <= k < w else 0

    def aa(k: int) -> int:
        return a[k] if 0 <= k < w else 0

    D = w // 2 + 1
    const = 0
    for i in range(D):
        x2, x1, x0 = bb(2 * i + 1), bb(2 * i), bb(2 * i - 1)
        one = g.XOR(x1, x0)
        two = g.OR(g.AND(x2, g.AND(x1 ^ 1, x0 ^ 1)), g.AND(x2 ^ 1, g.AND(x1, x0)))
        neg = g.AND(x2, g.AND(x1, x0) ^ 1)
        for j in range(w + 1):
            m = g.OR(g.AND(one, aa(j)), g.AND(two, aa(j - 1)))
            col = 2 * i + j
            if col < W:
                cols[col].append(g.XOR(m, neg))
        if 2 * i < W:
            cols[2 * i].append(neg)
        if 2 * i + w + 1 < W:
            cols[2 * i + w + 1].append(neg ^ 1)
        const += 1 << (w + 1 + 2 * i)
    cbits = (-const) % (1 << W)
    for j in range(W):
        if (cbits >> j) & 1:
            cols[j].append(1)
    return cols


def _fold_constants(cols: List[List[int]]) -> List[List[int]]:
    """Sum the constant-one bits of each column arithmetically (carrying into
    higher columns) so the reduction trees see at most one constant per column."""
    W = len(cols)
    out = [[x for x in c if x != 0 and x != 1] for c in cols]
    carry = 0
    for j in range(W):
        ones = sum(1 for x in cols[j] if x == 1) + carry
        if ones & 1:
            out[j].append(1)
        carry = ones >> 1
    return out


def wallace_reduce(g: AigBuilder, cols: List[List[int]]) -> List[List[int]]:
    """Wallace tree: each stage, full adders on every triple, a half adder on a
    leftover pair, until every column holds at most two bits."""
    W = len(cols)
    cols = _fold_constants(cols)
    for _ in range(64):
        if max((len(c) for c in cols), default=0) <= 2:
            return cols
        new: List[List[int]] = [[] for _ in range(W)]
        for j in range(W):
            bits = cols[j]
            k = 0
            while len(bits) - k >= 3:
                s, c = g.full_adder(bits[k], bits[k + 1], bits[k + 2])
                new[j].append(s)
                if j + 1 < W:
                    new[j + 1].append(c)
                k += 3
            if len(bits) - k == 2 and len(bits) > 2:
                s, c = g.half_adder(bits[k], bits[k + 1])
                new[j].append(s)
                if j + 1 < W:
                    new[j + 1].append(c)
                k += 2
            new[j].extend(bits[k:])
        cols = new
    raise RuntimeError("Wallace reduction did not converge")


def dadda_reduce(g: AigBuilder, cols: List[List[int]]) -> List[List[int]]:
    """Dadda tree: reduce column heights through the sequence 2,3,4,6,9,13,...
    using as few full/half adders as each stage needs."""
    W = len(cols)
    cols = [list(c) for c in _fold_constants(cols)]
    heights = [2]
    while heights[-1] < max(len(c) for c in cols):
        heights.append(heights[-1] * 3 // 2)
    for d in reversed(heights[:-1]):
        nxt: List[List[int]] = [[] for _ in range(W)]
        for j in range(W):
            bits = cols[j] + nxt[j]  # carries from column j-1 of this stage
            nxt[j] = []
            # sums produced in this stage stay in column j
            while len(bits) > d:
                if len(bits) - d >= 2:
                    s, c = g.full_adder(bits[0], bits[1], bits[2])
                    bits = bits[3:] + [s]
                else:
                    s, c = g.half_adder(bits[0], bits[1])
                    bits = bits[2:] + [s]
                if j + 1 < W:
                    nxt[j + 1].append(c)
            nxt[j] = bits
        cols = nxt
    assert max(len(c) for c in cols) <= 2
    return cols


def booth_multiplier(g: AigBuilder, a: Sequence[int], b: Sequence[int], tree: str = "wallace") -> List[int]:
    """Unsigned radix-4 Booth multiplier, Wallace or Dadda reduction, Kogge-Stone
    final adder (carry-out dropped: the product fits in 2w bits)."""
    w = len(a)
    cols = booth_partial_products(g, a, b)
    if tree == "wallace":
        cols = wallace_reduce(g, cols)
    elif tree == "dadda":
        cols = dadda_reduce(g, cols)
    else:
        raise ValueError(tree)
    x = [c[0] if len(c) > 0 else 0 for c in cols]
    y = [c[1] if len(c) > 1 else 0 for c in cols]
    return kogge_stone_adder(g, x, y)[: 2 * w]


# ----------------------------------------------------------------------------
# Miters and workloads
# ----------------------------------------------------------------------------

def miter_outputs(g: AigBuilder, xs: Sequence[int], ys: Sequence[int]) -> int:
    """§2.1: XOR corresponding outputs, OR the XORs (balanced tree)."""
    assert len(xs) == len(ys)
    return g.or_tree([g.XOR(x, y) for x, y in zip(xs, ys)])


def _two_operand_builder(w: int) -> Tuple[AigBuilder, List[int], List[int]]:
    g = AigBuilder(2 * w)
    a = [g.pi(i) for i in range(w)]
    b = [g.pi(w + i) for i in range(w)]
    return g, a, b


def build_adder_pair(w: int = 8) -> Aig:
    """w-bit RCA (side A) and KS (side B) over a[0..w-1] = PIs 0..w-1 and
    b[0..w-1] = PIs w..2w-1, with their miter as the single output."""
    g, a, b = _two_operand_builder(w)
    sa = g.next_var
    oa = ripple_carry_adder(g, a, b)
    g.new_scope()
    sb = g.next_var
    ob = kogge_stone_adder(g, a, b)
    eb = g.next_var
    g.new_scope()
    out = miter_outputs(g, oa, ob)
    return g.finish([out], side_ranges={"A": (sa, sb), "B": (sb, eb)},
                    side_outputs={"A": oa, "B": ob})


def build_multiplier_pair(w: int, tree: str = "wallace", msb_all_ones_mutant: bool = False,
                          product_bits: Optional[Sequence[int]] = None,
                          planted_minterm: Optional[int] = None, planted_bit: Optional[int] = None) -> Aig:
    """w x w array multiplier (side A) vs radix-4 Booth multiplier (side B),
    built in separate hashing scopes.  Outputs: the miter of all 2w product
    bits (default) or one XOR output per requested product bit.

    ``msb_all_ones_mutant`` XORs the AND of all 2w PIs into side B's MSB, so the
    two sides differ only at a = b = 2^w - 1.  ``planted_minterm`` = p
    generalises it: the minterm of p (PI k taken plain where bit k of p is 1,
    complemented where it is 0) is XORed into side B's product bit
    ``planted_bit`` (default the MSB), so the sides differ at pattern p alone
    and p is the miter's only (hence lowest) counterexample.
    """
    g, a, b = _two_operand_builder(w)
    sa = g.next_var
    oa = array_multiplier(g, a, b)
    g.new_scope()
    sb = g.next_var
    ob = booth_multiplier(g, a, b, tree=tree)
    if msb_all_ones_mutant:
        allp = g.and_tree(a + b)
        ob = ob[:-1] + [g.XOR(ob[-1], allp)]
    if planted_minterm is not None:
        assert 0 <= planted_minterm < (1 << (2 * w))
        k = 2 * w - 1 if planted_bit is None else planted_bit
        pis = a + b
        lits = [pis[i] if (planted_minterm >> i) & 1 else pis[i] ^ 1 for i in range(2 * w)]
        ob = list(ob)
        ob[k] = g.XOR(ob[k], g.and_tree(lits))
    eb = g.next_var
    g.new_scope()
    if product_bits is None:
        outs = [miter_outputs(g, oa, ob)]
    else:
        outs = [g.XOR(oa[k], ob[k]) for k in product_bits]
    return g.finish(outs, side_ranges={"A": (sa, sb), "B": (sb, eb)},
                    side_outputs={"A": oa, "B": ob})


# ----------------------------------------------------------------------------
# Random simulation (input selection only) and seeded mutants
# ----------------------------------------------------------------------------

def _splitmix64(state: int) -> Tuple[int, int]:
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Xoshiro256ss:
    """xoshiro256** seeded through splitmix64 (Blackman & Vigna, 2018)."""

    def __init__(self, seed: int):
        st = seed & MASK64
        self.s = []
        for _ in range(4):
            st, z = _splitmix64(st)
            self.s.append(z)

    def next(self) -> int:
        s = self.s
        r = (((s[1] * 5) & MASK64) << 7 | ((s[1] * 5) & MASK64) >> 57) & MASK64
        r = (r * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = ((s[3] << 45) | (s[3] >> 19)) & MASK64
        return r

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection."""
        assert n > 0
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next()
            if x < lim:
                return x % n

    def words(self, k: int) -> np.ndarray:
        return np.array([self.next() for _ in range(k)], dtype=np.uint64)


def random_signatures(aig: Aig, nwords: int, seed: int) -> np.ndarray:
    """64*nwords random patterns propagated through every node (input
    selection only).  Row v holds node v's signature."""
    rng = Xoshiro256ss(seed)
    V = aig.max_var + 1
    sig = np.zeros((V, nwords), dtype=np.uint64)
    for k in range(aig.num_pis):
        sig[k + 1] = rng.words(nwords)
    ones = np.uint64(MASK64)
    f = aig.fanins
    base = aig.num_pis + 1
    for i in range(aig.num_ands):
        l0, l1 = int(f[i, 0]), int(f[i, 1])
        x = sig[l0 >> 1] ^ ones if l0 & 1 else sig[l0 >> 1]
        y = sig[l1 >> 1] ^ ones if l1 & 1 else sig[l1 >> 1]
        sig[base + i] = x & y
    return sig


def lit_signature(sig: np.ndarray, lit: int) -> np.ndarray:
    s = sig[lit >> 1]
    return s ^ np.uint64(MASK64) if lit & 1 else s


def _tfi_ands(aig: Aig, roots: Sequence[int], lo: int, hi: int) -> List[int]:
    """AND variables in [lo, hi) reachable from the root literals (input
    selection: which ANDs a seeded flip may touch)."""
    seen = set()
    stack = [r >> 1 for r in roots]
    base = aig.num_pis + 1
    while stack:
        v = stack.pop()
        if v < base or v in seen:
            continue
        seen.add(v)
        f = aig.fanins[v - base]
        stack.append(int(f[0]) >> 1)
        stack.append(int(f[1]) >> 1)
    return sorted(v for v in seen if lo <= v < hi)


def inject_edge_inversion(aig: Aig, side: str, seed: int, max_tries: int = 64,
                          nwords: int = 16) -> Tuple[Aig, dict]:
    """Seeded single-edge inversion inside ``side``: one fanin complement bit of
    one AND in that side's output cone is flipped.  A flip that random
    simulation (16 words, same seed stream) cannot observe at the miter output
    is redrawn; each redraw is logged in the returned info."""
    lo, hi = aig.side_ranges[side]
    cand = _tfi_ands(aig, aig.side_outputs[side], lo, hi)
    rng = Xoshiro256ss(seed)
    redraws = []
    for _ in range(max_tries):
        v = cand[rng.below(len(cand))]
        e = rng.below(2)
        mut = Aig(aig.num_pis, aig.fanins.copy(), list(aig.outputs),
                  dict(aig.side_ranges), {k: list(x) for k, x in aig.side_outputs.items()})
        mut.fanins[v - aig.num_pis - 1, e] ^= 1
        sig = random_signatures(mut, nwords, seed ^ 0x5EED)
        if any(np.any(lit_signature(sig, o)) for o in mut.outputs):
            return mut, {"var": v, "edge": e, "redraws": redraws}
        redraws.append((v, e))
    raise RuntimeError("no observable edge inversion found")


# ----------------------------------------------------------------------------
# The five synthetic workloads
# ----------------------------------------------------------------------------

def config1_adders(mutant_seed: Optional[int] = None) -> Aig:
    """8-bit RCA vs 8-bit Kogge-Stone miter (16 PIs); optional KS-side flip."""
    m = build_adder_pair(8)
    if mutant_seed is not None:
        m, _ = inject_edge_inversion(m, "B", mutant_seed)
    return m


def config2_mult12(mutant_seed: Optional[int] = None) -> Aig:
    """12x12 array vs Booth/Wallace/KS miter (24 PIs); optional Booth-side flip."""
    m = build_multiplier_pair(12, tree="wallace")
    if mutant_seed is not None:
        m, _ = inject_edge_inversion(m, "B", mutant_seed)
    return m


def config3_mult16(mutant: bool = False, minterm: Optional[int] = None, bit: Optional[int] = None) -> Aig:
    """16x16 array vs Booth/Dadda miter (32 PIs, no hashing across sides);
    the mutant differs only at a = b = 0xFFFF.  ``minterm`` = p plants the
    minterm of p into product bit ``bit`` of the Booth side instead (see
    build_multiplier_pair): the only counterexample is then p = a | b << 16."""
    return build_multiplier_pair(16, tree="dadda", msb_all_ones_mutant=mutant,
                                 planted_minterm=minterm, planted_bit=bit)


def build_golden_revised_multipliers(w: int) -> Aig:
    """Four w x w multipliers over shared PIs: array (A), Booth/Wallace (B),
    and re-synthesized copies A* and B* (alternative XOR/majority forms).
    Outputs: A's product bits then B's."""
    g, a, b = _two_operand_builder(w)
    ranges = {}
    outs = {}
    for name, style, kind in (("A", "plain", "array"), ("B", "plain", "booth"),
                              ("A*", "alt", "array"), ("B*", "alt", "booth")):
        g.new_scope()
        g.style = style
        lo = g.next_var
        o = array_multiplier(g, a, b) if kind == "array" else booth_multiplier(g, a, b)
        ranges[name] = (lo, g.next_var)
        outs[name] = o
    g.style = "plain"
    return g.finish(outs["A"] + outs["B"], side_ranges=ranges, side_outputs=outs)


def build_revised_pair(w: int, kind: str = "array", mutant_seed: Optional[int] = None) -> Aig:
    """w x w multiplier (side A, plain XOR/majority forms) against its locally
    re-synthesized copy (side B, the alternative forms), as one miter over
    all 2w product bits: the golden-vs-revised setting of equivalence
    checking, where internal nodes correspond one to one.  ``kind`` is
    "array" or "booth"; an optional seeded edge inversion goes into side B."""
    g, a, b = _two_operand_builder(w)
    build = array_multiplier if kind == "array" else booth_multiplier
    g.new_scope()
    sa = g.next_var
    oa = build(g, a, b)
    g.new_scope()
    g.style = "alt"
    sb = g.next_var
    ob = build(g, a, b)
    eb = g.next_var
    g.style = "plain"
    g.new_scope()
    m = g.finish([miter_outputs(g, oa, ob)], side_ranges={"A": (sa, sb), "B": (sb, eb)},
                 side_outputs={"A": oa, "B": ob})
    if mutant_seed is not None:
        m, _ = inject_edge_inversion(m, "B", mutant_seed)
    return m


def _copy_path_with_flip(g_f0: List[int], g_f1: List[int], num_pis: int, root: int,
                         flip_var: int, flip_edge: int) -> int:
    """Append to (g_f0, g_f1) a copy of every AND on a path from ``flip_var`` to
    ``root`` (a literal), with one fanin edge of ``flip_var`` inverted.  Nodes
    off those paths are shared.  Returns the copied root literal."""
    base = num_pis + 1
    memo: Dict[int, int] = {}

    def reaches(v: int, cache: Dict[int, bool]) -> bool:
        # iterative reachability of flip_var from v through fanins
        stack = [v]
        order = []
        while stack:
            u = stack.pop()
            if u in cache or u < base:
                continue
            order.append(u)
            cache[u] = False  # placeholder
            stack.append(g_f0[u - base] >> 1)
            stack.append(g_f1[u - base] >> 1)
        for u in sorted(order):
            a0, a1 = g_f0[u - base] >> 1, g_f1[u - base] >> 1
            cache[u] = (u == flip_var) or cache.get(a0, False) or cache.get(a1, False)
        return cache.get(v, False)

    cache: Dict[int, bool] = {}
    reaches(root >> 1, cache)
    todo = sorted(u for u, r in cache.items() if r)
    for u in todo:
        l0, l1 = g_f0[u - base], g_f1[u - base]
        if u == flip_var:
            if flip_edge == 0:
                l0 ^= 1
            else:
                l1 ^= 1
        n0 = memo.get(l0 >> 1, l0 >> 1) * 2 | (l0 & 1) if (l0 >> 1) in memo else l0
        n1 = memo.get(l1 >> 1, l1 >> 1) * 2 | (l1 & 1) if (l1 >> 1) in memo else l1
        nv = num_pis + 1 + len(g_f0)
        g_f0.append(n0)
        g_f1.append(n1)
        memo[u] = nv
    rv = root >> 1
    if rv in memo:
        return 2 * memo[rv] | (root & 1)
    return root


def support_masks(aig: Aig) -> List[int]:
    """Python-int PI bitmask per variable (input selection for the support filter)."""
    V = aig.max_var + 1
    m = [0] * V
    for k in range(aig.num_pis):
        m[k + 1] = 1 << k
    base = aig.num_pis + 1
    f = aig.fanins
    for i in range(aig.num_ands):
        m[base + i] = m[int(f[i, 0]) >> 1] | m[int(f[i, 1]) >> 1]
    return m


def signature_words(aig: Aig, nwords: int, seed: int) -> np.ndarray:
    """The (num_pis, nwords) random PI words random_signatures draws."""
    rng = Xoshiro256ss(seed)
    return np.stack([rng.words(nwords) for _ in range(aig.num_pis)]) if aig.num_pis else \
        np.zeros((0, nwords), dtype=np.uint64)


def candidate_pairs(base: Aig, sig_words: int, seed: int, max_support: int):
    """Node pairs with equal random-simulation signatures (input selection):
    classes of identical non-constant signatures over the AND nodes, each
    member paired with the class's lowest variable, kept if the joint PI
    support has at most max_support PIs.  Returns (sorted pairs, masks)."""
    sig = random_signatures(base, sig_words, seed)
    masks = support_masks(base)
    V = base.max_var + 1
    first = base.num_pis + 1
    classes: Dict[bytes, List[int]] = {}
    zero = np.zeros(sig_words, dtype=np.uint64)
    ones = zero ^ np.uint64(MASK64)
    for v in range(first, V):
        s = sig[v]
        if np.array_equal(s, zero) or np.array_equal(s, ones):
            continue
        classes.setdefault(s.tobytes(), []).append(v)
    cands: List[Tuple[int, int]] = []
    for members in classes.values():
        if len(members) < 2:
            continue
        rep = members[0]
        for v in members[1:]:
            if bin(masks[rep] | masks[v]).count("1") <= max_support:
                cands.append((rep, v))
    cands.sort()
    return cands, masks


@dataclasses.dataclass
class PairBatch:
    """Node-pair miters sharing one AIG: miter j is (aig, outputs[j])."""

    aig: Aig
    pairs: List[Tuple[int, int]]       # (x_lit, y_lit) before mutation
    mutated: List[bool]
    support_sizes: List[int]


def config4_pairs(num_pairs: int = 4096, w: int = 32, max_support: int = 28, seed: int = 4,
                  mutant_frac: float = 0.02, sig_words: int = 64) -> PairBatch:
    """Node-pair miters from a w x w array-vs-Booth multiplier pair.

    The graph holds the array multiplier and the Booth multiplier, each in its
    generator form and in a locally re-synthesized form (every XOR and
    majority built from a different AND decomposition, as a synthesis tool
    would leave them), all in separate hashing scopes.  An array-vs-Booth
    pair alone shares almost no internal functions (only its low product
    bits), so the re-synthesized copies are what give internal equivalences.
    Nodes are grouped by equal 64-word random-simulation signatures (§2.3 step
    (1)); within a class every member is paired with the class's lowest
    variable.  Constant-signature classes and pairs whose joint PI support
    exceeds ``max_support`` are dropped.  A seeded sample of ``num_pairs`` is
    taken (all of them if fewer exist); ``mutant_frac`` of them get a seeded
    single-edge inversion inside the y cone (the path from the flipped AND to
    y is copied, so other pairs are untouched).  Each miter's output is
    x XOR y'.
    """
    base = build_golden_revised_multipliers(w)
    cands, masks = candidate_pairs(base, sig_words, seed, max_support)
    V = base.max_var + 1
    first = base.num_pis + 1
    rng = Xoshiro256ss(seed ^ 0xBA7C4)
    if len(cands) > num_pairs:
        idx = list(range(len(cands)))
        for i in range(num_pairs):  # partial Fisher-Yates
            j = i + rng.below(len(idx) - i)
            idx[i], idx[j] = idx[j], idx[i]
        chosen = sorted(idx[:num_pairs])
        cands = [cands[i] for i in chosen]
    f0 = [int(x) for x in base.fanins[:, 0]]
    f1 = [int(x) for x in base.fanins[:, 1]]
    n_mut = int(round(mutant_frac * len(cands)))
    mut_idx = set()
    while len(mut_idx) < n_mut:
        mut_idx.add(rng.below(len(cands)))
    outs, pairs, mutated, sup = [], [], [], []
    for j, (x, y) in enumerate(cands):
        ylit = 2 * y
        if j in mut_idx:
            cone = _tfi_ands(Aig(base.num_pis, np.stack([np.array(f0, dtype=np.uint32),
                                                         np.array(f1, dtype=np.uint32)], axis=1),
                                 []), [ylit], first, V)
            fv = cone[rng.below(len(cone))]
            ylit = _copy_path_with_flip(f0, f1, base.num_pis, ylit, fv, rng.below(2))
        # x XOR y' as three ANDs appended to the shared graph
        n = base.num_pis + 1 + len(f0)
        xl = 2 * x
        f0.append(xl); f1.append(ylit ^ 1)
        f0.append(xl ^ 1); f1.append(ylit)
        f0.append(2 * n ^ 1); f1.append(2 * (n + 1) ^ 1)
        outs.append(2 * (n + 2) ^ 1)
        pairs.append((2 * x, 2 * y))
        mutated.append(j in mut_idx)
        sup.append(bin(masks[x] | masks[y]).count("1"))
    f = np.stack([np.array(f0, dtype=np.uint32), np.array(f1, dtype=np.uint32)], axis=1)
    aig = Aig(base.num_pis, f, outs, dict(base.side_ranges), dict(base.side_outputs))
    return PairBatch(aig, pairs, mutated, sup)


@dataclasses.dataclass
class ProductBitRequest:
    w: int
    bit: int
    mutant: bool
    arrival_s: float


def config5_stream(num_requests: int = 20000, rate_per_s: float = 50.0, seed: int = 5,
                   w_lo: int = 8, w_hi: int = 18, mutant_frac: float = 0.01) -> List[ProductBitRequest]:
    """Seeded Poisson arrival stream of product-bit miter requests: w uniform in
    [w_lo, w_hi], product bit uniform in [w-1, 2w-1] (so the support is all 2w
    PIs), ``mutant_frac`` of them mutated."""
    rng = Xoshiro256ss(seed)
    t = 0.0
    out = []
    for _ in range(num_requests):
        u = (rng.next() >> 11) * (1.0 / (1 << 53))
        t += -np.log1p(-u) / rate_per_s
        w = w_lo + rng.below(w_hi - w_lo + 1)
        bit = (w - 1) + rng.below(w + 1)
        mut = rng.below(1_000_000) < int(mutant_frac * 1_000_000)
        out.append(ProductBitRequest(w, bit, mut, t))
    return out


class ProductBitMiters:
    """Per-width cache of product-bit miters (array vs Booth/Wallace), with
    seeded Booth-side mutants made by copying the flipped path."""

    def __init__(self, seed: int = 5):
        self.seed = seed
        self._base: Dict[int, Aig] = {}

    def base(self, w: int) -> Aig:
        if w not in self._base:
            self._base[w] = build_multiplier_pair(w, tree="wallace", product_bits=list(range(2 * w)))
        return self._base[w]

    def miter(self, w: int, bit: int, mutant: bool = False, mutant_seed: int = 0) -> Tuple[Aig, int]:
        """Returns (aig, out_lit) for product bit ``bit``."""
        b = self.base(w)
        if not mutant:
            return b, b.outputs[bit]
        f0 = [int(x) for x in b.fanins[:, 0]]
        f1 = [int(x) for x in b.fanins[:, 1]]
        lo, hi = b.side_ranges["B"]
        ob = b.side_outputs["B"][bit]
        rng = Xoshiro256ss(self.seed * 1000003 + w * 1009 + bit * 7 + mutant_seed)
        cone = _tfi_ands(b, [ob], lo, hi)
        for _ in range(64):
            fv = cone[rng.below(len(cone))]
            e = rng.below(2)
            g0, g1 = list(f0), list(f1)
            nb = _copy_path_with_flip(g0, g1, b.num_pis, ob, fv, e)
            oa = b.side_outputs["A"][bit]
            n = b.num_pis + 1 + len(g0)
            g0.append(oa); g1.append(nb ^ 1)
            g0.append(oa ^ 1); g1.append(nb)
            g0.append(2 * n ^ 1); g1.append(2 * (n + 1) ^ 1)
            out = 2 * (n + 2) ^ 1
            f = np.stack([np.array(g0, dtype=np.uint32), np.array(g1, dtype=np.uint32)], axis=1)
            m = Aig(b.num_pis, f, [out], dict(b.side_ranges), dict(b.side_outputs))
            sig = random_signatures(m, 16, rng.next())
            if np.any(lit_signature(sig, out)):
                return m, out
        raise RuntimeError("no observable mutant")


def build_four_multiplier_miter(w: int) -> Aig:
    """The four w x w multipliers of build_golden_revised_multipliers (array,
    Booth, and their re-synthesized copies) mitered together: the OR of the
    array-vs-copy, Booth-vs-copy and array-vs-Booth miters over all 2w
    product bits, one output whose cone holds all four multipliers."""
    g, a, b = _two_operand_builder(w)
    outs = {}
    for name, style, kind in (("A", "plain", "array"), ("B", "plain", "booth"),
                              ("A*", "alt", "array"), ("B*", "alt", "booth")):
        g.new_scope()
        g.style = style
        outs[name] = array_multiplier(g, a, b) if kind == "array" else booth_multiplier(g, a, b)
    g.style = "plain"
    g.new_scope()
    out = g.or_tree([miter_outputs(g, outs["A"], outs["A*"]), miter_outputs(g, outs["B"], outs["B*"]),
                     miter_outputs(g, outs["A"], outs["B"])])
    return g.finish([out], side_outputs=outs)


def config4_spread(num: int = 4096, seed: int = 4, min_support: int = 10, max_support: int = 28,
                   mutant_frac: float = 0.02) -> List[Tuple[Aig, int, str]]:
    """The batched workload at its stated spread: ``num`` miters of
    ``min_support``..``max_support`` PIs, from node pairs up to whole
    multiplier miters.  Sources (all seeded):
      pair      node-pair miters (as config4_pairs) from the w x w
                four-multiplier graphs, w = 32 and 14..10, whose joint
                support has at least min_support PIs (~2% mutated);
      bit       product-bit miters of w x w array vs Booth, w = 5..14,
                every product bit whose support has at least min_support
                PIs, 1 in 50 a seeded Booth-side mutant;
      revised   whole array (and Booth) multipliers against their
                re-synthesized copies, w = 5..14;
      four      the four w x w multipliers mitered together, w = 5..14.
    Every bit, revised and four miter is kept (the heavy end); the node
    pairs fill the rest by a seeded sample.  Returns (aig, out_lit, source)
    triples; many share one aig."""
    heavy: List[Tuple[Aig, int, str]] = []
    pm = ProductBitMiters(seed=seed)
    rng = Xoshiro256ss(seed ^ 0x5EED5)
    for w in range(min_support // 2, max_support // 2 + 1):
        masks = support_masks(pm.base(w))
        for bit in range(2 * w):
            mut = rng.below(50) == 0
            if bin(masks[pm.base(w).outputs[bit] >> 1]).count("1") < min_support:
                continue  # a low product bit: too few PIs
            aig, out = pm.miter(w, bit, mut, mutant_seed=bit)
            heavy.append((aig, out, "bit"))
        for kind in ("array", "booth"):
            r = build_revised_pair(w, kind)
            heavy.append((r, r.outputs[0], "revised"))
        f = build_four_multiplier_miter(w)
        heavy.append((f, f.outputs[0], "four"))
    pairs: List[Tuple[Aig, int, str]] = []
    for w in (32, 14, 13, 12, 11, 10):
        pb = config4_pairs(num_pairs=1 << 30, w=w, max_support=max_support, seed=seed + w,
                           mutant_frac=mutant_frac)
        pairs += [(pb.aig, pb.aig.outputs[j], "pair") for j, n in enumerate(pb.support_sizes)
                  if n >= min_support]
    want = max(0, num - len(heavy))
    if len(pairs) > want:
        idx = list(range(len(pairs)))
        for i in range(want):  # partial Fisher-Yates
            j = i + rng.below(len(idx) - i)
            idx[i], idx[j] = idx[j], idx[i]
        pairs = [pairs[i] for i in sorted(idx[:want])]
    return heavy + pairs


# ----------------------------------------------------------------------------
# AIGER I/O (format of Biere's AIGER 1.9 documentation, combinational subset)
# ----------------------------------------------------------------------------

def write_aag(aig: Aig) -> str:
    M = aig.max_var
    lines = [f"aag {M} {aig.num_pis} 0 {len(aig.outputs)} {aig.num_ands}"]
    lines += [str(2 * (k + 1)) for k in range(aig.num_pis)]
    lines += [str(o) for o in aig.outputs]
    base = aig.num_pis + 1
    for i in range(aig.num_ands):
        lines.append(f"{2 * (base + i)} {int(aig.fanins[i, 0])} {int(aig.fanins[i, 1])}")
    return "\n".join(lines) + "\n"


def _enc_delta(x: int) -> bytes:
    out = bytearray()
    while x & ~0x7F:
        out.append((x & 0x7F) | 0x80)
        x >>= 7
    out.append(x)
    return bytes(out)


def write_aig_binary(aig: Aig) -> bytes:
    M = aig.max_var
    hdr = f"aig {M} {aig.num_pis} 0 {len(aig.outputs)} {aig.num_ands}\n".encode()
    body = "".join(f"{o}\n" for o in aig.outputs).encode()
    base = aig.num_pis + 1
    out = bytearray(hdr + body)
    for i in range(aig.num_ands):
        lhs = 2 * (base + i)
        r0, r1 = int(aig.fanins[i, 0]), int(aig.fanins[i, 1])
        if r0 < r1:
            r0, r1 = r1, r0
        out += _enc_delta(lhs - r0)
        out += _enc_delta(r0 - r1)
    return bytes(out)


class AigerError(ValueError):
    pass


def read_aiger(data: bytes) -> Aig:
    """Parse ASCII (aag) or binary (aig) combinational AIGER.  ASCII AND
    definitions may come in any order; they are renumbered topologically."""
    if isinstance(data, str):
        data = data.encode()
    nl = data.find(b"\n")
    if nl < 0:
        raise AigerError("missing header")
    hdr = data[:nl].split()
    if len(hdr) < 6 or hdr[0] not in (b"aag", b"aig"):
        raise AigerError("bad header")
    try:
        M, I, L, O, A = (int(x) for x in hdr[1:6])
    except ValueError as e:
        raise AigerError("bad header numbers") from e
    if L != 0:
        raise AigerError("latches are not supported (combinational AIGs only)")
    if M < I + A:
        raise AigerError("M < I + A")
    pos = nl + 1
    binary = hdr[0] == b"aig"

    def line() -> List[int]:
        nonlocal pos
        e = data.find(b"\n", pos)
        if e < 0:
            e = len(data)
        ln = data[pos:e]
        pos = e + 1
        try:
            return [int(x) for x in ln.split()]
        except ValueError as ex:
            raise AigerError("bad number") from ex

    if binary:
        inputs = [2 * (k + 1) for k in range(I)]
    else:
        inputs = [line()[0] for _ in range(I)]
    outs = []
    for _ in range(O):
        ln = line()
        if not ln:
            raise AigerError("missing output")
        outs.append(ln[0])
    defs = []
    if binary:
        def dec() -> int:
            nonlocal pos
            x, sh = 0, 0
            while True:
                if pos >= len(data):
                    raise AigerError("truncated binary AND section")
                c = data[pos]
                pos += 1
                x |= (c & 0x7F) << sh
                if not c & 0x80:
                    return x
                sh += 7
        for i in range(A):
            lhs = 2 * (I + 1 + i)
            d0 = dec()
            d1 = dec()
            r0 = lhs - d0
            r1 = r0 - d1
            if r0 < 0 or r1 < 0:
                raise AigerError("bad delta")
            defs.append((lhs, r0, r1))
    else:
        for _ in range(A):
            ln = line()
            if len(ln) != 3:
                raise AigerError("bad AND line")
            defs.append(tuple(ln))
    # renumber: PIs first in declaration order, ANDs topologically
    remap = {0: 0}
    for k, lit in enumerate(inputs):
        if lit & 1 or lit < 2 or (lit >> 1) in remap:
            raise AigerError("bad input literal")
        remap[lit >> 1] = k + 1
    by_var = {}
    for lhs, r0, r1 in defs:
        if lhs & 1 or (lhs >> 1) in remap or (lhs >> 1) in by_var:
            raise AigerError("bad AND lhs")
        by_var[lhs >> 1] = (r0, r1)
    for lit in [x for d in defs for x in d[1:]] + outs:
        if (lit >> 1) > M:
            raise AigerError("literal exceeds M")
    order: List[int] = []
    state: Dict[int, int] = {}
    for root in sorted(by_var):
        if state.get(root) == 2:
            continue
        stack = [(root, 0)]
        while stack:
            v, k = stack.pop()
            if v in remap and v not in by_var:
                continue
            if v not in by_var:
                raise AigerError(f"undefined variable {v}")
            st = state.get(v, 0)
            if st == 2:
                continue
            if k == 0:
                if st == 1:
                    raise AigerError("combinational cycle")
                state[v] = 1
                stack.append((v, 1))
                for r in by_var[v]:
                    u = r >> 1
                    if u != 0 and state.get(u, 0) != 2 and not (u in remap and u not in by_var):
                        if state.get(u, 0) == 1:
                            raise AigerError("combinational cycle")
                        stack.append((u, 0))
            else:
                state[v] = 2
                order.append(v)
    nxt = I + 1
    for v in order:
        remap[v] = nxt
        nxt += 1

    def rl(lit: int) -> int:
        return 2 * remap[lit >> 1] | (lit & 1)

    f = np.zeros((len(order), 2), dtype=np.uint32)
    for i, v in enumerate(order):
        r0, r1 = by_var[v]
        f[i, 0] = rl(r0)
        f[i, 1] = rl(r1)
    return Aig(I, f, [rl(o) for o in outs])
