"""Writes spread1024_oracle.json: the CPU oracle's lowest counterexample of
each of the 1,024 miters of circuits.config4_spread(num=1024, seed=9) (the
batched workload at its stated spread, 10..28 PIs, node pairs up to whole
four-multiplier miters), so the GPU batch test can compare every result with
the oracle.  Calls only the oracle and the input generator; the file records
a fingerprint of the generated miters, and the tests refuse a stale file.

    python tests/golden/make_spread_oracle.py     # a few minutes on 8 threads
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2512_06627_b300 import circuits as C  # noqa: E402

OUT = os.path.join(HERE, "spread1024_oracle.json")
NUM, SEED = 1024, 9


def fingerprint(trip) -> str:
    """SHA-256 over every miter: its graph's fanins, PI count and output."""
    h = hashlib.sha256()
    seen = {}
    for aig, out, kind in trip:
        key = id(aig)
        if key not in seen:
            seen[key] = len(seen)
            h.update(b"graph")
            h.update(aig.flat_fanins().tobytes())
            h.update(repr(aig.num_pis).encode())
        h.update(repr((seen[key], int(out), kind)).encode())
    return h.hexdigest()


def main():
    trip = C.config4_spread(num=NUM, seed=SEED)
    threads = os.cpu_count() or 1
    t0 = time.time()
    cex = []
    for i, (aig, out, _) in enumerate(trip):
        cex.append(O.check_parallel(aig.num_pis, aig.fanins, out, threads)[0])
        if i % 128 == 127:
            print(i + 1, "of", len(trip), f"{time.time() - t0:.0f} s", flush=True)
    json.dump({"what": "oracle lowest counterexample per config4_spread(num=1024, seed=9) miter (null: equivalent)",
               "fingerprint": fingerprint(trip), "cex": cex}, open(OUT, "w"))
    print(OUT, sum(1 for x in cex if x is not None), "non-equivalent of", len(cex), f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
