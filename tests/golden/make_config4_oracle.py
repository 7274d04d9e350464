"""Writes config4_pairs_oracle.json: the CPU oracle's lowest counterexample
of each of the 4,096 node-pair miters of circuits.config4_pairs() (the
batched workload), so GPU tests can compare every batch result with the
oracle without re-running it.  Calls only the oracle and the input
generator; the file records a fingerprint of the generated graph, and the
tests refuse a stale file.

    python tests/golden/make_config4_oracle.py     # a few minutes on 8 threads
"""
import hashlib
import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2512_06627_b300 import circuits as C  # noqa: E402

OUT = os.path.join(HERE, "config4_pairs_oracle.json")


def fingerprint(aig) -> str:
    h = hashlib.sha256()
    h.update(aig.flat_fanins().tobytes())
    h.update(repr((aig.num_pis, list(aig.outputs))).encode())
    return h.hexdigest()


def main():
    pb = C.config4_pairs()
    a = pb.aig
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        cex = list(ex.map(lambda o: O.check(a.num_pis, a.fanins, o)[0], a.outputs))
    json.dump({"what": "oracle lowest counterexample per config4_pairs() miter (null: equivalent)",
               "fingerprint": fingerprint(a), "cex": cex}, open(OUT, "w"))
    print(OUT, sum(1 for x in cex if x is not None), "non-equivalent of", len(cex))


if __name__ == "__main__":
    main()
