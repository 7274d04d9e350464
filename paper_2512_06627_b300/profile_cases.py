"""Small, fixed workloads for profiling one kernel at a time.

    python -m paper_2512_06627_b300.profile_cases <case> [--runs N]

Cases:
  mult16-jit      the 16x16 array vs Booth/Dadda miter on the specialised kernel
  mult16-interp   the same miter on the shared-memory interpreter
  mult12-interp   the 12x12 miter on the interpreter (short launches)
  pairs-light     the node-pair miters light enough for the tile queue, one batch
  pairs-all       all 4,096 node-pair miters, one prepared batch
  pair-jit        one node-pair miter of support --n on the specialised kernel
  sweep-32x32     random-simulation signatures of the 32x32 four-multiplier graph

Each case prepares its work first and then runs it N times (default 2), so a
profiler can skip the first launch(es) and capture one.
"""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["mult16-jit", "mult16-interp", "mult12-interp", "pairs-light", "pairs-all",
                                     "pair-jit", "sweep-32x32"])
    ap.add_argument("--runs", type=int, default=2)
    ap.add_argument("--n", type=int, default=24, help="support size for pair-jit")
    a = ap.parse_args(argv)
    from paper_2512_06627_b300 import circuits as C
    from paper_2512_06627_b300 import lec_es as L
    ctx = L.lec_es_create(0, arena_bytes=1 << 30)
    if a.case == "sweep-32x32":
        base = C.build_golden_revised_multipliers(32)
        pw = C.signature_words(base, 64, 4)
        for _ in range(a.runs):
            pairs = L.lec_es_match_pairs(ctx, base.num_pis, base.flat_fanins(), pw, 28)
            print(f"pairs {len(pairs)}")
    elif a.case.startswith("mult"):
        aig = C.config3_mult16() if a.case.startswith("mult16") else C.config2_mult12()
        tier = L.TIER_JIT if a.case.endswith("jit") else L.TIER_INTERP
        p = L.lec_es_prepare(ctx, L.miter_of(aig), L.options(tier=tier))
        for _ in range(a.runs):
            L.lec_es_run_async(ctx, p)
            r = L.lec_es_plan_result(ctx, p)
            print(f"verdict {r.verdict} tier {r.tier} device_ms {r.device_ms:.3f}")
        L.lec_es_plan_free(ctx, p)
    elif a.case == "pair-jit":
        pb = C.config4_pairs()
        f = pb.aig.flat_fanins()
        m = None
        for o in pb.aig.outputs:
            cand = L.Miter(pb.aig.num_pis, f, o)
            info = L.lec_es_compile(cand)[0]
            if info.n == a.n and info.num_luts >= 64:
                m = cand
                break
        if m is None:
            sys.exit(f"no node-pair miter with support {a.n}")
        p = L.lec_es_prepare(ctx, m, L.options(tier=L.TIER_JIT))
        for _ in range(a.runs):
            L.lec_es_run_async(ctx, p)
            r = L.lec_es_plan_result(ctx, p)
            print(f"n {info.n} tables {info.num_luts} verdict {r.verdict} device_ms {r.device_ms:.4f}")
        L.lec_es_plan_free(ctx, p)
    else:
        pb = C.config4_pairs()
        f = pb.aig.flat_fanins()
        ms = [L.Miter(pb.aig.num_pis, f, o) for o in pb.aig.outputs]
        opt = None
        if a.case == "pairs-light":
            infos = [L.lec_es_compile(m)[0] for m in ms]
            ms = [m for m, i in zip(ms, infos) if i.num_records * float(1 << max(0, i.n - 5)) < 5e7]
            opt = L.options(tier=L.TIER_INTERP)
        b = L.lec_es_batch_prepare(ctx, ms, opt)
        for _ in range(a.runs):
            L.lec_es_batch_run_async(ctx, b)
            rs = L.lec_es_batch_results(ctx, b, len(ms))
            print(f"miters {len(ms)} device_ms {rs[0].device_ms:.3f}")
        L.lec_es_batch_free(ctx, b)
    L.lec_es_destroy(ctx)


if __name__ == "__main__":
    sys.exit(main())
