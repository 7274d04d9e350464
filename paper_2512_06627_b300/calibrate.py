"""Measure the ES time model's calibration set on this GPU and fit it.

    python -m paper_2512_06627_b300.calibrate [--tiers interp,jit] [--out fit.json]

The time model (paper §3.2, refit per tier: t = a + c * gates + alpha *
gates * 2^(n - 23)) starts every context from built-in B300 values.  This
tool times full, equivalent checks of a fixed calibration set -- the adder,
12x12 and 16x16 multiplier miters, single product-bit miters of 8..18-bit
multipliers and node-pair miters of 4..28 PIs -- on the requested tiers with
the library's default geometry (median of three launches after one warm-up)
and prints the least-relative-error fit of each tier, its median relative
error, and the error of the built-in values on the same set.  Specialised
kernels are also fitted by their executed lop3 per pass (x = (lop3 + 40) *
2^(n - 23)), the form the library uses once it holds a kernel.
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys

import numpy as np

from . import circuits as C
from . import lec_es as L

KERNEL_PASS_OVERHEAD = 40  # lop3-equivalents per pass outside the tables (as in the library)


def calibration_set(max_n: int = 32):
    """(name, Miter) pairs: equivalent miters only (full enumerations)."""
    out = [("adders", L.miter_of(C.config1_adders())), ("mult12", L.miter_of(C.config2_mult12())),
           ("mult16", L.miter_of(C.config3_mult16()))]
    rng = np.random.default_rng(11)
    for w in (8, 10, 12, 14, 16, 18):
        aig = C.build_multiplier_pair(w, tree="wallace", product_bits=list(range(2 * w)))
        f = aig.flat_fanins()
        for k in sorted(set(int(x) for x in rng.choice(2 * w, size=4, replace=False))):
            m = L.Miter(aig.num_pis, f, aig.outputs[k])
            if L.lec_es_compile(m)[0].n <= min(max_n, 30):
                out.append((f"mult{w}_bit{k}", m))
    pb = C.config4_pairs()
    f = pb.aig.flat_fanins()
    by_n = {}
    for i, s in enumerate(pb.support_sizes):
        if not pb.mutated[i] and 4 <= s <= 28:
            by_n.setdefault(s, []).append(i)
    for s in sorted(by_n):
        for i in by_n[s][:2]:
            out.append((f"pair{i}_n{s}", L.Miter(pb.aig.num_pis, f, pb.aig.outputs[i])))
    return out


def time_tier(ctx, m, tier, runs=3):
    p = L.lec_es_prepare(ctx, m, L.options(tier=tier))
    try:
        info = L.lec_es_plan_info(p)
        ts = []
        for i in range(runs + 1):
            L.lec_es_run_async(ctx, p)
            r = L.lec_es_plan_result(ctx, p)
            if r.cex != L.NO_CEX:
                return None
            if i:
                ts.append(r.device_ms)
        return statistics.median(ts), info
    finally:
        L.lec_es_plan_free(ctx, p)


def _median_rel_err(coef, gates, n, ms):
    pred = coef.a_ms + coef.c_ms * gates + coef.alpha_ms * gates * np.exp2(n - 23.0)
    return float(np.median(np.abs(pred - ms) / ms))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tiers", default="interp,jit")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    tiers = {"interp": L.TIER_INTERP, "jit": L.TIER_JIT}
    ctx = L.lec_es_create(0, arena_bytes=4 << 30)
    cases = calibration_set()
    report = {"cases": len(cases)}
    try:
        for name in args.tiers.split(","):
            tier = tiers[name]
            gates, ns, ms, lop = [], [], [], []
            for label, m in cases:
                got = time_tier(ctx, m, tier)
                if got is None:
                    continue
                t, info = got
                gates.append(info.cone_ands)
                ns.append(info.n)
                ms.append(t)
                lop.append(getattr(info, "lop3_per_pass", 0.0))
            g, n, t = np.array(gates, float), np.array(ns, float), np.array(ms)
            fit = L.lec_es_cost_fit(gates, ns, ms)
            builtin = L.lec_es_cost_model(None, tier)
            entry = {"samples": len(ms),
                     "fit": {"a_ms": fit.a_ms, "c_ms": fit.c_ms, "alpha_ms": fit.alpha_ms},
                     "median_rel_err_fit": _median_rel_err(fit, g, n, t),
                     "median_rel_err_builtin": _median_rel_err(builtin, g, n, t)}
            if tier == L.TIER_JIT and any(lop):
                lg = [int(round(x + KERNEL_PASS_OVERHEAD)) for x in lop]
                kf = L.lec_es_cost_fit(lg, ns, ms)
                kb = L.lec_es_cost_model(None, L.TIER_KERNEL)
                entry["by_lop3"] = {"fit": {"a_ms": kf.a_ms, "c_ms": kf.c_ms, "alpha_ms": kf.alpha_ms},
                                    "median_rel_err_fit": _median_rel_err(kf, np.array(lg, float), n, t),
                                    "median_rel_err_builtin": _median_rel_err(kb, np.array(lg, float), n, t)}
            report[name] = entry
    finally:
        L.lec_es_destroy(ctx)
    text = json.dumps(report, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
