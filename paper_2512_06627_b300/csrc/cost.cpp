// cost.cpp -- the ES time model of §3.2, refit for this GPU.
//
// The paper predicts exact-simulation time as alpha * gates * 2^(n - beta)
// (linear in the cone's gates, exponential in its PIs) and fits alpha and
// beta to measurements (its footnote: alpha = 0.0003 s, beta = 23 for one CPU
// core).  alpha * 2^-beta is a single factor, so here beta stays at the
// paper's 23 and each execution tier gets its own alpha (ms), plus a fixed
// launch cost a and a per-gate cost c for one pass over the program, which
// is what a small support costs on a GPU (too few patterns to fill it):
//
//     t_ms = a + c * gates + alpha * x,   x = gates * 2^(n - 23).
//
// The fit minimises relative error (weights 1/t^2) with a, c, alpha >= 0.  A
// context starts from values measured on B300 (entered as pseudo-samples, so
// they act as a prior) and folds in every full, equivalent single run it
// times; kernel builds are fitted as a + c * tables.  A built specialised
// kernel reports the lop3 it executes per 32-pattern pass, which tracks its
// time far better than the gates do (hoisted tables and folded pass PIs
// remove 10-90% of the work, by cone), so runs of a known kernel are also
// fitted and predicted with x = (lop3 + 40) * 2^(n - 23), 40 being the
// per-pass loop and result-check overhead in lop3-equivalents (20 for a
// kernel whose passes run in straight-line groups; the value
// with the least median error over the calibration set).  The model decides the
// tier of AUTO runs (jit_auto_tier), which batch miters get their own
// kernel, and the priority class of served requests.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lec_es.h"
#include "es_ctx.h"
#include "es_internal.h"

namespace lec {

namespace {

// Built-in B300 values (148 SMs at 2,032 MHz): lec_es_cost_fit over the
// single-launch device times of equivalent miters -- the 12x12 and 16x16
// multiplier miters, the adders, product-bit miters of 8..18-bit multipliers
// and node-pair miters of 4..28 PIs (python -m paper_2512_06627_b300.calibrate
// times that set).  Interpreter: 71 miters (four-record steps, barrier-free
// resident passes, wider blocks where shared memory allows), median relative
// error 8%; specialised kernel: 74 miters, 18% (small
// kernels are dominated by launch latency, which three terms only
// approximate).
struct Builtin {
  double a_ms, c_ms, alpha_ms;
};
constexpr Builtin kRun[4] = {
    {0.0, 0.0, 0.0},                  // AUTO: unused
    {8.360e-3, 4.120e-5, 1.3133e-4},  // INTERP: word-wide interpreter
    {7.743e-3, 2.742e-6, 6.018e-7},   // JIT: specialised kernel
    {2.0e-2, 1.0e-4, 2.0e-3},         // SPILL: global-memory interpreter (rough)
};
// By the kernel's executed lop3 (less 20 per pass for kernels with pass
// groups, JitKernel::model_lop3), over 225 kernel times (the calibration set
// and the served stream's 154 distinct programs, generator version 24):
// median relative error 5%, 90th percentile 21%.
constexpr Builtin kKernel = {7.887e-3, 1.074e-6, 1.3907e-5};
constexpr double kPassOverhead = 40.0;  // lop3-equivalents per pass outside the tables
constexpr Builtin kCompile = {14.2, 0.084, 0.0};  // kernel build: ms + ms per table
constexpr double kPriorWeight = 4.0;             // the built-in values count as this many samples each
constexpr double kBinCap = 8.0;                  // a (n, log2 gates) bin counts as at most this many

// Solve S[sel] c = b[sel] for the selected coefficients (others zero).
bool solve_subset(const double S[3][3], const double b[3], unsigned sel, double out[3]) {
  int idx[3], m = 0;
  for (int i = 0; i < 3; i++)
    if (sel >> i & 1u) idx[m++] = i;
  double A[3][4];
  for (int r = 0; r < m; r++) {
    for (int q = 0; q < m; q++) A[r][q] = S[idx[r]][idx[q]];
    A[r][m] = b[idx[r]];
  }
  for (int col = 0; col < m; col++) {  // Gaussian elimination, partial pivoting
    int piv = col;
    for (int r = col + 1; r < m; r++)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (!(fabs(A[piv][col]) > 1e-300)) return false;
    if (piv != col)
      for (int q = 0; q <= m; q++) std::swap(A[col][q], A[piv][q]);
    for (int r = 0; r < m; r++) {
      if (r == col) continue;
      const double f = A[r][col] / A[col][col];
      for (int q = col; q <= m; q++) A[r][q] -= f * A[col][q];
    }
  }
  out[0] = out[1] = out[2] = 0;
  for (int r = 0; r < m; r++) out[idx[r]] = A[r][m] / A[r][r];
  return true;
}

// Minimise c^T S c - 2 b^T c over c >= 0: the unconstrained solution if it
// is feasible, else the best feasible solution with some coefficients at 0.
void solve(const CostFit &f, double coef[3]) {
  double best[3] = {0, 0, 0}, best_e = INFINITY;
  for (unsigned sel = 7; sel >= 1; sel--) {
    double c[3];
    if (!solve_subset(f.S, f.b, sel, c)) continue;
    if (c[0] < 0 || c[1] < 0 || c[2] < 0) continue;
    double e = 0;
    for (int i = 0; i < 3; i++) {
      e -= 2 * f.b[i] * c[i];
      for (int j = 0; j < 3; j++) e += c[i] * f.S[i][j] * c[j];
    }
    if (e < best_e) {
      best_e = e;
      memcpy(best, c, sizeof(best));
    }
    if (sel == 7) break;  // the unconstrained optimum is feasible
  }
  if (best_e < INFINITY) memcpy(coef, best, sizeof(best));
}

template <class T>
void add_point(T &f, double g, double x, double t, double w) {
  const double fe[3] = {1.0, g, x};
  const double it = 1.0 / t;
  for (int i = 0; i < 3; i++) {
    f.b[i] += w * fe[i] * it;
    for (int j = 0; j < 3; j++) f.S[i][j] += w * fe[i] * fe[j] * it * it;
  }
}

// Prior plus every bin, each scaled to count at most kBinCap samples.
void totals(const CostFit &f, CostFit &tot) {
  memcpy(tot.S, f.S, sizeof(tot.S));
  memcpy(tot.b, f.b, sizeof(tot.b));
  for (const auto &kv : f.bins) {
    const CostSums &s = kv.second;
    const double w = s.count > kBinCap ? kBinCap / (double)s.count : 1.0;
    for (int i = 0; i < 3; i++) {
      tot.b[i] += w * s.b[i];
      for (int j = 0; j < 3; j++) tot.S[i][j] += w * s.S[i][j];
    }
  }
}

double eval(const double coef[3], double g, double x) { return coef[0] + coef[1] * g + coef[2] * x; }

// The built-in values as pseudo-samples spread over the model's range: a
// small cone with few patterns, a small cone with many, a large cone with
// few and a large one with many.
void seed(CostFit &f, Builtin bi) {
  f = CostFit();
  f.coef[0] = bi.a_ms;
  f.coef[1] = bi.c_ms;
  f.coef[2] = bi.alpha_ms;
  if (bi.a_ms <= 0) return;
  for (double g : {100.0, 5000.0})
    for (int n : {12, 32}) {
      const double x = g * ldexp(1.0, n - 23);
      add_point(f, g, x, eval(f.coef, g, x), kPriorWeight);
    }
}

void seed_compile(CostFit &f) {
  f = CostFit();
  f.coef[0] = kCompile.a_ms;
  f.coef[1] = kCompile.c_ms;
  for (double tables : {100.0, 2000.0}) {  // plain least squares in (1, tables)
    const double t = kCompile.a_ms + kCompile.c_ms * tables, fe[2] = {1.0, tables};
    for (int i = 0; i < 2; i++) {
      f.b[i] += kPriorWeight * fe[i] * t;
      for (int j = 0; j < 2; j++) f.S[i][j] += kPriorWeight * fe[i] * fe[j];
    }
  }
}

void ensure(CostModel &m) {
  if (m.ready) return;
  for (int t = 0; t < 4; t++) seed(m.tier[t], kRun[t]);
  seed(m.kernel, kKernel);
  seed_compile(m.compile);
  m.ready = true;
}

}  // namespace

double cost_x(uint32_t gates, uint32_t n) { return (double)gates * ldexp(1.0, (int)n - 23); }

double cost_kernel_x(double lop3, uint32_t n) { return (lop3 + kPassOverhead) * ldexp(1.0, (int)n - 23); }

double cost_run_ms(lec_es_ctx *c, uint32_t tier, uint32_t gates, uint32_t n, double lop3) {
  if (tier > 3 || tier == 0) tier = LEC_ES_TIER_INTERP;
  const bool by_lop3 = tier == LEC_ES_TIER_JIT && lop3 > 0;
  const double x = by_lop3 ? cost_kernel_x(lop3, n) : cost_x(gates, n);
  if (!c) {
    const Builtin b = by_lop3 ? kKernel : kRun[tier];
    const double co[3] = {b.a_ms, b.c_ms, b.alpha_ms};
    return eval(co, gates, x);
  }
  std::lock_guard<std::mutex> g(c->cost.mu);
  ensure(c->cost);
  return eval(by_lop3 ? c->cost.kernel.coef : c->cost.tier[tier].coef, gates, x);
}

double cost_compile_ms(lec_es_ctx *c, uint32_t tables) {
  if (!c) return kCompile.a_ms + kCompile.c_ms * tables;
  std::lock_guard<std::mutex> g(c->cost.mu);
  ensure(c->cost);
  return c->cost.compile.coef[0] + c->cost.compile.coef[1] * tables;
}

void cost_add_run(lec_es_ctx *c, uint32_t tier, uint32_t gates, uint32_t n, double ms, double lop3) {
  if (!c || tier == 0 || tier > 3 || !(ms > 0)) return;
  std::lock_guard<std::mutex> g(c->cost.mu);
  ensure(c->cost);
  const uint32_t lg = gates ? 32u - (uint32_t)__builtin_clz(gates) : 0u;
  auto fold = [&](CostFit &f, double x) {
    CostSums &bin = f.bins[n << 8 | lg];
    add_point(bin, gates, x, ms, 1.0);
    bin.count++;
    f.samples++;
    CostFit tot;
    totals(f, tot);
    solve(tot, f.coef);
  };
  fold(c->cost.tier[tier], cost_x(gates, n));
  if (tier == LEC_ES_TIER_JIT && lop3 > 0) fold(c->cost.kernel, cost_kernel_x(lop3, n));
}

void cost_add_compile(lec_es_ctx *c, uint32_t tables, double ms) {
  if (!c || !(ms > 0)) return;
  std::lock_guard<std::mutex> g(c->cost.mu);
  ensure(c->cost);
  CostFit &f = c->cost.compile;
  const double fe[2] = {1.0, (double)tables};
  for (int i = 0; i < 2; i++) {
    f.b[i] += fe[i] * ms;
    for (int j = 0; j < 2; j++) f.S[i][j] += fe[i] * fe[j];
  }
  f.samples++;
  const double det = f.S[0][0] * f.S[1][1] - f.S[0][1] * f.S[1][0];
  if (det > 0) {
    const double a = (f.b[0] * f.S[1][1] - f.S[0][1] * f.b[1]) / det;
    const double b = (f.S[0][0] * f.b[1] - f.S[1][0] * f.b[0]) / det;
    if (a >= 0 && b >= 0) {
      f.coef[0] = a;
      f.coef[1] = b;
    }
  }
}

bool cost_fit(const double *g, const double *x, const double *t, size_t k, double coef[3]) {
  CostFit f;
  for (size_t i = 0; i < k; i++) {
    if (!(t[i] > 0) || !(x[i] >= 0) || !(g[i] >= 0)) return false;
    add_point(f, g[i], x[i], t[i], 1.0);
  }
  if (!k) return false;
  coef[0] = coef[1] = coef[2] = 0;
  solve(f, coef);
  return true;
}

}  // namespace lec

using namespace lec;

extern "C" int lec_es_cost_fit(const uint32_t *gates, const uint32_t *n, const double *ms, size_t k,
                               lec_es_cost_coeffs *out) {
  if (!gates || !n || !ms || !out || k == 0) return LEC_ES_EINVAL;
  std::vector<double> g(k), x(k), t(k);
  for (size_t i = 0; i < k; i++) {
    if (n[i] > 63) return LEC_ES_EINVAL;
    g[i] = gates[i];
    x[i] = cost_x(gates[i], n[i]);
    t[i] = ms[i];
  }
  double co[3];
  if (!cost_fit(g.data(), x.data(), t.data(), k, co)) return LEC_ES_EINVAL;
  out->a_ms = co[0];
  out->c_ms = co[1];
  out->alpha_ms = co[2];
  out->samples = k;
  return LEC_ES_OK;
}

extern "C" int lec_es_cost_model(lec_es_ctx *c, uint32_t tier, lec_es_cost_coeffs *out) {
  if (!out || tier == 0 || tier > 5) return LEC_ES_EINVAL;
  if (!c) {
    const Builtin b = tier == 5 ? kKernel : tier == 4 ? kCompile : kRun[tier];
    out->a_ms = b.a_ms;
    out->c_ms = b.c_ms;
    out->alpha_ms = b.alpha_ms;
    out->samples = 0;
    return LEC_ES_OK;
  }
  std::lock_guard<std::mutex> g(c->cost.mu);
  ensure(c->cost);
  const CostFit &f = tier == 5 ? c->cost.kernel : tier == 4 ? c->cost.compile : c->cost.tier[tier];
  out->a_ms = f.coef[0];
  out->c_ms = f.coef[1];
  out->alpha_ms = f.coef[2];
  out->samples = f.samples;
  return LEC_ES_OK;
}

extern "C" int lec_es_cost_predict(lec_es_ctx *c, const lec_es_miter *m, uint32_t cpu_threads, lec_es_cost *out) {
  if (!m || !out) return LEC_ES_EINVAL;
  Program g;
  MiterView v{m->num_pis, m->num_ands, m->fanins, m->out_lit};
  int rc;
  try {
    if (c) {
      JitProbe jp{c, JitProbe::kInfo};
      const KernelProbe probe{jit_probe, &jp};
      rc = compile_program(v, LEC_ES_ORDER_AUTO, c->max_pis, g, &probe);
    } else {
      rc = compile_program(v, LEC_ES_ORDER_AUTO, 63, g);
    }
  } catch (const std::bad_alloc &) {
    return LEC_ES_ENOMEM;
  }
  if (rc) return rc;
  memset(out, 0, sizeof(*out));
  out->gates = g.cone_ands;
  out->n = g.n;
  out->num_luts = g.lut.count;
  out->interp_ms = cost_run_ms(c, LEC_ES_TIER_INTERP, g.cone_ands, g.n);
  out->jit_ms = cost_run_ms(c, LEC_ES_TIER_JIT, g.cone_ands, g.n, c ? jit_held_lop3(c, g) : 0.0);
  out->jit_compile_ms = g.lut.elided ? 0.0 : cost_compile_ms(c, g.lut.count);
  out->tier = jit_auto_tier(c, g, num_chunks(g.n));
  // an AUTO check never waits for a build: a cone whose kernel the context
  // does not hold starts on the interpreter (and may hand the rest of its
  // range to the kernel once the background build lands)
  if (out->tier == LEC_ES_TIER_JIT && c && !jit_held(c, g)) out->tier = LEC_ES_TIER_INTERP;
  // the paper's one-core CPU model and its GPU-offload rule (§3.2): ES goes
  // to the GPU when its predicted time on the given CPU threads exceeds 0.1 s
  out->paper_cpu_s = 0.0003 * cost_x(g.cone_ands, g.n);
  out->gpu_offload = out->paper_cpu_s / (double)std::max<uint32_t>(1, cpu_threads) > 0.1 ? 1u : 0u;
  return LEC_ES_OK;
}
