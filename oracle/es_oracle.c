/*
 * es_oracle.c -- CPU oracle for exact simulation (ES).  TEST INFRASTRUCTURE
 * ONLY: tests, the smoke check and the benchmark's CPU-baseline leg call it;
 * the product path never does.  It shares no code with the CUDA path.
 *
 * What it computes.  ES "enumerates all the possible assignments of PI and
 * checks the corresponding output of the miter" (paper §2.2, paragraph
 * "Exact Simulation"); a miter is equivalent iff its output is identically
 * zero (§2.1).  Because ES reaches exactly this definitional result, the
 * oracle is the definition written out, one 64-pattern word at a time in
 * ascending pattern order, with one value per AIG node (no slot reuse, so the
 * reference-count slot allocator of §3.3 is checked independently).
 *
 * Pattern numbering (the paper is silent; reading stated here):
 *   - the support S of the output is the set of PIs in its transitive fan-in
 *     cone (§2.1), sorted by PI index; n = |S|;
 *   - pattern p assigns bit k of p to support PI S[k];
 *   - word w holds patterns 64w .. 64w+63 (bit b of the word = pattern 64w+b),
 *     so PI S[k] for k < 6 is the constant mask MASK[k] and for k >= 6 is all
 *     ones iff bit (k-6) of w is set;
 *   - there are max(1, 2^(n-6)) words; for n < 6 only the low 2^n bits of the
 *     single word are patterns;
 *   - the counterexample returned is the lowest failing p.
 *
 * Error returns: 0 ok, -1 bad argument (literal out of range, fanin not below
 * its AND, n > 63), -2 out of memory.  Nothing aborts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static const uint64_t MASK[6] = {
    0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
    0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};

/* Cone of out_lit: marks reached variables, returns sorted support and the
 * ascending list of AND variables in the cone (ascending variable order is a
 * topological order because every fanin variable is below its AND). */
typedef struct {
  uint32_t n;         /* support size */
  uint32_t *support;  /* n PI indices, 0-based, ascending */
  uint32_t nands;
  uint32_t *ands;     /* AND variables of the cone, ascending */
} cone_t;

static void cone_free(cone_t *c) {
  free(c->support);
  free(c->ands);
  c->support = c->ands = NULL;
}

static int cone_build(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                      uint32_t out_lit, cone_t *c) {
  uint64_t maxvar = (uint64_t)num_pis + num_ands;
  memset(c, 0, sizeof(*c));
  if ((out_lit >> 1) > maxvar) return ORACLE_EINVAL;
  uint8_t *seen = calloc(maxvar + 1, 1);
  uint32_t *stack = malloc(sizeof(uint32_t) * (maxvar + 2));
  if (!seen || !stack) { free(seen); free(stack); return ORACLE_ENOMEM; }
  uint32_t sp = 0;
  stack[sp++] = out_lit >> 1;
  while (sp) {
    uint32_t v = stack[--sp];
    if (seen[v]) continue;
    seen[v] = 1;
    if (v > num_pis) {
      const uint32_t *f = fanins + 2 * (uint64_t)(v - num_pis - 1);
      for (int e = 0; e < 2; e++) {
        uint32_t u = f[e] >> 1;
        if (u >= v) { free(seen); free(stack); return ORACLE_EINVAL; }
        if (!seen[u]) stack[sp++] = u;
      }
    }
  }
  uint32_t n = 0, na = 0;
  for (uint64_t v = 1; v <= maxvar; v++) {
    if (!seen[v]) continue;
    if (v <= num_pis) n++; else na++;
  }
  if (n > 63) { free(seen); free(stack); return ORACLE_EINVAL; }
  c->support = malloc(sizeof(uint32_t) * (n + 1));
  c->ands = malloc(sizeof(uint32_t) * (na + 1));
  if (!c->support || !c->ands) { free(seen); free(stack); cone_free(c); return ORACLE_ENOMEM; }
  for (uint64_t v = 1; v <= maxvar; v++) {
    if (!seen[v]) continue;
    if (v <= num_pis) c->support[c->n++] = (uint32_t)(v - 1);
    else c->ands[c->nands++] = (uint32_t)v;
  }
  free(seen);
  free(stack);
  return ORACLE_OK;
}

/* value of literal l: node value, complemented when the literal's low bit is set */
static inline uint64_t lit_val(const uint64_t *val, uint32_t l) {
  return val[l >> 1] ^ ((l & 1) ? ~0ull : 0ull);
}

static uint64_t num_words(uint32_t n) { return n <= 6 ? 1ull : (1ull << (n - 6)); }

/* bits of the single word that are real patterns when n < 6 */
static uint64_t valid_mask(uint32_t n) {
  if (n >= 6) return ~0ull;
  return (1ull << (1u << n)) - 1ull; /* n = 0 gives 1: one pattern */
}

/* Set the support PIs for word w (the pattern layout in the header). */
static void load_pis(uint64_t *val, const cone_t *c, uint64_t w) {
  for (uint32_t k = 0; k < c->n; k++) {
    uint64_t x = (k < 6) ? MASK[k] : (((w >> (k - 6)) & 1) ? ~0ull : 0ull);
    val[c->support[k] + 1] = x;
  }
}

/* Evaluate every cone AND for the current PI values, ascending variable order. */
static void eval_cone(uint64_t *val, const cone_t *c, uint32_t num_pis, const uint32_t *fanins) {
  val[0] = 0; /* constant FALSE */
  for (uint32_t i = 0; i < c->nands; i++) {
    uint32_t v = c->ands[i];
    const uint32_t *f = fanins + 2 * (uint64_t)(v - num_pis - 1);
    val[v] = lit_val(val, f[0]) & lit_val(val, f[1]);
  }
}

/* Support of out_lit (sorted PI indices).  support must hold num_pis entries. */
int oracle_support(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, uint32_t out_lit,
                   uint32_t *support, uint32_t *n_out, uint32_t *cone_ands_out) {
  cone_t c;
  int rc = cone_build(num_pis, num_ands, fanins, out_lit, &c);
  if (rc) return rc;
  if (support) memcpy(support, c.support, sizeof(uint32_t) * c.n);
  if (n_out) *n_out = c.n;
  if (cone_ands_out) *cone_ands_out = c.nands;
  cone_free(&c);
  return ORACLE_OK;
}

/*
 * ES over words [word_begin, word_end) of the cone's pattern space (clipped to
 * its word count).  mode 0: stop at the first failing pattern (ascending), as
 * the verdict needs; mode 1: scan the whole range and count failing patterns.
 * *first_cex = lowest failing pattern in the range, or UINT64_MAX if none.
 */
int oracle_check(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, uint32_t out_lit,
                 uint64_t word_begin, uint64_t word_end, int mode, uint64_t *first_cex,
                 uint64_t *fail_count, uint32_t *n_out) {
  cone_t c;
  int rc = cone_build(num_pis, num_ands, fanins, out_lit, &c);
  if (rc) return rc;
  uint64_t *val = calloc((uint64_t)num_pis + num_ands + 1, sizeof(uint64_t));
  if (!val) { cone_free(&c); return ORACLE_ENOMEM; }
  uint64_t W = num_words(c.n);
  if (word_end > W) word_end = W;
  uint64_t vm = valid_mask(c.n);
  uint64_t first = UINT64_MAX, count = 0;
  for (uint64_t w = word_begin; w < word_end; w++) {
    load_pis(val, &c, w);
    eval_cone(val, &c, num_pis, fanins);
    uint64_t o = lit_val(val, out_lit) & vm;
    if (o) {
      if (first == UINT64_MAX) first = 64 * w + (uint64_t)__builtin_ctzll(o);
      count += (uint64_t)__builtin_popcountll(o);
      if (mode == 0) break;
    }
  }
  if (first_cex) *first_cex = first;
  if (fail_count) *fail_count = count;
  if (n_out) *n_out = c.n;
  free(val);
  cone_free(&c);
  return ORACLE_OK;
}

/*
 * Per-node truth tables over words [word_begin, word_end) of out_lit's cone
 * pattern space.  vars[j] must be 0, a support PI variable or an AND of the
 * cone; out[j * (word_end - word_begin) + (w - word_begin)] = value of var j.
 */
int oracle_truth_tables(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, uint32_t out_lit,
                        uint64_t word_begin, uint64_t word_end, const uint32_t *vars, uint32_t nvars,
                        uint64_t *out) {
  cone_t c;
  int rc = cone_build(num_pis, num_ands, fanins, out_lit, &c);
  if (rc) return rc;
  uint64_t W = num_words(c.n);
  if (word_end > W || word_begin > word_end) { cone_free(&c); return ORACLE_EINVAL; }
  uint64_t *val = calloc((uint64_t)num_pis + num_ands + 1, sizeof(uint64_t));
  if (!val) { cone_free(&c); return ORACLE_ENOMEM; }
  uint64_t nw = word_end - word_begin;
  for (uint32_t j = 0; j < nvars; j++)
    if (vars[j] > num_pis + num_ands) { free(val); cone_free(&c); return ORACLE_EINVAL; }
  for (uint64_t w = word_begin; w < word_end; w++) {
    load_pis(val, &c, w);
    eval_cone(val, &c, num_pis, fanins);
    for (uint32_t j = 0; j < nvars; j++) out[(uint64_t)j * nw + (w - word_begin)] = val[vars[j]];
  }
  free(val);
  cone_free(&c);
  return ORACLE_OK;
}

/*
 * Evaluate literals at explicit patterns.  pi_words[k * nw + j] holds PI k's
 * value in 64 patterns (word j); every AND of the graph is evaluated in
 * ascending order.  out[i * nw + j] = value of lits[i] in word j.
 */
int oracle_eval_patterns(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins,
                         const uint64_t *pi_words, uint64_t nw, const uint32_t *lits, uint32_t nl,
                         uint64_t *out) {
  uint64_t maxvar = (uint64_t)num_pis + num_ands;
  for (uint32_t i = 0; i < nl; i++)
    if ((lits[i] >> 1) > maxvar) return ORACLE_EINVAL;
  for (uint64_t a = 0; a < num_ands; a++)
    if ((fanins[2 * a] >> 1) > num_pis + a || (fanins[2 * a + 1] >> 1) > num_pis + a)
      return ORACLE_EINVAL;
  uint64_t *val = calloc(maxvar + 1, sizeof(uint64_t));
  if (!val) return ORACLE_ENOMEM;
  for (uint64_t j = 0; j < nw; j++) {
    val[0] = 0;
    for (uint32_t k = 0; k < num_pis; k++) val[k + 1] = pi_words[(uint64_t)k * nw + j];
    for (uint64_t a = 0; a < num_ands; a++)
      val[num_pis + 1 + a] = lit_val(val, fanins[2 * a]) & lit_val(val, fanins[2 * a + 1]);
    for (uint32_t i = 0; i < nl; i++) out[(uint64_t)i * nw + j] = lit_val(val, lits[i]);
  }
  free(val);
  return ORACLE_OK;
}
