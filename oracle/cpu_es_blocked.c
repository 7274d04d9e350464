/*
 * cpu_es_blocked.c -- a CPU exact-simulation baseline in the paper's CPU
 * setting.  TEST INFRASTRUCTURE ONLY: the benchmark's CPU-baseline leg times
 * it and tests pin it against es_oracle.c; the product path never runs it,
 * and it shares no code with the CUDA path (nor with es_oracle.c).
 *
 * What it computes: the same answer as the oracle -- ES of the miter output
 * over a word range, lowest failing pattern (paper §2.2 "Exact Simulation";
 * pattern numbering as in es_oracle.c).  How: the way the paper's CPU-ES
 * runs (§3.3, instructionalized ES and its "Effectiveness" paragraph): the
 * cone becomes an instruction stream over value rows reused once a node's
 * last reader has run (reference counts), and each thread simulates a block
 * of 2^14 patterns (256 64-bit words) per pass through the stream, over its
 * own contiguous share of the words.  Threads stop at their first failing
 * block, or as soon as another thread has found a failure below their
 * current block.
 *
 * Returns 0 ok, -1 bad argument (literal out of range, fanin not below its
 * AND, n > 63, block_words = 0), -2 out of memory.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const uint64_t PI_MASK[6] = {
    0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
    0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};

/* One instruction: row dst = (row a ^ ma) & (row b ^ mb). */
typedef struct {
  uint32_t dst, a, b;
  uint64_t ma, mb;
} instr_t;

typedef struct {
  uint32_t n;            /* support size */
  uint32_t npi_rows;     /* rows 0..n-1 hold the support PIs, row n the constant 0 */
  uint32_t nrows;        /* rows in all */
  uint32_t ninstr;
  instr_t *instr;
  uint32_t out_row;
  uint64_t out_mask;     /* complement of the output literal */
} stream_t;

/* Cone of out_lit, then the instruction stream in ascending variable order
 * with each AND's row freed after its last reader (the output's row is
 * never freed). */
static int build_stream(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, uint32_t out_lit,
                        stream_t *s) {
  memset(s, 0, sizeof(*s));
  const uint64_t maxvar = (uint64_t)num_pis + num_ands;
  if ((out_lit >> 1) > maxvar) return -1;
  uint8_t *in = calloc(maxvar + 1, 1);
  uint32_t *stack = malloc(sizeof(uint32_t) * (maxvar + 2));
  uint32_t *last = calloc(maxvar + 1, sizeof(uint32_t)); /* index of the last reading AND, +1 */
  uint32_t *row = malloc(sizeof(uint32_t) * (maxvar + 1));
  if (!in || !stack || !last || !row) {
    free(in); free(stack); free(last); free(row);
    return -2;
  }
  uint32_t sp = 0;
  stack[sp++] = out_lit >> 1;
  while (sp) {
    const uint32_t v = stack[--sp];
    if (in[v]) continue;
    in[v] = 1;
    if (v > num_pis) {
      const uint32_t *f = fanins + 2 * (uint64_t)(v - num_pis - 1);
      for (int e = 0; e < 2; e++) {
        const uint32_t u = f[e] >> 1;
        if (u >= v) { free(in); free(stack); free(last); free(row); return -1; }
        if (!in[u]) stack[sp++] = u;
      }
    }
  }
  uint32_t n = 0, na = 0;
  for (uint64_t v = 1; v <= maxvar; v++)
    if (in[v]) {
      if (v <= num_pis) row[v] = n++;
      else na++;
    }
  if (n > 63) { free(in); free(stack); free(last); free(row); return -1; }
  s->n = n;
  s->npi_rows = n;
  row[0] = n; /* the constant */
  /* last readers, in ascending order of the ANDs */
  uint32_t k = 0;
  for (uint64_t v = num_pis + 1; v <= maxvar; v++) {
    if (!in[v]) continue;
    k++;
    const uint32_t *f = fanins + 2 * (uint64_t)(v - num_pis - 1);
    last[f[0] >> 1] = k;
    last[f[1] >> 1] = k;
  }
  s->instr = malloc(sizeof(instr_t) * (na + 1));
  uint32_t *free_rows = malloc(sizeof(uint32_t) * (na + 1));
  if (!s->instr || !free_rows) { free(in); free(stack); free(last); free(row); free(free_rows); return -2; }
  uint32_t nfree = 0, next_row = n + 1;
  k = 0;
  const uint32_t out_var = out_lit >> 1;
  for (uint64_t v = num_pis + 1; v <= maxvar; v++) {
    if (!in[v]) continue;
    k++;
    const uint32_t *f = fanins + 2 * (uint64_t)(v - num_pis - 1);
    instr_t *ins = &s->instr[s->ninstr++];
    ins->a = row[f[0] >> 1];
    ins->b = row[f[1] >> 1];
    ins->ma = (f[0] & 1) ? ~0ull : 0ull;
    ins->mb = (f[1] & 1) ? ~0ull : 0ull;
    /* operands whose last reader this is give their rows back first, so the
     * result may take one of them (operands are read before the write) */
    for (int e = 0; e < 2; e++) {
      const uint32_t u = f[e] >> 1;
      if (u > num_pis && u != out_var && last[u] == k && (e == 0 || (f[1] >> 1) != (f[0] >> 1)))
        free_rows[nfree++] = row[u];
    }
    row[v] = nfree ? free_rows[--nfree] : next_row++;
    ins->dst = row[v];
  }
  s->nrows = next_row;
  s->out_row = row[out_var];
  s->out_mask = (out_lit & 1) ? ~0ull : 0ull;
  free(in); free(stack); free(last); free(row); free(free_rows);
  return 0;
}

typedef struct {
  const stream_t *s;
  uint64_t lo, hi;          /* this thread's words */
  uint32_t block;
  _Atomic uint64_t *best;   /* lowest failing pattern found by any thread */
  uint64_t first;           /* this thread's result */
  int err;
} job_t;

static void *run_job(void *arg) {
  job_t *j = (job_t *)arg;
  const stream_t *s = j->s;
  const uint32_t B = j->block;
  j->first = UINT64_MAX;
  j->err = 0;
  uint64_t *rows = malloc(sizeof(uint64_t) * (uint64_t)s->nrows * B);
  if (!rows) { j->err = -2; return NULL; }
  memset(rows + (uint64_t)s->n * B, 0, sizeof(uint64_t) * B); /* the constant row */
  const uint64_t vm = s->n >= 6 ? ~0ull : ((1ull << (1u << s->n)) - 1ull);
  for (uint64_t w0 = j->lo; w0 < j->hi; w0 += B) {
    if (w0 * 64 >= atomic_load(j->best)) break; /* nothing lower left here */
    const uint64_t cnt = (j->hi - w0 < B) ? j->hi - w0 : B;
    for (uint32_t k = 0; k < s->n; k++) {
      uint64_t *r = rows + (uint64_t)k * B;
      for (uint64_t i = 0; i < cnt; i++)
        r[i] = k < 6 ? PI_MASK[k] : ((((w0 + i) >> (k - 6)) & 1) ? ~0ull : 0ull);
    }
    for (uint32_t q = 0; q < s->ninstr; q++) {
      const instr_t *ins = &s->instr[q];
      const uint64_t *a = rows + (uint64_t)ins->a * B, *b = rows + (uint64_t)ins->b * B;
      uint64_t *d = rows + (uint64_t)ins->dst * B;
      const uint64_t ma = ins->ma, mb = ins->mb;
      for (uint64_t i = 0; i < cnt; i++) d[i] = (a[i] ^ ma) & (b[i] ^ mb);
    }
    const uint64_t *o = rows + (uint64_t)s->out_row * B;
    for (uint64_t i = 0; i < cnt; i++) {
      const uint64_t x = (o[i] ^ s->out_mask) & vm;
      if (x) {
        j->first = 64 * (w0 + i) + (uint64_t)__builtin_ctzll(x);
        uint64_t cur = atomic_load(j->best);
        while (j->first < cur && !atomic_compare_exchange_weak(j->best, &cur, j->first)) {
        }
        break;
      }
    }
    if (j->first != UINT64_MAX) break;
  }
  free(rows);
  return NULL;
}

int cpu_es_blocked(uint32_t num_pis, uint32_t num_ands, const uint32_t *fanins, uint32_t out_lit,
                   uint64_t word_begin, uint64_t word_end, uint32_t block_words, uint32_t threads,
                   uint64_t *first_cex, uint32_t *n_out) {
  if (block_words == 0 || threads == 0) return -1;
  stream_t s;
  int rc = build_stream(num_pis, num_ands, fanins, out_lit, &s);
  if (rc) { free(s.instr); return rc; }
  const uint64_t W = s.n <= 6 ? 1ull : (1ull << (s.n - 6));
  if (word_end > W) word_end = W;
  uint64_t first = UINT64_MAX;
  if (word_begin < word_end) {
    const uint64_t total = word_end - word_begin;
    if (threads > total) threads = (uint32_t)total;
    job_t *jobs = calloc(threads, sizeof(job_t));
    pthread_t *th = calloc(threads, sizeof(pthread_t));
    _Atomic uint64_t best = UINT64_MAX;
    if (!jobs || !th) { free(jobs); free(th); free(s.instr); return -2; }
    const uint64_t per = (total + threads - 1) / threads;
    for (uint32_t t = 0; t < threads; t++) {
      jobs[t].s = &s;
      jobs[t].lo = word_begin + t * per < word_end ? word_begin + t * per : word_end;
      jobs[t].hi = jobs[t].lo + per < word_end ? jobs[t].lo + per : word_end;
      jobs[t].block = block_words;
      jobs[t].best = &best;
      if (pthread_create(&th[t], NULL, run_job, &jobs[t]) != 0) {
        jobs[t].err = -2;
        th[t] = 0;
      }
    }
    for (uint32_t t = 0; t < threads; t++) {
      if (th[t]) pthread_join(th[t], NULL);
      if (jobs[t].err) rc = jobs[t].err;
      if (jobs[t].first < first) first = jobs[t].first;
    }
    free(jobs);
    free(th);
  }
  free(s.instr);
  if (rc) return rc;
  if (first_cex) *first_cex = first;
  if (n_out) *n_out = s.n;
  return 0;
}
