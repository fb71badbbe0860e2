/*
 * CPU ORACLE -- test infrastructure, not part of the product.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code with the CUDA library: it is a plain, slow,
 * obviously correct restatement of the metrics of Napoli, Pappalardo and
 * Tramontana (CISIS 2013), written from the paper's definitions:
 *
 *   fan-in / fan-out ......... Sec. II.A (methods calling m / called by m)
 *   CBO ...................... Sec. II.B (other classes used by C)
 *   LCOM (Chidamber-Kemerer).. Sec. II.B (pairs sharing no attribute minus
 *                              pairs sharing one), clamped at zero
 *   LCOM (Henderson-Sellers).. Sec. II.B (1 - average over methods of the
 *                              fraction of C's attributes they use), kept as
 *                              an exact integer fraction
 *   move evaluation .......... Sec. III.A rules + Sec. IV.C (change the class
 *                              representation, compute the metrics again)
 *
 * Three evaluators live here:
 *   - metrics by definition (pair loops over sorted sets);
 *   - O0: for a candidate move (m -> D) it changes cls(m), recomputes every
 *     affected class by the definitions and compares (the paper's way);
 *   - O1: the incremental formulas (source/target LCOM updates and the
 *     class multigraph CBO update), checked against O0 by the tests.
 * Multi-threading (pthreads) only splits candidate rows; it changes no result.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n_classes, n_methods, n_attrs, cbo_attrs;
  const int32_t *method_class, *attr_class;
  const int64_t *acc_rowptr, *call_rowptr;
  const int32_t *acc_idx, *call_idx;
} or_input;

typedef struct {
  uint32_t metric_mask; /* 1 = LCOM_CK, 2 = LCOM_HS, 4 = CBO */
  int32_t min_improved;
} or_criteria;

/* per-class metric values */
typedef struct {
  int64_t n, a, P, Q, S, ck, hs_num, hs_den, cbo;
} or_cm;

/* the 16-byte move record: s, t, dCBO(source), dCBO(target), #improved,
 * #worsened, sign flags (2 bits per metric and class; 1 = lower, 2 = higher),
 * bit 15 = kept */
typedef struct {
  int32_t s;
  uint16_t t;
  int16_t dcbo_src, dcbo_dst;
  uint16_t n_improved, n_worsened, flags;
} or_record;

typedef struct {
  int32_t m, d, n_improved, d_ck_sum, d_cbo_sum, pad;
} or_kept;

typedef struct {
  or_input in;
  int32_t *mem_rowptr, *mem;     /* members of each class, ascending ids */
  int32_t *acount;               /* attributes owned per class */
  int64_t *caller_rowptr;        /* callers of each method, ascending */
  int32_t *caller;
  or_cm *cm;                     /* base class metrics */
  int32_t *fan_in, *fan_out, *own, *q;
  /* class multigraph without intra edges: row Y sorted by E, counts */
  int64_t *mg_rowptr;
  int32_t *mg_dst, *mg_cnt;
  uint64_t *mg_bits;             /* existence bitmap, c x ceil(c/64) */
  int64_t mg_words;
} or_sys;

/* ------------------------------------------------------------------ */
/* small helpers                                                        */

static int sgn64(int64_t v) { return (v > 0) - (v < 0); }

/* exact comparison of two fractions x1/y1 and x2/y2 with y1, y2 > 0 */
static int frac_cmp(int64_t x1, int64_t y1, int64_t x2, int64_t y2) {
  __int128 l = (__int128)x1 * y2, r = (__int128)x2 * y1;
  return (l > r) - (l < r);
}

/* is there an attribute owned by Y accessed by both x and y? (sorted merge) */
static int shares(const or_input *in, int32_t x, int32_t y, int32_t Y) {
  int64_t i = in->acc_rowptr[x], ie = in->acc_rowptr[x + 1];
  int64_t j = in->acc_rowptr[y], je = in->acc_rowptr[y + 1];
  while (i < ie && j < je) {
    int32_t u = in->acc_idx[i], v = in->acc_idx[j];
    if (u < v) ++i;
    else if (v < u) ++j;
    else {
      if (in->attr_class[u] == Y) return 1;
      ++i; ++j;
    }
  }
  return 0;
}

static int64_t own_count(const or_input *in, int32_t x, int32_t Y) {
  int64_t k = 0;
  for (int64_t e = in->acc_rowptr[x]; e < in->acc_rowptr[x + 1]; ++e)
    if (in->attr_class[in->acc_idx[e]] == Y) ++k;
  return k;
}

/* ------------------------------------------------------------------ */
/* class metrics by definition                                          */

/*
 * Metrics of class Y whose members are mem[0..n) under the class map cls
 * (cls is only used to find the classes of called methods).  stamp/tag give
 * a scratch "seen" array of n_classes entries for the distinct-class count.
 */
static void class_metrics_def(const or_sys *s, int32_t Y, const int32_t *mem, int64_t n,
                              const int32_t *cls, int64_t *stamp, int64_t tag, or_cm *out) {
  const or_input *in = &s->in;
  or_cm r;
  r.n = n;
  r.a = s->acount[Y];
  r.P = 0; r.Q = 0; r.S = 0;
  for (int64_t i = 0; i < n; ++i) {
    r.S += own_count(in, mem[i], Y);
    for (int64_t j = i + 1; j < n; ++j) {
      if (shares(in, mem[i], mem[j], Y)) r.Q++;
      else r.P++;
    }
  }
  r.ck = r.P > r.Q ? r.P - r.Q : 0;
  if (r.n * r.a == 0) { r.hs_num = 0; r.hs_den = 1; }
  else { r.hs_num = r.n * r.a - r.S; r.hs_den = r.n * r.a; }
  /* CBO: distinct other classes used by the members */
  int64_t cbo = 0;
  stamp[Y] = tag;
  for (int64_t i = 0; i < n; ++i) {
    int32_t x = mem[i];
    for (int64_t e = in->call_rowptr[x]; e < in->call_rowptr[x + 1]; ++e) {
      int32_t E = cls[in->call_idx[e]];
      if (stamp[E] != tag) { stamp[E] = tag; ++cbo; }
    }
    if (in->cbo_attrs)
      for (int64_t e = in->acc_rowptr[x]; e < in->acc_rowptr[x + 1]; ++e) {
        int32_t E = in->attr_class[in->acc_idx[e]];
        if (stamp[E] != tag) { stamp[E] = tag; ++cbo; }
      }
  }
  r.cbo = cbo;
  *out = r;
}

/* ------------------------------------------------------------------ */
/* system set-up                                                        */

void or_free(or_sys *s) {
  if (!s) return;
  free(s->mem_rowptr); free(s->mem); free(s->acount); free(s->caller_rowptr); free(s->caller);
  free(s->cm); free(s->fan_in); free(s->fan_out); free(s->own); free(s->q);
  free(s->mg_rowptr); free(s->mg_dst); free(s->mg_cnt); free(s->mg_bits);
  free(s);
}

typedef struct {
  or_sys *s;
  int32_t next, end;
  pthread_mutex_t mu;
} base_job;

static void *base_worker(void *arg) {
  base_job *j = (base_job *)arg;
  or_sys *s = j->s;
  const or_input *in = &s->in;
  int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)in->n_classes);
  for (int32_t i = 0; i < in->n_classes; ++i) stamp[i] = -1;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    int32_t Y = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (Y >= j->end) break;
    const int32_t *mem = s->mem + s->mem_rowptr[Y];
    int64_t n = s->mem_rowptr[Y + 1] - s->mem_rowptr[Y];
    class_metrics_def(s, Y, mem, n, in->method_class, stamp, Y, &s->cm[Y]);
    for (int64_t i = 0; i < n; ++i) {
      int32_t x = mem[i], qx = 0;
      for (int64_t k = 0; k < n; ++k)
        if (k != i && shares(in, x, mem[k], Y)) ++qx;
      s->q[x] = qx;
      s->own[x] = (int32_t)own_count(in, x, Y);
    }
  }
  free(stamp);
  return NULL;
}

static int cmp_pair64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

/*
 * Copy the input, build member lists, callers, base metrics (by definition)
 * and the class multigraph.  Returns NULL on allocation failure or invalid
 * input (ids out of range).
 */
or_sys *or_build(const or_input *inp, int n_threads) {
  or_sys *s = (or_sys *)calloc(1, sizeof(or_sys));
  if (!s) return NULL;
  s->in = *inp;
  const or_input *in = &s->in;
  int32_t c = in->n_classes, M = in->n_methods;
  for (int32_t x = 0; x < M; ++x)
    if (in->method_class[x] < 0 || in->method_class[x] >= c) { or_free(s); return NULL; }
  s->mem_rowptr = (int32_t *)calloc((size_t)c + 1, sizeof(int32_t));
  s->mem = (int32_t *)malloc(sizeof(int32_t) * ((size_t)M + 1));
  s->acount = (int32_t *)calloc((size_t)c + 1, sizeof(int32_t));
  s->cm = (or_cm *)calloc((size_t)c + 1, sizeof(or_cm));
  s->fan_in = (int32_t *)calloc((size_t)M + 1, sizeof(int32_t));
  s->fan_out = (int32_t *)calloc((size_t)M + 1, sizeof(int32_t));
  s->own = (int32_t *)calloc((size_t)M + 1, sizeof(int32_t));
  s->q = (int32_t *)calloc((size_t)M + 1, sizeof(int32_t));
  s->caller_rowptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
  int64_t ncall = in->call_rowptr[M];
  s->caller = (int32_t *)malloc(sizeof(int32_t) * ((size_t)ncall + 1));
  if (!s->mem_rowptr || !s->mem || !s->acount || !s->cm || !s->fan_in || !s->fan_out || !s->own ||
      !s->q || !s->caller_rowptr || !s->caller) { or_free(s); return NULL; }
  /* members: ascending method ids per class */
  for (int32_t x = 0; x < M; ++x) s->mem_rowptr[in->method_class[x] + 1]++;
  for (int32_t Y = 0; Y < c; ++Y) s->mem_rowptr[Y + 1] += s->mem_rowptr[Y];
  {
    int32_t *fill = (int32_t *)calloc((size_t)c, sizeof(int32_t));
    for (int32_t x = 0; x < M; ++x) {
      int32_t Y = in->method_class[x];
      s->mem[s->mem_rowptr[Y] + fill[Y]++] = x;
    }
    free(fill);
  }
  for (int32_t a = 0; a < in->n_attrs; ++a) s->acount[in->attr_class[a]]++;
  /* fan-out = number of called methods; fan-in = number of callers */
  for (int32_t x = 0; x < M; ++x) {
    s->fan_out[x] = (int32_t)(in->call_rowptr[x + 1] - in->call_rowptr[x]);
    for (int64_t e = in->call_rowptr[x]; e < in->call_rowptr[x + 1]; ++e) s->fan_in[in->call_idx[e]]++;
  }
  for (int32_t x = 0; x < M; ++x) s->caller_rowptr[x + 1] = s->caller_rowptr[x] + s->fan_in[x];
  {
    int64_t *fill = (int64_t *)calloc((size_t)M, sizeof(int64_t));
    for (int32_t y = 0; y < M; ++y) /* ascending y => ascending caller lists */
      for (int64_t e = in->call_rowptr[y]; e < in->call_rowptr[y + 1]; ++e) {
        int32_t x = in->call_idx[e];
        s->caller[s->caller_rowptr[x] + fill[x]++] = y;
      }
    free(fill);
  }
  /* base metrics by definition */
  {
    base_job j;
    j.s = s; j.next = 0; j.end = c;
    pthread_mutex_init(&j.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t th[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, base_worker, &j);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
  }
  /* multigraph: (Y, E) for every use edge with E != Y; sort, run-length */
  {
    int64_t cap = ncall + (in->cbo_attrs ? in->acc_rowptr[M] : 0);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)cap + 1));
    int64_t k = 0;
    for (int32_t x = 0; x < M; ++x) {
      int32_t Y = in->method_class[x];
      for (int64_t e = in->call_rowptr[x]; e < in->call_rowptr[x + 1]; ++e) {
        int32_t E = in->method_class[in->call_idx[e]];
        if (E != Y) keys[k++] = ((uint64_t)(uint32_t)Y << 32) | (uint32_t)E;
      }
      if (in->cbo_attrs)
        for (int64_t e = in->acc_rowptr[x]; e < in->acc_rowptr[x + 1]; ++e) {
          int32_t E = in->attr_class[in->acc_idx[e]];
          if (E != Y) keys[k++] = ((uint64_t)(uint32_t)Y << 32) | (uint32_t)E;
        }
    }
    qsort(keys, (size_t)k, sizeof(uint64_t), cmp_pair64);
    int64_t u = 0;
    for (int64_t i = 0; i < k; ++i)
      if (i == 0 || keys[i] != keys[i - 1]) ++u;
    s->mg_rowptr = (int64_t *)calloc((size_t)c + 1, sizeof(int64_t));
    s->mg_dst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)u + 1));
    s->mg_cnt = (int32_t *)malloc(sizeof(int32_t) * ((size_t)u + 1));
    s->mg_words = ((int64_t)c + 63) / 64;
    s->mg_bits = (uint64_t *)calloc((size_t)(s->mg_words * c) + 1, sizeof(uint64_t));
    if (!s->mg_rowptr || !s->mg_dst || !s->mg_cnt || !s->mg_bits) { free(keys); or_free(s); return NULL; }
    int64_t w = -1;
    for (int64_t i = 0; i < k; ++i) {
      if (i == 0 || keys[i] != keys[i - 1]) {
        ++w;
        int32_t Y = (int32_t)(keys[i] >> 32), E = (int32_t)(keys[i] & 0xffffffffu);
        s->mg_dst[w] = E;
        s->mg_cnt[w] = 0;
        s->mg_rowptr[Y + 1]++;
        s->mg_bits[(int64_t)Y * s->mg_words + E / 64] |= 1ULL << (E % 64);
      }
      s->mg_cnt[w]++;
    }
    for (int32_t Y = 0; Y < c; ++Y) s->mg_rowptr[Y + 1] += s->mg_rowptr[Y];
    free(keys);
  }
  return s;
}

/* number of use edges from class Y into class E (Y != E), before any move */
static int32_t mg_count(const or_sys *s, int32_t Y, int32_t E) {
  if (!((s->mg_bits[(int64_t)Y * s->mg_words + E / 64] >> (E % 64)) & 1)) return 0;
  int64_t lo = s->mg_rowptr[Y], hi = s->mg_rowptr[Y + 1];
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (s->mg_dst[mid] < E) lo = mid + 1; else hi = mid;
  }
  return (lo < s->mg_rowptr[Y + 1] && s->mg_dst[lo] == E) ? s->mg_cnt[lo] : 0;
}

/* ------------------------------------------------------------------ */
/* accessors                                                            */

void or_class_metrics(const or_sys *s, or_cm *out) {
  memcpy(out, s->cm, sizeof(or_cm) * (size_t)s->in.n_classes);
}

void or_method_metrics(const or_sys *s, int32_t *fan_in, int32_t *fan_out, int32_t *own, int32_t *q) {
  size_t M = (size_t)s->in.n_methods;
  memcpy(fan_in, s->fan_in, M * 4); memcpy(fan_out, s->fan_out, M * 4);
  memcpy(own, s->own, M * 4); memcpy(q, s->q, M * 4);
}

int64_t or_multigraph(const or_sys *s, int64_t *rowptr, int32_t *dst, int32_t *cnt) {
  int64_t u = s->mg_rowptr[s->in.n_classes];
  if (rowptr) memcpy(rowptr, s->mg_rowptr, sizeof(int64_t) * ((size_t)s->in.n_classes + 1));
  if (dst) memcpy(dst, s->mg_dst, sizeof(int32_t) * (size_t)u);
  if (cnt) memcpy(cnt, s->mg_cnt, sizeof(int32_t) * (size_t)u);
  return u;
}

/* ------------------------------------------------------------------ */
/* record assembly shared by O0 and O1 (pure bookkeeping of signs)      */

static uint16_t sat_u16(int64_t v) { return v < 0 ? 0 : (v > 65535 ? 65535 : (uint16_t)v); }
static int16_t sat_i16(int64_t v) { return v < -32768 ? -32768 : (v > 32767 ? 32767 : (int16_t)v); }
static uint16_t enc(int sg) { return sg < 0 ? 1 : (sg > 0 ? 2 : 0); }

/* per-class outcome: improved (no metric higher, one lower) / worsened */
static void tally(uint32_t mask, int s_ck, int s_hs, int s_cbo, int64_t *imp, int64_t *wor) {
  int up = 0, down = 0;
  if (mask & 1) { up |= s_ck > 0; down |= s_ck < 0; }
  if (mask & 2) { up |= s_hs > 0; down |= s_hs < 0; }
  if (mask & 4) { up |= s_cbo > 0; down |= s_cbo < 0; }
  if (up) ++*wor;
  else if (down) ++*imp;
}

static int hs_sign(const or_cm *before, const or_cm *after) {
  /* LCOM_HS after vs before, as exact fractions */
  return frac_cmp(after->hs_num, after->hs_den, before->hs_num, before->hs_den);
}

/* ------------------------------------------------------------------ */
/* O0: change cls(m), recompute affected classes by definition          */

typedef struct {
  int32_t *cls;     /* private copy of method_class */
  int64_t *stamp;   /* n_classes */
  int64_t tag;
  int32_t *memb;    /* scratch member list */
  int32_t *aff;     /* affected classes */
} o0_scratch;

static void o0_eval(const or_sys *s, const or_criteria *cr, int32_t m, int32_t D, o0_scratch *w,
                    or_record *rec, int64_t *d_ck_sum, int64_t *d_cbo_sum) {
  const or_input *in = &s->in;
  int32_t C = in->method_class[m];
  /* affected classes: source, target, and classes of m's callers */
  int32_t naff = 0;
  w->tag++;
  w->aff[naff++] = C; w->stamp[C] = w->tag;
  if (w->stamp[D] != w->tag) { w->aff[naff++] = D; w->stamp[D] = w->tag; }
  for (int64_t e = s->caller_rowptr[m]; e < s->caller_rowptr[m + 1]; ++e) {
    int32_t X = in->method_class[s->caller[e]];
    if (w->stamp[X] != w->tag) { w->stamp[X] = w->tag; w->aff[naff++] = X; }
  }
  w->cls[m] = D;
  int64_t imp = 0, wor = 0;
  int sck[2] = {0, 0}, shs[2] = {0, 0}, scb[2] = {0, 0};
  int64_t dcbo[2] = {0, 0}, dck[2] = {0, 0};
  for (int32_t i = 0; i < naff; ++i) {
    int32_t Y = w->aff[i];
    /* members of Y after the move */
    int64_t n = 0;
    for (int32_t k = s->mem_rowptr[Y]; k < s->mem_rowptr[Y + 1]; ++k)
      if (s->mem[k] != m) w->memb[n++] = s->mem[k];
    if (Y == D) { /* insert m keeping ascending order */
      int64_t p = n;
      while (p > 0 && w->memb[p - 1] > m) { w->memb[p] = w->memb[p - 1]; --p; }
      w->memb[p] = m; ++n;
    }
    or_cm after;
    w->tag++;
    class_metrics_def(s, Y, w->memb, n, w->cls, w->stamp, w->tag, &after);
    const or_cm *before = &s->cm[Y];
    int c_ck = sgn64(after.ck - before->ck);
    int c_hs = hs_sign(before, &after);
    int c_cb = sgn64(after.cbo - before->cbo);
    tally(cr->metric_mask, c_ck, c_hs, c_cb, &imp, &wor);
    int slot = (Y == C) ? 0 : (Y == D ? 1 : -1);
    if (slot >= 0) {
      sck[slot] = c_ck; shs[slot] = c_hs; scb[slot] = c_cb;
      dcbo[slot] = after.cbo - before->cbo;
      dck[slot] = after.ck - before->ck;
    }
  }
  w->cls[m] = C;
  /* t = m's accesses to D's attributes; s = members of D sharing one of them */
  int64_t t = own_count(in, m, D), sh = 0;
  for (int32_t k = s->mem_rowptr[D]; k < s->mem_rowptr[D + 1]; ++k)
    if (shares(in, m, s->mem[k], D)) ++sh;
  rec->s = (int32_t)sh;
  rec->t = sat_u16(t);
  rec->dcbo_src = sat_i16(dcbo[0]);
  rec->dcbo_dst = sat_i16(dcbo[1]);
  rec->n_improved = sat_u16(imp);
  rec->n_worsened = sat_u16(wor);
  uint16_t f = (uint16_t)(enc(sck[0]) | enc(shs[0]) << 2 | enc(scb[0]) << 4 |
                          enc(sck[1]) << 6 | enc(shs[1]) << 8 | enc(scb[1]) << 10);
  if (wor == 0 && imp >= cr->min_improved) f |= 1u << 15;
  rec->flags = f;
  *d_ck_sum = dck[0] + dck[1];
  *d_cbo_sum = dcbo[0] + dcbo[1];
}

/* ------------------------------------------------------------------ */
/* O1: incremental formulas                                             */

typedef struct { int32_t key, val, aux; } kv3;

static int cmp_kv3(const void *a, const void *b) {
  int32_t x = ((const kv3 *)a)->key, y = ((const kv3 *)b)->key;
  return (x > y) - (x < y);
}

static const kv3 *kv_find(const kv3 *v, int32_t n, int32_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) { int32_t mid = (lo + hi) / 2; if (v[mid].key < key) lo = mid + 1; else hi = mid; }
  return (lo < n && v[lo].key == key) ? &v[lo] : NULL;
}

typedef struct {
  kv3 *T;  int32_t nT;   /* E -> out_m[E] (use edges of m into E), E != C */
  kv3 *R;  int32_t nR;   /* X -> in_m[X] (callers of m in X), X != C */
  kv3 *O;  int32_t nO;   /* D -> (t, s) for classes owning attributes m accesses, D != C */
  int32_t out_self, in_self;  /* m's use edges into C; m's callers inside C */
  int32_t cap;
} o1_pre;

static void o1_prepare(const or_sys *s, int32_t m, o1_pre *p) {
  const or_input *in = &s->in;
  int32_t C = in->method_class[m];
  int64_t nc = in->call_rowptr[m + 1] - in->call_rowptr[m];
  int64_t na = in->acc_rowptr[m + 1] - in->acc_rowptr[m];
  int64_t nr = s->caller_rowptr[m + 1] - s->caller_rowptr[m];
  int64_t need = nc + na + nr + 1;
  if (need > p->cap) {
    p->cap = (int32_t)need;
    p->T = (kv3 *)realloc(p->T, sizeof(kv3) * (size_t)need);
    p->R = (kv3 *)realloc(p->R, sizeof(kv3) * (size_t)need);
    p->O = (kv3 *)realloc(p->O, sizeof(kv3) * (size_t)need);
  }
  /* T: all use edges of m by target class, then merged */
  int32_t k = 0;
  for (int64_t e = in->call_rowptr[m]; e < in->call_rowptr[m + 1]; ++e)
    p->T[k++] = (kv3){in->method_class[in->call_idx[e]], 1, 0};
  if (in->cbo_attrs)
    for (int64_t e = in->acc_rowptr[m]; e < in->acc_rowptr[m + 1]; ++e)
      p->T[k++] = (kv3){in->attr_class[in->acc_idx[e]], 1, 0};
  qsort(p->T, (size_t)k, sizeof(kv3), cmp_kv3);
  int32_t w = 0;
  p->out_self = 0;
  for (int32_t i = 0; i < k; ++i) {
    if (p->T[i].key == C) { p->out_self++; continue; }
    if (w > 0 && p->T[w - 1].key == p->T[i].key) p->T[w - 1].val++;
    else p->T[w++] = p->T[i];
  }
  p->nT = w;
  /* R: callers by class */
  k = 0;
  for (int64_t e = s->caller_rowptr[m]; e < s->caller_rowptr[m + 1]; ++e)
    p->R[k++] = (kv3){in->method_class[s->caller[e]], 1, 0};
  qsort(p->R, (size_t)k, sizeof(kv3), cmp_kv3);
  w = 0;
  p->in_self = 0;
  for (int32_t i = 0; i < k; ++i) {
    if (p->R[i].key == C) { p->in_self++; continue; }
    if (w > 0 && p->R[w - 1].key == p->R[i].key) p->R[w - 1].val++;
    else p->R[w++] = p->R[i];
  }
  p->nR = w;
  /* O: owner classes of m's attributes, with t and s */
  k = 0;
  for (int64_t e = in->acc_rowptr[m]; e < in->acc_rowptr[m + 1]; ++e) {
    int32_t D = in->attr_class[in->acc_idx[e]];
    if (D != C) p->O[k++] = (kv3){D, 1, 0};
  }
  qsort(p->O, (size_t)k, sizeof(kv3), cmp_kv3);
  w = 0;
  for (int32_t i = 0; i < k; ++i) {
    if (w > 0 && p->O[w - 1].key == p->O[i].key) p->O[w - 1].val++;
    else p->O[w++] = p->O[i];
  }
  p->nO = w;
  for (int32_t i = 0; i < w; ++i) {
    int32_t D = p->O[i].key, sh = 0;
    for (int32_t j = s->mem_rowptr[D]; j < s->mem_rowptr[D + 1]; ++j)
      if (shares(in, m, s->mem[j], D)) ++sh;
    p->O[i].aux = sh;
  }
}

static int pos(int64_t v) { return v > 0; }

static void o1_eval(const or_sys *s, const or_criteria *cr, int32_t m, int32_t D, const o1_pre *p,
                    or_record *rec, int64_t *d_ck_sum, int64_t *d_cbo_sum) {
  const or_input *in = &s->in;
  int32_t C = in->method_class[m];
  const or_cm *bc = &s->cm[C], *bd = &s->cm[D];
  /* source class after the move: one method fewer */
  or_cm ac = *bc;
  ac.n = bc->n - 1;
  ac.S = bc->S - s->own[m];
  ac.Q = bc->Q - s->q[m];
  ac.P = bc->P - (bc->n - 1 - s->q[m]);
  /* target class after the move: one method more */
  const kv3 *o = kv_find(p->O, p->nO, D);
  int64_t t = o ? o->val : 0, sh = o ? o->aux : 0;
  or_cm ad = *bd;
  ad.n = bd->n + 1;
  ad.S = bd->S + t;
  ad.Q = bd->Q + sh;
  ad.P = bd->P + (bd->n - sh);
  or_cm *pair[2] = {&ac, &ad};
  for (int i = 0; i < 2; ++i) {
    or_cm *r = pair[i];
    r->ck = r->P > r->Q ? r->P - r->Q : 0;
    if (r->n * r->a == 0) { r->hs_num = 0; r->hs_den = 1; }
    else { r->hs_num = r->n * r->a - r->S; r->hs_den = r->n * r->a; }
  }
  /* CBO through the class multigraph cnt[Y][E]:
   *   row C loses m's out-edges and gains C->D for m's callers in C;
   *   row D gains m's out-edges and loses D->C for m's callers in D;
   *   row X (other caller classes) moves in_m[X] edges from X->C to X->D. */
  const kv3 *tD = kv_find(p->T, p->nT, D);
  const kv3 *rD = kv_find(p->R, p->nR, D);
  int64_t outD = tD ? tD->val : 0, inD = rD ? rD->val : 0;
  int64_t dC = 0, dD = 0;
  for (int32_t i = 0; i < p->nT; ++i) { /* E in T(m), E != C */
    int32_t E = p->T[i].key;
    int64_t o_e = p->T[i].val;
    if (E != D) {
      int64_t b = mg_count(s, C, E);
      dC += pos(b - o_e) - pos(b);
      int64_t bd2 = mg_count(s, D, E);
      dD += pos(bd2 + o_e) - pos(bd2);
    }
  }
  { /* E = D for row C */
    int64_t b = mg_count(s, C, D);
    dC += pos(b - outD + p->in_self) - pos(b);
  }
  { /* E = C for row D */
    int64_t b = mg_count(s, D, C);
    dD += pos(b + p->out_self - inD) - pos(b);
  }
  ac.cbo = bc->cbo + dC;
  ad.cbo = bd->cbo + dD;
  int64_t imp = 0, wor = 0;
  int sck0 = sgn64(ac.ck - bc->ck), shs0 = hs_sign(bc, &ac), scb0 = sgn64(dC);
  int sck1 = sgn64(ad.ck - bd->ck), shs1 = hs_sign(bd, &ad), scb1 = sgn64(dD);
  tally(cr->metric_mask, sck0, shs0, scb0, &imp, &wor);
  tally(cr->metric_mask, sck1, shs1, scb1, &imp, &wor);
  for (int32_t i = 0; i < p->nR; ++i) { /* other classes calling m: only CBO moves */
    int32_t X = p->R[i].key;
    if (X == D) continue;
    int64_t inX = p->R[i].val;
    int64_t bxc = mg_count(s, X, C), bxd = mg_count(s, X, D);
    int64_t dx = pos(bxc - inX) - pos(bxc) + pos(bxd + inX) - pos(bxd);
    tally(cr->metric_mask, 0, 0, sgn64(dx), &imp, &wor);
  }
  rec->s = (int32_t)sh;
  rec->t = sat_u16(t);
  rec->dcbo_src = sat_i16(dC);
  rec->dcbo_dst = sat_i16(dD);
  rec->n_improved = sat_u16(imp);
  rec->n_worsened = sat_u16(wor);
  uint16_t f = (uint16_t)(enc(sck0) | enc(shs0) << 2 | enc(scb0) << 4 |
                          enc(sck1) << 6 | enc(shs1) << 8 | enc(scb1) << 10);
  if (wor == 0 && imp >= cr->min_improved) f |= 1u << 15;
  rec->flags = f;
  *d_ck_sum = (ac.ck - bc->ck) + (ad.ck - bd->ck);
  *d_cbo_sum = dC + dD;
}

/* ------------------------------------------------------------------ */
/* digest of a record: SplitMix64 (published output function) chained  */

static uint64_t smix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_record_hash(int32_t m, int32_t D, const or_record *r) {
  uint64_t lo, hi;
  memcpy(&lo, r, 8);
  memcpy(&hi, (const char *)r + 8, 8);
  uint64_t key = ((uint64_t)(uint32_t)m << 32) | (uint32_t)D;
  return smix(key ^ smix(lo ^ smix(hi)));
}

/* ------------------------------------------------------------------ */
/* threaded driver over candidate rows                                  */

typedef struct {
  const or_sys *s;
  const or_criteria *cr;
  const int64_t *cand_rowptr;  /* NULL => all D != cls(m) */
  const int32_t *cand_dst;
  int32_t row_begin, row_end;
  int method;                  /* 0 = O0, 1 = O1 */
  or_record *records;          /* nullable; indexed from the first candidate of row_begin */
  int64_t base_index;
  int32_t next;
  pthread_mutex_t mu;
  uint64_t digest;
  or_kept *kept;
  int64_t n_kept, kept_cap;
  int64_t n_cand;
  int status;
} drive_job;

static int64_t row_start(const drive_job *j, int32_t m) {
  if (j->cand_rowptr) return j->cand_rowptr[m];
  return (int64_t)m * (j->s->in.n_classes - 1);
}

static void *drive_worker(void *arg) {
  drive_job *j = (drive_job *)arg;
  const or_sys *s = j->s;
  const or_input *in = &s->in;
  int32_t c = in->n_classes;
  o0_scratch w0;
  memset(&w0, 0, sizeof w0);
  o1_pre p1;
  memset(&p1, 0, sizeof p1);
  if (j->method == 0) {
    w0.cls = (int32_t *)malloc(sizeof(int32_t) * (size_t)in->n_methods);
    memcpy(w0.cls, in->method_class, sizeof(int32_t) * (size_t)in->n_methods);
    w0.stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)c);
    for (int32_t i = 0; i < c; ++i) w0.stamp[i] = 0;
    w0.tag = 0;
    w0.memb = (int32_t *)malloc(sizeof(int32_t) * ((size_t)in->n_methods + 1));
    w0.aff = (int32_t *)malloc(sizeof(int32_t) * ((size_t)c + 1));
  }
  uint64_t dig = 0;
  or_kept *kl = NULL;
  int64_t nk = 0, kcap = 0, ncand = 0;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    int32_t m0 = j->next;
    j->next += 16;
    pthread_mutex_unlock(&j->mu);
    if (m0 >= j->row_end) break;
    int32_t m1 = m0 + 16 < j->row_end ? m0 + 16 : j->row_end;
    for (int32_t m = m0; m < m1; ++m) {
      int32_t C = in->method_class[m];
      if (j->method == 1) o1_prepare(s, m, &p1);
      int64_t i0 = row_start(j, m);
      int64_t len = j->cand_rowptr ? j->cand_rowptr[m + 1] - j->cand_rowptr[m] : c - 1;
      for (int64_t k = 0; k < len; ++k) {
        int32_t D = j->cand_rowptr ? j->cand_dst[i0 + k] : (int32_t)(k < C ? k : k + 1);
        if (D < 0 || D >= c || D == C) { j->status = 1; continue; }
        or_record r;
        int64_t dck, dcb;
        if (j->method == 0) o0_eval(s, j->cr, m, D, &w0, &r, &dck, &dcb);
        else o1_eval(s, j->cr, m, D, &p1, &r, &dck, &dcb);
        ++ncand;
        dig += or_record_hash(m, D, &r);
        if (j->records) j->records[i0 + k - j->base_index] = r;
        if (r.flags & 0x8000u) {
          if (nk == kcap) { kcap = kcap ? 2 * kcap : 1024; kl = (or_kept *)realloc(kl, sizeof(or_kept) * (size_t)kcap); }
          kl[nk++] = (or_kept){m, D, r.n_improved, (int32_t)dck, (int32_t)dcb, 0};
        }
      }
    }
  }
  pthread_mutex_lock(&j->mu);
  j->digest += dig;
  j->n_cand += ncand;
  if (nk) {
    if (j->n_kept + nk > j->kept_cap) {
      j->kept_cap = (j->n_kept + nk) * 2;
      j->kept = (or_kept *)realloc(j->kept, sizeof(or_kept) * (size_t)j->kept_cap);
    }
    memcpy(j->kept + j->n_kept, kl, sizeof(or_kept) * (size_t)nk);
    j->n_kept += nk;
  }
  pthread_mutex_unlock(&j->mu);
  free(kl);
  free(w0.cls); free(w0.stamp); free(w0.memb); free(w0.aff);
  free(p1.T); free(p1.R); free(p1.O);
  return NULL;
}

/* suggestion order: more improved classes first, then the lower LCOM_CK
 * change sum, then the lower CBO change sum, then method id, then class id */
static int cmp_kept(const void *a, const void *b) {
  const or_kept *x = (const or_kept *)a, *y = (const or_kept *)b;
  if (x->n_improved != y->n_improved) return x->n_improved > y->n_improved ? -1 : 1;
  if (x->d_ck_sum != y->d_ck_sum) return x->d_ck_sum < y->d_ck_sum ? -1 : 1;
  if (x->d_cbo_sum != y->d_cbo_sum) return x->d_cbo_sum < y->d_cbo_sum ? -1 : 1;
  if (x->m != y->m) return x->m < y->m ? -1 : 1;
  return (x->d > y->d) - (x->d < y->d);
}

typedef struct {
  uint64_t digest;
  int64_t n_cand, n_kept, n_methods_with_kept;
  or_kept *kept;   /* sorted; free with or_free_kept */
  int status;
} or_eval_result;

/*
 * Evaluate candidate rows [row_begin, row_end) with O0 (method=0) or O1
 * (method=1).  records (nullable) receives the record of candidate i at
 * records[i - first candidate index of row_begin].
 */
int or_evaluate(const or_sys *s, const or_criteria *cr, const int64_t *cand_rowptr, const int32_t *cand_dst,
                int32_t row_begin, int32_t row_end, int method, int n_threads, or_record *records,
                or_eval_result *res) {
  drive_job j;
  memset(&j, 0, sizeof j);
  j.s = s; j.cr = cr; j.cand_rowptr = cand_rowptr; j.cand_dst = cand_dst;
  j.row_begin = row_begin; j.row_end = row_end; j.method = method;
  j.records = records; j.next = row_begin;
  j.base_index = cand_rowptr ? cand_rowptr[row_begin] : (int64_t)row_begin * (s->in.n_classes - 1);
  pthread_mutex_init(&j.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, drive_worker, &j);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&j.mu);
  if (j.n_kept > 1) qsort(j.kept, (size_t)j.n_kept, sizeof(or_kept), cmp_kept);
  /* distinct methods among kept moves */
  int64_t nm = 0;
  if (j.n_kept) {
    uint8_t *seen = (uint8_t *)calloc((size_t)s->in.n_methods, 1);
    for (int64_t i = 0; i < j.n_kept; ++i)
      if (!seen[j.kept[i].m]) { seen[j.kept[i].m] = 1; ++nm; }
    free(seen);
  }
  res->digest = j.digest;
  res->n_cand = j.n_cand;
  res->n_kept = j.n_kept;
  res->n_methods_with_kept = nm;
  res->kept = j.kept;
  res->status = j.status;
  return j.status;
}

void or_free_kept(or_kept *k) { free(k); }

/* Evaluate one candidate with O0 or O1 (single-threaded convenience). */
int or_evaluate_one(const or_sys *s, const or_criteria *cr, int32_t m, int32_t D, int method,
                    or_record *rec, int64_t *d_ck_sum, int64_t *d_cbo_sum) {
  const or_input *in = &s->in;
  if (m < 0 || m >= in->n_methods || D < 0 || D >= in->n_classes || D == in->method_class[m]) return 1;
  if (method == 0) {
    o0_scratch w;
    w.cls = (int32_t *)malloc(sizeof(int32_t) * (size_t)in->n_methods);
    memcpy(w.cls, in->method_class, sizeof(int32_t) * (size_t)in->n_methods);
    w.stamp = (int64_t *)calloc((size_t)in->n_classes, sizeof(int64_t));
    w.tag = 0;
    w.memb = (int32_t *)malloc(sizeof(int32_t) * ((size_t)in->n_methods + 1));
    w.aff = (int32_t *)malloc(sizeof(int32_t) * ((size_t)in->n_classes + 1));
    o0_eval(s, cr, m, D, &w, rec, d_ck_sum, d_cbo_sum);
    free(w.cls); free(w.stamp); free(w.memb); free(w.aff);
  } else {
    o1_pre p;
    memset(&p, 0, sizeof p);
    o1_prepare(s, m, &p);
    o1_eval(s, cr, m, D, &p, rec, d_ck_sum, d_cbo_sum);
    free(p.T); free(p.R); free(p.O);
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Jaccard similarity of method pairs (Sec. II.A) and rule R1 (Sec.      */
/* III.A, first rule and its footnote)                                    */
/*                                                                        */
/* The properties of a method are the methods it calls and the          */
/* attributes it accesses (two id spaces, never equal to each other).    */
/* sim(x, y) = |P(x) and P(y)| / |P(x) or P(y)|, kept as the exact pair   */
/* (i, u).  Only pairs with i > 0 are values (a pair sharing nothing has  */
/* similarity 0 and is not stored, Sec. IV.C).                            */

/* number of common elements of two strictly increasing rows (sorted merge) */
static int64_t common_sorted(const int32_t *a, int64_t na, const int32_t *b, int64_t nb) {
  int64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) ++i;
    else if (b[j] < a[i]) ++j;
    else { ++k; ++i; ++j; }
  }
  return k;
}

/* i and u of the pair (x, y) by the definition */
static void sim_pair(const or_input *in, int32_t x, int32_t y, int64_t *i_out, int64_t *u_out) {
  const int64_t ax = in->acc_rowptr[x], nax = in->acc_rowptr[x + 1] - ax;
  const int64_t ay = in->acc_rowptr[y], nay = in->acc_rowptr[y + 1] - ay;
  const int64_t cx = in->call_rowptr[x], ncx = in->call_rowptr[x + 1] - cx;
  const int64_t cy = in->call_rowptr[y], ncy = in->call_rowptr[y + 1] - cy;
  const int64_t i = common_sorted(in->acc_idx + ax, nax, in->acc_idx + ay, nay) +
                    common_sorted(in->call_idx + cx, ncx, in->call_idx + cy, ncy);
  *i_out = i;
  *u_out = nax + ncx + nay + ncy - i;
}

typedef struct {
  const or_sys *s;
  int32_t x0, x1;                  /* rows of this worker */
  int64_t n;                       /* pairs found */
  int32_t *px, *py, *pi, *pu;      /* output (NULL: count only) */
  int64_t cap;
} sim_job;

static void *sim_worker(void *arg) {
  sim_job *j = (sim_job *)arg;
  const or_input *in = &j->s->in;
  int64_t n = 0;
  for (int32_t x = j->x0; x < j->x1; ++x)
    for (int32_t y = x + 1; y < in->n_methods; ++y) {
      int64_t i, u;
      sim_pair(in, x, y, &i, &u);
      if (i == 0) continue;
      if (j->px && n < j->cap) {
        j->px[n] = x; j->py[n] = y; j->pi[n] = (int32_t)i; j->pu[n] = (int32_t)u;
      }
      ++n;
    }
  j->n = n;
  return NULL;
}

/*
 * Every pair x < y with a common property, in (x, y) order: x, y, i, u.
 * Returns the number of such pairs; with NULL outputs only counts.  Rows of
 * x are split over threads in two passes (count, then write at the offsets).
 */
int64_t or_similarity(const or_sys *s, int n_threads, int32_t *px, int32_t *py, int32_t *pi, int32_t *pu) {
  const int32_t M = s->in.n_methods;
  if (n_threads < 1) n_threads = 1;
  /* rows split so that each thread gets about the same number of pairs */
  int32_t *bounds = (int32_t *)calloc((size_t)n_threads + 1, sizeof(int32_t));
  sim_job *jobs = (sim_job *)calloc((size_t)n_threads, sizeof(sim_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!bounds || !jobs || !th) { free(bounds); free(jobs); free(th); return -1; }
  {
    const double total = (double)M * (M - 1) / 2.0;
    int32_t x = 0;
    double acc = 0;
    for (int t = 1; t < n_threads; ++t) {
      while (x < M && acc < total * t / n_threads) { acc += (double)(M - 1 - x); ++x; }
      bounds[t] = x;
    }
    bounds[n_threads] = M;
  }
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].s = s; jobs[t].x0 = bounds[t]; jobs[t].x1 = bounds[t + 1];
    jobs[t].px = NULL;
    pthread_create(&th[t], NULL, sim_worker, &jobs[t]);
  }
  int64_t total = 0;
  for (int t = 0; t < n_threads; ++t) { pthread_join(th[t], NULL); total += jobs[t].n; }
  if (px) {
    int64_t off = 0;
    for (int t = 0; t < n_threads; ++t) {
      const int64_t nt = jobs[t].n;
      jobs[t].px = px + off; jobs[t].py = py + off; jobs[t].pi = pi + off; jobs[t].pu = pu + off;
      jobs[t].cap = nt;
      off += nt;
      pthread_create(&th[t], NULL, sim_worker, &jobs[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  }
  free(bounds); free(jobs); free(th);
  return total;
}

/* every y != x with a common property with x, ascending y: y, i, u */
int64_t or_similarity_row(const or_sys *s, int32_t x, int32_t *py, int32_t *pi, int32_t *pu) {
  int64_t n = 0;
  for (int32_t y = 0; y < s->in.n_methods; ++y) {
    if (y == x) continue;
    int64_t i, u;
    sim_pair(&s->in, x, y, &i, &u);
    if (i == 0) continue;
    if (py) { py[n] = y; pi[n] = (int32_t)i; pu[n] = (int32_t)u; }
    ++n;
  }
  return n;
}

/*
 * The R1 threshold (footnote of Sec. III.A: the average of the system's
 * similarity values; the values are the pairs that share a property).  The
 * average is taken in double precision in one fixed order -- the sum over u
 * ascending of (sum of i over the pairs with union u) / u, divided by the
 * number of pairs -- and a pair is "high" when (double)i / (double)u exceeds
 * it.  thr[u] (u = 0 .. umax) receives the smallest i for which that holds
 * (u + 1 when none).  Returns the average.
 */
double or_r1_threshold(const int32_t *pi, const int32_t *pu, int64_t n, int32_t umax, int32_t *thr) {
  int64_t *sum_i = (int64_t *)calloc((size_t)umax + 1, sizeof(int64_t));
  if (!sum_i) return -1.0;
  for (int64_t k = 0; k < n; ++k) sum_i[pu[k]] += pi[k];
  double s = 0.0;
  for (int32_t u = 1; u <= umax; ++u)
    if (sum_i[u]) s += (double)sum_i[u] / (double)u;
  const double avg = n > 0 ? s / (double)n : 0.0;
  for (int32_t u = 0; u <= umax; ++u) {
    int32_t t = u + 1;
    for (int32_t i = 0; i <= u; ++i)
      if (u > 0 && (double)i / (double)u > avg) { t = i; break; }
    thr[u] = t;
  }
  free(sum_i);
  return avg;
}

/* ------------------------------------------------------------------ */
/* metric variants (Sec. II.B)                                          */
/*
 * The paper states LCOM as pairs sharing no attribute minus pairs sharing one
 * without saying whose attributes, and CBO as the classes C uses; the CK suite
 * it cites counts coupling in both directions.  The variants, by definition:
 *   P_all, Q_all, ck_all: LCOM_CK with sharing over every accessed attribute
 *                         (of any class), clamped at 0 like ck;
 *   pq, pq_all:           the unclamped differences P - Q and P_all - Q_all;
 *   cbo_out:              CBO as above (classes C uses);
 *   cbo_in:               other classes that use C;
 *   cbo_bi:               other classes coupled to C either way (|out u in|).
 * q_all[x]: methods of x's class sharing an accessed attribute with x.
 */
typedef struct {
  int64_t P_all, Q_all, ck_all, pq, pq_all, cbo_out, cbo_in, cbo_bi;
} or_cv;

/* is there an attribute (of any class) accessed by both x and y? (sorted merge) */
static int shares_any(const or_input *in, int32_t x, int32_t y) {
  int64_t i = in->acc_rowptr[x], ie = in->acc_rowptr[x + 1];
  int64_t j = in->acc_rowptr[y], je = in->acc_rowptr[y + 1];
  while (i < ie && j < je) {
    int32_t u = in->acc_idx[i], v = in->acc_idx[j];
    if (u < v) ++i;
    else if (v < u) ++j;
    else return 1;
  }
  return 0;
}

typedef struct {
  const or_sys *s;
  or_cv *out;
  int32_t *q_all;
  int32_t next, end;
  pthread_mutex_t mu;
} var_job;

static void *var_worker(void *arg) {
  var_job *j = (var_job *)arg;
  const or_sys *s = j->s;
  const or_input *in = &s->in;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    int32_t Y = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (Y >= j->end) break;
    const int32_t *mem = s->mem + s->mem_rowptr[Y];
    int64_t n = s->mem_rowptr[Y + 1] - s->mem_rowptr[Y];
    int64_t twice = 0; /* every sharing pair, once from each of its methods */
    for (int64_t i = 0; i < n; ++i) {
      int32_t qx = 0;
      for (int64_t k = 0; k < n; ++k)
        if (k != i && shares_any(in, mem[i], mem[k])) ++qx;
      j->q_all[mem[i]] = qx;
      twice += qx;
    }
    or_cv *r = &j->out[Y];
    r->Q_all = twice / 2;
    r->P_all = n * (n - 1) / 2 - r->Q_all;
    r->ck_all = r->P_all > r->Q_all ? r->P_all - r->Q_all : 0;
    r->pq = s->cm[Y].P - s->cm[Y].Q;
    r->pq_all = r->P_all - r->Q_all;
  }
  return NULL;
}

/* Fills out[n_classes] and q_all[n_methods]; 0 on success, -1 when out of memory. */
int or_class_variants(const or_sys *s, int n_threads, or_cv *out, int32_t *q_all) {
  const int32_t c = s->in.n_classes;
  var_job j;
  j.s = s; j.out = out; j.q_all = q_all; j.next = 0; j.end = c;
  pthread_mutex_init(&j.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, var_worker, &j);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&j.mu);
  /* coupling both ways: out(Y) is row Y of the multigraph (ascending E);
   * in(E) lists the rows Y that contain E, built by a counting pass over the
   * rows in ascending Y, so each in-list is ascending too */
  const int64_t u = s->mg_rowptr[c];
  int64_t *in_ptr = (int64_t *)calloc((size_t)c + 1, sizeof(int64_t));
  int32_t *in_row = (int32_t *)malloc(sizeof(int32_t) * ((size_t)u + 1));
  int64_t *fill = (int64_t *)calloc((size_t)c + 1, sizeof(int64_t));
  if (!in_ptr || !in_row || !fill) { free(in_ptr); free(in_row); free(fill); return -1; }
  for (int64_t k = 0; k < u; ++k) in_ptr[s->mg_dst[k] + 1]++;
  for (int32_t E = 0; E < c; ++E) in_ptr[E + 1] += in_ptr[E];
  for (int32_t Y = 0; Y < c; ++Y)
    for (int64_t k = s->mg_rowptr[Y]; k < s->mg_rowptr[Y + 1]; ++k) {
      int32_t E = s->mg_dst[k];
      in_row[in_ptr[E] + fill[E]++] = Y;
    }
  for (int32_t C = 0; C < c; ++C) {
    int64_t i = s->mg_rowptr[C], ie = s->mg_rowptr[C + 1], k = in_ptr[C], ke = in_ptr[C + 1];
    out[C].cbo_out = ie - i;
    out[C].cbo_in = ke - k;
    int64_t both = 0; /* size of the union of the two ascending lists */
    while (i < ie || k < ke) {
      if (k >= ke || (i < ie && s->mg_dst[i] < in_row[k])) ++i;
      else if (i >= ie || in_row[k] < s->mg_dst[i]) ++k;
      else { ++i; ++k; }
      ++both;
    }
    out[C].cbo_bi = both;
  }
  free(in_ptr); free(in_row); free(fill);
  return 0;
}
