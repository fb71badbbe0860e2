/*
 * Seeded synthetic-system generator.
 *
 * Produces object-oriented "systems" (classes, methods, attributes, method ->
 * attribute accesses, method -> method calls) shaped like the Java code bases
 * of the paper's evaluation (Table I: thousands of classes, methods roughly
 * 6-12x the class count, a Zipf-like class-size distribution).  The paper's
 * systems themselves are not available; these seeded inputs stand in for them.
 *
 * This module holds input generation only: it computes none of the metrics
 * (fan-in/out, LCOM, CBO) nor any move evaluation.  Both the CUDA library and
 * the CPU oracle consume its output.
 *
 * Randomness: one counter-based generator, u64 = splitmix64(seed*K1 ^ stream*K2
 * ^ index), where splitmix64 is the published SplitMix64 output function
 * (Steele, Lea and Flood, OOPSLA 2014).  Every draw has its own (stream, index)
 * so results do not depend on evaluation order.
 *
 * Layout of the generated system:
 *   - class sizes: rank-size Zipf law n_r = clamp(floor(K r^-s), 1, max) with
 *     the largest K whose total does not exceed M, then +1 to ranks 1,2,... still
 *     below max until the total is exactly M; ranks are mapped to class ids by a
 *     seeded Fisher-Yates shuffle.
 *   - method ids are contiguous by class id.
 *   - attributes: largest-remainder apportionment of n_attrs proportional to the
 *     class sizes (ties to the lower class id); ids contiguous by class.
 *   - accesses: Poisson(lambda_acc) draws per method; each draw takes, with
 *     probability p_loc, a uniform attribute of the own class (if it has any),
 *     otherwise a uniform attribute of a uniform other class that owns
 *     attributes.  Deduplicated and sorted.
 *   - calls: Poisson(lambda_call) draws per method; with probability p_loc a
 *     uniform other method of the own class (if the class has >= 2 methods),
 *     otherwise a uniform method of a uniform other class.  Deduplicated,
 *     sorted, never a self-call.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define K1 0xD1B54A32D192ED03ULL
#define K2 0xABC98388FB8FAC03ULL

enum {
  ST_SHUFFLE = 1,
  ST_POIS_ACC = 2,
  ST_ACC_LOC = 3,
  ST_ACC_CLS = 4,
  ST_ACC_ITEM = 5,
  ST_POIS_CALL = 6,
  ST_CALL_LOC = 7,
  ST_CALL_CLS = 8,
  ST_CALL_ITEM = 9,
  ST_CAND = 10,
  ST_SYS = 11,
  ST_EDIT = 12
};

static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_u64(uint64_t seed, uint64_t stream, uint64_t index) {
  return splitmix64(seed * K1 ^ stream * K2 ^ index);
}

/* uniform integer in [0, n), n < 2^32 */
static uint32_t uni_int(uint64_t seed, uint64_t stream, uint64_t index, uint32_t n) {
  uint64_t u32 = synth_u64(seed, stream, index) >> 32;
  return (uint32_t)((u32 * (uint64_t)n) >> 32);
}

/* uniform real in [0, 1) with 53 random bits */
static double uni_real(uint64_t seed, uint64_t stream, uint64_t index) {
  return (double)(synth_u64(seed, stream, index) >> 11) * (1.0 / 9007199254740992.0);
}

/* index of draw j of item x: x * 2^20 + j (j < 2^20) */
static uint64_t didx(int64_t x, int64_t j) { return ((uint64_t)x << 20) | (uint64_t)j; }

/* Poisson(lambda) by multiplying uniforms until the product drops below
 * exp(-lambda) (Knuth's method); each factor is its own counter draw. */
static int poisson(uint64_t seed, uint64_t stream, int64_t x, double lambda) {
  double limit = exp(-lambda), p = 1.0;
  int k = 0;
  for (;;) {
    p *= uni_real(seed, stream, didx(x, k));
    if (p < limit || k >= (1 << 19)) return k;
    ++k;
  }
}

typedef struct {
  int32_t n_classes, n_methods, n_attrs, max_class;
  double zipf_s, lambda_acc, lambda_call, p_loc;
  uint64_t seed;
} synth_params;

typedef struct {
  int32_t n_classes, n_methods, n_attrs, pad;
  int64_t n_acc, n_call;
  int32_t *method_class, *attr_class;
  int64_t *acc_rowptr, *call_rowptr;
  int32_t *acc_idx, *call_idx;
  int32_t *class_size; /* methods per class */
} synth_system;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* sort + dedupe in place, returns the new length */
static int64_t sort_unique(int32_t *v, int64_t n) {
  if (n <= 1) return n;
  qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
  int64_t w = 1;
  for (int64_t i = 1; i < n; ++i)
    if (v[i] != v[w - 1]) v[w++] = v[i];
  return w;
}

static int64_t g_rem_A, g_rem_M;
static const int32_t *g_rem_size;
static int cmp_rem(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  int64_t rx = (g_rem_A * g_rem_size[x]) % g_rem_M, ry = (g_rem_A * g_rem_size[y]) % g_rem_M;
  if (rx != ry) return rx > ry ? -1 : 1;
  return (x > y) - (x < y);
}

static int64_t zipf_total(double K, int32_t c, double s, int32_t mx) {
  int64_t t = 0;
  for (int32_t r = 1; r <= c; ++r) {
    double v = floor(K * pow((double)r, -s));
    int64_t n = v < 1.0 ? 1 : (v > (double)mx ? mx : (int64_t)v);
    t += n;
  }
  return t;
}

/* Rank-size class sizes with exact total; returns 0 on success. */
int synth_class_sizes(const synth_params *p, int32_t *size_by_class) {
  int32_t c = p->n_classes, M = p->n_methods, mx = p->max_class;
  if (c <= 0 || M < c || (int64_t)c * mx < M) return 1;
  int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
  if (!n) return 2;
  double lo = 0.0, hi = (double)mx * pow((double)c, p->zipf_s) + 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (zipf_total(mid, c, p->zipf_s, mx) <= M) lo = mid; else hi = mid;
  }
  int64_t tot = 0;
  for (int32_t r = 1; r <= c; ++r) {
    double v = floor(lo * pow((double)r, -p->zipf_s));
    n[r - 1] = v < 1.0 ? 1 : (v > (double)mx ? mx : (int32_t)v);
    tot += n[r - 1];
  }
  while (tot < M) {
    int progressed = 0;
    for (int32_t r = 0; r < c && tot < M; ++r)
      if (n[r] < mx) { n[r]++; tot++; progressed = 1; }
    if (!progressed) { free(n); return 1; }
  }
  /* rank -> class id by a seeded Fisher-Yates shuffle of the identity */
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
  if (!perm) { free(n); return 2; }
  for (int32_t i = 0; i < c; ++i) perm[i] = i;
  for (int32_t i = c - 1; i >= 1; --i) {
    int32_t j = (int32_t)uni_int(p->seed, ST_SHUFFLE, (uint64_t)i, (uint32_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  for (int32_t r = 0; r < c; ++r) size_by_class[perm[r]] = n[r];
  free(perm);
  free(n);
  return 0;
}

void synth_free(synth_system *s) {
  if (!s) return;
  free(s->method_class); free(s->attr_class); free(s->acc_rowptr); free(s->call_rowptr);
  free(s->acc_idx); free(s->call_idx); free(s->class_size);
  free(s);
}

int synth_generate(const synth_params *p, synth_system **out) {
  *out = NULL;
  int32_t c = p->n_classes, M = p->n_methods, A = p->n_attrs;
  if (c <= 0 || M <= 0 || A < 0) return 1;
  synth_system *s = (synth_system *)calloc(1, sizeof(synth_system));
  if (!s) return 2;
  s->n_classes = c; s->n_methods = M; s->n_attrs = A;
  s->class_size = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
  int32_t *mstart = (int32_t *)malloc(sizeof(int32_t) * ((size_t)c + 1));
  int32_t *astart = (int32_t *)malloc(sizeof(int32_t) * ((size_t)c + 1));
  int32_t *acnt = (int32_t *)calloc((size_t)c, sizeof(int32_t));
  int32_t *with_attrs = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
  s->method_class = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
  s->attr_class = (int32_t *)malloc(sizeof(int32_t) * ((size_t)A + 1));
  s->acc_rowptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)M + 1));
  s->call_rowptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)M + 1));
  int rc = 0;
  if (!s->class_size || !mstart || !astart || !acnt || !with_attrs || !s->method_class ||
      !s->attr_class || !s->acc_rowptr || !s->call_rowptr) { rc = 2; goto fail; }
  if ((rc = synth_class_sizes(p, s->class_size)) != 0) goto fail;

  mstart[0] = 0;
  for (int32_t C = 0; C < c; ++C) mstart[C + 1] = mstart[C] + s->class_size[C];
  for (int32_t C = 0; C < c; ++C)
    for (int32_t x = mstart[C]; x < mstart[C + 1]; ++x) s->method_class[x] = C;

  /* largest-remainder apportionment of A attributes proportional to sizes */
  {
    int64_t given = 0;
    for (int32_t C = 0; C < c; ++C) {
      acnt[C] = (int32_t)(((int64_t)A * s->class_size[C]) / M);
      given += acnt[C];
    }
    int64_t left = A - given;
    if (left > 0) {
      /* order classes by remainder (descending), ties to the lower id */
      int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
      if (!ord) { rc = 2; goto fail; }
      for (int32_t C = 0; C < c; ++C) ord[C] = C;
      g_rem_A = A; g_rem_M = M; g_rem_size = s->class_size;
      qsort(ord, (size_t)c, sizeof(int32_t), cmp_rem);
      for (int64_t i = 0; i < left; ++i) acnt[ord[i]]++;
      free(ord);
    }
  }
  astart[0] = 0;
  int32_t n_with = 0;
  for (int32_t C = 0; C < c; ++C) {
    astart[C + 1] = astart[C] + acnt[C];
    if (acnt[C] > 0) with_attrs[n_with++] = C;
  }
  for (int32_t C = 0; C < c; ++C)
    for (int32_t a = astart[C]; a < astart[C + 1]; ++a) s->attr_class[a] = C;

  /* accesses */
  {
    int64_t cap = 0;
    int *kk = (int *)malloc(sizeof(int) * (size_t)M);
    if (!kk) { rc = 2; goto fail; }
    for (int32_t x = 0; x < M; ++x) { kk[x] = poisson(p->seed, ST_POIS_ACC, x, p->lambda_acc); cap += kk[x]; }
    s->acc_idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cap + 1));
    if (!s->acc_idx) { free(kk); rc = 2; goto fail; }
    int64_t w = 0;
    s->acc_rowptr[0] = 0;
    for (int32_t x = 0; x < M; ++x) {
      int32_t C = s->method_class[x];
      int32_t aC = acnt[C];
      int32_t others = n_with - (aC > 0 ? 1 : 0);
      int64_t row0 = w;
      for (int j = 0; j < kk[x]; ++j) {
        double u = uni_real(p->seed, ST_ACC_LOC, didx(x, j));
        int32_t E;
        if (u < p->p_loc && aC > 0) {
          E = C;
        } else if (others > 0) {
          int32_t k = (int32_t)uni_int(p->seed, ST_ACC_CLS, didx(x, j), (uint32_t)others);
          /* k-th class with attributes, skipping the own class */
          E = with_attrs[k];
          if (aC > 0) {
            /* with_attrs is sorted; the own class sits at some position pos */
            int32_t lo2 = 0, hi2 = n_with;
            while (lo2 < hi2) { int32_t mid = (lo2 + hi2) / 2; if (with_attrs[mid] < C) lo2 = mid + 1; else hi2 = mid; }
            if (k >= lo2) E = with_attrs[k + 1];
          }
        } else if (aC > 0) {
          E = C;
        } else {
          continue;
        }
        s->acc_idx[w++] = astart[E] + (int32_t)uni_int(p->seed, ST_ACC_ITEM, didx(x, j), (uint32_t)acnt[E]);
      }
      w = row0 + sort_unique(s->acc_idx + row0, w - row0);
      s->acc_rowptr[x + 1] = w;
    }
    s->n_acc = w;
    free(kk);
  }

  /* calls */
  {
    int64_t cap = 0;
    int *kk = (int *)malloc(sizeof(int) * (size_t)M);
    if (!kk) { rc = 2; goto fail; }
    for (int32_t x = 0; x < M; ++x) { kk[x] = poisson(p->seed, ST_POIS_CALL, x, p->lambda_call); cap += kk[x]; }
    s->call_idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cap + 1));
    if (!s->call_idx) { free(kk); rc = 2; goto fail; }
    int64_t w = 0;
    s->call_rowptr[0] = 0;
    for (int32_t x = 0; x < M; ++x) {
      int32_t C = s->method_class[x];
      int32_t nC = s->class_size[C];
      int64_t row0 = w;
      for (int j = 0; j < kk[x]; ++j) {
        double u = uni_real(p->seed, ST_CALL_LOC, didx(x, j));
        int32_t t;
        if (u < p->p_loc && nC >= 2) {
          int32_t k = (int32_t)uni_int(p->seed, ST_CALL_ITEM, didx(x, j), (uint32_t)(nC - 1));
          t = mstart[C] + k;
          if (t >= x) ++t; /* skip self */
        } else if (c >= 2) {
          int32_t k = (int32_t)uni_int(p->seed, ST_CALL_CLS, didx(x, j), (uint32_t)(c - 1));
          int32_t E = k >= C ? k + 1 : k;
          t = mstart[E] + (int32_t)uni_int(p->seed, ST_CALL_ITEM, didx(x, j), (uint32_t)s->class_size[E]);
        } else {
          continue;
        }
        s->call_idx[w++] = t;
      }
      w = row0 + sort_unique(s->call_idx + row0, w - row0);
      s->call_rowptr[x + 1] = w;
    }
    s->n_call = w;
    free(kk);
  }
  free(mstart); free(astart); free(acnt); free(with_attrs);
  *out = s;
  return 0;
fail:
  free(mstart); free(astart); free(acnt); free(with_attrs);
  synth_free(s);
  return rc ? rc : 1;
}

/*
 * Restricted candidate destinations (the R2/R3 destination rule: classes of the
 * methods m calls and of the attributes m accesses) plus n_extra distinct
 * classes drawn uniformly from the remaining classes (never cls(m)).  Output is
 * a CSR over methods with each row sorted; rowptr has n_methods+1 entries.
 * Call with dst == NULL to get the row lengths only (rowptr filled).
 */
int synth_candidates(const synth_system *s, int32_t n_extra, uint64_t seed,
                     int64_t *rowptr, int32_t *dst) {
  int32_t c = s->n_classes;
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)c);
  int32_t *row = (int32_t *)malloc(sizeof(int32_t) * ((size_t)c + 1));
  if (!mark || !row) { free(mark); free(row); return 2; }
  for (int32_t E = 0; E < c; ++E) mark[E] = -1;
  int64_t w = 0;
  rowptr[0] = 0;
  for (int32_t x = 0; x < s->n_methods; ++x) {
    int32_t C = s->method_class[x];
    int32_t k = 0;
    mark[C] = x;
    for (int64_t e = s->acc_rowptr[x]; e < s->acc_rowptr[x + 1]; ++e) {
      int32_t E = s->attr_class[s->acc_idx[e]];
      if (mark[E] != x) { mark[E] = x; row[k++] = E; }
    }
    for (int64_t e = s->call_rowptr[x]; e < s->call_rowptr[x + 1]; ++e) {
      int32_t E = s->method_class[s->call_idx[e]];
      if (mark[E] != x) { mark[E] = x; row[k++] = E; }
    }
    int32_t avail = c - 1 - k;
    int32_t want = n_extra < avail ? n_extra : avail;
    for (int32_t j = 0, att = 0; j < want; ++att) {
      int32_t E = (int32_t)uni_int(seed, ST_CAND, didx(x, att), (uint32_t)c);
      if (mark[E] != x) { mark[E] = x; row[k++] = E; ++j; }
    }
    qsort(row, (size_t)k, sizeof(int32_t), cmp_i32);
    if (dst) memcpy(dst + w, row, sizeof(int32_t) * (size_t)k);
    w += k;
    rowptr[x + 1] = w;
  }
  free(mark); free(row);
  return 0;
}

/* Class count of batched system i: round(exp(ln lo + u ln(hi/lo))). */
int32_t synth_logu_classes(uint64_t seed, int32_t lo, int32_t hi) {
  double u = uni_real(seed, ST_SYS, 0);
  return (int32_t)llround(exp(log((double)lo) + u * log((double)hi / (double)lo)));
}
