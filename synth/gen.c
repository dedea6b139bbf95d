/*
 * Seeded synthetic inputs for spherical k-means (shared by the oracle side
 * and the CUDA side of the tests and the benchmark).
 *
 * This file holds NO arithmetic of the clustering method: it only draws
 * data with the shapes of the paper's workloads (Section 6, Table 1:
 * sparse TF-IDF document vectors; plus dense embedding-like vectors drawn
 * from a von Mises-Fisher mixture).  Every random number comes from a
 * counter-based splitmix64 stream keyed by (seed, purpose, index), so the
 * output does not depend on the number of threads used.
 *
 * Recipes (the paper gives no generator; these are the stated synthetic
 * stand-ins):
 *  - nnz per row: Poisson(lambda) redrawn while 0, or lognormal with a given
 *    arithmetic mean m and log-sigma s (mu = ln m - s^2/2), rounded to the
 *    nearest integer and clipped to [lo, hi] (hi is also capped at d/2).
 *  - term ids: finite Zipf over ranks 1..d, P(r) ~ r^-z, drawn with
 *    replacement and duplicates rejected until the row holds its nnz
 *    distinct terms; rank r maps to term perm[r-1] (seeded Fisher-Yates).
 *  - tf ~ Geometric(1/2) on {1,2,...}; value = log(1+tf) * idf(t),
 *    idf(t) = ln((1+n)/(1+df(t))) + 1; rows scaled to unit L2 norm in
 *    double and rounded to float.  Column indices sorted within each row.
 *  - dense: mixture of vMF(mu_c, kappa) with uniform weights and means
 *    uniform on the sphere; the cosine w to the mean is drawn with Wood's
 *    (1994) rejection sampler, the tangent direction uniformly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

typedef struct {
  uint64_t key;
  uint64_t ctr;
} stream_t;

static inline stream_t stream_make(uint64_t seed, uint64_t purpose, uint64_t index) {
  stream_t s;
  s.key = mix64(mix64(seed ^ 0x5EEDull) ^ mix64(purpose * 0x100000001B3ull + 0x9E37ull) ^ (index * 0xD1B54A32D192ED03ull));
  s.ctr = 0;
  return s;
}
static inline uint64_t next_u64(stream_t* s) { return mix64(s->key + (s->ctr++) * 0x9E3779B97F4A7C15ull); }
/* uniform in (0,1): 53 random bits, never exactly 0 */
static inline double next_unif(stream_t* s) { return ((double)(next_u64(s) >> 11) + 0.5) * 0x1.0p-53; }
static inline double next_normal(stream_t* s) {
  double u1 = next_unif(s), u2 = next_unif(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

enum { P_NNZ = 1, P_TERMS = 2, P_PERM = 3, P_MEANS = 4, P_POINTS = 5, P_INIT = 6 };

/* Poisson by inversion, summing pmf terms from 0 (fine for lambda <= ~500). */
static int64_t draw_poisson(stream_t* s, double lam) {
  double u = next_unif(s);
  double p = exp(-lam), c = p;
  int64_t x = 0;
  while (u > c && x < 100000) {
    x++;
    p *= lam / (double)x;
    c += p;
  }
  return x;
}

static int64_t draw_nnz(stream_t* s, int kind, double a, double b, int64_t lo, int64_t hi) {
  if (kind == 0) {
    int64_t x;
    do {
      x = draw_poisson(s, a);
    } while (x == 0);
    if (x > hi) x = hi;
    return x;
  }
  double mu = log(a) - 0.5 * b * b;
  double v = exp(mu + b * next_normal(s));
  int64_t x = (int64_t)llround(v);
  if (x < lo) x = lo;
  if (x > hi) x = hi;
  return x;
}

/* ---------------------------------------------------------------- sparse */

typedef struct {
  int64_t n, d;
  uint64_t seed;
  double zipf_s;
  const double* cdf; /* cumulative Zipf weights over ranks, cdf[d-1] = 1 */
  const int32_t* perm;
  const int64_t* row_ptr;
  int32_t* col;
  uint8_t* tf;
  int64_t r0, r1;
  int32_t* df; /* per-thread document-frequency counts (d) */
} sp_job;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void* sp_rows(void* arg) {
  sp_job* j = (sp_job*)arg;
  int64_t d = j->d;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  for (int64_t t = 0; t < d; ++t) mark[t] = -1;
  for (int64_t i = j->r0; i < j->r1; ++i) {
    stream_t s = stream_make(j->seed, P_TERMS, (uint64_t)i);
    int64_t b = j->row_ptr[i], m = j->row_ptr[i + 1] - b;
    int32_t* out = j->col + b;
    int64_t got = 0;
    while (got < m) {
      double u = next_unif(&s);
      /* smallest rank index r with cdf[r] >= u */
      int64_t lo = 0, hi = d - 1;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (j->cdf[mid] >= u) hi = mid; else lo = mid + 1;
      }
      int32_t term = j->perm[lo];
      if (mark[term] == (int32_t)(i & 0x7fffffff) ) continue;
      mark[term] = (int32_t)(i & 0x7fffffff);
      out[got++] = term;
    }
    qsort(out, (size_t)m, sizeof(int32_t), cmp_i32);
    for (int64_t p = 0; p < m; ++p) {
      uint64_t r = next_u64(&s);
      int tfv = 1;
      while ((r & 1ull) == 0 && tfv < 64) { r >>= 1; tfv++; }
      j->tf[b + p] = (uint8_t)tfv;
      j->df[out[p]]++;
    }
  }
  free(mark);
  return NULL;
}

typedef struct {
  const int64_t* row_ptr;
  const int32_t* col;
  const uint8_t* tf;
  const double* idf;
  float* val;
  int64_t r0, r1;
} val_job;

static void* sp_vals(void* arg) {
  val_job* j = (val_job*)arg;
  for (int64_t i = j->r0; i < j->r1; ++i) {
    int64_t b = j->row_ptr[i], e = j->row_ptr[i + 1];
    double ss = 0.0;
    for (int64_t p = b; p < e; ++p) {
      double v = log(1.0 + (double)j->tf[p]) * j->idf[j->col[p]];
      ss += v * v;
    }
    double r = 1.0 / sqrt(ss);
    for (int64_t p = b; p < e; ++p) {
      double v = log(1.0 + (double)j->tf[p]) * j->idf[j->col[p]];
      j->val[p] = (float)(v * r);
    }
  }
  return NULL;
}

/* Step 1: nnz per row (row_nnz has n entries). */
void synth_row_nnz(int64_t n, int64_t d, uint64_t seed, int kind, double a, double b, int64_t lo,
                   int64_t hi, int64_t* row_nnz) {
  if (hi > d / 2) hi = d / 2;
  if (lo > hi) lo = hi;
  for (int64_t i = 0; i < n; ++i) {
    stream_t s = stream_make(seed, P_NNZ, (uint64_t)i);
    row_nnz[i] = draw_nnz(&s, kind, a, b, lo, hi);
  }
}

/* Step 2: terms, tf-idf values.  row_ptr has n+1 entries (prefix sums of the
 * nnz from step 1); col and val have row_ptr[n] entries. */
int synth_tfidf_fill(int64_t n, int64_t d, uint64_t seed, double zipf_s, const int64_t* row_ptr,
                     int32_t* col, float* val, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  int64_t nnz = row_ptr[n];
  double* cdf = (double*)malloc(sizeof(double) * (size_t)d);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)d);
  uint8_t* tf = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
  int32_t* df = (int32_t*)calloc((size_t)nthreads * (size_t)d, sizeof(int32_t));
  double* idf = (double*)malloc(sizeof(double) * (size_t)d);
  if (!cdf || !perm || !tf || !df || !idf) return -1;
  double acc = 0.0;
  for (int64_t r = 0; r < d; ++r) {
    acc += pow((double)(r + 1), -zipf_s);
    cdf[r] = acc;
  }
  for (int64_t r = 0; r < d; ++r) cdf[r] /= acc;
  cdf[d - 1] = 1.0;
  for (int64_t r = 0; r < d; ++r) perm[r] = (int32_t)r;
  stream_t ps = stream_make(seed, P_PERM, 0);
  for (int64_t r = d - 1; r > 0; --r) {
    int64_t q = (int64_t)(next_u64(&ps) % (uint64_t)(r + 1));
    int32_t tmp = perm[r]; perm[r] = perm[q]; perm[q] = tmp;
  }
  pthread_t th[256];
  sp_job jobs[256];
  for (int w = 0; w < nthreads; ++w) {
    sp_job* j = &jobs[w];
    j->n = n; j->d = d; j->seed = seed; j->zipf_s = zipf_s; j->cdf = cdf; j->perm = perm;
    j->row_ptr = row_ptr; j->col = col; j->tf = tf;
    j->r0 = n * w / nthreads; j->r1 = n * (w + 1) / nthreads;
    j->df = df + (size_t)w * (size_t)d;
    pthread_create(&th[w], NULL, sp_rows, j);
  }
  for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
  for (int64_t t = 0; t < d; ++t) {
    int64_t c = 0;
    for (int w = 0; w < nthreads; ++w) c += df[(size_t)w * (size_t)d + (size_t)t];
    idf[t] = log((1.0 + (double)n) / (1.0 + (double)c)) + 1.0;
  }
  val_job vj[256];
  for (int w = 0; w < nthreads; ++w) {
    val_job* j = &vj[w];
    j->row_ptr = row_ptr; j->col = col; j->tf = tf; j->idf = idf; j->val = val;
    j->r0 = n * w / nthreads; j->r1 = n * (w + 1) / nthreads;
    pthread_create(&th[w], NULL, sp_vals, j);
  }
  for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
  free(cdf); free(perm); free(tf); free(df); free(idf);
  return 0;
}

/* ----------------------------------------------------------------- dense */

/* Gamma(alpha, 1) for alpha >= 1 (Marsaglia & Tsang 2000). */
static double draw_gamma(stream_t* s, double alpha) {
  double dd = alpha - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * dd);
  for (;;) {
    double x, v;
    do {
      x = next_normal(s);
      v = 1.0 + c * x;
    } while (v <= 0.0);
    v = v * v * v;
    double u = next_unif(s);
    if (log(u) < 0.5 * x * x + dd - dd * v + dd * log(v)) return dd * v;
  }
}

typedef struct {
  int64_t n, d, ncomp;
  uint64_t seed;
  double kappa;
  const double* means;
  float* X;
  int32_t* comp;
  int64_t r0, r1;
} vmf_job;

static void* vmf_rows(void* arg) {
  vmf_job* j = (vmf_job*)arg;
  int64_t d = j->d;
  double dm1 = (double)(d - 1), kap = j->kappa;
  double b = (-2.0 * kap + sqrt(4.0 * kap * kap + dm1 * dm1)) / dm1;
  double x0 = (1.0 - b) / (1.0 + b);
  double cst = kap * x0 + dm1 * log(1.0 - x0 * x0);
  double* g = (double*)malloc(sizeof(double) * (size_t)d);
  for (int64_t i = j->r0; i < j->r1; ++i) {
    stream_t s = stream_make(j->seed, P_POINTS, (uint64_t)i);
    int64_t c = (int64_t)(next_u64(&s) % (uint64_t)j->ncomp);
    const double* mu = j->means + (size_t)c * (size_t)d;
    double w;
    for (;;) {
      double ga = draw_gamma(&s, 0.5 * dm1), gb = draw_gamma(&s, 0.5 * dm1);
      double z = ga / (ga + gb);
      w = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z);
      double u = next_unif(&s);
      if (kap * w + dm1 * log(1.0 - x0 * w) - cst >= log(u)) break;
    }
    double dot = 0.0;
    for (int64_t t = 0; t < d; ++t) {
      g[t] = next_normal(&s);
      dot += g[t] * mu[t];
    }
    double nn = 0.0;
    for (int64_t t = 0; t < d; ++t) {
      g[t] -= dot * mu[t];
      nn += g[t] * g[t];
    }
    double sc = sqrt(1.0 - w * w) / sqrt(nn);
    double ss = 0.0;
    for (int64_t t = 0; t < d; ++t) {
      g[t] = w * mu[t] + sc * g[t];
      ss += g[t] * g[t];
    }
    double r = 1.0 / sqrt(ss);
    float* out = j->X + (size_t)i * (size_t)d;
    for (int64_t t = 0; t < d; ++t) out[t] = (float)(g[t] * r);
    if (j->comp) j->comp[i] = (int32_t)c;
  }
  free(g);
  return NULL;
}

/* Dense n x d rows (row-major float) from a mixture of ncomp vMF(kappa)
 * components; comp (optional, n) receives each row's component. */
int synth_vmf(int64_t n, int64_t d, int64_t ncomp, double kappa, uint64_t seed, float* X,
              int32_t* comp, double* means_out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  double* means = (double*)malloc(sizeof(double) * (size_t)ncomp * (size_t)d);
  if (!means) return -1;
  for (int64_t c = 0; c < ncomp; ++c) {
    stream_t s = stream_make(seed, P_MEANS, (uint64_t)c);
    double ss = 0.0;
    double* m = means + (size_t)c * (size_t)d;
    for (int64_t t = 0; t < d; ++t) {
      m[t] = next_normal(&s);
      ss += m[t] * m[t];
    }
    double r = 1.0 / sqrt(ss);
    for (int64_t t = 0; t < d; ++t) m[t] *= r;
  }
  pthread_t th[256];
  vmf_job jobs[256];
  for (int w = 0; w < nthreads; ++w) {
    vmf_job* j = &jobs[w];
    j->n = n; j->d = d; j->ncomp = ncomp; j->seed = seed; j->kappa = kappa; j->means = means;
    j->X = X; j->comp = comp;
    j->r0 = n * w / nthreads; j->r1 = n * (w + 1) / nthreads;
    pthread_create(&th[w], NULL, vmf_rows, j);
  }
  for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
  if (means_out) memcpy(means_out, means, sizeof(double) * (size_t)ncomp * (size_t)d);
  free(means);
  return 0;
}

/* k distinct row ids in [0, n), drawn by a seeded partial Fisher-Yates over
 * a virtual identity array (hash map free: rejection against earlier picks). */
int synth_init_rows(int64_t n, int64_t k, uint64_t seed, int64_t* out) {
  if (k > n) return -1;
  stream_t s = stream_make(seed, P_INIT, 0);
  for (int64_t j = 0; j < k; ++j) {
    for (;;) {
      int64_t r = (int64_t)(next_u64(&s) % (uint64_t)n);
      int dup = 0;
      for (int64_t q = 0; q < j; ++q)
        if (out[q] == r) { dup = 1; break; }
      if (!dup) { out[j] = r; break; }
    }
  }
  return 0;
}
