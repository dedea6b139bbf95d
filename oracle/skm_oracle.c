/*
 * Spherical k-means ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded FP64 implementation of what the GPU path
 * computes, written from the paper (Schubert, Lang, Feher: "Accelerating
 * Spherical k-Means", arXiv 2107.04074).  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code with the
 * CUDA library: no headers, no helpers, no tables.
 *
 * What it computes, and where the paper defines it:
 *   - cosine similarity of unit vectors = dot product (Section 2);
 *     rows are normalised once at the start (Section 5, first paragraph);
 *   - the standard Lloyd iteration: a(i) = argmax_j <x(i), c(j)>, then
 *     c(j) = sum of members / its norm (Section 5, the two update rules);
 *   - the center drift p(j) = <c(j), c'(j)> and the bound updates
 *     Eq. (eqn:l-bound) and Eq. (eqn:u-elkan) (Section 4), built on the
 *     cosine triangle inequalities Eq. (eq:tri-cosine), (eq:tri-cosine2);
 *   - center-center bounds cc(i,j) = sqrt((<c(i),c(j)>+1)/2) and
 *     s(i) = max_{j!=i} cc(i,j) (Section 5.2);
 *   - Simplified Elkan (5.1), Elkan (5.2), Hamerly with Eq. (eqn:u-hamerly-2)
 *     (5.3), Hamerly's center test and Simplified Hamerly (5.4), each walked
 *     point by point in the paper's order;
 *   - spherical k-means++ seeding (Section 5.6): the first center uniform,
 *     the others drawn proportional to 1 - max_c <x(i), c>; and the bound
 *     pre-initialisation from the seeding's similarities (Section 5.6 and
 *     the outlook of Section 7);
 *   - Yin-Yang group bounds (Section 5.5 names them without a cosine form;
 *     reading YY below).
 *
 * Readings where the paper is silent (stated once here):
 *   T  ties: the current label wins; among other centers the lowest index
 *      wins, i.e. a point only moves on a strict improvement.  Before the
 *      first assignment there is no current label.
 *   E  a cluster whose member sum has norm 0 keeps its previous center.
 *   CL the bound updates are clamped to what the triangle inequality on
 *      angles allows: if arccos u < arccos p the upper bound is 1; if
 *      arccos l + arccos p > pi the lower bound is -1.
 *   HG Eq. (eqn:u-hamerly-2) is used when u >= 0 and p' >= 0; otherwise (or
 *      with the "tight" option) the clamped single-center update with p'.
 *   V  one iteration = assignment + center update; the run stops after an
 *      assignment that changes no label (its update would be a no-op).
 *   D  1 - p^2 is evaluated as q(2 - q), q = |c/|c| - c'/|c'||^2 / 2, which
 *      avoids the cancellation the paper warns about (Section 2).
 *   YY Yin-Yang on cosines: the centers are split into groups of YY_GROUP
 *      consecutive indices; l(i) bounds <x_i, c_a(i)> from below and u(i,G)
 *      bounds max_{j in G, j != a(i)} <x_i, c_j> from above.  After the
 *      centers move, l follows Eq. (eqn:l-bound) with p(a) and u(i,G) the
 *      clamped Eq. (eqn:u-elkan) with the group's smallest p (valid for every
 *      center of the group: that update grows as p shrinks).  A point is
 *      skipped if l >= max_G u(i,G); otherwise l is made tight and every group
 *      with l < u(i,G) is recomputed exactly; the best of a(i) and those
 *      centers is the new label (rule T); recomputed groups get their exact
 *      bound, and the old label's group takes its similarity if it left it.
 *   M  pruning keeps the exact labels of the standard variant: a bound test
 *      is passed with a margin of 2*delta_i, delta_i covering the FP64
 *      rounding of a similarity of row i, and every bound update carries a
 *      slack of 4e-15 for its own rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SKO_STANDARD 0
#define SKO_HAMERLY 1
#define SKO_ELKAN 2
#define SKO_SIMP_HAMERLY 3
#define SKO_SIMP_ELKAN 4
#define SKO_YINYANG 5
#define YY_GROUP 8 /* centers per Yin-Yang group: j / YY_GROUP */

#define UPD_SLACK 4e-15

typedef struct {
  int64_t n, d;
  int dense;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val; /* CSR values or dense n*d values, promoted to double */
} sko_data;

static int64_t row_len(const sko_data* X, int64_t i) {
  return X->dense ? X->d : X->row_ptr[i + 1] - X->row_ptr[i];
}

/* 1/|x_i| of the stored row (Section 5: rows normalised at initialisation). */
void sko_rinv(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
              const double* val, double* rinv) {
  (void)col;
  for (int64_t i = 0; i < n; ++i) {
    double ss = 0.0;
    if (dense) {
      for (int64_t t = 0; t < d; ++t) ss += val[i * d + t] * val[i * d + t];
    } else {
      for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) ss += val[p] * val[p];
    }
    rinv[i] = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
  }
}

/* sim(x_i, c) = <x_i, c> with x_i = stored_i * rinv_i (Section 2: on unit
 * vectors the cosine is the dot product; the sparse form only visits the
 * non-zeros of x_i). */
static double sim(const sko_data* X, const double* rinv, int64_t i, const double* c) {
  double s = 0.0, r = rinv[i];
  if (X->dense) {
    const double* x = X->val + i * X->d;
    for (int64_t t = 0; t < X->d; ++t) s += (x[t] * r) * c[t];
  } else {
    for (int64_t p = X->row_ptr[i]; p < X->row_ptr[i + 1]; ++p) s += (X->val[p] * r) * c[X->col[p]];
  }
  return s;
}

double sko_sim(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
               const double* val, const double* rinv, int64_t i, const double* c) {
  sko_data X = {n, d, dense, row_ptr, col, val};
  return sim(&X, rinv, i, c);
}

/* The margin of reading M for row i. */
static double delta_row(const sko_data* X, int64_t i) {
  return (double)(row_len(X, i) + 16) * 0x1.0p-52;
}

/* ---------------------------------------------------------------- bounds */

/* Eq. (eqn:l-bound) with reading CL: the new lower bound of the similarity to
 * a center that moved by an angle with cosine p (sine sp >= 0). */
double sko_l_update(double l, double p, double sp) {
  if (l + p < 0.0) return -1.0; /* arccos l + arccos p > pi */
  double v = l * p - sqrt((1.0 - l) * (1.0 + l)) * sp - UPD_SLACK;
  return v < -1.0 ? -1.0 : v;
}

/* Eq. (eqn:u-elkan) with reading CL. */
double sko_u_update(double u, double p, double sp) {
  if (u > p) return 1.0; /* arccos u < arccos p: the angle may close to 0 */
  double v = u * p + sqrt((1.0 - u) * (1.0 + u)) * sp + UPD_SLACK;
  return v > 1.0 ? 1.0 : v;
}

/* Hamerly's single upper bound (Section 5.3): Eq. (eqn:u-hamerly-2) with
 * p' = min_{j != a} p(j), under reading HG. */
double sko_u_hamerly(double u, double pp, double spp, int tight) {
  if (!tight && u >= 0.0 && pp >= 0.0) {
    double v = u + sqrt((1.0 - u) * (1.0 + u)) * spp + UPD_SLACK;
    return v > 1.0 ? 1.0 : v;
  }
  return sko_u_update(u, pp, spp);
}

/* ------------------------------------------------------- assignment (T) */

static int32_t pick_rule_t(const double* s, int64_t k, int32_t cur) {
  int32_t best = cur;
  double bs = cur >= 0 ? s[cur] : -INFINITY;
  for (int64_t j = 0; j < k; ++j) {
    if (j == cur) continue;
    if (s[j] > bs) { bs = s[j]; best = (int32_t)j; }
  }
  return best;
}

/* Standard assignment of all rows (Section 5).  a: in = current labels (-1 =
 * none), out = new labels.  s_best[i] = sim to the new label, s_second[i] =
 * max over the other centers (-inf if k = 1), top_gap[i] = largest minus
 * second-largest similarity regardless of labels.  Any output may be NULL.
 * Returns the number of changed labels. */
int64_t sko_assign(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
                   const double* val, const double* rinv, int64_t k, const double* C, int32_t* a,
                   double* s_best, double* s_second, double* top_gap) {
  sko_data X = {n, d, dense, row_ptr, col, val};
  double* s = (double*)malloc(sizeof(double) * (size_t)k);
  int64_t changed = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < k; ++j) s[j] = sim(&X, rinv, i, C + j * d);
    int32_t cur = a[i];
    int32_t nb = pick_rule_t(s, k, cur);
    if (nb != cur) changed++;
    a[i] = nb;
    double m1 = -INFINITY, m2 = -INFINITY, other = -INFINITY;
    for (int64_t j = 0; j < k; ++j) {
      if (s[j] > m1) { m2 = m1; m1 = s[j]; }
      else if (s[j] > m2) m2 = s[j];
      if (j != nb && s[j] > other) other = s[j];
    }
    if (s_best) s_best[i] = s[nb];
    if (s_second) s_second[i] = other;
    if (top_gap) top_gap[i] = m1 - m2;
  }
  free(s);
  return changed;
}

/* -------------------------------------------------------- center update */

/* c(j) = sum_{a(i)=j} x(i) / |sum| (Section 5), reading E for empty sums.
 * norms[j] = |S_j|; returns J = sum_j |S_j| (= sum_i <x_i, c_a(i)>). */
double sko_update(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
                  const double* val, const double* rinv, int64_t k, const int32_t* a,
                  const double* C_old, double* C_new, double* norms) {
  memset(C_new, 0, sizeof(double) * (size_t)(k * d));
  for (int64_t i = 0; i < n; ++i) {
    if (a[i] < 0 || a[i] >= k) continue;
    double* S = C_new + (int64_t)a[i] * d;
    if (dense) {
      for (int64_t t = 0; t < d; ++t) S[t] += val[i * d + t] * rinv[i];
    } else {
      for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) S[col[p]] += val[p] * rinv[i];
    }
  }
  double J = 0.0;
  for (int64_t j = 0; j < k; ++j) {
    double* S = C_new + j * d;
    double ss = 0.0;
    for (int64_t t = 0; t < d; ++t) ss += S[t] * S[t];
    double nr = sqrt(ss);
    if (norms) norms[j] = nr;
    J += nr;
    if (nr > 0.0) {
      for (int64_t t = 0; t < d; ++t) S[t] /= nr;
    } else {
      memcpy(S, C_old + j * d, sizeof(double) * (size_t)d);
    }
  }
  return J;
}

/* p(j) = <c(j), c'(j)> (Section 4) with its sine, under reading D. */
void sko_drift(int64_t k, int64_t d, const double* C_old, const double* C_new, double* p, double* sp) {
  for (int64_t j = 0; j < k; ++j) {
    const double* a = C_old + j * d;
    const double* b = C_new + j * d;
    double na = 0.0, nb = 0.0;
    for (int64_t t = 0; t < d; ++t) { na += a[t] * a[t]; nb += b[t] * b[t]; }
    na = sqrt(na); nb = sqrt(nb);
    double q = 0.0;
    for (int64_t t = 0; t < d; ++t) {
      double df = b[t] / nb - a[t] / na;
      q += df * df;
    }
    q *= 0.5;
    if (q > 2.0) q = 2.0;
    p[j] = 1.0 - q;
    sp[j] = sqrt(q * (2.0 - q));
  }
}

/* cc(i,j) = sqrt((<c(i),c(j)> + 1)/2) and s(i) = max_{j != i} cc(i,j)
 * (Section 5.2; cos of half the angle between two centers). */
void sko_center_bounds(int64_t k, int64_t d, const double* C, double* cc, double* s) {
  for (int64_t i = 0; i < k; ++i) {
    for (int64_t j = 0; j < k; ++j) {
      double g = 0.0;
      for (int64_t t = 0; t < d; ++t) g += C[i * d + t] * C[j * d + t];
      double h = 0.5 * (g + 1.0);
      if (h < 0.0) h = 0.0;
      if (h > 1.0) h = 1.0;
      cc[i * k + j] = sqrt(h) + 1e-15;
    }
  }
  for (int64_t i = 0; i < k; ++i) {
    double m = -INFINITY;
    for (int64_t j = 0; j < k; ++j)
      if (j != i && cc[i * k + j] > m) m = cc[i * k + j];
    s[i] = m;
  }
}

/* ------------------------------------------------------------ full runs */

/*
 * One spherical k-means run from the initial centers C (k x d, unit rows; on
 * return the final centers).  Records per iteration t < iters_done:
 *   labels_trace[t*n + i]  labels after the assignment of iteration t
 *   changed_trace[t]       labels changed by that assignment
 *   sims_trace[t]          exact similarities computed by that assignment
 *   J_trace[t]             objective after that iteration's center update
 *                          (after the last, converged one: unchanged)
 * check_bounds != 0 verifies, each iteration, every maintained bound against
 * the exact similarities (not counted in sims_trace) and returns the number of
 * violations in *violations.
 */
int sko_run(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
            const double* val, const double* rinv, int64_t k, int variant, double* C,
            int32_t max_iters, int hamerly_tight, int check_bounds, int32_t* labels_trace,
            int64_t* changed_trace, int64_t* sims_trace, double* J_trace, int32_t* iters_done,
            int64_t* violations) {
  sko_data X = {n, d, dense, row_ptr, col, val};
  int elkan = (variant == SKO_ELKAN || variant == SKO_SIMP_ELKAN);
  int hamerly = (variant == SKO_HAMERLY || variant == SKO_SIMP_HAMERLY);
  int full = (variant == SKO_ELKAN || variant == SKO_HAMERLY);
  int yy = (variant == SKO_YINYANG);
  int64_t ng = (k + YY_GROUP - 1) / YY_GROUP;
  double* ug = yy ? (double*)malloc(sizeof(double) * (size_t)(n * ng)) : NULL;
  double* pg = yy ? (double*)malloc(sizeof(double) * (size_t)ng) : NULL;
  double* spg = yy ? (double*)malloc(sizeof(double) * (size_t)ng) : NULL;
  char* live = yy ? (char*)malloc((size_t)ng) : NULL;
  int32_t* a = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  double* l = (double*)malloc(sizeof(double) * (size_t)n);
  double* uh = (double*)malloc(sizeof(double) * (size_t)n);
  double* ue = elkan ? (double*)malloc(sizeof(double) * (size_t)(n * k)) : NULL;
  double* s = (double*)malloc(sizeof(double) * (size_t)k);
  double* Cn = (double*)malloc(sizeof(double) * (size_t)(k * d));
  double* p = (double*)malloc(sizeof(double) * (size_t)k);
  double* sp = (double*)malloc(sizeof(double) * (size_t)k);
  double* cc = full ? (double*)malloc(sizeof(double) * (size_t)(k * k)) : NULL;
  double* sc = (double*)malloc(sizeof(double) * (size_t)k);
  if (!a || !l || !uh || (elkan && !ue) || !s || !Cn || !p || !sp || (full && !cc) || !sc) return -1;
  for (int64_t i = 0; i < n; ++i) a[i] = -1;
  int64_t viol = 0;
  double Jlast = 0.0;
  int32_t it;
  for (it = 0; it < max_iters; ++it) {
    int64_t changed = 0, sims = 0;
    if (it == 0 || variant == SKO_STANDARD) {
      /* full assignment; the first one also initialises the bounds */
      for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < k; ++j) s[j] = sim(&X, rinv, i, C + j * d);
        sims += k;
        int32_t nb = pick_rule_t(s, k, a[i]);
        if (nb != a[i]) changed++;
        a[i] = nb;
        double dl = delta_row(&X, i);
        l[i] = s[nb] - dl;
        double o = -INFINITY;
        for (int64_t j = 0; j < k; ++j)
          if (j != nb && s[j] > o) o = s[j];
        uh[i] = (k > 1) ? o + dl : -1.0;
        if (elkan)
          for (int64_t j = 0; j < k; ++j) ue[i * k + j] = s[j] + dl;
        if (yy)
          for (int64_t g = 0; g < ng; ++g) {
            double o2 = -INFINITY;
            for (int64_t j = g * YY_GROUP; j < k && j < (g + 1) * YY_GROUP; ++j)
              if (j != nb && s[j] > o2) o2 = s[j];
            ug[i * ng + g] = (o2 == -INFINITY) ? -1.0 : o2 + dl;
          }
      }
    } else if (yy) {
      /* the worst drift of each group */
      for (int64_t g = 0; g < ng; ++g) {
        int64_t jm = g * YY_GROUP;
        for (int64_t j = jm; j < k && j < (g + 1) * YY_GROUP; ++j)
          if (p[j] < p[jm]) jm = j;
        pg[g] = p[jm];
        spg[g] = sp[jm];
      }
      for (int64_t i = 0; i < n; ++i) {
        int32_t ai = a[i];
        double dl = delta_row(&X, i);
        l[i] = sko_l_update(l[i], p[ai], sp[ai]);
        double umax = -INFINITY;
        for (int64_t g = 0; g < ng; ++g) {
          ug[i * ng + g] = sko_u_update(ug[i * ng + g], pg[g], spg[g]);
          if (ug[i * ng + g] > umax) umax = ug[i * ng + g];
        }
        if (check_bounds) {
          for (int64_t j = 0; j < k; ++j) s[j] = sim(&X, rinv, i, C + j * d);
          if (l[i] > s[ai] + dl) viol++;
          for (int64_t j = 0; j < k; ++j)
            if (j != ai && ug[i * ng + j / YY_GROUP] < s[j] - dl) viol++;
        }
        double L = l[i] - 2.0 * dl;
        if (L >= umax) continue; /* global test */
        double sa = sim(&X, rinv, i, C + ai * d);
        sims++;
        l[i] = sa - dl;
        L = l[i] - 2.0 * dl;
        if (L >= umax) continue;
        /* group test; the recomputed groups' similarities (a(i) known) */
        for (int64_t j = 0; j < k; ++j) s[j] = -INFINITY;
        s[ai] = sa;
        for (int64_t g = 0; g < ng; ++g) {
          live[g] = L < ug[i * ng + g];
          if (!live[g]) continue;
          for (int64_t j = g * YY_GROUP; j < k && j < (g + 1) * YY_GROUP; ++j) {
            if (j == ai) continue;
            s[j] = sim(&X, rinv, i, C + j * d);
            sims++;
          }
        }
        int32_t nb = pick_rule_t(s, k, ai);
        if (nb != ai) changed++;
        a[i] = nb;
        l[i] = s[nb] - dl;
        for (int64_t g = 0; g < ng; ++g) {
          if (!live[g]) continue;
          double o2 = -INFINITY;
          for (int64_t j = g * YY_GROUP; j < k && j < (g + 1) * YY_GROUP; ++j)
            if (j != nb && s[j] > o2) o2 = s[j];
          ug[i * ng + g] = (o2 == -INFINITY) ? -1.0 : o2 + dl;
        }
        /* the old label left a group that was not recomputed */
        int64_t go = ai / YY_GROUP;
        if (nb != ai && !live[go] && sa + dl > ug[i * ng + go]) ug[i * ng + go] = sa + dl;
      }
    } else {
      /* p'(j) = min_{j' != j} p(j') for Hamerly (Section 5.3) */
      int64_t jmin = 0;
      for (int64_t j = 1; j < k; ++j)
        if (p[j] < p[jmin]) jmin = j;
      int64_t jmin2 = -1;
      for (int64_t j = 0; j < k; ++j)
        if (j != jmin && (jmin2 < 0 || p[j] < p[jmin2])) jmin2 = j;
      for (int64_t i = 0; i < n; ++i) {
        int32_t ai = a[i];
        double dl = delta_row(&X, i);
        /* bound updates (Section 4) */
        l[i] = sko_l_update(l[i], p[ai], sp[ai]);
        if (hamerly) {
          int64_t jp = (ai == jmin) ? jmin2 : jmin;
          if (jp >= 0) uh[i] = sko_u_hamerly(uh[i], p[jp], sp[jp], hamerly_tight);
        } else {
          for (int64_t j = 0; j < k; ++j) ue[i * k + j] = sko_u_update(ue[i * k + j], p[j], sp[j]);
        }
        if (check_bounds) {
          for (int64_t j = 0; j < k; ++j) s[j] = sim(&X, rinv, i, C + j * d);
          if (l[i] > s[ai] + dl) viol++;
          for (int64_t j = 0; j < k; ++j) {
            if (j == ai) continue;
            if (hamerly && uh[i] < s[j] - dl) viol++;
            if (elkan && ue[i * k + j] < s[j] - dl) viol++;
          }
        }
        double L = l[i] - 2.0 * dl;
        if (hamerly) {
          /* Section 5.3 / 5.4: prune if l >= u, or (full) l >= s(a) */
          if (L >= uh[i]) continue;
          if (full && L >= 0.0 && L >= sc[ai]) continue;
          double sa = sim(&X, rinv, i, C + ai * d);
          sims++;
          l[i] = sa - dl;
          L = l[i] - 2.0 * dl;
          if (L >= uh[i]) continue;
          if (full && L >= 0.0 && L >= sc[ai]) continue;
          for (int64_t j = 0; j < k; ++j) {
            if (j == ai) { s[j] = sa; continue; }
            s[j] = sim(&X, rinv, i, C + j * d);
            sims++;
          }
          int32_t nb = pick_rule_t(s, k, ai);
          if (nb != ai) changed++;
          a[i] = nb;
          l[i] = s[nb] - dl;
          double o = -INFINITY;
          for (int64_t j = 0; j < k; ++j)
            if (j != nb && s[j] > o) o = s[j];
          uh[i] = o + dl;
        } else {
          /* Section 5.2: skip the point if s(a) <= l; Section 5.1 / 5.2 per center */
          if (full && L >= 0.0 && sc[ai] <= L) continue;
          int tight = 0;
          double sa = 0.0;
          int32_t cur = ai;
          for (int64_t j = 0; j < k; ++j) {
            if (j == cur) continue;
            if (ue[i * k + j] <= L) continue;
            if (full && L >= 0.0 && cc[cur * k + j] <= L) continue;
            if (!tight) {
              sa = sim(&X, rinv, i, C + cur * d);
              sims++;
              l[i] = sa - dl;
              L = l[i] - 2.0 * dl;
              tight = 1;
              if (ue[i * k + j] <= L) continue;
              if (full && L >= 0.0 && cc[cur * k + j] <= L) continue;
            }
            double sj = sim(&X, rinv, i, C + j * d);
            sims++;
            ue[i * k + j] = sj + dl;
            if (sj > sa) {
              ue[i * k + cur] = sa + dl;
              cur = (int32_t)j;
              sa = sj;
              l[i] = sj - dl;
              L = l[i] - 2.0 * dl;
            }
          }
          if (cur != ai) changed++;
          a[i] = cur;
        }
      }
    }
    if (labels_trace) memcpy(labels_trace + (int64_t)it * n, a, sizeof(int32_t) * (size_t)n);
    if (changed_trace) changed_trace[it] = changed;
    if (sims_trace) sims_trace[it] = sims;
    if (changed == 0) {
      if (J_trace) J_trace[it] = Jlast;
      it++;
      break;
    }
    Jlast = sko_update(n, d, dense, row_ptr, col, val, rinv, k, a, C, Cn, NULL);
    if (J_trace) J_trace[it] = Jlast;
    sko_drift(k, d, C, Cn, p, sp);
    memcpy(C, Cn, sizeof(double) * (size_t)(k * d));
    if (full) {
      if (elkan) {
        sko_center_bounds(k, d, C, cc, sc);
      } else {
        double* tmp = (double*)malloc(sizeof(double) * (size_t)(k * k));
        sko_center_bounds(k, d, C, tmp, sc);
        free(tmp);
      }
    }
  }
  if (iters_done) *iters_done = it;
  if (violations) *violations = viol;
  free(a); free(l); free(uh); free(ue); free(s); free(Cn); free(p); free(sp); free(cc); free(sc);
  free(ug); free(pg); free(spg); free(live);
  return 0;
}

/* Spherical k-means++ (Section 5.6).  The caller supplies the uniform draws
 * u[0..k-1] in [0, 1).  Row floor(u[0] n) is the first center.  Then, with
 * m_i = max over the chosen centers of <x_i, c> (kept up to date as centers
 * are added), each row weighs 1 - m_i, quantised to q_i = round((1 - m_i) 2^40)
 * (0 if negative); with W = sum q_i and T = floor(u[j] W) the next center is
 * the first row whose running sum of q exceeds T, or, if W = 0, the first row
 * not chosen yet.  Writes the k chosen rows; returns 0.
 *
 * Bound pre-initialisation (the remark of Section 5.6 and the outlook of
 * Section 7: the similarities the seeding computes can initialise the
 * bounds): when a is not NULL the similarities to the last center are
 * computed as well, and each row keeps, over the centers in the order they
 * were chosen, its best similarity s1 (at the lowest index among equal
 * values, rule T with no current label), that index a(i), and its second
 * best s2 (the largest of the others; -inf with k = 1); S (n x k, may be
 * NULL) receives every similarity.  That is the first assignment from the
 * seeded centers, with Hamerly's bounds l = s1, u = s2 and Elkan's
 * u(i,j) = S[i][j], without a separate pass over the data. */
static int kmeanspp_impl(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
                         const double* val, const double* rinv, int64_t k, const double* u, int64_t* rows,
                         int32_t* a, double* s1, double* s2, double* S) {
  sko_data X = {n, d, dense, row_ptr, col, val};
  double* c = (double*)malloc(sizeof(double) * (size_t)d);
  double* m = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t r = (int64_t)(u[0] * (double)n);
  if (r >= n) r = n - 1;
  for (int64_t j = 0; j < k; ++j) {
    rows[j] = r;
    /* the new center: the chosen row, normalised */
    memset(c, 0, sizeof(double) * (size_t)d);
    if (dense) {
      for (int64_t t = 0; t < d; ++t) c[t] = val[r * d + t] * rinv[r];
    } else {
      for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) c[col[p]] = val[p] * rinv[r];
    }
    if (j + 1 == k && !a) break;
    long long W = 0;
    for (int64_t i = 0; i < n; ++i) {
      const double s = sim(&X, rinv, i, c);
      m[i] = (j == 0 || s > m[i]) ? s : m[i];
      long long q = llround((1.0 - m[i]) * 0x1.0p40);
      W += q > 0 ? q : 0;
      if (a) {
        if (S) S[i * k + j] = s;
        if (j == 0) {
          a[i] = 0;
          s1[i] = s;
          s2[i] = -INFINITY;
        } else if (s > s1[i]) {
          s2[i] = s1[i];
          s1[i] = s;
          a[i] = (int32_t)j;
        } else if (s > s2[i]) {
          s2[i] = s;
        }
      }
    }
    if (j + 1 == k) break;
    int64_t next = -1;
    if (W > 0) {
      long long T = (long long)(u[j + 1] * (double)W);
      if (T >= W) T = W - 1;
      long long acc = 0;
      for (int64_t i = 0; i < n && next < 0; ++i) {
        long long q = llround((1.0 - m[i]) * 0x1.0p40);
        acc += q > 0 ? q : 0;
        if (acc > T) next = i;
      }
    } else {
      for (int64_t i = 0; i < n && next < 0; ++i) {
        int taken = 0;
        for (int64_t cc = 0; cc <= j && !taken; ++cc) taken = rows[cc] == i;
        if (!taken) next = i;
      }
    }
    r = next;
  }
  free(c);
  free(m);
  return 0;
}

int sko_kmeanspp(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
                 const double* val, const double* rinv, int64_t k, const double* u, int64_t* rows) {
  return kmeanspp_impl(n, d, dense, row_ptr, col, val, rinv, k, u, rows, NULL, NULL, NULL, NULL);
}

int sko_kmeanspp_bounds(int64_t n, int64_t d, int dense, const int64_t* row_ptr, const int32_t* col,
                        const double* val, const double* rinv, int64_t k, const double* u, int64_t* rows,
                        int32_t* a, double* s1, double* s2, double* S) {
  return kmeanspp_impl(n, d, dense, row_ptr, col, val, rinv, k, u, rows, a, s1, s2, S);
}
