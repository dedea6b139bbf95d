// The center update (Section 5): S_j = sum_{a(i)=j} x(i), c(j) = S_j/|S_j|;
// the drift p(j) = <c(j), c'(j)> that moves the bounds (Section 4); and the
// center-center bounds cc(i,j), s(i) of Section 5.2.
//
// The sums are kept between iterations as exact 64-bit fixed-point integers
// S64[t][j] (x scaled by 2^s and rounded).  Integer addition is exact and
// associative, so the sums do not depend on any order, and -- the paper's
// optimisation (iii), Section 5 -- a later iteration may add and subtract only
// the rows whose label changed and obtain bit for bit the sums a full
// recomputation would give.  Only clusters whose sum changed ("dirty") are
// renormalised, get a drift, and get their Gram row recomputed.
//
//   k_center_sum        full recompute: warp per chunk of a term's column,
//                       per-cluster bins in shared memory (native 32-bit
//                       atomics on two 20-bit halves, exact), no atomics in
//                       global memory.
//   k_center_sum_multi  terms with several chunks: exact sum of the partials.
//   k_center_delta      incremental: warp per changed row, +x to the new and
//                       -x to the old cluster (exact integer atomics).
//   k_dirty             the dirty cluster list (all clusters after a full sum).
//   k_colnorm_*         |S_j| for dirty clusters (compensated FP32 per thread,
//                       FP64 across threads and blocks, fixed order).
//   k_normalize_drift   c(j) = S_j/|S_j| in place for dirty clusters (an empty
//                       cluster keeps c'(j)), partial sums for the drift.
//   k_drift_final       per center an interval [pd, pu] for cos(angle(c, c'))
//                       and an upper bound q of its sine, rounded outward.
//   k_hsel_obj          J = sum_j |S_j| and Hamerly's worst-drift summary; zeroes
//                       the assignment counters for the next assignment.
//   k_gram_*            <c_i, c_j> (FP32 products, FP64 across 256-term
//                       chunks): all tiles when many clusters moved, else only
//                       the rows of the (at most 64) dirty clusters; then cc
//                       and s.
//   k_hsel_runs, k_gram_plan, k_gram_batch, k_gram_final_batch
//                       a batch of runs: Hamerly's worst-drift summary per run,
//                       and each run's own (block-diagonal) Gram entries of its
//                       dirty centers, then its cc rows and s.
#include <cfloat>
#include <climits>

#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kChunk = 1024;  // must match the chunking built in k_prep.cu
constexpr int kTB = 256;      // rows (terms) per reduction block

// Fixed-point value of x: |x| <= 1 maps below 2^40 (the 20 + 20 bit split).
__device__ __forceinline__ long long to_fixed(float x, float scale) { return __float2ll_rn(__fmul_rn(x, scale)); }

// The FP32 sum a fixed-point sum stands for (the value every kernel uses).
__device__ __forceinline__ float from_fixed(long long s, float inv) { return __fmul_rn(__ll2float_rn(s), inv); }

// Full recompute.  fx = round(x * 2^s) is split into hi = fx >> 20 and
// lo = fx & (2^20 - 1); a chunk holds at most 2^10 entries, so both halves sum
// exactly in 32-bit integers and the shared atomics are native 32-bit ones.
// A column of the term-major copy: a term, or for a batch a (run, term)
// pair whose sums fill the run's slice koff .. koff + kw of the term's row.
struct SumCol {
  int64_t t;
  int32_t koff, k, kw;
};
__device__ __forceinline__ SumCol sum_col(int64_t key, int32_t k, int64_t kst, const RunDesc* __restrict__ runs,
                                          int64_t dterm) {
  SumCol c;
  if (!runs) {
    c.t = key;
    c.koff = 0;
    c.k = k;
    c.kw = (int32_t)kst;
  } else {
    const int64_t r = key / dterm;
    c.t = key - r * dterm;
    c.koff = runs[r].koff;
    c.k = runs[r].k;
    c.kw = runs[r].kst;
  }
  return c;
}

__global__ void __launch_bounds__(256) k_center_sum(int64_t nchunks, const int32_t* __restrict__ ch_term,
                                                    const int32_t* __restrict__ ch_idx,
                                                    const int64_t* __restrict__ ch_part,
                                                    const int64_t* __restrict__ t_ptr, const int32_t* __restrict__ t_row,
                                                    const float* __restrict__ t_x, const int32_t* __restrict__ a,
                                                    int32_t k, int64_t kst, const RunDesc* __restrict__ runs,
                                                    int64_t dterm, int32_t kbins, float scale,
                                                    long long* __restrict__ S64, long long* __restrict__ part,
                                                    int s64_valid, const unsigned long long* __restrict__ cnt,
                                                    int64_t n, unsigned long long* __restrict__ glog) {
  // graph replay: the first kernel of the update records the assignment's
  // changed count and similarities (glog[0] = entries written so far)
  if (glog && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long pos = glog[0];
    if (pos < (unsigned long long)kLogCap) {
      glog[2 + 2 * pos] = cnt[C_CHANGED];
      glog[3 + 2 * pos] = cnt[C_SIMS];
    }
    glog[0] = pos + 1;
  }
  if (!full_update(s64_valid, cnt, n)) return;
  extern __shared__ int bins_all[];
  const int lane = threadIdx.x & 31;
  int* hi = bins_all + (int64_t)(threadIdx.x >> 5) * 2 * kbins;
  int* lo = hi + kbins;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nchunks; g += nw) {
    const int64_t key = ch_term[g];
    const SumCol sc = sum_col(key, k, kst, runs, dterm);
    const int64_t b = t_ptr[key] + (int64_t)ch_idx[g] * kChunk;
    const int64_t e = min(t_ptr[key + 1], b + kChunk);
    for (int j = lane; j < sc.k; j += 32) {
      hi[j] = 0;
      lo[j] = 0;
    }
    __syncwarp();
    // four entries per lane per step: their loads and label gathers are
    // issued before any of the (order-free, exact) integer additions
    for (int64_t p0 = b + lane; p0 < e; p0 += 128) {
      int32_t r[4];
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t p = p0 + 32 * u;
        r[u] = p < e ? t_row[p] : -1;
        x[u] = p < e ? t_x[p] : 0.f;
      }
      int32_t lab[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) lab[u] = r[u] >= 0 ? a[r[u]] - sc.koff : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (lab[u] >= 0) {
          const long long fx = to_fixed(x[u], scale);
          atomicAdd(hi + lab[u], (int)(fx >> 20));
          atomicAdd(lo + lab[u], (int)(fx & 0xFFFFF));
        }
    }
    __syncwarp();
    const int64_t ps = ch_part[g];
    long long* dst = ps < 0 ? S64 + sc.t * kst + sc.koff : part + ps * kbins;
    const int lim = ps < 0 ? sc.kw : sc.k;
    for (int j = lane; j < lim; j += 32) dst[j] = (j < sc.k) ? ((long long)hi[j] << 20) + (long long)lo[j] : 0ll;
    __syncwarp();
  }
}

__global__ void k_center_sum_multi(int64_t nmulti, const int32_t* __restrict__ mterm, const int64_t* __restrict__ mbase,
                                   const int32_t* __restrict__ mcnt, const long long* __restrict__ part, int32_t k,
                                   int64_t kst, const RunDesc* __restrict__ runs, int64_t dterm, int32_t kbins,
                                   long long* __restrict__ S64, int s64_valid,
                                   const unsigned long long* __restrict__ cnt, int64_t n) {
  if (!full_update(s64_valid, cnt, n)) return;
  const int64_t kbw = runs ? kbins : kst;  // slice width iterated per column
  const int64_t total = nmulti * kbw;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = q / kbw;
    const int j = (int)(q - m * kbw);
    const SumCol sc = sum_col(mterm[m], k, kst, runs, dterm);
    if (j >= sc.kw) continue;
    long long s = 0;
    if (j < sc.k) {
      const long long* pr = part + mbase[m] * kbins + j;
      const int nc = mcnt[m];
      int c = 0;
      for (; c + 8 <= nc; c += 8) {
        long long v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = pr[(int64_t)(c + u) * kbins];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
      }
      for (; c < nc; ++c) s += pr[(int64_t)c * kbins];
    }
    S64[sc.t * kst + sc.koff + j] = s;
  }
}

// Incremental: warp per changed row i (old label -> a[i]); each entry's fixed
// point value -- the same x = v / |x_i| as the term-major copy -- moves from
// the old cluster's sum to the new one.  Both clusters become dirty.
template <typename VT>
__global__ void __launch_bounds__(256) k_center_delta(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const VT* __restrict__ val, const float* __restrict__ rinv,
                                                      const int32_t* __restrict__ chg_i,
                                                      const int32_t* __restrict__ chg_old, const int32_t* __restrict__ a,
                                                      int64_t kst, float scale, long long* __restrict__ S64,
                                                      int32_t* __restrict__ dflag, int s64_valid,
                                                      const unsigned long long* __restrict__ cnt, int64_t n) {
  if (full_update(s64_valid, cnt, n)) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nchg = (int64_t)cnt[C_CHG];
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nchg; q += nw) {
    const int32_t i = chg_i[q], old = chg_old[q], nu = a[i];
    if (lane == 0) {
      dflag[old] = 1;
      dflag[nu] = 1;
    }
    const float ri = rinv[i];
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int64_t t = col[p];
      const long long fx = to_fixed(__fmul_rn(to_f32(val[p]), ri), scale);
      atomicAdd(reinterpret_cast<unsigned long long*>(S64 + t * kst + old), (unsigned long long)(-fx));
      atomicAdd(reinterpret_cast<unsigned long long*>(S64 + t * kst + nu), (unsigned long long)fx);
    }
  }
}

// One block: the list of dirty clusters in ascending order (all clusters
// after a full recompute), dmark[j] / dpos[j] for lookups, flags cleared.
__global__ void __launch_bounds__(1024) k_dirty(int32_t k, int32_t* __restrict__ dflag, int32_t* __restrict__ dmark,
                                                int32_t* __restrict__ dpos, int32_t* __restrict__ dlist,
                                                unsigned long long* __restrict__ cnt, int s64_valid, int64_t n) {
  __shared__ int wsum[32];
  __shared__ int base;
  const bool full = full_update(s64_valid, cnt, n);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int j0 = 0; j0 < k; j0 += 1024) {
    const int j = j0 + threadIdx.x;
    const bool d = (j < k) && (full || dflag[j] != 0);
    const unsigned ball = __ballot_sync(SKM_FULL_MASK, d);
    if (lane == 0) wsum[wid] = __popc(ball);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    const int pos = base + before + __popc(ball & ((1u << lane) - 1u));
    if (j < k) {
      dmark[j] = d ? 1 : 0;
      dpos[j] = d ? pos : -1;
      if (d) dlist[pos] = j;
      dflag[j] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < 32; ++w) tot += wsum[w];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[C_NDIRTY] = (unsigned long long)base;
}

// grid (ceil(d/kTB), ceil(k/32)), block (32, 8): thread (x, y) handles dirty
// slot 32 blockIdx.y + x and terms t = y, y+8, ... of the block's range.
// Squares summed in FP32 with a compensation term (Neumaier), accurate to
// ~2u per thread; threads and blocks combine in FP64.
__global__ void k_colnorm_part(const long long* __restrict__ S64, float inv, int64_t d, int64_t kst,
                               const int32_t* __restrict__ dlist, const unsigned long long* __restrict__ cnt,
                               double* __restrict__ red) {
  __shared__ double sh[8][33];
  const int nd = (int)cnt[C_NDIRTY];
  const int slot = blockIdx.y * 32 + threadIdx.x;
  if ((int)(blockIdx.y * 32) >= nd) return;
  const int64_t t0 = (int64_t)blockIdx.x * kTB;
  float s = 0.f, comp = 0.f;
  if (slot < nd) {
    const int j = dlist[slot];
    for (int64_t t = t0 + threadIdx.y; t < min(d, t0 + kTB); t += 8) {
      const float v = from_fixed(S64[t * kst + j], inv);
      const float sq = __fmul_rn(v, v);
      const float err_sq = __fmaf_rn(v, v, -sq);  // exact low part of v*v
      const float ns = __fadd_rn(s, sq);
      comp += (fabsf(s) >= fabsf(sq)) ? ((s - ns) + sq) : ((sq - ns) + s);
      comp += err_sq;
      s = ns;
    }
  }
  sh[threadIdx.y][threadIdx.x] = (double)s + (double)comp;
  __syncthreads();
  if (threadIdx.y == 0 && slot < nd) {
    double r = 0.0;
    for (int y = 0; y < 8; ++y) r += sh[y][threadIdx.x];
    red[(int64_t)blockIdx.x * kst + slot] = r;
  }
}

// Block per dirty slot: |S_j| from the per-block partials in a fixed order.
__global__ void __launch_bounds__(128) k_colnorm_final(const double* __restrict__ red, int64_t nblk, int64_t kst,
                                                       const int32_t* __restrict__ dlist,
                                                       const unsigned long long* __restrict__ cnt,
                                                       double* __restrict__ nrm) {
  __shared__ double sh[128];
  const int slot = blockIdx.x;
  if (slot >= (int)cnt[C_NDIRTY]) return;
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += red[b * kst + slot];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 64; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) nrm[dlist[slot]] = sqrt(sh[0]);
}

// grid (ceil(d/kTB), ceil(k/32)), block (32, 8), dirty slots as above.  The
// dirty centers are overwritten in place; red2 receives per block and slot
// sum c^2, sum c'^2 and sum (c - c')^2 (FP32 per thread over 32 terms --
// relative error <= 36u, covered by the slack of k_drift_final).
__global__ void k_normalize_drift(const long long* __restrict__ S64, float inv, float* __restrict__ Ct,
                                  const double* __restrict__ nrm, int64_t d, int64_t kst,
                                  const int32_t* __restrict__ dlist, const unsigned long long* __restrict__ cnt,
                                  double* __restrict__ red2) {
  __shared__ double sh[3][8][33];
  const int nd = (int)cnt[C_NDIRTY];
  const int slot = blockIdx.y * 32 + threadIdx.x;
  if ((int)(blockIdx.y * 32) >= nd) return;
  const int64_t t0 = (int64_t)blockIdx.x * kTB;
  float sn = 0.f, so = 0.f, sd = 0.f;
  if (slot < nd) {
    const int j = dlist[slot];
    const double nr = nrm[j];
    const bool empty = !(nr > 0.0);
    const float rn = empty ? 0.f : (float)(1.0 / nr);
    for (int64_t t = t0 + threadIdx.y; t < min(d, t0 + kTB); t += 8) {
      float* cp = Ct + t * kst + j;
      const float co = *cp;
      const float cn = empty ? co : __fmul_rn(from_fixed(S64[t * kst + j], inv), rn);
      *cp = cn;
      const float df = cn - co;
      sn = __fmaf_rn(cn, cn, sn);
      so = __fmaf_rn(co, co, so);
      sd = __fmaf_rn(df, df, sd);
    }
  }
  sh[0][threadIdx.y][threadIdx.x] = sn;
  sh[1][threadIdx.y][threadIdx.x] = so;
  sh[2][threadIdx.y][threadIdx.x] = sd;
  __syncthreads();
  if (threadIdx.y == 0 && slot < nd) {
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    for (int y = 0; y < 8; ++y) {
      r0 += sh[0][y][threadIdx.x];
      r1 += sh[1][y][threadIdx.x];
      r2 += sh[2][y][threadIdx.x];
    }
    double* o = red2 + ((int64_t)blockIdx.x * kst + slot) * 3;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
  }
}

// Block per center (grid kst).  Clean centers did not move: p = 1, sine 0.
// Dirty ones: from N = |c|, N' = |c'| and D = |c - c'|^2 (relative error <= e,
// e = 40u + d 2^-53):  1 - cos = (D - (N - N')^2) / (2 N N'), hence
//   q_up = D (1+4e) / (2 N N')                           >= 1 - cos
//   q_dn = (D (1-e) - (|N-N'| + e)^2) / (2 N N' (1+3e))  <= 1 - cos
// pd = rd(1 - q_up), pu = ru(1 - q_dn), q = ru(max sin over [q_dn, q_up]).
__global__ void __launch_bounds__(128) k_drift_final(const double* __restrict__ red2, int64_t nblk, int32_t k,
                                                     int64_t kst, int64_t d, const int32_t* __restrict__ dmark,
                                                     const int32_t* __restrict__ dpos, float* __restrict__ pdn,
                                                     float* __restrict__ pup, float* __restrict__ qup,
                                                     double* __restrict__ cnorm) {
  __shared__ double sh[3][128];
  const int j = blockIdx.x;
  if (j >= k || !dmark[j]) {
    if (threadIdx.x == 0) {
      pdn[j] = 1.f;
      pup[j] = 1.f;
      qup[j] = 0.f;
    }
    return;
  }
  const int slot = dpos[j];
  double sn = 0.0, so = 0.0, sd = 0.0;
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
    const double* r = red2 + (b * kst + slot) * 3;
    sn += r[0];
    so += r[1];
    sd += r[2];
  }
  sh[0][threadIdx.x] = sn;
  sh[1][threadIdx.x] = so;
  sh[2][threadIdx.x] = sd;
  __syncthreads();
  for (int o = 64; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  sn = sh[0][0];
  so = sh[1][0];
  sd = sh[2][0];
  const double e = 40.0 * 0x1.0p-24 + ((double)d + 8.0) * 0x1.0p-53;
  const double N = sqrt(sn), No = sqrt(so);
  cnorm[j] = N;
  float pd, pu, q;
  if (sd == 0.0) {
    pd = 1.f;
    pu = 1.f;
    q = 0.f;
  } else {
    const double den = 2.0 * N * No;
    const double qu = sd * (1.0 + 4.0 * e) / den;
    const double dn = fabs(N - No) + e;
    double qd = (sd * (1.0 - e) - dn * dn) / (den * (1.0 + 3.0 * e));
    if (qd < 0.0) qd = 0.0;
    double lo = 1.0 - qu, hi = 1.0 - qd;
    lo = lo < -1.0 ? -1.0 : lo;
    hi = hi > 1.0 ? 1.0 : hi;
    pd = fmaxf(__double2float_rd(lo - 0x1.0p-60), -1.f);
    pu = fminf(__double2float_ru(hi + 0x1.0p-60), 1.f);
    double smax;
    if (qd <= 1.0 && qu >= 1.0) smax = 1.0;
    else if (qu < 1.0) smax = sqrt(qu * (2.0 - qu));
    else smax = sqrt(qd * (2.0 - qd));
    q = fminf(__double2float_ru(smax * (1.0 + 4.0 * e) + 0x1.0p-60), 1.f);
  }
  pdn[j] = pd;
  pup[j] = pu;
  qup[j] = q;
}

// One block: the objective J = sum_j |S_j| (fixed order) and Hamerly's
// worst-drift summary -- argmin / min / second min of pd and of pu, argmax /
// max / second max of q, lowest index on ties (Section 5.3: p' is the minimum
// over the other centers, hence the second value for the argmin's members).
__global__ void __launch_bounds__(1024) k_hsel_obj(const float* __restrict__ pdn, const float* __restrict__ pup,
                                                   const float* __restrict__ qup, const double* __restrict__ nrm,
                                                   int32_t k, float* __restrict__ hsel, double* __restrict__ obj,
                                                   unsigned long long* __restrict__ cnt) {
  // the last kernel of the update to read the assignment's counters has run:
  // zero them for the next assignment (which then needs no memset)
  if (threadIdx.x < C_ERR) cnt[threadIdx.x] = 0ull;
  __shared__ float s_pd[1024], s_pu[1024], s_q[1024], s_pd2[1024], s_pu2[1024], s_q2[1024];
  __shared__ int s_jd[1024], s_ju[1024], s_jq[1024];
  __shared__ double s_J[1024];
  float bd = FLT_MAX, bd2 = FLT_MAX, bu = FLT_MAX, bu2 = FLT_MAX, bq = -FLT_MAX, bq2 = -FLT_MAX;
  int jd = INT_MAX, ju = INT_MAX, jq = INT_MAX;
  double J = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const float x = pdn[j], y = pup[j], z = qup[j];
    if (x < bd) { bd2 = bd; bd = x; jd = j; } else if (x < bd2) bd2 = x;
    if (y < bu) { bu2 = bu; bu = y; ju = j; } else if (y < bu2) bu2 = y;
    if (z > bq) { bq2 = bq; bq = z; jq = j; } else if (z > bq2) bq2 = z;
    J += nrm[j];
  }
  s_pd[threadIdx.x] = bd; s_pd2[threadIdx.x] = bd2; s_jd[threadIdx.x] = jd;
  s_pu[threadIdx.x] = bu; s_pu2[threadIdx.x] = bu2; s_ju[threadIdx.x] = ju;
  s_q[threadIdx.x] = bq; s_q2[threadIdx.x] = bq2; s_jq[threadIdx.x] = jq;
  s_J[threadIdx.x] = J;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const int a = threadIdx.x, b = threadIdx.x + o;
      if (s_pd[b] < s_pd[a] || (s_pd[b] == s_pd[a] && s_jd[b] < s_jd[a])) {
        s_pd2[a] = fminf(s_pd2[b], s_pd[a]);
        s_pd[a] = s_pd[b];
        s_jd[a] = s_jd[b];
      } else {
        s_pd2[a] = fminf(s_pd2[a], s_pd[b]);
      }
      if (s_pu[b] < s_pu[a] || (s_pu[b] == s_pu[a] && s_ju[b] < s_ju[a])) {
        s_pu2[a] = fminf(s_pu2[b], s_pu[a]);
        s_pu[a] = s_pu[b];
        s_ju[a] = s_ju[b];
      } else {
        s_pu2[a] = fminf(s_pu2[a], s_pu[b]);
      }
      if (s_q[b] > s_q[a] || (s_q[b] == s_q[a] && s_jq[b] < s_jq[a])) {
        s_q2[a] = fmaxf(s_q2[b], s_q[a]);
        s_q[a] = s_q[b];
        s_jq[a] = s_jq[b];
      } else {
        s_q2[a] = fmaxf(s_q2[a], s_q[b]);
      }
      s_J[a] += s_J[b];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // with a single center there is no "other" center: no drift to account for
    const bool one = (k == 1);
    hsel[0] = (float)s_jd[0];
    hsel[1] = s_pd[0];
    hsel[2] = one ? 1.f : s_pd2[0];
    hsel[3] = (float)s_ju[0];
    hsel[4] = s_pu[0];
    hsel[5] = one ? 1.f : s_pu2[0];
    hsel[6] = (float)s_jq[0];
    hsel[7] = s_q[0];
    hsel[8] = one ? 0.f : s_q2[0];
    obj[0] = s_J[0];
  }
}

// The Gram by 64 x 64 tiles: grid (ceil(k/64), ceil(k/64), nsplit), block
// 256 = 16 x 16.  Each thread owns a 4 x 4 block of <c_i, c_j>; per term it
// reads 4 + 4 center values from shared memory (float4) for 16 FMAs.  FP32
// products are accumulated over 256 terms, then added to FP64 accumulators
// (the error bound used by k_gram_final).
// ROWS = false: many dirty clusters, tiles (bi, bj) with bi <= bj of the whole
//   Gram into gpart[z][i][j].
// ROWS = true: 1..row_max (<= 64) dirty clusters; the A tile holds the dirty
//   centers (gathered by dlist), only bi = 0 runs, into gpart[z][r][j].
constexpr int kGT = 64;
template <bool ROWS>
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ Ct, int64_t d, int32_t k, int64_t kst,
                                                   int64_t per_split, double* __restrict__ gpart,
                                                   const int32_t* __restrict__ dlist,
                                                   const unsigned long long* __restrict__ cnt, int32_t row_max) {
  const int nd = (int)cnt[C_NDIRTY];
  if (ROWS ? (nd == 0 || nd > row_max || blockIdx.x != 0) : (blockIdx.x > blockIdx.y || nd <= row_max)) return;
  __shared__ __align__(16) float A[32][kGT], B[32][kGT];
  const int i0 = blockIdx.x * kGT, j0 = blockIdx.y * kGT;
  const int64_t tb = (int64_t)blockIdx.z * per_split, te = min(d, tb + per_split);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc64[4][4];
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      acc64[x][y] = 0.0;
      acc[x][y] = 0.f;
    }
  int steps = 0;
  for (int64_t t0 = tb; t0 < te; t0 += 32) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + 256 * h;
      const int r = q >> 4, c4 = (q & 15) * 4;
      const int64_t t = t0 + r;
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (t < te) {
        if (ROWS) {
          const float* row = Ct + t * kst;
          va.x = (c4 + 0 < nd) ? row[dlist[c4 + 0]] : 0.f;
          va.y = (c4 + 1 < nd) ? row[dlist[c4 + 1]] : 0.f;
          va.z = (c4 + 2 < nd) ? row[dlist[c4 + 2]] : 0.f;
          va.w = (c4 + 3 < nd) ? row[dlist[c4 + 3]] : 0.f;
        } else if (i0 + c4 < kst) {
          va = *reinterpret_cast<const float4*>(Ct + t * kst + i0 + c4);
        }
        if (j0 + c4 < kst) vb = *reinterpret_cast<const float4*>(Ct + t * kst + j0 + c4);
      }
      *reinterpret_cast<float4*>(&A[r][c4]) = va;
      *reinterpret_cast<float4*>(&B[r][c4]) = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float4 av = *reinterpret_cast<const float4*>(&A[r][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&B[r][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = __fmaf_rn(ar[x], br[y], acc[x][y]);
    }
    __syncthreads();
    if (++steps == 8) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          acc64[x][y] += (double)acc[x][y];
          acc[x][y] = 0.f;
        }
      steps = 0;
    }
  }
  const int rows = ROWS ? row_max : k;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + ty * 4 + x, j = j0 + tx * 4 + y;
      if (i < (ROWS ? nd : k) && j < k)
        gpart[((int64_t)blockIdx.z * rows + i) * k + j] = acc64[x][y] + (double)acc[x][y];
    }
}

// Thread per (i, j), i <= j: the Gram entry as the sum of the split partials
// in split order (loads coalesced across threads).
__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ gpart, int32_t nsplit, int32_t k,
                                                     double* __restrict__ G, const unsigned long long* __restrict__ cnt,
                                                     int32_t row_max) {
  if ((int)cnt[C_NDIRTY] <= row_max) return;
  const int64_t kk = (int64_t)k * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kk; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / k), j = (int)(q - (int64_t)i * k);
    if (i > j) continue;
    double g = 0.0;
    int s = 0;
    for (; s + 8 <= nsplit; s += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = gpart[(int64_t)(s + u) * kk + q];
#pragma unroll
      for (int u = 0; u < 8; ++u) g += v[u];
    }
    for (; s < nsplit; ++s) g += gpart[(int64_t)s * kk + q];
    G[q] = g;
  }
}

__global__ void __launch_bounds__(256) k_gram_rows_reduce(const double* __restrict__ rpart, int32_t nsplit,
                                                          int32_t k, const int32_t* __restrict__ dlist,
                                                          const unsigned long long* __restrict__ cnt, int32_t row_max,
                                                          double* __restrict__ G) {
  const int nd = (int)cnt[C_NDIRTY];
  if (nd > row_max) return;
  const int64_t tot = (int64_t)nd * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / k), j = (int)(q - (int64_t)r * k);
    double g = 0.0;
    for (int s = 0; s < nsplit; ++s) g += rpart[((int64_t)s * row_max + r) * k + j];
    const int i = dlist[r];
    // the same dot product is computed by both rows when i and j are dirty;
    // the two values are identical (same products, same term ranges)
    G[(int64_t)min(i, j) * k + max(i, j)] = g;
  }
}

// Block per center i: <c_i, c_j> (upper triangle of G), normalised by the FP64
// norms and widened by the error bound eg, then cc(i,j) = sqrt((g+1)/2)
// rounded up and s(i) = max_{j != i} cc(i,j).
__global__ void __launch_bounds__(256) k_gram_final(const double* __restrict__ G, int32_t k, int64_t kst,
                                                    const double* __restrict__ cnorm, double eg,
                                                    float* __restrict__ cc, float* __restrict__ sc) {
  __shared__ float sh[256];
  const int i = blockIdx.x;
  float best = -1.f;
  for (int j = threadIdx.x; j < kst; j += blockDim.x) {
    if (j >= k) {
      cc[(int64_t)i * kst + j] = 1.f;
      continue;
    }
    const int lo = min(i, j), hi = max(i, j);
    const double g = G[(int64_t)lo * k + hi];
    const double den = cnorm[i] * cnorm[j];
    double gh = (den > 0.0 ? g / den : 0.0) + eg;
    double h = 0.5 * (gh + 1.0);
    h = h < 0.0 ? 0.0 : (h > 1.0 ? 1.0 : h);
    const float v = fminf(__double2float_ru(sqrt(h) * (1.0 + 0x1.0p-50)), 1.f);
    cc[(int64_t)i * kst + j] = v;
    if (j != i) best = fmaxf(best, v);
  }
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) sc[i] = sh[0];
}

// ---------------------------------------------------------------- batches

// Block per run: Hamerly's worst-drift summary over the run's own centers
// koff .. koff + k - 1 (global ids), the rule of k_hsel_obj.
__global__ void __launch_bounds__(256) k_hsel_runs(const float* __restrict__ pdn, const float* __restrict__ pup,
                                                   const float* __restrict__ qup, const RunDesc* __restrict__ runs,
                                                   float* __restrict__ hsel) {
  const RunDesc R = runs[blockIdx.x];
  __shared__ float s_pd[256], s_pu[256], s_q[256], s_pd2[256], s_pu2[256], s_q2[256];
  __shared__ int s_jd[256], s_ju[256], s_jq[256];
  float bd = FLT_MAX, bd2 = FLT_MAX, bu = FLT_MAX, bu2 = FLT_MAX, bq = -FLT_MAX, bq2 = -FLT_MAX;
  int jd = INT_MAX, ju = INT_MAX, jq = INT_MAX;
  for (int j = R.koff + threadIdx.x; j < R.koff + R.k; j += blockDim.x) {
    const float x = pdn[j], y = pup[j], z = qup[j];
    if (x < bd) { bd2 = bd; bd = x; jd = j; } else if (x < bd2) bd2 = x;
    if (y < bu) { bu2 = bu; bu = y; ju = j; } else if (y < bu2) bu2 = y;
    if (z > bq) { bq2 = bq; bq = z; jq = j; } else if (z > bq2) bq2 = z;
  }
  s_pd[threadIdx.x] = bd; s_pd2[threadIdx.x] = bd2; s_jd[threadIdx.x] = jd;
  s_pu[threadIdx.x] = bu; s_pu2[threadIdx.x] = bu2; s_ju[threadIdx.x] = ju;
  s_q[threadIdx.x] = bq; s_q2[threadIdx.x] = bq2; s_jq[threadIdx.x] = jq;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const int a = threadIdx.x, b = threadIdx.x + o;
      if (s_pd[b] < s_pd[a] || (s_pd[b] == s_pd[a] && s_jd[b] < s_jd[a])) {
        s_pd2[a] = fminf(s_pd2[b], s_pd[a]);
        s_pd[a] = s_pd[b];
        s_jd[a] = s_jd[b];
      } else {
        s_pd2[a] = fminf(s_pd2[a], s_pd[b]);
      }
      if (s_pu[b] < s_pu[a] || (s_pu[b] == s_pu[a] && s_ju[b] < s_ju[a])) {
        s_pu2[a] = fminf(s_pu2[b], s_pu[a]);
        s_pu[a] = s_pu[b];
        s_ju[a] = s_ju[b];
      } else {
        s_pu2[a] = fminf(s_pu2[a], s_pu[b]);
      }
      if (s_q[b] > s_q[a] || (s_q[b] == s_q[a] && s_jq[b] < s_jq[a])) {
        s_q2[a] = fmaxf(s_q2[b], s_q[a]);
        s_q[a] = s_q[b];
        s_jq[a] = s_jq[b];
      } else {
        s_q2[a] = fmaxf(s_q2[a], s_q[b]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool one = (R.k == 1);
    float* h = hsel + (int64_t)HSEL_N * blockIdx.x;
    h[0] = (float)s_jd[0];
    h[1] = s_pd[0];
    h[2] = one ? 1.f : s_pd2[0];
    h[3] = (float)s_ju[0];
    h[4] = s_pu[0];
    h[5] = one ? 1.f : s_pu2[0];
    h[6] = (float)s_jq[0];
    h[7] = s_q[0];
    h[8] = one ? 0.f : s_q2[0];
  }
}

// First position p in the ascending list[0..len) with list[p] >= v.
__device__ __forceinline__ int lower_pos(const int32_t* __restrict__ list, int len, int32_t v) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (list[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One block: per run the range of its real dirty centers in the ascending
// dirty list (dbeg, dcnt) and its tile count ceil(dcnt / 64) * ceil(k / 64);
// task_off = the exclusive prefix over runs (task_off[nruns] = total).
__global__ void __launch_bounds__(1024) k_gram_plan(const int32_t* __restrict__ dlist,
                                                    const unsigned long long* __restrict__ cnt,
                                                    const RunDesc* __restrict__ runs, int32_t nruns,
                                                    int32_t* __restrict__ dbeg, int32_t* __restrict__ dcnt,
                                                    int64_t* __restrict__ task_off) {
  __shared__ long long part[1024];
  const int nd = (int)cnt[C_NDIRTY];
  const int per = (nruns + (int)blockDim.x - 1) / (int)blockDim.x;
  const int r0 = (int)threadIdx.x * per, r1 = min(nruns, r0 + per);
  long long mine = 0;
  for (int r = r0; r < r1; ++r) {
    const int lo = lower_pos(dlist, nd, runs[r].koff), hi = lower_pos(dlist, nd, runs[r].koff + runs[r].k);
    dbeg[r] = lo;
    dcnt[r] = hi - lo;
    mine += (long long)((hi - lo + kGT - 1) / kGT) * ((runs[r].k + kGT - 1) / kGT);
  }
  part[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = s;
      s += v;
    }
    task_off[nruns] = s;
  }
  __syncthreads();
  long long s = part[threadIdx.x];
  for (int r = r0; r < r1; ++r) {
    task_off[r] = s;
    s += (long long)((dcnt[r] + kGT - 1) / kGT) * ((runs[r].k + kGT - 1) / kGT);
  }
}

// Persistent blocks over the batch's Gram tasks: a task is (run, block of <= 64
// dirty centers of the run, tile of 64 of the run's centers).  Its 64 x 64
// dot products over all d terms (threads own 4 x 4, FP32 products summed over
// 256 terms, then in FP64 -- the chunking of k_gram_part, so the error bound
// eg holds) are written to both G[i][j] and G[j][i] of the run's block: a
// moved center changes its row and its column.  When i and j both moved,
// both tasks compute the same value (the same products in the same order).
__global__ void __launch_bounds__(256) k_gram_batch(const float* __restrict__ Ct, int64_t d, int64_t K,
                                                    const RunDesc* __restrict__ runs, int32_t nruns,
                                                    const int32_t* __restrict__ dlist,
                                                    const int32_t* __restrict__ dbeg,
                                                    const int32_t* __restrict__ dcnt,
                                                    const int64_t* __restrict__ task_off, double* __restrict__ G) {
  __shared__ __align__(16) float A[32][kGT], B[32][kGT];
  __shared__ int rows_g[kGT];
  const int64_t total = task_off[nruns];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int64_t task = blockIdx.x; task < total; task += gridDim.x) {
    int lo = 0, hi = nruns - 1;  // the run: last r with task_off[r] <= task
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (task_off[mid] <= task) lo = mid;
      else hi = mid - 1;
    }
    const RunDesc R = runs[lo];
    const int64_t t_in = task - task_off[lo];
    const int nj = (R.k + kGT - 1) / kGT;
    const int db = (int)(t_in / nj), j0 = (int)(t_in % nj) * kGT;  // j0: local
    const int nrow = min(kGT, dcnt[lo] - db * kGT);
    __syncthreads();  // the previous task's readers of rows_g are done
    if (tid < kGT) rows_g[tid] = tid < nrow ? dlist[dbeg[lo] + db * kGT + tid] : -1;
    __syncthreads();
    double acc64[4][4];
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        acc64[x][y] = 0.0;
        acc[x][y] = 0.f;
      }
    int steps = 0;
    for (int64_t t0 = 0; t0 < d; t0 += 32) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = tid + 256 * h;
        const int r = q >> 4, c4 = (q & 15) * 4;
        const int64_t t = t0 + r;
        float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
        if (t < d) {
          const float* row = Ct + t * K;
          va.x = rows_g[c4 + 0] >= 0 ? row[rows_g[c4 + 0]] : 0.f;
          va.y = rows_g[c4 + 1] >= 0 ? row[rows_g[c4 + 1]] : 0.f;
          va.z = rows_g[c4 + 2] >= 0 ? row[rows_g[c4 + 2]] : 0.f;
          va.w = rows_g[c4 + 3] >= 0 ? row[rows_g[c4 + 3]] : 0.f;
          // the run's slice is kst wide (a multiple of 8): 16-byte loads stay inside it
          if (j0 + c4 < R.kst) vb = *reinterpret_cast<const float4*>(row + R.koff + j0 + c4);
        }
        *reinterpret_cast<float4*>(&A[r][c4]) = va;
        *reinterpret_cast<float4*>(&B[r][c4]) = vb;
      }
      __syncthreads();
#pragma unroll 8
      for (int r = 0; r < 32; ++r) {
        const float4 av = *reinterpret_cast<const float4*>(&A[r][ty * 4]);
        const float4 bv = *reinterpret_cast<const float4*>(&B[r][tx * 4]);
        const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = __fmaf_rn(ar[x], br[y], acc[x][y]);
      }
      __syncthreads();
      if (++steps == 8) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            acc64[x][y] += (double)acc[x][y];
            acc[x][y] = 0.f;
          }
        steps = 0;
      }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int ri = ty * 4 + x, jl = j0 + tx * 4 + y;
        if (ri < nrow && jl < R.k) {
          const int il = rows_g[ri] - R.koff;
          const double g = acc64[x][y] + (double)acc[x][y];
          G[R.ccoff + (int64_t)il * R.kst + jl] = g;
          G[R.ccoff + (int64_t)jl * R.kst + il] = g;
        }
      }
  }
}

// Block per global center i of a batch: its run's cc row (the rule of
// k_gram_final on the run's block of G) and s(i).  A run's padding centers
// (local ids k .. kst - 1) label no row, so their rows are skipped; their
// columns get cc = 1.
__global__ void __launch_bounds__(256) k_gram_final_batch(const double* __restrict__ G,
                                                          const RunDesc* __restrict__ runs, int32_t nruns,
                                                          const double* __restrict__ cnorm, double eg,
                                                          float* __restrict__ cc, float* __restrict__ sc) {
  __shared__ float sh[256];
  const int i = blockIdx.x;
  int lo = 0, hi = nruns - 1;  // the run: last r with koff <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (runs[mid].koff <= i) lo = mid;
    else hi = mid - 1;
  }
  const RunDesc R = runs[lo];
  const int il = i - R.koff;
  if (il >= R.k) {
    if (threadIdx.x == 0) sc[i] = 1.f;
    return;
  }
  float best = -1.f;
  for (int j = threadIdx.x; j < R.kst; j += blockDim.x) {
    float* out = cc + R.ccoff + (int64_t)il * R.kst + j;
    if (j >= R.k) {
      *out = 1.f;
      continue;
    }
    const double g = G[R.ccoff + (int64_t)il * R.kst + j];
    const double den = cnorm[i] * cnorm[R.koff + j];
    double gh = (den > 0.0 ? g / den : 0.0) + eg;
    double h = 0.5 * (gh + 1.0);
    h = h < 0.0 ? 0.0 : (h > 1.0 ? 1.0 : h);
    const float v = fminf(__double2float_ru(sqrt(h) * (1.0 + 0x1.0p-50)), 1.f);
    *out = v;
    if (j != il) best = fmaxf(best, v);
  }
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) sc[i] = sh[0];
}

inline unsigned grid_cap(int64_t items, int per_block, int nsm, int per_sm = 16) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g > (int64_t)nsm * per_sm) g = (int64_t)nsm * per_sm;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename VT>
int center_delta_t(skm_ctx* c) {
  SKM_PROF_BEGIN(c, "k_center_delta");
  k_center_delta<VT><<<grid_cap(c->n * 32, 256, c->nsm), 256, 0, c->st>>>(
      c->rp, c->col, (const VT*)c->val, c->rinv, c->chg_i, c->chg_old, c->a, c->kst, c->fx_scale, c->S64, c->dflag,
      c->s64_valid, c->cnt, c->n);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

}  // namespace

int64_t reduction_blocks(int64_t d) { return (d + kTB - 1) / kTB; }

int update_centers(skm_ctx* c) {
  const int k = c->k;
  if (c->layout == SKM_DENSE) {
    const int rc = dense_center_sums(c);
    if (rc) return rc;
    return finish_update(c);
  }
  // ---- sums: a full recompute, or only the changed rows (decided on the device)
  const int32_t kbins = c->nruns > 0 ? c->kmax : k;
  int wpb = (int)((96 * 1024) / ((int64_t)kbins * 8));  // two int32 bins per cluster per warp
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  const size_t smem = (size_t)wpb * kbins * 8;
  if (smem > 48 * 1024)
    SKM_CUDA_TRY(cudaFuncSetAttribute(k_center_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SKM_PROF_BEGIN(c, "k_center_sum");
  k_center_sum<<<grid_cap(c->nchunks, wpb, c->nsm), wpb * 32, smem, c->st>>>(
      c->nchunks, c->ch_term, c->ch_idx, c->ch_part, c->t_ptr, c->t_row, (const float*)c->t_val, c->a, k, c->kst,
      c->runs, c->d, kbins, c->fx_scale, c->S64, c->part64, c->s64_valid, c->cnt, c->n, c->glog_active);
  SKM_LAUNCHED(c);
  if (c->nmulti > 0) {
    const int64_t kbw = c->nruns > 0 ? kbins : c->kst;
    SKM_PROF_BEGIN(c, "k_center_sum_multi");
    k_center_sum_multi<<<grid_cap(c->nmulti * kbw, 256, c->nsm), 256, 0, c->st>>>(
        c->nmulti, c->multi_term, c->multi_base, c->multi_cnt, c->part64, k, c->kst, c->runs, c->d, kbins, c->S64,
        c->s64_valid, c->cnt, c->n);
    SKM_LAUNCHED(c);
  }
  int rc = SKM_OK;
  switch (c->dtype) {
    case SKM_F32: rc = center_delta_t<float>(c); break;
    case SKM_F16: rc = center_delta_t<__half>(c); break;
    default: rc = center_delta_t<__nv_bfloat16>(c); break;
  }
  if (rc) return rc;
  return finish_update(c);
}

// Dirty list, norms, new centers, drift and (full variants) the center-center
// bounds, shared by the sparse and dense paths.
int finish_update(skm_ctx* c) {
  const int k = c->k;
  SKM_PROF_BEGIN(c, "k_dirty");
  k_dirty<<<1, 1024, 0, c->st>>>(k, c->dflag, c->dmark, c->dpos, c->dlist, c->cnt, c->s64_valid, c->n);
  SKM_LAUNCHED(c);
  c->s64_valid = 1;
  // ---- norms, new centers and drift of the dirty clusters
  const int64_t nblk = reduction_blocks(c->d);
  dim3 grid((unsigned)nblk, (unsigned)((k + 31) / 32));
  SKM_PROF_BEGIN(c, "k_colnorm_part");
  k_colnorm_part<<<grid, dim3(32, 8), 0, c->st>>>(c->S64, c->fx_inv, c->d, c->kst, c->dlist, c->cnt, c->red);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_colnorm_final");
  k_colnorm_final<<<k, 128, 0, c->st>>>(c->red, nblk, c->kst, c->dlist, c->cnt, c->nrm);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_normalize_drift");
  k_normalize_drift<<<grid, dim3(32, 8), 0, c->st>>>(c->S64, c->fx_inv, c->Ct, c->nrm, c->d, c->kst, c->dlist,
                                                     c->cnt, c->red);
  SKM_LAUNCHED(c);
  double* cnorm = c->nrm + c->kst;  // second half of the norm buffer: |c(j)| of the centers
  SKM_PROF_BEGIN(c, "k_drift_final");
  k_drift_final<<<c->kst, 128, 0, c->st>>>(c->red, nblk, k, c->kst, c->d, c->dmark, c->dpos, c->pdn, c->pup, c->qup,
                                           cnorm);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_hsel_obj");
  k_hsel_obj<<<1, 1024, 0, c->st>>>(c->pdn, c->pup, c->qup, c->nrm, k, c->hsel, c->obj, c->cnt);
  SKM_LAUNCHED(c);
  const bool hamv = (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY);
  const bool full = (c->variant == SKM_ELKAN || c->variant == SKM_HAMERLY);
  // |error| of an FP32 sum of 256 products <= gamma_256 |c_i||c_j|, plus
  // the normalisation by FP64 norms of FP32 vectors.
  const double eg = 260.0 * 0x1.0p-24 / (1.0 - 260.0 * 0x1.0p-24) + 1e-12;
  if (c->nruns > 0) {
    // a batch: per-run drift summaries, per-run (block-diagonal) Gram
    if (hamv) {
      SKM_PROF_BEGIN(c, "k_hsel_runs");
      k_hsel_runs<<<(unsigned)c->nruns, 256, 0, c->st>>>(c->pdn, c->pup, c->qup, c->runs, c->hsel);
      SKM_LAUNCHED(c);
    }
    if (full) {
      SKM_PROF_BEGIN(c, "k_gram_plan");
      k_gram_plan<<<1, 1024, 0, c->st>>>(c->dlist, c->cnt, c->runs, c->nruns, c->gdbeg, c->gdcnt, c->gtask);
      SKM_LAUNCHED(c);
      SKM_PROF_BEGIN(c, "k_gram_batch");
      k_gram_batch<<<(unsigned)(c->nsm * 4), 256, 0, c->st>>>(c->Ct, c->d, c->kst, c->runs, c->nruns, c->dlist,
                                                              c->gdbeg, c->gdcnt, c->gtask, c->G);
      SKM_LAUNCHED(c);
      SKM_PROF_BEGIN(c, "k_gram_final");
      k_gram_final_batch<<<(unsigned)k, 256, 0, c->st>>>(c->G, c->runs, c->nruns, cnorm, eg, c->cc, c->sc);
      SKM_LAUNCHED(c);
    }
    return SKM_OK;
  }
  // ---- center-center bounds (full variants)
  if (full) {
    const int32_t row_max = c->grow_max;
    const int64_t per = (c->d + c->gsplit - 1) / c->gsplit;
    const unsigned tk = (unsigned)((k + kGT - 1) / kGT);
    SKM_PROF_BEGIN(c, "k_gram_part");
    k_gram_part<false><<<dim3(tk, tk, (unsigned)c->gsplit), 256, 0, c->st>>>(c->Ct, c->d, k, c->kst, per, c->gpart,
                                                                             c->dlist, c->cnt, row_max);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_gram_reduce");
    k_gram_reduce<<<grid_cap((int64_t)k * k, 256, c->nsm), 256, 0, c->st>>>(c->gpart, c->gsplit, k, c->G, c->cnt,
                                                                             row_max);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_gram_rows");
    k_gram_part<true><<<dim3(1, tk, (unsigned)c->gsplit), 256, 0, c->st>>>(c->Ct, c->d, k, c->kst, per, c->rpart,
                                                                           c->dlist, c->cnt, row_max);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_gram_rows_reduce");
    k_gram_rows_reduce<<<grid_cap((int64_t)row_max * k, 256, c->nsm), 256, 0, c->st>>>(c->rpart, c->gsplit, k,
                                                                                       c->dlist, c->cnt, row_max, c->G);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_gram_final");
    k_gram_final<<<k, 256, 0, c->st>>>(c->G, k, c->kst, cnorm, eg, c->cc, c->sc);
    SKM_LAUNCHED(c);
  }
  return SKM_OK;
}

}  // namespace skm
