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
//   k_drift_hsel        per center an interval [pd, pu] for cos(angle(c, c'))
//                       and an upper bound q of its sine, rounded outward;
//                       then, by the last block, J = sum_j |S_j| and Hamerly's
//                       worst-drift summary, and the assignment counters
//                       zeroed for the next assignment.
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
// the old cluster's sum to the new one, and both clusters' squared norms
// take the change of the entries' squares (n2_add).  Both clusters become
// dirty.
template <typename VT>
__global__ void __launch_bounds__(256) k_center_delta(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const VT* __restrict__ val, const float* __restrict__ rinv,
                                                      const int32_t* __restrict__ chg_i,
                                                      const int32_t* __restrict__ chg_old, const int32_t* __restrict__ a,
                                                      int64_t kst, float scale, long long* __restrict__ S64,
                                                      int32_t* __restrict__ dflag, int s64_valid,
                                                      const unsigned long long* __restrict__ cnt, int64_t n,
                                                      long long* __restrict__ n2l) {
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
    __int128 co = 0, cn = 0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int64_t t = col[p];
      const long long fx = to_fixed(__fmul_rn(to_f32(val[p]), ri), scale);
      const long long po =
          (long long)atomicAdd(reinterpret_cast<unsigned long long*>(S64 + t * kst + old), (unsigned long long)(-fx));
      const long long pn =
          (long long)atomicAdd(reinterpret_cast<unsigned long long*>(S64 + t * kst + nu), (unsigned long long)fx);
      const __int128 sq = (__int128)fx * fx;
      co += sq - 2 * (__int128)po * fx;
      cn += sq + 2 * (__int128)pn * fx;
    }
    co = warp_sum128(co);
    cn = warp_sum128(cn);
    if (lane == 0) {
      n2_add(n2l, kst, old, co);
      n2_add(n2l, kst, nu, cn);
    }
  }
}

// ------------------------------------------------------------------
// The phases after the sums.  Each is a device routine so that the separate
// kernels below and the fused cooperative kernel (k_finish_fused) run the
// same arithmetic in the same order: their results are bit-identical.  Data
// that another block may have written earlier in the fused launch is read
// with __ldcg (from L2, past this SM's L1).

// One block: the list of dirty clusters in ascending order (all clusters
// after a full recompute), dmark[j] / dpos[j] for lookups, flags cleared.
// wsum: shared, one int per warp of the block.
__device__ __forceinline__ void dev_dirty(int32_t k, int32_t* __restrict__ dflag, int32_t* __restrict__ dmark,
                                          int32_t* __restrict__ dpos, int32_t* __restrict__ dlist,
                                          unsigned long long* __restrict__ cnt, bool full, int* wsum, int* base) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) *base = 0;
  __syncthreads();
  for (int j0 = 0; j0 < k; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const bool d = (j < k) && (full || dflag[j] != 0);
    const unsigned ball = __ballot_sync(SKM_FULL_MASK, d);
    if (lane == 0) wsum[wid] = __popc(ball);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    const int pos = *base + before + __popc(ball & ((1u << lane) - 1u));
    if (j < k) {
      dmark[j] = d ? 1 : 0;
      dpos[j] = d ? pos : -1;
      if (d) dlist[pos] = j;
      dflag[j] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < nwarp; ++w) tot += wsum[w];
      *base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[C_NDIRTY] = (unsigned long long)*base;
}

__global__ void __launch_bounds__(1024) k_dirty(int32_t k, int32_t* __restrict__ dflag, int32_t* __restrict__ dmark,
                                                int32_t* __restrict__ dpos, int32_t* __restrict__ dlist,
                                                unsigned long long* __restrict__ cnt, int s64_valid, int64_t n) {
  __shared__ int wsum[32];
  __shared__ int base;
  dev_dirty(k, dflag, dmark, dpos, dlist, cnt, full_update(s64_valid, cnt, n), wsum, &base);
}

// Tile (bx, by) of 256 terms x 32 dirty slots, threads (x, y) = (tid & 31,
// tid >> 5) of 256: thread (x, y) handles dirty slot 32 by + x and terms
// t = y, y+8, ... of the tile.  After a full recomputation of the sums: the
// exact sum of the squares of the tile's fixed-point values (an __int128,
// see n2_add) into red as (low, high) words; after an incremental update the
// squared norms were kept up to date by k_center_delta and there is nothing
// to do.  sh: shared long long[2][8][33].
__device__ __forceinline__ void dev_colnorm_part(const long long* __restrict__ S64, int64_t d, int64_t kst,
                                                 const int32_t* __restrict__ dlist, int nd, double* __restrict__ red,
                                                 int bx, int by, long long (*sh)[8][33], bool full) {
  if (!full) return;  // the same for the whole block
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int slot = by * 32 + tx;
  const int64_t t0 = (int64_t)bx * kTB;
  __int128 acc = 0;
  if (slot < nd) {
    const int j = __ldcg(dlist + slot);
    const int64_t tend = min(d, t0 + kTB);
    int64_t t = t0 + ty;
    // eight loads in flight
    for (; t + 56 < tend; t += 64) {
      long long raw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) raw[u] = S64[(t + 8 * u) * kst + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += (__int128)raw[u] * raw[u];
    }
    for (; t < tend; t += 8) {
      const long long v = S64[t * kst + j];
      acc += (__int128)v * v;
    }
  }
  sh[0][ty][tx] = (long long)acc;
  sh[1][ty][tx] = (long long)(acc >> 64);
  __syncthreads();
  if (ty == 0 && slot < nd) {
    __int128 r = 0;
    for (int y = 0; y < 8; ++y) r += (((__int128)sh[1][y][tx]) << 64) | (unsigned long long)sh[0][y][tx];
    long long* red64 = reinterpret_cast<long long*>(red);
    red64[((int64_t)bx * kst + slot) * 2] = (long long)r;
    red64[((int64_t)bx * kst + slot) * 2 + 1] = (long long)(r >> 64);
  }
  __syncthreads();
}

// grid (ceil(d/kTB), ceil(k/32)), block 256.
__global__ void __launch_bounds__(256) k_colnorm_part(const long long* __restrict__ S64, int64_t d, int64_t kst,
                                                      const int32_t* __restrict__ dlist,
                                                      const unsigned long long* __restrict__ cnt,
                                                      double* __restrict__ red, int s64_valid, int64_t n) {
  __shared__ long long sh[2][8][33];
  const int nd = (int)cnt[C_NDIRTY];
  if ((int)(blockIdx.y * 32) >= nd) return;
  dev_colnorm_part(S64, d, kst, dlist, nd, red, blockIdx.x, blockIdx.y, sh, full_update(s64_valid, cnt, n));
}

// Dirty slot `slot`: |S_j|^2 exactly -- after a full recomputation the sum
// of the per-tile partials (by the block's first 128 threads; integer sums,
// so their order does not matter), else the value the incremental update
// kept in the limbs -- stored back as limbs in range, and |S_j| = sqrt of it
// times the fixed-point scale inv.  sh: shared long long[256].
__device__ __forceinline__ void dev_colnorm_final(const double* __restrict__ red, int64_t nblk, int64_t kst,
                                                  const int32_t* __restrict__ dlist, int slot,
                                                  double* __restrict__ nrm, long long* sh, long long* __restrict__ n2l,
                                                  bool full, float inv) {
  const int j = __ldcg(dlist + slot);
  __int128 v = 0;
  if (full) {
    const long long* red64 = reinterpret_cast<const long long*>(red);
    const bool on = threadIdx.x < 128;
    __int128 s = 0;
    if (on)
      for (int64_t b = threadIdx.x; b < nblk; b += 128)
        s += (((__int128)__ldcg(red64 + (b * kst + slot) * 2 + 1)) << 64) |
             (unsigned long long)__ldcg(red64 + (b * kst + slot) * 2);
    if (on) {
      sh[threadIdx.x] = (long long)s;
      sh[128 + threadIdx.x] = (long long)(s >> 64);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < 128; ++q) v += (((__int128)sh[128 + q]) << 64) | (unsigned long long)sh[q];
  } else if (threadIdx.x == 0) {
    v = n2_get(n2l, kst, j);
  }
  if (threadIdx.x == 0) {
    n2_set(n2l, kst, j, v);
    nrm[j] = sqrt((double)v) * (double)inv;
  }
  __syncthreads();
}

// Block per dirty slot.
__global__ void __launch_bounds__(128) k_colnorm_final(const double* __restrict__ red, int64_t nblk, int64_t kst,
                                                       const int32_t* __restrict__ dlist,
                                                       const unsigned long long* __restrict__ cnt,
                                                       double* __restrict__ nrm, long long* __restrict__ n2l,
                                                       int s64_valid, int64_t n, float inv) {
  __shared__ long long sh[256];
  if ((int)blockIdx.x >= (int)cnt[C_NDIRTY]) return;
  dev_colnorm_final(red, nblk, kst, dlist, blockIdx.x, nrm, sh, n2l, full_update(s64_valid, cnt, n), inv);
}

// Tile (bx, by), threads as dev_colnorm_part.  The dirty centers are
// overwritten in place; red2 receives per tile and slot sum c^2, sum c'^2 and
// sum (c - c')^2 (FP32 per thread over 32 terms -- relative error <= 36u,
// covered by the slack of dev_drift_final).  With Ct16 (screened contexts)
// the new values are also written rounded to FP16, and e2p receives per tile
// and slot the FP64 sum of the squared rounding errors (each difference is
// exact in FP32, its square exact in FP64).  sh: shared double[4][8][33].
__device__ __forceinline__ void dev_normalize_drift(const long long* __restrict__ S64, float inv,
                                                    float* __restrict__ Ct, const double* __restrict__ nrm,
                                                    int64_t d, int64_t kst, const int32_t* __restrict__ dlist,
                                                    int nd, double* __restrict__ red2, int bx, int by,
                                                    double (*sh)[8][33], __half* __restrict__ Ct16,
                                                    double* __restrict__ e2p) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int slot = by * 32 + tx;
  const int64_t t0 = (int64_t)bx * kTB;
  float sn = 0.f, so = 0.f, sd = 0.f;
  double se = 0.0;
  if (slot < nd) {
    const int j = __ldcg(dlist + slot);
    const double nr = __ldcg(nrm + j);
    const bool empty = !(nr > 0.0);
    const float rn = empty ? 0.f : (float)(1.0 / nr);
    const int64_t tend = min(d, t0 + kTB);
    auto step = [&](int64_t t, float co, long long raw) {
      const float cn = empty ? co : __fmul_rn(from_fixed(raw, inv), rn);
      Ct[t * kst + j] = cn;
      if (Ct16) {
        const __half h = __float2half_rn(cn);
        Ct16[t * kst + j] = h;
        const double er = (double)__fsub_rn(cn, __half2float(h));  // exact
        se += er * er;
      }
      const float df = cn - co;
      sn = __fmaf_rn(cn, cn, sn);
      so = __fmaf_rn(co, co, so);
      sd = __fmaf_rn(df, df, sd);
    };
    int64_t t = t0 + ty;
    // eight terms' loads in flight, then the updates in the same order
    for (; t + 56 < tend; t += 64) {
      float co[8];
      long long raw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        co[u] = Ct[(t + 8 * u) * kst + j];
        raw[u] = S64[(t + 8 * u) * kst + j];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) step(t + 8 * u, co[u], raw[u]);
    }
    for (; t < tend; t += 8) step(t, Ct[t * kst + j], S64[t * kst + j]);
  }
  sh[0][ty][tx] = sn;
  sh[1][ty][tx] = so;
  sh[2][ty][tx] = sd;
  sh[3][ty][tx] = se;
  __syncthreads();
  if (ty == 0 && slot < nd) {
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
    for (int y = 0; y < 8; ++y) {
      r0 += sh[0][y][tx];
      r1 += sh[1][y][tx];
      r2 += sh[2][y][tx];
      r3 += sh[3][y][tx];
    }
    double* o = red2 + ((int64_t)bx * kst + slot) * 3;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    if (Ct16) e2p[(int64_t)bx * kst + slot] = r3;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_normalize_drift(const long long* __restrict__ S64, float inv,
                                                         float* __restrict__ Ct, const double* __restrict__ nrm,
                                                         int64_t d, int64_t kst, const int32_t* __restrict__ dlist,
                                                         const unsigned long long* __restrict__ cnt,
                                                         double* __restrict__ red2, __half* __restrict__ Ct16,
                                                         double* __restrict__ e2p) {
  __shared__ double sh[4][8][33];
  const int nd = (int)cnt[C_NDIRTY];
  if ((int)(blockIdx.y * 32) >= nd) return;
  dev_normalize_drift(S64, inv, Ct, nrm, d, kst, dlist, nd, red2, blockIdx.x, blockIdx.y, sh, Ct16, e2p);
}

// Center j (the block's first 128 threads).  Clean centers did not move:
// p = 1, sine 0.  Dirty ones: from N = |c|, N' = |c'| and D = |c - c'|^2
// (relative error <= e, e = 40u + d 2^-53):  1 - cos = (D - (N - N')^2) /
// (2 N N'), hence
//   q_up = D (1+4e) / (2 N N')                           >= 1 - cos
//   q_dn = (D (1-e) - (|N-N'| + e)^2) / (2 N N' (1+3e))  <= 1 - cos
// pd = rd(1 - q_up), pu = ru(1 - q_dn), q = ru(max sin over [q_dn, q_up]).
// sh: shared double[3][128].
// With e2c (screened contexts) also e2c[j] = the sum of the FP16 error
// partials of the moved center (fixed order); clean centers keep theirs.
// sh: shared double[4][128].
__device__ __forceinline__ void dev_drift_final(const double* __restrict__ red2, int64_t nblk, int32_t k,
                                                int64_t kst, int64_t d, const int32_t* __restrict__ dmark,
                                                const int32_t* __restrict__ dpos, float* __restrict__ pdn,
                                                float* __restrict__ pup, float* __restrict__ qup,
                                                double* __restrict__ cnorm, int j, double (*sh)[128],
                                                const double* __restrict__ e2p, double* __restrict__ e2c) {
  if (j >= k || !__ldcg(dmark + j)) {
    if (threadIdx.x == 0) {
      pdn[j] = 1.f;
      pup[j] = 1.f;
      qup[j] = 0.f;
    }
    return;  // the same for the whole block
  }
  const bool on = threadIdx.x < 128;
  const int slot = __ldcg(dpos + j);
  double sn = 0.0, so = 0.0, sd = 0.0, se = 0.0;
  if (on)
    for (int64_t b = threadIdx.x; b < nblk; b += 128) {
      const double* r = red2 + (b * kst + slot) * 3;
      sn += __ldcg(r);
      so += __ldcg(r + 1);
      sd += __ldcg(r + 2);
      if (e2c) se += __ldcg(e2p + b * kst + slot);
    }
  if (on) {
    sh[0][threadIdx.x] = sn;
    sh[1][threadIdx.x] = so;
    sh[2][threadIdx.x] = sd;
    sh[3][threadIdx.x] = se;
  }
  __syncthreads();
  for (int o = 64; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
      sh[3][threadIdx.x] += sh[3][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (e2c) e2c[j] = sh[3][0];
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
  __syncthreads();
}

// One block: the objective J = sum_j |S_j| (fixed order) and Hamerly's
// worst-drift summary -- argmin / min / second min of pd and of pu, argmax /
// max / second max of q, lowest index on ties (Section 5.3: p' is the minimum
// over the other centers, hence the second value for the argmin's members).
// Also zeroes the assignment counters for the next assignment: the last
// reader of them (the update) is done.
// With e2c (screened contexts): escr = E >= max_j |fp16(c_j) - c_j| (the FP64
// sums carry a relative error below 10^-9, covered by the slack).
__device__ __forceinline__ void dev_fp16_err_max(const double* __restrict__ e2c, int32_t k, float* __restrict__ escr,
                                                 double* sh /* >= blockDim.x doubles */) {
  double m = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) m = fmax(m, __ldcg(e2c + j));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) escr[0] = __double2float_ru(sqrt(sh[0] * (1.0 + 1e-9)) * (1.0 + 1e-15));
  __syncthreads();
}

// dev_hsel_obj_256 (a 256-thread block) computes it: 256 slots for the minima
// and maxima (which do not depend on the order they are combined in: values,
// then the lowest index on ties) and 1024 slots for J (slot v sums centers
// v, v + 1024, ...; then a fixed tree).
struct HselSmall {
  float pd[256], pu[256], q[256], pd2[256], pu2[256], q2[256];
  int jd[256], ju[256], jq[256];
  double J[1024];
};
__device__ __forceinline__ void dev_hsel_obj_256(const float* __restrict__ pdn, const float* __restrict__ pup,
                                                 const float* __restrict__ qup, const double* __restrict__ nrm,
                                                 int32_t k, float* __restrict__ hsel, double* __restrict__ obj,
                                                 unsigned long long* __restrict__ cnt, HselSmall& S,
                                                 const double* __restrict__ e2c, float* __restrict__ escr) {
  if (threadIdx.x < C_ERR) cnt[threadIdx.x] = 0ull;
  const int tid = threadIdx.x;
  float bd = FLT_MAX, bd2 = FLT_MAX, bu = FLT_MAX, bu2 = FLT_MAX, bq = -FLT_MAX, bq2 = -FLT_MAX;
  int jd = INT_MAX, ju = INT_MAX, jq = INT_MAX;
  for (int j = tid; j < k; j += 256) {
    const float x = __ldcg(pdn + j), y = __ldcg(pup + j), z = __ldcg(qup + j);
    if (x < bd) { bd2 = bd; bd = x; jd = j; } else if (x < bd2) bd2 = x;
    if (y < bu) { bu2 = bu; bu = y; ju = j; } else if (y < bu2) bu2 = y;
    if (z > bq) { bq2 = bq; bq = z; jq = j; } else if (z > bq2) bq2 = z;
  }
  S.pd[tid] = bd; S.pd2[tid] = bd2; S.jd[tid] = jd;
  S.pu[tid] = bu; S.pu2[tid] = bu2; S.ju[tid] = ju;
  S.q[tid] = bq; S.q2[tid] = bq2; S.jq[tid] = jq;
  for (int v = tid; v < 1024; v += 256) {
    double J = 0.0;
    for (int j = v; j < k; j += 1024) J += __ldcg(nrm + j);
    S.J[v] = J;
  }
  __syncthreads();
  for (int o = 512; o; o >>= 1) {
    for (int a = tid; a < o; a += 256) S.J[a] += S.J[a + o];
    if (o < 256 && tid < o) {
      const int a = tid, b = tid + o;
      if (S.pd[b] < S.pd[a] || (S.pd[b] == S.pd[a] && S.jd[b] < S.jd[a])) {
        S.pd2[a] = fminf(S.pd2[b], S.pd[a]);
        S.pd[a] = S.pd[b];
        S.jd[a] = S.jd[b];
      } else {
        S.pd2[a] = fminf(S.pd2[a], S.pd[b]);
      }
      if (S.pu[b] < S.pu[a] || (S.pu[b] == S.pu[a] && S.ju[b] < S.ju[a])) {
        S.pu2[a] = fminf(S.pu2[b], S.pu[a]);
        S.pu[a] = S.pu[b];
        S.ju[a] = S.ju[b];
      } else {
        S.pu2[a] = fminf(S.pu2[a], S.pu[b]);
      }
      if (S.q[b] > S.q[a] || (S.q[b] == S.q[a] && S.jq[b] < S.jq[a])) {
        S.q2[a] = fmaxf(S.q2[b], S.q[a]);
        S.q[a] = S.q[b];
        S.jq[a] = S.jq[b];
      } else {
        S.q2[a] = fmaxf(S.q2[a], S.q[b]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const bool one = (k == 1);
    hsel[0] = (float)S.jd[0];
    hsel[1] = S.pd[0];
    hsel[2] = one ? 1.f : S.pd2[0];
    hsel[3] = (float)S.ju[0];
    hsel[4] = S.pu[0];
    hsel[5] = one ? 1.f : S.pu2[0];
    hsel[6] = (float)S.jq[0];
    hsel[7] = S.q[0];
    hsel[8] = one ? 0.f : S.q2[0];
    obj[0] = S.J[0];
  }
  __syncthreads();
  if (e2c) dev_fp16_err_max(e2c, k, escr, S.J);
}

// The drift per center and the summary in one launch: block per center (grid
// kst, 256 threads) for the drift, then the last block to finish writes J and
// Hamerly's summary (dev_hsel_obj_256).  done: a counter
// that only grows, so launches and graph replays need no reset.
__global__ void __launch_bounds__(256) k_drift_hsel(const double* __restrict__ red2, int64_t nblk, int32_t k,
                                                    int64_t kst, int64_t d, const int32_t* __restrict__ dmark,
                                                    const int32_t* __restrict__ dpos, float* __restrict__ pdn,
                                                    float* __restrict__ pup, float* __restrict__ qup,
                                                    double* __restrict__ cnorm, const double* __restrict__ e2p,
                                                    double* __restrict__ e2c, const double* __restrict__ nrm,
                                                    float* __restrict__ hsel, double* __restrict__ obj,
                                                    unsigned long long* __restrict__ cnt, float* __restrict__ escr,
                                                    unsigned long long* __restrict__ done) {
  __shared__ union {
    double fin[4][128];
    HselSmall hs;
  } sm;
  __shared__ int last_sh;
  dev_drift_final(red2, nblk, k, kst, d, dmark, dpos, pdn, pup, qup, cnorm, blockIdx.x, sm.fin, e2p, e2c);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long v = atomicAdd(done, 1ull);
    last_sh = (v % gridDim.x) == gridDim.x - 1;
    __threadfence();
  }
  __syncthreads();
  if (last_sh) dev_hsel_obj_256(pdn, pup, qup, nrm, k, hsel, obj, cnt, sm.hs, e2c, escr);
}

// ------------------------------------------------------------------
// All the phases above in one cooperative launch (every block resident at
// once, so blocks may wait on one another), with grid barriers between the
// phases that read what the previous one wrote:
//   block 0: dirty list | tiles: partial norms | dirty slots: norms |
//   tiles: normalise + drift partials | centers: drift | last block: J and
//   Hamerly's summary.
// Each barrier waits on a 64-bit counter that only grows (kFinishBars
// arrivals per block per launch), so no reset is needed between launches or
// graph replays: a block finds its launch's base by rounding the counter it
// reads at the start down to a multiple of kFinishBars * gridDim.x (no block
// can pass the first barrier before every block has started).  Every wait
// gives up after one second, raises E_TIMEOUT and the blocks leave.
constexpr int kFinishBars = 4;
constexpr uint64_t kFinishTimeoutNs = 1000000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier number `which` (1-based) of this launch; false if the wait gave up.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long base, int which,
                                             unsigned long long* __restrict__ cnt, int* ok_sh,
                                             uint64_t timeout_ns = kFinishTimeoutNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1ull);
    const unsigned long long target = base + (unsigned long long)which * gridDim.x;
    const uint64_t t0 = globaltimer_ns();
    int ok = 1;
    while (*reinterpret_cast<volatile unsigned long long*>(bar) < target) {
      if (globaltimer_ns() - t0 > timeout_ns) {
        ok = 0;
        atomicOr(cnt + C_ERR, (unsigned long long)E_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

// Self-test of the barrier's failure path: two cooperative blocks, block 1
// never arrives, so block 0's wait must give up after timeout_ns and raise
// E_TIMEOUT in flag[C_ERR].
__global__ void k_barrier_selftest(unsigned long long* bar, uint64_t timeout_ns, unsigned long long* flag) {
  __shared__ int ok_sh;
  if (blockIdx.x != 0) return;
  (void)grid_barrier(bar, 0, 1, flag, &ok_sh, timeout_ns);
}

__global__ void __launch_bounds__(256) k_finish_fused(int32_t k, int64_t kst, int64_t d, int64_t nblk, float inv,
                                                      int s64_valid, int64_t n, int32_t* __restrict__ dflag,
                                                      int32_t* __restrict__ dmark, int32_t* __restrict__ dpos,
                                                      int32_t* __restrict__ dlist, const long long* __restrict__ S64,
                                                      float* __restrict__ Ct, double* __restrict__ nrm,
                                                      double* __restrict__ red, float* __restrict__ pdn,
                                                      float* __restrict__ pup, float* __restrict__ qup,
                                                      double* __restrict__ cnorm, float* __restrict__ hsel,
                                                      double* __restrict__ obj, unsigned long long* __restrict__ cnt,
                                                      unsigned long long* __restrict__ bar, __half* __restrict__ Ct16,
                                                      double* __restrict__ e2p, double* __restrict__ e2c,
                                                      float* __restrict__ escr, long long* __restrict__ n2l) {
  __shared__ union {
    long long cn[2][8][33];
    long long cf[256];
    double part[4][8][33];
    double fin[4][128];
    HselSmall hs;
  } sm;
  __shared__ int wsum[8];
  __shared__ int base_sh, ok_sh, last_sh;
  __shared__ unsigned long long bar0_sh;
  if (threadIdx.x == 0) {
    const unsigned long long per = (unsigned long long)kFinishBars * gridDim.x;
    const unsigned long long v = *reinterpret_cast<volatile unsigned long long*>(bar);
    bar0_sh = v - v % per;
  }
  __syncthreads();
  const unsigned long long b0 = bar0_sh;
  const bool full = full_update(s64_valid, cnt, n);
  if (blockIdx.x == 0) dev_dirty(k, dflag, dmark, dpos, dlist, cnt, full, wsum, &base_sh);
  if (!grid_barrier(bar, b0, 1, cnt, &ok_sh)) return;
  const int nd = (int)__ldcg(cnt + C_NDIRTY);
  const int ngroups = (nd + 31) / 32;
  const int64_t ntile = nblk * ngroups;
  for (int64_t w = blockIdx.x; w < ntile; w += gridDim.x)
    dev_colnorm_part(S64, d, kst, dlist, nd, red, (int)(w % nblk), (int)(w / nblk), sm.cn, full);
  if (!grid_barrier(bar, b0, 2, cnt, &ok_sh)) return;
  for (int slot = blockIdx.x; slot < nd; slot += gridDim.x)
    dev_colnorm_final(red, nblk, kst, dlist, slot, nrm, sm.cf, n2l, full, inv);
  if (!grid_barrier(bar, b0, 3, cnt, &ok_sh)) return;
  for (int64_t w = blockIdx.x; w < ntile; w += gridDim.x)
    dev_normalize_drift(S64, inv, Ct, nrm, d, kst, dlist, nd, red, (int)(w % nblk), (int)(w / nblk), sm.part, Ct16,
                        e2p);
  if (!grid_barrier(bar, b0, 4, cnt, &ok_sh)) return;
  for (int64_t j = blockIdx.x; j < kst; j += gridDim.x)
    dev_drift_final(red, nblk, k, kst, d, dmark, dpos, pdn, pup, qup, cnorm, (int)j, sm.fin, e2p, e2c);
  // the last block to get here writes J and Hamerly's summary
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long v = atomicAdd(bar + 1, 1ull);
    last_sh = (v % gridDim.x) == gridDim.x - 1;
    __threadfence();
  }
  __syncthreads();
  if (last_sh) dev_hsel_obj_256(pdn, pup, qup, nrm, k, hsel, obj, cnt, sm.hs, e2c, escr);
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
// koff .. koff + k - 1 (global ids), the rule of dev_hsel_obj_256.
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
      c->s64_valid, c->cnt, c->n, c->n2l);
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

int barrier_selftest(int64_t timeout_ns, cudaStream_t st) {
  unsigned long long* buf = nullptr;  // [0] the barrier counter, [1 + C_ERR] the error word
  SKM_CUDA_TRY(cudaMallocAsync((void**)&buf, sizeof(unsigned long long) * (2 + C_NUM), st));
  SKM_CUDA_TRY(cudaMemsetAsync(buf, 0, sizeof(unsigned long long) * (2 + C_NUM), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SKM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_barrier_selftest, buf, (uint64_t)timeout_ns, buf + 1));
  note_launch();
  unsigned long long h = 0;
  SKM_CUDA_TRY(cudaMemcpyAsync(&h, buf + 1 + C_ERR, sizeof(h), cudaMemcpyDeviceToHost, st));
  SKM_CUDA_TRY(cudaFreeAsync(buf, st));
  SKM_CUDA_TRY(cudaStreamSynchronize(st));
  return (h & E_TIMEOUT) ? SKM_ETIMEOUT : SKM_OK;
}

// Screened contexts, after Ct was set outside a center update (initial rows,
// skm_set_centers): the FP16 copy of every center and its rounding error.
// Tile (blockIdx.x: 256 terms, blockIdx.y: 32 centers), threads as
// dev_colnorm_part; e2p gets the per-tile sums, then k_ct16_final sums them
// per center in a fixed order and takes the maximum.
__global__ void __launch_bounds__(256) k_ct16_part(const float* __restrict__ Ct, int64_t d, int64_t kst,
                                                   __half* __restrict__ Ct16, double* __restrict__ e2p) {
  __shared__ double sh[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.y * 32 + tx;
  const int64_t t0 = (int64_t)blockIdx.x * kTB;
  double se = 0.0;
  if (j < kst)
    for (int64_t t = t0 + ty; t < min(d, t0 + kTB); t += 8) {
      const float c = Ct[t * kst + j];
      const __half h = __float2half_rn(c);
      Ct16[t * kst + j] = h;
      const double er = (double)__fsub_rn(c, __half2float(h));  // exact
      se += er * er;
    }
  sh[ty][tx] = se;
  __syncthreads();
  if (ty == 0 && j < kst) {
    double r = 0.0;
    for (int y = 0; y < 8; ++y) r += sh[y][tx];
    e2p[(int64_t)blockIdx.x * kst + j] = r;
  }
}

__global__ void __launch_bounds__(1024) k_ct16_final(const double* __restrict__ e2p, int64_t nblk, int32_t k,
                                                     int64_t kst, double* __restrict__ e2c, float* __restrict__ escr) {
  __shared__ double sh[1024];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int64_t b = 0; b < nblk; ++b) s += e2p[b * kst + j];
    e2c[j] = s;
  }
  __syncthreads();
  dev_fp16_err_max(e2c, k, escr, sh);
}

// Blocks of the fused finishing kernel: enough for its largest phase, at most
// what is resident at once (its blocks wait on one another); 0 if it is not
// asked for (opt.fused_update; on the RCV-1-like workload its four grid
// barriers and serial dirty-list phase cost more than the launch gaps of the
// separate kernels save: 2251 vs 2331 iterations/s) or this device cannot
// launch cooperative kernels.
int finish_fused_grid(const skm_ctx* c) {
  if (!c->opt.fused_update) return 0;
  static int per_sm = -1, coop = -1;
  if (per_sm < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      v = 0;
    coop = v;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_finish_fused, 256, 0) != cudaSuccess) nb = 0;
    (void)cudaGetLastError();
    per_sm = nb;
  }
  if (!coop || per_sm < 1 || !c->fbar) return 0;
  const int64_t want = reduction_blocks(c->d) * ((c->kst + 31) / 32);
  int64_t g = (int64_t)c->nsm * per_sm;
  if (want < g) g = want;
  return (int)(g < 1 ? 1 : g);
}

int ct16_all(skm_ctx* c) {
  if (!c->Ct16) return SKM_OK;
  const int64_t nblk = reduction_blocks(c->d);
  dim3 grid((unsigned)nblk, (unsigned)((c->kst + 31) / 32));
  SKM_PROF_BEGIN(c, "k_ct16_part");
  k_ct16_part<<<grid, 256, 0, c->st>>>(c->Ct, c->d, c->kst, c->Ct16, c->e2p);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_ct16_final");
  k_ct16_final<<<1, 1024, 0, c->st>>>(c->e2p, nblk, c->k, c->kst, c->e2c, c->escr);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

// Dirty list, norms, new centers, drift and (full variants) the center-center
// bounds, shared by the sparse and dense paths.
int finish_update(skm_ctx* c) {
  const int k = c->k;
  const int64_t nblk = reduction_blocks(c->d);
  double* cnorm = c->nrm + c->kst;  // second half of the norm buffer: |c(j)| of the centers
  const int s64_was_valid = c->s64_valid;
  c->s64_valid = 1;
  const int fg = finish_fused_grid(c);
  if (fg > 0) {
    // ---- dirty list, norms, new centers, drift, J and Hamerly's summary: one cooperative launch
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)fg);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SKM_PROF_BEGIN(c, "k_finish_fused");
    SKM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_finish_fused, k, (int64_t)c->kst, c->d, nblk, c->fx_inv, s64_was_valid,
                                    c->n, c->dflag, c->dmark, c->dpos, c->dlist, (const long long*)c->S64, c->Ct,
                                    c->nrm, c->red, c->pdn, c->pup, c->qup, cnorm, c->hsel, c->obj, c->cnt,
                                    c->fbar, c->Ct16, c->e2p, c->e2c, c->escr, c->n2l));
    SKM_LAUNCHED(c);
  } else {
    SKM_PROF_BEGIN(c, "k_dirty");
    k_dirty<<<1, 1024, 0, c->st>>>(k, c->dflag, c->dmark, c->dpos, c->dlist, c->cnt, s64_was_valid, c->n);
    SKM_LAUNCHED(c);
    // ---- norms, new centers and drift of the dirty clusters
    dim3 grid((unsigned)nblk, (unsigned)((k + 31) / 32));
    SKM_PROF_BEGIN(c, "k_colnorm_part");
    k_colnorm_part<<<grid, 256, 0, c->st>>>(c->S64, c->d, c->kst, c->dlist, c->cnt, c->red, s64_was_valid, c->n);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_colnorm_final");
    k_colnorm_final<<<k, 128, 0, c->st>>>(c->red, nblk, c->kst, c->dlist, c->cnt, c->nrm, c->n2l, s64_was_valid,
                                          c->n, c->fx_inv);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_normalize_drift");
    k_normalize_drift<<<grid, 256, 0, c->st>>>(c->S64, c->fx_inv, c->Ct, c->nrm, c->d, c->kst, c->dlist, c->cnt,
                                               c->red, c->Ct16, c->e2p);
    SKM_LAUNCHED(c);
    SKM_PROF_BEGIN(c, "k_drift_hsel");
    k_drift_hsel<<<c->kst, 256, 0, c->st>>>(c->red, nblk, k, c->kst, c->d, c->dmark, c->dpos, c->pdn, c->pup,
                                            c->qup, cnorm, c->e2p, c->e2c, c->nrm, c->hsel, c->obj, c->cnt, c->escr,
                                            c->fbar + 2);
    SKM_LAUNCHED(c);
  }
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
