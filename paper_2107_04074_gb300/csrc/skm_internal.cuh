// Internal declarations of libskm: the context, device helpers shared by the
// kernels, and the host-side launch wrappers each kernel file exports.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/skm.h"

#define SKM_FULL_MASK 0xffffffffu

namespace skm {

// ---------------------------------------------------------------- counters
// Device counters of one assignment (reset at its start).
enum Counter {
  C_CHANGED = 0,  // labels changed
  C_SIMS = 1,     // exact similarities computed
  C_W1 = 2,       // points failing the first bound test
  C_W2 = 3,       // points needing a full row of similarities
  C_CHG = 4,      // entries of the changed-row list
  C_W3 = 5,       // dense precision form: rows rechecked against a few candidates
  C_W1L = 6,      // Elkan: survivors with long rows (kept at the top of w1)
  C_CURSOR = 7,   // next work item of k_rows_top2 (dynamic scheduling)
  C_CURSOR_R = 8,  // ... of k_elk_recompute
  C_CURSOR_L = 9,  // ... of k_elk_recompute_long
  C_W3S = 10,     // screened whole rows left open, short rows (pair recompute, from the bottom of w3)
  C_W3L = 11,     // ... long rows (from the top of w3)
  C_W4 = 12,      // rows for an exact FP32 whole-row pass after the screened one
  C_CURSOR_2 = 13,   // cursors of the second launches of an assignment: k_rows_top2,
  C_CURSOR_R2 = 14,  // k_elk_recompute,
  C_CURSOR_L2 = 15,  // k_elk_recompute_long
  C_SKIP = 16,    // 1: this assignment skipped Elkan's bound pass or Hamerly's tightening
  C_ERR = 17,     // error flags (bit field)
  C_NDIRTY = 18,  // clusters whose sum changed in the last center update
  C_NUM = 19
};

// Data-preparation error bits (C_ERR).
enum ErrBits { E_COLIDX = 1, E_ORDER = 2, E_ZERO_ROW = 4, E_NONFINITE = 8, E_ROWPTR = 16, E_TIMEOUT = 32 };

// Hamerly drift summary (Section 5.3): for the worst-moving center over all
// j != a(i) we keep, for "a(i) is the argmin/argmax" and "it is not":
//   [0] argmin p_dn   [1] min p_dn    [2] second min p_dn
//   [3] argmin p_up   [4] min p_up    [5] second min p_up
//   [6] argmax q_up   [7] max q_up    [8] second max q_up
constexpr int HSEL_N = 9;

// --------------------------------------------------------------- helpers
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Canonical similarity of row i to center j: sequential FMA over the row's
// stored entries in CSR order, starting from 0, then times 1/|x_i|.  Every
// kernel that produces a similarity uses exactly this order, so all variants
// see bit-identical values and take identical decisions.  Eight entries are
// loaded (and their center values gathered) before they are accumulated, to
// keep several loads in flight; the accumulation order is unchanged.
template <typename VT>
__device__ __forceinline__ float dot_row_center(int64_t b, int64_t e, const int32_t* __restrict__ col,
                                                const VT* __restrict__ val, const float* __restrict__ Ct,
                                                int64_t kst, int j) {
  float acc = 0.f;
  int64_t p = b;
  for (; p + 8 <= e; p += 8) {
    int t[8];
    float v[8], c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      t[u] = __ldg(col + p + u);
      v[u] = to_f32(val[p + u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = __ldg(Ct + (int64_t)t[u] * kst + j);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = __fmaf_rn(v[u], c[u], acc);
  }
  for (; p < e; ++p) acc = __fmaf_rn(to_f32(val[p]), __ldg(Ct + (int64_t)__ldg(col + p) * kst + j), acc);
  return acc;
}

// Warp-cooperative canonical similarity to ONE center j (all lanes return
// it): the warp loads 32 entries and their center values at once, then runs
// the sequential FMA chain over them through shuffles.  The next chunk's
// loads are issued before the current chunk is accumulated.
template <typename VT>
__device__ __forceinline__ float warp_dot_one(int64_t b, int64_t e, const int32_t* __restrict__ col,
                                              const VT* __restrict__ val, const float* __restrict__ Ct, int64_t kst,
                                              int j) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  float v = 0.f, c = 0.f;
  if (b + lane < e) {
    v = to_f32(val[b + lane]);
    c = __ldg(Ct + (int64_t)__ldg(col + b + lane) * kst + j);
  }
  for (int64_t p0 = b; p0 < e; p0 += 32) {
    const float cv = v, cc = c;
    const int64_t pn = p0 + 32 + lane;
    if (pn < e) {
      v = to_f32(val[pn]);
      c = __ldg(Ct + (int64_t)__ldg(col + pn) * kst + j);
    }
    const int nq = (int)min((int64_t)32, e - p0);
    for (int q = 0; q < nq; ++q)
      acc = __fmaf_rn(__shfl_sync(SKM_FULL_MASK, cv, q), __shfl_sync(SKM_FULL_MASK, cc, q), acc);
  }
  return acc;
}

// Warp-cooperative canonical similarities to one center PER LANE (my_j < 0:
// the lane computes nothing useful).  Row entries are broadcast by shuffles
// in CSR order; for each chunk of 32 entries every lane first gathers all its
// center values (one round trip), then accumulates them in order.
template <typename VT>
__device__ __forceinline__ float warp_dot_lanes(int64_t b, int64_t e, const int32_t* __restrict__ col,
                                                const VT* __restrict__ val, const float* __restrict__ Ct,
                                                int64_t kst, int my_j) {
  const int lane = threadIdx.x & 31;
  const bool on = my_j >= 0;
  const float* cbase = Ct + (on ? my_j : 0);
  float acc = 0.f;
  int tt = 0;
  float vv = 0.f;
  if (b + lane < e) {
    tt = __ldg(col + b + lane);
    vv = to_f32(val[b + lane]);
  }
  for (int64_t p0 = b; p0 < e; p0 += 32) {
    const int ct = tt;
    const float cv = vv;
    const int64_t pn = p0 + 32 + lane;
    if (pn < e) {
      tt = __ldg(col + pn);
      vv = to_f32(val[pn]);
    }
    const int nq = (int)min((int64_t)32, e - p0);
    if (nq == 32) {
      float c[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int t = __shfl_sync(SKM_FULL_MASK, ct, q);
        c[q] = on ? __ldg(cbase + (int64_t)t * kst) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) acc = __fmaf_rn(__shfl_sync(SKM_FULL_MASK, cv, q), c[q], acc);
    } else {
      for (int q = 0; q < nq; ++q) {
        const int t = __shfl_sync(SKM_FULL_MASK, ct, q);
        const float v = __shfl_sync(SKM_FULL_MASK, cv, q);
        acc = __fmaf_rn(v, on ? __ldg(cbase + (int64_t)t * kst) : 0.f, acc);
      }
    }
  }
  return acc;
}

// Precision form: bound on |BF16 tensor-core similarity - exact similarity|
// for row i against every center, eps_i = ex_i (1 + 6u + E_c) + E_c + acc
// (rounded up), from the row's and the centers' rounding errors as vectors
// (Cauchy-Schwarz); ebc holds the two per-iteration terms.
__device__ __forceinline__ float bf16_eps(const float* __restrict__ exr, const float* __restrict__ ebc, int64_t i) {
  return __fmaf_ru(exr[i], ebc[0], ebc[1]);
}

// Eq. (eqn:l-bound) with the clamp of the angle triangle inequality, in FP32
// rounded towards -inf.  The drift of the center is an interval: its cosine p
// lies in [pd, pu] and its sine is at most q.
__device__ __forceinline__ float bound_l(float l, float pd, float pu, float q) {
  if (l < -pd) return -1.f;  // arccos l + arccos p may exceed pi
  const float lp = (l >= 0.f) ? __fmul_rd(l, pd) : __fmul_rd(l, pu);
  const float om = __fmul_ru(__fsub_ru(1.f, l), __fadd_ru(1.f, l));
  const float v = __fsub_rd(lp, __fmul_ru(__fsqrt_ru(om), q));
  return fmaxf(v, -1.f);
}

// Eq. (eqn:u-elkan) with the clamp, rounded towards +inf.
__device__ __forceinline__ float bound_u(float u, float pd, float pu, float q) {
  if (u > pd) return 1.f;  // arccos u may be below arccos p: the angle can close
  const float up = (u >= 0.f) ? __fmul_ru(u, pu) : __fmul_ru(u, pd);
  const float om = __fmul_ru(__fsub_ru(1.f, u), __fadd_ru(1.f, u));
  const float v = __fadd_ru(up, __fmul_ru(__fsqrt_ru(om), q));
  return fminf(v, 1.f);
}

// Hamerly's single upper bound, Eq. (eqn:u-hamerly-2), used when u >= 0 and
// every other center moved by at most 90 degrees; otherwise (or when tight)
// the clamped single-center form with the worst drift p' = min_{j != a} p(j).
__device__ __forceinline__ float bound_u_hamerly(float u, float pd_min, float pu_min, float q_max, int tight) {
  if (!tight && u >= 0.f && pd_min >= 0.f) {
    const float om = __fmul_ru(__fsub_ru(1.f, u), __fadd_ru(1.f, u));
    return fminf(__fadd_ru(u, __fmul_ru(__fsqrt_ru(om), q_max)), 1.f);
  }
  return bound_u(u, pd_min, pu_min, q_max);
}

// ---- squared norms of the sums, exactly
// S64 holds fixed-point values S = x 2^s with the scale chosen so that the
// squared norm of a cluster's column, at most (n_j 2^s)^2 < 2^124, fits an
// __int128, as does every partial sum of it: the squared norm is an integer
// computed exactly, whatever the order of the additions.  The full
// recomputation sums the squares of the dirty columns (the colnorm pass);
// the incremental update adds, for every entry a moved row touches, the
// change of its square, (S + x)^2 - S^2 = 2 S x + x^2 from the value S its
// atomic add replaced (these changes telescope to the exact new value, in
// any order of the atomics).  Both give the same bits.  A cluster's running
// value is kept as three limbs, n2l[j] + n2l[kst + j] 2^42 + n2l[2 kst + j]
// 2^84, so that 64-bit atomics can add to it (each added piece below 2^42
// in magnitude); the norm pass carries them back into range once per
// update.
constexpr int kLimb = 42;

__device__ __forceinline__ void n2_add(long long* __restrict__ n2l, int64_t kst, int32_t j, __int128 c) {
  const long long mask = (1ll << kLimb) - 1;
  const long long c0 = (long long)c & mask;
  const long long c1 = (long long)(c >> kLimb) & mask;
  const long long c2 = (long long)(c >> (2 * kLimb));
  atomicAdd(reinterpret_cast<unsigned long long*>(n2l + j), (unsigned long long)c0);
  atomicAdd(reinterpret_cast<unsigned long long*>(n2l + kst + j), (unsigned long long)c1);
  atomicAdd(reinterpret_cast<unsigned long long*>(n2l + 2 * kst + j), (unsigned long long)c2);
}
__device__ __forceinline__ __int128 n2_get(const long long* __restrict__ n2l, int64_t kst, int32_t j) {
  return (__int128)__ldcg(n2l + j) + ((__int128)__ldcg(n2l + kst + j) << kLimb) +
         ((__int128)__ldcg(n2l + 2 * kst + j) << (2 * kLimb));
}
__device__ __forceinline__ void n2_set(long long* __restrict__ n2l, int64_t kst, int32_t j, __int128 v) {
  const long long mask = (1ll << kLimb) - 1;
  n2l[j] = (long long)v & mask;
  n2l[kst + j] = (long long)(v >> kLimb) & mask;
  n2l[2 * kst + j] = (long long)(v >> (2 * kLimb));
}
// A warp's sum of one __int128 per lane (every lane gets it).
__device__ __forceinline__ __int128 warp_sum128(__int128 v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(SKM_FULL_MASK, (unsigned long long)v, o);
    const long long hi = __shfl_xor_sync(SKM_FULL_MASK, (long long)(v >> 64), o);
    v += (((__int128)hi) << 64) | lo;
  }
  return v;
}

// Append (i, old) to the changed-row list through a per-warp buffer: lane r
// holds the r-th pending entry; the warp flushes 32 at a time with one atomic.
// All arguments but the buffer are warp-uniform.
struct ChangedBuf {
  int n = 0;
  int32_t bi = 0, bo = 0;
  __device__ __forceinline__ void flush(int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
                                        unsigned long long* __restrict__ cnt) {
    if (n == 0) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cnt + C_CHG, (unsigned long long)n);
    base = __shfl_sync(SKM_FULL_MASK, base, 0);
    if (lane < n) {
      chg_i[base + lane] = bi;
      chg_old[base + lane] = bo;
    }
    n = 0;
  }
  __device__ __forceinline__ void push(int32_t i, int32_t old, int32_t* __restrict__ chg_i,
                                       int32_t* __restrict__ chg_old, unsigned long long* __restrict__ cnt) {
    if ((threadIdx.x & 31) == n) {
      bi = i;
      bo = old;
    }
    if (++n == 32) flush(chg_i, chg_old, cnt);
  }
};

// Warp-aggregated append of `item` (when take) to list[*count]; returns nothing.
__device__ __forceinline__ void warp_push(bool take, int32_t item, int32_t* __restrict__ list,
                                          unsigned long long* __restrict__ count) {
  const unsigned m = __ballot_sync(SKM_FULL_MASK, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
  base = __shfl_sync(SKM_FULL_MASK, base, leader);
  if (take) list[base + __popc(m & ((1u << lane) - 1u))] = item;
}

// The same, filling the list downwards from list_top (list_top[-pos]).
__device__ __forceinline__ void warp_push_down(bool take, int32_t item, int32_t* __restrict__ list_top,
                                               unsigned long long* __restrict__ count) {
  const unsigned m = __ballot_sync(SKM_FULL_MASK, take);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
  base = __shfl_sync(SKM_FULL_MASK, base, leader);
  if (take) list_top[-(int64_t)(base + __popc(m & ((1u << lane) - 1u)))] = item;
}

// Is this center update a full recomputation of the sums?  (Else only the
// rows whose label changed are moved; decided on the device.)
__device__ __forceinline__ bool full_update(int s64_valid, const unsigned long long* cnt, int64_t n) {
  return !s64_valid || cnt[C_CHG] * 8ull > (unsigned long long)n;
}

// ---------------------------------------------------------------- context
}  // namespace skm

constexpr int kLogCap = 256;  // iterations a graph replay logs between host reads

// One run of a batch (many independent clusterings in one context): rows
// [row0, row0 + n) of the concatenated data, centers koff .. koff + k - 1 in
// global numbering (the run's slice of the term-major arrays is kst wide, a
// multiple of 8, so koff is too), Elkan bound rows of kst floats from uoff,
// and (full variants) its block of center-center bounds and Gram entries,
// k rows of kst, from ccoff.  Labels are global center ids.
struct RunDesc {
  int64_t row0, n, uoff, ccoff;
  int32_t koff, k, kst, cap;
};

// Where a row's centers and bounds live: its run's slice, or for a single
// run the whole center range (ccoff: the first center-center row; kst: the
// row stride of the bound and center-center rows).
struct RowGeom {
  int64_t ubase, ccoff;
  int32_t koff, k, cap, kst;
  int64_t ybase, ystride;  // Yin-Yang in a batch: u(i,G) at ybase + G ystride (the run's group-major block)
};
template <bool BATCH>
__device__ __forceinline__ RowGeom row_geom(int64_t i, int32_t k, int64_t kst, int32_t cap,
                                            const int32_t* __restrict__ row_run,
                                            const RunDesc* __restrict__ runs) {
  RowGeom g;
  if (!BATCH) {
    g.ubase = i * kst;
    g.ccoff = 0;
    g.koff = 0;
    g.k = k;
    g.cap = cap;
    g.kst = (int32_t)kst;
    g.ybase = 0;  // single runs address u(i,G) as G n + i
    g.ystride = 0;
  } else {
    const RunDesc& R = runs[row_run[i]];
    g.ubase = R.uoff + (i - R.row0) * (int64_t)R.kst;
    g.ccoff = R.ccoff;
    g.koff = R.koff;
    g.k = R.k;
    g.cap = R.cap;
    g.kst = R.kst;
    g.ybase = R.uoff + (i - R.row0);  // Yin-Yang batches lay uoff out per group block
    g.ystride = R.n;
  }
  return g;
}

struct skm_ctx {
  cudaStream_t st;
  int dev;
  int nsm;
  // problem
  int64_t n, d, nnz;
  int32_t k, kst;  // kst = row stride of the term-major center arrays (k rounded up to 8)
  int32_t variant, layout, dtype;
  // batch of independent runs (nruns == 0: a single run)
  int32_t nruns;
  int32_t kmax;         // widest run slice (bins of the center sums)
  RunDesc* runs;        // [nruns] device
  int32_t* row_run;     // [n] run of each row
  void* hruns;          // std::vector<RunDesc> host copy
  void* hinit;          // std::vector<int64_t>: the initial rows (global), for resets
  // whole iteration as a CUDA graph (skm_run with opt.graph)
  cudaGraphExec_t gexec;
  cudaStream_t cap_st;
  int64_t gkernels;       // kernel nodes in the graph
  unsigned long long* glog;  // [2 + 2 * kLogCap]: position, then (changed, sims) per iteration
  skm_options opt;
  // data (borrowed, or owned copies when given in host memory)
  const int64_t* rp;
  const int32_t* col;
  const void* val;
  void* own[3];
  // preparation
  float* rinv;         // [n] 1/|x_i| (FP32 of the FP64 value)
  float* dlt;          // [n] delta_i: bound on the FP32 error of a similarity of row i
  int64_t* t_ptr;      // [d+1] term-major (CSC) offsets
  int32_t* t_row;      // [nnz]
  int32_t* hst;        // [4] Hamerly: skip tightening this iteration, iterations skipped, blocks done
  long long* n2l;      // [3 kst] exact squared norms of the cluster sums as 42-bit limbs
  int32_t scr_off;     // 1: the screened whole-row pass is not used although Ct16 is kept (skm_autotune)
  void* t_val;         // [nnz] dtype
  int64_t nchunks;     // center-sum work items
  int32_t* ch_term;    // [nchunks]
  int32_t* ch_idx;     // [nchunks] chunk number within its term
  int64_t* ch_part;    // [nchunks] partial slot (-1: the term has a single chunk)
  int64_t nparts;      // number of partial slots
  int64_t nmulti;      // terms with several chunks
  int32_t* multi_term; // [nmulti]
  int64_t* multi_base; // [nmulti] first partial slot of the term
  int32_t* multi_cnt;  // [nmulti] chunks of the term
  long long* part64;   // [nparts * k] fixed-point partial sums
  float fx_scale, fx_inv;
  // centers (term-major, d x kst)
  float* Ct;        // current centers
  __half* Ct16;     // screened whole-row passes: FP16 copy of Ct (same layout), or NULL
  double* e2p;      // per (256-term tile, dirty slot): sum of the squared FP16 rounding errors
  double* e2c;      // [kst] per center: |fp16(c_j) - c_j|^2 (FP64 sum of exact squares)
  float* escr;      // [1] E >= max_j |fp16(c_j) - c_j| (rounded up, with slack)
  int32_t* w4;      // [n] rows for the exact whole-row pass after a screened one
  long long* S64;   // exact fixed-point cluster sums (d x kst)
  int s64_valid;    // S64 matches the current labels (else: full recompute)
  int chg_fresh;    // the changed-row list belongs to the last assignment
  int cnt_clear;    // the counters [0, C_ERR) were zeroed by the last center update
  unsigned long long* glog_active;  // while capturing the replayed iteration: glog (k_center_sum logs into it)
  int32_t* chg_i;   // [n] rows whose label changed in the last assignment
  int32_t* chg_old; // [n] their previous labels
  int32_t* dflag;   // [k] cluster sum touched by the incremental update
  int32_t* dmark;   // [k] cluster dirty in this update
  int32_t* dpos;    // [k] its position in dlist
  int32_t* dlist;   // [k] dirty clusters, ascending
  double* nrm;  // [k] |S_j|
  double* red;  // reduction partials
  int64_t red_blocks;
  double* obj;  // [1] objective
  float* pdn;   // [kst] drift cosine lower bound
  float* pup;   // [kst] drift cosine upper bound
  float* qup;   // [kst] drift sine upper bound
  float* gdrift;  // [3 ng] Yin-Yang: per group of 8 centers min pd, max pu, max q
  float* hsel;  // [HSEL_N] Hamerly drift summary (a batch: one per run)
  float* cc;    // [k * kst] center-center bounds (full variants; a batch: per run from ccoff)
  float* sc;    // [k] s(j)
  double* gpart;  // Gram partials (all tiles)
  double* G;      // [k * k] Gram, upper triangle (a batch: each run's k x kst block from ccoff, both triangles)
  int32_t* gdbeg;   // batch Gram plan: per run the first of its dirty centers in dlist
  int32_t* gdcnt;   // ... and their number
  int64_t* gtask;   // [nruns + 1] exclusive prefix of the runs' tile counts
  double* rpart;  // Gram partials of dirty rows
  int32_t gsplit, rsplit, grow_max;
  // dense rows (layout SKM_DENSE)
  int32_t precision;  // SKM_PREC_*
  int32_t kpad;       // centers padded to the tensor-core tile (256)
  float* exr;         // [n] |bf16(x_i/|x_i|) - x_i/|x_i||, rounded up (precision form)
  float* ebc;         // [2] {1 + 6u + E_c, E_c + accumulation term}, E_c = max_j |bf16(c_j) - c_j|
  unsigned* ebw;      // [2] k_center_err's running max (float bits) and block counter; zero between launches
  void* Xb;           // [n x d] BF16 unit rows, or FP8-E4M3 rows scaled by 2^e_i
  float* rsc;         // [n] FP8: 2^-(e_i + 8), accumulator -> similarity
  float* Cr;          // [k x d] FP32 centers, row-major
  void* Cb;           // [kpad x d] BF16 centers, or FP8-E4M3 of 2^8 c
  float* topv;        // [n x 8] best BF16 similarities per row, descending
  int32_t* topi;      // [n x 8] their centers
  uint2* cand;        // [2 x 16 x n] the tensor kernel's per-group lists (value bits, center)
  uint8_t* cand_n;    // [2 x n] their lengths
  int32_t* w3;        // [n] rows rechecked against their candidates
  int32_t* lcount;    // [k] members per cluster
  int32_t* loff;      // [k+1]
  int32_t* lcursor;   // [k]
  int32_t* lmembers;  // [n] rows sorted by label
  // labels and bounds
  int32_t* a;
  float* lb;  // [n]
  float* ub;  // [n] (Hamerly) or [n * kst] (Elkan)
  // worklists: points failing the first bound test, points needing a whole row
  int32_t* w1;
  int32_t* w2;
  // counters
  unsigned long long* cnt;   // device [C_NUM]
  unsigned long long* fbar;  // device [3]: k_finish_fused's barrier and last-block counters, k_drift_hsel's
                             // last-block counter (all only grow)
  unsigned long long* hcnt;  // pinned host mirror [C_NUM]
  double* hobj;              // pinned host [1]
  // per-kernel CUDA-event timing (skm_profile)
  int prof_on;
  void* prof;  // std::vector of (name, start event, end event)
  // state
  int have_bounds;
  int moved;  // centers changed since the last assignment (drift valid)
  skm_stats stats;
};

namespace skm {

// Library-wide kernel launch counter (host side).
void note_launch(int n = 1);

// Per-kernel timing: when enabled on the context, the launch between
// prof_begin and prof_end is bracketed by two CUDA events on its stream.
void prof_begin(skm_ctx* c, const char* name);
void prof_end(skm_ctx* c);

// ------------------------------------------------------- kernel wrappers
// prep (k_prep.cu)
int prep_rows(skm_ctx* c);             // validate CSR, rinv, delta
int prep_transpose(skm_ctx* c);        // CSC copy + center-sum chunks
int init_centers(skm_ctx* c, const int64_t* rows_dev);
int scan_i64(cudaStream_t st, const int64_t* in, int64_t* out, int64_t len);  // exclusive, out[len] = total
int centers_to_rows(skm_ctx* c, float* out /* k x d */);
int rows_to_centers(skm_ctx* c, const float* in /* k x d */);

// assignment (k_assign.cu)
int assign_full(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows);
int hamerly_step(skm_ctx* c);
int hamerly_bounds_only(skm_ctx* c);
int elkan_step(skm_ctx* c);

// update (k_update.cu)
int update_centers(skm_ctx* c);
int finish_update(skm_ctx* c);
int ct16_all(skm_ctx* c);  // Ct16, e2c and escr from the whole of Ct (after Ct was set outside an update)

// dense rows (k_dense.cu, k_mma.cu)
int dense_prep_bf16(skm_ctx* c);
int dense_prep_fp8(skm_ctx* c);
int dense_refresh_centers(skm_ctx* c);
int dense_bf16_eps(skm_ctx* c, float* out);
int dense_rows(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt);
int dense_classify(skm_ctx* c, bool hamerly, const int32_t* list, const unsigned long long* list_cnt);
int dense_tighten(skm_ctx* c);
int dense_center_sums(skm_ctx* c);
int bf16_mma_supported(int64_t d);
int fp8_mma_supported(int64_t d);
constexpr int kTopK = 8;  // BF16 candidates kept per row
int bf16_topk(skm_ctx* c, const void* Xb, const void* Cb, int use_thr, float* topv, int32_t* topi);
int dense_lower(skm_ctx* c);
int dense_recheck_cands(skm_ctx* c, bool hamerly);
int wait_selftest(int64_t timeout_ns, cudaStream_t st);
int barrier_selftest(int64_t timeout_ns, cudaStream_t st);
// The first assignment kept by a seeding (seed_kmeanspp with first != NULL):
// per row the best similarity, its center and the second best (device
// buffers the seeding allocates and seed_finish frees); elkan: the seeding
// also writes Elkan's bounds u(i,j) into the context's array.
struct SeedFirst {
  int elkan, keep_l, keep_u;
  float* m;
  int32_t* best;
  float* second;
};
int seed_kmeanspp(skm_ctx* c, const double* u, int64_t* rows_host, SeedFirst* first = nullptr);
int seed_finish(skm_ctx* c, SeedFirst* first);
int yinyang_step(skm_ctx* c);

}  // namespace skm

#define SKM_CUDA_TRY(x)                      \
  do {                                       \
    cudaError_t e__ = (x);                   \
    if (e__ != cudaSuccess) return SKM_ECUDA; \
  } while (0)

#define SKM_LAUNCH_CHECK()                                 \
  do {                                                     \
    skm::note_launch();                                    \
    if (cudaPeekAtLastError() != cudaSuccess) {            \
      (void)cudaGetLastError();                            \
      return SKM_ECUDA;                                    \
    }                                                      \
  } while (0)

// Profiled launch: name the kernel before the launch, close it after.
#define SKM_PROF_BEGIN(c, name) skm::prof_begin((c), (name))
#define SKM_LAUNCHED(c)   \
  do {                    \
    skm::prof_end(c);     \
    SKM_LAUNCH_CHECK();   \
  } while (0)
