// The assignment step (Section 5) and its pruned forms: Hamerly (5.3, 5.4)
// and Elkan (5.1, 5.2) with bounds kept on cosines (Section 4).
//
// Kernels:
//   k_rows_top2     warp per row: all k similarities of a CSR row against the
//                   term-major centers (an SpMM row fused with a top-2 argmax
//                   under the tie rule); initialises / refreshes the bounds.
//   k_ham_bounds    thread per point: Eq. (eqn:l-bound), Eq. (eqn:u-hamerly-2),
//                   prune test, compaction of the survivors.
//   k_tighten       thread per survivor: exact <x, c_a> (l made tight), retest.
//   k_elk_bounds    warp per point: Eq. (eqn:l-bound) and Eq. (eqn:u-elkan) on
//                   the whole bound row, prune tests, compaction.
//   k_elk_compact   warp per survivor: retest with the tight l, append the
//                   surviving (point, center) pairs in ascending center order.
//   k_pair_sims     thread per pair: the exact similarity, u(i,j) refreshed.
//   k_elk_merge     thread per survivor: best candidate under the tie rule.
#include <climits>

#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kBlock = 256;

// MODE 0: labels only (standard).  MODE 1: also l(i) and Hamerly's u(i).
// MODE 2: also l(i) and every Elkan bound u(i,j).
template <typename VT, int NT, int MODE>
__global__ void __launch_bounds__(kBlock) k_rows_top2(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int32_t k,
    int64_t kst, const int32_t* __restrict__ list, const unsigned long long* __restrict__ list_cnt, int64_t nrows,
    int32_t* __restrict__ a, float* __restrict__ lb, float* __restrict__ ub, unsigned long long* __restrict__ cnt) {
  constexpr int KT = 32 * NT;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = list ? (int64_t)(*list_cnt) : nrows;
  unsigned long long my_changed = 0, my_sims = 0;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    const int64_t i = list ? (int64_t)list[w] : w;
    const int64_t b = rp[i], e = rp[i + 1];
    const float ri = rinv[i];
    const float dl = dlt[i];
    const int32_t cur = a[i];
    float v1 = -INFINITY, v2 = -INFINITY, vcur = -INFINITY;
    int j1 = INT_MAX;
    for (int j0 = 0; j0 < k; j0 += KT) {
      float acc[NT];
      bool ok[NT];
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        acc[m] = 0.f;
        ok[m] = (j0 + m * 32 + lane) < k;
      }
      for (int64_t p0 = b; p0 < e; p0 += 32) {
        int tt = 0;
        float vv = 0.f;
        if (p0 + lane < e) {
          tt = __ldg(col + p0 + lane);
          vv = to_f32(val[p0 + lane]);
        }
        const int nq = (int)min((int64_t)32, e - p0);
#pragma unroll 4
        for (int q = 0; q < nq; ++q) {
          const int t = __shfl_sync(SKM_FULL_MASK, tt, q);
          const float v = __shfl_sync(SKM_FULL_MASK, vv, q);
          const float* crow = Ct + (int64_t)t * kst + j0 + lane;
#pragma unroll
          for (int m = 0; m < NT; ++m)
            if (ok[m]) acc[m] = __fmaf_rn(v, __ldg(crow + m * 32), acc[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const int j = j0 + m * 32 + lane;
        if (ok[m]) {
          const float s = __fmul_rn(acc[m], ri);
          if (MODE == 2) ub[i * kst + j] = __fadd_ru(s, dl);
          if (j == cur) vcur = s;
          if (s > v1) {
            v2 = v1;
            v1 = s;
            j1 = j;
          } else if (s > v2) {
            v2 = s;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float ov1 = __shfl_xor_sync(SKM_FULL_MASK, v1, o);
      const int oj1 = __shfl_xor_sync(SKM_FULL_MASK, j1, o);
      const float ov2 = __shfl_xor_sync(SKM_FULL_MASK, v2, o);
      if (ov1 > v1 || (ov1 == v1 && oj1 < j1)) {
        v2 = fmaxf(ov2, v1);
        v1 = ov1;
        j1 = oj1;
      } else {
        v2 = fmaxf(v2, ov1);
      }
      vcur = fmaxf(vcur, __shfl_xor_sync(SKM_FULL_MASK, vcur, o));
    }
    int32_t nb;
    float ssec;
    if (cur >= 0 && vcur == v1) {  // the current label is among the maxima: it stays
      nb = cur;
      ssec = (j1 == cur) ? v2 : v1;
    } else {
      nb = j1;
      ssec = v2;
    }
    if (lane == 0) {
      a[i] = nb;
      my_changed += (nb != cur);
      my_sims += (unsigned long long)k;
      if (MODE >= 1) lb[i] = __fsub_rd(v1, dl);
      if (MODE == 1) ub[i] = (k > 1) ? __fadd_ru(ssec, dl) : -1.f;
    }
  }
  if (lane == 0) {
    if (my_changed) atomicAdd(cnt + C_CHANGED, my_changed);
    if (my_sims) atomicAdd(cnt + C_SIMS, my_sims);
  }
}

// ------------------------------------------------------------- Hamerly

template <bool FULL>
__global__ void __launch_bounds__(kBlock) k_ham_bounds(int64_t n, const int32_t* __restrict__ a,
                                                       float* __restrict__ lb, float* __restrict__ ub,
                                                       const float* __restrict__ dlt, const float* __restrict__ pdn,
                                                       const float* __restrict__ pup, const float* __restrict__ qup,
                                                       const float* __restrict__ hsel, const float* __restrict__ sc,
                                                       int tight, int moved, int32_t* __restrict__ w1,
                                                       unsigned long long* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int jmin_d = (int)hsel[0], jmin_u = (int)hsel[3], jmax_q = (int)hsel[6];
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool take = false;
    if (i < n) {
      const int32_t ai = a[i];
      float l = lb[i], u = ub[i];
      if (moved) {
        // p'(a) = min_{j != a} p(j): the worst drift among the other centers
        const float pdm = (ai == jmin_d) ? hsel[2] : hsel[1];
        const float pum = (ai == jmin_u) ? hsel[5] : hsel[4];
        const float qm = (ai == jmax_q) ? hsel[8] : hsel[7];
        l = bound_l(l, pdn[ai], pup[ai], qup[ai]);
        u = bound_u_hamerly(u, pdm, pum, qm, tight);
        lb[i] = l;
        ub[i] = u;
      }
      const float L = __fsub_rd(l, 2.f * dlt[i]);
      const bool prune = (L >= u) || (FULL && L >= 0.f && L >= sc[ai]);
      take = !prune;
    }
    warp_push(take, (int32_t)i, w1, cnt + C_W1);
  }
}

// Thread per survivor: l(i) <- <x(i), c(a(i))> (made tight), then the test
// again; the points still failing go to `out` (Hamerly) -- for Elkan the
// tight similarity is kept for the merge and no retest is done here.
template <typename VT, bool FULL, bool HAMERLY>
__global__ void __launch_bounds__(kBlock) k_tighten(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int64_t kst,
    const int32_t* __restrict__ w1, const unsigned long long* __restrict__ w1_cnt, const int32_t* __restrict__ a,
    float* __restrict__ lb, const float* __restrict__ ub, const float* __restrict__ sc, float* __restrict__ w1s,
    int32_t* __restrict__ out, unsigned long long* __restrict__ cnt) {
  const int64_t total = (int64_t)(*w1_cnt);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long sims = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t idx = base + threadIdx.x;
    bool take = false;
    int32_t i = 0;
    if (idx < total) {
      i = w1[idx];
      const int32_t ai = a[i];
      const float s = __fmul_rn(dot_row_center<VT>(rp[i], rp[i + 1], col, val, Ct, kst, ai), rinv[i]);
      ++sims;
      const float dl = dlt[i];
      const float l = __fsub_rd(s, dl);
      lb[i] = l;
      if (HAMERLY) {
        const float L = __fsub_rd(l, 2.f * dl);
        take = !((L >= ub[i]) || (FULL && L >= 0.f && L >= sc[ai]));
      } else {
        w1s[idx] = s;
      }
    }
    if (HAMERLY) warp_push(take, i, out, cnt + C_W2);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
  if ((threadIdx.x & 31) == 0 && sims) atomicAdd(cnt + C_SIMS, sims);
}

// --------------------------------------------------------------- Elkan

// Is (i, j) still a candidate: u(i,j) > L and, for full Elkan, cc(a,j) > L
// (Section 5.2: cc(a,j) <= l with l >= 0 rules c(j) out).
template <bool FULL>
__device__ __forceinline__ bool elk_cand(int j, int32_t ai, float u, float L, const float* __restrict__ ccrow) {
  if (j == ai || !(u > L)) return false;
  if (FULL && L >= 0.f && __ldg(ccrow + j) <= L) return false;
  return true;
}

// Warp per point; each warp walks 32 consecutive points and pushes the
// survivors of the tile with one atomic.
template <bool FULL>
__global__ void __launch_bounds__(kBlock) k_elk_bounds(int64_t n, int32_t k, int64_t kst, const int32_t* __restrict__ a,
                                                       float* __restrict__ lb, float* __restrict__ ub,
                                                       const float* __restrict__ dlt, const float* __restrict__ pdn,
                                                       const float* __restrict__ pup, const float* __restrict__ qup,
                                                       const float* __restrict__ cc, const float* __restrict__ sc,
                                                       int moved, int32_t* __restrict__ w1,
                                                       unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 32 < n; tile += nw) {
    unsigned surv = 0;
    const int64_t i0 = tile * 32;
    const int rows = (int)min((int64_t)32, n - i0);
    for (int r = 0; r < rows; ++r) {
      const int64_t i = i0 + r;
      const int32_t ai = a[i];
      float l = lb[i];
      if (moved) l = bound_l(l, pdn[ai], pup[ai], qup[ai]);
      const float L = __fsub_rd(l, 2.f * dlt[i]);
      const bool skip_pt = FULL && L >= 0.f && sc[ai] <= L;
      float* urow = ub + i * kst;
      const float* ccrow = cc + (int64_t)ai * kst;
      bool any = false;
      for (int j4 = lane * 4; j4 < k; j4 += 128) {
        float4 u4 = *reinterpret_cast<const float4*>(urow + j4);
        if (moved) {
          const float4 pd = *reinterpret_cast<const float4*>(pdn + j4);
          const float4 pu = *reinterpret_cast<const float4*>(pup + j4);
          const float4 q = *reinterpret_cast<const float4*>(qup + j4);
          u4.x = bound_u(u4.x, pd.x, pu.x, q.x);
          u4.y = bound_u(u4.y, pd.y, pu.y, q.y);
          u4.z = bound_u(u4.z, pd.z, pu.z, q.z);
          u4.w = bound_u(u4.w, pd.w, pu.w, q.w);
          *reinterpret_cast<float4*>(urow + j4) = u4;
        }
        if (!skip_pt) {
          any |= (j4 + 0 < k) && elk_cand<FULL>(j4 + 0, ai, u4.x, L, ccrow);
          any |= (j4 + 1 < k) && elk_cand<FULL>(j4 + 1, ai, u4.y, L, ccrow);
          any |= (j4 + 2 < k) && elk_cand<FULL>(j4 + 2, ai, u4.z, L, ccrow);
          any |= (j4 + 3 < k) && elk_cand<FULL>(j4 + 3, ai, u4.w, L, ccrow);
        }
      }
      if (__any_sync(SKM_FULL_MASK, any)) surv |= 1u << r;
      if (moved && lane == 0) lb[i] = l;
    }
    warp_push((surv >> lane) & 1u, (int32_t)(i0 + lane), w1, cnt + C_W1);
  }
}

// Warp per survivor: test every center again with the tight l, append the
// remaining pairs in ascending center order as one contiguous segment.
template <bool FULL>
__global__ void __launch_bounds__(kBlock) k_elk_compact(
    int32_t k, int64_t kst, const int32_t* __restrict__ w1, const unsigned long long* __restrict__ w1_cnt,
    const int32_t* __restrict__ a, const float* __restrict__ lb, const float* __restrict__ ub,
    const float* __restrict__ dlt, const float* __restrict__ cc, const float* __restrict__ sc,
    int64_t* __restrict__ poff, int32_t* __restrict__ pnum, int32_t* __restrict__ pslot, int32_t* __restrict__ pj,
    int64_t pcap, int32_t row_thresh, int32_t* __restrict__ w2, unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = (int64_t)(*w1_cnt);
  for (int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total; slot += nw) {
    const int32_t i = w1[slot];
    const int32_t ai = a[i];
    const float L = __fsub_rd(lb[i], 2.f * dlt[i]);
    const bool skip_pt = FULL && L >= 0.f && sc[ai] <= L;
    const float* urow = ub + (int64_t)i * kst;
    const float* ccrow = cc + (int64_t)ai * kst;
    int mine = 0;
    if (!skip_pt) {
      for (int j4 = lane * 4; j4 < k; j4 += 128) {
        const float4 u4 = *reinterpret_cast<const float4*>(urow + j4);
        mine += (j4 + 0 < k) && elk_cand<FULL>(j4 + 0, ai, u4.x, L, ccrow);
        mine += (j4 + 1 < k) && elk_cand<FULL>(j4 + 1, ai, u4.y, L, ccrow);
        mine += (j4 + 2 < k) && elk_cand<FULL>(j4 + 2, ai, u4.z, L, ccrow);
        mine += (j4 + 3 < k) && elk_cand<FULL>(j4 + 3, ai, u4.w, L, ccrow);
      }
    }
    int tot = mine;
#pragma unroll
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(SKM_FULL_MASK, tot, o);
    if (tot == 0) {
      if (lane == 0) pnum[slot] = 0;
      continue;
    }
    if (tot > row_thresh) {
      // many candidates: the whole row through the SpMM kernel is cheaper
      // (same similarity order, so the same values)
      if (lane == 0) {
        pnum[slot] = 0;
        const unsigned long long pos = atomicAdd(cnt + C_W2, 1ull);
        w2[pos] = i;
      }
      continue;
    }
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(cnt + C_PAIRS, (unsigned long long)tot);
    off = __shfl_sync(SKM_FULL_MASK, off, 0);
    if ((int64_t)(off + tot) > pcap) {
      // no room: mark the reserved entries that exist as unused and send the
      // point to the full recompute
      for (int64_t q = (int64_t)off + lane; q < pcap && q < (int64_t)off + tot; q += 32) pslot[q] = -1;
      if (lane == 0) {
        pnum[slot] = 0;
        const unsigned long long pos = atomicAdd(cnt + C_W2, 1ull);
        w2[pos] = i;
      }
      continue;
    }
    if (lane == 0) {
      poff[slot] = (int64_t)off;
      pnum[slot] = tot;
    }
    int64_t pos0 = (int64_t)off;
    for (int g = 0; g * 128 < k; ++g) {
      const int j4 = g * 128 + lane * 4;
      unsigned m = 0;
      if (j4 < k) {
        const float4 u4 = *reinterpret_cast<const float4*>(urow + j4);
        m |= ((j4 + 0 < k) && elk_cand<FULL>(j4 + 0, ai, u4.x, L, ccrow)) ? 1u : 0u;
        m |= ((j4 + 1 < k) && elk_cand<FULL>(j4 + 1, ai, u4.y, L, ccrow)) ? 2u : 0u;
        m |= ((j4 + 2 < k) && elk_cand<FULL>(j4 + 2, ai, u4.z, L, ccrow)) ? 4u : 0u;
        m |= ((j4 + 3 < k) && elk_cand<FULL>(j4 + 3, ai, u4.w, L, ccrow)) ? 8u : 0u;
      }
      const int c = __popc(m);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(SKM_FULL_MASK, incl, o);
        if (lane >= o) incl += y;
      }
      int64_t pos = pos0 + (incl - c);
      for (int b = 0; b < 4; ++b)
        if (m & (1u << b)) {
          pslot[pos] = (int32_t)slot;
          pj[pos] = j4 + b;
          ++pos;
        }
      pos0 += __shfl_sync(SKM_FULL_MASK, incl, 31);
    }
  }
}

template <typename VT>
__global__ void __launch_bounds__(kBlock) k_pair_sims(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int64_t kst,
    const int32_t* __restrict__ w1, const int32_t* __restrict__ pslot, const int32_t* __restrict__ pj,
    const unsigned long long* __restrict__ pcnt, int64_t pcap, float* __restrict__ psim, float* __restrict__ ub,
    unsigned long long* __restrict__ cnt) {
  int64_t total = (int64_t)(*pcnt);
  if (total > pcap) total = pcap;
  unsigned long long sims = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = pslot[q];
    if (slot < 0) continue;
    const int32_t i = w1[slot], j = pj[q];
    const float s = __fmul_rn(dot_row_center<VT>(rp[i], rp[i + 1], col, val, Ct, kst, j), rinv[i]);
    psim[q] = s;
    ub[(int64_t)i * kst + j] = __fadd_ru(s, dlt[i]);
    ++sims;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
  if ((threadIdx.x & 31) == 0 && sims) atomicAdd(cnt + C_SIMS, sims);
}

// Thread per survivor with pairs: the pairs are in ascending center order, so
// "strictly greater" keeps the current label on ties and otherwise the lowest
// index -- the standard variant's rule.
__global__ void __launch_bounds__(kBlock) k_elk_merge(
    int64_t kst, const int32_t* __restrict__ w1, const unsigned long long* __restrict__ w1_cnt,
    const float* __restrict__ w1s, const int64_t* __restrict__ poff, const int32_t* __restrict__ pnum,
    const int32_t* __restrict__ pj, const float* __restrict__ psim, const float* __restrict__ dlt,
    int32_t* __restrict__ a, float* __restrict__ lb, float* __restrict__ ub, unsigned long long* __restrict__ cnt) {
  const int64_t total = (int64_t)(*w1_cnt);
  unsigned long long changed = 0;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < total;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int32_t np = pnum[slot];
    if (np == 0) continue;
    const int32_t i = w1[slot];
    const int32_t ai = a[i];
    const int64_t o = poff[slot];
    float best = w1s[slot];
    int32_t bj = ai;
    for (int32_t q = 0; q < np; ++q) {
      const float s = psim[o + q];
      if (s > best) {
        best = s;
        bj = pj[o + q];
      }
    }
    if (bj != ai) {
      const float dl = dlt[i];
      a[i] = bj;
      lb[i] = __fsub_rd(best, dl);
      ub[(int64_t)i * kst + ai] = __fadd_ru(w1s[slot], dl);
      ++changed;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
  if ((threadIdx.x & 31) == 0 && changed) atomicAdd(cnt + C_CHANGED, changed);
}

inline int persistent_grid(const skm_ctx* c, int per_sm = 8) { return c->nsm * per_sm; }

template <typename VT, int NT>
int launch_rows(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows) {
  int64_t g = list ? (int64_t)persistent_grid(c, 8) : (nrows * 32 + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)c->nsm * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  const VT* v = (const VT*)c->val;
  SKM_PROF_BEGIN(c, list ? "k_rows_top2(list)" : "k_rows_top2");
  switch (mode) {
    case 0:
      k_rows_top2<VT, NT, 0><<<(unsigned)g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst,
                                                                 list, list_cnt, nrows, c->a, c->lb, c->ub, c->cnt);
      break;
    case 1:
      k_rows_top2<VT, NT, 1><<<(unsigned)g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst,
                                                                 list, list_cnt, nrows, c->a, c->lb, c->ub, c->cnt);
      break;
    default:
      k_rows_top2<VT, NT, 2><<<(unsigned)g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst,
                                                                 list, list_cnt, nrows, c->a, c->lb, c->ub, c->cnt);
  }
  SKM_LAUNCHED(c);
  return SKM_OK;
}

template <typename VT>
int assign_full_t(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows) {
  const int k = c->k;
  if (k <= 32) return launch_rows<VT, 1>(c, mode, list, list_cnt, nrows);
  if (k <= 64) return launch_rows<VT, 2>(c, mode, list, list_cnt, nrows);
  if (k <= 128) return launch_rows<VT, 4>(c, mode, list, list_cnt, nrows);
  if (k <= 256) return launch_rows<VT, 8>(c, mode, list, list_cnt, nrows);
  if (k <= 512) return launch_rows<VT, 16>(c, mode, list, list_cnt, nrows);
  return launch_rows<VT, 32>(c, mode, list, list_cnt, nrows);
}

template <typename VT>
int hamerly_step_t(skm_ctx* c) {
  const bool full = (c->variant == SKM_HAMERLY);
  const int g = persistent_grid(c);
  SKM_PROF_BEGIN(c, "k_ham_bounds");
  if (full) {
    k_ham_bounds<true><<<g, kBlock, 0, c->st>>>(c->n, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup, c->qup, c->hsel,
                                                c->sc, c->opt.hamerly_tight, c->moved, c->w1, c->cnt);
  } else {
    k_ham_bounds<false><<<g, kBlock, 0, c->st>>>(c->n, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup, c->qup, c->hsel,
                                                 c->sc, c->opt.hamerly_tight, c->moved, c->w1, c->cnt);
  }
  SKM_LAUNCHED(c);
  const VT* v = (const VT*)c->val;
  SKM_PROF_BEGIN(c, "k_tighten");
  if (full) {
    k_tighten<VT, true, true><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1,
                                                       c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w1s, c->w2, c->cnt);
  } else {
    k_tighten<VT, false, true><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1,
                                                        c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w1s, c->w2,
                                                        c->cnt);
  }
  SKM_LAUNCHED(c);
  return assign_full_t<VT>(c, 1, c->w2, c->cnt + C_W2, 0);
}

template <typename VT>
int elkan_step_t(skm_ctx* c) {
  const bool full = (c->variant == SKM_ELKAN);
  const int g = persistent_grid(c);
  SKM_PROF_BEGIN(c, "k_elk_bounds");
  if (full) {
    k_elk_bounds<true><<<g, kBlock, 0, c->st>>>(c->n, c->k, c->kst, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup,
                                                c->qup, c->cc, c->sc, c->moved, c->w1, c->cnt);
  } else {
    k_elk_bounds<false><<<g, kBlock, 0, c->st>>>(c->n, c->k, c->kst, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup,
                                                 c->qup, c->cc, c->sc, c->moved, c->w1, c->cnt);
  }
  SKM_LAUNCHED(c);
  const VT* v = (const VT*)c->val;
  SKM_PROF_BEGIN(c, "k_tighten");
  k_tighten<VT, false, false><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1,
                                                       c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w1s, nullptr,
                                                       c->cnt);
  SKM_LAUNCHED(c);
  // a point with more than k/8 candidate pairs is recomputed as a full row
  const int32_t row_thresh = c->opt.row_threshold > 0 ? c->opt.row_threshold : (c->k + 7) / 8;
  SKM_PROF_BEGIN(c, "k_elk_compact");
  if (full) {
    k_elk_compact<true><<<g, kBlock, 0, c->st>>>(c->k, c->kst, c->w1, c->cnt + C_W1, c->a, c->lb, c->ub, c->dlt, c->cc,
                                                 c->sc, c->poff, c->pnum, c->pslot, c->pj, c->pcap, row_thresh, c->w2, c->cnt);
  } else {
    k_elk_compact<false><<<g, kBlock, 0, c->st>>>(c->k, c->kst, c->w1, c->cnt + C_W1, c->a, c->lb, c->ub, c->dlt,
                                                  c->cc, c->sc, c->poff, c->pnum, c->pslot, c->pj, c->pcap,
                                                  row_thresh, c->w2, c->cnt);
  }
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_pair_sims");
  k_pair_sims<VT><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1, c->pslot, c->pj,
                                           c->cnt + C_PAIRS, c->pcap, c->psim, c->ub, c->cnt);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_elk_merge");
  k_elk_merge<<<g, kBlock, 0, c->st>>>(c->kst, c->w1, c->cnt + C_W1, c->w1s, c->poff, c->pnum, c->pj, c->psim, c->dlt,
                                       c->a, c->lb, c->ub, c->cnt);
  SKM_LAUNCHED(c);
  return assign_full_t<VT>(c, 2, c->w2, c->cnt + C_W2, 0);
}

}  // namespace

int assign_full(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows) {
  switch (c->dtype) {
    case SKM_F32: return assign_full_t<float>(c, mode, list, list_cnt, nrows);
    case SKM_F16: return assign_full_t<__half>(c, mode, list, list_cnt, nrows);
    case SKM_BF16: return assign_full_t<__nv_bfloat16>(c, mode, list, list_cnt, nrows);
  }
  return SKM_EINVAL;
}

int hamerly_step(skm_ctx* c) {
  switch (c->dtype) {
    case SKM_F32: return hamerly_step_t<float>(c);
    case SKM_F16: return hamerly_step_t<__half>(c);
    case SKM_BF16: return hamerly_step_t<__nv_bfloat16>(c);
  }
  return SKM_EINVAL;
}

int elkan_step(skm_ctx* c) {
  switch (c->dtype) {
    case SKM_F32: return elkan_step_t<float>(c);
    case SKM_F16: return elkan_step_t<__half>(c);
    case SKM_BF16: return elkan_step_t<__nv_bfloat16>(c);
  }
  return SKM_EINVAL;
}

}  // namespace skm
