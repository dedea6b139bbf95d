// The center update (Section 5): S_j = sum_{a(i)=j} x(i), c(j) = S_j/|S_j|;
// the drift p(j) = <c(j), c'(j)> that moves the bounds (Section 4); and the
// center-center bounds cc(i,j), s(i) of Section 5.2.
//
//   k_center_sum        warp per chunk of a term's column (term-major data):
//                       sums x_it into per-cluster bins in shared memory in
//                       64-bit fixed point.  Integer addition is exact and
//                       associative, so the result does not depend on the
//                       order of the entries or of the atomics: the center
//                       sum is deterministic with no atomics in global memory.
//   k_center_sum_multi  terms with several chunks: exact sum of the partials.
//   k_colnorm_part/final  |S_j| in FP64 over fixed blocks (deterministic).
//   k_normalize_drift   c(j) = S_j/|S_j| (empty cluster keeps c'(j)); FP64
//                       partial sums for the drift.
//   k_drift_final       per center: an interval [pd, pu] for cos(angle(c, c'))
//                       and an upper bound q for its sine, rounded outward to
//                       FP32; the Hamerly worst-drift summary.
//   k_gram_part/final   <c_i, c_j> (FP32 products, FP64 across 256-term
//                       chunks), widened by its error bound, -> cc and s.
#include <cfloat>

#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kChunk = 2048;  // must match the chunking built in k_prep.cu
constexpr int kTB = 256;      // rows (terms) per reduction block

template <typename VT>
__global__ void __launch_bounds__(256) k_center_sum(int64_t nchunks, const int32_t* __restrict__ ch_term,
                                                    const int32_t* __restrict__ ch_idx,
                                                    const int64_t* __restrict__ ch_part,
                                                    const int64_t* __restrict__ t_ptr, const int32_t* __restrict__ t_row,
                                                    const VT* __restrict__ t_val, const float* __restrict__ rinv,
                                                    const int32_t* __restrict__ a, int32_t k, int64_t kst, float scale,
                                                    float inv, float* __restrict__ S, long long* __restrict__ part) {
  extern __shared__ long long bins_all[];
  const int lane = threadIdx.x & 31;
  long long* bins = bins_all + (int64_t)(threadIdx.x >> 5) * k;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nchunks; g += nw) {
    const int64_t t = ch_term[g];
    const int64_t b = t_ptr[t] + (int64_t)ch_idx[g] * kChunk;
    const int64_t e = min(t_ptr[t + 1], b + kChunk);
    for (int j = lane; j < k; j += 32) bins[j] = 0;
    __syncwarp();
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t r = t_row[p];
      const float x = __fmul_rn(to_f32(t_val[p]), rinv[r]);
      const long long fx = __float2ll_rn(__fmul_rn(x, scale));
      atomicAdd(reinterpret_cast<unsigned long long*>(bins + a[r]), (unsigned long long)fx);
    }
    __syncwarp();
    const int64_t ps = ch_part[g];
    if (ps < 0) {
      float* row = S + t * kst;
      for (int j = lane; j < kst; j += 32) row[j] = (j < k) ? __fmul_rn(__ll2float_rn(bins[j]), inv) : 0.f;
    } else {
      long long* pr = part + ps * k;
      for (int j = lane; j < k; j += 32) pr[j] = bins[j];
    }
    __syncwarp();
  }
}

__global__ void k_center_sum_multi(int64_t nmulti, const int32_t* __restrict__ mterm, const int64_t* __restrict__ mbase,
                                   const int32_t* __restrict__ mcnt, const long long* __restrict__ part, int32_t k,
                                   int64_t kst, float inv, float* __restrict__ S) {
  const int64_t total = nmulti * kst;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = q / kst;
    const int j = (int)(q - m * kst);
    const int64_t t = mterm[m];
    float out = 0.f;
    if (j < k) {
      long long s = 0;
      const long long* pr = part + mbase[m] * k + j;
      for (int c = 0; c < mcnt[m]; ++c) s += pr[(int64_t)c * k];
      out = __fmul_rn(__ll2float_rn(s), inv);
    }
    S[t * kst + j] = out;
  }
}

// grid (ceil(d/kTB), ceil(k/32)), block (32, 8)
__global__ void k_colnorm_part(const float* __restrict__ S, int64_t d, int32_t k, int64_t kst,
                               double* __restrict__ red) {
  __shared__ double sh[8][33];
  const int j = blockIdx.y * 32 + threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * kTB;
  double s = 0.0;
  if (j < k)
    for (int64_t t = t0 + threadIdx.y; t < min(d, t0 + kTB); t += 8) {
      const double v = S[t * kst + j];
      s = fma(v, v, s);
    }
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < k) {
    double r = 0.0;
    for (int y = 0; y < 8; ++y) r += sh[y][threadIdx.x];
    red[(int64_t)blockIdx.x * kst + j] = r;
  }
}

// one block: |S_j| and J = sum_j |S_j|, in a fixed order
__global__ void __launch_bounds__(1024) k_colnorm_final(const double* __restrict__ red, int64_t nblk, int32_t k,
                                                        int64_t kst, double* __restrict__ nrm,
                                                        double* __restrict__ obj) {
  __shared__ double sh[1024];
  double mine = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int64_t b = 0; b < nblk; ++b) s += red[b * kst + j];
    const double nr = sqrt(s);
    nrm[j] = nr;
    mine += nr;
  }
  sh[threadIdx.x] = mine;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) obj[0] = sh[0];
}

// grid (ceil(d/kTB), ceil(k/32)), block (32, 8).  S is overwritten with the
// new centers; red2 receives, per block and center, sum c^2, sum c'^2 and
// sum (c - c')^2.
__global__ void k_normalize_drift(float* __restrict__ S, const float* __restrict__ Cold, const double* __restrict__ nrm,
                                  int64_t d, int32_t k, int64_t kst, double* __restrict__ red2) {
  __shared__ double sh[3][8][33];
  const int j = blockIdx.y * 32 + threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * kTB;
  double sn = 0.0, so = 0.0, sd = 0.0;
  if (j < k) {
    const double nr = nrm[j];
    const bool empty = !(nr > 0.0);
    const float inv = empty ? 0.f : (float)(1.0 / nr);
    for (int64_t t = t0 + threadIdx.y; t < min(d, t0 + kTB); t += 8) {
      const float co = Cold[t * kst + j];
      const float cn = empty ? co : __fmul_rn(S[t * kst + j], inv);
      S[t * kst + j] = cn;
      const double dn = cn, dv = co, df = dn - dv;
      sn = fma(dn, dn, sn);
      so = fma(dv, dv, so);
      sd = fma(df, df, sd);
    }
  }
  sh[0][threadIdx.y][threadIdx.x] = sn;
  sh[1][threadIdx.y][threadIdx.x] = so;
  sh[2][threadIdx.y][threadIdx.x] = sd;
  __syncthreads();
  if (threadIdx.y == 0 && j < k) {
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;
    for (int y = 0; y < 8; ++y) {
      r0 += sh[0][y][threadIdx.x];
      r1 += sh[1][y][threadIdx.x];
      r2 += sh[2][y][threadIdx.x];
    }
    double* o = red2 + ((int64_t)blockIdx.x * kst + j) * 3;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
  }
}

struct ArgMin {
  float v;
  int j;
};

// One block.  From N = |c|, N' = |c'| and D = |c - c'|^2 (all FP64 with
// relative error <= e):  1 - cos = (D - (N - N')^2) / (2 N N'), hence
//   q_up = D (1+4e) / (2 N N')           >= 1 - cos
//   q_dn = (D (1-e) - (|N-N'| + e)^2) / (2 N N' (1+3e))  <= 1 - cos
// pd = rd(1 - q_up), pu = ru(1 - q_dn), q = ru(max sin over [q_dn, q_up]).
// Identical vectors (D = 0) give exactly p = 1, sin = 0.
__global__ void __launch_bounds__(1024) k_drift_final(const double* __restrict__ red2, int64_t nblk, int32_t k,
                                                      int64_t kst, int64_t d, float* __restrict__ pdn,
                                                      float* __restrict__ pup, float* __restrict__ qup,
                                                      double* __restrict__ cnorm, float* __restrict__ hsel) {
  __shared__ float s_pd[1024], s_pu[1024], s_q[1024];
  __shared__ int s_jd[1024], s_ju[1024], s_jq[1024];
  const double e = ((double)d + 8.0) * 0x1.0p-53;
  for (int j = threadIdx.x; j < kst; j += blockDim.x) {
    if (j >= k) {
      pdn[j] = 1.f;
      pup[j] = 1.f;
      qup[j] = 0.f;
      continue;
    }
    double sn = 0.0, so = 0.0, sd = 0.0;
    for (int64_t b = 0; b < nblk; ++b) {
      const double* r = red2 + (b * kst + j) * 3;
      sn += r[0];
      so += r[1];
      sd += r[2];
    }
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
      pd = __double2float_rd(lo - 0x1.0p-60);
      pu = __double2float_ru(hi + 0x1.0p-60);
      pd = fmaxf(pd, -1.f);
      pu = fminf(pu, 1.f);
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
  // Hamerly summary: argmin / min / second min of pd and pu, argmax / max /
  // second max of q (lowest index on ties).  Sequential per thread over a
  // strided slice, then a fixed tree.
  float bd = FLT_MAX, bd2 = FLT_MAX, bu = FLT_MAX, bu2 = FLT_MAX, bq = -FLT_MAX, bq2 = -FLT_MAX;
  int jd = INT_MAX, ju = INT_MAX, jq = INT_MAX;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const float x = pdn[j], y = pup[j], z = qup[j];
    if (x < bd) { bd2 = bd; bd = x; jd = j; } else if (x < bd2) bd2 = x;
    if (y < bu) { bu2 = bu; bu = y; ju = j; } else if (y < bu2) bu2 = y;
    if (z > bq) { bq2 = bq; bq = z; jq = j; } else if (z > bq2) bq2 = z;
  }
  // two-value reductions via shared memory, pairwise in a fixed order
  __shared__ float s_pd2[1024], s_pu2[1024], s_q2[1024];
  s_pd[threadIdx.x] = bd; s_pd2[threadIdx.x] = bd2; s_jd[threadIdx.x] = jd;
  s_pu[threadIdx.x] = bu; s_pu2[threadIdx.x] = bu2; s_ju[threadIdx.x] = ju;
  s_q[threadIdx.x] = bq; s_q2[threadIdx.x] = bq2; s_jq[threadIdx.x] = jq;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const int a = threadIdx.x, b = threadIdx.x + o;
      // min pd
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
  }
}

// Gram partials: grid (ceil(k/32), ceil(k/32), nsplit), block (32, 8); tile
// (bi, bj) with bi <= bj only.  Each thread owns 4 entries; FP32 products are
// accumulated over 256 terms, then added to FP64 accumulators.
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ Ct, int64_t d, int32_t k, int64_t kst,
                                                   int64_t per_split, double* __restrict__ gpart) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ float A[32][33], B[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int64_t tb = (int64_t)blockIdx.z * per_split, te = min(d, tb + per_split);
  const int tx = threadIdx.x, ty = threadIdx.y;
  double acc64[4] = {0.0, 0.0, 0.0, 0.0};
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  int steps = 0;
  for (int64_t t0 = tb; t0 < te; t0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int64_t t = t0 + r;
      A[r][tx] = (t < te && i0 + tx < k) ? Ct[t * kst + i0 + tx] : 0.f;
      B[r][tx] = (t < te && j0 + tx < k) ? Ct[t * kst + j0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float bv = B[r][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = __fmaf_rn(A[r][ty + 8 * q], bv, acc[q]);
    }
    __syncthreads();
    if (++steps == 8) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc64[q] += (double)acc[q];
        acc[q] = 0.f;
      }
      steps = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc64[q] += (double)acc[q];
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < k && j < k) gpart[((int64_t)blockIdx.z * k + i) * k + j] = acc64[q];
  }
}

// Block per center i: <c_i, c_j> from the partials (fixed order), normalised by
// the FP64 norms and widened by the error bound eg, then
// cc(i,j) = sqrt((g+1)/2) rounded up and s(i) = max_{j != i} cc(i,j).
__global__ void __launch_bounds__(256) k_gram_final(const double* __restrict__ gpart, int32_t nsplit, int32_t k,
                                                    int64_t kst, const double* __restrict__ cnorm, double eg,
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
    double g = 0.0;
    for (int s = 0; s < nsplit; ++s) g += gpart[((int64_t)s * k + lo) * k + hi];
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

template <typename VT>
int center_sum_t(skm_ctx* c) {
  const int k = c->k;
  int wpb = (int)((96 * 1024) / ((int64_t)k * 8));
  if (wpb > 8) wpb = 8;
  if (wpb < 1) wpb = 1;
  const size_t smem = (size_t)wpb * k * 8;
  if (smem > 48 * 1024)
    SKM_CUDA_TRY(cudaFuncSetAttribute(k_center_sum<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t g = (c->nchunks + wpb - 1) / wpb;
  const int64_t cap = (int64_t)c->nsm * 16;
  if (g > cap) g = cap;
  SKM_PROF_BEGIN(c, "k_center_sum");
  k_center_sum<VT><<<(unsigned)g, wpb * 32, smem, c->st>>>(c->nchunks, c->ch_term, c->ch_idx, c->ch_part, c->t_ptr,
                                                           c->t_row, (const VT*)c->t_val, c->rinv, c->a, k, c->kst,
                                                           c->fx_scale, c->fx_inv, c->S, c->part64);
  SKM_LAUNCHED(c);
  if (c->nmulti > 0) {
    int64_t tot = c->nmulti * c->kst;
    int64_t gb = (tot + 255) / 256;
    if (gb > cap) gb = cap;
    SKM_PROF_BEGIN(c, "k_center_sum_multi");
    k_center_sum_multi<<<(unsigned)gb, 256, 0, c->st>>>(c->nmulti, c->multi_term, c->multi_base, c->multi_cnt,
                                                         c->part64, k, c->kst, c->fx_inv, c->S);
    SKM_LAUNCHED(c);
  }
  return SKM_OK;
}

}  // namespace

int64_t reduction_blocks(int64_t d) { return (d + kTB - 1) / kTB; }

int update_centers(skm_ctx* c) {
  int rc = SKM_OK;
  switch (c->dtype) {
    case SKM_F32: rc = center_sum_t<float>(c); break;
    case SKM_F16: rc = center_sum_t<__half>(c); break;
    case SKM_BF16: rc = center_sum_t<__nv_bfloat16>(c); break;
    default: return SKM_EINVAL;
  }
  if (rc) return rc;
  const int64_t nblk = reduction_blocks(c->d);
  dim3 grid((unsigned)nblk, (unsigned)((c->k + 31) / 32));
  SKM_PROF_BEGIN(c, "k_colnorm_part");
  k_colnorm_part<<<grid, dim3(32, 8), 0, c->st>>>(c->S, c->d, c->k, c->kst, c->red);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_colnorm_final");
  k_colnorm_final<<<1, 1024, 0, c->st>>>(c->red, nblk, c->k, c->kst, c->nrm, c->obj);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_normalize_drift");
  k_normalize_drift<<<grid, dim3(32, 8), 0, c->st>>>(c->S, c->Ct, c->nrm, c->d, c->k, c->kst, c->red);
  SKM_LAUNCHED(c);
  double* cnorm = c->nrm + c->kst;  // second half of the norm buffer: |c(j)| of the new centers
  SKM_PROF_BEGIN(c, "k_drift_final");
  k_drift_final<<<1, 1024, 0, c->st>>>(c->red, nblk, c->k, c->kst, c->d, c->pdn, c->pup, c->qup, cnorm, c->hsel);
  SKM_LAUNCHED(c);
  // the new centers become current
  float* tmp = c->Ct;
  c->Ct = c->S;
  c->S = tmp;
  if (c->variant == SKM_ELKAN || c->variant == SKM_HAMERLY) {
    const int64_t per = (c->d + c->gsplit - 1) / c->gsplit;
    const unsigned tk = (unsigned)((c->k + 31) / 32);
    SKM_PROF_BEGIN(c, "k_gram_part");
    k_gram_part<<<dim3(tk, tk, (unsigned)c->gsplit), dim3(32, 8), 0, c->st>>>(c->Ct, c->d, c->k, c->kst, per,
                                                                                c->gpart);
    SKM_LAUNCHED(c);
    // |error| of an FP32 sum of 256 products <= gamma_256 |c_i||c_j|, plus
    // the normalisation by FP64 norms of FP32 vectors.
    const double eg = 260.0 * 0x1.0p-24 / (1.0 - 260.0 * 0x1.0p-24) + 1e-12;
    SKM_PROF_BEGIN(c, "k_gram_final");
    k_gram_final<<<c->k, 256, 0, c->st>>>(c->gpart, c->gsplit, c->k, c->kst, cnorm, eg, c->cc, c->sc);
    SKM_LAUNCHED(c);
  }
  return SKM_OK;
}

}  // namespace skm
