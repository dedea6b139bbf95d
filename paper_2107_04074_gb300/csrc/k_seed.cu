// Spherical k-means++ seeding (Section 5.6): the first center is a row drawn
// uniformly, each further center a row drawn with probability proportional to
// 1 - max_c <x(i), c> over the centers chosen so far (the analogue of the
// squared Euclidean distance of k-means++), the maximum cached per row so the
// whole seeding costs O(nk) similarities.
//
// The uniform draws u_0 .. u_{k-1} in [0, 1) are inputs.  Discrete rule: the
// first row is floor(u_0 n); the weights are quantised to integers
// q_i = round((1 - m_i) 2^40) (0 when negative), W = sum q_i, T = floor(u_j W),
// and the chosen row is the first whose inclusive prefix sum of q exceeds T;
// integer sums make the choice independent of summation order.  If W = 0
// (every row already equals a center) the first row not chosen yet is taken.
//
// Each chosen row becomes its center column of the term-major array Ct, the
// same values k_init_centers writes, and the similarities use the canonical
// FP32 chain of the assignment kernels.
//   k_seed_column  center column j <- row rows[j] (normalised), also as a
//                  contiguous vector
//   k_seed_sims    m_i = max(m_i, <x_i, c_j>), q_i, block sums (dense rows: a
//                  warp per row; CSR rows: k_seed_sims_lane, a lane per row)
//   k_seed_pick    one block: W, T, the chosen row for column j + 1
//   k_seed_finish  bound pre-initialisation (the remark of Section 5.6 and
//                  the outlook of Section 7): the seeding's similarities are
//                  those of the first assignment from the seeded centers, so
//                  the similarity passes also keep each row's best center,
//                  its best and second best similarity and (Elkan) every
//                  u(i,j), and this kernel installs the labels and bounds --
//                  the first assignment without another pass over the data.
#include <climits>

#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kSeedRows = 64;  // rows per block of k_seed_sims (8 per warp)

// Also writes the center as a contiguous vector cvec (d values, all zero but
// the current center's terms for CSR data), which the similarity pass gathers
// from: nearby terms share its cache lines, unlike the strided column of Ct.
template <typename VT>
__global__ void k_seed_column(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const VT* __restrict__ val, const float* __restrict__ rinv, int64_t n, int64_t d,
                              int dense, int64_t kst, int j, const int64_t* __restrict__ rows, float* __restrict__ Ct,
                              float* __restrict__ cvec) {
  const int64_t r = rows[j];
  if (r < 0 || r >= n) return;  // not reachable: the pick always finds a row
  const float ri = rinv[r];
  if (dense) {
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
      const float v = __fmul_rn(to_f32(val[r * d + t]), ri);
      Ct[t * kst + j] = v;
      cvec[t] = v;
    }
  } else {
    // clear the previous center's entries of the vector, then write this one
    if (j > 0) {
      const int64_t r0 = rows[j - 1];
      if (r0 >= 0 && r0 < n)
        for (int64_t p = rp[r0] + threadIdx.x; p < rp[r0 + 1]; p += blockDim.x) cvec[col[p]] = 0.f;
      __syncthreads();
    }
    for (int64_t p = rp[r] + threadIdx.x; p < rp[r + 1]; p += blockDim.x) {
      const float v = __fmul_rn(to_f32(val[p]), ri);
      Ct[(int64_t)col[p] * kst + j] = v;
      cvec[col[p]] = v;
    }
  }
}

// Canonical dense similarity chain (t in order) against center column j.
template <typename VT>
__device__ __forceinline__ float warp_dot_dense_col(const VT* __restrict__ x, int64_t d,
                                                    const float* __restrict__ Ct, int64_t kst, int j) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (int64_t t0 = 0; t0 < d; t0 += 32) {
    const float xv = (t0 + lane < d) ? to_f32(x[t0 + lane]) : 0.f;
    const float cv = (t0 + lane < d) ? __ldg(Ct + (t0 + lane) * kst + j) : 0.f;
    const int nq = (int)min((int64_t)32, d - t0);
    for (int q = 0; q < nq; ++q)
      acc = __fmaf_rn(__shfl_sync(SKM_FULL_MASK, xv, q), __shfl_sync(SKM_FULL_MASK, cv, q), acc);
  }
  return acc;
}

// What the similarity passes keep for the first assignment (all pointers
// NULL: plain seeding).  Over the centers in the order they are chosen, each
// row keeps its best similarity (m, the seeding's own maximum), the lowest
// center index reaching it (best) and the second best (second, the largest
// of the others: equal to m on a tie); Elkan's u(i,j) = s_ij + delta_i
// rounded up goes to uelk[i si + j sj]: a center-major staging array (si = 1,
// sj = n: the pass over center j writes one contiguous row, coalesced), later
// transposed into the row-major bounds, or the bounds themselves (si = their
// row stride, sj = 1) when the staging array would exceed kSeedStageBytes.
struct SeedTrack {
  int32_t* best;
  float* second;
  float* uelk;
  int64_t si, sj;
  const float* dlt;
};
constexpr int64_t kSeedStageBytes = int64_t(2) << 30;

__device__ __forceinline__ void seed_track(const SeedTrack& tr, int64_t i, int j, float sim, float m_old) {
  if (!tr.best) return;
  if (j == 0) {
    tr.best[i] = 0;
    tr.second[i] = -INFINITY;
  } else if (sim > m_old) {
    tr.second[i] = m_old;
    tr.best[i] = j;
  } else if (sim > tr.second[i]) {
    tr.second[i] = sim;
  }
  if (tr.uelk) tr.uelk[i * tr.si + j * tr.sj] = __fadd_ru(sim, tr.dlt[i]);
}

template <typename VT>
__global__ void __launch_bounds__(256) k_seed_sims(int64_t n, int64_t d, int dense, const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                   const float* __restrict__ rinv, const float* __restrict__ Ct,
                                                   int64_t kst, int jc, int j, float* __restrict__ m,
                                                   long long* __restrict__ q, long long* __restrict__ bsum,
                                                   SeedTrack tr) {
  __shared__ long long wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long s = 0;
  for (int u = 0; u < kSeedRows / 8; ++u) {
    const int64_t i = (int64_t)blockIdx.x * kSeedRows + warp * (kSeedRows / 8) + u;
    if (i >= n) break;
    float dot;
    if (dense) dot = warp_dot_dense_col<VT>(val + i * d, d, Ct, kst, jc);
    else dot = warp_dot_one<VT>(rp[i], rp[i + 1], col, val, Ct, kst, jc);
    const float sim = __fmul_rn(dot, rinv[i]);
    if (lane == 0) {
      seed_track(tr, i, j, sim, m[i]);
      const float mi = j == 0 ? sim : fmaxf(m[i], sim);
      m[i] = mi;
      long long qi = __double2ll_rn((1.0 - (double)mi) * 0x1.0p40);
      if (qi < 0) qi = 0;
      q[i] = qi;
      s += qi;
    }
  }
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    bsum[blockIdx.x] = t;
  }
}

// CSR rows, a lane per row (32 rows per warp, kSeedRowsLane per block): the
// lane walks its row entry by entry -- four entries' columns, values and
// center values loaded together -- so that many short FMA chains run side by
// side instead of one warp-wide chain per row; the chain is the canonical one
// (CSR order from 0), so the similarities equal warp_dot_one's.
constexpr int kSeedRowsLane = 256;

template <typename VT>
__global__ void __launch_bounds__(256) k_seed_sims_lane(int64_t n, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                        const float* __restrict__ rinv,
                                                        const float* __restrict__ cvec, int j,
                                                        float* __restrict__ m, long long* __restrict__ q,
                                                        long long* __restrict__ bsum, SeedTrack tr) {
  __shared__ long long wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kSeedRowsLane + threadIdx.x;
  long long qi = 0;
  if (i < n) {
    const int64_t b = rp[i], e = rp[i + 1];
    float acc = 0.f;
    int64_t p = b;
    for (; p + 4 <= e; p += 4) {
      int t[4];
      float x[4], c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        t[u] = __ldg(col + p + u);
        x[u] = to_f32(val[p + u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = __ldg(cvec + t[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = __fmaf_rn(x[u], c[u], acc);
    }
    for (; p < e; ++p) acc = __fmaf_rn(to_f32(val[p]), __ldg(cvec + __ldg(col + p)), acc);
    const float sim = __fmul_rn(acc, rinv[i]);
    seed_track(tr, i, j, sim, m[i]);
    const float mi = j == 0 ? sim : fmaxf(m[i], sim);
    m[i] = mi;
    qi = __double2ll_rn((1.0 - (double)mi) * 0x1.0p40);
    if (qi < 0) qi = 0;
    q[i] = qi;
  }
  long long s = qi;
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(SKM_FULL_MASK, s, o);
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_seed_pick(const long long* __restrict__ bsum, int64_t nblk,
                                                    int64_t rows_per_block, const long long* __restrict__ q,
                                                    int64_t n, double u, int64_t* __restrict__ rows, int j) {
  __shared__ long long part[1024];
  __shared__ long long total, target, before;
  __shared__ int owner;
  __shared__ int64_t found;
  const int tid = threadIdx.x;
  const int64_t per = (nblk + 1023) / 1024;
  const int64_t b0 = tid * per, b1 = min(nblk, b0 + per);
  long long s = 0;
  for (int64_t b = b0; b < b1; ++b) s += bsum[b];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    long long t = 0;
    for (int w = 0; w < 1024; ++w) t += part[w];
    total = t;
    long long T = (long long)(u * (double)t);
    if (T >= t) T = t - 1;
    target = T;
    found = -1;
    owner = -1;
    long long acc = 0;
    for (int w = 0; w < 1024 && t > 0; ++w) {
      if (T < acc + part[w]) {
        owner = w;
        before = acc;
        break;
      }
      acc += part[w];
    }
  }
  __syncthreads();
  if (total <= 0) {
    // every row equals a chosen center: the first row not chosen yet
    if (tid == 0) {
      for (int64_t i = 0; i < n && found < 0; ++i) {
        bool taken = false;
        for (int c = 0; c < j && !taken; ++c) taken = rows[c] == i;
        if (!taken) found = i;
      }
      rows[j] = found < 0 ? 0 : found;
    }
    return;
  }
  // the owner thread walks its blocks, then the rows of the block that holds the target
  if (tid == owner) {
    long long acc = before;
    for (int64_t b = b0; b < b1; ++b) {
      if (target < acc + bsum[b]) {
        const int64_t r0 = b * rows_per_block, r1 = min(n, r0 + rows_per_block);
        for (int64_t i = r0; i < r1; ++i) {
          acc += q[i];
          if (acc > target) {
            found = i;
            break;
          }
        }
        break;
      }
      acc += bsum[b];
    }
    rows[j] = found;
  }
}

// The staged bounds (center-major, k x n) into the row-major bound array
// (n x kst): 32 x 32 tiles through shared memory, both sides coalesced.
__global__ void k_seed_stage_out(const float* __restrict__ ucol, int64_t n, int32_t k, int64_t kst,
                                 float* __restrict__ ub) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (j < k && i < n) tile[r][threadIdx.x] = ucol[j * n + i];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < k) ub[i * kst + j] = tile[threadIdx.x][r];
  }
}

// Thread per row: the first assignment from the seeding's similarities, as
// k_rows_top2 leaves it (no label was current, so every label changes):
// a(i) = best, l(i) = s1 - delta rounded down, Hamerly's u(i) = s2 + delta
// rounded up (-1 with one center); the counters count n changed labels and
// n k similarities.
__global__ void __launch_bounds__(256) k_seed_finish(int64_t n, int32_t k, const float* __restrict__ m,
                                                     const int32_t* __restrict__ best,
                                                     const float* __restrict__ second,
                                                     const float* __restrict__ dlt, int32_t* __restrict__ a,
                                                     float* __restrict__ lb, float* __restrict__ ub_one,
                                                     unsigned long long* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    a[i] = best[i];
    const float dl = dlt[i];
    if (lb) lb[i] = __fsub_rd(m[i], dl);
    if (ub_one) ub_one[i] = (k > 1) ? __fadd_ru(second[i], dl) : -1.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt[C_CHANGED] = (unsigned long long)n;
    cnt[C_SIMS] = (unsigned long long)n * (unsigned long long)k;
  }
}

template <typename VT>
int seed_t(skm_ctx* c, const double* u, int64_t* rows_host, SeedFirst* first) {
  const int64_t n = c->n, d = c->d, kst = c->kst;
  const int k = c->k;
  const int dense = c->layout == SKM_DENSE;
  const int64_t rpb = dense ? kSeedRows : kSeedRowsLane;  // rows per block of the similarity pass
  const int64_t nblk = (n + rpb - 1) / rpb;
  float *m = nullptr, *cvec = nullptr;
  long long *q = nullptr, *bsum = nullptr;
  int64_t* rows = nullptr;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&m, sizeof(float) * n, c->st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&cvec, sizeof(float) * d, c->st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&q, sizeof(long long) * n, c->st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&bsum, sizeof(long long) * nblk, c->st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&rows, sizeof(int64_t) * k, c->st));
  SeedTrack tr = {nullptr, nullptr, nullptr, 0, 0, nullptr};
  float* ucol = nullptr;  // center-major staging of Elkan's bounds
  if (first) {
    SKM_CUDA_TRY(cudaMallocAsync((void**)&tr.best, sizeof(int32_t) * n, c->st));
    SKM_CUDA_TRY(cudaMallocAsync((void**)&tr.second, sizeof(float) * n, c->st));
    if (first->elkan) {
      if ((int64_t)sizeof(float) * k * n <= kSeedStageBytes &&
          cudaMallocAsync((void**)&ucol, sizeof(float) * k * n, c->st) == cudaSuccess) {
        tr.uelk = ucol;
        tr.si = 1;
        tr.sj = n;
      } else {
        (void)cudaGetLastError();
        ucol = nullptr;
        tr.uelk = c->ub;
        tr.si = kst;
        tr.sj = 1;
      }
    }
    tr.dlt = c->dlt;
  }
  SKM_CUDA_TRY(cudaMemsetAsync(c->Ct, 0, sizeof(float) * d * kst, c->st));
  int64_t r0 = (int64_t)(u[0] * (double)n);
  if (r0 >= n) r0 = n - 1;
  rows_host[0] = r0;
  SKM_CUDA_TRY(cudaMemcpyAsync(rows, rows_host, sizeof(int64_t), cudaMemcpyHostToDevice, c->st));
  const VT* v = (const VT*)c->val;
  if (!dense) SKM_CUDA_TRY(cudaMemsetAsync(cvec, 0, sizeof(float) * d, c->st));
  for (int j = 0; j < k; ++j) {
    k_seed_column<VT><<<1, 256, 0, c->st>>>(c->rp, c->col, v, c->rinv, n, d, dense, kst, j, rows, c->Ct, cvec);
    SKM_LAUNCH_CHECK();
    // the last center's similarities are needed only for the first assignment
    if (j + 1 == k && !first) break;
    // the similarities to center j, read from its contiguous copy (the same
    // FP32 values as column j of Ct)
    if (dense)
      k_seed_sims<VT><<<(unsigned)nblk, 256, 0, c->st>>>(n, d, dense, c->rp, c->col, v, c->rinv, cvec, 1, 0, j, m,
                                                         q, bsum, tr);
    else
      k_seed_sims_lane<VT><<<(unsigned)nblk, 256, 0, c->st>>>(n, c->rp, c->col, v, c->rinv, cvec, j, m, q, bsum,
                                                              tr);
    SKM_LAUNCH_CHECK();
    if (j + 1 == k) break;
    k_seed_pick<<<1, 1024, 0, c->st>>>(bsum, nblk, rpb, q, n, u[j + 1], rows, j + 1);
    SKM_LAUNCH_CHECK();
  }
  SKM_CUDA_TRY(cudaMemcpyAsync(rows_host, rows, sizeof(int64_t) * k, cudaMemcpyDeviceToHost, c->st));
  if (ucol) {
    k_seed_stage_out<<<dim3((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32)), dim3(32, 8), 0, c->st>>>(
        ucol, n, k, kst, c->ub);
    SKM_LAUNCH_CHECK();
    cudaFreeAsync(ucol, c->st);
  }
  if (first) {
    // handed to seed_finish, which frees them
    first->m = m;
    first->best = tr.best;
    first->second = tr.second;
    m = nullptr;
  }
  if (m) cudaFreeAsync(m, c->st);
  cudaFreeAsync(cvec, c->st);
  cudaFreeAsync(q, c->st);
  cudaFreeAsync(bsum, c->st);
  cudaFreeAsync(rows, c->st);
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  return SKM_OK;
}

}  // namespace

int seed_kmeanspp(skm_ctx* c, const double* u, int64_t* rows_host, SeedFirst* first) {
  switch (c->dtype) {
    case SKM_F32: return seed_t<float>(c, u, rows_host, first);
    case SKM_F16: return seed_t<__half>(c, u, rows_host, first);
    case SKM_BF16: return seed_t<__nv_bfloat16>(c, u, rows_host, first);
  }
  return SKM_EINVAL;
}

// After the context restarted from the seeded rows: install the first
// assignment kept by the seeding (labels; l for every variant that keeps
// it; Hamerly's single u; Elkan's u(i,j) were written during the seeding)
// and free the seeding's per-row buffers.
int seed_finish(skm_ctx* c, SeedFirst* first) {
  const int64_t g = (c->n + 255) / 256, gcap = (int64_t)c->nsm * 16;
  SKM_PROF_BEGIN(c, "k_seed_finish");
  k_seed_finish<<<(unsigned)(g < gcap ? g : gcap), 256, 0, c->st>>>(c->n, c->k, first->m, first->best,
                                                                    first->second, c->dlt, c->a,
                                                                    first->keep_l ? c->lb : nullptr,
                                                                    first->keep_u ? c->ub : nullptr, c->cnt);
  SKM_LAUNCHED(c);
  cudaFreeAsync(first->m, c->st);
  cudaFreeAsync(first->best, c->st);
  cudaFreeAsync(first->second, c->st);
  return SKM_OK;
}

}  // namespace skm
