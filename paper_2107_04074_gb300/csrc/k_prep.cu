// Data preparation (run once per context): CSR validation, row norms, the
// per-row similarity error bound, the term-major copy used by the center
// sum, the initial centers and center layout conversions.
#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kChunk = 1024;  // entries of a term handled by one warp in the center sum

// Warp per row: structure checks, 1/|x_i| (Section 5: rows are normalised)
// and delta_i, an upper bound on |computed - exact| of any similarity of row
// i: sequential FP32 FMA over m terms (gamma_m), the FP32 1/|x_i| and final
// product (2u), and centers whose norm is within 6u of 1 (FP32 normalisation
// by a compensated norm) -> (m+10)u/(1-(m+10)u).
template <typename VT>
__global__ void __launch_bounds__(256) k_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const VT* __restrict__ val, int64_t n, int64_t d,
                                              float* __restrict__ rinv, float* __restrict__ dlt,
                                              unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned err = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int64_t b = rp[i], e = rp[i + 1];
    if (i == 0 && b != 0) err |= E_ROWPTR;
    if (e < b) {
      err |= E_ROWPTR;
      continue;
    }
    double ss = 0.0;
    for (int64_t p = b + lane; p < e; p += 32) {
      const int32_t t = col[p];
      if (t < 0 || t >= d) err |= E_COLIDX;
      if (p > b && col[p - 1] >= t) err |= E_ORDER;
      const double v = (double)to_f32(val[p]);
      if (!isfinite(v)) err |= E_NONFINITE;
      ss = fma(v, v, ss);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(SKM_FULL_MASK, ss, o);
    if (lane == 0) {
      if (!(ss > 0.0)) err |= E_ZERO_ROW;
      if (!isfinite(ss)) err |= E_NONFINITE;
      rinv[i] = (ss > 0.0) ? __double2float_rn(1.0 / sqrt(ss)) : 0.f;
      const double m = (double)(e - b) + 10.0;
      const double g = m * 0x1.0p-24;
      dlt[i] = (g < 0.5) ? __double2float_ru(g / (1.0 - g)) : 1.f;
    }
  }
  err = __reduce_or_sync(SKM_FULL_MASK, err);
  if (lane == 0 && err) atomicOr(cnt + C_ERR, (unsigned long long)err);
}

// Dense rows: the same quantities with m = d.
template <typename VT>
__global__ void __launch_bounds__(256) k_rows_dense(const VT* __restrict__ X, int64_t n, int64_t d,
                                                    float* __restrict__ rinv, float* __restrict__ dlt,
                                                    unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned err = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    double ss = 0.0;
    for (int64_t t = lane; t < d; t += 32) {
      const double v = (double)to_f32(X[i * d + t]);
      if (!isfinite(v)) err |= E_NONFINITE;
      ss = fma(v, v, ss);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(SKM_FULL_MASK, ss, o);
    if (lane == 0) {
      if (!(ss > 0.0)) err |= E_ZERO_ROW;
      rinv[i] = (ss > 0.0) ? __double2float_rn(1.0 / sqrt(ss)) : 0.f;
      const double g = ((double)d + 10.0) * 0x1.0p-24;
      dlt[i] = (g < 0.5) ? __double2float_ru(g / (1.0 - g)) : 1.f;
    }
  }
  err = __reduce_or_sync(SKM_FULL_MASK, err);
  if (lane == 0 && err) atomicOr(cnt + C_ERR, (unsigned long long)err);
}

__global__ void k_term_count(const int32_t* __restrict__ col, int64_t nnz, unsigned long long* __restrict__ tc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(tc + col[p], 1ull);
}

// Batch: the columns of the term-major copy are (run, term) pairs, key =
// run * d + term, so that each run's center sums see only its own rows.
__global__ void __launch_bounds__(256) k_term_count_runs(const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, int64_t n,
                                                         const int32_t* __restrict__ row_run, int64_t d,
                                                         unsigned long long* __restrict__ tc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int64_t base = (int64_t)row_run[i] * d;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) atomicAdd(tc + base + col[p], 1ull);
  }
}

// Warp per row: place each entry, already normalised (x = v / |row|, FP32),
// in its term's column.  The order inside a column is arbitrary; the center
// sum is exact (fixed point), so the order cannot change any result.
template <typename VT>
__global__ void __launch_bounds__(256) k_scatter(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                 const VT* __restrict__ val, const float* __restrict__ rinv,
                                                 int64_t n, const int32_t* __restrict__ row_run, int64_t d,
                                                 unsigned long long* __restrict__ cursor,
                                                 int32_t* __restrict__ t_row, float* __restrict__ t_x) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const float ri = rinv[i];
    const int64_t base = row_run ? (int64_t)row_run[i] * d : 0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const unsigned long long pos = atomicAdd(cursor + base + col[p], 1ull);
      t_row[pos] = (int32_t)i;
      t_x[pos] = __fmul_rn(to_f32(val[p]), ri);
    }
  }
}

// Chunks per term (>= 1 so that every term writes its row of the sums) and
// partial slots for the terms with more than one chunk.
__global__ void k_chunk_counts(const int64_t* __restrict__ t_ptr, int64_t d, int64_t* __restrict__ nch,
                               int64_t* __restrict__ npart, int64_t* __restrict__ ismulti) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < d; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = t_ptr[t + 1] - t_ptr[t];
    const int64_t c = len > kChunk ? (len + kChunk - 1) / kChunk : 1;
    nch[t] = c;
    npart[t] = c > 1 ? c : 0;
    ismulti[t] = c > 1 ? 1 : 0;
  }
}

__global__ void k_chunk_fill(const int64_t* __restrict__ ch_ptr, const int64_t* __restrict__ pbase,
                             const int64_t* __restrict__ mpos, int64_t d, int32_t* __restrict__ ch_term,
                             int32_t* __restrict__ ch_idx, int64_t* __restrict__ ch_part,
                             int32_t* __restrict__ multi_term, int64_t* __restrict__ multi_base,
                             int32_t* __restrict__ multi_cnt) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < d; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c0 = ch_ptr[t], c = ch_ptr[t + 1] - c0;
    for (int64_t q = 0; q < c; ++q) {
      ch_term[c0 + q] = (int32_t)t;
      ch_idx[c0 + q] = (int32_t)q;
      ch_part[c0 + q] = c > 1 ? pbase[t] + q : -1;
    }
    if (c > 1) {
      const int64_t m = mpos[t];
      multi_term[m] = (int32_t)t;
      multi_base[m] = pbase[t];
      multi_cnt[m] = (int32_t)c;
    }
  }
}

// Exclusive scan of len int64 values by one block; out[len] = total.
__global__ void __launch_bounds__(1024) k_scan_i64(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                   int64_t len) {
  __shared__ int64_t sh[1024];
  const int tid = threadIdx.x;
  const int64_t per = (len + 1023) / 1024;
  const int64_t b = tid * per, e = min(len, b + per);
  int64_t s = 0;
#pragma unroll 8
  for (int64_t q = b; q < e; ++q) s += in[q];
  sh[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = tid >= off ? sh[tid - off] : 0;
    __syncthreads();
    sh[tid] += v;
    __syncthreads();
  }
  int64_t run = sh[tid] - s;
#pragma unroll 8
  for (int64_t q = b; q < e; ++q) {
    const int64_t v = in[q];
    out[q] = run;
    run += v;
  }
  if (tid == 1023) out[len] = sh[1023];
}

// Warp per center: c(j) = x(rows[j]) (Section 6: initial centers are random
// rows), written into the term-major array (zeroed before).
template <typename VT>
__global__ void k_init_centers(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const VT* __restrict__ val, const float* __restrict__ rinv,
                               const int64_t* __restrict__ rows, int32_t k, int64_t kst, float* __restrict__ Ct) {
  const int lane = threadIdx.x & 31;
  const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (j >= k) return;
  const int64_t r = rows[j];
  if (r < 0) return;  // padding column of a batch: stays zero
  const float ri = rinv[r];
  for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) Ct[(int64_t)col[p] * kst + j] = __fmul_rn(to_f32(val[p]), ri);
}

template <typename VT>
__global__ void k_init_centers_dense(const VT* __restrict__ X, int64_t d, const float* __restrict__ rinv,
                                     const int64_t* __restrict__ rows, int32_t k, int64_t kst,
                                     float* __restrict__ Ct) {
  const int lane = threadIdx.x & 31;
  const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (j >= k) return;
  const int64_t r = rows[j];
  const float ri = rinv[r];
  for (int64_t t = lane; t < d; t += 32) Ct[t * kst + j] = __fmul_rn(to_f32(X[r * d + t]), ri);
}

// Term-major d x kst  <->  row-major k x d, through a 32x32 shared tile.
__global__ void k_ct_to_rows(const float* __restrict__ Ct, int64_t d, int32_t k, int64_t kst, float* __restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (t < d && j < k) ? Ct[t * kst + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, t = t0 + threadIdx.x;
    if (j < k && t < d) out[j * d + t] = tile[threadIdx.x][r];
  }
}

__global__ void k_rows_to_ct(const float* __restrict__ in, int64_t d, int32_t k, int64_t kst, float* __restrict__ Ct) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = (j < k && t < d) ? in[j * d + t] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r, j = j0 + threadIdx.x;
    if (t < d && j < kst) Ct[t * kst + j] = tile[threadIdx.x][r];
  }
}

inline int grid_for(int64_t items, int per_block, int nsm, int max_per_sm = 16) {
  int64_t g = (items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)nsm * max_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename VT>
int prep_rows_t(skm_ctx* c) {
  if (c->layout == SKM_CSR) {
    k_rows<VT><<<grid_for(c->n * 32, 256, c->nsm), 256, 0, c->st>>>(c->rp, c->col, (const VT*)c->val, c->n, c->d,
                                                                     c->rinv, c->dlt, c->cnt);
  } else {
    k_rows_dense<VT><<<grid_for(c->n * 32, 256, c->nsm), 256, 0, c->st>>>((const VT*)c->val, c->n, c->d, c->rinv,
                                                                           c->dlt, c->cnt);
  }
  SKM_LAUNCH_CHECK();
  return SKM_OK;
}

template <typename VT>
int prep_transpose_t(skm_ctx* c) {
  cudaStream_t st = c->st;
  // columns: terms, or (run, term) pairs for a batch
  const int64_t d = c->d * (c->nruns > 0 ? c->nruns : 1), nnz = c->nnz;
  unsigned long long* tc = nullptr;
  int64_t *nch = nullptr, *npart = nullptr, *ism = nullptr, *ch_ptr = nullptr, *pbase = nullptr, *mpos = nullptr;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&tc, sizeof(unsigned long long) * (d + 1), st));
  SKM_CUDA_TRY(cudaMemsetAsync(tc, 0, sizeof(unsigned long long) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->t_ptr, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->t_row, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->t_val, sizeof(float) * (nnz > 0 ? nnz : 1), st));
  if (nnz > 0) {
    if (c->nruns > 0)
      k_term_count_runs<<<grid_for(c->n * 32, 256, c->nsm), 256, 0, st>>>(c->rp, c->col, c->n, c->row_run, c->d, tc);
    else
      k_term_count<<<grid_for(nnz, 256, c->nsm, 32), 256, 0, st>>>(c->col, nnz, tc);
    SKM_LAUNCH_CHECK();
  }
  k_scan_i64<<<1, 1024, 0, st>>>((const int64_t*)tc, c->t_ptr, d);
  SKM_LAUNCH_CHECK();
  SKM_CUDA_TRY(cudaMemcpyAsync(tc, c->t_ptr, sizeof(int64_t) * d, cudaMemcpyDeviceToDevice, st));
  k_scatter<VT><<<grid_for(c->n * 32, 256, c->nsm), 256, 0, st>>>(c->rp, c->col, (const VT*)c->val, c->rinv, c->n,
                                                                   c->nruns > 0 ? c->row_run : nullptr, c->d, tc,
                                                                   c->t_row, (float*)c->t_val);
  SKM_LAUNCH_CHECK();
  // chunk tables
  SKM_CUDA_TRY(cudaMallocAsync((void**)&nch, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&npart, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&ism, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&ch_ptr, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&pbase, sizeof(int64_t) * (d + 1), st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&mpos, sizeof(int64_t) * (d + 1), st));
  k_chunk_counts<<<grid_for(d, 256, c->nsm), 256, 0, st>>>(c->t_ptr, d, nch, npart, ism);
  SKM_LAUNCH_CHECK();
  k_scan_i64<<<1, 1024, 0, st>>>(nch, ch_ptr, d);
  SKM_LAUNCH_CHECK();
  k_scan_i64<<<1, 1024, 0, st>>>(npart, pbase, d);
  SKM_LAUNCH_CHECK();
  k_scan_i64<<<1, 1024, 0, st>>>(ism, mpos, d);
  SKM_LAUNCH_CHECK();
  int64_t tot[3];
  SKM_CUDA_TRY(cudaMemcpyAsync(&tot[0], ch_ptr + d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SKM_CUDA_TRY(cudaMemcpyAsync(&tot[1], pbase + d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SKM_CUDA_TRY(cudaMemcpyAsync(&tot[2], mpos + d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SKM_CUDA_TRY(cudaStreamSynchronize(st));
  c->nchunks = tot[0];
  c->nparts = tot[1];
  c->nmulti = tot[2];
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->ch_term, sizeof(int32_t) * c->nchunks, st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->ch_idx, sizeof(int32_t) * c->nchunks, st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->ch_part, sizeof(int64_t) * c->nchunks, st));
  const int64_t nm = c->nmulti > 0 ? c->nmulti : 1;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->multi_term, sizeof(int32_t) * nm, st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->multi_base, sizeof(int64_t) * nm, st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->multi_cnt, sizeof(int32_t) * nm, st));
  const int64_t kbins = c->nruns > 0 ? c->kmax : c->k;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&c->part64, sizeof(long long) * (c->nparts > 0 ? c->nparts : 1) * kbins, st));
  k_chunk_fill<<<grid_for(d, 256, c->nsm), 256, 0, st>>>(ch_ptr, pbase, mpos, d, c->ch_term, c->ch_idx, c->ch_part,
                                                          c->multi_term, c->multi_base, c->multi_cnt);
  SKM_LAUNCH_CHECK();
  cudaFreeAsync(tc, st);
  cudaFreeAsync(nch, st);
  cudaFreeAsync(npart, st);
  cudaFreeAsync(ism, st);
  cudaFreeAsync(ch_ptr, st);
  cudaFreeAsync(pbase, st);
  cudaFreeAsync(mpos, st);
  return SKM_OK;
}

}  // namespace

int prep_rows(skm_ctx* c) {
  switch (c->dtype) {
    case SKM_F32: return prep_rows_t<float>(c);
    case SKM_F16: return prep_rows_t<__half>(c);
    case SKM_BF16: return prep_rows_t<__nv_bfloat16>(c);
  }
  return SKM_EINVAL;
}

int prep_transpose(skm_ctx* c) {
  switch (c->dtype) {
    case SKM_F32: return prep_transpose_t<float>(c);
    case SKM_F16: return prep_transpose_t<__half>(c);
    case SKM_BF16: return prep_transpose_t<__nv_bfloat16>(c);
  }
  return SKM_EINVAL;
}

int scan_i64(cudaStream_t st, const int64_t* in, int64_t* out, int64_t len) {
  k_scan_i64<<<1, 1024, 0, st>>>(in, out, len);
  SKM_LAUNCH_CHECK();
  return SKM_OK;
}

template <typename VT>
static int init_centers_t(skm_ctx* c, const int64_t* rows_dev) {
  SKM_CUDA_TRY(cudaMemsetAsync(c->Ct, 0, sizeof(float) * c->d * c->kst, c->st));
  const int blocks = (c->k * 32 + 255) / 256;
  if (c->layout == SKM_CSR)
    k_init_centers<VT><<<blocks, 256, 0, c->st>>>(c->rp, c->col, (const VT*)c->val, c->rinv, rows_dev, c->k, c->kst,
                                                  c->Ct);
  else
    k_init_centers_dense<VT><<<blocks, 256, 0, c->st>>>((const VT*)c->val, c->d, c->rinv, rows_dev, c->k, c->kst,
                                                        c->Ct);
  SKM_LAUNCH_CHECK();
  return SKM_OK;
}

int init_centers(skm_ctx* c, const int64_t* rows_dev) {
  switch (c->dtype) {
    case SKM_F32: return init_centers_t<float>(c, rows_dev);
    case SKM_F16: return init_centers_t<__half>(c, rows_dev);
    case SKM_BF16: return init_centers_t<__nv_bfloat16>(c, rows_dev);
  }
  return SKM_EINVAL;
}

int centers_to_rows(skm_ctx* c, float* out) {
  dim3 g((unsigned)((c->d + 31) / 32), (unsigned)((c->k + 31) / 32));
  k_ct_to_rows<<<g, dim3(32, 8), 0, c->st>>>(c->Ct, c->d, c->k, c->kst, out);
  SKM_LAUNCH_CHECK();
  return SKM_OK;
}

int rows_to_centers(skm_ctx* c, const float* in) {
  dim3 g((unsigned)((c->d + 31) / 32), (unsigned)((c->kst + 31) / 32));
  k_rows_to_ct<<<g, dim3(32, 8), 0, c->st>>>(in, c->d, c->k, c->kst, c->Ct);
  SKM_LAUNCH_CHECK();
  return SKM_OK;
}

}  // namespace skm
