// skm_assign_noalloc: the standard assignment step for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or under a strict memory budget, real-time
// services that must not allocate after start-up, and code recorded into a
// graph where allocation is not allowed.  For them this file keeps the only
// scratch the step needs -- a term-major copy of the centers and two
// counters -- in a file-scope static device array of fixed size.  Every GPU
// that loads the library holds that array until the process exits.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.  All calls on a device share the
// array and it keeps the last call's contents, so calls that overlap on the
// GPU (different streams, or different host threads) race: serialise them.
//
// The similarities are computed in the same order as k_rows_top2 and the row
// norms as in k_rows, so the labels equal those of skm_assign (standard).
#include <climits>
#include <mutex>

#include "skm_internal.cuh"

namespace {

constexpr int64_t kMaxCenterFloats = int64_t(1) << 22;  // d * round_up(k, 8) <= 4 Mi floats (16 MiB)
constexpr int kCounterFloats = 4;                        // two 64-bit counters

// [0, kMaxCenterFloats): term-major centers; then the counters.
static __device__ __align__(256) float g_noalloc_scratch[kMaxCenterFloats + kCounterFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return SKM_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return SKM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SKM_OK;
}

// row-major k x d centers -> term-major d x kst (padding columns zeroed);
// the grid walks the center tiles (y) with a stride, so any kst fits.
__global__ void k_na_transpose(const float* __restrict__ C, int64_t d, int32_t k, int64_t kst, float* __restrict__ Ct) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  for (int64_t j0 = (int64_t)blockIdx.y * 32; j0 < kst; j0 += (int64_t)gridDim.y * 32) {
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t j = j0 + r, t = t0 + threadIdx.x;
      tile[r][threadIdx.x] = (j < k && t < d) ? C[j * d + t] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t t = t0 + r, j = j0 + threadIdx.x;
      if (t < d && j < kst) Ct[t * kst + j] = tile[threadIdx.x][r];
    }
    __syncthreads();
  }
}

// Warp per row: 1/|x_i| computed in the row's own warp, then all k
// similarities and the argmax under the tie rule.  A row with a column index
// outside [0, d), a zero or non-finite norm (a NaN or an infinite value), or
// one whose similarities leave no best center (NaN centers) gets label -1 and
// raises the error counter.  The row is checked before any center value is
// gathered, so a bad column index is never dereferenced.
template <typename VT, int NT>
__global__ void __launch_bounds__(256) k_na_rows_top2(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const VT* __restrict__ val, int64_t n, int64_t d,
                                                      const float* __restrict__ Ct, int32_t k, int64_t kst,
                                                      int32_t* __restrict__ a, unsigned long long* __restrict__ cnt) {
  constexpr int KT = 32 * NT;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long my_changed = 0, my_err = 0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int64_t b = rp[i], e = rp[i + 1];
    double ss = 0.0;
    bool bad = false;
    for (int64_t p = b + lane; p < e; p += 32) {
      const double v = (double)skm::to_f32(val[p]);
      ss = fma(v, v, ss);
      const int32_t t = col[p];
      bad |= (t < 0 || (int64_t)t >= d);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(SKM_FULL_MASK, ss, o);
    bad = __any_sync(SKM_FULL_MASK, bad) || !(ss > 0.0) || !isfinite(ss) || e < b;
    const int32_t cur = a[i];
    if (bad) {
      if (lane == 0) {
        a[i] = -1;
        ++my_err;
        my_changed += (cur != -1);
      }
      continue;
    }
    const float ri = __double2float_rn(1.0 / sqrt(ss));
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
          vv = skm::to_f32(val[p0 + lane]);
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
    // no finite maximum (every similarity NaN): no label
    const bool none = (j1 == INT_MAX);
    const int32_t nb = none ? -1 : (cur >= 0 && cur < k && vcur == v1) ? cur : j1;
    if (lane == 0) {
      a[i] = nb;
      my_changed += (nb != cur);
      my_err += none ? 1 : 0;
    }
  }
  if (lane == 0) {
    if (my_changed) atomicAdd(cnt + 0, my_changed);
    if (my_err) atomicAdd(cnt + 1, my_err);
  }
}

template <typename VT, int NT>
void launch_na(const skm_data* x, const float* Ct, int32_t k, int64_t kst, int32_t* labels,
               unsigned long long* cnt, int nsm, cudaStream_t st) {
  int64_t g = (x->n * 32 + 255) / 256;
  if (g > (int64_t)nsm * 16) g = (int64_t)nsm * 16;
  if (g < 1) g = 1;
  k_na_rows_top2<VT, NT><<<(unsigned)g, 256, 0, st>>>(x->row_ptr, x->col_idx, (const VT*)x->values, x->n, x->d, Ct,
                                                      k, kst, labels, cnt);
}

template <typename VT>
void dispatch_na(const skm_data* x, const float* Ct, int32_t k, int64_t kst, int32_t* labels,
                 unsigned long long* cnt, int nsm, cudaStream_t st) {
  if (k <= 32) return launch_na<VT, 1>(x, Ct, k, kst, labels, cnt, nsm, st);
  if (k <= 64) return launch_na<VT, 2>(x, Ct, k, kst, labels, cnt, nsm, st);
  if (k <= 128) return launch_na<VT, 4>(x, Ct, k, kst, labels, cnt, nsm, st);
  if (k <= 256) return launch_na<VT, 8>(x, Ct, k, kst, labels, cnt, nsm, st);
  if (k <= 512) return launch_na<VT, 16>(x, Ct, k, kst, labels, cnt, nsm, st);
  return launch_na<VT, 32>(x, Ct, k, kst, labels, cnt, nsm, st);
}

}  // namespace

extern "C" int skm_assign_noalloc(const skm_data* x, int32_t k, const float* centers, int32_t* labels,
                                  int64_t* n_changed, void* stream) {
  if (!x || !centers || !labels || k < 1 || x->n < 1 || x->d < 1 || x->reserved != 0) return SKM_EINVAL;
  if (x->layout != SKM_CSR || x->memspace != SKM_DEVICE || !x->row_ptr || !x->col_idx || !x->values)
    return SKM_EINVAL;
  if (x->dtype < SKM_F32 || x->dtype > SKM_BF16) return SKM_EINVAL;
  if (x->d > INT32_MAX || x->n > INT32_MAX) return SKM_ETOOBIG;
  const int64_t kst = ((int64_t)k + 7) / 8 * 8;
  if (x->d > kMaxCenterFloats || x->d * kst > kMaxCenterFloats) return SKM_ETOOBIG;
  float* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != SKM_OK) return rc;
  float* Ct = base;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(base + kMaxCenterFloats);
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 1;
  SKM_CUDA_TRY(cudaGetDevice(&dev));
  SKM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // the counters keep the previous call's values: clear them
  SKM_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
  const int64_t gy = (kst + 31) / 32;
  dim3 g((unsigned)((x->d + 31) / 32), (unsigned)(gy < 65535 ? gy : 65535));
  k_na_transpose<<<g, dim3(32, 8), 0, st>>>(centers, x->d, k, kst, Ct);
  skm::note_launch();
  if (cudaPeekAtLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SKM_ECUDA;
  }
  switch (x->dtype) {
    case SKM_F32: dispatch_na<float>(x, Ct, k, kst, labels, cnt, nsm, st); break;
    case SKM_F16: dispatch_na<__half>(x, Ct, k, kst, labels, cnt, nsm, st); break;
    default: dispatch_na<__nv_bfloat16>(x, Ct, k, kst, labels, cnt, nsm, st); break;
  }
  skm::note_launch();
  if (cudaPeekAtLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SKM_ECUDA;
  }
  if (n_changed) {
    unsigned long long h[2] = {0, 0};
    SKM_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
    SKM_CUDA_TRY(cudaStreamSynchronize(st));
    *n_changed = (int64_t)h[0];
    if (h[1]) return SKM_EINVAL;
  }
  return SKM_OK;
}
