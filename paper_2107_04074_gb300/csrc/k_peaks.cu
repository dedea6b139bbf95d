// Peak arithmetic rates of this GPU, measured rather than quoted: the FP32
// and FP64 FMA roofs that the SIMT kernels of this library (the sparse
// similarity gathers, the FP32 dense GEMM, the FP64 drift sums) are reported
// against.  The paper has no counterpart; this is measurement support.
//
// Each thread runs 8 independent FMA chains (enough independent work to
// cover the pipeline latency with 8 warps per scheduler), the grid fills
// every SM 8 times over, and the chains' results are folded into one store
// so that none of the work can be dropped.  Time = CUDA events around one
// launch after a warm-up launch; rate = 2 FLOP per FMA.
#include "skm_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(int iters, T b, T c, T* __restrict__ out) {
  T a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == (T)-1.2345) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

// The same with packed FP32 FMAs (two lanes per instruction, each rounded as
// one FMA): one issue slot per two FMAs, so a kernel limited by issue rather
// than by the FP32 pipe can only reach the pipe's rate this way.
__global__ void __launch_bounds__(256) k_peak_fma2(int iters, float b, float c, float* __restrict__ out) {
  float2 a[kChains / 2];
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q)
    a[q] = make_float2((float)(threadIdx.x + 2 * q) * 1e-3f, (float)(threadIdx.x + 2 * q + 1) * 1e-3f);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int q = 0; q < kChains / 2; ++q) a[q] = __ffma2_rn(a[q], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains / 2; ++q) s += a[q].x + a[q].y;
  if (s == -1.2345f) out[blockIdx.x] = s;
}

// L2-resident gather rate at the whole-row kernel's granularity: every warp
// gathers rows of 416 bytes (26 lanes x 16 B: the center slice of one row
// entry at k = 100) at pseudo-random rows of a 20.8 MB table (50,000 rows:
// L2 keeps it, L1 does not), 16 rows in flight per warp at two 256-thread
// blocks per SM, and folds what it loaded into one store so that no load can
// be dropped.  Rate = 416 bytes per row gathered.
constexpr int kGatherRows = 50000;
constexpr int kGatherVec = 26;  // float4 per row
constexpr int kGatherInFlight = 16;

__global__ void __launch_bounds__(256, 2) k_peak_gather(const float4* __restrict__ tab, int iters,
                                                       float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t h = w * 2654435761u + 12345u;  // the same sequence in every lane of the warp
  float4 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int it = 0; it < iters; ++it) {
    uint32_t r[kGatherInFlight];
#pragma unroll
    for (int u = 0; u < kGatherInFlight; ++u) {
      h = h * 1664525u + 1013904223u;
      r[u] = (uint32_t)(((uint64_t)h * kGatherRows) >> 32);
    }
    float4 v[kGatherInFlight];
#pragma unroll
    for (int u = 0; u < kGatherInFlight; ++u)
      v[u] = lane < kGatherVec ? __ldg(tab + (size_t)r[u] * kGatherVec + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kGatherInFlight; ++u) {
      acc[u & 3].x += v[u].x;
      acc[u & 3].y += v[u].y;
      acc[u & 3].z += v[u].z;
      acc[u & 3].w += v[u].w;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += acc[q].x + acc[q].y + acc[q].z + acc[q].w;
  if (s == -1.2345f) out[blockIdx.x] = s;  // the table holds zeros: never true
}

int measure_gather(double* tbps, cudaStream_t st) {
  int dev = 0, nsm = 0;
  SKM_CUDA_TRY(cudaGetDevice(&dev));
  SKM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t tab_bytes = sizeof(float4) * (size_t)kGatherRows * kGatherVec;
  const unsigned grid = (unsigned)nsm * 2;
  const int iters = 4000;
  float4* tab = nullptr;
  float* out = nullptr;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&tab, tab_bytes, st));
  SKM_CUDA_TRY(cudaMallocAsync((void**)&out, sizeof(float) * grid, st));
  SKM_CUDA_TRY(cudaMemsetAsync(tab, 0, tab_bytes, st));
  cudaEvent_t e0, e1;
  SKM_CUDA_TRY(cudaEventCreate(&e0));
  SKM_CUDA_TRY(cudaEventCreate(&e1));
  for (int rep = 0; rep < 2; ++rep) {  // a warm-up launch (which also brings the table into L2), then the timed one
    if (rep == 1) SKM_CUDA_TRY(cudaEventRecord(e0, st));
    k_peak_gather<<<grid, 256, 0, st>>>(tab, iters, out);
    skm::note_launch();
  }
  SKM_CUDA_TRY(cudaEventRecord(e1, st));
  SKM_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  SKM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SKM_CUDA_TRY(cudaFreeAsync(tab, st));
  SKM_CUDA_TRY(cudaFreeAsync(out, st));
  SKM_CUDA_TRY(cudaStreamSynchronize(st));
  const double rows = (double)grid * 8.0 * (double)iters * kGatherInFlight;  // 8 warps per block
  *tbps = rows * 16.0 * kGatherVec / ((double)ms * 1e-3) / 1e12;
  return SKM_OK;
}

template <typename T, bool PACKED = false>
int measure(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, nsm = 0;
  SKM_CUDA_TRY(cudaGetDevice(&dev));
  SKM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  T* out = nullptr;
  const unsigned grid = (unsigned)nsm * 8;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&out, sizeof(T) * grid, st));
  cudaEvent_t e0, e1;
  SKM_CUDA_TRY(cudaEventCreate(&e0));
  SKM_CUDA_TRY(cudaEventCreate(&e1));
  const T b = (T)0.999999, c = (T)1e-7;
  for (int rep = 0; rep < 2; ++rep) {  // a warm-up launch, then the timed one
    if (rep == 1) SKM_CUDA_TRY(cudaEventRecord(e0, st));
    if constexpr (PACKED) k_peak_fma2<<<grid, 256, 0, st>>>(iters, (float)b, (float)c, (float*)out);
    else k_peak_fma<T><<<grid, 256, 0, st>>>(iters, b, c, out);
    skm::note_launch();
  }
  SKM_CUDA_TRY(cudaEventRecord(e1, st));
  SKM_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  SKM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SKM_CUDA_TRY(cudaFreeAsync(out, st));
  SKM_CUDA_TRY(cudaStreamSynchronize(st));
  const double fmas = (double)grid * 256.0 * (double)iters * kUnroll * kChains;
  *tflops = 2.0 * fmas / ((double)ms * 1e-3) / 1e12;
  return SKM_OK;
}

}  // namespace

extern "C" int skm_measure_peak(int32_t kind, double* tflops, void* stream) {
  if (!tflops) return SKM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == SKM_PEAK_FP32_FMA) return measure<float>(4096, tflops, st);
  if (kind == SKM_PEAK_FP64_FMA) return measure<double>(256, tflops, st);
  if (kind == SKM_PEAK_FP32_FMA2) return measure<float, true>(4096, tflops, st);
  if (kind == SKM_PEAK_L2_GATHER) return measure_gather(tflops, st);
  return SKM_EINVAL;
}
