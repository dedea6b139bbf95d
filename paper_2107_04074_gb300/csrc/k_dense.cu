// Dense rows (embedding-like data): the same Lloyd iteration as the sparse
// path, with the similarity bulk as a GEMM.
//
// Canonical dense similarity: s_ij = fl32(fl32_seq(sum_{t=0..d-1} x_it c_jt)
// * 1/|x_i|), a sequential FP32 FMA chain over t in order.  k_dense_top2 (a
// tiled SIMT GEMM) accumulates every output exactly in that order, and so do
// k_dense_tighten and the FP32 recheck, so all paths agree bit for bit.
//
//   k_dense_bf16        unit rows rounded to BF16 (A operand of k_bf16_topk)
//   k_dense_fp8         unit rows scaled by a power of two and rounded to
//                       FP8-E4M3 (the A operand of the FP8 form)
//   k_dense_centers     term-major FP32 centers -> row-major FP32 and BF16
//                       (or FP8-E4M3 of 2^8 c)
//   k_dense_top2        FP32 GEMM + fused top-2 (plain FP32 path, whole rows
//                       for Hamerly, recheck of ambiguous rows)
//   k_dense_classify    precision form: the BF16 top-2 decides the label when its
//                       margin exceeds the error bound, else the row is rechecked
//   k_dense_cands       precision form: FP32 recheck of an ambiguous row against
//                       the BF16 candidates that can still win
//   k_dense_tighten     Hamerly: exact <x, c_a> (warp per survivor)
//   k_label_*, k_dense_cluster_sum, k_dense_delta
//                       exact fixed-point cluster sums: full (rows sorted by
//                       label) or only the rows whose label changed
#include <cuda_fp8.h>

#include <climits>

#include "skm_internal.cuh"

namespace skm {

namespace {

// Sum over a warp, each step rounded up (an upper bound for terms >= 0).
__device__ __forceinline__ float warp_sum_up(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(SKM_FULL_MASK, v, o));
  return v;
}

// Xb = bf16(y_i), y_i = fl(x_i * rinv_i) (a warp per row), and
// exr_i >= |Xb_i - x_i/|x_i||.  The BF16 rounding error y - bf16(y) of an
// FP32 value is exact in FP32, and its squares are summed with every step
// rounded up; y_i itself is within 2^-23 (1 + (d + 8) 2^-30) of the exact
// unit row (one rounding of each product, one of rinv from an FP64 norm of d
// squares), added at the end.
__global__ void k_dense_bf16(const float* __restrict__ X, const float* __restrict__ rinv, int64_t n, int64_t d,
                             __nv_bfloat16* __restrict__ Xb, float* __restrict__ exr) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float yerr = __fmul_ru(0x1.0p-23f, __fadd_ru(1.f, __fmul_ru((float)(d + 8), 0x1.0p-30f)));
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const float ri = rinv[i];
    float e2 = 0.f;
    for (int64_t t = lane; t < d; t += 32) {
      const float y = __fmul_rn(X[i * d + t], ri);
      const __nv_bfloat16 b = __float2bfloat16_rn(y);
      Xb[i * d + t] = b;
      const float e = __fsub_rn(y, __bfloat162float(b));  // exact
      e2 = __fmaf_ru(e, e, e2);
    }
    e2 = warp_sum_up(e2);
    if (lane == 0) exr[i] = __fadd_ru(__fsqrt_ru(e2), yerr);
  }
}

// E4M3 rounding (to nearest even; no saturation is reached: callers keep
// |v| < 256) and its exact value as FP32.
__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(uint8_t q) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3)));
}

// Xq = e4m3(y_i 2^e_i), y_i = fl(x_i * rinv_i) (a warp per row), with the
// power of two 2^e_i chosen from the row's largest |y|, m in [2^q, 2^(q+1)):
// e_i = 7 - q puts every scaled entry below 256 (no saturation) and the
// largest at or above 128.  rsc_i = 2^-(e_i + 8) turns an accumulator of the
// row against centers scaled by 2^8 back into a similarity, exactly.
// exr_i >= |Xq_i 2^-e_i - x_i/|x_i||: y - e4m3(y 2^e) 2^-e is exact in FP32
// (the difference between a float and its rounding to a coarser
// power-of-two grid), its squares are summed rounding up, and y's own error
// is added as in k_dense_bf16.
__global__ void k_dense_fp8(const float* __restrict__ X, const float* __restrict__ rinv, int64_t n, int64_t d,
                            uint8_t* __restrict__ Xq, float* __restrict__ exr, float* __restrict__ rsc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float yerr = __fmul_ru(0x1.0p-23f, __fadd_ru(1.f, __fmul_ru((float)(d + 8), 0x1.0p-30f)));
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const float ri = rinv[i];
    float m = 0.f;
    for (int64_t t = lane; t < d; t += 32) m = fmaxf(m, fabsf(__fmul_rn(X[i * d + t], ri)));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(SKM_FULL_MASK, m, o));
    // unit rows: m >= 1/sqrt(d) is a normal float, q = its exponent
    const int q = (int)((__float_as_uint(m) >> 23) & 0xFF) - 127;
    const int e = 7 - q;
    const float sc = ldexpf(1.f, e), isc = ldexpf(1.f, -e);
    float e2 = 0.f;
    for (int64_t t = lane; t < d; t += 32) {
      const float y = __fmul_rn(X[i * d + t], ri);
      const uint8_t b = to_e4m3(__fmul_rn(y, sc));  // y * 2^e is exact
      Xq[i * d + t] = b;
      const float err = __fsub_rn(y, __fmul_rn(from_e4m3(b), isc));  // exact
      e2 = __fmaf_ru(err, err, e2);
    }
    e2 = warp_sum_up(e2);
    if (lane == 0) {
      exr[i] = __fadd_ru(__fsqrt_ru(e2), yerr);
      rsc[i] = ldexpf(1.f, -(e + 8));
    }
  }
}

// ec_j = |bf16(c_j) - c_j| for every center (a warp each; the differences
// are exact in FP32, their squares summed rounding up), reduced to
// E_c = max_j ec_j (float bits compare as unsigned for values >= 0); the
// last block to finish writes ebc = {1 + 6u + E_c, E_c + 1.02 (d + 16) 2^-23}
// rounded up -- the per-row bound's center terms: |c_j| <= 1 + 6u, and the
// FP32 accumulation of d products adds at most 2^-23 of the running sum of
// |products| <= (1 + ex_i)(1 + 6u + E_c) < 1.02 per step (reading TC) --
// and zeroes the max and the counter for the next launch.
__global__ void __launch_bounds__(256) k_center_err(const float* __restrict__ Cr, const __nv_bfloat16* __restrict__ Cb,
                                                    int64_t d, int32_t k, unsigned* __restrict__ ebw,
                                                    float* __restrict__ ebc) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j < k) {
    float e2 = 0.f;
    for (int64_t t = lane; t < d; t += 32) {
      const float e = __fsub_rn(Cr[j * d + t], __bfloat162float(Cb[j * d + t]));  // exact
      e2 = __fmaf_ru(e, e, e2);
    }
    e2 = warp_sum_up(e2);
    if (lane == 0) {
      atomicMax(ebw, __float_as_uint(__fsqrt_ru(e2)));
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ebw + 1, 1u) == gridDim.x - 1) {
      __threadfence();
      const double ec = (double)__uint_as_float(atomicExch(ebw, 0u));
      ebc[0] = __double2float_ru(__dadd_ru(1.0 + 6.0 * 0x1.0p-24, ec));
      ebc[1] = __double2float_ru(__dadd_ru(ec, ((double)d + 16.0) * 0x1.0p-23 * 1.02));
      atomicExch(ebw + 1, 0u);
    }
  }
}

// The same for the FP8 centers e4m3(2^8 c_j): ec_j = |e4m3(2^8 c_j) 2^-8 - c_j|
// (exact differences); the accumulation term uses 1.25 >= (1 + ex_i)(1 + 6u +
// E_c): an E4M3 rounding of a normal value errs by at most 2^-4 of it, and a
// subnormal one (scaled magnitude below 2^-6) by at most 2^-10 of the scale,
// so ex_i, E_c < 0.063 for unit rows and centers.
__global__ void __launch_bounds__(256) k_center_err_fp8(const float* __restrict__ Cr, const uint8_t* __restrict__ Cq,
                                                        int64_t d, int32_t k, unsigned* __restrict__ ebw,
                                                        float* __restrict__ ebc) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j < k) {
    float e2 = 0.f;
    for (int64_t t = lane; t < d; t += 32) {
      const float e = __fsub_rn(Cr[j * d + t], __fmul_rn(from_e4m3(Cq[j * d + t]), 0x1.0p-8f));  // exact
      e2 = __fmaf_ru(e, e, e2);
    }
    e2 = warp_sum_up(e2);
    if (lane == 0) {
      atomicMax(ebw, __float_as_uint(__fsqrt_ru(e2)));
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ebw + 1, 1u) == gridDim.x - 1) {
      __threadfence();
      const double ec = (double)__uint_as_float(atomicExch(ebw, 0u));
      ebc[0] = __double2float_ru(__dadd_ru(1.0 + 6.0 * 0x1.0p-24, ec));
      ebc[1] = __double2float_ru(__dadd_ru(ec, ((double)d + 16.0) * 0x1.0p-23 * 1.25));
      atomicExch(ebw + 1, 0u);
    }
  }
}

__global__ void k_bf16_eps_rows(const float* __restrict__ exr, const float* __restrict__ ebc, int64_t n,
                                float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = bf16_eps(exr, ebc, i);
}

// Ct (d x kst, term-major) -> Cr (k x d FP32) and Cb (kpad x d BF16, zero
// rows past k) or Cq (kpad x d FP8-E4M3 of 2^8 c), through 32 x 32 shared
// tiles.
__global__ void k_dense_centers(const float* __restrict__ Ct, int64_t d, int32_t k, int64_t kst, int32_t kpad,
                                float* __restrict__ Cr, __nv_bfloat16* __restrict__ Cb, uint8_t* __restrict__ Cq) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (t < d && j < k) ? Ct[t * kst + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, t = t0 + threadIdx.x;
    if (t < d && j < kpad) {
      const float v = tile[threadIdx.x][r];
      if (j < k) Cr[j * d + t] = v;
      if (Cb) Cb[j * d + t] = __float2bfloat16_rn(v);
      if (Cq) Cq[j * d + t] = to_e4m3(__fmul_rn(v, 0x1.0p8f));
    }
  }
}

// FP32 GEMM with fused top-2.  CTA: 128 rows x all centers (tiles of 128),
// 256 threads (16 x 16), each thread 8 rows x 8 centers (trow: two runs of 4,
// 64 apart, so that the 16 threads of a row group read consecutive 16-byte
// words of a shared-memory tile row, free of bank conflicts), K in chunks of 32
// through shared memory, double-buffered: the asynchronous copies of the next
// chunk (4-byte cp.async into the transposed tiles, zero-filled outside the
// data) are in flight while this one is multiplied.  Rows: all (list ==
// nullptr) or list[0..*list_cnt).  MODE 0: labels only; MODE 1: also
// Hamerly's l = s1 - delta, u = s2 + delta.  Two blocks per SM (128
// registers): the running top-2 of each thread's rows lives in shared memory.
constexpr int kTR = 128, kTC = 128, kKC = 32;

// The tile row (or center) of a thread's x-th row: 4 consecutive ones at
// 4 g, then 4 more at 64 + 4 g.
__device__ __forceinline__ int trow(int g, int x) { return (x < 4 ? 0 : 60) + g * 4 + x; }
constexpr size_t kDenseSmem = sizeof(float) * 2 * kKC * (kTR + 4) * 2;

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(in ? 4 : 0)
               : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) k_dense_top2(const float* __restrict__ X, const float* __restrict__ rinv,
                                                       const float* __restrict__ dlt, const float* __restrict__ Cr,
                                                       int64_t n, int64_t d, int32_t k,
                                                       const int32_t* __restrict__ list,
                                                       const unsigned long long* __restrict__ list_cnt,
                                                       int64_t few_limit, int32_t* __restrict__ a,
                                                       float* __restrict__ lb, float* __restrict__ ub,
                                                       int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
                                                       unsigned long long* __restrict__ cnt) {
  extern __shared__ __align__(16) float dense_smem[];
  float(*As)[kKC][kTR + 4] = reinterpret_cast<float(*)[kKC][kTR + 4]>(dense_smem);                      // [2]
  float(*Bs)[kKC][kTC + 4] = reinterpret_cast<float(*)[kKC][kTC + 4]>(dense_smem + 2 * kKC * (kTR + 4));  // [2]
  // per tile row: its index, current label and 1/|x|; per thread and row of
  // its 8: the running top-2 over the center tiles done so far and the
  // current label's similarity (kept here, not in registers, so that two
  // blocks fit on an SM)
  __shared__ int rows_sh[kTR], cur_sh[kTR];
  __shared__ float ri_sh[kTR];
  __shared__ float tv1[8][256], tv2[8][256], tvc[8][256];
  __shared__ int tj1[8][256];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
  const int64_t total = list ? (int64_t)(*list_cnt) : n;
  if (list && total <= few_limit) return;  // k_dense_rows_few takes short lists
  const int64_t ntiles = (total + kTR - 1) / kTR;
  unsigned long long changed = 0, sims = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    if (tid < kTR) {
      const int64_t q = tile * kTR + tid;
      const int32_t row = (q < total) ? (list ? list[q] : (int32_t)q) : -1;
      rows_sh[tid] = row;
      cur_sh[tid] = row >= 0 ? a[row] : -1;
      ri_sh[tid] = row >= 0 ? rinv[row] : 0.f;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      tv1[x][tid] = tv2[x][tid] = tvc[x][tid] = -INFINITY;
      tj1[x][tid] = INT_MAX;
    }
    __syncthreads();
    // chunks ci = (center tile, term chunk) in order; chunk ci + 1 is copied
    // while chunk ci is multiplied
    const int nkc = (int)((d + kKC - 1) / kKC), nct = (k + kTC - 1) / kTC, nch = nkc * nct;
    auto issue = [&](int ci) {
      const int64_t j0c = (int64_t)(ci / nkc) * kTC, t0c = (int64_t)(ci % nkc) * kKC;
      const int sb = ci & 1;
      // A: 128 rows x 32 terms, B: 128 centers x 32 terms, both transposed
      for (int q = tid; q < kTR * kKC; q += 256) {
        const int r = q / kKC, kk = q % kKC;
        const int32_t row = rows_sh[r];
        const int64_t t = t0c + kk, j = j0c + r;
        const bool ina = row >= 0 && t < d, inb = j < k && t < d;
        cp_async4(&As[sb][kk][r], ina ? X + (int64_t)row * d + t : X, ina);
        cp_async4(&Bs[sb][kk][r], inb ? Cr + j * d + t : Cr, inb);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    float2 acc[8][4];  // [row][center pair]: packed FMAs, each lane rounded as one FMA
    for (int ci = 0; ci < nch; ++ci) {
      if (ci + 1 < nch) issue(ci + 1);
      else asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      __syncthreads();
      const int kc = ci % nkc, sb = ci & 1;
      if (kc == 0) {
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = make_float2(0.f, 0.f);
      }
#pragma unroll 4
      for (int kk = 0; kk < kKC; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[sb][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[sb][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[sb][kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[sb][kk][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = __ffma2_rn(make_float2(av[x], av[x]), bv[y], acc[x][y]);
      }
      __syncthreads();  // this stage is refilled by the copies of chunk ci + 2
      if (kc != nkc - 1) continue;
      const int j0 = (ci / nkc) * kTC;
      // fold this center tile into the running top-2 of each row
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const float ri = ri_sh[trow(ty, x)];
        const int cur = cur_sh[trow(ty, x)];
        float v1 = tv1[x][tid], v2 = tv2[x][tid], vc = tvc[x][tid];
        int j1 = tj1[x][tid];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const int j = j0 + trow(tx, y);
          if (j < k) {
            const float s = __fmul_rn((y & 1) ? acc[x][y >> 1].y : acc[x][y >> 1].x, ri);
            if (j == cur) vc = s;
            if (s > v1) {  // j ascends within a thread: ties keep the lowest index
              v2 = v1;
              v1 = s;
              j1 = j;
            } else if (s > v2) {
              v2 = s;
            }
          }
        }
        tv1[x][tid] = v1;
        tv2[x][tid] = v2;
        tvc[x][tid] = vc;
        tj1[x][tid] = j1;
      }
    }
    // merge across the 16 threads that share these rows (lanes of one half-warp)
#pragma unroll 1
    for (int x = 0; x < 8; ++x) {
      float v1 = tv1[x][tid], v2 = tv2[x][tid], vc = tvc[x][tid];
      int j1 = tj1[x][tid];
#pragma unroll
      for (int o = 8; o; o >>= 1) {
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
        vc = fmaxf(vc, __shfl_xor_sync(SKM_FULL_MASK, vc, o));
      }
      const int32_t row = rows_sh[trow(ty, x)];
      const int32_t cur = cur_sh[trow(ty, x)];
      int32_t nb = -1;
      bool moved = false;
      if (row >= 0) {
        float ssec;
        if (cur >= 0 && vc == v1) {
          nb = cur;
          ssec = (j1 == cur) ? v2 : v1;
        } else {
          nb = j1;
          ssec = v2;
        }
        moved = (nb != cur);
        if (tx == 0) {
          a[row] = nb;
          changed += moved;
          sims += (unsigned long long)k;
          const float dl = dlt[row];
          if (MODE == 1) {
            lb[row] = __fsub_rd(v1, dl);
            ub[row] = (k > 1) ? __fadd_ru(ssec, dl) : -1.f;
          }
        }
      }
      // changed-row list: one entry per moved row (lane tx == 0 of its half-warp)
      const bool take = moved && tx == 0;
      const unsigned m = __ballot_sync(SKM_FULL_MASK, take);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(cnt + C_CHG, (unsigned long long)__popc(m));
        base = __shfl_sync(SKM_FULL_MASK, base, leader);
        if (take) {
          const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
          chg_i[pos] = row;
          chg_old[pos] = cur;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
    sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
  }
  if (lane == 0) {
    if (changed) atomicAdd(cnt + C_CHANGED, changed);
    if (sims) atomicAdd(cnt + C_SIMS, sims);
  }
}

// Whole-row FP32 recheck of a short list (at most `limit` rows; the tile
// kernel above takes longer lists): a block of 1024 threads per kFR rows,
// thread per center (tiles of 1024), reading the term-major centers Ct
// coalesced while the rows' terms come broadcast from shared memory; each
// (row, center) dot is the same sequential chain over t.  Top-2 merged across
// the block with the tie rule.
constexpr int kFR = 4, kXC = 1024, kFT = 1024;

template <int MODE>
__global__ void __launch_bounds__(kFT) k_dense_rows_few(const float* __restrict__ X, const float* __restrict__ rinv,
                                                        const float* __restrict__ dlt, const float* __restrict__ Ct,
                                                        int64_t d, int64_t kst, int32_t k,
                                                        const int32_t* __restrict__ list,
                                                        const unsigned long long* __restrict__ list_cnt, int64_t limit,
                                                        int32_t* __restrict__ a, float* __restrict__ lb,
                                                        float* __restrict__ ub, int32_t* __restrict__ chg_i,
                                                        int32_t* __restrict__ chg_old,
                                                        unsigned long long* __restrict__ cnt) {
  const int64_t total = (int64_t)(*list_cnt);
  if (total > limit) return;
  constexpr int NW = kFT / 32;
  __shared__ float xs[kFR][kXC];
  __shared__ float sv1[NW][kFR], sv2[NW][kFR], svc[NW][kFR];
  __shared__ int sj1[NW][kFR];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t g0 = (int64_t)blockIdx.x * kFR; g0 < total; g0 += (int64_t)gridDim.x * kFR) {
    int32_t row[kFR], cur[kFR];
    float v1[kFR], v2[kFR], vc[kFR];
    int j1[kFR];
#pragma unroll
    for (int r = 0; r < kFR; ++r) {
      row[r] = (g0 + r < total) ? list[g0 + r] : -1;
      cur[r] = row[r] >= 0 ? a[row[r]] : -1;
      v1[r] = v2[r] = vc[r] = -INFINITY;
      j1[r] = INT_MAX;
    }
    for (int j0 = 0; j0 < k; j0 += kFT) {
      const int j = j0 + tid;
      float acc[kFR];
#pragma unroll
      for (int r = 0; r < kFR; ++r) acc[r] = 0.f;
      for (int64_t t0 = 0; t0 < d; t0 += kXC) {
        const int nt = (int)((d - t0) < kXC ? (d - t0) : kXC);
        __syncthreads();
        for (int q = tid; q < kFR * kXC; q += kFT) {
          const int r = q / kXC, tt = q % kXC;
          xs[r][tt] = (row[r] >= 0 && tt < nt) ? X[(int64_t)row[r] * d + t0 + tt] : 0.f;
        }
        __syncthreads();
        if (j < k) {
          const float* cp = Ct + t0 * kst + j;
#pragma unroll 8
          for (int tt = 0; tt < nt; ++tt) {
            const float cv = __ldg(cp + (int64_t)tt * kst);
#pragma unroll
            for (int r = 0; r < kFR; ++r) acc[r] = __fmaf_rn(xs[r][tt], cv, acc[r]);
          }
        }
      }
      if (j < k) {
#pragma unroll
        for (int r = 0; r < kFR; ++r) {
          if (row[r] < 0) continue;
          const float s = __fmul_rn(acc[r], rinv[row[r]]);
          if (j == cur[r]) vc[r] = s;
          if (s > v1[r]) {  // j ascends within a thread: ties keep the lowest index
            v2[r] = v1[r];
            v1[r] = s;
            j1[r] = j;
          } else if (s > v2[r]) {
            v2[r] = s;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kFR; ++r) {
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float ov1 = __shfl_xor_sync(SKM_FULL_MASK, v1[r], o);
        const int oj1 = __shfl_xor_sync(SKM_FULL_MASK, j1[r], o);
        const float ov2 = __shfl_xor_sync(SKM_FULL_MASK, v2[r], o);
        if (ov1 > v1[r] || (ov1 == v1[r] && oj1 < j1[r])) {
          v2[r] = fmaxf(ov2, v1[r]);
          v1[r] = ov1;
          j1[r] = oj1;
        } else {
          v2[r] = fmaxf(v2[r], ov1);
        }
        vc[r] = fmaxf(vc[r], __shfl_xor_sync(SKM_FULL_MASK, vc[r], o));
      }
      if (lane == 0) {
        sv1[warp][r] = v1[r];
        sv2[warp][r] = v2[r];
        svc[warp][r] = vc[r];
        sj1[warp][r] = j1[r];
      }
    }
    __syncthreads();
    if (tid < kFR && row[tid] >= 0) {
      const int r = tid;
      float b1 = sv1[0][r], b2 = sv2[0][r], bc = svc[0][r];
      int bj = sj1[0][r];
      for (int w = 1; w < NW; ++w) {
        const float ov1 = sv1[w][r];
        const int oj1 = sj1[w][r];
        if (ov1 > b1 || (ov1 == b1 && oj1 < bj)) {
          b2 = fmaxf(sv2[w][r], b1);
          b1 = ov1;
          bj = oj1;
        } else {
          b2 = fmaxf(b2, ov1);
        }
        bc = fmaxf(bc, svc[w][r]);
      }
      const int32_t i = row[r], ci = cur[r];
      int32_t nb;
      float ssec;
      if (ci >= 0 && bc == b1) {
        nb = ci;
        ssec = (bj == ci) ? b2 : b1;
      } else {
        nb = bj;
        ssec = b2;
      }
      a[i] = nb;
      atomicAdd(cnt + C_SIMS, (unsigned long long)k);
      if (MODE == 1) {
        const float dl = dlt[i];
        lb[i] = __fsub_rd(b1, dl);
        ub[i] = (k > 1) ? __fadd_ru(ssec, dl) : -1.f;
      }
      if (nb != ci) {
        atomicAdd(cnt + C_CHANGED, 1ull);
        const unsigned long long pos = atomicAdd(cnt + C_CHG, 1ull);
        chg_i[pos] = i;
        chg_old[pos] = ci;
      }
    }
  }
}

// Precision form, standard variant: after the centers moved, l(i) <- the
// lower bound of Eq. (eqn:l-bound) with the drift of c(a(i)), so that l stays
// a lower bound on the best similarity (the tensor-core pass starts each
// row's candidate list above l - eps_b - 2 (eps_b + delta_i)).
__global__ void k_dense_lower(int64_t n, const int32_t* __restrict__ a, float* __restrict__ lb,
                              const float* __restrict__ pdn, const float* __restrict__ pup,
                              const float* __restrict__ qup) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ai = a[i];
    lb[i] = bound_l(lb[i], pdn[ai], pup[ai], qup[ai]);
  }
}

// Precision form, first pass.  For each row (all, or the Hamerly survivors
// w1) the BF16 top-8 is within eps_b = bf16_eps(row) of the exact ones (v1 the best
// at j1, v2 the next); the canonical FP32 similarities are within delta_i of
// exact.  If v1 - v2 > 2 (eps_b + delta_i) the FP32 standard variant
// necessarily picks j1, so j1 is the label, and Hamerly's bounds become
// l = v1 - eps_b, u = v2 + eps_b (exact-similarity bounds).  Otherwise the row
// goes to `amb` for k_dense_cands.
template <bool HAMERLY>
__global__ void __launch_bounds__(256) k_dense_classify(const float* __restrict__ topv, const int32_t* __restrict__ topi,
                                                        const float* __restrict__ dlt, const float* __restrict__ exr,
                                                        const float* __restrict__ ebc, int64_t n,
                                                        const int32_t* __restrict__ list,
                                                        const unsigned long long* __restrict__ list_cnt,
                                                        int32_t* __restrict__ a, float* __restrict__ lb,
                                                        float* __restrict__ ub, int32_t* __restrict__ amb_out,
                                                        int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
                                                        unsigned long long* __restrict__ cnt) {
  const int64_t total = list ? (int64_t)(*list_cnt) : n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long changed = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t q = base + threadIdx.x;
    bool amb = false, moved = false;
    int32_t row = 0, cur = -1;
    if (q < total) {
      row = list ? list[q] : (int32_t)q;
      const float2 t = *reinterpret_cast<const float2*>(topv + (int64_t)row * kTopK);
      const float v1 = t.x, v2 = t.y;
      const int j1 = topi[(int64_t)row * kTopK];
      const float eps_b = bf16_eps(exr, ebc, row);
      const float margin = __fadd_ru(eps_b, dlt[row]);
      cur = a[row];
      if (j1 >= 0 && __fsub_rd(v1, v2) > __fmul_ru(2.f, margin)) {
        moved = (j1 != cur);
        a[row] = j1;
        changed += moved;
        if (HAMERLY) {
          lb[row] = __fsub_rd(v1, eps_b);
          ub[row] = fmaxf(__fadd_ru(v2, eps_b), -1.f);
        }
      } else {
        amb = true;
      }
    }
    warp_push(amb, row, amb_out, cnt + C_W3);
    const unsigned m = __ballot_sync(SKM_FULL_MASK, moved);
    if (m) {
      const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
      unsigned long long b0 = 0;
      if (lane == leader) b0 = atomicAdd(cnt + C_CHG, (unsigned long long)__popc(m));
      b0 = __shfl_sync(SKM_FULL_MASK, b0, leader);
      if (moved) {
        const unsigned long long pos = b0 + __popc(m & ((1u << lane) - 1u));
        chg_i[pos] = row;
        chg_old[pos] = cur;
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
  if ((threadIdx.x & 31) == 0 && changed) atomicAdd(cnt + C_CHANGED, changed);
}

// Canonical FP32 dot of a stored row with a center row: one FMA chain over
// t = 0..d-1 in order (float4 loads when both rows are 16-byte aligned).
// Canonical FP32 dot of a stored row with a center row: one FMA chain over
// t = 0..d-1 in order.  V = 8: 32-byte loads (rows 32-byte aligned, d % 8 == 0),
// V = 4: 16-byte loads, V = 1: scalar loads; the chain is the same.
__device__ __forceinline__ void ldg_v8(const float* p, float (&r)[8]) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
               : "l"(p));
}

template <int V>
__device__ __forceinline__ float dense_dot_seq(const float* __restrict__ x, const float* __restrict__ c, int64_t d) {
  float acc = 0.f;
  if (V == 8) {
#pragma unroll 2
    for (int64_t t = 0; t < d; t += 8) {
      float xv[8], cv[8];
      ldg_v8(x + t, xv);
      ldg_v8(c + t, cv);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = __fmaf_rn(xv[q], cv[q], acc);
    }
  } else if (V == 4) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* c4 = reinterpret_cast<const float4*>(c);
#pragma unroll 4
    for (int64_t t = 0; t < (d >> 2); ++t) {
      const float4 xv = x4[t], cv = c4[t];
      acc = __fmaf_rn(xv.x, cv.x, acc);
      acc = __fmaf_rn(xv.y, cv.y, acc);
      acc = __fmaf_rn(xv.z, cv.z, acc);
      acc = __fmaf_rn(xv.w, cv.w, acc);
    }
  } else {
#pragma unroll 4
    for (int64_t t = 0; t < d; ++t) acc = __fmaf_rn(x[t], c[t], acc);
  }
  return acc;
}

// Precision form, second pass, over the ambiguous rows.  With w = eps_b +
// delta_i, a center whose BF16 similarity is below v1 - 2w has an FP32
// similarity below that of j1, so only the leading candidates of a row's list
// with v >= v1 - 2w can win; each gets its canonical FP32 similarity and the
// winner follows the tie rule (the current label, else the lowest index).
// Centers outside the top-8 have BF16 similarity <= v8; when all eight are
// candidates the winner must beat v8 + w, else the row goes to `out` for a
// whole-row recheck.  Hamerly: l = f_a - delta_i, u = max(other candidates'
// f + delta_i, next BF16 value + eps_b).
// A warp takes 32 rows at a time (lane r: row r) and spreads their
// (row, candidate) pairs over its lanes, 32 pairs per round, so that no lane
// idles while a row has few candidates; each pair's similarity is one lane's
// FMA chain.  Lane r then decides row r from the similarities in shared memory.
template <bool HAMERLY, int V>
__global__ void __launch_bounds__(256) k_dense_cands(const float* __restrict__ X, const float* __restrict__ rinv,
                                                     const float* __restrict__ dlt, const float* __restrict__ Cr,
                                                     int64_t d, int32_t k, const float* __restrict__ exr,
                                                     const float* __restrict__ ebc,
                                                     const float* __restrict__ topv, const int32_t* __restrict__ topi,
                                                     const int32_t* __restrict__ list,
                                                     const unsigned long long* __restrict__ list_cnt,
                                                     int32_t* __restrict__ a, float* __restrict__ lb,
                                                     float* __restrict__ ub, int32_t* __restrict__ out,
                                                     int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
                                                     unsigned long long* __restrict__ cnt) {
  __shared__ int32_t s_j[8][32][kTopK];  // per warp: the listed centers of its 32 rows
  __shared__ float s_f[8][32][kTopK];    // their FP32 similarities (candidates only)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t total = (int64_t)(*list_cnt);
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long changed = 0, sims = 0;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < total;
       base += nwarps * 32) {
    const int64_t slot = base + lane;
    const bool act = slot < total;
    const int32_t row = act ? list[slot] : 0;
    float v[kTopK];
    int32_t jj[kTopK];
    float dl = 0.f, w = 0.f, eps_b = 0.f;
    int ncand = 0;
    if (act) {
      const float4* vp = reinterpret_cast<const float4*>(topv + (int64_t)row * kTopK);
      const int4* ip = reinterpret_cast<const int4*>(topi + (int64_t)row * kTopK);
      const float4 v0 = vp[0], v1 = vp[1];
      const int4 i0 = ip[0], i1 = ip[1];
      v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w; v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
      jj[0] = i0.x; jj[1] = i0.y; jj[2] = i0.z; jj[3] = i0.w; jj[4] = i1.x; jj[5] = i1.y; jj[6] = i1.z; jj[7] = i1.w;
      dl = dlt[row];
      eps_b = bf16_eps(exr, ebc, row);
      w = __fadd_ru(eps_b, dl);
      const float theta = __fsub_rd(v[0], __fmul_ru(2.f, w));
      // the candidates are a prefix of the descending list
#pragma unroll
      for (int q = 0; q < kTopK; ++q) ncand += (jj[q] >= 0 && v[q] >= theta) ? 1 : 0;
#pragma unroll
      for (int q = 0; q < kTopK; ++q) s_j[warp][lane][q] = jj[q];
    } else {
#pragma unroll
      for (int q = 0; q < kTopK; ++q) {
        v[q] = -INFINITY;
        jj[q] = -1;
      }
    }
    // pairs: exclusive prefix of the candidate counts over the lanes
    int incl = ncand;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(SKM_FULL_MASK, incl, o);
      if (lane >= o) incl += y;
    }
    const int npairs = __shfl_sync(SKM_FULL_MASK, incl, 31);
    __syncwarp();
    for (int p0 = 0; p0 < npairs; p0 += 32) {
      const int p = p0 + lane;
      // the row r of pair p: the first lane whose inclusive count exceeds p
      int r = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int c = __shfl_sync(SKM_FULL_MASK, incl, r + step - 1);
        if (c <= p) r += step;
      }
      const int excl_r = __shfl_sync(SKM_FULL_MASK, incl - ncand, r);
      const int32_t row_r = __shfl_sync(SKM_FULL_MASK, row, r);
      if (p < npairs) {
        const int q = p - excl_r;
        const int32_t j = s_j[warp][r][q];
        s_f[warp][r][q] = __fmul_rn(dense_dot_seq<V>(X + (int64_t)row_r * d, Cr + (int64_t)j * d, d), rinv[row_r]);
      }
    }
    __syncwarp();
    if (act) {
      const int32_t cur = a[row];
      // best candidate under the tie rule (a total order: any scan order)
      float bf = -INFINITY;
      int32_t bj = INT_MAX;
      for (int q = 0; q < ncand; ++q) {
        const float of = s_f[warp][lane][q];
        const int32_t oj = jj[q];
        const bool take = (of > bf) || (of == bf && oj != bj && (oj == cur || (bj != cur && oj < bj)));
        if (take) {
          bf = of;
          bj = oj;
        }
      }
      // largest BF16 value among the non-candidates (or a bound on it)
      const bool all8 = (ncand == kTopK) && (k > kTopK);
      float vnext = -INFINITY;
#pragma unroll
      for (int q = 0; q < kTopK; ++q)
        if (q == ncand) vnext = v[q];
      if (ncand == kTopK) vnext = all8 ? v[kTopK - 1] : -INFINITY;
      const bool resolved = ncand > 0 && ((ncand < kTopK) || !all8 || (bf > __fadd_ru(v[kTopK - 1], w)));
      sims += (unsigned long long)ncand;
      if (resolved) {
        a[row] = bj;
        if (bj != cur) {
          ++changed;
          const unsigned long long pos = atomicAdd(cnt + C_CHG, 1ull);
          chg_i[pos] = row;
          chg_old[pos] = cur;
        }
        if (HAMERLY) {
          float f2 = -INFINITY;
          for (int q = 0; q < ncand; ++q)
            if (jj[q] != bj) f2 = fmaxf(f2, s_f[warp][lane][q]);
          lb[row] = __fsub_rd(bf, dl);
          const float u1 = (f2 == -INFINITY) ? -1.f : __fadd_ru(f2, dl);
          const float u2 = (vnext == -INFINITY) ? -1.f : __fadd_ru(vnext, eps_b);
          ub[row] = fmaxf(fmaxf(u1, u2), -1.f);
        }
      } else {
        const unsigned long long pos = atomicAdd(cnt + C_W2, 1ull);
        out[pos] = row;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
    sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
  }
  if (lane == 0) {
    if (changed) atomicAdd(cnt + C_CHANGED, changed);
    if (sims) atomicAdd(cnt + C_SIMS, sims);
  }
}

// Hamerly on dense rows: warp per survivor, exact <x, c_a> (32 terms loaded at
// once, sequential FMA chain through shuffles), then the test again; points
// still failing go to `out`.
template <bool FULL>
__global__ void __launch_bounds__(256) k_dense_tighten(const float* __restrict__ X, const float* __restrict__ rinv,
                                                       const float* __restrict__ dlt, const float* __restrict__ Cr,
                                                       int64_t d, const int32_t* __restrict__ w1,
                                                       const unsigned long long* __restrict__ w1_cnt,
                                                       const int32_t* __restrict__ a, float* __restrict__ lb,
                                                       const float* __restrict__ ub, const float* __restrict__ sc,
                                                       int32_t* __restrict__ out, unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)(*w1_cnt);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long sims = 0;
  for (int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total; slot += nw) {
    const int32_t i = w1[slot];
    const int32_t ai = a[i];
    const float* xr = X + (int64_t)i * d;
    const float* cr = Cr + (int64_t)ai * d;
    float acc = 0.f;
    for (int64_t t0 = 0; t0 < d; t0 += 32) {
      const float xv = (t0 + lane < d) ? xr[t0 + lane] : 0.f;
      const float cv = (t0 + lane < d) ? cr[t0 + lane] : 0.f;
      const int nq = (int)min((int64_t)32, d - t0);
      for (int q = 0; q < nq; ++q)
        acc = __fmaf_rn(__shfl_sync(SKM_FULL_MASK, xv, q), __shfl_sync(SKM_FULL_MASK, cv, q), acc);
    }
    const float sim = __fmul_rn(acc, rinv[i]);
    const float dl = dlt[i];
    const float l = __fsub_rd(sim, dl);
    const float L = __fsub_rd(l, 2.f * dl);
    const bool fail = !((L >= ub[i]) || (FULL && L >= 0.f && L >= sc[ai]));
    if (lane == 0) {
      lb[i] = l;
      ++sims;
      if (fail) {
        const unsigned long long pos = atomicAdd(cnt + C_W2, 1ull);
        out[pos] = i;
      }
    }
  }
  if (lane == 0 && sims) atomicAdd(cnt + C_SIMS, sims);
}

// ---- exact fixed-point cluster sums of dense rows

__global__ void k_label_zero(int32_t* __restrict__ cntk, int32_t k, int s64_valid,
                             const unsigned long long* __restrict__ cnt, int64_t n) {
  if (!full_update(s64_valid, cnt, n)) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) cntk[j] = 0;
}

__global__ void k_label_count(const int32_t* __restrict__ a, int64_t n, int32_t* __restrict__ cntk, int s64_valid,
                              const unsigned long long* __restrict__ cnt) {
  if (!full_update(s64_valid, cnt, n)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cntk + a[i], 1);
}

// one block: exclusive scan of k counts into off (k+1) and a cursor copy
__global__ void __launch_bounds__(1024) k_label_scan(const int32_t* __restrict__ cntk, int32_t k,
                                                     int32_t* __restrict__ off, int32_t* __restrict__ cursor,
                                                     int s64_valid, const unsigned long long* __restrict__ cnt,
                                                     int64_t n) {
  if (!full_update(s64_valid, cnt, n)) return;
  __shared__ int sh[1024];
  const int per = (k + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(k, b + per);
  int s = 0;
  for (int q = b; q < e; ++q) s += cntk[q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - s;
  for (int q = b; q < e; ++q) {
    off[q] = run;
    cursor[q] = run;
    run += cntk[q];
  }
  if (threadIdx.x == 1023) off[k] = sh[1023];
}

__global__ void k_label_place(const int32_t* __restrict__ a, int64_t n, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ members, int s64_valid, const unsigned long long* __restrict__ cnt) {
  if (!full_update(s64_valid, cnt, n)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    members[atomicAdd(cursor + a[i], 1)] = (int32_t)i;
}

// Block per (cluster, 128-term slice): sum of the members' fixed-point values
// (order-free, exact) -> S64[t][j].
__global__ void __launch_bounds__(128) k_dense_cluster_sum(const float* __restrict__ X, const float* __restrict__ rinv,
                                                           int64_t d, int64_t kst, const int32_t* __restrict__ off,
                                                           const int32_t* __restrict__ members, float scale,
                                                           long long* __restrict__ S64, int s64_valid,
                                                           const unsigned long long* __restrict__ cnt, int64_t n) {
  if (!full_update(s64_valid, cnt, n)) return;
  const int j = blockIdx.x;
  const int64_t t = (int64_t)blockIdx.y * 128 + threadIdx.x;
  if (t >= d) return;
  long long s = 0;
  const int b = off[j], e = off[j + 1];
  int m = b;
  for (; m + 4 <= e; m += 4) {
    int32_t r[4];
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = members[m + u];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __fmul_rn(X[(int64_t)r[u] * d + t], rinv[r[u]]);
#pragma unroll
    for (int u = 0; u < 4; ++u) s += __float2ll_rn(__fmul_rn(x[u], scale));
  }
  for (; m < e; ++m) {
    const int32_t r = members[m];
    s += __float2ll_rn(__fmul_rn(__fmul_rn(X[(int64_t)r * d + t], rinv[r]), scale));
  }
  S64[t * kst + j] = s;
}

// Incremental: warp per changed row, -x from the old and +x to the new sum;
// both clusters' exact squared norms take the change of the squares (n2_add).
__global__ void __launch_bounds__(256) k_dense_delta(const float* __restrict__ X, const float* __restrict__ rinv,
                                                     int64_t d, int64_t kst, const int32_t* __restrict__ chg_i,
                                                     const int32_t* __restrict__ chg_old, const int32_t* __restrict__ a,
                                                     float scale, long long* __restrict__ S64,
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
    for (int64_t t = lane; t < d; t += 32) {
      const long long fx = __float2ll_rn(__fmul_rn(__fmul_rn(X[(int64_t)i * d + t], ri), scale));
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

inline unsigned grid_cap(int64_t items, int per_block, int nsm, int per_sm = 16) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g > (int64_t)nsm * per_sm) g = (int64_t)nsm * per_sm;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int dense_prep_bf16(skm_ctx* c) {
  SKM_PROF_BEGIN(c, "k_dense_bf16");
  k_dense_bf16<<<grid_cap(c->n, 8, c->nsm), 256, 0, c->st>>>((const float*)c->val, c->rinv, c->n, c->d,
                                                             (__nv_bfloat16*)c->Xb, c->exr);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

// out[i] = the row's current BF16 error bound (device memory, n floats).
int dense_prep_fp8(skm_ctx* c) {
  SKM_PROF_BEGIN(c, "k_dense_fp8");
  k_dense_fp8<<<grid_cap(c->n, 8, c->nsm), 256, 0, c->st>>>((const float*)c->val, c->rinv, c->n, c->d,
                                                            (uint8_t*)c->Xb, c->exr, c->rsc);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

int dense_bf16_eps(skm_ctx* c, float* out) {
  SKM_PROF_BEGIN(c, "k_bf16_eps_rows");
  k_bf16_eps_rows<<<grid_cap(c->n, 256, c->nsm), 256, 0, c->st>>>(c->exr, c->ebc, c->n, out);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

int dense_refresh_centers(skm_ctx* c) {
  dim3 g((unsigned)((c->d + 31) / 32), (unsigned)((c->kpad + 31) / 32));
  const bool fp8 = c->precision == SKM_PREC_FP8;
  SKM_PROF_BEGIN(c, "k_dense_centers");
  k_dense_centers<<<g, dim3(32, 8), 0, c->st>>>(c->Ct, c->d, c->k, c->kst, c->kpad, c->Cr,
                                                fp8 ? nullptr : (__nv_bfloat16*)c->Cb,
                                                fp8 ? (uint8_t*)c->Cb : nullptr);
  SKM_LAUNCHED(c);
  if (c->Cb && fp8) {
    SKM_PROF_BEGIN(c, "k_center_err");
    k_center_err_fp8<<<(unsigned)((c->k + 7) / 8), 256, 0, c->st>>>(c->Cr, (const uint8_t*)c->Cb, c->d, c->k,
                                                                   c->ebw, c->ebc);
    SKM_LAUNCHED(c);
  } else if (c->Cb) {
    SKM_PROF_BEGIN(c, "k_center_err");
    k_center_err<<<(unsigned)((c->k + 7) / 8), 256, 0, c->st>>>(c->Cr, (const __nv_bfloat16*)c->Cb, c->d, c->k,
                                                              c->ebw, c->ebc);
    SKM_LAUNCHED(c);
  }
  return SKM_OK;
}

int dense_rows(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt) {
  const int64_t ntiles = (c->n + kTR - 1) / kTR;
  const unsigned g = (unsigned)(list ? c->nsm * 2 : (ntiles < (int64_t)c->nsm * 4 ? ntiles : (int64_t)c->nsm * 4));
  // a list of at most few_limit rows goes to k_dense_rows_few, a longer one
  // to the tile kernel (each returns at once when the other one applies)
  const int64_t few_limit = (int64_t)c->nsm * 32;
  const float* X = (const float*)c->val;
  static bool attr = false;
  if (!attr) {
    SKM_CUDA_TRY(cudaFuncSetAttribute(k_dense_top2<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem));
    SKM_CUDA_TRY(cudaFuncSetAttribute(k_dense_top2<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem));
    attr = true;
  }
  SKM_PROF_BEGIN(c, list ? "k_dense_top2(list)" : "k_dense_top2");
  if (mode == 0)
    k_dense_top2<0><<<g, 256, kDenseSmem, c->st>>>(X, c->rinv, c->dlt, c->Cr, c->n, c->d, c->k, list, list_cnt,
                                                   few_limit, c->a, c->lb, c->ub, c->chg_i, c->chg_old, c->cnt);
  else
    k_dense_top2<1><<<g, 256, kDenseSmem, c->st>>>(X, c->rinv, c->dlt, c->Cr, c->n, c->d, c->k, list, list_cnt,
                                                   few_limit, c->a, c->lb, c->ub, c->chg_i, c->chg_old, c->cnt);
  SKM_LAUNCHED(c);
  if (list) {
    SKM_PROF_BEGIN(c, "k_dense_rows_few");
    const unsigned gf = c->nsm * 2;
    if (mode == 0)
      k_dense_rows_few<0><<<gf, kFT, 0, c->st>>>(X, c->rinv, c->dlt, c->Ct, c->d, c->kst, c->k, list, list_cnt,
                                                 few_limit, c->a, c->lb, c->ub, c->chg_i, c->chg_old, c->cnt);
    else
      k_dense_rows_few<1><<<gf, kFT, 0, c->st>>>(X, c->rinv, c->dlt, c->Ct, c->d, c->kst, c->k, list, list_cnt,
                                                 few_limit, c->a, c->lb, c->ub, c->chg_i, c->chg_old, c->cnt);
    SKM_LAUNCHED(c);
  }
  return SKM_OK;
}

int dense_lower(skm_ctx* c) {
  SKM_PROF_BEGIN(c, "k_dense_lower");
  k_dense_lower<<<grid_cap(c->n, 256, c->nsm), 256, 0, c->st>>>(c->n, c->a, c->lb, c->pdn, c->pup, c->qup);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

int dense_classify(skm_ctx* c, bool hamerly, const int32_t* list, const unsigned long long* list_cnt) {
  SKM_PROF_BEGIN(c, "k_dense_classify");
  const unsigned g = c->nsm * 8;
  if (hamerly)
    k_dense_classify<true><<<g, 256, 0, c->st>>>(c->topv, c->topi, c->dlt, c->exr, c->ebc, c->n, list, list_cnt, c->a,
                                                 c->lb, c->ub, c->w3, c->chg_i, c->chg_old, c->cnt);
  else
    k_dense_classify<false><<<g, 256, 0, c->st>>>(c->topv, c->topi, c->dlt, c->exr, c->ebc, c->n, list, list_cnt, c->a,
                                                  c->lb, c->ub, c->w3, c->chg_i, c->chg_old, c->cnt);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

// Blocks of k_dense_cands<H, V> resident on one SM (the occupancy calculator).
template <bool H, int V>
int cands_fit() {
  static int nb = 0;
  if (nb == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dense_cands<H, V>, 256, 0) != cudaSuccess || nb < 1) {
      (void)cudaGetLastError();
      nb = 1;
    }
  }
  return nb;
}

int dense_recheck_cands(skm_ctx* c, bool hamerly) {
  SKM_PROF_BEGIN(c, "k_dense_cands");
  const uintptr_t xa = (uintptr_t)c->val, ca = (uintptr_t)c->Cr;
  const int v = (c->d % 8 == 0 && xa % 32 == 0 && ca % 32 == 0) ? 8 : (c->d % 4 == 0 && xa % 16 == 0) ? 4 : 1;
  const float* X = (const float*)c->val;
  // one resident wave: every warp takes 32 rows at a time
#define SKM_CANDS(H, V)                                                                                            \
  k_dense_cands<H, V><<<c->nsm * cands_fit<H, V>(), 256, 0, c->st>>>(X, c->rinv, c->dlt, c->Cr, c->d, c->k, c->exr, c->ebc, c->topv, c->topi,     \
                                            c->w3, c->cnt + C_W3, c->a, c->lb, c->ub, c->w2, c->chg_i, c->chg_old, \
                                            c->cnt)
  if (hamerly) {
    if (v == 8) SKM_CANDS(true, 8);
    else if (v == 4) SKM_CANDS(true, 4);
    else SKM_CANDS(true, 1);
  } else {
    if (v == 8) SKM_CANDS(false, 8);
    else if (v == 4) SKM_CANDS(false, 4);
    else SKM_CANDS(false, 1);
  }
#undef SKM_CANDS
  SKM_LAUNCHED(c);
  return SKM_OK;
}

int dense_tighten(skm_ctx* c) {
  SKM_PROF_BEGIN(c, "k_dense_tighten");
  const unsigned g = c->nsm * 8;
  if (c->variant == SKM_HAMERLY)
    k_dense_tighten<true><<<g, 256, 0, c->st>>>((const float*)c->val, c->rinv, c->dlt, c->Cr, c->d, c->w1,
                                                c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w2, c->cnt);
  else
    k_dense_tighten<false><<<g, 256, 0, c->st>>>((const float*)c->val, c->rinv, c->dlt, c->Cr, c->d, c->w1,
                                                 c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w2, c->cnt);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

// Cluster sums of dense rows: a full recomputation (rows sorted by label,
// then a block per cluster and 128-term slice) or only the changed rows; the
// same device-side rule as the sparse path picks one (the other's kernels
// return at once).
int dense_center_sums(skm_ctx* c) {
  const int64_t n = c->n;
  SKM_PROF_BEGIN(c, "k_label_zero");
  k_label_zero<<<grid_cap(c->k, 256, c->nsm), 256, 0, c->st>>>(c->lcount, c->k, c->s64_valid, c->cnt, n);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_label_count");
  k_label_count<<<grid_cap(n, 256, c->nsm), 256, 0, c->st>>>(c->a, n, c->lcount, c->s64_valid, c->cnt);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_label_scan");
  k_label_scan<<<1, 1024, 0, c->st>>>(c->lcount, c->k, c->loff, c->lcursor, c->s64_valid, c->cnt, n);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_label_place");
  k_label_place<<<grid_cap(n, 256, c->nsm), 256, 0, c->st>>>(c->a, n, c->lcursor, c->lmembers, c->s64_valid, c->cnt);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_dense_cluster_sum");
  k_dense_cluster_sum<<<dim3((unsigned)c->k, (unsigned)((c->d + 127) / 128)), 128, 0, c->st>>>(
      (const float*)c->val, c->rinv, c->d, c->kst, c->loff, c->lmembers, c->fx_scale, c->S64, c->s64_valid, c->cnt, n);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_dense_delta");
  k_dense_delta<<<grid_cap(n * 32, 256, c->nsm), 256, 0, c->st>>>((const float*)c->val, c->rinv, c->d, c->kst,
                                                                   c->chg_i, c->chg_old, c->a, c->fx_scale, c->S64,
                                                                   c->dflag, c->s64_valid, c->cnt, n, c->n2l);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

}  // namespace skm
