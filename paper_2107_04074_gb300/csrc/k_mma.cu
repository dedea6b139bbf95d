// Dense similarity bulk on the 5th-generation tensor cores (precision form):
// S^b = X_b * C_b^T with BF16 operands and FP32 accumulation in tensor memory,
// fused with a per-row top-2 (and the similarity to the current label).
//
// One CTA per SM, persistent over tiles of 128 rows.  Warp roles:
//   warp 0  TMA producer: the row tile A (128 x d, all K blocks, resident in
//           shared memory) and 256 x 64 tiles of the centers B through a
//           3-stage ring, 128-byte swizzled;
//   warp 1  allocates 512 TMEM columns; one lane issues tcgen05.mma
//           (M = 128, N = 256, K = 16 per instruction) into one of two
//           256-column accumulators, and tcgen05.commit to the barriers;
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane TMEM quarter, top-2 per
//           row while the other accumulator is being filled.
// Every barrier wait gives up after one second (globaltimer): the kernel
// then records an error word and leaves its loops; TMEM is freed on exit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <climits>

#include "skm_internal.cuh"

namespace skm {

namespace {

constexpr int kBM = 128;          // rows per tile (UMMA M)
constexpr int kBN = 256;          // centers per accumulator (UMMA N)
constexpr int kBK = 64;           // K elements per 128-byte swizzled row
constexpr int kStages = 3;        // B ring
constexpr int kMaxKB = 7;         // K blocks of A kept resident (d <= 448)
constexpr int kThreads = 192;
constexpr uint32_t kABytes = kBM * kBK * 2;  // 16 KB per K block
constexpr uint32_t kBBytes = kBN * kBK * 2;  // 32 KB per stage
constexpr uint64_t kTimeoutNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout (which
// also raises the CTA's abort flag so that the other roles stop too) or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (now_ns() - t0 > kTimeoutNs) {
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) atoms; start address advances 32 bytes per
// K = 16 step inside the atom.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);  // start address
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct MmaShared {
  uint64_t a_full, a_empty;
  uint64_t b_full[kStages], b_empty[kStages];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem_base;
  int abort_flag;
};

// Per row: v1 (best BF16 similarity), j1 (its center, lowest index on ties),
// v2 (best over the other centers) and vc (similarity to the current label).
__global__ void __launch_bounds__(kThreads, 1) k_bf16_top2(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, int64_t n,
                                                          int32_t k, int nkb, int nnt, const int32_t* __restrict__ a,
                                                          float4* __restrict__ top2, unsigned long long* __restrict__ cnt) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the swizzled tiles
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* As = base;                                // nkb x 16 KB
  unsigned char* Bs = base + (size_t)kMaxKB * kABytes;     // kStages x 32 KB
  MmaShared* sh = reinterpret_cast<MmaShared*>(Bs + (size_t)kStages * kBBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (n + kBM - 1) / kBM;
  const uint32_t idesc = idesc_bf16(kBM, kBN);

  if (threadIdx.x == 0) {
    mbar_init(&sh->a_full, 1);
    mbar_init(&sh->a_empty, 1);
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh->b_full[s], 1);
      mbar_init(&sh->b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->acc_full[b], 1);
      mbar_init(&sh->acc_empty[b], 128);
    }
    sh->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh->tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;
  volatile int* abort_flag = &sh->abort_flag;
  bool ok = true;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t gidx = 0;
      int lt = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        if (lt > 0) ok = mbar_wait(&sh->a_empty, (lt - 1) & 1, abort_flag);
        if (!ok) break;
        mbar_expect_tx(&sh->a_full, kABytes * nkb);
        for (int kb = 0; kb < nkb; ++kb)
          tma_load_2d(&mapA, &sh->a_full, As + (size_t)kb * kABytes, kb * kBK, (int)(tile * kBM));
        for (int nt = 0; nt < nnt && ok; ++nt)
          for (int kb = 0; kb < nkb; ++kb, ++gidx) {
            const int s = gidx % kStages;
            if (gidx >= (uint32_t)kStages) ok = mbar_wait(&sh->b_empty[s], ((gidx / kStages) - 1) & 1, abort_flag);
            if (!ok) break;
            mbar_expect_tx(&sh->b_full[s], kBBytes);
            tma_load_2d(&mapB, &sh->b_full[s], Bs + (size_t)s * kBBytes, kb * kBK, nt * kBN);
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t gidx = 0, accidx = 0;
      int lt = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        ok = mbar_wait(&sh->a_full, lt & 1, abort_flag);
        if (!ok) break;
        for (int nt = 0; nt < nnt && ok; ++nt, ++accidx) {
          const uint32_t buf = accidx & 1, use = accidx >> 1;
          if (use > 0) ok = mbar_wait(&sh->acc_empty[buf], (use - 1) & 1, abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d_tmem = tmem + buf * kBN;
          for (int kb = 0; kb < nkb; ++kb, ++gidx) {
            const int s = gidx % kStages;
            ok = mbar_wait(&sh->b_full[s], (gidx / kStages) & 1, abort_flag);
            if (!ok) break;
            tc_fence_after();
            const uint32_t a_addr = smem_u32(As + (size_t)kb * kABytes);
            const uint32_t b_addr = smem_u32(Bs + (size_t)s * kBBytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              umma_bf16(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc,
                        (kb > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&sh->b_empty[s]);  // the stage is free once these MMAs are done
          }
          if (!ok) break;
          umma_commit(&sh->acc_full[buf]);
        }
        if (!ok) break;
        umma_commit(&sh->a_empty);
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2-5)
    const int quarter = warp & 3;  // the TMEM lanes this warp may read
    const int r_in_tile = quarter * 32 + lane;
    uint32_t accidx = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t row = tile * kBM + r_in_tile;
      const int32_t cur = (row < n) ? a[row] : -1;
      float v1 = -INFINITY, v2 = -INFINITY, vc = -INFINITY;
      int j1 = INT_MAX;
      for (int nt = 0; nt < nnt; ++nt, ++accidx) {
        const uint32_t buf = accidx & 1, use = accidx >> 1;
        ok = mbar_wait(&sh->acc_full[buf], use & 1, abort_flag);
        if (!ok) break;
        tc_fence_after();
        for (int c = 0; c < kBN / 32; ++c) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + buf * kBN + c * 32, r);
          const int jb = nt * kBN + c * 32;
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = jb + q;
            const float s = __uint_as_float(r[q]);
            if (j < k) {
              if (j == cur) vc = s;
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
        tc_fence_before();
        mbar_arrive(&sh->acc_empty[buf]);
      }
      if (ok && row < n) top2[row] = make_float4(v1, __int_as_float(j1), v2, vc);
    }
  }
  if (!ok) atomicOr(cnt + C_ERR, (unsigned long long)E_TIMEOUT);  // a device wait gave up
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// rows x cols BF16, row-major (cols contiguous); boxes of 64 columns x box_rows.
int make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return SKM_EUNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SKM_OK : SKM_EINVAL;
}

}  // namespace

size_t bf16_mma_smem_bytes() { return 1024 + (size_t)kMaxKB * kABytes + (size_t)kStages * kBBytes + sizeof(MmaShared); }

int bf16_mma_supported(int64_t d) { return (d % 8 == 0) && ((d + kBK - 1) / kBK <= kMaxKB); }

// Xb: n x d BF16 (unit rows); Cb: (ceil(k/256)*256) x d BF16 (zero rows past k).
int bf16_top2(skm_ctx* c, const void* Xb, const void* Cb, float4* top2) {
  if (!bf16_mma_supported(c->d)) return SKM_EUNSUPPORTED;
  CUtensorMap mA, mB;
  const int nnt = (c->k + kBN - 1) / kBN;
  int rc = make_map(&mA, Xb, c->n, c->d, kBM);
  if (rc) return rc;
  rc = make_map(&mB, Cb, (int64_t)nnt * kBN, c->d, kBN);
  if (rc) return rc;
  const size_t smem = bf16_mma_smem_bytes();
  SKM_CUDA_TRY(cudaFuncSetAttribute(k_bf16_top2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ntiles = (c->n + kBM - 1) / kBM;
  const int grid = (int)(ntiles < c->nsm ? ntiles : c->nsm);
  const int nkb = (int)((c->d + kBK - 1) / kBK);
  SKM_PROF_BEGIN(c, "k_bf16_top2");
  k_bf16_top2<<<grid, kThreads, smem, c->st>>>(mA, mB, c->n, c->k, nkb, nnt, c->a, top2, c->cnt);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

}  // namespace skm
