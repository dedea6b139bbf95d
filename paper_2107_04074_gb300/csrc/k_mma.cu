// Dense similarity bulk on the 5th-generation tensor cores (precision form):
// S^b = X_b * C_b^T with BF16 operands (kind::f16) or FP8-E4M3 operands
// (kind::f8f6f4) and FP32 accumulation in tensor memory, fused with the
// selection of each row's recheck candidates.  FP8 operands carry power-of-two
// scales (per row for the data, 2^8 for every center), so the epilogue turns
// an accumulator into a similarity by one exact multiplication per value.
//
// One CTA per SM, persistent over tiles of 128 rows.  Warp roles:
//   warp 0  TMA producer: per (center tile, K block) one stage of a 4-stage
//           ring holding the row tile's 128 x 128-byte slice of A and the
//           256 x 128-byte slice of the centers B (64 BF16 or 128 FP8
//           elements of K), 128-byte swizzled (A comes from L2 after the
//           first center tile);
//   warp 1  allocates 512 TMEM columns; one lane issues tcgen05.mma
//           (M = 128, N = 256, K = 32 bytes per instruction: 16 BF16 or 32
//           FP8 elements) into one of two 256-column accumulators, and
//           tcgen05.commit to the barriers;
//   warps 2-9  epilogue, two groups of four: group g drains accumulator g
//           (tcgen05.ld of the warp's 32-lane TMEM quarter) while the other
//           group drains the other one.
// Selection.  A center can be a recheck candidate only if its BF16 similarity
// is within 2w of the row's best v1 (w = eps_b + delta_i).  Each 64-column
// chunk first raises the running best, then appends every value above
// thr = max(tau, v1_run - W2) (W2 slightly above 2w; tau from a lower bound l
// on the best similarity when one is known) to the row's buffer in shared
// memory: a predicated store, no divergent code; a buffer more than half full
// first drops the entries the rising threshold has passed.  At the end of the
// row tile each group compacts its buffer to its final threshold and writes it
// out; k_topk_merge then merges the two lists of a row into the output list,
// off the tensor kernel's critical path.  A buffer that still overflows marks
// the row for a whole-row recheck.
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
constexpr int kRowBytes = 128;    // K bytes per 128-byte swizzled row of a stage
constexpr int kStages = 4;        // A + B ring
constexpr int kCap = 16;          // appended values a row's buffer holds per group
constexpr int kThreads = 320;     // 2 + 8 warps
constexpr uint32_t kABytes = kBM * kRowBytes;  // 16 KB per stage
constexpr uint32_t kBBytes = kBN * kRowBytes;  // 32 KB per stage
constexpr uint32_t kStageBytes = kABytes + kBBytes;
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t timeout_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (now_ns() - t0 > timeout_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Self-test of the bounded wait: one warp waits on a barrier that nothing
// completes; the wait must give up after timeout_ns and report E_TIMEOUT.
__global__ void k_wait_selftest(uint64_t timeout_ns, unsigned long long* __restrict__ flag) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, &abort_flag, timeout_ns);
  if (!ok && threadIdx.x == 0) atomicOr(flag, (unsigned long long)E_TIMEOUT);
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

// Instruction descriptors, D = F32, A and B K-major: kind::f16 with
// A = B = BF16 (type code 1), kind::f8f6f4 with A = B = E4M3 (type code 0).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
  if (FP8)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, "
        "p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
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

// max(a, b, c) in one instruction.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Two 32-column loads in flight, one wait.
__device__ __forceinline__ void tmem_ld32x2(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr + 32));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct MmaShared {
  uint64_t full[kStages], empty[kStages];
  uint64_t acc_full[2], acc_empty[2];
  uint32_t tmem_base;
  int abort_flag;
};

// A group's list of a row as written out: cand_n[g n + row] = its length
// (0..kCap) or kCandOverflow; entry q at cand[(g kCap + q) n + row].
constexpr uint8_t kCandOverflow = 0xFF;

// Insert (s, j) into a list ordered by value (descending), then center
// (ascending), if it ranks above the last entry; entries with center -1
// rank below real ones of the same value.
__device__ __forceinline__ bool ranks_above(float s, int32_t j, float v, int32_t i) {
  return s > v || (s == v && (i < 0 || j < i));
}
__device__ __forceinline__ void topk_insert(float (&tv)[kTopK], int32_t (&ti)[kTopK], float s, int32_t j) {
  if (!ranks_above(s, j, tv[kTopK - 1], ti[kTopK - 1])) return;
#pragma unroll
  for (int p = kTopK - 1; p > 0; --p) {
    if (ranks_above(s, j, tv[p - 1], ti[p - 1])) {
      tv[p] = tv[p - 1];
      ti[p] = ti[p - 1];
    } else if (ranks_above(s, j, tv[p], ti[p])) {
      tv[p] = s;
      ti[p] = j;
    }
  }
  if (ranks_above(s, j, tv[0], ti[0])) {
    tv[0] = s;
    ti[0] = j;
  }
}

// Keep the buffer entries above thr (in order); returns the count.
__device__ __forceinline__ int compact_buf(uint2* b, int nap, float thr) {
  int w = 0;
  for (int q = 0; q < nap; ++q) {
    const uint2 e = b[q * kBM];
    if (__uint_as_float(e.x) > thr) {
      b[w * kBM] = e;
      ++w;
    }
  }
  return w;
}

// Per row and group: the reduced-precision similarities above the group's
// final threshold (with their centers), or an overflow mark.  FP8: rsc[row]
// is the exact power of two 1 / (row scale * center scale) that turns the
// row's accumulators into similarities.
template <bool FP8>
__global__ void __launch_bounds__(kThreads, 1) k_bf16_topk(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, int64_t n,
                                                          int32_t k, int nkb, int nnt, const float* __restrict__ lb,
                                                          const float* __restrict__ dlt, const float* __restrict__ exr,
                                                          const float* __restrict__ ebc, const float* __restrict__ rsc,
                                                          int use_thr, uint2* __restrict__ cand,
                                                          uint8_t* __restrict__ cand_n,
                                                          unsigned long long* __restrict__ cnt) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the swizzled tiles
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* St = base;                                         // kStages x (A 16 KB, B 32 KB)
  uint2* buf = reinterpret_cast<uint2*>(base + (size_t)kStages * kStageBytes);  // [2][kCap][kBM]
  MmaShared* sh = reinterpret_cast<MmaShared*>(buf + 2 * kCap * kBM);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (n + kBM - 1) / kBM;
  const uint32_t idesc = FP8 ? idesc_e4m3(kBM, kBN) : idesc_bf16(kBM, kBN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
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
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
        for (int nt = 0; nt < nnt && ok; ++nt)
          for (int kb = 0; kb < nkb; ++kb, ++gidx) {
            const int s = gidx % kStages;
            if (gidx >= (uint32_t)kStages) ok = mbar_wait(&sh->empty[s], ((gidx / kStages) - 1) & 1, abort_flag);
            if (!ok) break;
            unsigned char* st = St + (size_t)s * kStageBytes;
            mbar_expect_tx(&sh->full[s], kStageBytes);
            // x = the first K element of the block: 128 bytes per block, so
            // x times the element size is a multiple of 16 bytes
            const int kx = kb * (FP8 ? kRowBytes : kRowBytes / 2);
            tma_load_2d(&mapA, &sh->full[s], st, kx, (int)(tile * kBM));
            tma_load_2d(&mapB, &sh->full[s], st + kABytes, kx, nt * kBN);
          }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t gidx = 0, accidx = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int nt = 0; nt < nnt && ok; ++nt, ++accidx) {
          const uint32_t b = accidx & 1, use = accidx >> 1;
          if (use > 0) ok = mbar_wait(&sh->acc_empty[b], (use - 1) & 1, abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d_tmem = tmem + b * kBN;
          for (int kb = 0; kb < nkb; ++kb, ++gidx) {
            const int s = gidx % kStages;
            ok = mbar_wait(&sh->full[s], (gidx / kStages) & 1, abort_flag);
            if (!ok) break;
            tc_fence_after();
            const uint32_t a_addr = smem_u32(St + (size_t)s * kStageBytes);
            const uint32_t b_addr = a_addr + kABytes;
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk)
              umma<FP8>(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc,
                        (kb > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&sh->empty[s]);  // the stage is free once these MMAs are done
          }
          if (!ok) break;
          umma_commit(&sh->acc_full[b]);
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2-9)
    const int grp = (warp - 2) >> 2;  // drains accumulator buffer grp
    const int quarter = warp & 3;     // the TMEM lanes this warp may read
    const int r_in_tile = quarter * 32 + lane;
    uint2* mybuf = buf + (size_t)grp * kCap * kBM + r_in_tile;  // slot c at mybuf[c * kBM]
    uint32_t accidx = 0;
    int lt = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
      const int64_t row = tile * kBM + r_in_tile;
      const bool valid = row < n;
      float tau = -INFINITY, W2 = 0.f, f = 1.f;
      if (valid) {
        if (FP8) f = rsc[row];
        const float eps_b = bf16_eps(exr, ebc, row);
        W2 = __fadd_ru(__fmul_ru(2.f, __fadd_ru(eps_b, dlt[row])), 0x1.0p-20f);
        if (use_thr) tau = __fsub_rd(__fsub_rd(__fsub_rd(lb[row], eps_b), W2), 0x1.0p-20f);
      }
      float v1 = tau;
      int nap = 0;  // values appended (may exceed kCap: overflow)
      for (int nt = 0; nt < nnt; ++nt, ++accidx) {
        const uint32_t b = accidx & 1, use = accidx >> 1;
        if ((int)b != grp) continue;
        ok = __all_sync(SKM_FULL_MASK, mbar_wait(&sh->acc_full[b], use & 1, abort_flag));
        if (!ok) break;
        tc_fence_after();
        for (int c = 0; c < kBN / 64; ++c) {
          const int jb = nt * kBN + c * 64;
          if (jb >= k) break;  // the same for the whole warp
          uint32_t r[64];
          tmem_ld32x2(tmem + ((uint32_t)(quarter * 32) << 16) + b * kBN + c * 64, r);
          if (FP8) {  // accumulators -> similarities (exact: f is a power of two)
#pragma unroll
            for (int q = 0; q < 64; ++q) r[q] = __float_as_uint(__fmul_rn(__uint_as_float(r[q]), f));
          }
          if (jb + 64 > k) {  // last chunk: columns past k belong to padding centers
#pragma unroll
            for (int q = 0; q < 64; ++q)
              if (jb + q >= k) r[q] = __float_as_uint(-INFINITY);
          }
          // chunk maximum by a tree of three-input maxima (64 -> 22 -> 8 -> 3 -> 1)
          float m1[22];
#pragma unroll
          for (int q = 0; q < 21; ++q)
            m1[q] = fmax3(__uint_as_float(r[3 * q]), __uint_as_float(r[3 * q + 1]), __uint_as_float(r[3 * q + 2]));
          m1[21] = __uint_as_float(r[63]);
          float m2[8];
#pragma unroll
          for (int q = 0; q < 7; ++q) m2[q] = fmax3(m1[3 * q], m1[3 * q + 1], m1[3 * q + 2]);
          m2[7] = m1[21];
          const float cm = fmax3(fmax3(m2[0], m2[1], m2[2]), fmax3(m2[3], m2[4], m2[5]), fmaxf(m2[6], m2[7]));
          v1 = fmaxf(v1, cm);
          const float thr = fmaxf(tau, __fsub_rd(v1, W2));
          // a buffer more than half full drops the entries the threshold has
          // passed by since (one warp-uniform test per chunk; rarely taken)
          if (__any_sync(SKM_FULL_MASK, nap > kCap / 2)) {
            if (nap > kCap / 2 && nap <= kCap) {
              int w = 0;
              for (int q = 0; q < nap; ++q) {
                const uint2 e = mybuf[q * kBM];
                if (__uint_as_float(e.x) > thr) {
                  mybuf[w * kBM] = e;
                  ++w;
                }
              }
              nap = w;
            }
          }
          // predicated appends, no branches: the store happens only while the
          // row's buffer has room, the count goes on (overflow is detected)
#pragma unroll
          for (int q = 0; q < 64; ++q) {
            const bool keep = __uint_as_float(r[q]) > thr;
            const bool room = nap < kCap;
            if (keep && room) mybuf[nap * kBM] = make_uint2(r[q], (uint32_t)(jb + q));
            nap += keep ? 1 : 0;
          }
        }
        tc_fence_before();
        mbar_arrive(&sh->acc_empty[b]);
      }
      if (!ok) break;
      // keep only the entries above the group's final threshold, and write
      // them out (coalesced: consecutive rows of a slot are adjacent)
      if (nap <= kCap) nap = compact_buf(mybuf, nap, fmaxf(tau, __fsub_rd(v1, W2)));
      if (valid) {
        cand_n[(int64_t)grp * n + row] = nap > kCap ? kCandOverflow : (uint8_t)nap;
        if (nap <= kCap)
          for (int q = 0; q < nap; ++q) cand[(int64_t)(grp * kCap + q) * n + row] = mybuf[q * kBM];
      }
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

// Thread per row: the two groups' lists of k_bf16_topk merged into the
// output.  Per row: the (at most 8) largest BF16 similarities above B in
// descending order with their centers, then entries with center -1 holding
// B = max(tau, best - W2), where best is the row's largest value (each group
// appended its running best whenever it rose) -- B bounds every center not
// listed.  A row with an overflowed list, or with nothing above B, gets
// center -1 and value +inf throughout (a whole-row recheck).
__global__ void __launch_bounds__(256) k_topk_merge(const uint2* __restrict__ cand, const uint8_t* __restrict__ cand_n,
                                                    int64_t n, const float* __restrict__ lb,
                                                    const float* __restrict__ dlt, const float* __restrict__ exr,
                                                    const float* __restrict__ ebc, int use_thr,
                                                    float* __restrict__ topv, int32_t* __restrict__ topi) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const float eps_b = bf16_eps(exr, ebc, row);
    const float W2 = __fadd_ru(__fmul_ru(2.f, __fadd_ru(eps_b, dlt[row])), 0x1.0p-20f);
    const float tau = use_thr ? __fsub_rd(__fsub_rd(__fsub_rd(lb[row], eps_b), W2), 0x1.0p-20f) : -INFINITY;
    const int c0 = cand_n[row], c1 = cand_n[n + row];
    const bool over = c0 == kCandOverflow || c1 == kCandOverflow;
    float tv[kTopK];
    int32_t ti[kTopK];
#pragma unroll
    for (int q = 0; q < kTopK; ++q) {
      tv[q] = INFINITY;
      ti[q] = -1;
    }
    if (!over) {
      float best = tau;
      for (int q = 0; q < c0; ++q) best = fmaxf(best, __uint_as_float(cand[(int64_t)q * n + row].x));
      for (int q = 0; q < c1; ++q) best = fmaxf(best, __uint_as_float(cand[(int64_t)(kCap + q) * n + row].x));
      const float bnd = fmaxf(tau, __fsub_rd(best, W2));
#pragma unroll
      for (int q = 0; q < kTopK; ++q) tv[q] = bnd;
      for (int q = 0; q < c0; ++q) {
        const uint2 e = cand[(int64_t)q * n + row];
        const float sv = __uint_as_float(e.x);
        if (sv > bnd) topk_insert(tv, ti, sv, (int32_t)e.y);
      }
      for (int q = 0; q < c1; ++q) {
        const uint2 e = cand[(int64_t)(kCap + q) * n + row];
        const float sv = __uint_as_float(e.x);
        if (sv > bnd) topk_insert(tv, ti, sv, (int32_t)e.y);
      }
      if (ti[0] < 0) {
#pragma unroll
        for (int q = 0; q < kTopK; ++q) tv[q] = INFINITY;
      }
    }
    float4* vo = reinterpret_cast<float4*>(topv + row * kTopK);
    int4* io = reinterpret_cast<int4*>(topi + row * kTopK);
    vo[0] = make_float4(tv[0], tv[1], tv[2], tv[3]);
    vo[1] = make_float4(tv[4], tv[5], tv[6], tv[7]);
    io[0] = make_int4(ti[0], ti[1], ti[2], ti[3]);
    io[1] = make_int4(ti[4], ti[5], ti[6], ti[7]);
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

// rows x cols of BF16 (esize 2) or FP8 (esize 1), row-major (cols
// contiguous); boxes of 128 bytes of columns x box_rows.
int make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows, int esize) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return SKM_EUNSUPPORTED;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * esize};
  const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esize), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                         const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SKM_OK : SKM_EINVAL;
}

}  // namespace

size_t bf16_mma_smem_bytes() {
  return 1024 + (size_t)kStages * kStageBytes + sizeof(uint2) * 2 * kCap * kBM + sizeof(MmaShared);
}

// rows of 16-byte multiples for the tensor maps
int bf16_mma_supported(int64_t d) { return d % 8 == 0; }
int fp8_mma_supported(int64_t d) { return d % 16 == 0; }

// Xb: n x d BF16 or FP8 (scaled unit rows); Cb: (ceil(k/256)*256) x d of the
// same type (zero rows past k).  Columns past d read as zeros (the tensor
// map's out-of-bounds fill).  use_thr: lb holds a lower bound on every row's
// best exact similarity.
int bf16_topk(skm_ctx* c, const void* Xb, const void* Cb, int use_thr, float* topv, int32_t* topi) {
  const bool fp8 = c->precision == SKM_PREC_FP8;
  if (fp8 ? !fp8_mma_supported(c->d) : !bf16_mma_supported(c->d)) return SKM_EUNSUPPORTED;
  const int esize = fp8 ? 1 : 2;
  CUtensorMap mA, mB;
  const int nnt = (c->k + kBN - 1) / kBN;
  int rc = make_map(&mA, Xb, c->n, c->d, kBM, esize);
  if (rc) return rc;
  rc = make_map(&mB, Cb, (int64_t)nnt * kBN, c->d, kBN, esize);
  if (rc) return rc;
  const size_t smem = bf16_mma_smem_bytes();
  const void* kern = fp8 ? (const void*)k_bf16_topk<true> : (const void*)k_bf16_topk<false>;
  SKM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ntiles = (c->n + kBM - 1) / kBM;
  const int grid = (int)(ntiles < c->nsm ? ntiles : c->nsm);
  const int kblk = kRowBytes / esize;  // K elements per block
  const int nkb = (int)((c->d + kblk - 1) / kblk);
  SKM_PROF_BEGIN(c, fp8 ? "k_fp8_topk" : "k_bf16_topk");
  if (fp8)
    k_bf16_topk<true><<<grid, kThreads, smem, c->st>>>(mA, mB, c->n, c->k, nkb, nnt, c->lb, c->dlt, c->exr, c->ebc,
                                                       c->rsc, use_thr, c->cand, c->cand_n, c->cnt);
  else
    k_bf16_topk<false><<<grid, kThreads, smem, c->st>>>(mA, mB, c->n, c->k, nkb, nnt, c->lb, c->dlt, c->exr,
                                                        c->ebc, nullptr, use_thr, c->cand, c->cand_n, c->cnt);
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_topk_merge");
  const int64_t gm = (c->n + 255) / 256, gcap = (int64_t)c->nsm * 16;
  k_topk_merge<<<(unsigned)(gm < gcap ? gm : gcap), 256, 0, c->st>>>(c->cand, c->cand_n, c->n, c->lb, c->dlt,
                                                                     c->exr, c->ebc, use_thr, topv, topi);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

int wait_selftest(int64_t timeout_ns, cudaStream_t st) {
  unsigned long long* flag = nullptr;
  SKM_CUDA_TRY(cudaMallocAsync((void**)&flag, sizeof(unsigned long long), st));
  SKM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned long long), st));
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)timeout_ns, flag);
  SKM_CUDA_TRY(cudaGetLastError());
  note_launch(1);
  unsigned long long h = 0;
  SKM_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(h), cudaMemcpyDeviceToHost, st));
  SKM_CUDA_TRY(cudaFreeAsync(flag, st));
  SKM_CUDA_TRY(cudaStreamSynchronize(st));
  return (h & E_TIMEOUT) ? SKM_ETIMEOUT : SKM_OK;
}

}  // namespace skm
