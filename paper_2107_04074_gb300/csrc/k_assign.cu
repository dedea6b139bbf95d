// The assignment step (Section 5) and its pruned forms: Hamerly (5.3, 5.4)
// and Elkan (5.1, 5.2) with bounds kept on cosines (Section 4).
//
// Kernels:
//   k_rows_top2      warp per row: all k similarities of a CSR row against the
//                    term-major centers (an SpMM row fused with a top-2 argmax
//                    under the tie rule); initialises / refreshes the bounds.
//   k_ham_bounds     thread per point: Eq. (eqn:l-bound), Eq. (eqn:u-hamerly-2),
//                    prune test, compaction of the survivors into a worklist.
//   k_ham_tighten    warp per survivor: exact <x, c_a> (l made tight), retest,
//                    compaction of the points that need a whole row.
//   k_elk_bounds     warp per point: Eq. (eqn:l-bound) and Eq. (eqn:u-elkan) on
//                    the whole bound row, prune tests, compaction of survivors.
//   k_elk_recompute  8-lane group per survivor: its surviving (point, center)
//                    pairs compacted into lanes, their exact similarities in
//                    one pass over the row, reassignment under the tie rule.
//   k_elk_recompute_long  the same for survivors with long rows, a warp per
//                    point (32 row entries gathered per round trip).
//   k_rows_top2 MODE 4  the screened whole-row pass of the Elkan variants for
//                    k > 128: all k similarities against an FP16 copy of the
//                    centers (half the bytes gathered: with k = 1000 the
//                    center table is far larger than L2 and the FP32 pass
//                    streams it from DRAM) with a proven error bound; rows
//                    whose label the bound decides are done, the others go
//                    to an exact pass (pairs or whole rows).
#include <climits>
#include <mutex>
#include <unordered_map>

#include "skm_internal.cuh"

namespace skm {

namespace {

#define TRY_K(x)                   \
  do {                             \
    const int r__ = (x);           \
    if (r__ != SKM_OK) return r__; \
  } while (0)

constexpr int kBlock = 256;
constexpr int kTile = 8;       // points per warp tile of k_elk_bounds
constexpr int kLongRow = 256;  // Elkan survivors with longer rows go to the warp-per-point recompute

// Dynamic scheduling over `total` items by `nworkers` warps (or 8-lane
// groups): worker w takes item w first, then items nworkers + c for
// c = 0, 1, ... from the kernel's own cursor counter (one atomic per item,
// issued while the worker is busy with its current item and read when it is
// done), so that long rows do not leave the rest of a persistent grid idle.
// When every item fits the first round no atomic is issued.  The cursors are
// zeroed with the other counters at the start of each assignment (each of
// these kernels runs at most once per assignment), so no memset separates
// the kernels of an iteration.
__device__ __forceinline__ unsigned long long grab_issue(unsigned long long* cursor, bool leader, int64_t nworkers,
                                                         int64_t total) {
  return (leader && total > nworkers) ? (unsigned long long)nworkers + atomicAdd(cursor, 1ull) : ~0ull >> 1;
}
__device__ __forceinline__ int64_t grab_take(unsigned long long v, unsigned mask, int width) {
  return (int64_t)__shfl_sync(mask, v, 0, width);
}

// acc += v * c for four center sums (scalar FMAs: packed fma.rn.f32x2 pairs
// were measured 3 % slower in the whole-row pass, which is bound by its
// gathers, not by issue).
__device__ __forceinline__ void fma4(float4& acc, float v, const float4& c) {
  acc.x = __fmaf_rn(v, c.x, acc.x);
  acc.y = __fmaf_rn(v, c.y, acc.y);
  acc.z = __fmaf_rn(v, c.z, acc.z);
  acc.w = __fmaf_rn(v, c.w, acc.w);
}

// NB consecutive entries (offsets and values) of a warp's 32-entry buffer in
// shared memory, read by every lane with broadcast vector loads (one shared
// wavefront per four entries, against one per entry and array for shuffles).
// q is a multiple of NB, and NB divides 32.
template <int NB>
__device__ __forceinline__ void entries_from_smem(const uint32_t* st, const float* sv, int q, uint32_t (&t)[NB],
                                                  float (&v)[NB]) {
  if constexpr (NB % 4 == 0) {
#pragma unroll
    for (int x = 0; x < NB / 4; ++x) {
      const uint4 a = *reinterpret_cast<const uint4*>(st + q + 4 * x);
      const float4 c = *reinterpret_cast<const float4*>(sv + q + 4 * x);
      t[4 * x] = a.x;
      t[4 * x + 1] = a.y;
      t[4 * x + 2] = a.z;
      t[4 * x + 3] = a.w;
      v[4 * x] = c.x;
      v[4 * x + 1] = c.y;
      v[4 * x + 2] = c.z;
      v[4 * x + 3] = c.w;
    }
  } else if constexpr (NB == 2) {
    const uint2 a = *reinterpret_cast<const uint2*>(st + q);
    const float2 c = *reinterpret_cast<const float2*>(sv + q);
    t[0] = a.x;
    t[1] = a.y;
    v[0] = c.x;
    v[1] = c.y;
  } else {
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      t[u] = st[q + u];
      v[u] = sv[q + u];
    }
  }
}

// Raw loads of four center values, converted just before the FMAs: FP16
// centers take half the registers, so twice as many row entries' gathers can
// be in flight at once.
template <typename CT>
struct RawC4;
template <>
struct RawC4<float> {
  using type = float4;
  static __device__ __forceinline__ type load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ type load_v(const type* p) { return __ldg(p); }
  static __device__ __forceinline__ type zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ float4 f4(type r) { return r; }
};
template <>
struct RawC4<__half> {
  using type = uint2;
  static __device__ __forceinline__ type load(const __half* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }
  static __device__ __forceinline__ type load_v(const type* p) { return __ldg(p); }
  static __device__ __forceinline__ type zero() { return make_uint2(0u, 0u); }
  static __device__ __forceinline__ float4 f4(type r) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

// MODE 0: labels only (standard).  MODE 1: also l(i) and Hamerly's u(i).
// MODE 2: also l(i) and every Elkan bound u(i,j).  MODE 3 (Yin-Yang): only
// the centers of the live groups (a group of 8 consecutive centers is live
// when its bound u(i,G) = ub[G * ustride + i] exceeds l(i) - 2 delta, and
// always for the group of a(i); before the first assignment all are live)
// are gathered and compared; l(i) and the live groups' bounds are rewritten.
// A lane's four centers always lie in one group.
// Lane L owns the centers j = 128 g + 4 L + c (c = 0..3, g = 0..G-1) and
// gathers them with one 16-byte load per row entry and group; each center's
// sum runs over the row entries in CSR order (the canonical order).
// For a batch (runs != nullptr) each row works on its run's slice of the
// centers (global ids koff + j) and its run's bound row.
// MODE 4 (screened Elkan whole rows, CT = __half, single runs, one pass):
// the similarities s^ against the FP16 centers h_j satisfy |s^ - s| <= eps_i
// for the exact cosine s, with eps_i = E + 1.001 delta_i (E = escr[0] bounds
// |h_j - c_j| for every j, so |<x^, h_j - c_j>| <= E by Cauchy-Schwarz; the
// FP32 chain over the products with h, |h_j| <= 1 + 6u + E, errs by at most
// delta_i (1 + E), and E < 10^-3).  So |s^ - f| <= w_i = eps_i + delta_i for
// the canonical FP32 similarity f.  Every u(i,j) becomes s^_ij + eps_i.  If
// the best two differ by more than 2 w_i the best center is the one the
// exact pass would pick: label and l(i) = s^_1 - eps_i.  Otherwise the
// current label stays, l(i) = s^_cur - eps_i, and the row goes to the exact
// pass: the pair recompute (w3) when at most 7 centers pass Elkan's test
// against these bounds (counted from the bound row just written), else an
// FP32 whole row (w4).
// MODE 5 (screened Hamerly whole rows, the same bound): a row whose best two
// FP16 similarities differ by more than 2 w_i takes the best center as its
// label, l(i) = s^_1 - eps_i and u(i) = s^_2 + eps_i (bounds on the exact
// similarities); any other row goes to an FP32 whole row (w4).
// Resident blocks asked of the compiler: two (128 registers, no spills).
// Latency-bound as it is, the kernel runs faster with more gathers in flight
// than with more warps: at 128 centers, 16 row entries per warp with 16 warps
// per SM beat 8 entries with 24 warps (9 % per pass), and at 256 and 512
// centers two blocks without spills beat three with them (2-4 % per run).
constexpr int rows_min_blocks(int) { return 2; }

template <typename VT, typename CT, int G, int MODE, bool BATCH>
__global__ void __launch_bounds__(kBlock, rows_min_blocks(G)) k_rows_top2(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const CT* __restrict__ Ct, int32_t k,
    int64_t kst, const int32_t* __restrict__ row_run, const RunDesc* __restrict__ runs,
    const int32_t* __restrict__ list, const unsigned long long* __restrict__ list_cnt, int64_t nrows,
    int64_t ustride, int32_t* __restrict__ a, float* __restrict__ lb, float* __restrict__ ub,
    int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old, unsigned long long* __restrict__ cnt,
    unsigned long long* __restrict__ cursor, const float* __restrict__ escr, int32_t* __restrict__ w3,
    int32_t* __restrict__ w4) {
  constexpr int KT = 128 * G;                     // centers per pass over the row
  // row entries batched per step (their gathers in flight together): 16 for
  // one group of centers; for wider forms, twice as many with FP16 centers,
  // whose raw loads take half the registers
  constexpr int NB = G == 1 ? 16 : (sizeof(CT) == 2 ? 2 : 1) * (G >= 8 ? 1 : 8 / G);
  using Raw = RawC4<CT>;
  const int lane = threadIdx.x & 31;
  // each warp's current 32 row entries (vector offsets, values), read back by
  // all lanes with broadcast loads
  __shared__ __align__(16) uint32_t ent_t[kBlock / 32][32];
  __shared__ __align__(16) float ent_v[kBlock / 32][32];
  uint32_t* const et = ent_t[threadIdx.x >> 5];
  float* const ev = ent_v[threadIdx.x >> 5];
  const int64_t total = list ? (int64_t)(*list_cnt) : nrows;
  unsigned long long my_changed = 0, my_sims = 0;
  ChangedBuf chb;
  // screened pass: E, and whether it is small enough for the bound (else every row goes to the exact pass)
  constexpr bool SCR = (MODE == 4 || MODE == 5);
  const float Escr = SCR ? escr[0] : 0.f;
  const bool scr_ok = SCR && Escr < 1e-3f;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nxt;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
       w = grab_take(nxt, SKM_FULL_MASK, 32)) {
    nxt = grab_issue(cursor, lane == 0, nw, total);
    const int64_t i = list ? (int64_t)list[w] : w;
    const RowGeom rg = row_geom<BATCH>(i, k, kst, 0, row_run, runs);
    const int32_t kr = rg.k;
    const int64_t b = rp[i], e = rp[i + 1];
    const float ri = rinv[i];
    const float dl = dlt[i];
    const int32_t cur = a[i] - rg.koff;  // local; negative before the first assignment
    float v1 = -INFINITY, v2 = -INFINITY, vcur = -INFINITY;
    int j1 = INT_MAX;
    float sv[MODE == 3 ? G : 1][4];  // Yin-Yang: this lane's similarities (-inf: not live)
    bool live[MODE == 3 ? G : 1];
    const float eps = SCR ? __fadd_ru(Escr, __fmul_ru(dl, 1.001f)) : 0.f;
    unsigned live_cnt = 0;
    const float L3 = (MODE == 3 && cur >= 0) ? __fsub_rd(lb[i], 2.f * dl) : -INFINITY;
    for (int j0 = 0; j0 < kr; j0 += KT) {
      float4 acc[G];
      bool ok[G];  // this lane's 4-center slot of group g lies inside the padded row
#pragma unroll
      for (int g = 0; g < G; ++g) {
        acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        ok[g] = (j0 + g * 128 + lane * 4) < kr;
        if (MODE == 3) {
          const int grp = (j0 + g * 128 + lane * 4) >> 3;
          const int64_t ya = BATCH ? rg.ybase + (int64_t)grp * rg.ystride : (int64_t)grp * ustride + i;
          live[g] = ok[g] && (cur < 0 || grp == (cur >> 3) || __ldg(ub + ya) > L3);
          ok[g] = live[g];
        }
      }
      // this lane's four centers of group 0 as one vector; an entry's term t
      // becomes the 32-bit offset t kst / 4 in vectors (d kst < 2^32 is
      // checked at init), computed once by the lane that loads the entry
      const typename Raw::type* cbase = reinterpret_cast<const typename Raw::type*>(Ct + rg.koff + j0 + lane * 4);
      const uint32_t kv = (uint32_t)(kst >> 2);
      // the row's entries 32 at a time, the next 32 loaded ahead
      uint32_t tt_n = 0;
      float vv_n = 0.f;
      if (b + lane < e) {
        tt_n = (uint32_t)__ldg(col + b + lane) * kv;
        vv_n = to_f32(val[b + lane]);
      }
      for (int64_t p0 = b; p0 < e; p0 += 32) {
        __syncwarp();  // the previous chunk's reads are done
        et[lane] = tt_n;
        ev[lane] = vv_n;
        __syncwarp();
        if (p0 + 32 + lane < e) {
          tt_n = (uint32_t)__ldg(col + p0 + 32 + lane) * kv;
          vv_n = to_f32(val[p0 + 32 + lane]);
        }
        const int nq = (int)min((int64_t)32, e - p0);
        // full batches of NB entries (NB divides 32), then the row's ragged
        // tail as one more batch whose missing entries load and add nothing,
        // so that it costs one round trip, not one per entry
        int q = 0;
        for (; q + NB <= nq; q += NB) {
          uint32_t t[NB];
          float v[NB];
          typename Raw::type cv[NB][G];
          entries_from_smem<NB>(et, ev, q, t, v);
#pragma unroll
          for (int u = 0; u < NB; ++u)
#pragma unroll
            for (int g = 0; g < G; ++g)
              cv[u][g] = ok[g] ? Raw::load_v(cbase + t[u] + g * 32) : Raw::zero();
#pragma unroll
          for (int u = 0; u < NB; ++u)
#pragma unroll
            for (int g = 0; g < G; ++g) fma4(acc[g], v[u], Raw::f4(cv[u][g]));
        }
        if (q < nq) {
          const int nb = nq - q;  // 1 .. NB - 1 entries left
          uint32_t t[NB];
          float v[NB];
          typename Raw::type cv[NB][G];
          entries_from_smem<NB>(et, ev, q, t, v);  // entries past the row's end are stale; not used
#pragma unroll
          for (int u = 0; u < NB; ++u)
#pragma unroll
            for (int g = 0; g < G; ++g)
              cv[u][g] = (ok[g] && u < nb) ? Raw::load_v(cbase + t[u] + g * 32) : Raw::zero();
#pragma unroll
          for (int u = 0; u < NB; ++u)
            if (u < nb)
#pragma unroll
              for (int g = 0; g < G; ++g) fma4(acc[g], v[u], Raw::f4(cv[u][g]));
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const float av[4] = {acc[g].x, acc[g].y, acc[g].z, acc[g].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + g * 128 + lane * 4 + c;
          if (MODE == 3) sv[g][c] = -INFINITY;
          if (j < kr && (MODE != 3 || live[g])) {
            const float s = __fmul_rn(av[c], ri);
            if (MODE == 3) {
              sv[g][c] = s;
              ++live_cnt;
            }
            if (MODE == 2) ub[rg.ubase + j] = __fadd_ru(s, dl);
            if (MODE == 4) ub[rg.ubase + j] = __fadd_ru(s, eps);
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
    // screened: decided (scr_dec 0), pair recompute (1) or exact whole row (2)
    int scr_dec = 0;
    float scr_l = 0.f;
    if (MODE == 5) {
      const float w2x = __fmul_ru(2.f, __fadd_ru(eps, dl));
      if (scr_ok && __fsub_rd(v1, v2) > w2x) {
        nb = j1;
        scr_l = __fsub_rd(v1, eps);
      } else {
        nb = cur;
        scr_dec = 2;
      }
    }
    if (MODE == 4) {
      const float w2x = __fmul_ru(2.f, __fadd_ru(eps, dl));
      if (scr_ok && __fsub_rd(v1, v2) > w2x) {
        nb = j1;  // the exact standard pass picks j1: it beats every other center strictly
        scr_l = __fsub_rd(v1, eps);
      } else if (scr_ok && cur >= 0) {
        // keep the label; count the centers Elkan's test (u(i,j) > l - 2 delta)
        // lets through against the bound row written above, as the pair
        // recompute will
        nb = cur;
        scr_l = __fsub_rd(vcur, eps);
        const float L = __fsub_rd(scr_l, 2.f * dl);
        __syncwarp();
        int m = 0;
        for (int jb = lane * 4; jb < kr; jb += 128) {
          const float4 u4 = *reinterpret_cast<const float4*>(ub + rg.ubase + jb);
          m += (jb + 0 < kr && jb + 0 != cur && u4.x > L) ? 1 : 0;
          m += (jb + 1 < kr && jb + 1 != cur && u4.y > L) ? 1 : 0;
          m += (jb + 2 < kr && jb + 2 != cur && u4.z > L) ? 1 : 0;
          m += (jb + 3 < kr && jb + 3 != cur && u4.w > L) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(SKM_FULL_MASK, m, o);
        scr_dec = m <= 7 ? 1 : 2;
      } else {
        nb = cur;
        scr_dec = 2;
      }
    }
    if (MODE == 3) {
      // the live groups' new bounds: the best of their other centers (two
      // lanes per group)
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int jb = g * 128 + lane * 4;  // one pass: kr <= KT for this variant
        float m = -INFINITY;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (jb + c != nb) m = fmaxf(m, sv[g][c]);
        m = fmaxf(m, __shfl_xor_sync(SKM_FULL_MASK, m, 1));
        const int64_t ya = BATCH ? rg.ybase + (int64_t)(jb >> 3) * rg.ystride : (int64_t)(jb >> 3) * ustride + i;
        if (live[g] && (lane & 1) == 0) ub[ya] = (m == -INFINITY) ? -1.f : __fadd_ru(m, dl);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) live_cnt += __shfl_xor_sync(SKM_FULL_MASK, live_cnt, o);
    }
    if (lane == 0) {
      if (!SCR || nb >= 0) a[i] = rg.koff + nb;
      my_changed += (nb != cur);
      my_sims += MODE == 3 ? (unsigned long long)live_cnt : (unsigned long long)kr;
      if (MODE >= 1 && MODE <= 3) lb[i] = __fsub_rd(v1, dl);
      if (MODE == 1) ub[i] = (kr > 1) ? __fadd_ru(ssec, dl) : -1.f;
      if (MODE == 5) {
        if (scr_dec == 0) {
          lb[i] = scr_l;
          ub[i] = (kr > 1) ? __fadd_ru(v2, eps) : -1.f;
        } else {
          w4[atomicAdd(cnt + C_W4, 1ull)] = (int32_t)i;
        }
      }
      if (MODE == 4) {
        if (scr_dec < 2 || cur >= 0) lb[i] = scr_l;
        if (scr_dec == 1) {
          // long rows from the top of w3 down (ustride = n for this mode)
          if (e - b > kLongRow) w3[(ustride - 1) - (int64_t)atomicAdd(cnt + C_W3L, 1ull)] = (int32_t)i;
          else w3[atomicAdd(cnt + C_W3S, 1ull)] = (int32_t)i;
        } else if (scr_dec == 2) {
          w4[atomicAdd(cnt + C_W4, 1ull)] = (int32_t)i;
        }
      }
    }
    if (nb != cur) chb.push((int32_t)i, cur < 0 ? -1 : rg.koff + cur, chg_i, chg_old, cnt);
  }
  chb.flush(chg_i, chg_old, cnt);
  if (lane == 0) {
    if (my_changed) atomicAdd(cnt + C_CHANGED, my_changed);
    if (my_sims) atomicAdd(cnt + C_SIMS, my_sims);
  }
}

// ------------------------------------------------------------- Hamerly

// Thread per point.  A batch keeps one drift summary per run (the other
// centers of a point are those of its run), read through row_run.
template <bool FULL, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_ham_bounds(int64_t n, const int32_t* __restrict__ a,
                                                       float* __restrict__ lb, float* __restrict__ ub,
                                                       const float* __restrict__ dlt, const float* __restrict__ pdn,
                                                       const float* __restrict__ pup, const float* __restrict__ qup,
                                                       const float* __restrict__ hsel, const float* __restrict__ sc,
                                                       const int32_t* __restrict__ row_run, int tight, int moved,
                                                       const int32_t* __restrict__ hst, int32_t* __restrict__ w1,
                                                       int32_t* __restrict__ w2, unsigned long long* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // tightening skipped this iteration: the survivors go to the whole-row list
  // at once (and are still counted as survivors)
  const bool skip_t = hst[0] != 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool take = false;
    if (i < n) {
      const int32_t ai = a[i];
      float l = lb[i], u = ub[i];
      if (moved) {
        // p'(a) = min_{j != a} p(j): the worst drift among the other centers
        const float* hs = BATCH ? hsel + (int64_t)HSEL_N * row_run[i] : hsel;
        const int jmin_d = (int)hs[0], jmin_u = (int)hs[3], jmax_q = (int)hs[6];
        const float pdm = (ai == jmin_d) ? hs[2] : hs[1];
        const float pum = (ai == jmin_u) ? hs[5] : hs[4];
        const float qm = (ai == jmax_q) ? hs[8] : hs[7];
        l = bound_l(l, pdn[ai], pup[ai], qup[ai]);
        u = bound_u_hamerly(u, pdm, pum, qm, tight);
        lb[i] = l;
        ub[i] = u;
      }
      const float L = __fsub_rd(l, 2.f * dlt[i]);
      const bool prune = (L >= u) || (FULL && L >= 0.f && L >= sc[ai]);
      take = !prune;
    }
    if (skip_t) {
      warp_push(take, (int32_t)i, w2, cnt + C_W2);
      const unsigned m = __ballot_sync(SKM_FULL_MASK, take);
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(cnt + C_W1, (unsigned long long)__popc(m));
    } else {
      warp_push(take, (int32_t)i, w1, cnt + C_W1);
    }
  }
}

// Warp per survivor (Hamerly): l(i) <- <x(i), c(a(i))> (made tight) with the
// warp-cooperative canonical similarity, then the test again; the points still
// failing go to `out`.  Each warp walks 8 consecutive survivors and pushes its
// failures with one atomic.
// Tightening costs a fraction of a whole row per survivor (about 0.4 of one
// at 128 centers or fewer, less beyond) and pays only for the survivors it
// prunes.  When Hamerly's single bound fails for nearly every point (one
// center that moves far loosens every u), it prunes almost none, so the last
// block to finish decides for the next iteration: if fewer than `thr` of at
// least 1024 tightened survivors were pruned, the next iterations send their
// survivors straight to the whole-row pass (hst[0] = 1), tightening again
// every kTightProbe-th iteration to re-measure.  Labels do not depend on it
// (the whole row computes <x, c_a> too); the similarity count does.
// hst: [0] skip this iteration, [1] iterations skipped in a row, [2] blocks done.
constexpr int kTightProbe = 8;

template <typename VT, bool FULL>
__global__ void __launch_bounds__(kBlock) k_ham_tighten(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int64_t kst,
    const int32_t* __restrict__ w1, const unsigned long long* __restrict__ w1_cnt, const int32_t* __restrict__ a,
    float* __restrict__ lb, const float* __restrict__ ub, const float* __restrict__ sc, int32_t* __restrict__ out,
    unsigned long long* __restrict__ cnt, int32_t* __restrict__ hst, float thr) {
  constexpr int TP = 8;
  const int lane = threadIdx.x & 31;
  const bool skip_t = hst[0] != 0;
  if (skip_t && blockIdx.x == 0 && threadIdx.x == 0) cnt[C_SKIP] = 1ull;
  const int64_t total = skip_t ? 0 : (int64_t)(*w1_cnt);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long sims = 0;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * TP < total; tile += nw) {
    const int64_t s0 = tile * TP;
    const int rows = (int)min((int64_t)TP, total - s0);
    int32_t my_i = 0, my_a = 0;
    int64_t my_b = 0, my_e = 0;
    if (lane < rows) {
      my_i = w1[s0 + lane];
      my_a = a[my_i];
      my_b = rp[my_i];
      my_e = rp[my_i + 1];
    }
    unsigned keep = 0;
    for (int r = 0; r < rows; ++r) {
      const int32_t i = __shfl_sync(SKM_FULL_MASK, my_i, r);
      const int32_t ai = __shfl_sync(SKM_FULL_MASK, my_a, r);
      const int64_t b = __shfl_sync(SKM_FULL_MASK, my_b, r), e = __shfl_sync(SKM_FULL_MASK, my_e, r);
      const float sim = __fmul_rn(warp_dot_one<VT>(b, e, col, val, Ct, kst, ai), rinv[i]);
      const float dl = dlt[i];
      const float l = __fsub_rd(sim, dl);
      const float L = __fsub_rd(l, 2.f * dl);
      if (lane == 0) lb[i] = l;
      if (!((L >= ub[i]) || (FULL && L >= 0.f && L >= sc[ai]))) keep |= 1u << r;
    }
    sims += (unsigned long long)rows;
    warp_push((keep >> lane) & 1u, my_i, out, cnt + C_W2);
  }
  if (lane == 0 && sims) atomicAdd(cnt + C_SIMS, sims);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(reinterpret_cast<unsigned*>(hst + 2), 1u);
    if (done == gridDim.x - 1) {  // the last block: every push and count is in
      __threadfence();
      if (!skip_t) {
        const unsigned long long t = *reinterpret_cast<volatile unsigned long long*>(cnt + C_W1);
        const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(cnt + C_W2);
        hst[0] = (t >= 1024 && (double)(t - w) < (double)thr * (double)t) ? 1 : 0;
        hst[1] = 0;
      } else if (++hst[1] >= kTightProbe - 1) {
        hst[0] = 0;
      }
      hst[2] = 0;
    }
  }
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

// ------------------------------------------------------------- Yin-Yang

// Per group of 8 consecutive centers, the worst drift: the smallest cosine
// lower bound, the largest upper bound and the largest sine bound of its
// centers (together they bound the drift of every center of the group).
__global__ void k_yy_drift(int32_t k, int32_t ng, const float* __restrict__ pdn, const float* __restrict__ pup,
                           const float* __restrict__ qup, float* __restrict__ gd) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    float pd = 1.f, pu = -1.f, q = 0.f;
    for (int j = 8 * g; j < k && j < 8 * g + 8; ++j) {
      pd = fminf(pd, pdn[j]);
      pu = fmaxf(pu, pup[j]);
      q = fmaxf(q, qup[j]);
    }
    gd[g] = pd;
    gd[ng + g] = pu;
    gd[2 * ng + g] = q;
  }
}

// Thread per point: Eq. (eqn:l-bound) for l(i) with the drift of c(a(i)),
// the clamped Eq. (eqn:u-elkan) for every group bound with the group's worst
// drift (the update grows as the drift grows, so it bounds every center of
// the group), then the global test l - 2 delta >= max_G u(i,G).  Group bounds
// are group-major (ug[G * n + i]; in a batch each run has its own block,
// ug[uoff + G n_r + (i - row0)], and its groups are the global groups
// koff / 8 ...).  Survivors go to w1.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock) k_yy_bounds(int64_t n, int32_t ng, const int32_t* __restrict__ a,
                                                      float* __restrict__ lb, float* __restrict__ ug,
                                                      const float* __restrict__ dlt, const float* __restrict__ pdn,
                                                      const float* __restrict__ pup, const float* __restrict__ qup,
                                                      const float* __restrict__ gd, int moved,
                                                      const int32_t* __restrict__ row_run,
                                                      const RunDesc* __restrict__ runs,
                                                      int32_t* __restrict__ w1, unsigned long long* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool take = false;
    if (i < n) {
      const int32_t ai = a[i];
      float l = lb[i];
      if (moved) {
        l = bound_l(l, pdn[ai], pup[ai], qup[ai]);
        lb[i] = l;
      }
      // this row's groups: all ng of a single run, or its run's own
      int32_t g0 = 0, ngr = ng;
      int64_t yb = i, ys = n;
      if (BATCH) {
        const RunDesc& R = runs[row_run[i]];
        g0 = R.koff >> 3;
        ngr = (R.k + 7) >> 3;
        yb = R.uoff + (i - R.row0);
        ys = R.n;
      }
      float umax = -INFINITY;
      for (int g = 0; g < ngr; ++g) {
        float u = ug[yb + (int64_t)g * ys];
        if (moved) {
          const int gg = g0 + g;
          u = bound_u(u, gd[gg], gd[ng + gg], gd[2 * ng + gg]);
          ug[yb + (int64_t)g * ys] = u;
        }
        umax = fmaxf(umax, u);
      }
      take = !(__fsub_rd(l, 2.f * dlt[i]) >= umax);
    }
    warp_push(take, (int32_t)i, w1, cnt + C_W1);
  }
}

// Warp per point; each warp walks a tile of kTile consecutive points: lanes
// 0..kTile-1 first update l and test the point-level rule for one point each
// (so the scalar loads overlap), then the warp streams each point's bound
// row and counts its candidate centers.  A point with 1..cap candidates goes
// to w1 (recomputed pair by pair) -- from the bottom of w1 up when its row
// has at most kLongRow entries, else from the top down (w1[n - 1 - pos], for
// the warp-per-point recompute) -- and one with more to w2 (recomputed as a
// whole row); each list gets one atomic per tile.
// While nearly every point goes to w2 (the bounds prune nothing in the early
// iterations), the bound pass is skipped: the last block to finish decides
// for the next iteration from this one's count (hst[0] = 1 when at least 98 %
// of n >= 4096 points went to w2), and a skipped pass sends every point to
// w2 without reading or writing a bound -- the whole-row pass rewrites l and
// every u(i,j) of each row anyway -- and passes the bounds again every
// kElkProbe-th iteration to re-measure.  Labels do not depend on it.
// hst: [0] skip this iteration, [1] passes skipped in a row, [2] blocks done.
constexpr int kElkProbe = 8;

template <bool FULL, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_elk_bounds(int64_t n, int32_t k, int64_t kst,
                                                       const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ row_run,
                                                       const RunDesc* __restrict__ runs, const int32_t* __restrict__ a,
                                                       float* __restrict__ lb, float* __restrict__ ub,
                                                       const float* __restrict__ dlt, const float* __restrict__ pdn,
                                                       const float* __restrict__ pup, const float* __restrict__ qup,
                                                       const float* __restrict__ cc, const float* __restrict__ sc,
                                                       int moved, int32_t cap, int32_t* __restrict__ w1,
                                                       int32_t* __restrict__ w2, unsigned long long* __restrict__ cnt,
                                                       int32_t* __restrict__ hst) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool skip_b = hst[0] != 0;
  if (skip_b) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[C_SKIP] = 1ull;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31; base < n;
         base += (int64_t)gridDim.x * blockDim.x)
      warp_push(base + lane < n, (int32_t)(base + lane), w2, cnt + C_W2);
  }
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; !skip_b && tile * kTile < n;
       tile += nw) {
    const int64_t i0 = tile * kTile;
    const int rows = (int)min((int64_t)kTile, n - i0);
    int32_t my_a = 0;
    float my_L = 0.f;
    bool my_skip = true, my_long = false;
    if (lane < rows) {
      const int64_t i = i0 + lane;
      my_long = rp[i + 1] - rp[i] > kLongRow;
      my_a = a[i];
      float l = lb[i];
      if (moved) {
        l = bound_l(l, pdn[my_a], pup[my_a], qup[my_a]);
        lb[i] = l;
      }
      my_L = __fsub_rd(l, 2.f * dlt[i]);
      my_skip = FULL && my_L >= 0.f && sc[my_a] <= my_L;
    }
    unsigned few = 0, many = 0;
    for (int r = 0; r < rows; ++r) {
      const int64_t i = i0 + r;
      const RowGeom rg = row_geom<BATCH>(i, k, kst, cap, row_run, runs);
      const int32_t kr = rg.k;
      const int32_t ai = __shfl_sync(SKM_FULL_MASK, my_a, r) - rg.koff;  // local
      const float L = __shfl_sync(SKM_FULL_MASK, my_L, r);
      const bool skip_pt = __shfl_sync(SKM_FULL_MASK, (int)my_skip, r) != 0;
      float* urow = ub + rg.ubase;
      const float* ccrow = cc + rg.ccoff + (int64_t)ai * rg.kst;
      const float* pdr = pdn + rg.koff;
      const float* pur = pup + rg.koff;
      const float* qr = qup + rg.koff;
      int mine = 0;
      for (int j4 = lane * 4; j4 < kr; j4 += 128) {
        float4 u4 = *reinterpret_cast<const float4*>(urow + j4);
        if (moved) {
          const float4 pd = *reinterpret_cast<const float4*>(pdr + j4);
          const float4 pu = *reinterpret_cast<const float4*>(pur + j4);
          const float4 q = *reinterpret_cast<const float4*>(qr + j4);
          u4.x = bound_u(u4.x, pd.x, pu.x, q.x);
          u4.y = bound_u(u4.y, pd.y, pu.y, q.y);
          u4.z = bound_u(u4.z, pd.z, pu.z, q.z);
          u4.w = bound_u(u4.w, pd.w, pu.w, q.w);
          *reinterpret_cast<float4*>(urow + j4) = u4;
        }
        if (!skip_pt) {
          mine += (j4 + 0 < kr) && elk_cand<FULL>(j4 + 0, ai, u4.x, L, ccrow);
          mine += (j4 + 1 < kr) && elk_cand<FULL>(j4 + 1, ai, u4.y, L, ccrow);
          mine += (j4 + 2 < kr) && elk_cand<FULL>(j4 + 2, ai, u4.z, L, ccrow);
          mine += (j4 + 3 < kr) && elk_cand<FULL>(j4 + 3, ai, u4.w, L, ccrow);
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(SKM_FULL_MASK, mine, o);
      if (mine > rg.cap) many |= 1u << r;
      else if (mine > 0) few |= 1u << r;
    }
    const bool is_few = (few >> lane) & 1u;
    warp_push(is_few && !my_long, (int32_t)(i0 + lane), w1, cnt + C_W1);
    warp_push_down(is_few && my_long, (int32_t)(i0 + lane), w1 + (n - 1), cnt + C_W1L);
    warp_push((many >> lane) & 1u, (int32_t)(i0 + lane), w2, cnt + C_W2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(reinterpret_cast<unsigned*>(hst + 2), 1u);
    if (done == gridDim.x - 1) {  // the last block: every push is counted
      __threadfence();
      if (!skip_b) {
        const unsigned long long whole = *reinterpret_cast<volatile unsigned long long*>(cnt + C_W2);
        hst[0] = (n >= 4096 && (double)whole >= 0.98 * (double)n) ? 1 : 0;
        hst[1] = 0;
      } else if (++hst[1] >= kElkProbe - 1) {
        hst[0] = 0;
      }
      hst[2] = 0;
    }
  }
}

// Canonical similarity to one center per lane of an 8-lane group (my_j < 0:
// the lane computes nothing useful).  The group walks the row 16 entries at a
// time: each lane loads two entries, the group broadcasts them by width-8
// shuffles, every lane gathers its 16 center values, then accumulates them in
// CSR order.  The next chunk's entries are loaded ahead.
template <typename VT>
__device__ __forceinline__ float group8_dot(int64_t b, int64_t e, const int32_t* __restrict__ col,
                                            const VT* __restrict__ val, const float* __restrict__ Ct, int64_t kst,
                                            int my_j, unsigned gmask, int gl, uint32_t* __restrict__ gt,
                                            float* __restrict__ gv) {
  const bool on = my_j >= 0;
  const float* cbase = Ct + (on ? my_j : 0);
  // an entry's term t as the 32-bit offset t kst (d kst < 2^32, checked at
  // init), computed by the lane that loads the entry
  const uint32_t ku = (uint32_t)kst;
  float acc = 0.f;
  uint32_t t0 = 0, t1 = 0;
  float v0 = 0.f, v1 = 0.f;
  if (b + gl < e) {
    t0 = (uint32_t)__ldg(col + b + gl) * ku;
    v0 = to_f32(val[b + gl]);
  }
  if (b + 8 + gl < e) {
    t1 = (uint32_t)__ldg(col + b + 8 + gl) * ku;
    v1 = to_f32(val[b + 8 + gl]);
  }
  int64_t p0 = b;
  // full batches of 16 entries, without per-entry tests
  for (; p0 + 16 <= e; p0 += 16) {
    const uint32_t ct0 = t0, ct1 = t1;
    const float cv0 = v0, cv1 = v1;
    if (p0 + 16 + gl < e) {
      t0 = (uint32_t)__ldg(col + p0 + 16 + gl) * ku;
      v0 = to_f32(val[p0 + 16 + gl]);
    }
    if (p0 + 24 + gl < e) {
      t1 = (uint32_t)__ldg(col + p0 + 24 + gl) * ku;
      v1 = to_f32(val[p0 + 24 + gl]);
    }
    // the batch's 16 entries through the group's shared buffer (broadcast
    // vector reads cost less of the load/store path than 32 shuffles)
    __syncwarp(gmask);
    gt[gl] = ct0;
    gt[8 + gl] = ct1;
    gv[gl] = cv0;
    gv[8 + gl] = cv1;
    __syncwarp(gmask);
    float c[16];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint4 t4 = *reinterpret_cast<const uint4*>(gt + 4 * x);
      c[4 * x] = on ? __ldg(cbase + t4.x) : 0.f;
      c[4 * x + 1] = on ? __ldg(cbase + t4.y) : 0.f;
      c[4 * x + 2] = on ? __ldg(cbase + t4.z) : 0.f;
      c[4 * x + 3] = on ? __ldg(cbase + t4.w) : 0.f;
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float4 v4 = *reinterpret_cast<const float4*>(gv + 4 * x);
      acc = __fmaf_rn(v4.x, c[4 * x], acc);
      acc = __fmaf_rn(v4.y, c[4 * x + 1], acc);
      acc = __fmaf_rn(v4.z, c[4 * x + 2], acc);
      acc = __fmaf_rn(v4.w, c[4 * x + 3], acc);
    }
  }
  // the ragged tail: one more batch whose missing entries load and add nothing
  if (p0 < e) {
    const int nq = (int)(e - p0);
    __syncwarp(gmask);
    gt[gl] = t0;  // past the row's end: an earlier entry's offset (or 0), never used
    gt[8 + gl] = t1;
    gv[gl] = v0;
    gv[8 + gl] = v1;
    __syncwarp(gmask);
    float c[16];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint4 t4 = *reinterpret_cast<const uint4*>(gt + 4 * x);
      c[4 * x] = (on && 4 * x < nq) ? __ldg(cbase + t4.x) : 0.f;
      c[4 * x + 1] = (on && 4 * x + 1 < nq) ? __ldg(cbase + t4.y) : 0.f;
      c[4 * x + 2] = (on && 4 * x + 2 < nq) ? __ldg(cbase + t4.z) : 0.f;
      c[4 * x + 3] = (on && 4 * x + 3 < nq) ? __ldg(cbase + t4.w) : 0.f;
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float4 v4 = *reinterpret_cast<const float4*>(gv + 4 * x);
      if (4 * x < nq) acc = __fmaf_rn(v4.x, c[4 * x], acc);
      if (4 * x + 1 < nq) acc = __fmaf_rn(v4.y, c[4 * x + 1], acc);
      if (4 * x + 2 < nq) acc = __fmaf_rn(v4.z, c[4 * x + 2], acc);
      if (4 * x + 3 < nq) acc = __fmaf_rn(v4.w, c[4 * x + 3], acc);
    }
  }
  return acc;
}

// The candidates of an Elkan survivor, for an 8-lane group (lane gl): a(i)
// itself in slot 0, then every j != a with u(i,j) > L and, for full Elkan,
// cc(a,j) > L (Section 5.2), in ascending center order (lane gl scans 4
// consecutive centers per step of 32).  Returns their number minus one.
template <bool FULL>
__device__ __forceinline__ int elk_candidates(const float* __restrict__ urow, const float* __restrict__ ccrow,
                                              int32_t ai, float L, int32_t kr, unsigned gmask, int gl, int* sj) {
  __syncwarp(gmask);
  if (gl == 0) sj[0] = ai;
  int m = 0;
  for (int j0 = 0; j0 < kr; j0 += 32) {
    const int jb = j0 + gl * 4;
    unsigned bits = 0;
    if (jb < kr) {
      const float4 u4 = *reinterpret_cast<const float4*>(urow + jb);
      bits |= ((jb + 0 < kr) && elk_cand<FULL>(jb + 0, ai, u4.x, L, ccrow)) ? 1u : 0u;
      bits |= ((jb + 1 < kr) && elk_cand<FULL>(jb + 1, ai, u4.y, L, ccrow)) ? 2u : 0u;
      bits |= ((jb + 2 < kr) && elk_cand<FULL>(jb + 2, ai, u4.z, L, ccrow)) ? 4u : 0u;
      bits |= ((jb + 3 < kr) && elk_cand<FULL>(jb + 3, ai, u4.w, L, ccrow)) ? 8u : 0u;
    }
    const int nb = __popc(bits);
    int incl = nb;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int y = __shfl_up_sync(gmask, incl, o, 8);
      if (gl >= o) incl += y;
    }
    int pos = m + 1 + (incl - nb);
    for (int c = 0; c < 4; ++c)
      if (bits & (1u << c)) {
        if (pos < 8) sj[pos] = jb + c;  // ascending center order
        ++pos;
      }
    m += __shfl_sync(gmask, incl, 7, 8);
  }
  __syncwarp(gmask);
  return m;
}

// The decision for an Elkan survivor from its candidates' canonical
// similarities (lane gl holds candidate sj[gl]; lane 0 is a(i)): the best
// candidate replaces a(i) only on a strict improvement, and among equal maxima
// the lowest index wins -- the standard variant's rule, because every center
// left out satisfies sim <= sim(a) (bounds with the 2 delta margin).  Writes
// the exact u(i,j) of the candidates, l(i), and the label.
__device__ __forceinline__ void elk_decide(int32_t i, int32_t koff, int32_t ai, int m, int my_j, float sim, float dl,
                                           float* __restrict__ urow, int32_t* __restrict__ a,
                                           float* __restrict__ lb, int32_t* __restrict__ chg_i,
                                           int32_t* __restrict__ chg_old, unsigned long long* __restrict__ cnt,
                                           unsigned gmask, int gl, unsigned long long& sims,
                                           unsigned long long& changed) {
  const float sa = __shfl_sync(gmask, sim, 0, 8);
  float bv = (gl >= 1 && gl <= m) ? sim : -INFINITY;
  int bj = (gl >= 1 && gl <= m) ? my_j : INT_MAX;
#pragma unroll
  for (int o = 4; o; o >>= 1) {
    const float ov = __shfl_xor_sync(gmask, bv, o, 8);
    const int oj = __shfl_xor_sync(gmask, bj, o, 8);
    if (ov > bv || (ov == bv && oj < bj)) {
      bv = ov;
      bj = oj;
    }
  }
  if (gl >= 1 && gl <= m) urow[my_j] = __fadd_ru(sim, dl);
  if (gl == 0) {
    if (m > 0 && bv > sa) {
      a[i] = koff + bj;
      lb[i] = __fsub_rd(bv, dl);
      urow[ai] = __fadd_ru(sa, dl);
      ++changed;
      const unsigned long long pos = atomicAdd(cnt + C_CHG, 1ull);
      chg_i[pos] = i;
      chg_old[pos] = koff + ai;
    } else {
      lb[i] = __fsub_rd(sa, dl);
    }
    sims += (unsigned long long)(m + 1);
  }
}

// Elkan survivors, an 8-lane group per point (four points per warp).  The
// surviving (point, center) pairs of the point are compacted into the group's
// lanes (elk_candidates); one pass over the row computes all their canonical
// similarities.  This makes l(i) tight (<x, c_a>, Section 5.1) and gives the
// exact u(i,j) of every candidate (elk_decide).  The bound kernel only sends
// points with 1..7 candidates and rows of at most kLongRow entries here.
template <typename VT, bool FULL, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_elk_recompute(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int32_t k,
    int64_t kst, const int32_t* __restrict__ row_run, const RunDesc* __restrict__ runs,
    const int32_t* __restrict__ w1, const unsigned long long* __restrict__ w1_cnt,
    int32_t* __restrict__ a, float* __restrict__ lb, float* __restrict__ ub, const float* __restrict__ cc,
    int32_t* __restrict__ w2, int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
    unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ cursor,
    unsigned long long* __restrict__ w2_cnt) {
  const int lane = threadIdx.x & 31, gid = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xFFu << (8 * gid);
  const int64_t total = (int64_t)(*w1_cnt);
  __shared__ int slot_j[kBlock / 8][8];  // per group: center of each compacted lane
  __shared__ __align__(16) uint32_t ent_t[kBlock / 8][16];  // per group: a batch of row entries
  __shared__ __align__(16) float ent_v[kBlock / 8][16];
  int* sj = slot_j[threadIdx.x >> 3];
  unsigned long long sims = 0, changed = 0;
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) >> 3;
  unsigned long long nxt;
  for (int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3; slot < total;
       slot = grab_take(nxt, gmask, 8)) {
    nxt = grab_issue(cursor, gl == 0, ngroups, total);
    const int32_t i = w1[slot];
    const RowGeom rg = row_geom<BATCH>(i, k, kst, 0, row_run, runs);
    const int32_t ai = a[i] - rg.koff;  // local center ids from here on
    const float dl = dlt[i];
    const float L = __fsub_rd(lb[i], 2.f * dl);
    float* urow = ub + rg.ubase;
    const int m = elk_candidates<FULL>(urow, cc + rg.ccoff + (int64_t)ai * rg.kst, ai, L, rg.k, gmask, gl, sj);
    if (m > 7) {  // not expected (the bound kernel routes such points), handled anyway
      if (gl == 0) {
        const unsigned long long pos = atomicAdd(w2_cnt, 1ull);
        w2[pos] = i;
      }
      continue;
    }
    const int my_j = (gl <= m) ? sj[gl] : -1;
    const float sim = __fmul_rn(
        group8_dot<VT>(rp[i], rp[i + 1], col, val, Ct, kst, my_j >= 0 ? rg.koff + my_j : -1, gmask, gl,
                       ent_t[threadIdx.x >> 3], ent_v[threadIdx.x >> 3]),
        rinv[i]);
    elk_decide(i, rg.koff, ai, m, my_j, sim, dl, urow, a, lb, chg_i, chg_old, cnt, gmask, gl, sims, changed);
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
    changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
  }
  if (lane == 0) {
    if (sims) atomicAdd(cnt + C_SIMS, sims);
    if (changed) atomicAdd(cnt + C_CHANGED, changed);
  }
}

// The same for survivors with long rows (more than kLongRow entries), a warp
// per point: lanes 0-7 find the candidates and decide as above.  The dot
// walks the row 64 entries at a time: every lane takes two entries of a chunk
// and gathers the center values of all candidates for them into the warp's
// half of a double buffer in shared memory; the gathers of the next chunk are
// in flight while the candidate lanes run their FMA chains over this one in
// CSR order (the chain of group8_dot, so the similarities are bit-identical).
constexpr int kLongChunk = 64;

template <typename VT, bool FULL, bool BATCH>
__global__ void __launch_bounds__(kBlock) k_elk_recompute_long(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ val,
    const float* __restrict__ rinv, const float* __restrict__ dlt, const float* __restrict__ Ct, int32_t k,
    int64_t kst, const int32_t* __restrict__ row_run, const RunDesc* __restrict__ runs,
    const int32_t* __restrict__ w1_top, const unsigned long long* __restrict__ w1_cnt,
    int32_t* __restrict__ a, float* __restrict__ lb, float* __restrict__ ub, const float* __restrict__ cc,
    int32_t* __restrict__ w2, int32_t* __restrict__ chg_i, int32_t* __restrict__ chg_old,
    unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ cursor,
    unsigned long long* __restrict__ w2_cnt) {
  constexpr int NW = kBlock / 32, CH = kLongChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t total = (int64_t)(*w1_cnt);
  __shared__ int slot_j[NW][8];
  // [buffer][candidate][entry of the chunk]: a candidate lane reads four
  // consecutive entries with one 16-byte load (rows padded to 68 floats, so
  // that the eight candidate lanes hit different banks)
  __shared__ __align__(16) float tile[NW][2][8][CH + 4];
  __shared__ __align__(16) float tvl[NW][2][CH];  // the chunk's values
  int* sj = slot_j[warp];
  unsigned long long sims = 0, changed = 0;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nxt;
  for (int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total;
       slot = grab_take(nxt, SKM_FULL_MASK, 32)) {
    nxt = grab_issue(cursor, lane == 0, nwarps, total);
    const int32_t i = w1_top[-slot];
    const RowGeom rg = row_geom<BATCH>(i, k, kst, 0, row_run, runs);
    const int32_t ai = a[i] - rg.koff;
    const float dl = dlt[i];
    const float L = __fsub_rd(lb[i], 2.f * dl);
    float* urow = ub + rg.ubase;
    int m = 0;
    if (lane < 8) m = elk_candidates<FULL>(urow, cc + rg.ccoff + (int64_t)ai * rg.kst, ai, L, rg.k, 0xFFu, lane, sj);
    m = __shfl_sync(SKM_FULL_MASK, m, 0);
    __syncwarp();
    if (m > 7) {
      if (lane == 0) {
        const unsigned long long pos = atomicAdd(w2_cnt, 1ull);
        w2[pos] = i;
      }
      continue;
    }
    const int64_t b = rp[i], e = rp[i + 1];
    const float* cb = Ct + rg.koff;
    int jq[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) jq[q] = q <= m ? sj[q] : 0;
    // entries p0 + lane and p0 + 32 + lane of chunk p0: columns, values, gathers
    // an entry's term t as the 32-bit offset t kst (d kst < 2^32, checked at init)
    const uint32_t ku = (uint32_t)kst;
    uint32_t t0 = b + lane < e ? (uint32_t)__ldg(col + b + lane) * ku : 0u;
    uint32_t t1 = b + 32 + lane < e ? (uint32_t)__ldg(col + b + 32 + lane) * ku : 0u;
    float x0 = b + lane < e ? to_f32(val[b + lane]) : 0.f;
    float x1 = b + 32 + lane < e ? to_f32(val[b + 32 + lane]) : 0.f;
    float g0[8], g1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      g0[q] = (b + lane < e && q <= m) ? __ldg(cb + t0 + jq[q]) : 0.f;
      g1[q] = (b + 32 + lane < e && q <= m) ? __ldg(cb + t1 + jq[q]) : 0.f;
    }
    float acc = 0.f;
    int buf = 0;
    for (int64_t p0 = b; p0 < e; p0 += CH, buf ^= 1) {
      // this chunk into the buffer (the previous reader of this half finished
      // before the __syncwarp of the last chunk)
      tvl[warp][buf][lane] = x0;
      tvl[warp][buf][32 + lane] = x1;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        tile[warp][buf][q][lane] = g0[q];
        tile[warp][buf][q][32 + lane] = g1[q];
      }
      __syncwarp();
      // the next chunk's gathers go out before this chunk's FMA chains
      const int64_t pn = p0 + CH;
      const bool in0 = pn + lane < e, in1 = pn + 32 + lane < e;
      t0 = in0 ? (uint32_t)__ldg(col + pn + lane) * ku : 0u;
      t1 = in1 ? (uint32_t)__ldg(col + pn + 32 + lane) * ku : 0u;
      x0 = in0 ? to_f32(val[pn + lane]) : 0.f;
      x1 = in1 ? to_f32(val[pn + 32 + lane]) : 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        g0[q] = (in0 && q <= m) ? __ldg(cb + t0 + jq[q]) : 0.f;
        g1[q] = (in1 && q <= m) ? __ldg(cb + t1 + jq[q]) : 0.f;
      }
      if (lane <= m) {
        const float* tv = tvl[warp][buf];
        const float* tl = tile[warp][buf][lane];
        if (e - p0 >= CH) {
#pragma unroll 4
          for (int q = 0; q < CH; q += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(tv + q);
            const float4 cv = *reinterpret_cast<const float4*>(tl + q);
            acc = __fmaf_rn(xv.x, cv.x, acc);
            acc = __fmaf_rn(xv.y, cv.y, acc);
            acc = __fmaf_rn(xv.z, cv.z, acc);
            acc = __fmaf_rn(xv.w, cv.w, acc);
          }
        } else {
          const int nq = (int)(e - p0);
          for (int q = 0; q < nq; ++q) acc = __fmaf_rn(tv[q], tl[q], acc);
        }
      }
      __syncwarp();
    }
    if (lane < 8) {
      const int my_j = (lane <= m) ? sj[lane] : -1;
      const float sim = __fmul_rn(acc, rinv[i]);
      elk_decide(i, rg.koff, ai, m, my_j, sim, dl, urow, a, lb, chg_i, chg_old, cnt, 0xFFu, lane, sims, changed);
    }
    __syncwarp();
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    sims += __shfl_xor_sync(SKM_FULL_MASK, sims, o);
    changed += __shfl_xor_sync(SKM_FULL_MASK, changed, o);
  }
  if (lane == 0) {
    if (sims) atomicAdd(cnt + C_SIMS, sims);
    if (changed) atomicAdd(cnt + C_CHANGED, changed);
  }
}

// Blocks of a kernel (kBlock threads, static shared memory) resident on one
// SM, from the occupancy calculator; cached per kernel.
int fit_blocks(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kBlock, 0) != cudaSuccess || nb < 1) {
    (void)cudaGetLastError();
    nb = 1;
  }
  cache.emplace(kernel, nb);
  return nb;
}

// Persistent kernels: as many blocks as are resident at once (at most the
// blocks per SM of the options, which skm_autotune sets), so that no block
// waits for a second wave.
inline int persistent_grid(const skm_ctx* c, const void* kernel) {
  int per_sm = fit_blocks(kernel);
  if (c->opt.blocks_per_sm > 0 && c->opt.blocks_per_sm < per_sm) per_sm = c->opt.blocks_per_sm;
  return c->nsm * per_sm;
}


// One whole-row launch.  mode 0-3 as k_rows_top2 (FP32 centers); modes 4, 5:
// the screened Elkan / Hamerly passes (FP16 centers, single runs, one pass
// over k).
// cursor: the work cursor of this launch (each launch of an assignment has
// its own).
template <typename VT, int G, bool BATCH>
int launch_rows_b(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows,
                  int cursor) {
  const void* kern = mode == 0   ? (const void*)k_rows_top2<VT, float, G, 0, BATCH>
                     : mode == 1 ? (const void*)k_rows_top2<VT, float, G, 1, BATCH>
                     : mode == 2 ? (const void*)k_rows_top2<VT, float, G, 2, BATCH>
                     : mode == 3 ? (const void*)k_rows_top2<VT, float, G, 3, BATCH>
                     : mode == 4 ? (const void*)k_rows_top2<VT, __half, G, 4, BATCH>
                                 : (const void*)k_rows_top2<VT, __half, G, 5, BATCH>;
  int64_t g = persistent_grid(c, kern);
  if (!list && g > (nrows * 32 + kBlock - 1) / kBlock) g = (nrows * 32 + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  const VT* v = (const VT*)c->val;
  SKM_PROF_BEGIN(c, mode >= 4 ? "k_rows_top2(screen)" : list ? "k_rows_top2(list)" : "k_rows_top2");
#define SKM_ROWS(CT, CP, M)                                                                                        \
  k_rows_top2<VT, CT, G, M, BATCH><<<(unsigned)g, kBlock, 0, c->st>>>(                                            \
      c->rp, c->col, v, c->rinv, c->dlt, CP, c->k, c->kst, c->row_run, c->runs, list, list_cnt, nrows, c->n, c->a, \
      c->lb, c->ub, c->chg_i, c->chg_old, c->cnt, c->cnt + cursor, c->escr, c->w3, c->w4)
  switch (mode) {
    case 0: SKM_ROWS(float, c->Ct, 0); break;
    case 1: SKM_ROWS(float, c->Ct, 1); break;
    case 2: SKM_ROWS(float, c->Ct, 2); break;
    case 3: SKM_ROWS(float, c->Ct, 3); break;
    case 4: SKM_ROWS(__half, c->Ct16, 4); break;
    default: SKM_ROWS(__half, c->Ct16, 5);
  }
#undef SKM_ROWS
  SKM_LAUNCHED(c);
  return SKM_OK;
}

// Yin-Yang in a batch: the whole-row kernel with four groups of 128 centers,
// one pass over every run's row (runs of at most 512 centers).
template <typename VT>
int launch_rows_yy_batch(skm_ctx* c, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows,
                         int cursor) {
  const void* kern = (const void*)k_rows_top2<VT, float, 4, 3, true>;
  int64_t g = persistent_grid(c, kern);
  if (!list && g > (nrows * 32 + kBlock - 1) / kBlock) g = (nrows * 32 + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  SKM_PROF_BEGIN(c, list ? "k_rows_top2(list)" : "k_rows_top2");
  k_rows_top2<VT, float, 4, 3, true><<<(unsigned)g, kBlock, 0, c->st>>>(
      c->rp, c->col, (const VT*)c->val, c->rinv, c->dlt, c->Ct, c->k, c->kst, c->row_run, c->runs, list, list_cnt,
      nrows, c->n, c->a, c->lb, c->ub, c->chg_i, c->chg_old, c->cnt, c->cnt + cursor, c->escr, c->w3, c->w4);
  SKM_LAUNCHED(c);
  return SKM_OK;
}

template <typename VT, int G>
int launch_rows(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows,
                int cursor) {
  return launch_rows_b<VT, G, false>(c, mode, list, list_cnt, nrows, cursor);
}

template <typename VT>
int assign_full_t(skm_ctx* c, int mode, const int32_t* list, const unsigned long long* list_cnt, int64_t nrows,
                  int cursor = C_CURSOR) {
  const int k = c->k;
  // a batch walks each row's own slice 128 centers at a time
  // (Yin-Yang in a batch: every run has at most 512 centers, walked in one
  // pass, which its group bounds need)
  if (c->nruns > 0 && mode == 3) return launch_rows_yy_batch<VT>(c, list, list_cnt, nrows, cursor);
  if (c->nruns > 0) return launch_rows_b<VT, 1, true>(c, mode, list, list_cnt, nrows, cursor);
  // centers per pass over a row: the chosen tile, else the smallest that holds k
  const int kt = c->opt.k_tile > 0 ? c->opt.k_tile : k <= 128 ? 128 : k <= 256 ? 256 : k <= 512 ? 512 : 1024;
  if (kt == 128) return launch_rows<VT, 1>(c, mode, list, list_cnt, nrows, cursor);
  if (kt == 256) return launch_rows<VT, 2>(c, mode, list, list_cnt, nrows, cursor);
  if (kt == 512) return launch_rows<VT, 4>(c, mode, list, list_cnt, nrows, cursor);
  return launch_rows<VT, 8>(c, mode, list, list_cnt, nrows, cursor);
}

// Hamerly's bound pass (k_ham_bounds for the context's variant and form).
int ham_bounds_launch(skm_ctx* c) {
  const bool full = (c->variant == SKM_HAMERLY), batch = c->nruns > 0;
#define SKM_HAMB(F, B)                                                                                            \
  k_ham_bounds<F, B><<<persistent_grid(c, (const void*)k_ham_bounds<F, B>), kBlock, 0, c->st>>>(                  \
      c->n, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup, c->qup, c->hsel, c->sc, c->row_run, c->opt.hamerly_tight, \
      c->moved, c->hst, c->w1, c->w2, c->cnt)
  SKM_PROF_BEGIN(c, "k_ham_bounds");
  if (full && batch) SKM_HAMB(true, true);
  else if (full) SKM_HAMB(true, false);
  else if (batch) SKM_HAMB(false, true);
  else SKM_HAMB(false, false);
#undef SKM_HAMB
  SKM_LAUNCHED(c);
  return SKM_OK;
}

template <typename VT>
int hamerly_step_t(skm_ctx* c) {
  const bool full = (c->variant == SKM_HAMERLY);
  const int rc = ham_bounds_launch(c);
  if (rc) return rc;
  const int g = persistent_grid(c, full ? (const void*)k_ham_tighten<VT, true> : (const void*)k_ham_tighten<VT, false>);
  const VT* v = (const VT*)c->val;
  const float thr = (c->nruns > 0 ? c->kmax : c->k) <= 128 ? 0.4f : 0.15f;
  SKM_PROF_BEGIN(c, "k_ham_tighten");
  if (full) {
    k_ham_tighten<VT, true><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1,
                                                     c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w2, c->cnt,
                                                     c->hst, thr);
  } else {
    k_ham_tighten<VT, false><<<g, kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->kst, c->w1,
                                                      c->cnt + C_W1, c->a, c->lb, c->ub, c->sc, c->w2, c->cnt,
                                                      c->hst, thr);
  }
  SKM_LAUNCHED(c);
  if (!c->Ct16 || c->scr_off || c->nruns > 0) return assign_full_t<VT>(c, 1, c->w2, c->cnt + C_W2, 0);
  // screened whole rows (FP16 centers), then FP32 whole rows for the rows the bound left open
  TRY_K(assign_full_t<VT>(c, 5, c->w2, c->cnt + C_W2, 0));
  return assign_full_t<VT>(c, 1, c->w4, c->cnt + C_W4, 0, C_CURSOR_2);
}

template <typename VT>
int elkan_step_t(skm_ctx* c) {
  const bool full = (c->variant == SKM_ELKAN);
  const bool batch = c->nruns > 0;
  // a point with more than min(k/8, 7) candidate centers is recomputed as a
  // whole row (the per-pair path gives each point an 8-lane group)
  int32_t row_thresh = c->opt.row_threshold > 0 ? c->opt.row_threshold : (c->k + 7) / 8;
  if (row_thresh > 7) row_thresh = 7;
  SKM_PROF_BEGIN(c, "k_elk_bounds");
#define SKM_ELKB(F, B)                                                                                            \
  k_elk_bounds<F, B><<<persistent_grid(c, (const void*)k_elk_bounds<F, B>), kBlock, 0, c->st>>>(c->n, c->k, c->kst, c->rp, c->row_run, c->runs, c->a, c->lb, c->ub, \
                                              c->dlt,                                                              \
                                              c->pdn, c->pup, c->qup, c->cc, c->sc, c->moved, row_thresh, c->w1,   \
                                              c->w2, c->cnt, c->hst)
  if (batch && full) SKM_ELKB(true, true);
  else if (batch) SKM_ELKB(false, true);
  else if (full) SKM_ELKB(true, false);
  else SKM_ELKB(false, false);
#undef SKM_ELKB
  SKM_LAUNCHED(c);
  const VT* v = (const VT*)c->val;
  SKM_PROF_BEGIN(c, "k_elk_recompute");
#define SKM_ELKR(F, B)                                                                                           \
  k_elk_recompute<VT, F, B><<<persistent_grid(c, (const void*)k_elk_recompute<VT, F, B>), kBlock, 0, c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst,     \
                                                     c->row_run, c->runs, c->w1, c->cnt + C_W1, c->a, c->lb, c->ub, \
                                                     c->cc, c->w2, c->chg_i, c->chg_old, c->cnt,               \
                                                     c->cnt + C_CURSOR_R, c->cnt + C_W2)
  if (batch && full) SKM_ELKR(true, true);
  else if (batch) SKM_ELKR(false, true);
  else if (full) SKM_ELKR(true, false);
  else SKM_ELKR(false, false);
#undef SKM_ELKR
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_elk_recompute_long");
#define SKM_ELKL(F, B)                                                                                         \
  k_elk_recompute_long<VT, F, B><<<persistent_grid(c, (const void*)k_elk_recompute_long<VT, F, B>), kBlock, 0, \
                                   c->st>>>(                                                                   \
      c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst, c->row_run, c->runs, c->w1 + (c->n - 1),         \
      c->cnt + C_W1L, c->a, c->lb, c->ub, c->cc, c->w2, c->chg_i, c->chg_old, c->cnt, c->cnt + C_CURSOR_L,    \
      c->cnt + C_W2)
  if (batch && full) SKM_ELKL(true, true);
  else if (batch) SKM_ELKL(false, true);
  else if (full) SKM_ELKL(true, false);
  else SKM_ELKL(false, false);
#undef SKM_ELKL
  SKM_LAUNCHED(c);
  if (!c->Ct16 || c->scr_off || batch) return assign_full_t<VT>(c, 2, c->w2, c->cnt + C_W2, 0);
  // screened whole rows (FP16 centers), then the exact pass for the rows the
  // bound left open: pairs (w3, short rows from the bottom, long ones from
  // the top) and FP32 whole rows (w4)
  TRY_K(assign_full_t<VT>(c, 4, c->w2, c->cnt + C_W2, 0));
  SKM_PROF_BEGIN(c, "k_elk_recompute(screen)");
#define SKM_ELKR2(F)                                                                                           \
  k_elk_recompute<VT, F, false><<<persistent_grid(c, (const void*)k_elk_recompute<VT, F, false>), kBlock, 0,  \
                                  c->st>>>(c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst, c->row_run, \
                                           c->runs, c->w3, c->cnt + C_W3S, c->a, c->lb, c->ub, c->cc, c->w4,   \
                                           c->chg_i, c->chg_old, c->cnt, c->cnt + C_CURSOR_R2, c->cnt + C_W4)
  if (full) SKM_ELKR2(true);
  else SKM_ELKR2(false);
#undef SKM_ELKR2
  SKM_LAUNCHED(c);
  SKM_PROF_BEGIN(c, "k_elk_recompute_long(screen)");
#define SKM_ELKL2(F)                                                                                             \
  k_elk_recompute_long<VT, F, false><<<persistent_grid(c, (const void*)k_elk_recompute_long<VT, F, false>),     \
                                       kBlock, 0, c->st>>>(                                                      \
      c->rp, c->col, v, c->rinv, c->dlt, c->Ct, c->k, c->kst, c->row_run, c->runs, c->w3 + (c->n - 1),           \
      c->cnt + C_W3L, c->a, c->lb, c->ub, c->cc, c->w4, c->chg_i, c->chg_old, c->cnt, c->cnt + C_CURSOR_L2,      \
      c->cnt + C_W4)
  if (full) SKM_ELKL2(true);
  else SKM_ELKL2(false);
#undef SKM_ELKL2
  SKM_LAUNCHED(c);
  return assign_full_t<VT>(c, 2, c->w4, c->cnt + C_W4, 0, C_CURSOR_2);
}

template <typename VT>
int yinyang_step_t(skm_ctx* c) {
  const bool batch = c->nruns > 0;
  const int g = persistent_grid(c, batch ? (const void*)k_yy_bounds<true> : (const void*)k_yy_bounds<false>);
  const int32_t ng = (c->k + 7) / 8;  // a batch: every run's slice, each a whole number of groups
  if (c->moved) {
    SKM_PROF_BEGIN(c, "k_yy_drift");
    k_yy_drift<<<(ng + 127) / 128, 128, 0, c->st>>>(c->k, ng, c->pdn, c->pup, c->qup, c->gdrift);
    SKM_LAUNCHED(c);
  }
  SKM_PROF_BEGIN(c, "k_yy_bounds");
  if (batch)
    k_yy_bounds<true><<<g, kBlock, 0, c->st>>>(c->n, ng, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup, c->qup,
                                               c->gdrift, c->moved, c->row_run, c->runs, c->w1, c->cnt);
  else
    k_yy_bounds<false><<<g, kBlock, 0, c->st>>>(c->n, ng, c->a, c->lb, c->ub, c->dlt, c->pdn, c->pup, c->qup,
                                                c->gdrift, c->moved, nullptr, nullptr, c->w1, c->cnt);
  SKM_LAUNCHED(c);
  // the survivors go straight to the group pass: its group test uses the
  // moved (not tightened) l, and a(i)'s own group is always recomputed
  return assign_full_t<VT>(c, 3, c->w1, c->cnt + C_W1, 0);
}

}  // namespace

int hamerly_bounds_only(skm_ctx* c) { return ham_bounds_launch(c); }

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

namespace skm {

int yinyang_step(skm_ctx* c) {
  switch (c->dtype) {
    case SKM_F32: return yinyang_step_t<float>(c);
    case SKM_F16: return yinyang_step_t<__half>(c);
    case SKM_BF16: return yinyang_step_t<__nv_bfloat16>(c);
  }
  return SKM_EINVAL;
}

}  // namespace skm
