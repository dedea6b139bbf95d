// The C ABI of libskm (declared in include/skm.h): argument checks, device
// memory of a context, and the order of the kernels of one Lloyd iteration.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_set>
#include <vector>

#include "skm_internal.cuh"

namespace skm {

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t reduction_blocks(int64_t d);

struct ProfRec {
  const char* name;
  cudaEvent_t b, e;
};
using ProfList = std::vector<ProfRec>;

void prof_begin(skm_ctx* c, const char* name) {
  if (!c->prof_on) return;
  ProfRec r{name, nullptr, nullptr};
  if (cudaEventCreate(&r.b) != cudaSuccess || cudaEventCreate(&r.e) != cudaSuccess) {
    (void)cudaGetLastError();
    return;
  }
  cudaEventRecord(r.b, c->st);
  static_cast<ProfList*>(c->prof)->push_back(r);
}

void prof_end(skm_ctx* c) {
  if (!c->prof_on) return;
  ProfList* L = static_cast<ProfList*>(c->prof);
  if (!L->empty()) cudaEventRecord(L->back().e, c->st);
}

static void prof_clear(skm_ctx* c) {
  if (!c->prof) return;
  ProfList* L = static_cast<ProfList*>(c->prof);
  for (auto& r : *L) {
    cudaEventDestroy(r.b);
    cudaEventDestroy(r.e);
  }
  L->clear();
}

}  // namespace skm

using namespace skm;

namespace {

inline unsigned grid_cap(int64_t items, int per_block, int nsm, int per_sm = 16) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g > (int64_t)nsm * per_sm) g = (int64_t)nsm * per_sm;
  return (unsigned)(g < 1 ? 1 : g);
}

// Batch: global label -> label local to the row's run.
__global__ void k_labels_local(const int32_t* __restrict__ a, int64_t n, const int32_t* __restrict__ row_run,
                               const RunDesc* __restrict__ runs, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = a[i];
    out[i] = v < 0 ? v : v - runs[row_run[i]].koff;
  }
}

// Batch: the runs' centers one after the other as rows (out: sum_r k_r x d);
// thread per (output row, term), the run found by a walk over the table.
__global__ void k_centers_batch(const float* __restrict__ Ct, int64_t d, int64_t kst, const RunDesc* __restrict__ runs,
                                int32_t nruns, int64_t ktot, float* __restrict__ out) {
  const int64_t total = ktot * d;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = q / d, t = q - o * d;
    int64_t base = 0;
    int r = 0;
    while (r + 1 < nruns && base + runs[r].k <= o) base += runs[r++].k;
    out[q] = Ct[t * kst + runs[r].koff + (o - base)];
  }
}


template <typename T>
int dalloc(skm_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMallocAsync((void**)p, sizeof(T) * count, c->st) != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return SKM_ENOMEM;
  }
  return SKM_OK;
}

#define TRY(x)                   \
  do {                           \
    int r__ = (x);               \
    if (r__ != SKM_OK) return r__; \
  } while (0)

size_t dtype_size(int dt) { return dt == SKM_F32 ? 4 : 2; }

uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// k distinct rows from a seed (used when the caller gives no init rows).
void seeded_rows(int64_t n, int32_t k, uint64_t seed, std::vector<int64_t>& out) {
  std::unordered_set<int64_t> seen;
  out.clear();
  uint64_t ctr = 0;
  while ((int32_t)out.size() < k) {
    const int64_t r = (int64_t)(mix64(seed * 0x9E3779B97F4A7C15ull + (ctr++)) % (uint64_t)n);
    if (seen.insert(r).second) out.push_back(r);
  }
}

int start_from_rows(skm_ctx* c, const std::vector<int64_t>& rows) {
  // rows: one global row per center column (-1: a batch's padding column)
  if (!c->hinit) {
    c->hinit = new (std::nothrow) std::vector<int64_t>();
    if (!c->hinit) return SKM_ENOMEM;
  }
  *static_cast<std::vector<int64_t>*>(c->hinit) = rows;
  int64_t* drows = nullptr;
  TRY(dalloc(c, &drows, (size_t)c->k));
  SKM_CUDA_TRY(cudaMemcpyAsync(drows, rows.data(), sizeof(int64_t) * c->k, cudaMemcpyHostToDevice, c->st));
  int rc = init_centers(c, drows);
  cudaFreeAsync(drows, c->st);
  if (rc == SKM_OK) rc = ct16_all(c);
  // the host vector must outlive the copy
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (rc) return rc;
  SKM_CUDA_TRY(cudaMemsetAsync(c->a, 0xff, sizeof(int32_t) * c->n, c->st));
  SKM_CUDA_TRY(cudaMemsetAsync(c->hst, 0, sizeof(int32_t) * 4, c->st));
  c->have_bounds = 0;
  c->moved = 0;
  c->s64_valid = 0;
  c->chg_fresh = 0;
  c->cnt_clear = 0;
  std::memset(&c->stats, 0, sizeof(c->stats));
  return SKM_OK;
}

int set_init(skm_ctx* c, const int64_t* init_rows, uint64_t seed) {
  std::vector<int64_t> rows;
  if (c->nruns > 0) {
    // per run: ks[r] local rows, placed in the run's slice of the columns
    const auto& R = *static_cast<std::vector<RunDesc>*>(c->hruns);
    rows.assign((size_t)c->k, -1);
    int64_t q = 0;
    std::vector<int64_t> loc;
    for (size_t r = 0; r < R.size(); ++r) {
      if (init_rows) {
        std::unordered_set<int64_t> seen;
        loc.clear();
        for (int32_t j = 0; j < R[r].k; ++j, ++q) {
          const int64_t v = init_rows[q];
          if (v < 0 || v >= R[r].n || !seen.insert(v).second) return SKM_EINVAL;
          loc.push_back(v);
        }
      } else {
        seeded_rows(R[r].n, R[r].k, seed + r, loc);
      }
      for (int32_t j = 0; j < R[r].k; ++j) rows[(size_t)(R[r].koff + j)] = R[r].row0 + loc[(size_t)j];
    }
  } else if (init_rows) {
    std::unordered_set<int64_t> seen;
    for (int32_t j = 0; j < c->k; ++j) {
      if (init_rows[j] < 0 || init_rows[j] >= c->n || !seen.insert(init_rows[j]).second) return SKM_EINVAL;
      rows.push_back(init_rows[j]);
    }
  } else {
    seeded_rows(c->n, c->k, seed, rows);
  }
  return start_from_rows(c, rows);
}

void release(skm_ctx* c) {
  if (!c) return;
  if (c->prof) {
    skm::prof_clear(c);
    delete static_cast<ProfList*>(c->prof);
    c->prof = nullptr;
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  delete static_cast<std::vector<RunDesc>*>(c->hruns);
  delete static_cast<std::vector<int64_t>*>(c->hinit);
  void* ptrs[] = {c->gdrift, c->runs,   c->row_run, c->glog,  c->own[0], c->own[1], c->own[2], c->rinv,  c->dlt,
                  c->t_ptr,  c->t_row,   c->t_val, c->ch_term, c->ch_idx, c->ch_part, c->multi_term,
                  c->multi_base, c->multi_cnt, c->part64, c->Ct, c->S64, c->nrm, c->red, c->obj, c->pdn,
                  c->pup,    c->qup,     c->hsel,  c->cc,     c->sc,     c->gpart,  c->a,     c->lb,
                  c->ub,     c->w1,      c->w2,    c->cnt,    c->chg_i,  c->chg_old, c->dflag, c->dmark,
                  c->dpos,   c->dlist,   c->G,     c->rpart,  c->Xb,     c->Cr,     c->Cb,    c->topv,
                  c->topi,   c->w3,      c->lcount, c->loff,  c->lcursor, c->lmembers, c->cand, c->cand_n,
                  c->exr,    c->ebc,     c->ebw,   c->rsc,    c->gdbeg,  c->gdcnt,  c->gtask,  c->fbar,
                  c->Ct16,   c->e2p,     c->e2c,   c->escr,   c->w4,     c->hst,    c->n2l};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, c->st);
  cudaStreamSynchronize(c->st);
  if (c->hcnt) cudaFreeHost(c->hcnt);
  if (c->hobj) cudaFreeHost(c->hobj);
  (void)cudaGetLastError();
  delete c;
}

int read_counters(skm_ctx* c) {
  SKM_CUDA_TRY(cudaMemcpyAsync(c->hcnt, c->cnt, sizeof(unsigned long long) * C_NUM, cudaMemcpyDeviceToHost, c->st));
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->stats.last_changed = (int64_t)c->hcnt[C_CHANGED];
  c->stats.last_sims = (int64_t)c->hcnt[C_SIMS];
  c->stats.last_survivors = (int64_t)(c->hcnt[C_W1] + c->hcnt[C_W1L]);
  c->stats.last_rechecks = (int64_t)c->hcnt[C_W2];
  c->stats.last_cand_rechecks = (int64_t)c->hcnt[C_W3];
  c->stats.last_skipped = (int64_t)c->hcnt[C_SKIP];
  return SKM_OK;
}

int build_ctx(skm_ctx* c, const skm_data* x, const int64_t* init_rows, uint64_t seed) {
  SKM_CUDA_TRY(cudaGetDevice(&c->dev));
  SKM_CUDA_TRY(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev));
  const int64_t n = c->n, d = c->d;
  // ---- data
  if (x->layout == SKM_CSR) {
    int64_t nnz = 0;
    if (x->memspace == SKM_HOST) {
      nnz = x->row_ptr[n];
      if (x->row_ptr[0] != 0 || nnz < 0) return SKM_EINVAL;
    } else {
      SKM_CUDA_TRY(cudaMemcpyAsync(&nnz, x->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
      SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
      if (nnz < 0) return SKM_EINVAL;
    }
    c->nnz = nnz;
    if (x->memspace == SKM_HOST) {
      int64_t* rp = nullptr;
      int32_t* col = nullptr;
      char* val = nullptr;
      TRY(dalloc(c, &rp, (size_t)(n + 1)));
      c->own[0] = rp;
      TRY(dalloc(c, &col, (size_t)nnz));
      c->own[1] = col;
      TRY(dalloc(c, &val, (size_t)nnz * dtype_size(c->dtype)));
      c->own[2] = val;
      SKM_CUDA_TRY(cudaMemcpyAsync(rp, x->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->st));
      SKM_CUDA_TRY(cudaMemcpyAsync(col, x->col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, c->st));
      SKM_CUDA_TRY(cudaMemcpyAsync(val, x->values, nnz * dtype_size(c->dtype), cudaMemcpyHostToDevice, c->st));
      c->rp = rp;
      c->col = col;
      c->val = val;
    } else {
      c->rp = x->row_ptr;
      c->col = x->col_idx;
      c->val = x->values;
    }
  } else {
    // dense rows: n x d FP32
    c->nnz = n * d;
    if (x->memspace == SKM_HOST) {
      float* X = nullptr;
      TRY(dalloc(c, &X, (size_t)(n * d)));
      c->own[2] = X;
      SKM_CUDA_TRY(cudaMemcpyAsync(X, x->values, sizeof(float) * n * d, cudaMemcpyHostToDevice, c->st));
      c->val = X;
    } else {
      c->val = x->values;
    }
  }
  // ---- counters and per-row data
  TRY(dalloc(c, &c->cnt, C_NUM));
  SKM_CUDA_TRY(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * C_NUM, c->st));
  TRY(dalloc(c, &c->fbar, 3));
  SKM_CUDA_TRY(cudaMemsetAsync(c->fbar, 0, sizeof(unsigned long long) * 3, c->st));
  TRY(dalloc(c, &c->hst, 4));
  SKM_CUDA_TRY(cudaMemsetAsync(c->hst, 0, sizeof(int32_t) * 4, c->st));
  SKM_CUDA_TRY(cudaMallocHost((void**)&c->hcnt, sizeof(unsigned long long) * C_NUM));
  SKM_CUDA_TRY(cudaMallocHost((void**)&c->hobj, sizeof(double)));
  TRY(dalloc(c, &c->rinv, (size_t)n));
  TRY(dalloc(c, &c->dlt, (size_t)n));
  TRY(prep_rows(c));
  TRY(read_counters(c));
  if (c->hcnt[C_ERR]) return SKM_EINVAL;
  if (c->layout == SKM_CSR) TRY(prep_transpose(c));
  // ---- centers
  const int64_t kst = c->kst, k = c->k;
  TRY(dalloc(c, &c->Ct, (size_t)(d * kst)));
  TRY(dalloc(c, &c->S64, (size_t)(d * kst)));
  TRY(dalloc(c, &c->n2l, (size_t)(3 * kst)));
  SKM_CUDA_TRY(cudaMemsetAsync(c->n2l, 0, sizeof(long long) * 3 * kst, c->st));
  SKM_CUDA_TRY(cudaMemsetAsync(c->S64, 0, sizeof(long long) * d * kst, c->st));
  TRY(dalloc(c, &c->chg_i, (size_t)n));
  TRY(dalloc(c, &c->chg_old, (size_t)n));
  TRY(dalloc(c, &c->dflag, (size_t)k));
  SKM_CUDA_TRY(cudaMemsetAsync(c->dflag, 0, sizeof(int32_t) * k, c->st));
  TRY(dalloc(c, &c->dmark, (size_t)k));
  TRY(dalloc(c, &c->dpos, (size_t)k));
  TRY(dalloc(c, &c->dlist, (size_t)k));
  TRY(dalloc(c, &c->nrm, (size_t)(2 * kst)));
  c->red_blocks = reduction_blocks(d);
  TRY(dalloc(c, &c->red, (size_t)(c->red_blocks * kst * 3)));
  TRY(dalloc(c, &c->obj, 1));
  TRY(dalloc(c, &c->pdn, (size_t)kst));
  TRY(dalloc(c, &c->pup, (size_t)kst));
  TRY(dalloc(c, &c->qup, (size_t)kst));
  TRY(dalloc(c, &c->hsel, (size_t)HSEL_N * (c->nruns > 0 ? c->nruns : 1)));
  const bool full = (c->variant == SKM_ELKAN || c->variant == SKM_HAMERLY);
  const bool elk = (c->variant == SKM_ELKAN || c->variant == SKM_SIMP_ELKAN);
  const bool yy = (c->variant == SKM_YINYANG);
  const bool ham = (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY) || c->layout == SKM_DENSE || yy;
  if (full && c->nruns > 0) {
    // a batch: each run's k x kst block of cc and of the Gram (FP64), and the
    // per-run plan of the Gram tasks
    const auto& R = *static_cast<std::vector<RunDesc>*>(c->hruns);
    const int64_t blk = R.back().ccoff + (int64_t)R.back().k * R.back().kst;
    TRY(dalloc(c, &c->cc, (size_t)blk));
    TRY(dalloc(c, &c->sc, (size_t)k));
    TRY(dalloc(c, &c->G, (size_t)blk));
    TRY(dalloc(c, &c->gdbeg, (size_t)c->nruns));
    TRY(dalloc(c, &c->gdcnt, (size_t)c->nruns));
    TRY(dalloc(c, &c->gtask, (size_t)c->nruns + 1));
  } else if (full) {
    // enough d-splits of the Gram (64 x 64 tiles) for ~4 blocks per SM, each
    // split >= 256 terms
    const int64_t tk = (k + 63) / 64, tiles = tk * (tk + 1) / 2;
    int64_t sp = (4 * c->nsm + tiles - 1) / tiles;
    if (sp > 128) sp = 128;
    const int64_t spmax = (d + 255) / 256;
    if (sp > spmax) sp = spmax;
    c->gsplit = (int32_t)(sp < 1 ? 1 : sp);
    TRY(dalloc(c, &c->cc, (size_t)(k * kst)));
    TRY(dalloc(c, &c->sc, (size_t)k));
    TRY(dalloc(c, &c->gpart, (size_t)(c->gsplit * k * k)));
    TRY(dalloc(c, &c->G, (size_t)(k * k)));
    // Gram rows of at most min(k/4, 64) dirty clusters (same d-splits)
    c->grow_max = (int32_t)((k + 3) / 4 < 64 ? (k + 3) / 4 : 64);
    c->rsplit = c->gsplit;
    TRY(dalloc(c, &c->rpart, (size_t)(c->gsplit * c->grow_max * k)));
  }
  // ---- dense rows: row-major centers, label sort, BF16 operands
  if (c->layout == SKM_DENSE) {
    c->precision = c->opt.precision;
    c->kpad = (int32_t)((k + 255) / 256 * 256);
    TRY(dalloc(c, &c->Cr, (size_t)(k * d)));
    TRY(dalloc(c, &c->lcount, (size_t)k));
    TRY(dalloc(c, &c->loff, (size_t)(k + 1)));
    TRY(dalloc(c, &c->lcursor, (size_t)k));
    TRY(dalloc(c, &c->lmembers, (size_t)n));
    if (c->precision != SKM_PREC_FP32) {
      if (c->precision == SKM_PREC_FP8) {
        uint8_t *xq = nullptr, *cq = nullptr;
        TRY(dalloc(c, &xq, (size_t)(n * d)));
        c->Xb = xq;
        TRY(dalloc(c, &cq, (size_t)(c->kpad * d)));
        c->Cb = cq;
        TRY(dalloc(c, &c->rsc, (size_t)n));
      } else {
        __nv_bfloat16 *xb = nullptr, *cb = nullptr;
        TRY(dalloc(c, &xb, (size_t)(n * d)));
        c->Xb = xb;
        TRY(dalloc(c, &cb, (size_t)(c->kpad * d)));
        c->Cb = cb;
      }
      TRY(dalloc(c, &c->topv, (size_t)(n * kTopK)));
      TRY(dalloc(c, &c->topi, (size_t)(n * kTopK)));
      TRY(dalloc(c, &c->cand, (size_t)(n * 2 * 16)));
      TRY(dalloc(c, &c->cand_n, (size_t)(n * 2)));
      TRY(dalloc(c, &c->w3, (size_t)n));
      // |BF16 similarity - exact| for the unit row x and a center c (|c| <= 1 + 6u)
      // rounded to xb and cb: <xb, cb> - <x, c> = <xb - x, cb> + <x, cb - c>, so by
      // Cauchy-Schwarz it is at most |xb - x| (1 + 6u + |cb - c|) + |cb - c|, plus
      // the FP32 accumulation of d products.  exr holds |xb - x| per row (set here,
      // once), ebc the center terms (set after every center refresh).
      TRY(dalloc(c, &c->exr, (size_t)n));
      TRY(dalloc(c, &c->ebc, (size_t)2));
      TRY(dalloc(c, &c->ebw, (size_t)2));
      SKM_CUDA_TRY(cudaMemsetAsync(c->ebw, 0, sizeof(unsigned) * 2, c->st));
      TRY(c->precision == SKM_PREC_FP8 ? dense_prep_fp8(c) : dense_prep_bf16(c));
    }
  }
  // ---- labels, bounds, worklists
  TRY(dalloc(c, &c->a, (size_t)n));
  if (ham || elk) {
    TRY(dalloc(c, &c->lb, (size_t)n));
    int64_t ucount = elk ? n * kst : yy ? n * ((k + 7) / 8) : n;
    if (yy) TRY(dalloc(c, &c->gdrift, (size_t)(3 * ((k + 7) / 8))));
    if ((elk || yy) && c->nruns > 0) {
      const auto& R = *static_cast<std::vector<RunDesc>*>(c->hruns);
      ucount = R.back().uoff + R.back().n * (yy ? R.back().kst / 8 : R.back().kst);
    }
    TRY(dalloc(c, &c->ub, (size_t)ucount));
    TRY(dalloc(c, &c->w1, (size_t)n));
    TRY(dalloc(c, &c->w2, (size_t)n));
  }
  // ---- screened whole-row passes (Elkan and Hamerly variants, single runs, 128 < k <= 1024)
  const int scr = c->opt.screen;  // 0 auto, 1 on, 2 off
  const bool hamv = (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY);
  if ((elk || hamv) && c->nruns == 0 && c->layout == SKM_CSR && k <= 1024 &&
      (scr == 1 || (scr == 0 && k > 128))) {
    TRY(dalloc(c, &c->Ct16, (size_t)(d * kst)));
    TRY(dalloc(c, &c->e2p, (size_t)(reduction_blocks(d) * kst)));
    TRY(dalloc(c, &c->e2c, (size_t)kst));
    SKM_CUDA_TRY(cudaMemsetAsync(c->e2c, 0, sizeof(double) * kst, c->st));
    TRY(dalloc(c, &c->escr, (size_t)1));
    TRY(dalloc(c, &c->w3, (size_t)n));
    TRY(dalloc(c, &c->w4, (size_t)n));
  }
  // fixed-point scale of the center sums: an entry |x| <= 1 maps below 2^40
  // (the 20 + 20 bit split of k_center_sum) and |sum| <= n must stay below
  // 2^62 in the 64-bit partials
  int bits = 1;
  while ((int64_t(1) << bits) <= n) ++bits;
  const int sbits = (62 - bits) < 40 ? (62 - bits) : 40;
  c->fx_scale = std::ldexp(1.0f, sbits);
  c->fx_inv = std::ldexp(1.0f, -sbits);
  TRY(set_init(c, init_rows, seed));
  return SKM_OK;
}

}  // namespace

extern "C" {

void skm_default_options(skm_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->validate = 1;
}

int skm_init(skm_ctx** out, const skm_data* x, int32_t k, int32_t variant, const int64_t* init_rows, uint64_t seed,
             const skm_options* opt, void* stream) {
  if (!out) return SKM_EINVAL;
  *out = nullptr;
  if (!x || x->n < 1 || x->d < 1 || k < 1 || k > x->n || x->reserved != 0) return SKM_EINVAL;
  if (variant < SKM_STANDARD || variant > SKM_YINYANG) return SKM_EINVAL;
  if (x->dtype < SKM_F32 || x->dtype > SKM_BF16) return SKM_EINVAL;
  if (x->layout != SKM_CSR && x->layout != SKM_DENSE) return SKM_EINVAL;
  if (variant == SKM_YINYANG && x->layout != SKM_CSR) return SKM_EUNSUPPORTED;
  if (x->memspace != SKM_DEVICE && x->memspace != SKM_HOST) return SKM_EINVAL;
  if (!x->values || (x->layout == SKM_CSR && (!x->row_ptr || !x->col_idx))) return SKM_EINVAL;
  if (x->d > INT32_MAX || x->n > INT32_MAX) return SKM_EUNSUPPORTED;
  if ((variant == SKM_ELKAN || variant == SKM_SIMP_ELKAN) && k > 4096) return SKM_EUNSUPPORTED;
  // Yin-Yang keeps a row's similarities of one pass over the row (up to 1024 centers) for its group bounds
  if (variant == SKM_YINYANG && k > 1024) return SKM_EUNSUPPORTED;
  // the sparse kernels address the term-major centers with 32-bit offsets:
  // d round8(k) < 2^32 (a center table below 16 GB)
  if (x->layout == SKM_CSR && x->d * (((int64_t)k + 7) / 8 * 8) >= (int64_t(1) << 32)) return SKM_EUNSUPPORTED;
  skm_ctx* c = new (std::nothrow) skm_ctx();
  if (!c) return SKM_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->st = (cudaStream_t)stream;
  c->n = x->n;
  c->d = x->d;
  c->k = k;
  c->kst = (k + 7) / 8 * 8;
  c->variant = variant;
  c->layout = x->layout;
  c->dtype = x->dtype;
  if (opt) c->opt = *opt;
  else skm_default_options(&c->opt);
  {
    const int kt = c->opt.k_tile;
    if (kt != 0 && kt != 128 && kt != 256 && kt != 512 && kt != 1024) {
      delete c;
      return SKM_EINVAL;
    }
    if (kt != 0 && (variant == SKM_YINYANG || x->layout != SKM_CSR)) {
      delete c;
      return SKM_EUNSUPPORTED;
    }
  }
  if (x->layout == SKM_DENSE) {
    if (x->dtype != SKM_F32 || variant == SKM_ELKAN || variant == SKM_SIMP_ELKAN) {
      delete c;
      return SKM_EUNSUPPORTED;
    }
    if (c->opt.precision < SKM_PREC_FP32 || c->opt.precision > SKM_PREC_FP8) {
      delete c;
      return SKM_EINVAL;
    }
    if ((c->opt.precision == SKM_PREC_BF16 && !bf16_mma_supported(x->d)) ||
        (c->opt.precision == SKM_PREC_FP8 && !fp8_mma_supported(x->d))) {
      delete c;
      return SKM_EUNSUPPORTED;
    }
  }
  c->prof = new (std::nothrow) ProfList();
  if (!c->prof) {
    delete c;
    return SKM_ENOMEM;
  }
  const int rc = build_ctx(c, x, init_rows, seed);
  if (rc != SKM_OK) {
    release(c);
    return rc;
  }
  *out = c;
  return SKM_OK;
}

int skm_batch_init(skm_ctx** out, const skm_data* x, const int64_t* run_rows, const int32_t* ks, int32_t nruns,
                   int32_t variant, const int64_t* init_rows, uint64_t seed, const skm_options* opt, void* stream) {
  if (!out) return SKM_EINVAL;
  *out = nullptr;
  if (!x || !run_rows || !ks || nruns < 1 || x->n < 1 || x->d < 1 || x->reserved != 0) return SKM_EINVAL;
  if (opt && opt->k_tile != 0) return SKM_EUNSUPPORTED;  // a batch walks every run's slice 128 centers at a time
  if (x->layout != SKM_CSR) return SKM_EUNSUPPORTED;
  if (variant < SKM_STANDARD || variant > SKM_YINYANG) return SKM_EINVAL;
  if (x->dtype < SKM_F32 || x->dtype > SKM_BF16) return SKM_EINVAL;
  if (x->memspace != SKM_DEVICE && x->memspace != SKM_HOST) return SKM_EINVAL;
  if (!x->values || !x->row_ptr || !x->col_idx) return SKM_EINVAL;
  if (x->d > INT32_MAX || x->n > INT32_MAX || (int64_t)nruns * x->d > INT32_MAX) return SKM_EUNSUPPORTED;
  if (run_rows[0] != 0 || run_rows[nruns] != x->n) return SKM_EINVAL;
  std::vector<RunDesc> R((size_t)nruns);
  int64_t koff = 0, uoff = 0, ccoff = 0;
  int32_t kmax = 0;
  for (int32_t r = 0; r < nruns; ++r) {
    const int64_t nr = run_rows[r + 1] - run_rows[r];
    if (nr < 1 || ks[r] < 1 || ks[r] > nr) return SKM_EINVAL;
    if (ks[r] > 4096) return SKM_EUNSUPPORTED;
    if (variant == SKM_YINYANG && ks[r] > 512) return SKM_EUNSUPPORTED;  // group bounds from one pass
    RunDesc& d = R[(size_t)r];
    d.row0 = run_rows[r];
    d.n = nr;
    d.k = ks[r];
    d.kst = (ks[r] + 7) / 8 * 8;
    d.koff = (int32_t)koff;
    d.uoff = uoff;
    d.ccoff = ccoff;
    int32_t cap = opt && opt->row_threshold > 0 ? opt->row_threshold : (ks[r] + 7) / 8;
    d.cap = cap > 7 ? 7 : cap;
    koff += d.kst;
    uoff += nr * (variant == SKM_YINYANG ? d.kst / 8 : d.kst);  // Elkan: a bound per center; Yin-Yang: per group
    ccoff += (int64_t)d.k * d.kst;
    if (d.kst > kmax) kmax = d.kst;
  }
  if (koff > INT32_MAX / 2) return SKM_EUNSUPPORTED;
  if (x->d * koff >= (int64_t(1) << 32)) return SKM_EUNSUPPORTED;  // 32-bit offsets into Ct
  skm_ctx* c = new (std::nothrow) skm_ctx();
  if (!c) return SKM_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->st = (cudaStream_t)stream;
  c->n = x->n;
  c->d = x->d;
  c->k = (int32_t)koff;  // every run's slice, padding included
  c->kst = (int32_t)koff;
  c->kmax = kmax;
  c->nruns = nruns;
  c->variant = variant;
  c->layout = x->layout;
  c->dtype = x->dtype;
  if (opt) c->opt = *opt;
  else skm_default_options(&c->opt);
  c->prof = new (std::nothrow) ProfList();
  c->hruns = new (std::nothrow) std::vector<RunDesc>(R);
  if (!c->prof || !c->hruns) {
    release(c);
    return SKM_ENOMEM;
  }
  int rc = SKM_OK;
  std::vector<int32_t> rr((size_t)x->n);
  for (int32_t r = 0; r < nruns; ++r)
    for (int64_t i = run_rows[r]; i < run_rows[r + 1]; ++i) rr[(size_t)i] = r;
  if ((rc = dalloc(c, &c->runs, (size_t)nruns)) == SKM_OK && (rc = dalloc(c, &c->row_run, (size_t)x->n)) == SKM_OK) {
    if (cudaMemcpyAsync(c->runs, R.data(), sizeof(RunDesc) * nruns, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(c->row_run, rr.data(), sizeof(int32_t) * x->n, cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
      rc = SKM_ECUDA;
  }
  if (rc == SKM_OK) rc = build_ctx(c, x, init_rows, seed);
  if (rc != SKM_OK) {
    release(c);
    return rc;
  }
  *out = c;
  return SKM_OK;
}

int skm_reset(skm_ctx* c, const int64_t* init_rows, uint64_t seed) {
  if (!c) return SKM_EINVAL;
  return set_init(c, init_rows, seed);
}

namespace {

// One steady-state iteration (assignment, log of its counters, center
// update) captured from a private stream into a CUDA graph.  Launch counts of
// the capture are taken back out; each replay adds the graph's kernel nodes.
int capture_iteration(skm_ctx* c);

int build_graph(skm_ctx* c) {
  if (!c->cap_st) SKM_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  if (!c->glog) {
    TRY(dalloc(c, &c->glog, (size_t)(2 + 2 * kLogCap)));
    SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  const long long before = g_launches.load();
  const skm_stats saved = c->stats;  // the capture runs nothing
  cudaStream_t orig = c->st;
  c->st = c->cap_st;
  SKM_CUDA_TRY(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeRelaxed));
  const int rc = capture_iteration(c);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c->cap_st, &g);
  c->st = orig;
  c->stats = saved;
  g_launches.fetch_sub(g_launches.load() - before);
  if (rc != SKM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ec != cudaSuccess || !g) {
    (void)cudaGetLastError();
    return SKM_ECUDA;
  }
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  c->gkernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++c->gkernels;
  }
  const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    (void)cudaGetLastError();
    c->gexec = nullptr;
    return SKM_ECUDA;
  }
  return SKM_OK;
}

// One assignment of dense rows (standard or Hamerly; FP32 or BF16 bulk).
int assign_dense(skm_ctx* c) {
  TRY(dense_refresh_centers(c));
  const bool ham = (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY);
  const bool first = !c->have_bounds;
  if (c->precision != SKM_PREC_FP32) {
    // the precision form keeps Hamerly's l (and u) for every variant: l seeds
    // the candidate threshold of the tensor-core pass
    const int32_t* list = nullptr;
    const unsigned long long* lcnt = nullptr;
    if (!first) {
      if (ham) {
        TRY(hamerly_bounds_only(c));  // survivors of the bound test -> w1
        list = c->w1;
        lcnt = c->cnt + C_W1;
      } else if (c->moved) {
        TRY(dense_lower(c));
      }
    }
    TRY(bf16_topk(c, c->Xb, c->Cb, first ? 0 : 1, c->topv, c->topi));
    TRY(dense_classify(c, true, list, lcnt));  // ambiguous rows -> w3
    TRY(dense_recheck_cands(c, true));         // unresolved rows -> w2
    TRY(dense_rows(c, 1, c->w2, c->cnt + C_W2));
    c->have_bounds = 1;
  } else if (!ham || first) {
    TRY(dense_rows(c, ham ? 1 : 0, nullptr, nullptr));
  } else {
    TRY(hamerly_bounds_only(c));
    TRY(dense_tighten(c));
    TRY(dense_rows(c, 1, c->w2, c->cnt + C_W2));
  }
  if (ham) c->have_bounds = 1;
  return SKM_OK;
}

}  // namespace

int skm_assign(skm_ctx* c, int64_t* n_changed) {
  if (!c) return SKM_EINVAL;
  if (!c->cnt_clear) SKM_CUDA_TRY(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * C_ERR, c->st));
  c->cnt_clear = 0;
  int rc;
  if (c->layout == SKM_DENSE) {
    rc = assign_dense(c);
  } else if (!c->have_bounds || c->variant == SKM_STANDARD) {
    const int mode = (c->variant == SKM_STANDARD) ? 0
                     : (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY) ? 1
                     : (c->variant == SKM_YINYANG)                                   ? 3
                                                                                      : 2;
    rc = assign_full(c, mode, nullptr, nullptr, c->n);
    if (rc == SKM_OK) c->have_bounds = (c->variant != SKM_STANDARD);
  } else if (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY) {
    rc = hamerly_step(c);
  } else if (c->variant == SKM_YINYANG) {
    rc = yinyang_step(c);
  } else {
    rc = elkan_step(c);
  }
  if (rc) return rc;
  c->moved = 0;
  c->chg_fresh = 1;
  c->stats.iterations++;
  if (n_changed) {
    TRY(read_counters(c));
    if (c->hcnt[C_ERR] & E_TIMEOUT) return SKM_ETIMEOUT;
    c->stats.total_sims += c->stats.last_sims;
    *n_changed = c->stats.last_changed;
  } else {
    c->stats.last_changed = -1;
  }
  return SKM_OK;
}

int skm_update_centers(skm_ctx* c, double* objective) {
  if (!c) return SKM_EINVAL;
  // without an assignment since the last update no label changed
  if (!c->chg_fresh) SKM_CUDA_TRY(cudaMemsetAsync(c->cnt + C_CHG, 0, sizeof(unsigned long long), c->st));
  TRY(update_centers(c));
  c->chg_fresh = 0;
  c->cnt_clear = 1;  // its last kernel zeroed the assignment counters
  c->moved = 1;
  if (objective) {
    SKM_CUDA_TRY(cudaMemcpyAsync(c->hobj, c->obj, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
    *objective = *c->hobj;
    c->stats.objective = *c->hobj;
  }
  return SKM_OK;
}

int skm_run(skm_ctx* c, int32_t max_iters, int32_t* iters_done, double* objective) {
  if (!c || max_iters < 0) return SKM_EINVAL;
  int32_t it = 0;
  bool done = false;
  const bool use_graph = c->opt.graph && c->layout == SKM_CSR && !c->prof_on;
  // eager iterations (all of them, or the first one before the graph: the
  // graph holds the steady state, bounds present and centers moved)
  while (it < max_iters && !done) {
    int64_t ch = 0;
    TRY(skm_assign(c, &ch));
    ++it;
    if (ch == 0) {
      done = true;
      break;
    }
    TRY(skm_update_centers(c, nullptr));
    if (use_graph) break;
  }
  if (use_graph && !done && it < max_iters) {
    TRY(build_graph(c));
    int check = c->opt.graph_check > 0 ? c->opt.graph_check : 8;
    if (check > kLogCap) check = kLogCap;
    while (it < max_iters && !done) {
      const int m = (max_iters - it) < check ? (max_iters - it) : check;
      SKM_CUDA_TRY(cudaMemsetAsync(c->glog, 0, sizeof(unsigned long long), c->st));
      for (int q = 0; q < m; ++q) SKM_CUDA_TRY(cudaGraphLaunch(c->gexec, c->st));
      note_launch((int)(m * c->gkernels));
      std::vector<unsigned long long> lg((size_t)(2 + 2 * m));
      SKM_CUDA_TRY(cudaMemcpyAsync(lg.data(), c->glog, sizeof(unsigned long long) * lg.size(),
                                   cudaMemcpyDeviceToHost, c->st));
      SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
      for (int q = 0; q < m; ++q) {
        ++it;
        c->stats.iterations++;
        c->stats.last_changed = (int64_t)lg[(size_t)(2 + 2 * q)];
        c->stats.last_sims = (int64_t)lg[(size_t)(3 + 2 * q)];
        c->stats.total_sims += c->stats.last_sims;
        if (c->stats.last_changed == 0) {
          done = true;  // later replays of this chunk changed nothing
          break;
        }
      }
    }
    c->moved = 1;
    c->chg_fresh = 0;
    c->cnt_clear = 0;
  }
  SKM_CUDA_TRY(cudaMemcpyAsync(c->hobj, c->obj, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->stats.objective = *c->hobj;
  if (iters_done) *iters_done = it;
  if (objective) *objective = *c->hobj;
  return SKM_OK;
}

int skm_get_labels(skm_ctx* c, int32_t* out, int32_t space) {
  if (!c || !out) return SKM_EINVAL;
  if (c->nruns > 0) {
    // labels local to each run
    int32_t* tmp = nullptr;
    if (space == SKM_HOST) TRY(dalloc(c, &tmp, (size_t)c->n));
    int32_t* dst = space == SKM_HOST ? tmp : out;
    k_labels_local<<<grid_cap(c->n, 256, c->nsm), 256, 0, c->st>>>(c->a, c->n, c->row_run, c->runs, dst);
    note_launch(1);
    int rc = SKM_OK;
    if (space == SKM_HOST) {
      if (cudaMemcpyAsync(out, tmp, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        rc = SKM_ECUDA;
      cudaFreeAsync(tmp, c->st);
      if (cudaStreamSynchronize(c->st) != cudaSuccess) rc = SKM_ECUDA;
    }
    return rc;
  }
  SKM_CUDA_TRY(cudaMemcpyAsync(out, c->a, sizeof(int32_t) * c->n,
                               space == SKM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
  if (space == SKM_HOST) SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  return SKM_OK;
}

int skm_get_centers(skm_ctx* c, float* out, int32_t space) {
  if (!c || !out) return SKM_EINVAL;
  int64_t krows = c->k;
  if (c->nruns > 0) {
    krows = 0;
    for (const auto& r : *static_cast<std::vector<RunDesc>*>(c->hruns)) krows += r.k;
  }
  auto fill = [&](float* dst) -> int {
    if (c->nruns == 0) return centers_to_rows(c, dst);
    k_centers_batch<<<grid_cap(krows * c->d, 256, c->nsm), 256, 0, c->st>>>(c->Ct, c->d, c->kst, c->runs, c->nruns,
                                                                            krows, dst);
    note_launch(1);
    return SKM_OK;
  };
  if (space == SKM_DEVICE) return fill(out);
  float* tmp = nullptr;
  TRY(dalloc(c, &tmp, (size_t)(krows * c->d)));
  int rc = fill(tmp);
  if (rc == SKM_OK && cudaMemcpyAsync(out, tmp, sizeof(float) * krows * c->d, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
    rc = SKM_ECUDA;
  cudaFreeAsync(tmp, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) rc = SKM_ECUDA;
  return rc;
}

int skm_set_centers(skm_ctx* c, const float* C, int32_t space) {
  if (!c || !C) return SKM_EINVAL;
  if (c->nruns > 0) return SKM_EUNSUPPORTED;
  int rc;
  if (space == SKM_DEVICE) {
    rc = rows_to_centers(c, C);
  } else {
    float* tmp = nullptr;
    TRY(dalloc(c, &tmp, (size_t)(c->k * c->d)));
    SKM_CUDA_TRY(cudaMemcpyAsync(tmp, C, sizeof(float) * c->k * c->d, cudaMemcpyHostToDevice, c->st));
    rc = rows_to_centers(c, tmp);
    cudaFreeAsync(tmp, c->st);
    SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  if (rc == SKM_OK) rc = ct16_all(c);
  c->have_bounds = 0;
  c->moved = 0;
  c->s64_valid = 0;
  c->chg_fresh = 0;
  c->cnt_clear = 0;
  return rc;
}

int skm_set_labels(skm_ctx* c, const int32_t* lab, int32_t space) {
  if (!c || !lab) return SKM_EINVAL;
  if (c->nruns > 0) return SKM_EUNSUPPORTED;
  if (space == SKM_HOST)
    for (int64_t i = 0; i < c->n; ++i)
      if (lab[i] < 0 || lab[i] >= c->k) return SKM_EINVAL;
  SKM_CUDA_TRY(cudaMemcpyAsync(c->a, lab, sizeof(int32_t) * c->n,
                               space == SKM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
  if (space == SKM_HOST) SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->have_bounds = 0;
  c->s64_valid = 0;
  c->chg_fresh = 0;
  c->cnt_clear = 0;
  return SKM_OK;
}

int skm_get_bounds(skm_ctx* c, float* l, float* u, int32_t space) {
  if (!c) return SKM_EINVAL;
  if (c->nruns > 0) return SKM_EUNSUPPORTED;
  if (c->variant == SKM_STANDARD || !c->have_bounds) return SKM_ESTATE;
  const bool elk = (c->variant == SKM_ELKAN || c->variant == SKM_SIMP_ELKAN);
  const cudaMemcpyKind kind = space == SKM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (l) SKM_CUDA_TRY(cudaMemcpyAsync(l, c->lb, sizeof(float) * c->n, kind, c->st));
  if (u) {
    if (elk)
      SKM_CUDA_TRY(cudaMemcpy2DAsync(u, sizeof(float) * c->k, c->ub, sizeof(float) * c->kst, sizeof(float) * c->k,
                                     (size_t)c->n, kind, c->st));
    else if (c->variant == SKM_YINYANG)
      SKM_CUDA_TRY(cudaMemcpyAsync(u, c->ub, sizeof(float) * c->n * ((c->k + 7) / 8), kind, c->st));
    else
      SKM_CUDA_TRY(cudaMemcpyAsync(u, c->ub, sizeof(float) * c->n, kind, c->st));
  }
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  return SKM_OK;
}

int skm_get_bf16_topk(skm_ctx* c, float* vals, int32_t* idx, float* eps, int32_t space) {
  if (!c) return SKM_EINVAL;
  if (c->layout != SKM_DENSE || c->precision == SKM_PREC_FP32 || !c->have_bounds) return SKM_ESTATE;
  const cudaMemcpyKind kind = space == SKM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (eps) {
    float* out = eps;
    if (space == SKM_HOST) TRY(dalloc(c, &out, (size_t)c->n));
    int rc = dense_bf16_eps(c, out);
    if (space == SKM_HOST) {
      if (rc == SKM_OK &&
          cudaMemcpyAsync(eps, out, sizeof(float) * c->n, cudaMemcpyDeviceToHost, c->st) != cudaSuccess)
        rc = SKM_ECUDA;
      cudaFreeAsync(out, c->st);
    }
    if (rc != SKM_OK) {
      (void)cudaGetLastError();
      return rc;
    }
  }
  if (vals) SKM_CUDA_TRY(cudaMemcpyAsync(vals, c->topv, sizeof(float) * kTopK * c->n, kind, c->st));
  if (idx) SKM_CUDA_TRY(cudaMemcpyAsync(idx, c->topi, sizeof(int32_t) * kTopK * c->n, kind, c->st));
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  return SKM_OK;
}

int skm_get_stats(skm_ctx* c, skm_stats* out) {
  if (!c || !out) return SKM_EINVAL;
  *out = c->stats;
  return SKM_OK;
}

int skm_bound_bytes(int32_t variant, int64_t n, int32_t k, int64_t* bytes) {
  if (!bytes || n < 0 || k < 1) return SKM_EINVAL;
  switch (variant) {
    case SKM_STANDARD: *bytes = 0; return SKM_OK;
    case SKM_HAMERLY:
    case SKM_SIMP_HAMERLY: *bytes = 8 * n; return SKM_OK;
    case SKM_ELKAN:
    case SKM_SIMP_ELKAN: *bytes = 4 * n + 4 * n * (int64_t)k; return SKM_OK;
    case SKM_YINYANG: *bytes = 4 * n + 4 * n * (int64_t)((k + 7) / 8); return SKM_OK;
  }
  return SKM_EINVAL;
}

int64_t skm_kernel_launches(void) { return (int64_t)g_launches.load(); }

int skm_profile(skm_ctx* c, int32_t enable) {
  if (!c) return SKM_EINVAL;
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_clear(c);
  c->prof_on = enable ? 1 : 0;
  return SKM_OK;
}

int skm_profile_read(skm_ctx* c, int32_t idx, char* name, int32_t name_len, double* total_ms, int64_t* launches) {
  if (!c || idx < 0) return SKM_EINVAL;
  SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
  ProfList* L = static_cast<ProfList*>(c->prof);
  // distinct kernel names in order of first launch
  std::vector<const char*> names;
  for (auto& r : *L) {
    bool seen = false;
    for (const char* q : names) seen = seen || std::strcmp(q, r.name) == 0;
    if (!seen) names.push_back(r.name);
  }
  if (idx >= (int32_t)names.size()) return SKM_EINVAL;
  double tot = 0.0;
  int64_t cntl = 0;
  for (auto& r : *L) {
    if (std::strcmp(r.name, names[idx]) != 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.b, r.e) == cudaSuccess) {
      tot += ms;
      ++cntl;
    } else {
      (void)cudaGetLastError();
    }
  }
  if (name && name_len > 0) {
    std::strncpy(name, names[idx], (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = cntl;
  return SKM_OK;
}

int skm_autotune(skm_ctx* c, const char* cache_path, int32_t iters, int32_t* from_cache) {
  if (!c || iters < 1) return SKM_EINVAL;
  if (from_cache) *from_cache = 0;
  if (!c->hinit) return SKM_ESTATE;
  // shape bucket: device, variant, batch or not, log2 of n, k (widest run)
  // and mean nonzeros per row
  cudaDeviceProp prop;
  SKM_CUDA_TRY(cudaGetDeviceProperties(&prop, c->dev));
  auto lg2 = [](double v) { return v < 1.0 ? 0 : (int)std::floor(std::log2(v)); };
  const int32_t kb = c->nruns > 0 ? c->kmax : c->k;
  char key[320];
  std::snprintf(key, sizeof(key), "%s|sm%d|v%d|b%d|L%d|n%d|k%d|z%d", prop.name, c->nsm, c->variant,
                c->nruns > 0 ? 1 : 0, c->layout, lg2((double)c->n), lg2((double)kb),
                lg2((double)c->nnz / (double)c->n));
  for (char* q = key; *q; ++q)
    if (*q == ' ') *q = '_';
  const bool elk = (c->variant == SKM_ELKAN || c->variant == SKM_SIMP_ELKAN);
  auto apply = [&](int32_t bpsm, int32_t thr, int32_t kt, int32_t so) -> int {
    c->opt.blocks_per_sm = bpsm;
    c->opt.row_threshold = thr;
    c->opt.k_tile = kt;
    c->scr_off = so;
    if (c->nruns > 0) {
      auto& R = *static_cast<std::vector<RunDesc>*>(c->hruns);
      for (auto& r : R) {
        const int32_t cap = thr > 0 ? thr : (r.k + 7) / 8;
        r.cap = cap > 7 ? 7 : cap;
      }
      SKM_CUDA_TRY(cudaMemcpyAsync(c->runs, R.data(), sizeof(RunDesc) * R.size(), cudaMemcpyHostToDevice, c->st));
      SKM_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    return SKM_OK;
  };
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char line[512];
      int found = 0, bp = 0, th = 0, kt = 0, so = 0;
      while (std::fgets(line, sizeof(line), f)) {
        char k2[320];
        int b2, t2, k3 = 0, s3 = 0;
        const int nf = std::sscanf(line, "%319s %d %d %d %d", k2, &b2, &t2, &k3, &s3);
        if (nf >= 3 && std::strcmp(k2, key) == 0) {
          found = 1;
          bp = b2;
          th = t2;
          kt = nf >= 4 ? k3 : 0;
          so = nf >= 5 ? s3 : 0;
        }
      }
      std::fclose(f);
      if (found) {
        TRY(apply(bp, th, kt, so));
        if (from_cache) *from_cache = 1;
        return SKM_OK;
      }
    }
  }
  const std::vector<int64_t> init = *static_cast<std::vector<int64_t>*>(c->hinit);
  cudaEvent_t e0, e1;
  SKM_CUDA_TRY(cudaEventCreate(&e0));
  SKM_CUDA_TRY(cudaEventCreate(&e1));
  // time `iters` iterations under a setting, after 4 iters untimed ones
  // from the initial centers: the first iterations send nearly every row to
  // a whole-row recompute whatever the setting, so they do not tell the
  // settings apart
  auto timed = [&](int32_t bpsm, int32_t thr, int32_t kt, int32_t so, float* ms) -> int {
    TRY(apply(bpsm, thr, kt, so));
    TRY(start_from_rows(c, init));
    int rc = SKM_OK;
    for (int32_t it = 0; it < 5 * iters && rc == SKM_OK; ++it) {
      if (it == 4 * iters) cudaEventRecord(e0, c->st);
      rc = skm_assign(c, nullptr);
      if (rc == SKM_OK) rc = skm_update_centers(c, nullptr);
    }
    cudaEventRecord(e1, c->st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = SKM_ECUDA;
    if (rc == SKM_OK) cudaEventElapsedTime(ms, e0, e1);
    return rc;
  };
  // coordinate search: launch shape x Elkan whole-row threshold, then the
  // whole-row kernel's tile of centers (single CSR runs but Yin-Yang: the
  // default tile and up to two smaller ones), then the screened pass on or off
  // (where the context keeps the FP16 centers)
  const int32_t bps[3] = {4, 8, 16};  // blocks per SM of the persistent kernels, capped at what is resident
  const int32_t thrs[3] = {0, 2, 7};
  const int nthr = elk ? 3 : 1;
  float best = INFINITY, ms = 0.f;
  int32_t bb = 8, bt = 0, bk = 0, bs = 0;
  int rc = SKM_OK;
  for (int a = 0; a < 3 && rc == SKM_OK; ++a)
    for (int b = 0; b < nthr && rc == SKM_OK; ++b)
      if ((rc = timed(bps[a], thrs[b], 0, 0, &ms)) == SKM_OK && ms < best) {
        best = ms;
        bb = bps[a];
        bt = thrs[b];
      }
  if (rc == SKM_OK && c->nruns == 0 && c->layout == SKM_CSR && c->variant != SKM_YINYANG) {
    const int32_t k = c->k;
    const int32_t kt0 = k <= 128 ? 128 : k <= 256 ? 256 : k <= 512 ? 512 : 1024;
    for (int32_t kt = kt0 / 2; kt >= 128 && kt >= kt0 / 4 && rc == SKM_OK; kt /= 2)
      if ((rc = timed(bb, bt, kt, 0, &ms)) == SKM_OK && ms < best) {
        best = ms;
        bk = kt;
      }
  }
  if (rc == SKM_OK && c->Ct16 && (rc = timed(bb, bt, bk, 1, &ms)) == SKM_OK && ms < best) {
    best = ms;
    bs = 1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SKM_OK) return rc;
  TRY(apply(bb, bt, bk, bs));
  TRY(start_from_rows(c, init));
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s %d %d %d %d\n", key, bb, bt, bk, bs);
      std::fclose(f);
    }
  }
  return SKM_OK;
}

int skm_seed_kmeanspp(skm_ctx* c, const double* u, int64_t* rows_out) {
  if (!c || !u) return SKM_EINVAL;
  if (c->nruns > 0) return SKM_EUNSUPPORTED;
  for (int32_t j = 0; j < c->k; ++j)
    if (!(u[j] >= 0.0 && u[j] < 1.0)) return SKM_EINVAL;
  std::vector<int64_t> rows((size_t)c->k);
  TRY(seed_kmeanspp(c, u, rows.data()));
  {
    std::unordered_set<int64_t> seen;
    for (int64_t r : rows)
      if (r < 0 || r >= c->n || !seen.insert(r).second) return SKM_ECUDA;  // not reachable
  }
  TRY(start_from_rows(c, rows));
  if (rows_out) std::memcpy(rows_out, rows.data(), sizeof(int64_t) * rows.size());
  return SKM_OK;
}

int skm_seed_kmeanspp_assign(skm_ctx* c, const double* u, int64_t* rows_out, int64_t* n_changed) {
  if (!c || !u) return SKM_EINVAL;
  if (c->nruns > 0 || c->variant == SKM_YINYANG) return SKM_EUNSUPPORTED;
  for (int32_t j = 0; j < c->k; ++j)
    if (!(u[j] >= 0.0 && u[j] < 1.0)) return SKM_EINVAL;
  const bool elk = (c->variant == SKM_ELKAN || c->variant == SKM_SIMP_ELKAN);
  const bool ham = (c->variant == SKM_HAMERLY || c->variant == SKM_SIMP_HAMERLY);
  SeedFirst first = {elk ? 1 : 0, c->lb ? 1 : 0, (c->ub && !elk) ? 1 : 0, nullptr, nullptr, nullptr};
  std::vector<int64_t> rows((size_t)c->k);
  TRY(seed_kmeanspp(c, u, rows.data(), &first));
  {
    std::unordered_set<int64_t> seen;
    for (int64_t r : rows)
      if (r < 0 || r >= c->n || !seen.insert(r).second) return SKM_ECUDA;  // not reachable
  }
  TRY(start_from_rows(c, rows));
  // the assignment the seeding made: its counters start from zero, as in skm_assign
  SKM_CUDA_TRY(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * C_ERR, c->st));
  TRY(seed_finish(c, &first));
  c->have_bounds = c->layout == SKM_DENSE ? (ham || c->precision != SKM_PREC_FP32) : (c->variant != SKM_STANDARD);
  c->moved = 0;
  c->chg_fresh = 1;
  c->cnt_clear = 0;
  c->stats.iterations = 1;
  if (rows_out) std::memcpy(rows_out, rows.data(), sizeof(int64_t) * rows.size());
  if (n_changed) {
    TRY(read_counters(c));
    c->stats.total_sims += c->stats.last_sims;
    *n_changed = c->stats.last_changed;
  } else {
    c->stats.last_changed = -1;
  }
  return SKM_OK;
}

int skm_selftest_wait(int64_t timeout_ns, void* stream) {
  if (timeout_ns < 1 || timeout_ns > 2000000000ll) return SKM_EINVAL;
  const int a = wait_selftest(timeout_ns, (cudaStream_t)stream);
  if (a != SKM_OK && a != SKM_ETIMEOUT) return a;
  const int b = barrier_selftest(timeout_ns, (cudaStream_t)stream);
  if (b != SKM_OK && b != SKM_ETIMEOUT) return b;
  // both waits must have given up
  return (a == SKM_ETIMEOUT && b == SKM_ETIMEOUT) ? SKM_ETIMEOUT : SKM_OK;
}

void skm_destroy(skm_ctx* c) { release(c); }

const char* skm_strerror(int s) {
  switch (s) {
    case SKM_OK: return "ok";
    case SKM_EINVAL: return "invalid argument or malformed input";
    case SKM_ENOMEM: return "out of memory";
    case SKM_ECUDA: return "CUDA error";
    case SKM_ETIMEOUT: return "device wait timed out";
    case SKM_EUNSUPPORTED: return "unsupported configuration";
    case SKM_ESTATE: return "invalid state for this call";
    case SKM_ETOOBIG: return "problem exceeds the fixed-size limit of this call";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

int capture_iteration(skm_ctx* c) {
  TRY(skm_assign(c, nullptr));
  c->glog_active = c->glog;  // the update's first kernel logs the changed count
  const int rc = skm_update_centers(c, nullptr);
  c->glog_active = nullptr;
  return rc;
}

}  // namespace
