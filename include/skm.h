/*
 * skm.h -- C ABI of the GB300 spherical k-means library (libskm.so).
 *
 * Implements one Lloyd iteration of spherical k-means and its accelerated
 * variants from "Accelerating Spherical k-Means" (Schubert, Lang, Feher,
 * arXiv 2107.04074):
 *   - assignment a(i) = argmax_j <x(i), c(j)> on unit vectors (Section 5),
 *     pruned with cosine bounds kept directly on similarities (Section 4:
 *     Eq. eqn:l-bound, Eq. eqn:u-elkan; Section 5.3: Eq. eqn:u-hamerly-2);
 *   - center update c(j) = sum_{a(i)=j} x(i) / |sum| (Section 5).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: SKM_OK (0) or a negative SKM_E*
 *     code (skm_strerror names it).  No call aborts the process.
 *   - Work is enqueued on the CUDA stream given to skm_init (passed as a
 *     plain pointer, NULL = legacy default stream).  A call synchronises
 *     that stream only when it returns a host scalar (non-NULL host output).
 *   - Device pointers given to skm_init with memspace SKM_DEVICE are
 *     BORROWED: the caller keeps them alive and unchanged until
 *     skm_destroy.  With SKM_HOST the library copies them to device memory it
 *     owns.  All other device memory is allocated by the library
 *     (cudaMallocAsync on the context's stream) and released by skm_destroy.
 *   - Rows are normalised by the library (Section 5: all samples normalised
 *     at initialisation): stored rows need not be exactly unit length, but a
 *     row may not be all zero.
 *   - Ties follow one rule everywhere: the current label wins; among the
 *     other centers the lowest index wins (a point moves only on a strict
 *     improvement).  All variants therefore produce the label sequence of the
 *     standard variant.
 */
#ifndef SKM_H
#define SKM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SKM_OK 0
#define SKM_EINVAL (-1)       /* bad argument or malformed input data */
#define SKM_ENOMEM (-2)       /* device or host allocation failed */
#define SKM_ECUDA (-3)        /* a CUDA runtime call or a kernel launch failed */
#define SKM_ETIMEOUT (-4)     /* a bounded device-side wait expired */
#define SKM_EUNSUPPORTED (-5) /* valid request this build does not handle */
#define SKM_ESTATE (-6)       /* call not valid in the context's current state */
#define SKM_ETOOBIG (-7)      /* problem larger than a fixed-size limit of the call */

/* ---- enumerations ---- */
/* Variants (Section 5): standard Lloyd; Hamerly (5.3 + center test 5.4);
 * Elkan (5.2); Simplified Hamerly (5.4, no center test); Simplified Elkan
 * (5.1, no center-center tests); Yin-Yang group bounds (5.5, CSR data only,
 * k <= 1024: one upper bound per group of 8 consecutive centers, moved by the
 * group's worst drift). */
typedef enum {
  SKM_STANDARD = 0,
  SKM_HAMERLY = 1,
  SKM_ELKAN = 2,
  SKM_SIMP_HAMERLY = 3,
  SKM_SIMP_ELKAN = 4,
  SKM_YINYANG = 5
} skm_variant;

typedef enum { SKM_F32 = 0, SKM_F16 = 1, SKM_BF16 = 2 } skm_dtype;
typedef enum { SKM_CSR = 0, SKM_DENSE = 1 } skm_layout;
typedef enum { SKM_DEVICE = 0, SKM_HOST = 1 } skm_memspace;

/* Arithmetic of the dense similarity bulk.  FP32: the plain FP32 GEMM (the
 * reference point).  BF16: the precision form -- a BF16 x BF16 -> FP32
 * tensor-core GEMM whose per-row top-2 decides a label when its margin
 * exceeds the row's proven error bound (from the row's and the centers'
 * actual BF16 rounding errors, see skm_get_bf16_topk); the other rows are
 * rechecked in FP32 against the centers that can still win, so the labels
 * are those of the FP32 path.  FP8: the same with FP8-E4M3 operands
 * (E4M3 x E4M3 -> FP32): each unit row is scaled by its own power of two
 * 2^e_i (its largest entry lands in [128, 256)) and every center by 2^8
 * before rounding, so the accumulator times 2^-(e_i + 8) is the similarity,
 * exactly; E4M3 keeps 4 significant bits, so the error bound is about 16x
 * the BF16 one and most rows are rechecked. */
typedef enum { SKM_PREC_FP32 = 0, SKM_PREC_BF16 = 1, SKM_PREC_FP8 = 2 } skm_precision;

/* Input vectors x(1..n) in R^d (Section 2: sparse rows stored as sorted
 * (index, value) pairs; dense rows as plain arrays).
 *   CSR:   row_ptr int64[n+1] (row_ptr[0] = 0, non-decreasing), col_idx
 *          int32[nnz] strictly increasing within each row and in [0, d),
 *          values[nnz] of type dtype.
 *   DENSE: values[n*d] row-major FP32; row_ptr, col_idx unused.  Dense rows
 *          support the standard and Hamerly variants (SKM_EUNSUPPORTED for
 *          Elkan); precision BF16 needs d a multiple of 8 and FP8 a
 *          multiple of 16 (the tensor maps want 16-byte rows; any such d
 *          works: the K loop runs blocks of 128 bytes with the tail read as
 *          zeros).
 * memspace says where all three pointers live. */
typedef struct {
  int64_t n;
  int64_t d;
  int32_t layout;   /* skm_layout */
  int32_t dtype;    /* skm_dtype */
  int32_t memspace; /* skm_memspace */
  int32_t reserved; /* must be 0 */
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const void* values;
} skm_data;

/* Options; skm_default_options fills the defaults. */
typedef struct {
  int32_t hamerly_tight;   /* 0: Eq. eqn:u-hamerly-2 as in the paper (guarded);
                              1: the clamped single-center update with p' */
  int32_t validate;        /* 1 (default): check the CSR structure at init */
  int32_t row_threshold;   /* Elkan: a point with more candidate centers than
                              this (capped at 7) is recomputed as a whole row;
                              0 = min(k/8, 7) */
  int32_t precision;       /* skm_precision, dense rows only (default FP32) */
  int32_t graph;           /* skm_run on CSR data: 1 = after the first iteration,
                              replay one whole iteration (assignment and center
                              update) as a captured CUDA graph and read the
                              changed-label counts back every graph_check
                              iterations; iterations after convergence change
                              nothing.  0 (default): one host sync per iteration */
  int32_t graph_check;     /* 0 = 8 */
  int32_t blocks_per_sm;   /* grid of the persistent bound/recompute kernels:
                              at most this many blocks per SM (0 = as many
                              as are resident at once); skm_autotune sets it */
  int32_t fused_update;    /* 0 (default): the center update's phases after
                              the sums (dirty list, norms, normalisation,
                              drift, objective) run as separate kernels; 1:
                              as one cooperative launch whose blocks wait on
                              one another at bounded grid barriers (a wait
                              that gives up after 1 s makes the next
                              skm_assign return SKM_ETIMEOUT; destroy the
                              context then).  Results are bit-identical. */
  int32_t screen;          /* Elkan and Hamerly variants on CSR data (single
                              runs, k <= 1024):
                              the whole-row recomputes after the first
                              assignment screened against an FP16 copy of the
                              centers (half the bytes gathered; with k = 1000
                              the FP32 center table outgrows L2).  The center
                              update keeps E >= max_j |fp16(c_j) - c_j|; every
                              FP16 similarity is then within eps_i =
                              E + 1.001 delta_i of the exact one, so a row
                              whose best two differ by more than
                              2 (eps_i + delta_i) takes its label from them,
                              and the other rows are recomputed exactly
                              (labels identical either way; the bounds of
                              screened rows are looser by eps_i).
                              0 (default): on for k > 128; 1: on; 2: off. */
  int32_t k_tile;          /* centers per pass of the whole-row kernel (single
                              CSR runs, every variant but Yin-Yang): 0
                              (default) = the smallest of 128, 256, 512, 1024
                              that holds k; else one of those four, and a
                              row is walked once per tile of centers (fewer
                              registers per pass).  Results do not depend on
                              it; skm_autotune chooses it.  Other values, or
                              a nonzero value for a batch or Yin-Yang:
                              SKM_EINVAL / SKM_EUNSUPPORTED. */
  int32_t reserved[2];
} skm_options;

/* Counters of the last assignment and of the run so far. */
typedef struct {
  int64_t iterations;     /* assignments performed since init / reset */
  int64_t last_changed;   /* labels changed by the last assignment */
  int64_t last_sims;      /* exact similarities computed by the last assignment */
  int64_t total_sims;     /* ... summed over all assignments */
  int64_t last_survivors; /* points that failed the first bound test */
  int64_t last_rechecks;  /* points recomputed as a whole row of k similarities
                             (Hamerly: still failing after l was tightened;
                             Elkan: too many candidate centers) */
  double objective;       /* J = sum_j |S_j| after the last center update */
  int64_t last_cand_rechecks; /* precision form: ambiguous rows rechecked in
                                 FP32 against their BF16 candidates only */
  int64_t last_skipped;   /* 1 when the last assignment skipped Elkan's bound
                             pass (nearly every point had gone to a whole row)
                             or Hamerly's tightening (it had pruned almost
                             nothing): the survivors went to whole rows */
} skm_stats;

typedef struct skm_ctx skm_ctx;

void skm_default_options(skm_options* opt);

/* Create a clustering context for data x with k clusters and the given
 * variant.  init_rows (HOST, k distinct row ids in [0,n)) picks the initial
 * centers c(j) = x(init_rows[j]) (Section 6: uniform random rows); NULL draws
 * them from seed.  Prepares everything the iterations need (row norms, the
 * term-major copy of the data, work buffers).  stream: a cudaStream_t.
 * Errors: SKM_EINVAL (k < 1, k > n, malformed CSR, zero or non-finite row,
 * duplicate init rows), SKM_EUNSUPPORTED (Elkan with k > 4096; CSR data
 * whose term-major center table, d x round_up(k, 8) FP32 values, reaches
 * 16 GB), SKM_ENOMEM, SKM_ECUDA.  On error *out is NULL. */
int skm_init(skm_ctx** out, const skm_data* x, int32_t k, int32_t variant,
             const int64_t* init_rows, uint64_t seed, const skm_options* opt,
             void* stream);

/* Restart from new initial rows (HOST, k ids; NULL = draw from seed) without
 * repeating the data preparation. */
int skm_reset(skm_ctx* ctx, const int64_t* init_rows, uint64_t seed);

/* The assignment step (Section 5), pruned per the variant (Sections 5.1-5.4).
 * The first call after init/reset (or after skm_set_centers/labels) computes
 * all n*k similarities and initialises the bounds.  n_changed (HOST, may be
 * NULL): labels changed; non-NULL synchronises the stream. */
int skm_assign(skm_ctx* ctx, int64_t* n_changed);

/* The center update (Section 5): c(j) = normalised member sum; a cluster with
 * a zero sum keeps its center.  Also computes the center drift
 * p(j) = <c(j), c'(j)> (Section 4) and, for Elkan and Hamerly, the
 * center-center bounds cc and s (Section 5.2).  objective (HOST, may be NULL):
 * J = sum_j |S_j|; non-NULL synchronises. */
int skm_update_centers(skm_ctx* ctx, double* objective);

/* Iterate assign + update until an assignment changes no label or max_iters
 * assignments were done.  Outputs (HOST, may be NULL): iterations done and the
 * final objective.  Synchronises. */
int skm_run(skm_ctx* ctx, int32_t max_iters, int32_t* iters_done, double* objective);

/* Copy out the labels a(i) (int32[n]) or the centers (float[k*d], row-major
 * c(j)) to memory in memspace out_space. */
int skm_get_labels(skm_ctx* ctx, int32_t* out, int32_t out_space);
int skm_get_centers(skm_ctx* ctx, float* out, int32_t out_space);

/* Overwrite the centers (float[k*d] row-major, in memspace) or the labels
 * (int32[n], each in [0,k) ).  Invalidates the bounds: the next assignment
 * recomputes everything.  Used to resume from a checkpoint. */
int skm_set_centers(skm_ctx* ctx, const float* C, int32_t space);
int skm_set_labels(skm_ctx* ctx, const int32_t* a, int32_t space);

/* Copy out the bounds for inspection: l (float[n]); u is float[n] for the
 * Hamerly variants, float[n*k] (row-major u(i,j)) for the Elkan variants and
 * float[ceil(k/8)*n] (group-major u(i,G) at [G*n + i]) for Yin-Yang; either
 * pointer may be NULL.  SKM_ESTATE before the first assignment or for
 * the standard variant. */
int skm_get_bounds(skm_ctx* ctx, float* l, float* u, int32_t out_space);

int skm_get_stats(skm_ctx* ctx, skm_stats* out);

/* Diagnostic for the precision form (dense rows, precision BF16 or FP8): the
 * tensor-core result of the last assignment, per row the 8 largest BF16 (FP8)
 * similarities in descending order (vals, float[n*8]) and their centers
 * (idx, int32[n*8]; equal values: lower center first; -1 / -inf past k),
 * and per row the error bound eps (float[n]) that every BF16 similarity of
 * the row to the current centers satisfies against the exact one:
 * eps_i = |xb_i - x_i| (1 + 6u + E_c) + E_c + 1.02 (d + 16) 2^-23, rounded up,
 * with x_i the unit row, xb_i its BF16 copy, E_c = max_j |bf16(c_j) - c_j| and
 * u = 2^-24 (Cauchy-Schwarz on <xb, cb> - <x, c>; at most
 * 2^-7 + 2^-15 + (d + 16) 2^-23, the bound for the worst-case rounding).
 * FP8: the same form with xb_i = e4m3(2^e_i x_i) 2^-e_i, cb_j =
 * e4m3(2^8 c_j) 2^-8 and 1.25 in place of 1.02.
 * Rows the last Hamerly assignment pruned keep older values.  Any pointer may
 * be NULL; vals/idx/eps live in out_space.  SKM_ESTATE for other contexts, and
 * before the first assignment or after skm_set_centers / skm_set_labels. */
int skm_get_bf16_topk(skm_ctx* ctx, float* vals, int32_t* idx, float* eps, int32_t out_space);

/* Batched form: nruns independent clusterings of different row blocks of
 * one CSR matrix (same d) in one context, so that each phase of an iteration
 * is one launch for all runs.  x holds all rows; run r owns rows
 * run_rows[r] .. run_rows[r+1]-1 (host int64[nruns+1], run_rows[0] = 0,
 * run_rows[nruns] = x->n, increasing) and clusters them into ks[r] centers
 * (host int32[nruns], 1 <= ks[r] <= rows of the run, <= 4096).  init_rows:
 * host int64[sum ks], for each run in order ks[r] distinct row indices local
 * to the run, or NULL to draw them from seed (run r uses seed + r).
 * Every variant; Yin-Yang only with ks[r] <= 512 for every run (its group
 * bounds, one per 8 consecutive centers of a run, come from one pass over
 * the run's centers; else SKM_EUNSUPPORTED).  Hamerly's worst drift
 * p' (Section 5.3) is taken per run over the run's own centers, and the full
 * variants keep each run's own center-center bounds cc and s (Section 5.2):
 * the Gram is block-diagonal, one k_r x k_r block per run, whose rows and
 * columns of the centers that moved are recomputed after each update.
 * skm_assign / skm_update_centers / skm_run then advance every run;
 * skm_get_labels returns labels local to each run (in [0, ks[r]));
 * skm_get_centers returns the runs' centers one after the other
 * (float[sum ks * d]); the objective and counters are totals over the runs.
 * skm_set_centers, skm_set_labels and skm_get_bounds return
 * SKM_EUNSUPPORTED for a batch.  Ownership and errors as skm_init. */
int skm_batch_init(skm_ctx** out, const skm_data* x, const int64_t* run_rows, const int32_t* ks, int32_t nruns,
                   int32_t variant, const int64_t* init_rows, uint64_t seed, const skm_options* opt,
                   void* stream);

/* Choose, for this context's shape, by timing `iters` iterations per
 * candidate, after 4 * iters untimed ones from the initial centers (the
 * first iterations recompute nearly every row whatever the setting; results
 * do not depend on the choice):
 * the launch configuration of the persistent bound and recompute kernels
 * (4, 8 or 16 blocks per SM) with the Elkan whole-row threshold (auto, 2,
 * 7); then, for single CSR runs but Yin-Yang, the whole-row kernel's tile of
 * centers (the default one or up to two smaller ones, opt.k_tile); then,
 * where the context keeps FP16 centers (opt.screen), whether the screened
 * whole-row pass is used.  A coordinate search: each stage keeps the best of
 * the previous ones.  The initial state is restored afterwards.  The choice
 * is kept in the text file cache_path (one line per device and shape bucket:
 * key, blocks per SM, threshold, tile, screen off) when cache_path is not
 * NULL, and read from it instead of timing when the bucket is already there
 * (lines with only the first two values are read with the defaults for the
 * others).  *from_cache (may be NULL) tells which happened. */
int skm_autotune(skm_ctx* ctx, const char* cache_path, int32_t iters, int32_t* from_cache);

/* Spherical k-means++ seeding (Section 5.6) of a context's centers: the
 * first center is row floor(u[0] n); center j > 0 is drawn with probability
 * proportional to 1 - max_c <x(i), c> over the centers chosen so far, as
 * follows: q_i = round((1 - m_i) 2^40) (0 if negative), W = sum q_i,
 * T = floor(u[j] W), and the row whose inclusive prefix sum of q first
 * exceeds T is chosen (if W = 0, the first row not chosen yet).  u: host
 * double[k] of uniform draws in [0, 1) supplied by the caller.  The chosen
 * rows become the centers and the context restarts from them as after
 * skm_reset (labels unassigned, bounds dropped); rows_out (host int64[k], may
 * be NULL) receives them.  SKM_EUNSUPPORTED for a batch. */
int skm_seed_kmeanspp(skm_ctx* ctx, const double* u, int64_t* rows_out);

/* skm_seed_kmeanspp followed by the first assignment, which costs no extra
 * pass: the bound pre-initialisation that Section 5.6 remarks on and Section 7
 * names as future work.  The seeding computes every row's similarity to each
 * center it chooses (the last one included) with the assignment kernels'
 * arithmetic, so it keeps per row the best center, the best and second best
 * similarity and, for Elkan, every u(i,j); the labels and bounds are then
 * exactly those skm_assign would leave after skm_seed_kmeanspp (l = s1 - delta
 * rounded down, Hamerly's u = s2 + delta, Elkan's u(i,j) = s_ij + delta
 * rounded up), and the next call is skm_update_centers (skm_run begins with an
 * assignment, so call skm_update_centers before it).  n_changed (host, may
 * be NULL; non-NULL synchronises) receives n, as for a first assignment, and
 * skm_get_stats counts n k similarities for it.  SKM_EUNSUPPORTED for a batch
 * and for Yin-Yang bounds; u and rows_out as skm_seed_kmeanspp. */
int skm_seed_kmeanspp_assign(skm_ctx* ctx, const double* u, int64_t* rows_out, int64_t* n_changed);

/* Self-test of the failure path of every device-side wait: the tensor-core
 * kernel's barrier waits (one warp waits on an mbarrier nothing completes)
 * and the grid barrier of the fused center update (a cooperative launch of
 * two blocks, one of which never arrives), each with the given limit
 * (1 ns .. 2 s).  Returns SKM_ETIMEOUT when both waits gave up as they must
 * (the GPU context stays usable), SKM_OK if one completed (a defect),
 * SKM_ECUDA on a CUDA error. */
int skm_selftest_wait(int64_t timeout_ns, void* stream);

/* Bytes of bound state a variant keeps for n points and k centers (labels
 * excluded): standard 0; Hamerly 8n (two FP32 bounds); Elkan 4n + 4nk;
 * Yin-Yang 4n + 4n ceil(k/8). */
int skm_bound_bytes(int32_t variant, int64_t n, int32_t k, int64_t* bytes);

/* Number of CUDA kernels this library has launched in this process. */
int64_t skm_kernel_launches(void);

/* Per-kernel timing for profiling.  skm_profile(ctx, 1) starts bracketing
 * every kernel the context launches with two CUDA events on its stream (this
 * adds a little launch overhead); skm_profile(ctx, 0) stops; either call
 * drops what was recorded.  skm_profile_read reports kernel number idx (in
 * order of first launch): its name (NUL-terminated, truncated to name_len),
 * the summed event time in ms and the number of launches.  SKM_EINVAL once
 * idx is past the last kernel.  Both synchronise the stream. */
int skm_profile(skm_ctx* ctx, int32_t enable);
int skm_profile_read(skm_ctx* ctx, int32_t idx, char* name, int32_t name_len, double* total_ms,
                     int64_t* launches);

void skm_destroy(skm_ctx* ctx);
const char* skm_strerror(int status);

/* One standard assignment step that allocates no device memory (the paper has
 * no counterpart: this exists for callers that cannot call cudaMalloc, e.g.
 * code running inside another framework's memory pool or under a fixed
 * memory budget, or a service that must not allocate after start-up).
 *   x:        CSR data in DEVICE memory (not checked beyond what the kernel
 *             can see: a row with a column index outside [0,d), a zero norm or
 *             a non-finite value gets label -1, and so does a row whose
 *             similarities are all NaN, e.g. against NaN centers).
 *   centers:  DEVICE float[k*d], row-major unit centers c(j).
 *   labels:   DEVICE int32[n], in: current labels (-1 = none), out: the new
 *             labels a(i) = argmax_j <x(i), c(j)> under the library's tie rule
 *             -- identical to skm_assign of a standard context holding the
 *             same centers and labels.
 *   n_changed: HOST, may be NULL; non-NULL synchronises the stream, returns
 *             the number of changed labels, and makes the call return
 *             SKM_EINVAL if some row got label -1 for the reasons above.
 *             With NULL the call only enqueues its work: malformed rows then
 *             show only as label -1.
 * Scratch lives in a static device array of 16 MiB (plus 16 bytes) that every
 * GPU loading the library holds until exit: d * round_up(k, 8) must not
 * exceed 4,194,304, else SKM_ETOOBIG.  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress); make it before any stream capture.
 * All calls on a device share the array: calls that overlap on the GPU race
 * and must be serialised by the caller. */
int skm_assign_noalloc(const skm_data* x, int32_t k, const float* centers, int32_t* labels,
                       int64_t* n_changed, void* stream);

/* Measured peak arithmetic rate of the current GPU (the paper has no
 * counterpart: measurement support for the roofline fractions this library's
 * benchmark reports).  kind SKM_PEAK_FP32_FMA: FP32 FMA, the roof of the SIMT
 * similarity kernels; SKM_PEAK_FP64_FMA: FP64 FMA; SKM_PEAK_FP32_FMA2: FP32
 * FMA issued as packed pairs (fma.rn.f32x2, two FMAs per instruction, each
 * rounded as one FMA); SKM_PEAK_L2_GATHER: the rate (TB/s of bytes
 * gathered) of warps that gather 416-byte rows (26 lanes x 16 B, the
 * whole-row kernel's center slice at k = 100) at pseudo-random rows of an
 * L2-resident 20.8 MB table, 16 rows in flight per warp.  Runs one warm-up and one
 * timed launch of a kernel of independent FMA chains on every SM (a few to a
 * few tens of ms) on the given stream, synchronises it, and writes the rate
 * in TFLOP/s (2 FLOP per FMA) to *tflops (host).  SKM_EINVAL for another
 * kind or a NULL pointer. */
#define SKM_PEAK_FP32_FMA 0
#define SKM_PEAK_FP64_FMA 1
#define SKM_PEAK_FP32_FMA2 2
#define SKM_PEAK_L2_GATHER 3 /* TB/s, not TFLOP/s: see below */
int skm_measure_peak(int32_t kind, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SKM_H */
