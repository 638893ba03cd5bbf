/*
 * pt_sgemm -- portability-tuned single-precision GEMM for sm_103a (GB300).
 *
 * C ABI of the library libptsgemm.so.  Every call returns an int status
 * (PT_OK = 0, negative on error) and never aborts or prints (unless the
 * environment variable PT_VERBOSE is set).  After a failing call,
 * pt_last_error() gives a message and pt_last_error_arg() the 1-based index
 * of the offending argument (0 when no single argument is at fault); both are
 * per host thread.
 *
 * Operation (the problem statement of "A Few Fit Most: Improving Performance
 * Portability of SGEMM on GPUs using Multi-Versioning", Section V-B, in BLAS
 * form):
 *
 *     C <- alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T
 *
 * Storage is ROW-MAJOR.  op(A) is M x K, op(B) is K x N, C is M x N.
 *   transA 'N': A is M x K, lda >= max(1, K);  'T': A is K x M, lda >= max(1, M)
 *   transB 'N': B is K x N, ldb >= max(1, N);  'T': B is N x K, ldb >= max(1, K)
 *   C: ldc >= max(1, N).
 * beta == 0 means C is not read (NaN/Inf already in C do not propagate).
 * M == 0 or N == 0 returns at once; K == 0 or alpha == 0 sets C <- beta*C.
 *
 * A, B, C are DEVICE pointers owned by the caller; the library never frees
 * or retains them.  Calls on a stream are asynchronous with respect to the
 * host; `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  C must not alias A or B.
 */
#ifndef PT_SGEMM_H
#define PT_SGEMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PT_OK 0
#define PT_EINVAL (-1)        /* invalid argument (see pt_last_error_arg)   */
#define PT_EUNSUPPORTED (-2)  /* variant cannot run this shape/layout      */
#define PT_ECUDA (-3)         /* CUDA runtime or driver error              */
#define PT_EIO (-4)           /* file could not be opened/written          */
#define PT_EFORMAT (-5)       /* malformed table or manifest               */
#define PT_ETIMEOUT (-6)      /* a bounded device wait gave up             */

const char *pt_last_error(void);
int pt_last_error_arg(void);

/* ---- the operation ------------------------------------------------------
 * pt_sgemm: the multi-versioned entry.  The runtime selector (the
 * "classifier" of the paper's Fig. 1, Section III-C) maps the call's
 * (transA, transB, M, N, K) to one variant of the loaded set kappa
 * (pt_load_manifest): an exact shape hit takes the member timed fastest on
 * that shape.  Any other shape goes, in this order, to the manifest's
 * regression tree (PT_SELECT_TREE manifests), else to its time model (one
 * least-squares quadratic in (log2 M, log2 N, log2 K) of ln t per member,
 * corrected by the distance-weighted mean of its residuals at the training
 * shapes, fitted when they share one transpose pair and used only for
 * queries with that pair: the member of least predicted time, ties to the
 * earlier member), else to the pick of the nearest listed shape in
 * (log2 M, log2 N, log2 K), L1 distance, ties to the lower entry.  With no
 * manifest loaded, or when the picked variant cannot run the arguments
 * (alignment, transpose support), the next members of kappa are tried in
 * the order of the manifest and finally the built-in default variant, which
 * runs every valid argument set.
 */
int pt_sgemm(char transA, char transB, int64_t M, int64_t N, int64_t K,
             float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
             float beta, float *C, int64_t ldc, void *stream);

/* Runs variant `id` (0 <= id < pt_num_variants()): one code variant, i.e.
 * one configuration of the kernel's parameters compiled ahead of time
 * (Section III-A).  The tuner, the tests and single-variant callers use it.
 * PT_EUNSUPPORTED when the variant's layout or alignment rules exclude these
 * arguments; nothing is launched then. */
int pt_sgemm_variant(int id, char transA, char transB, int64_t M, int64_t N, int64_t K,
                     float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                     float beta, float *C, int64_t ldc, void *stream);

/* Screening reference kernel (the paper's "reference kernels", Section V-C):
 * one thread per output, compensated FP32 dot product (TwoProduct/TwoSum),
 * independent of the variant family.  Same arguments as pt_sgemm. */
int pt_sgemm_reference(char transA, char transB, int64_t M, int64_t N, int64_t K,
                       float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                       float beta, float *C, int64_t ldc, void *stream);

/* ---- variant registry (a parameter configuration compiled ahead of time;
 * Section III-A terminology, precompilation Section III-B) ---------------- */
#define PT_LOADER_CPASYNC 0   /* cp.async global->shared staging            */
#define PT_LOADER_TMA 1       /* cp.async.bulk.tensor (TMA) + mbarrier       */

/* How a variant's CTAs cover the output (pt_variant_desc_t.schedule). */
#define PT_SCHED_TILE 0        /* one CTA (or split-K cluster) per tile        */
#define PT_SCHED_PERSISTENT 1  /* one CTA per SM walks the tiles               */
#define PT_SCHED_STREAMK 2     /* one CTA per SM; whole tiles for all but the
                                  last full wave, the rest shared in 128-k
                                  chunks with partial tiles handed over       */

typedef struct pt_variant_desc {
    int id;
    int bm, bn, bk;    /* CTA tile M x N and K-step (two-CTA tensor-core
                          versions, names ending in _2sm: bm = 256 is the
                          tile of the CTA pair, 128 rows per CTA)       */
    int wm, wn;        /* warp tile                                          */
    int tm, tn;        /* per-thread register tile                           */
    int kl;            /* k-groups of lanes inside a warp, shuffle-reduced   */
    int vec;           /* floats per direct global load / store (1, 2, 4)    */
    int stages;        /* shared-memory pipeline depth                       */
    int splitk;        /* CTAs of a cluster splitting K, reduced over DSMEM  */
    int loader;        /* PT_LOADER_*                                        */
    int a_kmajor;      /* 1: A tile held K-major (swizzled) in shared memory */
    int threads;       /* threads per CTA                                    */
    int smem_bytes;    /* dynamic shared memory per CTA                      */
    int trans_mask;    /* bit (2*tA + tB) set when (transA, transB) runs;
                          tX = 0 for 'N', 1 for 'T'                          */
    int kind;          /* 0 = FP32 SIMT, 1 = 3xTF32 tensor core (tcgen05),
                          2 = BF16x3 tensor core (tcgen05, six products),
                          3 = scaled 3xF16 tensor core (tcgen05, three FP16
                          products, per-chunk power-of-two scales)         */
    int fma2;          /* 1: packed fma.rn.f32x2 register-tile updates       */
    int schedule;      /* PT_SCHED_*                                         */
    char name[96];     /* stable key used in tables and manifests           */
} pt_variant_desc_t;

int pt_num_variants(void);
int pt_variant_desc(int id, pt_variant_desc_t *out);
/* id of a variant by name, or PT_EINVAL */
int pt_variant_by_name(const char *name);
/* The split-precision tensor-core variants (kind 1, 2, 3) split both operands
 * into low-precision planes in a library workspace (see pt_shutdown) and run
 * tcgen05.mma with TMEM accumulators; they accept every layout and alignment.
 * Exception: fused versions (names with "_fa" / "_fb") split A (or B) inside
 * the GEMM kernel from the caller's matrix, so they need that operand
 * untransposed (trans_mask), 16-byte aligned, with a leading dimension
 * divisible by 4, and return PT_EUNSUPPORTED otherwise.
 * 3xTF32 (Markidis et al.-style split x = hi + lo, three products), BF16x3
 * (x = b0 + b1 + b2, six products) and scaled 3xF16 give FP32-level error.
 * 3xF16 ("tc3xf16_" names) multiplies, per 256 values of k, each row of
 * op(A) and each group of 32 consecutive columns of op(B) by a power of two
 * that brings its largest magnitude there into [2^14, 2^15), splits into two
 * FP16 planes (11-bit significands, as TF32) and undoes the scales on each
 * 256-k partial product: three MMAs at the FP16 rate, error relative to the
 * largest |a| of the row times the largest |b| of the column's group.  It
 * gives that accuracy while those maxima lie in [2^-49, 2^78]; larger values
 * overflow FP16 (C gets Inf or
 * NaN) and smaller ones keep fewer bits.  Names with "_2sm" run a cluster
 * of two CTAs per 256 x 128 or 256 x 256 tile with cta_group::2 MMAs of
 * M = 256 (each CTA loads its 128 rows of A and half of the tile's B; the
 * 256 x 256 ones run stream-K over CTA pairs when the last wave of pair
 * tiles is under 3/4 full, always with "_stk"); names with "n256" compute
 * 128 x 256 or 256 x 256 tiles whose three products accumulate in one
 * tensor-memory accumulator.  The paper has no tensor-core versions; they
 * are further members of the same variant space. */
/* the fixed default variant (128x128x8 CTA tile, cp.async, any layout) */
int pt_default_variant(void);

/* ---- portability tuning ------------------------------------------------ */
typedef struct pt_shape {
    int64_t m, n, k;
    char transA, transB;
} pt_shape_t;

typedef struct pt_tune_opts {
    int warmup;          /* untimed launches per entry (>= 0; default 2)       */
    int reps_min;        /* timed launches per entry, lower bound (default 5)  */
    int reps_max;        /* upper bound (default 50)                           */
    double target_ms;    /* aim for reps * t ~ target (default 5 ms)           */
    uint64_t seed;       /* SplitMix64 seed of the on-device inputs            */
    int resume;          /* 1: keep rows already in the table, skip them       */
    double tol;          /* screening bound on the normalised error (2e-6)     */
    int64_t pool_bytes;  /* rotating input pool; >= 2x L2 keeps L2 cold        */
    int verbose;         /* progress to stderr                                 */
    int64_t fail_launch; /* test hook: the n-th variant launch of this call
                            (1-based; screening and timed launches count)
                            is not made and reports PT_ECUDA; 0 = off      */
} pt_tune_opts_t;

/* Fills *o with the defaults above. */
void pt_tune_default_opts(pt_tune_opts_t *o);

/* Data collection (Section V-D): times every listed variant (ids == NULL:
 * all) on every shape and appends one CSV row per (shape, variant) to
 * table_path, flushing after each row, so the file is the checkpoint.  Each
 * variant is first screened against the reference kernel on the same inputs;
 * a launch error or a normalised error above opts->tol marks the row invalid
 * (status column = the error) and tuning goes on with the next variant; only
 * an error that leaves the CUDA context unusable stops it (PT_ECUDA).
 * Timing: per-launch CUDA events after warmup, inputs rotating through a pool
 * larger than L2; median and mean recorded.  The library allocates and frees
 * its own device buffers on the current device.  Synchronous. */
int pt_tune(const pt_shape_t *shapes, int n_shapes, const int *ids, int n_ids,
            const pt_tune_opts_t *opts, const char *table_path);

#define PT_SELECT_EXACT 0       /* enumerate every k-subset                    */
#define PT_SELECT_GREEDY_SWAP 1 /* greedy growth + 1-swap local search         */
#define PT_SELECT_AUTO 2        /* exact when C(n,k) <= 2e7, else greedy+swap  */
#define PT_SELECT_KMEANS 3      /* k-means on performance vectors (IV-C-2)     */
#define PT_SELECT_TREE 4        /* regression tree with k leaves (IV-C-3)      */

/* PortabilityTune (Section IV-B, cost Eq. 1): choose kappa, |kappa| <= k, of
 * table variants maximising the geometric mean over the training shapes
 * (indices into the table's distinct-shape list, in order of first
 * appearance; n_train == 0 trains on every shape of the table) of
 * t_best(s) / min_{v in kappa} t(v, s), t_best over every
 * valid variant of the table.  Writes the ids to out_ids[0..k) (-1 padded),
 * the training geomean to *out_train_geomean, and, when manifest_path is not
 * NULL, a manifest (kappa, each training shape's fastest member, the tree
 * of PT_SELECT_TREE, and each member's time model when every training shape
 * has the same transpose pair).  `seed`
 * drives the random restarts / initialisation of the heuristic methods.
 * CPU only. */
int pt_select(const char *table_path, const int *train_idx, int n_train, int k,
              int method, uint64_t seed, int *out_ids, double *out_train_geomean,
              const char *manifest_path);

#define PT_SCORE_BEST_OF_SET 0  /* each shape uses kappa's fastest member     */
#define PT_SCORE_SELECTOR 1     /* each shape uses the runtime selector's pick
                                   from the manifest at manifest_path         */

/* Held-out scoring (Section V-E): the geometric mean over the listed shapes
 * (indices into the table's distinct-shape list) of t_best(s) / t(chosen(s), s),
 * the reciprocal of the paper's slowdown over Oracle (S/O), with t_best over
 * every valid variant of the table.  chosen(s) is kappa's fastest member on s
 * (PT_SCORE_BEST_OF_SET, ids[0..k), the paper's measure) or the runtime
 * selector's pick from the manifest (PT_SCORE_SELECTOR; ids unused; where the
 * pick has no valid time, pt_sgemm's fallback order: the other members, then
 * the default variant).  If some listed shape has no valid time left, the
 * geomean is 0.  CPU only. */
int pt_score(const char *table_path, const int *ids, int k, const int *shape_idx,
             int n, int mode, const char *manifest_path, double *out_geomean);

/* Number of distinct shapes in a table and shape i of it. */
int pt_table_shapes(const char *table_path, int *out_n);
int pt_table_shape(const char *table_path, int i, pt_shape_t *out);

/* Installs the multi-versioned set and the classifier that picks from it at
 * run time (Fig. 1, Section III-C) for pt_sgemm (process-wide, mutex-guarded);
 * NULL clears it.  PT_EIO when the file cannot be read, PT_EFORMAT when it
 * is not a manifest of this form (one JSON object; pt_select writes it):
 *   "format": "pt-manifest-1"
 *   "kappa":  [variant names]          the multi-versioned set, in order
 *   "map":    [{"m", "n", "k", "transA", "transB", "variant"}]  (optional)
 *             listed shapes and the member of kappa each one takes
 *   "tree":   [nodes]  (optional; PT_SELECT_TREE) node 0 is the root; an
 *             inner node {"feature": 0|1|2 (log2 M, N, K), "threshold",
 *             "left", "right"} sends feature <= threshold left; children
 *             come after their parent; a leaf is {"variant": name}
 *   "model":  {"transA", "transB", "coef": [10 numbers or null per kappa
 *             member], "points": [[M, N, K]], "resid": [[number or null per
 *             point] or null per member]}  (optional; "points" and "resid"
 *             optional together) predicted ln t = coef . (1, u, v, w, u^2,
 *             v^2, w^2, uv, uw, vw), u = (log2 M - 9) / 3, v and w likewise
 *             for N and K, plus the 1/d^2-weighted mean of the member's
 *             residuals at the points (d: L1 distance in log2 M, N, K; at
 *             d = 0 the mean of the residuals there); used only for shapes
 *             with these transposes
 * "method", "k" and "train_geomean" are informative.  Variant names not in
 * this library are PT_EFORMAT. */
int pt_load_manifest(const char *path);
/* The variant id pt_sgemm would launch for these arguments (same rules). */
int pt_selected_variant(char transA, char transB, int64_t M, int64_t N, int64_t K,
                        const float *A, int64_t lda, const float *B, int64_t ldb,
                        const float *C, int64_t ldc);

/* ---- grouped SGEMM: many independent problems in a few persistent launches ---
 * (The paper tunes single GEMM calls; this batches uneven problems, each
 * with its own variant choice.)  One descriptor per problem; same operation
 * and conventions as pt_sgemm per problem.  `tile` is the problem's tile
 * configuration: 0: 64x64, 1: 128x64, 2: 128x128 SIMT tiles with 16-byte
 * aligned A, B, C and leading dimensions divisible by 4; 3: 64x64 SIMT for
 * any alignment; 4 (PT_GROUPED_TILE_TC): 128x128 scaled 3xF16 tensor-core
 * tile, any alignment, K > 0.  pt_grouped_plan fills it from the runtime
 * selector. */
typedef struct pt_gemm_problem {
    int64_t m, n, k;
    const float *A;
    int64_t lda;
    const float *B;
    int64_t ldb;
    float *C;
    int64_t ldc;
    float alpha, beta;
    char transA, transB;
    int16_t reserved;
    int32_t tile;
} pt_gemm_problem_t;

#define PT_GROUPED_MAX 4096  /* problems per pt_sgemm_grouped call */
#define PT_GROUPED_TILE_TC 4 /* tile value: 128 x 128 scaled 3xF16 tensor-core tile */

/* Sets problems[i].tile for every problem (host array): the variant the
 * loaded manifest's selector picks for that shape (see pt_sgemm) mapped to
 * the grouped tile of the nearest area, or to PT_GROUPED_TILE_TC when the
 * pick is a tensor-core version and K > 0; 3 when the problem's operands are
 * not 16-byte aligned. */
int pt_grouped_plan(pt_gemm_problem_t *problems, int count);

/* Runs `count` problems: the SIMT tiles in one launch of a persistent kernel
 * (a grid of resident CTAs walking all their tiles); problems with the
 * tensor-core tile through a plan kernel, one split kernel and one
 * persistent tensor-core kernel, whose planes live in the stream's library
 * workspace (see pt_shutdown; it grows only outside stream capture, so make
 * a first call on the stream before capturing one).  `problems` (host) is
 * validated; `problems_dev` must be a device copy of the same array,
 * caller-owned, left unchanged until the launches have completed (for a
 * captured graph: while it is replayed).  Asynchronous on `stream`. */
int pt_sgemm_grouped(const pt_gemm_problem_t *problems, const pt_gemm_problem_t *problems_dev, int count,
                     void *stream);

/* Frees the library's device workspaces (one buffer per device and stream
 * for the tensor-core variants: stream-K flags and partial tiles, then the
 * split planes; grown on first use of a larger shape; growing is refused with
 * PT_EUNSUPPORTED while the stream is being captured, and pt_sgemm then falls
 * back to another variant) and unloads the manifest.  Synchronises the
 * devices that hold a workspace.  Calls made afterwards allocate afresh. */
int pt_shutdown(void);

/* Allocation-free SGEMM (the paper has no counterpart; this is a library
 * convenience).  For callers that cannot allocate device memory during their
 * GEMM calls: programs whose device memory is handed to their own pool
 * allocator at start-up and which forbid raw cudaMalloc, latency-critical
 * loops in which an allocation (that may synchronise the device) is not
 * acceptable, and hosts that only run with memory reserved in advance.
 * Same operation and arguments as pt_sgemm; it always runs the 3xTF32
 * tensor-core kernel of the registry's tc3xtf32_m128n128_p3 (128 x 128
 * tiles, one CTA per SM) and gives the same bits, with the split planes in a
 * fixed array of PT_NOALLOC_SCRATCH_BYTES bytes of device memory that belongs
 * to the library image.  It calls no cudaMalloc, cudaFree or allocating
 * routine.
 * Limit: 2 * (M + N) * round_up(K, 8) * 4 bytes (plus up to 1 KiB of
 * alignment) must not exceed PT_NOALLOC_SCRATCH_BYTES, else PT_EINVAL and
 * nothing is launched.
 * First call on a device (that device current): under CUDA's default lazy
 * module loading it loads the library module that holds the array, which
 * commits the PT_NOALLOC_SCRATCH_BYTES of device memory at that moment (with
 * CUDA_MODULE_LOADING=EAGER this already happened when the context was
 * created); it also looks up the array's device address and sets the
 * kernel's shared-memory attribute.  Make that first call (any small shape)
 * at start-up, before a pool allocator takes the device's free memory and
 * before any stream capture; it returns PT_ECUDA if the memory is not free.
 * Later calls on the device allocate nothing.
 * Every call shares the one array and leaves its planes there: calls whose
 * kernels overlap on the GPU (e.g. on two streams without ordering between
 * them) race on it and give wrong results.  A bounded device wait that gives
 * up leaves C unwritten and is reported by pt_device_status. */
#define PT_NOALLOC_SCRATCH_BYTES (64u << 20)
int pt_sgemm_3xtf32_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K,
                            float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                            float beta, float *C, int64_t ldc, void *stream);

/* Device-side error word set by kernels whose bounded waits gave up
 * (PT_ETIMEOUT) on the current device; reading clears it.  Synchronises the
 * device. */
int pt_device_status(void);

/* Failure-path hook for the stream-K versions (a testing aid; the paper has
 * no counterpart).  In a stream-K launch, the CTA that finishes a tile shared
 * by several CTAs waits, with a time limit, for flags the others set when
 * their partial tiles are written; a wait that runs out skips that tile's
 * stores, sets the device error word (pt_device_status then returns
 * PT_ETIMEOUT) and lets the kernel end normally.  This call sets, for the
 * launches made after it in the process: the limit of that wait (limit_ns;
 * 0 restores the default of 2 s, larger values are PT_EINVAL), and, with
 * never_ready = 1, a flag value that no CTA writes, so every such wait runs
 * out.  never_ready = 0 and limit_ns = 0 restore normal operation.  Only
 * that inter-CTA wait is affected; the pipeline's own waits keep 2 s. */
int pt_debug_streamk_wait(uint64_t limit_ns, int never_ready);

/* Stream-K work partition (a testing aid; the paper has no counterpart): the
 * segments that scheduling unit `unit` (a CTA, or a CTA pair in pair
 * versions) of `units` processes when `tiles` output tiles of `nchunks`
 * k-chunks each are shared stream-K style, computed by the same code the
 * kernels run.  Each segment is three ints in `out` (host memory, caller
 * owned): tile index, first chunk, end chunk (exclusive), in the order the
 * unit visits them.  A unit first takes whole tiles unit, unit + units, ...
 * for all but the last full wave of tiles, then an equal contiguous range of
 * the remaining tiles x chunks, visited from its last tile to its first.
 * Returns the number of segments (only the first `cap` are written), or
 * PT_EINVAL for tiles, nchunks < 1, units outside [1, 2048], unit outside
 * [0, units), cap < 0 or out == NULL with cap > 0.  No device work. */
int pt_debug_streamk_segments(int tiles, int nchunks, int units, int unit, int *out, int cap);

/* Kernel timer (a measurement aid; the paper has no counterpart).  While it
 * runs on the calling host thread, every pt_sgemm / pt_sgemm_variant call
 * records a pair of CUDA events on its stream directly around its main GEMM
 * kernel, so that the time excludes the tensor-core versions' split kernel
 * and any host work.  Calls made while their stream is being captured record
 * nothing.  pt_kernel_timer_stop waits for the recorded events, returns the
 * summed duration in milliseconds and the number of timed launches (either
 * pointer may be NULL), and ends timing.  Starting an already running timer
 * discards what it holds.  PT_ECUDA if an event cannot be created, recorded
 * or read. */
int pt_kernel_timer_start(void);
int pt_kernel_timer_stop(double *total_ms, int *launches);

#ifdef __cplusplus
}
#endif

#endif /* PT_SGEMM_H */
