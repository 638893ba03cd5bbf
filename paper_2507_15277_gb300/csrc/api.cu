// Public SGEMM entry points, argument checking, runtime variant selection,
// the screening reference kernel and library-wide error reporting.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>

#include "common.h"
#include "launch.cuh"

namespace pt {

void free_workspaces();  // tc.cu

// ---- errors ---------------------------------------------------------------------
static thread_local char g_msg[512];
static thread_local int g_arg = 0;

bool verbose() {
    static const bool v = std::getenv("PT_VERBOSE") != nullptr;
    return v;
}

int set_error(int code, int arg, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    g_arg = arg;
    if (verbose()) std::fprintf(stderr, "[pt_sgemm] %d: %s\n", code, g_msg);
    return code;
}

void clear_error() {
    g_msg[0] = 0;
    g_arg = 0;
}

// ---- kernel timer -----------------------------------------------------------------
// Event pairs of the current host thread; the events are created on first use
// and kept for the life of the thread (destroying them at thread exit could
// run after the CUDA runtime has shut down).
struct KernelTimer {
    bool on = false, failed = false;
    int used = 0;
    std::vector<cudaEvent_t> ev;
};

KernelTimer &kernel_timer() {
    static thread_local KernelTimer t;
    return t;
}

void kernel_timer_mark(cudaStream_t st, bool begin) {
    KernelTimer &t = kernel_timer();
    if (!t.on || t.failed) return;
    // An unmatched begin (launch refused after it) is overwritten by the next one.
    if (begin && (t.used & 1)) --t.used;
    if (!begin && !(t.used & 1)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        if (!begin) --t.used;
        return;
    }
    if (t.used == (int)t.ev.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            t.failed = true;
            return;
        }
        t.ev.push_back(e);
    }
    if (cudaEventRecord(t.ev[t.used], st) != cudaSuccess) {
        t.failed = true;
        return;
    }
    ++t.used;
}

// ---- driver entry point and device helpers --------------------------------------
EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

// Error word written by kernels whose bounded waits gave up (one per device).
__device__ int g_err_word;

int *err_word(int dev) {
    static std::atomic<int *> ptrs[64];
    if (dev < 0 || dev >= 64) return nullptr;
    int *p = ptrs[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        if (cudaGetSymbolAddress(&q, g_err_word) != cudaSuccess) return nullptr;
        p = static_cast<int *>(q);
        ptrs[dev].store(p, std::memory_order_release);
    }
    return p;
}

// Stream-K finisher wait (pt_debug_streamk_wait): limit and awaited-value offset.
static std::atomic<uint64_t> g_sk_wait_ns{kWaitLimitNs};
static std::atomic<unsigned> g_sk_wait_bias{0};

void streamk_wait_settings(uint64_t *limit_ns, unsigned *bias) {
    *limit_ns = g_sk_wait_ns.load(std::memory_order_relaxed);
    *bias = g_sk_wait_bias.load(std::memory_order_relaxed);
}

// ---- small kernels -------------------------------------------------------------
__global__ void scale_kernel(float *C, int64_t ldc, int M, int N, float beta) {
    const int64_t total = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / N, c = i % N;
        float *p = C + r * ldc + c;
        *p = (beta == 0.f) ? 0.f : beta * *p;
    }
}

// Reference GEMM: one thread per output, compensated dot product in FP32
// (TwoProduct by FMA and TwoSum; Ogita, Rump and Oishi, "Accurate sum and dot
// product", SISC 2005).  The _rn intrinsics keep the compiler from
// contracting the error-free transformations.
__global__ void reference_kernel(GemmArgs a) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = blockIdx.y * blockDim.y + threadIdx.y;
    if (row >= a.M || col >= a.N) return;
    float s = 0.f, c = 0.f;
    for (int k = 0; k < a.K; ++k) {
        const float x = a.ta ? a.A[(int64_t)k * a.lda + row] : a.A[(int64_t)row * a.lda + k];
        const float y = a.tb ? a.B[(int64_t)col * a.ldb + k] : a.B[(int64_t)k * a.ldb + col];
        const float p = __fmul_rn(x, y);
        const float ep = fmaf(x, y, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fsub_rn(t, s);
        const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(ep, es));
    }
    const float r = __fadd_rn(s, c);
    float *out = a.C + (int64_t)row * a.ldc + col;
    *out = (a.beta != 0.f) ? __fadd_rn(__fmul_rn(a.alpha, r), __fmul_rn(a.beta, *out)) : __fmul_rn(a.alpha, r);
}

// ---- argument checking -------------------------------------------------------------
static int trans_flag(char t, int arg, int *out) {
    switch (t) {
        case 'N': case 'n': *out = 0; return PT_OK;
        case 'T': case 't': case 'C': case 'c': *out = 1; return PT_OK;
        default: return set_error(PT_EINVAL, arg, "trans must be 'N' or 'T' (got %d)", (int)t);
    }
}

enum Quick { kRun = 0, kNothing = 1, kScale = 2 };

// Argument indices are those of pt_sgemm (1-based).
static int check_args(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha, const float *A,
                      int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc, GemmArgs *g,
                      int *quick) {
    int ta, tb, rc;
    if ((rc = trans_flag(transA, 1, &ta)) != PT_OK) return rc;
    if ((rc = trans_flag(transB, 2, &tb)) != PT_OK) return rc;
    const int64_t lim = 0x7fffffff;
    if (M < 0 || M > lim) return set_error(PT_EINVAL, 3, "M out of range");
    if (N < 0 || N > lim) return set_error(PT_EINVAL, 4, "N out of range");
    if (K < 0 || K > lim) return set_error(PT_EINVAL, 5, "K out of range");
    const int64_t need_a = ta ? M : K, need_b = tb ? K : N;
    if (lda < (need_a > 1 ? need_a : 1)) return set_error(PT_EINVAL, 8, "lda too small");
    if (ldb < (need_b > 1 ? need_b : 1)) return set_error(PT_EINVAL, 10, "ldb too small");
    if (ldc < (N > 1 ? N : 1)) return set_error(PT_EINVAL, 13, "ldc too small");
    if (std::isnan(alpha)) return set_error(PT_EINVAL, 6, "alpha is NaN");
    if (M == 0 || N == 0) {
        *quick = kNothing;
        return PT_OK;
    }
    if (!C) return set_error(PT_EINVAL, 12, "C is NULL");
    *quick = (K == 0 || alpha == 0.f) ? kScale : kRun;
    if (*quick == kRun) {
        if (!A) return set_error(PT_EINVAL, 7, "A is NULL");
        if (!B) return set_error(PT_EINVAL, 9, "B is NULL");
    }
    g->A = A; g->B = B; g->C = C;
    g->lda = lda; g->ldb = ldb; g->ldc = ldc;
    g->M = (int)M; g->N = (int)N; g->K = (int)K;
    g->alpha = alpha; g->beta = beta;
    g->ta = ta; g->tb = tb;
    g->err = err_word(current_device());
    return PT_OK;
}

static int run_scale(const GemmArgs &g, cudaStream_t st) {
    if (g.beta == 1.f) return PT_OK;
    const int64_t total = (int64_t)g.M * g.N;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    scale_kernel<<<(unsigned)blocks, 256, 0, st>>>(g.C, g.ldc, g.M, g.N, g.beta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : set_error(PT_ECUDA, 0, "scale kernel: %s", cudaGetErrorString(e));
}

// ---- installed manifest -----------------------------------------------------------
static std::mutex g_manifest_mu;
static std::shared_ptr<const Manifest> g_manifest;

bool installed_manifest(Manifest *out) {
    std::lock_guard<std::mutex> lk(g_manifest_mu);
    if (!g_manifest) return false;
    *out = *g_manifest;
    return true;
}

static std::shared_ptr<const Manifest> current_manifest() {
    std::lock_guard<std::mutex> lk(g_manifest_mu);
    return g_manifest;
}

// Picks the variant pt_sgemm launches: the selector's pick, then the other
// members of kappa in manifest order, then the default variant.  Returns the
// id (>= 0) or an error status.
static int choose(const GemmArgs &g, cudaStream_t st) {
    const VariantEntry *tab = variant_table();
    std::shared_ptr<const Manifest> m = current_manifest();
    if (m && !m->kappa.empty()) {
        pt_shape_t s;
        s.m = g.M; s.n = g.N; s.k = g.K;
        s.transA = g.ta ? 'T' : 'N';
        s.transB = g.tb ? 'T' : 'N';
        const int pick = manifest_pick(*m, s);
        if (pick >= 0 && tab[pick].launch(g, st, true) == PT_OK) return pick;
        for (int id : m->kappa)
            if (id != pick && tab[id].launch(g, st, true) == PT_OK) return id;
    }
    const int rc = tab[0].launch(g, st, true);
    return rc == PT_OK ? 0 : rc;
}

}  // namespace pt

using namespace pt;

extern "C" {

const char *pt_last_error(void) { return g_msg; }
int pt_last_error_arg(void) { return g_arg; }

int pt_num_variants(void) { return variant_table_size(); }

int pt_variant_desc(int id, pt_variant_desc_t *out) {
    if (id < 0 || id >= variant_table_size()) return set_error(PT_EINVAL, 1, "variant id %d out of range", id);
    if (!out) return set_error(PT_EINVAL, 2, "out is NULL");
    *out = variant_table()[id].desc;
    return PT_OK;
}

int pt_variant_by_name(const char *name) {
    if (!name) return set_error(PT_EINVAL, 1, "name is NULL");
    const VariantEntry *t = variant_table();
    for (int i = 0; i < variant_table_size(); ++i)
        if (std::strcmp(t[i].desc.name, name) == 0) return i;
    return set_error(PT_EINVAL, 1, "unknown variant '%s'", name);
}

int pt_default_variant(void) { return 0; }

int pt_sgemm_variant(int id, char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha, const float *A,
                     int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc, void *stream) {
    clear_error();
    if (id < 0 || id >= variant_table_size()) return set_error(PT_EINVAL, 0, "variant id %d out of range", id);
    GemmArgs g;
    int quick = kRun;
    int rc = check_args(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, &g, &quick);
    if (rc != PT_OK || quick == kNothing) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (quick == kScale) return run_scale(g, st);
    return variant_table()[id].launch(g, st, false);
}

int pt_sgemm(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha, const float *A, int64_t lda,
             const float *B, int64_t ldb, float beta, float *C, int64_t ldc, void *stream) {
    clear_error();
    GemmArgs g;
    int quick = kRun;
    int rc = check_args(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, &g, &quick);
    if (rc != PT_OK || quick == kNothing) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (quick == kScale) return run_scale(g, st);
    const int id = choose(g, st);
    if (id < 0) return id;
    return variant_table()[id].launch(g, st, false);
}

int pt_selected_variant(char transA, char transB, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda,
                        const float *B, int64_t ldb, const float *C, int64_t ldc) {
    clear_error();
    GemmArgs g;
    int quick = kRun;
    const float one = 1.f;
    (void)one;
    int rc = check_args(transA, transB, M, N, K > 0 ? K : 1, 1.f, A ? A : reinterpret_cast<const float *>(16),
                        lda, B ? B : reinterpret_cast<const float *>(16), ldb, 0.f,
                        const_cast<float *>(C ? C : reinterpret_cast<const float *>(16)), ldc, &g, &quick);
    if (rc != PT_OK) return rc;
    if (quick == kNothing) return set_error(PT_EINVAL, 3, "empty output");
    return choose(g, nullptr);
}

int pt_sgemm_reference(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha, const float *A,
                       int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc, void *stream) {
    clear_error();
    GemmArgs g;
    int quick = kRun;
    int rc = check_args(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, &g, &quick);
    if (rc != PT_OK || quick == kNothing) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (quick == kScale) return run_scale(g, st);
    dim3 block(16, 16);
    dim3 grid((unsigned)((N + 15) / 16), (unsigned)((M + 15) / 16));
    if (grid.y > 65535) return set_error(PT_EUNSUPPORTED, 3, "M too large for the reference kernel");
    reference_kernel<<<grid, block, 0, st>>>(g);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : set_error(PT_ECUDA, 0, "reference kernel: %s", cudaGetErrorString(e));
}

int pt_debug_streamk_wait(uint64_t limit_ns, int never_ready) {
    clear_error();
    if (limit_ns > kWaitLimitNs) return set_error(PT_EINVAL, 1, "limit above the default %llu ns",
                                                  (unsigned long long)kWaitLimitNs);
    if (never_ready != 0 && never_ready != 1) return set_error(PT_EINVAL, 2, "never_ready must be 0 or 1");
    g_sk_wait_ns.store(limit_ns ? limit_ns : kWaitLimitNs, std::memory_order_relaxed);
    g_sk_wait_bias.store((unsigned)never_ready, std::memory_order_relaxed);
    return PT_OK;
}

int pt_debug_streamk_segments(int tiles, int nchunks, int units, int unit, int *out, int cap) {
    clear_error();
    if (tiles < 1) return set_error(PT_EINVAL, 1, "tiles must be at least 1");
    if (nchunks < 1) return set_error(PT_EINVAL, 2, "nchunks must be at least 1");
    constexpr int kMaxUnits = 2048;  // the stream-K header's flag slots (kSkMaxGrid in tc.cuh)
    if (units < 1 || units > kMaxUnits) return set_error(PT_EINVAL, 3, "units must be in [1, %d]", kMaxUnits);
    if (unit < 0 || unit >= units) return set_error(PT_EINVAL, 4, "unit must be in [0, units)");
    if (cap < 0 || (cap > 0 && out == nullptr)) return set_error(PT_EINVAL, 6, "out must hold cap triples");
    if ((int64_t)tiles * nchunks > 0x7fffffffLL) return set_error(PT_EINVAL, 2, "tiles x nchunks too large");
    return streamk_segments(tiles, nchunks, units, unit, out, cap);
}

int pt_kernel_timer_start(void) {
    clear_error();
    KernelTimer &t = kernel_timer();
    t.used = 0;
    t.failed = false;
    t.on = true;
    return PT_OK;
}

int pt_kernel_timer_stop(double *total_ms, int *launches) {
    clear_error();
    KernelTimer &t = kernel_timer();
    t.on = false;
    double sum = 0;
    int n = 0;
    bool bad = t.failed;
    for (int i = 0; i + 1 < t.used && !bad; i += 2) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.ev[i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]) != cudaSuccess) {
            bad = true;
            break;
        }
        sum += ms;
        ++n;
    }
    t.used = 0;
    if (bad) {
        cudaGetLastError();
        return set_error(PT_ECUDA, 0, "kernel timer: an event could not be created, recorded or read");
    }
    if (total_ms) *total_ms = sum;
    if (launches) *launches = n;
    return PT_OK;
}

int pt_device_status(void) {
    clear_error();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "device: %s", cudaGetErrorString(e));
    int v = 0;
    e = cudaMemcpyFromSymbol(&v, g_err_word, sizeof(int));
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "error word: %s", cudaGetErrorString(e));
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_err_word, &zero, sizeof(int));
        return set_error(PT_ETIMEOUT, 0, "a bounded device wait gave up (word %d)", v);
    }
    return PT_OK;
}

int pt_shutdown(void) {
    clear_error();
    free_workspaces();
    std::lock_guard<std::mutex> lk(g_manifest_mu);
    g_manifest.reset();
    return PT_OK;
}

int pt_load_manifest(const char *path) {
    clear_error();
    if (!path) {
        std::lock_guard<std::mutex> lk(g_manifest_mu);
        g_manifest.reset();
        return PT_OK;
    }
    auto m = std::make_shared<Manifest>();
    int rc = read_manifest(path, m.get());
    if (rc != PT_OK) return rc;
    std::lock_guard<std::mutex> lk(g_manifest_mu);
    g_manifest = m;
    return PT_OK;
}

}  // extern "C"
