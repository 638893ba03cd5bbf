// Allocation-free 3xTF32 SGEMM entry point.
//
// Some callers cannot allocate device memory while they run GEMMs: code that
// hands all device memory to its own pool allocator at start-up and forbids
// raw cudaMalloc, latency-bound loops where an allocation (which may
// synchronise the device) is unacceptable, and embedded or real-time hosts
// that only run with memory reserved up front.  pt_sgemm's tensor-core
// variants allocate their split-plane workspace on first use, so they are
// closed to such callers.  This entry point runs the same 3xTF32 kernel with
// its split planes in a fixed array of device memory that is part of the
// library image, so a call allocates nothing.
#include <atomic>
#include <cmath>
#include <cstring>

#include "common.h"
#include "launch.cuh"
#include "tc.cuh"

// Scratch for the split planes of both operands.  Every GPU on which this
// file's module is loaded holds these PT_NOALLOC_SCRATCH_BYTES bytes until the
// process exits.  With CUDA's default lazy module loading that happens at the
// first call on the device (the cudaGetSymbolAddress below loads the module);
// with CUDA_MODULE_LOADING=EAGER, when the context is created.  In host code
// this name is only a stand-in for the device array: its device address comes
// from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char pt_noalloc_scratch[PT_NOALLOC_SCRATCH_BYTES];

namespace pt {
namespace {

using NoAllocCfg = Tc<kTcTf32, 128, 3>;

std::atomic<unsigned char *> g_scratch_addr[64];
std::atomic<int> g_sms[64];
std::atomic<uint64_t> g_attr_done{0};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) on the first call; the same call
// caches the device's SM count (the persistent grid's size).
int scratch_address(int dev, unsigned char **out, int *sms) {
    if (dev < 0 || dev >= 64) return set_error(PT_EUNSUPPORTED, 0, "device ordinal %d out of range", dev);
    unsigned char *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_sms[dev].store(n, std::memory_order_relaxed);
        void *q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&q, pt_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(PT_ECUDA, 0,
                             "cudaGetSymbolAddress of the %u-byte scratch array (loading its module commits that "
                             "device memory; is it free?): %s",
                             (unsigned)PT_NOALLOC_SCRATCH_BYTES, cudaGetErrorString(e));
        }
        p = static_cast<unsigned char *>(q);
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    *sms = g_sms[dev].load(std::memory_order_relaxed);
    return PT_OK;
}

__global__ void noalloc_scale_kernel(float *C, int64_t ldc, int M, int N, float beta) {
    const int64_t total = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        float *p = C + (i / N) * ldc + (i % N);
        *p = (beta == 0.f) ? 0.f : beta * *p;
    }
}

int map_3d(CUtensorMap *map, const void *base, int64_t inner, int64_t rows, int64_t pitch_bytes,
           int64_t plane_bytes, int box_rows) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, 2};
    cuuint64_t strides[2] = {(cuuint64_t)pitch_bytes, (cuuint64_t)plane_bytes};
    cuuint32_t box[3] = {(cuuint32_t)NoAllocCfg::BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PT_OK;
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" int pt_sgemm_3xtf32_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha,
                                       const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
                                       float *C, int64_t ldc, void *stream) {
    clear_error();
    int ta, tb;
    if (transA == 'N' || transA == 'n') ta = 0;
    else if (transA == 'T' || transA == 't' || transA == 'C' || transA == 'c') ta = 1;
    else return set_error(PT_EINVAL, 1, "transA must be 'N' or 'T'");
    if (transB == 'N' || transB == 'n') tb = 0;
    else if (transB == 'T' || transB == 't' || transB == 'C' || transB == 'c') tb = 1;
    else return set_error(PT_EINVAL, 2, "transB must be 'N' or 'T'");
    const int64_t lim = 0x7fffffff;
    if (M < 0 || M > lim) return set_error(PT_EINVAL, 3, "M out of range");
    if (N < 0 || N > lim) return set_error(PT_EINVAL, 4, "N out of range");
    if (K < 0 || K > lim) return set_error(PT_EINVAL, 5, "K out of range");
    const int64_t need_a = ta ? M : K, need_b = tb ? K : N;
    if (lda < (need_a > 1 ? need_a : 1)) return set_error(PT_EINVAL, 8, "lda too small");
    if (ldb < (need_b > 1 ? need_b : 1)) return set_error(PT_EINVAL, 10, "ldb too small");
    if (ldc < (N > 1 ? N : 1)) return set_error(PT_EINVAL, 13, "ldc too small");
    if (std::isnan(alpha)) return set_error(PT_EINVAL, 6, "alpha is NaN");
    if (M == 0 || N == 0) return PT_OK;
    if (!C) return set_error(PT_EINVAL, 12, "C is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (K == 0 || alpha == 0.f) {
        if (beta == 1.f) return PT_OK;
        const int64_t total = M * N;
        const unsigned blocks = (unsigned)(total / 256 + 1 > 65536 ? 65536 : total / 256 + 1);
        noalloc_scale_kernel<<<blocks, 256, 0, st>>>(C, ldc, (int)M, (int)N, beta);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? PT_OK : set_error(PT_ECUDA, 0, "scale kernel: %s", cudaGetErrorString(e));
    }
    if (!A) return set_error(PT_EINVAL, 7, "A is NULL");
    if (!B) return set_error(PT_EINVAL, 9, "B is NULL");
    if ((M + NoAllocCfg::BM - 1) / NoAllocCfg::BM > 65535 || (M + 31) / 32 > 65535 || (N + 31) / 32 > 65535)
        return set_error(PT_EUNSUPPORTED, 3, "shape too large for the grid");

    // Two TF32 planes (hi, lo) of op(A) (M rows) and of op(B)^T (N rows), K-major,
    // row pitch rounded up to 8 floats, each plane 256-byte aligned.
    const int64_t pitch = (K + 7) / 8 * 8;
    const int64_t a_plane = align256(M * pitch * 4);
    const int64_t b_plane = align256(N * pitch * 4);
    const int64_t need = 2 * (a_plane + b_plane);
    if (need > (int64_t)PT_NOALLOC_SCRATCH_BYTES)
        return set_error(PT_EINVAL, 0,
                         "M=%lld N=%lld K=%lld needs %lld bytes of scratch (2 planes x (M + N) x round_up(K, 8) x 4 "
                         "bytes); the allocation-free entry point has %lld",
                         (long long)M, (long long)N, (long long)K, (long long)need,
                         (long long)PT_NOALLOC_SCRATCH_BYTES);

    const int dev = current_device();
    unsigned char *ws = nullptr;
    int sms = 1;
    int rc = scratch_address(dev, &ws, &sms);
    if (rc != PT_OK) return rc;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(g_attr_done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(tc_sgemm_kernel<NoAllocCfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             NoAllocCfg::SMEM_BYTES);
        if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        g_attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }

    // The split kernel overwrites every plane element that the GEMM reads
    // (rows x K; the pitch padding is outside the tensor maps), so nothing
    // left in the array by an earlier call is used.
    unsigned char *wA = ws;
    unsigned char *wB = ws + 2 * a_plane;
    const int va = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0) ? 1 : 0;
    const int vb = (reinterpret_cast<uintptr_t>(B) % 16 == 0 && ldb % 4 == 0) ? 1 : 0;
    // One launch splits both operands (grid rows: A's blocks, then B's; the
    // scratch limit keeps (M + N) / 32 far below the 65535 grid limit).
    const SplitOperand oa{A, lda, ta, (int)M, wA, a_plane, va};
    const SplitOperand ob{B, ldb, tb ? 0 : 1, (int)N, wB, b_plane, vb};
    const int ya = (int)((M + 31) / 32), yb = (int)((N + 31) / 32);
    const dim3 sgrid((unsigned)((pitch + SPLIT_K_PER_BLOCK - 1) / SPLIT_K_PER_BLOCK), (unsigned)(ya + yb));
    // Both kernels are launched with programmatic stream serialization, as the
    // registry's versions are: each waits (griddepcontrol.wait) for the
    // previous kernel of the stream before touching global memory, and its
    // launch and prologue overlap that kernel's tail.
    cudaLaunchAttribute pdl[1];
    unsigned npdl = 0;
    add_pdl_attr(pdl, npdl);
    cudaLaunchConfig_t scfg;
    std::memset(&scfg, 0, sizeof(scfg));
    scfg.gridDim = sgrid;
    scfg.blockDim = dim3(256, 1, 1);
    scfg.stream = st;
    scfg.attrs = pdl;
    scfg.numAttrs = npdl;
    cudaError_t e = cudaLaunchKernelEx(&scfg, tc_split_kernel<kTcTf32>, oa, ob, (int)K, pitch, ya);
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "split kernel: %s", cudaGetErrorString(e));

    CUtensorMap mA, mB;
    rc = map_3d(&mA, wA, K, M, pitch * 4, a_plane, NoAllocCfg::BM);
    if (rc != PT_OK) return rc;
    rc = map_3d(&mB, wB, K, N, pitch * 4, b_plane, NoAllocCfg::BN);
    if (rc != PT_OK) return rc;

    TcArgs t;
    t.C = C;
    t.ldc = ldc;
    t.M = (int)M;
    t.N = (int)N;
    t.K = (int)K;
    t.alpha = alpha;
    t.beta = beta;
    t.vec4 = (reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0) ? 1 : 0;
    t.tma_c = 0;  // the epilogue warps store C themselves (same values as through the TMA engine)
    t.err = err_word(dev);  // a file-scope device word as well: no allocation
    t.sk_words = nullptr;  // no stream-K in this entry point
    t.sk_partials = nullptr;
    t.sk_wait_ns = kWaitLimitNs;
    t.sk_wait_bias = 0;
    t.scale_a = nullptr;  // 3xTF32: no scales
    t.scale_b = nullptr;
    t.ld_sa = t.ld_sb = 0;
    // Persistent grid: one CTA per SM walks the tiles (as the registry's
    // tc3xtf32_m128n128_p3 does), so a CTA's producer runs ahead into its
    // next tile while the epilogue drains the previous one.
    const int64_t tiles = ((N + NoAllocCfg::BN - 1) / NoAllocCfg::BN) * ((M + NoAllocCfg::BM - 1) / NoAllocCfg::BM);
    const dim3 grid((unsigned)(tiles < sms ? tiles : sms));
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NoAllocCfg::THREADS, 1, 1);
    cfg.dynamicSmemBytes = NoAllocCfg::SMEM_BYTES;
    cfg.stream = st;
    cfg.attrs = pdl;
    cfg.numAttrs = npdl;
    e = cudaLaunchKernelEx(&cfg, tc_sgemm_kernel<NoAllocCfg>, t, mA, mB, mA);  // (no C map: tma_c = 0)
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "tensor-core kernel: %s", cudaGetErrorString(e));
    return PT_OK;
}
