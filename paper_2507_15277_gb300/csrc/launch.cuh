// Host-side launch of one SIMT variant: layout/alignment admission, TMA
// descriptors, cluster launch.
#pragma once

#include <atomic>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_runtime.h>

#include "pt_sgemm.h"
#include "simt.cuh"

namespace pt {

// Error reporting shared by the library's translation units (api.cu).
int set_error(int code, int arg, const char *fmt, ...);
void clear_error();

// cuTensorMapEncodeTiled from the driver, resolved once (no libcuda link).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

// Current device ordinal (cached per host thread is not safe across
// cudaSetDevice, so it is queried; the call is cheap).
int current_device();

// Device address of the library's error word on device `dev` (api.cu): kernels
// whose bounded waits give up write PT_ETIMEOUT's cause there, and
// pt_device_status reads and clears it.  A file-scope __device__ variable, so
// looking it up allocates nothing; NULL if the lookup fails.
int *err_word(int dev);

// The library's workspace of (current device, stream) with at least `need`
// bytes (tc.cu): its first kSkHeaderBytes hold the stream-K header.  Grown
// outside stream capture only (PT_EUNSUPPORTED while capturing); `dry`
// checks without allocating.
int stream_workspace(cudaStream_t st, size_t need, bool dry, void **out);

// The stream-K segments (tile, first chunk, end chunk) of unit `unit` of
// `units` over tiles x nchunks, from the kernels' own partition code (tc.cu,
// pt_debug_streamk_segments): their number; at most `cap` are written.
int streamk_segments(int tiles, int nchunks, int units, int unit, int *out, int cap);

// Stream-K finisher wait settings for the next launches (api.cu,
// pt_debug_streamk_wait): time limit in ns and the awaited-value offset.
void streamk_wait_settings(uint64_t *limit_ns, unsigned *bias);

// Kernel timer (api.cu): records an event on `st` before (begin = true) or
// after the main GEMM kernel of a call while pt_kernel_timer_start is active
// on this host thread; otherwise does nothing.
void kernel_timer_mark(cudaStream_t st, bool begin);

// Launch attribute: programmatic stream serialization (the kernel may be
// scheduled while the previous kernel of the stream finishes; every kernel
// launched this way calls pdl_wait before its first global memory access).
inline void add_pdl_attr(cudaLaunchAttribute *attrs, unsigned &n) {
    attrs[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
}

inline bool misaligned(const void *p, int bytes) { return (reinterpret_cast<uintptr_t>(p) % bytes) != 0; }

// 2-D fp32 tensor map: inner extent `inner` (contiguous), outer extent
// `outer`, row pitch `ld` floats, box box_inner x box_outer.
inline int make_map_2d(CUtensorMap *map, const float *base, int64_t inner, int64_t outer, int64_t ld, int box_inner,
                       int box_outer, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4u};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PT_OK;
}

inline CUtensorMapSwizzle swizzle_for_bytes(int row_bytes) {
    switch (row_bytes) {
        case 32: return CU_TENSOR_MAP_SWIZZLE_32B;
        case 64: return CU_TENSOR_MAP_SWIZZLE_64B;
        case 128: return CU_TENSOR_MAP_SWIZZLE_128B;
        default: return CU_TENSOR_MAP_SWIZZLE_NONE;
    }
}

// Admission rules of a variant for one argument set (no launch).
template <class V>
int admit_simt(const GemmArgs &a) {
    if (V::LOADER == kLoaderTma) {
        if (a.tb != 0 || (V::AKM ? a.ta != 0 : a.ta != 1))
            return set_error(PT_EUNSUPPORTED, 0, "TMA variant needs transB='N' and transA='%c'", V::AKM ? 'N' : 'T');
        if (misaligned(a.A, 16) || misaligned(a.B, 16) || (a.lda % 4) || (a.ldb % 4))
            return set_error(PT_EUNSUPPORTED, 0, "TMA needs 16-byte aligned A/B and lda, ldb multiples of 4");
    } else if (V::AKM && a.ta != 0) {
        return set_error(PT_EUNSUPPORTED, 0, "K-major-A variant needs transA='N'");
    }
    if (V::VEC > 1) {
        const int vb = 4 * V::VEC;
        const bool a_direct = V::LOADER == kLoaderCpAsync && (V::AKM ? true : a.ta == 1);
        const bool b_direct = V::LOADER == kLoaderCpAsync && a.tb == 0;
        if (a_direct && (misaligned(a.A, vb) || (a.lda % V::VEC)))
            return set_error(PT_EUNSUPPORTED, 7, "A / lda not aligned to %d floats", V::VEC);
        if (b_direct && (misaligned(a.B, vb) || (a.ldb % V::VEC)))
            return set_error(PT_EUNSUPPORTED, 9, "B / ldb not aligned to %d floats", V::VEC);
        if (misaligned(a.C, vb) || (a.ldc % V::VEC))
            return set_error(PT_EUNSUPPORTED, 12, "C / ldc not aligned to %d floats", V::VEC);
    }
    const int64_t gy = ((int64_t)a.M + V::BM - 1) / V::BM;
    if (gy > 65535) return set_error(PT_EUNSUPPORTED, 3, "M too large for this tile");
    return PT_OK;
}

template <class V>
int launch_simt(const GemmArgs &a, cudaStream_t st, bool dry) {
    int rc = admit_simt<V>(a);
    if (rc != PT_OK || dry) return rc;

    static std::atomic<uint64_t> attr_done{0};
    const int dev = current_device();
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(simt_sgemm_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             V::SMEM_BYTES);
        if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }

    CUtensorMap mA, mB;
    std::memset(&mA, 0, sizeof(mA));
    std::memset(&mB, 0, sizeof(mB));
    if (V::LOADER == kLoaderTma) {
        if (V::AKM) rc = make_map_2d(&mA, a.A, a.K, a.M, a.lda, V::BK, V::BM, swizzle_for_bytes(V::BK * 4));
        else rc = make_map_2d(&mA, a.A, a.M, a.K, a.lda, V::BM, V::BK, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (rc != PT_OK) return rc;
        rc = make_map_2d(&mB, a.B, a.N, a.K, a.ldb, V::BN, V::BK, CU_TENSOR_MAP_SWIZZLE_NONE);
        if (rc != PT_OK) return rc;
    }

    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)((a.N + V::BN - 1) / V::BN), (unsigned)((a.M + V::BM - 1) / V::BM), V::SPLITK);
    cfg.blockDim = dim3(V::THREADS, 1, 1);
    cfg.dynamicSmemBytes = V::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    unsigned nattr = 0;
    if (V::SPLITK > 1) {
        attr[nattr].id = cudaLaunchAttributeClusterDimension;
        attr[nattr].val.clusterDim.x = 1;
        attr[nattr].val.clusterDim.y = 1;
        attr[nattr].val.clusterDim.z = V::SPLITK;
        ++nattr;
    }
    add_pdl_attr(attr, nattr);
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    kernel_timer_mark(st, true);
    cudaError_t e = cudaLaunchKernelEx(&cfg, simt_sgemm_kernel<V>, a, mA, mB);
    kernel_timer_mark(st, false);
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "launch: %s", cudaGetErrorString(e));
    return PT_OK;
}

// One registry entry.
struct VariantEntry {
    pt_variant_desc_t desc;
    int (*launch)(const GemmArgs &, cudaStream_t, bool dry);
};

const VariantEntry *variant_table();
int variant_table_size();

}  // namespace pt
