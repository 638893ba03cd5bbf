// Split kernel of the tensor-core versions: FP32 operands to K-major
// low-precision planes (3xTF32: hi, lo; BF16x3: b0, b1, b2) in a workspace
// that the GEMM kernel reads through TMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"

namespace pt {

constexpr int kTcTf32 = 0;
constexpr int kTcBf16x3 = 1;

// ---- splitting --------------------------------------------------------------------
// Round to nearest even on the TF32 grid (10 explicit mantissa bits) by bit
// manipulation; infinities and NaNs keep their class.
__device__ __forceinline__ float tf32_rne(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u += 0xfffu + ((u >> 13) & 1u);
    else if (u & 0x007fffffu) u |= 0x00400000u;
    return __uint_as_float(u & 0xffffe000u);
}

// Two floats to BF16 with round-to-nearest-even (one cvt.rn.bf16x2.f32; NaN
// and infinity keep their class): x0 in the low half, x1 in the high half.
__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(x1), "f"(x0));
    return d;
}
__device__ __forceinline__ float bf16_lo_f32(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi_f32(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }

// Planes of 8 consecutive elements x[0..8) of row r starting at column k
// (k a multiple of 8, k + 8 <= pitch): one 16-byte store per plane for BF16,
// two per plane for TF32.  Elements at or beyond K are written as zero.
template <int KIND>
__device__ __forceinline__ void split_store8(unsigned char *ws, int64_t plane_bytes, int64_t pitch, int r, int k,
                                             const float (&x)[8]) {
    const int64_t off = (int64_t)r * pitch + k;
    if constexpr (KIND == kTcTf32) {
        float hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            hi[i] = tf32_rne(x[i]);
            lo[i] = tf32_rne(x[i] - hi[i]);
        }
        float4 *ph = reinterpret_cast<float4 *>(reinterpret_cast<float *>(ws) + off);
        float4 *pl = reinterpret_cast<float4 *>(reinterpret_cast<float *>(ws + plane_bytes) + off);
        ph[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        ph[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
        pl[0] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        pl[1] = make_float4(lo[4], lo[5], lo[6], lo[7]);
    } else {
        // b0 = RN(x), b1 = RN(x - b0), b2 = RN(x - b0 - b1); the residuals
        // are exact in FP32.
        uint32_t b[3][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            float v0 = x[i], v1 = x[i + 1];
#pragma unroll
            for (int pl = 0; pl < 3; ++pl) {
                const uint32_t q = bf16x2_rn(v0, v1);
                b[pl][i / 2] = q;
                v0 -= bf16_lo_f32(q);
                v1 -= bf16_hi_f32(q);
            }
        }
#pragma unroll
        for (int pl = 0; pl < 3; ++pl)
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(ws + pl * plane_bytes) + off) =
                make_uint4(b[pl][0], b[pl][1], b[pl][2], b[pl][3]);
    }
}

// Split of a logical rows x K operand X(r, k) into K-major planes with row
// pitch `pitch` (a multiple of 8 elements, >= round_up(K, 8)); the padding
// columns [K, pitch) are written as zero.
// trans == 0: X(r, k) at src[r*ld + k];  trans == 1: X(r, k) at src[k*ld + r].
// A block of 256 threads covers 32 rows x 64 columns; every thread writes 8
// consecutive columns of one row with 16-byte stores.  The transposed case
// goes through shared memory so that the global reads run along r.
// vec4: src and ld allow 16-byte loads along the contiguous direction.
// One operand of a split: rows x K values, element (r, k) at src[r * ld + k]
// (trans = 0) or src[k * ld + r] (trans = 1); planes written to ws.
struct SplitOperand {
    const float *src;
    int64_t ld;
    int trans;
    int rows;
    unsigned char *ws;
    int64_t plane_bytes;
    int vec4;  // src and ld allow 16-byte loads
};

// Both operands in one launch: blocks with blockIdx.y < ya split `a`, the
// others `b`.  A block converts 32 rows x SPLIT_KT * 64 values of k; each
// thread issues all of its loads (SPLIT_KT x 32 bytes) before converting, so
// that enough bytes are in flight to keep HBM busy.  Transposed sources go
// through shared memory so that both the loads and the 16-byte plane stores
// are contiguous.
constexpr int SPLIT_KT = 4;
constexpr int SPLIT_K_PER_BLOCK = 64 * SPLIT_KT;

template <int KIND>
__global__ void __launch_bounds__(256) tc_split_kernel(const SplitOperand a, const SplitOperand b, int K,
                                                       int64_t pitch, int ya) {
    __shared__ float tile[SPLIT_KT][64][33];
    const bool first = (int)blockIdx.y < ya;
    const SplitOperand &o = first ? a : b;
    const int by = first ? (int)blockIdx.y : (int)blockIdx.y - ya;
    const float *__restrict__ src = o.src;
    const int64_t ld = o.ld;
    const int rows = o.rows;
    const int r0 = by * 32, kb = blockIdx.x * SPLIT_K_PER_BLOCK;
    const int tid = threadIdx.x;
    const int r = r0 + (tid >> 3), kt8 = (tid & 7) * 8;
    float x[SPLIT_KT][8];
    // Launched with programmatic stream serialization: the previous kernel
    // (e.g. a GEMM still reading the planes) completes first.
    pdl_wait();
    if (o.trans) {
        // tile[t][kk][rr] <- X(r0 + rr, kb + 64 t + kk) = src[(kb + 64 t + kk) * ld + r0 + rr]
        float v[SPLIT_KT][2][4];
        const int rr = (tid & 7) * 4, gr = r0 + rr;
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int gk = kb + 64 * t + (tid >> 3) + 32 * j;
                const float *p = src + (int64_t)gk * ld + gr;
                if (gk < K && gr + 3 < rows && o.vec4) {
                    const float4 q = *reinterpret_cast<const float4 *>(p);
                    v[t][j][0] = q.x; v[t][j][1] = q.y; v[t][j][2] = q.z; v[t][j][3] = q.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[t][j][i] = (gk < K && gr + i < rows) ? p[i] : 0.f;
                }
            }
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) tile[t][(tid >> 3) + 32 * j][rr + i] = v[t][j][i];
        __syncthreads();
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t)
#pragma unroll
            for (int i = 0; i < 8; ++i) x[t][i] = tile[t][kt8 + i][tid >> 3];
    } else {
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t) {
            const int k = kb + 64 * t + kt8;
            const float *p = src + (int64_t)r * ld + k;
            if (r < rows && k + 7 < K && o.vec4) {
                const float4 q0 = *reinterpret_cast<const float4 *>(p);
                const float4 q1 = *reinterpret_cast<const float4 *>(p + 4);
                x[t][0] = q0.x; x[t][1] = q0.y; x[t][2] = q0.z; x[t][3] = q0.w;
                x[t][4] = q1.x; x[t][5] = q1.y; x[t][6] = q1.z; x[t][7] = q1.w;
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) x[t][i] = (r < rows && k + i < K) ? p[i] : 0.f;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < SPLIT_KT; ++t) {
        const int k = kb + 64 * t + kt8;
        if (r < rows && k < pitch) split_store8<KIND>(o.ws, o.plane_bytes, pitch, r, k, x[t]);
    }
    pdl_trigger();
}

}  // namespace pt
