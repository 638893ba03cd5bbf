// Split kernel of the tensor-core versions: FP32 operands to K-major
// low-precision planes (3xTF32: hi, lo; BF16x3: b0, b1, b2; scaled 3xF16:
// h0, h1 of the value times a power-of-two scale per 256 values of k)
// in a workspace that the GEMM kernel reads through TMA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"

namespace pt {

constexpr int kTcTf32 = 0;
constexpr int kTcBf16x3 = 1;
constexpr int kTcF16s = 2;  // scaled FP16 split, three products (3xTF32's precision, FP16 rate)

// Scaled FP16 split: k is cut into chunks of 256 values.  Chunk c of row r of
// op(A) is multiplied by 2^S_A(r, c); chunk c of a group of 32 consecutive
// columns g of op(B) (32 consecutive rows of the K-major B planes) by
// 2^S_B(g, c).  S = 14 - floor(log2 m), m the largest magnitude in that
// chunk of the row (of the 32 columns), clamped to [-63, 63] (63 when
// m = 0), so that largest magnitude lands in [2^14, 2^15) (FP16 holds up to
// 65504).  The GEMM multiplies each chunk's product by 2^-S_A * 2^-S_B, a
// power of two in [2^-126, 2^126] (exact), when it drains the chunk.  Maxima
// in [2^-49, 2^78] get the full scale; beyond 2^78 the planes overflow to
// infinity, below 2^-49 the values keep fewer bits (as FP32 products of such
// values do).
constexpr int kF16ScaleMin = -63, kF16ScaleMax = 63;
__device__ __forceinline__ int f16_scale_exp(float m) {
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu);  // biased exponent of m (0: zero or subnormal)
    int S = 141 - e;                                           // 14 - (e - 127)
    S = S < kF16ScaleMin ? kF16ScaleMin : S;
    return S > kF16ScaleMax ? kF16ScaleMax : S;
}
__device__ __forceinline__ float pow2f(int S) { return __uint_as_float((uint32_t)(S + 127) << 23); }

// Two floats to FP16 with round-to-nearest-even (one cvt.rn.f16x2.f32): x0 in
// the low half, x1 in the high half; and back to FP32 (exact).
__device__ __forceinline__ uint32_t f16x2_rn(float x0, float x1) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(x1), "f"(x0));
    return d;
}
__device__ __forceinline__ float f16_lo_f32(uint32_t p) {
    float f;
    asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %1;\n cvt.f32.f16 %0, lo;\n}" : "=f"(f) : "r"(p));
    return f;
}
__device__ __forceinline__ float f16_hi_f32(uint32_t p) {
    float f;
    asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %1;\n cvt.f32.f16 %0, hi;\n}" : "=f"(f) : "r"(p));
    return f;
}

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
    } else if constexpr (KIND == kTcF16s) {
        // h0 = RN(x), h1 = RN(x - h0) on the FP16 grid (x already scaled);
        // the residual is exact in FP32.
        uint32_t h[2][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            const uint32_t q = f16x2_rn(x[i], x[i + 1]);
            h[0][i / 2] = q;
            h[1][i / 2] = f16x2_rn(x[i] - f16_lo_f32(q), x[i + 1] - f16_hi_f32(q));
        }
#pragma unroll
        for (int pl = 0; pl < 2; ++pl)
            *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(ws + pl * plane_bytes) + off) =
                make_uint4(h[pl][0], h[pl][1], h[pl][2], h[pl][3]);
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
    // Scaled FP16 split only: 2^-S of chunk c at scale[c * ld_scale + i], i the
    // row (first operand) or the 32-row group (second operand).
    float *scale = nullptr;
    int64_t ld_scale = 0;
};

// Both operands in one launch: blocks with blockIdx.y < ya split `a`, the
// others `b`.  A block converts 32 rows x SPLIT_KT * 64 values of k; each
// thread issues all of its loads (SPLIT_KT x 32 bytes) before converting, so
// that enough bytes are in flight to keep HBM busy.  Transposed sources go
// through shared memory so that both the loads and the 16-byte plane stores
// are contiguous.
constexpr int SPLIT_KT = 4;
constexpr int SPLIT_K_PER_BLOCK = 64 * SPLIT_KT;

// The block's 32 rows x SPLIT_K_PER_BLOCK values of k starting at
// (r0, kb) into x (thread t: row r0 + t / 8, values kb + 64 s + 8 (t % 8) + i of
// slab s); values outside the operand are zero.  Transposed sources go
// through shared memory so that both the loads and the later 16-byte plane
// stores are contiguous.
__device__ __forceinline__ void split_load_block(const SplitOperand &o, int K, int r0, int kb, int tid,
                                                 float (&x)[SPLIT_KT][8], float (*tile)[64][33]) {
    const float *__restrict__ src = o.src;
    const int64_t ld = o.ld;
    const int rows = o.rows;
    const int r = r0 + (tid >> 3), kt8 = (tid & 7) * 8;
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
}

template <int KIND>
__global__ void __launch_bounds__(256) tc_split_kernel(const SplitOperand a, const SplitOperand b, int K,
                                                       int64_t pitch, int ya) {
    __shared__ float tile[SPLIT_KT][64][33];
    __shared__ float gmax[8];
    const bool first = (int)blockIdx.y < ya;
    const SplitOperand &o = first ? a : b;
    const int by = first ? (int)blockIdx.y : (int)blockIdx.y - ya;
    const int r0 = by * 32, kb = blockIdx.x * SPLIT_K_PER_BLOCK;
    const int tid = threadIdx.x;
    const int r = r0 + (tid >> 3), kt8 = (tid & 7) * 8;
    float x[SPLIT_KT][8];
    // Launched with programmatic stream serialization: the previous kernel
    // (e.g. a GEMM still reading the planes) completes first.  The GEMM that
    // reads these planes may be scheduled as soon as every block of this grid
    // has started (it waits for this grid to complete before it reads them),
    // so its launch and prologue overlap this grid's last wave.
    pdl_wait();
    pdl_trigger();
    split_load_block(o, K, r0, kb, tid, x, tile);
    if constexpr (KIND == kTcF16s) {
        // The block's 256 values of k are chunk blockIdx.x.  First operand:
        // the maximum of each row's chunk (its eight threads are consecutive
        // lanes); second operand: of the block's 32 rows (all threads).
        static_assert(SPLIT_K_PER_BLOCK == 256, "a block covers one 256-k chunk");
        float m = 0.f;
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t)
#pragma unroll
            for (int i = 0; i < 8; ++i) m = fmaxf(m, fabsf(x[t][i]));
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (!first) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
            if ((tid & 31) == 0) gmax[tid >> 5] = m;
            __syncthreads();
            m = gmax[0];
#pragma unroll
            for (int w = 1; w < 8; ++w) m = fmaxf(m, gmax[w]);
        }
        const int S = f16_scale_exp(m);
        const float sc = pow2f(S);
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t)
#pragma unroll
            for (int i = 0; i < 8; ++i) x[t][i] *= sc;
        const int gc = (int)blockIdx.x;
        if (first && (tid & 7) == 0 && r < o.rows) o.scale[(int64_t)gc * o.ld_scale + r] = pow2f(-S);
        if (!first && tid == 0) o.scale[(int64_t)gc * o.ld_scale + by] = pow2f(-S);
    }
#pragma unroll
    for (int t = 0; t < SPLIT_KT; ++t) {
        const int k = kb + 64 * t + kt8;
        if (r < o.rows && k < pitch) split_store8<KIND>(o.ws, o.plane_bytes, pitch, r, k, x[t]);
    }
}

}  // namespace pt
