// FP32 SIMT SGEMM variant family for sm_103a.
//
// One template, instantiated ahead of time for every parameter configuration
// of the variant space (the paper's "code variants": a kernel compiled with
// one combination of tuning parameters, Section III-A; precompiled rather
// than JIT-compiled, Section III-B).
//
//   C <- alpha * op(A) * op(B) + beta * C      (row-major, FP32 FMA, FP32 accumulate)
//
// Parameters
//   BM x BN   CTA output tile               BK      K-step per pipeline stage
//   WM x WN   warp output tile              TM x TN per-thread register tile
//   KL        lane groups of a warp that split each stage's K range; their
//             partial sums are combined with __shfl_xor_sync
//   VEC       floats per direct global load (cp.async 4/8/16 B) and store
//   STAGES    shared-memory ring depth
//   SPLITK    CTAs of one thread-block cluster (1,1,SPLITK) that split K; the
//             partial tiles are summed through distributed shared memory in
//             cluster-rank order (deterministic, no atomics, no workspace)
//   LOADER    0: cp.async (LDGSTS) staging by all threads
//             1: TMA (cp.async.bulk.tensor) issued by one thread, mbarrier
//   F2        1: the register tile is updated with packed fma.rn.f32x2 (two
//             FP32 FMAs per instruction, same IEEE results), halving FMA issue
//             slots; 0: one fmaf per product
//   AKM       1: the A tile is held K-major in shared memory (rows of BK
//             floats, XOR-swizzled in 16-byte units with the TMA swizzle of
//             span BK*4 bytes) and read four k at a time; 0: held M-major
//             (rows of BM(+4) floats) and read one k at a time.
//
// Shared-memory layouts (per stage):
//   A, AKM=0: sA[k][m], row stride BM+PAD        (PAD = 4 for cp.async, 0 for TMA)
//   A, AKM=1: sA[m][k], BK floats per row, swizzled
//   B:        sB[k][n], row stride BN+PAD
// cp.async variants accept any (transA, transB) at run time: an operand whose
// global layout already matches is copied VEC floats at a time; one that
// does not is transposed on the fly by 4-byte copies laid out so that the
// shared-memory stores are bank-conflict free (needs the +4 padding).  TMA
// cannot transpose 4-byte elements, so TMA variants need transB = 'N' and
// transA = 'N' for AKM=1 / 'T' for AKM=0.
//
// Thread mapping: lane = (g * LN + ln) * LM + lm, g the k-group.  A thread
// owns rows  wm0 + (i/4)*4*LM + 4*lm + i%4   (AKM=0, float4 reads along m)
//       or   wm0 + lm + i*LM                  (AKM=1, one float4 of 4 k per row)
// and columns wn0 + (j/4)*4*LN + 4*ln + j%4, so every quarter-warp reads
// distinct consecutive 16-byte words or broadcasts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"

namespace pt {

struct GemmArgs {
    const float *A;
    const float *B;
    float *C;
    int64_t lda, ldb, ldc;
    int M, N, K;
    float alpha, beta;
    int ta, tb;  // 0 = 'N', 1 = 'T'
    int *err;    // device error word: bit 0 set when a bounded wait gave up
};

constexpr int kLoaderCpAsync = 0;
constexpr int kLoaderTma = 1;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per bounded wait

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int BM_, int BN_, int BK_, int WM_, int WN_, int TM_, int TN_, int KL_, int VEC_, int STAGES_,
          int SPLITK_, int LOADER_, int AKM_, int F2_ = 0>
struct Simt {
    static constexpr int BM = BM_, BN = BN_, BK = BK_, WM = WM_, WN = WN_, TM = TM_, TN = TN_;
    static constexpr int KL = KL_, VEC = VEC_, STAGES = STAGES_, SPLITK = SPLITK_;
    static constexpr int LOADER = LOADER_, AKM = AKM_, F2 = F2_;

    static constexpr int WARPS_M = BM / WM, WARPS_N = BN / WN;
    static constexpr int WARPS = WARPS_M * WARPS_N;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int LANES = 32 / KL;
    static constexpr int LM = WM / TM, LN = WN / TN;
    static constexpr int PAD = (LOADER == kLoaderCpAsync) ? 4 : 0;
    static constexpr int A_LD = BM + PAD;  // AKM = 0
    static constexpr int B_LD = BN + PAD;
    static constexpr int A_STAGE_BYTES = round_up(AKM ? BM * BK * 4 : BK * A_LD * 4, 1024);
    static constexpr int B_STAGE_BYTES = round_up(BK * B_LD * 4, 1024);
    static constexpr int PIPE_BYTES = STAGES * (A_STAGE_BYTES + B_STAGE_BYTES);
    static constexpr int RED_LD = BN + 4;
    static constexpr int RED_BYTES = SPLITK > 1 ? BM * RED_LD * 4 : 0;
    static constexpr int BAR_OFFSET = cmax(PIPE_BYTES, RED_BYTES);
    static constexpr int BAR_BYTES = LOADER == kLoaderTma ? 16 * STAGES : 0;
    static constexpr int ALIGN_SLACK = 1024;
    static constexpr int SMEM_BYTES = BAR_OFFSET + BAR_BYTES + ALIGN_SLACK;
    // XOR swizzle of the K-major A tile: 16-byte unit index ^= (byte >> 7) & SW_MASK
    static constexpr int SW_MASK = BK / 4 - 1;
    // Resident CTAs per SM asked of the register allocator, from an estimate
    // of registers per thread: accumulators + fragments + addressing, more
    // for the K-major A fragments (4 k per row) and the split-K epilogue.
    static constexpr int REG_EST = TM * TN + 64 + (AKM ? 6 * TM : 0) + (SPLITK > 1 ? 16 : 0);
    static constexpr int MIN_BLOCKS_RAW = 65536 / (THREADS * REG_EST);
    static constexpr int MIN_BLOCKS = MIN_BLOCKS_RAW < 1 ? 1 : (MIN_BLOCKS_RAW > 8 ? 8 : MIN_BLOCKS_RAW);

    static_assert(BM % WM == 0 && BN % WN == 0, "warp tiling");
    static_assert(LM * LN == LANES, "lane layout");
    static_assert(TN % 4 == 0 && (AKM || TM % 4 == 0), "float4 fragments");
    static_assert(BK % 8 == 0 && BK <= 32, "BK");
    static_assert(BK % (4 * KL) == 0, "each k-group needs whole k4 chunks");
    static_assert(TM % KL == 0, "stores are split across k-groups by rows");
    static_assert(BM % SPLITK == 0, "split-K reduction slices rows");
    static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
    static_assert(THREADS <= 1024, "threads");
};

// ---- packed FP32x2 FMA (sm_100+): two IEEE fused multiply-adds per instruction
__device__ __forceinline__ uint64_t pack2(float x, float y) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}

__device__ __forceinline__ void unpack2(uint64_t v, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}

__device__ __forceinline__ void fma2(uint64_t &d, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// ---- global -> shared copies (cp.async) ------------------------------------

// Direct copy of a ROWS x COLS tile whose COLS direction is contiguous in
// both global and shared memory.  Out-of-range parts are zero-filled.
template <int THREADS, int ROWS, int COLS, int VEC, int LD, bool SWZ, int SW_MASK>
__device__ __forceinline__ void copy_direct(uint32_t dst, const float *__restrict__ g, int64_t ld, int row0,
                                            int col0, int rows_valid, int cols_valid, int tid) {
    constexpr int CPR = COLS / VEC;
    constexpr int TOTAL = ROWS * CPR;
#pragma unroll
    for (int it = 0; it < (TOTAL + THREADS - 1) / THREADS; ++it) {
        const int c = tid + it * THREADS;
        if (TOTAL % THREADS == 0 || c < TOTAL) {
            const int r = c / CPR;
            const int col = (c % CPR) * VEC;
            const int grow = row0 + r, gcol = col0 + col;
            int nb = cols_valid - gcol;
            nb = nb < 0 ? 0 : (nb > VEC ? VEC : nb);
            if (grow >= rows_valid) nb = 0;
            const float *src = nb ? g + (int64_t)grow * ld + gcol : g;
            uint32_t off;
            if constexpr (SWZ) {
                const uint32_t lin = (uint32_t)(r * COLS + col) * 4u;
                off = lin ^ (((lin >> 7) & SW_MASK) << 4);
            } else {
                off = (uint32_t)(r * LD + col) * 4u;
            }
            cp_async<VEC * 4>(dst + off, src, (uint32_t)nb * 4u);
        }
    }
}

// Transposing copy: global tile ROWS (mn) x BK (k, contiguous) into shared
// sX[k][mn] with row stride LD.  A warp moves blocks of 8 k x 4 rows: 32-byte
// global segments, and 32 distinct banks on the shared side when LD % 32 == 4.
template <int THREADS, int ROWS, int BK, int LD>
__device__ __forceinline__ void copy_transpose(uint32_t dst, const float *__restrict__ g, int64_t ld, int row0,
                                               int k0, int rows_valid, int k_valid, int tid) {
    constexpr int WARPS = THREADS / 32;
    constexpr int KB = BK / 8;
    constexpr int BLOCKS = KB * (ROWS / 4);
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int it = 0; it < (BLOCKS + WARPS - 1) / WARPS; ++it) {
        const int b = warp + it * WARPS;
        if (BLOCKS % WARPS == 0 || b < BLOCKS) {
            const int k = (b % KB) * 8 + (lane & 7);
            const int r = (b / KB) * 4 + (lane >> 3);
            const int grow = row0 + r, gk = k0 + k;
            const bool ok = grow < rows_valid && gk < k_valid;
            const float *src = ok ? g + (int64_t)grow * ld + gk : g;
            cp_async<4>(dst + (uint32_t)(k * LD + r) * 4u, src, ok ? 4u : 0u);
        }
    }
}

// ---- epilogue store of 4 consecutive columns --------------------------------
template <int VEC>
__device__ __forceinline__ void store4(float *__restrict__ c, float4 v, int ncols, float alpha, float beta) {
    float r[4] = {v.x, v.y, v.z, v.w};
    if (ncols >= 4 && VEC == 4) {
        float4 o;
        if (beta != 0.f) {
            const float4 old = *reinterpret_cast<const float4 *>(c);
            o = make_float4(alpha * r[0] + beta * old.x, alpha * r[1] + beta * old.y, alpha * r[2] + beta * old.z,
                            alpha * r[3] + beta * old.w);
        } else {
            o = make_float4(alpha * r[0], alpha * r[1], alpha * r[2], alpha * r[3]);
        }
        *reinterpret_cast<float4 *>(c) = o;
    } else if (ncols >= 4 && VEC == 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 o;
            if (beta != 0.f) {
                const float2 old = *reinterpret_cast<const float2 *>(c + 2 * h);
                o = make_float2(alpha * r[2 * h] + beta * old.x, alpha * r[2 * h + 1] + beta * old.y);
            } else {
                o = make_float2(alpha * r[2 * h], alpha * r[2 * h + 1]);
            }
            *reinterpret_cast<float2 *>(c + 2 * h) = o;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (q < ncols) c[q] = (beta != 0.f) ? alpha * r[q] + beta * c[q] : alpha * r[q];
        }
    }
}

// ---- one CTA tile -------------------------------------------------------------
// Computes the BM x BN tile at (m0, n0) of C (over k-tiles of split kz when
// SPLITK > 1).  Shared by the per-GEMM kernel below and the persistent
// grouped kernel (which calls it for successive tiles; it leaves shared
// memory free for the next call).
template <class V>
__device__ __forceinline__ void simt_body(const GemmArgs &args, const CUtensorMap *tmA, const CUtensorMap *tmB,
                                          const int m0, const int n0, const int kz, const bool trigger = false) {
    constexpr int BM = V::BM, BN = V::BN, BK = V::BK, TM = V::TM, TN = V::TN, KL = V::KL;
    constexpr int STAGES = V::STAGES, THREADS = V::THREADS, LM = V::LM, LN = V::LN;
    constexpr bool TMA = V::LOADER == kLoaderTma;
    constexpr bool AKM = V::AKM != 0;

    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base (TMA swizzle patterns use absolute address bits).
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
    unsigned char *smem = smem_raw + pad;
    const uint32_t sbase = raw_addr + pad;
    const uint32_t sA0 = sbase;
    const uint32_t sB0 = sbase + STAGES * V::A_STAGE_BYTES;
    const uint32_t bar0 = sbase + V::BAR_OFFSET;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int lm = lane % LM;
    const int ln = (lane / LM) % LN;
    const int g = lane / V::LANES;
    const int wm0 = (warp / V::WARPS_N) * V::WM;
    const int wn0 = (warp % V::WARPS_N) * V::WN;

    const int M = args.M, N = args.N, K = args.K;

    // K range of this CTA (split-K across the cluster's z dimension).
    const int kt_total = (K + BK - 1) / BK;
    int kt_begin = 0, nkt = kt_total;
    if constexpr (V::SPLITK > 1) {
        const int per = (kt_total + V::SPLITK - 1) / V::SPLITK;
        kt_begin = kz * per;
        const int kt_end = kt_begin + per < kt_total ? kt_begin + per : kt_total;
        nkt = kt_end > kt_begin ? kt_end - kt_begin : 0;
    }

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    // Packed accumulators for the FP32x2 path: acc2[i][p] holds columns 2p, 2p+1.
    uint64_t acc2[V::F2 ? TM : 1][V::F2 ? TN / 2 : 1];
    if constexpr (V::F2) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int p = 0; p < TN / 2; ++p) acc2[i][p] = 0ull;
    }

    auto load_stage = [&](int s, int kt) {
        const int k0 = kt * BK;
        const uint32_t dA = sA0 + s * V::A_STAGE_BYTES;
        const uint32_t dB = sB0 + s * V::B_STAGE_BYTES;
        if constexpr (TMA) {
            const uint32_t bar = bar0 + 8 * s;
            mbar_arrive_expect_tx(bar, (uint32_t)((BM * BK + BK * BN) * 4));
            if constexpr (AKM) tma_load_2d(dA, tmA, bar, k0, m0);
            else tma_load_2d(dA, tmA, bar, m0, k0);
            tma_load_2d(dB, tmB, bar, n0, k0);
        } else {
            if constexpr (AKM) {
                copy_direct<THREADS, BM, BK, V::VEC, BK, true, V::SW_MASK>(dA, args.A, args.lda, m0, k0, M, K, tid);
            } else {
                if (args.ta) copy_direct<THREADS, BK, BM, V::VEC, V::A_LD, false, 0>(dA, args.A, args.lda, k0, m0, K, M, tid);
                else copy_transpose<THREADS, BM, BK, V::A_LD>(dA, args.A, args.lda, m0, k0, M, K, tid);
            }
            if (args.tb) copy_transpose<THREADS, BN, BK, V::B_LD>(dB, args.B, args.ldb, n0, k0, N, K, tid);
            else copy_direct<THREADS, BK, BN, V::VEC, V::B_LD, false, 0>(dB, args.B, args.ldb, k0, n0, K, N, tid);
        }
    };

    // Per-thread fragment offsets (bytes, relative to a stage base).
    const uint32_t b_off = (uint32_t)(wn0 + 4 * ln + g * 4 * V::B_LD) * 4u;
    uint32_t a_off = 0;
    uint32_t a_row[AKM ? TM : 1];
    uint32_t a_xor[AKM ? TM : 1];
    if constexpr (AKM) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const uint32_t r = (uint32_t)(wm0 + lm + i * LM);
            a_row[i] = r * BK * 4u;
            a_xor[i] = (uint32_t)g ^ ((a_row[i] >> 7) & V::SW_MASK);
        }
    } else {
        a_off = (uint32_t)(wm0 + 4 * lm + g * 4 * V::A_LD) * 4u;
    }

    auto compute_stage = [&](int s) {
        const unsigned char *pA = smem + s * V::A_STAGE_BYTES;
        const unsigned char *pB = smem + STAGES * V::A_STAGE_BYTES + s * V::B_STAGE_BYTES;
#pragma unroll
        for (int t = 0; t < BK / (4 * KL); ++t) {
            float a4[AKM ? TM : 1][4];
            if constexpr (AKM) {
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    const uint32_t off = a_row[i] + ((((uint32_t)(t * KL)) ^ a_xor[i]) << 4);
                    const float4 v = *reinterpret_cast<const float4 *>(pA + off);
                    a4[i][0] = v.x; a4[i][1] = v.y; a4[i][2] = v.z; a4[i][3] = v.w;
                }
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k = t * KL * 4 + kk;  // this k-group's k is k + 4*g (folded into offsets)
                float a[TM], b[V::F2 ? 1 : TN];
                if constexpr (AKM) {
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = a4[i][kk];
                } else {
#pragma unroll
                    for (int c = 0; c < TM / 4; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(pA + a_off + (k * V::A_LD + c * 4 * LM) * 4);
                        a[4 * c] = v.x; a[4 * c + 1] = v.y; a[4 * c + 2] = v.z; a[4 * c + 3] = v.w;
                    }
                }
                if constexpr (V::F2) {
                    uint64_t b2[TN / 2];
#pragma unroll
                    for (int c = 0; c < TN / 4; ++c) {
                        const ulonglong2 v =
                            *reinterpret_cast<const ulonglong2 *>(pB + b_off + (k * V::B_LD + c * 4 * LN) * 4);
                        b2[2 * c] = v.x;
                        b2[2 * c + 1] = v.y;
                    }
#pragma unroll
                    for (int i = 0; i < TM; ++i) {
                        const uint64_t ad = pack2(a[i], a[i]);
#pragma unroll
                        for (int p = 0; p < TN / 2; ++p) fma2(acc2[i][p], ad, b2[p]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < TN / 4; ++c) {
                        const float4 v = *reinterpret_cast<const float4 *>(pB + b_off + (k * V::B_LD + c * 4 * LN) * 4);
                        b[4 * c] = v.x; b[4 * c + 1] = v.y; b[4 * c + 2] = v.z; b[4 * c + 3] = v.w;
                    }
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                }
            }
        }
    };

    bool failed = false;
    if constexpr (TMA) {
        // full[s] (bar0 + 8s): completes when stage s's TMA bytes have landed
        // (one arrive: the producer's expect_tx).  empty[s] (emp0 + 8s):
        // completes when every warp has finished reading stage s (one arrive
        // per warp).  Warps never wait for each other: the producer thread
        // refills the stage read one iteration earlier, so its empty wait is
        // normally already satisfied.
        const uint32_t emp0 = bar0 + 8 * STAGES;
        if (tid == 0) {
            prefetch_tensormap(tmA);
            prefetch_tensormap(tmB);
#pragma unroll
            for (int s = 0; s < STAGES; ++s) {
                mbar_init(bar0 + 8 * s, 1);
                mbar_init(emp0 + 8 * s, V::WARPS);
            }
            fence_mbarrier_init();
        }
        __syncthreads();
        const int pre = STAGES < nkt ? STAGES : nkt;
        int issued = 0, seen = 0;  // k-tiles issued / waited on (thread 0's view)
        if (tid == 0) {
            for (int s = 0; s < pre; ++s) load_stage(s, kt_begin + s);
            issued = pre;
        }
        bool ok = true;
        int s = 0;
        uint32_t phase = 0;
        for (int it = 0; it < nkt; ++it) {
            if (!mbar_wait_bounded(bar0 + 8 * s, phase, kWaitLimitNs)) {
                ok = false;
                break;
            }
            seen = it + 1;
            compute_stage(s);
            __syncwarp();
            if (lane == 0) mbar_arrive(emp0 + 8 * s);
            const int j = it - 1 + STAGES;  // refill the stage read at it - 1 with k-tile j
            if (tid == 0 && it >= 1 && j < nkt) {
                const int sp = (s + STAGES - 1) % STAGES;
                if (!mbar_wait_bounded(emp0 + 8 * sp, (uint32_t)(((it - 1) / STAGES) & 1), kWaitLimitNs)) {
                    ok = false;
                    break;
                }
                load_stage(sp, kt_begin + j);
                issued = j + 1;
            }
            if (++s == STAGES) { s = 0; phase ^= 1u; }
        }
        failed = __syncthreads_or(!ok);
        if (failed && tid == 0) {
            if (args.err) atomicOr(args.err, 1);
            // Let every TMA copy still in flight land before shared memory is
            // reused or the CTA exits.
            for (int q = seen; q < issued; ++q)
                (void)mbar_wait_bounded(bar0 + 8 * (q % STAGES), (uint32_t)((q / STAGES) & 1), kWaitLimitNs);
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int s = 0; s < STAGES - 1; ++s) {
            if (s < nkt) load_stage(s, kt_begin + s);
            cp_async_commit();
        }
        int s = 0;
        for (int it = 0; it < nkt; ++it) {
            cp_async_wait<STAGES - 2>();
            __syncthreads();
            const int nx = it + STAGES - 1;
            if (nx < nkt) load_stage((s + STAGES - 1) % STAGES, kt_begin + nx);
            cp_async_commit();
            compute_stage(s);
            if (++s == STAGES) s = 0;
        }
        cp_async_wait<0>();
        __syncthreads();
    }

    // Main loop done: the next kernel of the stream may be scheduled (it
    // still waits for this one to complete before touching memory).
    if (trigger) pdl_trigger();

    if constexpr (V::F2) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int p = 0; p < TN / 2; ++p) unpack2(acc2[i][p], acc[i][2 * p], acc[i][2 * p + 1]);
    }

    // Combine the k-groups of each warp (butterfly; every group ends with the
    // same bits since the last step adds the same two values in either order).
    if constexpr (KL > 1) {
#pragma unroll
        for (int off = 16; off >= V::LANES; off >>= 1)
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], off);
    }

    auto row_of = [&](int i) -> int {
        if constexpr (AKM) return wm0 + lm + i * LM;
        else return wm0 + (i / 4) * 4 * LM + 4 * lm + (i % 4);
    };

    const float alpha = args.alpha, beta = args.beta;
    if constexpr (V::SPLITK == 1) {
        if (!failed) {
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                if (KL > 1 && (i % KL) != g) continue;
                const int row = m0 + row_of(i);
                if (row >= M) continue;
                float *crow = args.C + (int64_t)row * args.ldc;
#pragma unroll
                for (int c = 0; c < TN / 4; ++c) {
                    const int col = n0 + wn0 + c * 4 * LN + 4 * ln;
                    if (col < N)
                        store4<V::VEC>(crow + col,
                                       make_float4(acc[i][4 * c], acc[i][4 * c + 1], acc[i][4 * c + 2], acc[i][4 * c + 3]),
                                       N - col, alpha, beta);
                }
            }
        }
    } else {
        // Partial tiles -> own shared memory -> cluster barrier -> CTA r sums
        // rows [r*BM/S, (r+1)*BM/S) over ranks 0..S-1 in order.
        float *red = reinterpret_cast<float *>(smem);
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            if (KL > 1 && (i % KL) != g) continue;
            const int r = row_of(i);
#pragma unroll
            for (int c = 0; c < TN / 4; ++c) {
                const int cl = wn0 + c * 4 * LN + 4 * ln;
                *reinterpret_cast<float4 *>(red + r * V::RED_LD + cl) =
                    make_float4(acc[i][4 * c], acc[i][4 * c + 1], acc[i][4 * c + 2], acc[i][4 * c + 3]);
            }
        }
        cluster_sync();
        const uint32_t rank = cluster_ctarank();
        constexpr int ROWS = BM / V::SPLITK;
        constexpr int C4 = BN / 4;
        const uint32_t red_addr = smem_u32(red);
        for (int idx = tid; idx < ROWS * C4; idx += THREADS) {
            const int rl = (int)rank * ROWS + idx / C4;
            const int cl = (idx % C4) * 4;
            const int row = m0 + rl, col = n0 + cl;
            if (failed || row >= M || col >= N) continue;
            const uint32_t a = red_addr + (uint32_t)(rl * V::RED_LD + cl) * 4u;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < V::SPLITK; ++q) {
                const float4 v = ld_dsmem_f4(mapa_shared(a, (uint32_t)q));
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            store4<V::VEC>(args.C + (int64_t)row * args.ldc + col, sum, N - col, alpha, beta);
        }
        cluster_sync();  // no CTA leaves while a peer may still read its tile
    }
}

template <class V>
__global__ void __launch_bounds__(V::THREADS, V::MIN_BLOCKS)
    simt_sgemm_kernel(const GemmArgs args, const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB) {
    pdl_wait();  // launched with programmatic stream serialization
    simt_body<V>(args, &tmA, &tmB, (int)blockIdx.y * V::BM, (int)blockIdx.x * V::BN, (int)blockIdx.z, true);
}

}  // namespace pt
