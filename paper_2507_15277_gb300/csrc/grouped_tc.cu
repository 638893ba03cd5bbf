// Grouped 3xF16 tensor-core SGEMM (layout and plan in grouped_tc.cuh): a
// plan kernel, a split kernel over all tensor-core problems, and one
// persistent GEMM kernel walking all their 128 x 128 tiles.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "common.h"
#include "grouped_tc.cuh"
#include "launch.cuh"
#include "tc.cuh"

namespace pt {
namespace {

constexpr int kGtcStages = 3;
constexpr int kGtcThreads = 192;  // 4 epilogue warps, producer warp, MMA warp
constexpr int kGtcStageBytes = 2 * kGtcBlockBytes;
constexpr int kGtcBarOffset = kGtcStages * kGtcStageBytes;
constexpr int kGtcBarBytes = 8 * (2 * kGtcStages + 6);
constexpr int kGtcStgLd = 36;
constexpr int kGtcStgOffset = (kGtcBarOffset + kGtcBarBytes + 15) / 16 * 16;
constexpr int kGtcSmem = kGtcStgOffset + 4 * 32 * kGtcStgLd * 4 + 1024;
static_assert(kGtcSmem <= 232448, "shared memory");
// Instruction descriptors: D = F32, A = B = F16, K-major, M = 128, N = 256
// (the paired A0 [B0 | B1] product) or 128.
constexpr uint32_t kGtcIdescW = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t kGtcIdesc = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ int gtc_find(const int *prefix, int count, int t) {
    int lo = 0, hi = count - 1;  // last problem whose first item is <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool gtc_trans(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }

// Prefix sums of tiles, split units and region bytes (one block).
__global__ void __launch_bounds__(256) gtc_plan_kernel(const pt_gemm_problem_t *__restrict__ probs, int count,
                                                      GtcPlan pl) {
    __shared__ int64_t s_part[3][256];
    const int tid = threadIdx.x;
    const int per = (count + 255) / 256;
    int64_t loc[3] = {0, 0, 0};
    for (int i = 0; i < per; ++i) {
        const int p = tid * per + i;
        if (p < count) {
            loc[0] += gtc_tiles(probs[p]);
            loc[1] += gtc_units(probs[p]);
            loc[2] += gtc_region_bytes(probs[p]);
        }
    }
    for (int j = 0; j < 3; ++j) s_part[j][tid] = loc[j];
    __syncthreads();
    if (tid == 0) {
        int64_t run[3] = {0, 0, 0};
        for (int w = 0; w < 256; ++w)
            for (int j = 0; j < 3; ++j) {
                const int64_t v = s_part[j][w];
                s_part[j][w] = run[j];
                run[j] += v;
            }
    }
    __syncthreads();
    int64_t run[3] = {s_part[0][tid], s_part[1][tid], s_part[2][tid]};
    for (int i = 0; i < per; ++i) {
        const int p = tid * per + i;
        if (p < count) {
            pl.tile_prefix[p] = (int)run[0];
            pl.unit_prefix[p] = (int)run[1];
            pl.off[p] = run[2];
            run[0] += gtc_tiles(probs[p]);
            run[1] += gtc_units(probs[p]);
            run[2] += gtc_region_bytes(probs[p]);
        }
    }
    if (count > 0 && tid == (count - 1) / per) {  // the thread holding the last problem: totals
        pl.tile_prefix[count] = (int)run[0];
        pl.unit_prefix[count] = (int)run[1];
        pl.off[count] = run[2];
    }
}

// Split of the tensor-core problems: unit u (32 rows x 256 values of k of A,
// or of op(B)^T) of problem p into its tiled, pre-swizzled FP16 planes and
// chunk scales (see grouped_tc.cuh).
__global__ void __launch_bounds__(256) gtc_split_kernel(const pt_gemm_problem_t *__restrict__ probs, int count,
                                                       GtcPlan pl) {
    __shared__ float tile[SPLIT_KT][64][33];
    __shared__ float gmax[SPLIT_KT / 2][8];
    const int tid = threadIdx.x;
    pdl_wait();  // the plan kernel has completed
    const int total = pl.unit_prefix[count];
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        const int p = gtc_find(pl.unit_prefix, count, u);
        const pt_gemm_problem_t &pr = probs[p];
        const GtcDims d = gtc_dims(pr);
        const int64_t kbs = (d.kt + 3) / 4;  // 256-k blocks
        int64_t lu = u - pl.unit_prefix[p];
        const bool isA = lu < d.mt * 4 * kbs;
        if (!isA) lu -= d.mt * 4 * kbs;
        const int rb = (int)(lu / kbs), kb = (int)(lu % kbs);
        unsigned char *reg = pl.regions + pl.off[p];
        SplitOperand o;
        if (isA) {
            o.src = pr.A;
            o.ld = pr.lda;
            o.trans = gtc_trans(pr.transA) ? 1 : 0;
            o.rows = (int)pr.m;
        } else {
            o.src = pr.B;
            o.ld = pr.ldb;
            o.trans = gtc_trans(pr.transB) ? 0 : 1;  // op(B)^T rows are B's columns unless B is stored N x K
            o.rows = (int)pr.n;
        }
        o.vec4 = (reinterpret_cast<uintptr_t>(o.src) % 16 == 0 && o.ld % 4 == 0) ? 1 : 0;
        const int K = (int)pr.k;
        const int r0 = rb * 32, k0 = kb * SPLIT_K_PER_BLOCK;
        const int r = r0 + (tid >> 3);
        float x[SPLIT_KT][8];
        __syncthreads();  // the previous unit's shared-memory reads are done
        split_load_block(o, K, r0, k0, tid, x, tile);
        unsigned char *blocks = reg + (isA ? 0 : gtc_a_bytes(d));
        float *scales = reinterpret_cast<float *>(reg + gtc_a_bytes(d) + gtc_b_bytes(d) + (isA ? 0 : gtc_sa_bytes(d)));
        const int64_t ld_scale = isA ? d.mt * 128 : d.nt * 4;
#pragma unroll
        for (int c = 0; c < SPLIT_KT / 2; ++c) {
            float m = 0.f;
#pragma unroll
            for (int t = 2 * c; t < 2 * c + 2; ++t)
#pragma unroll
                for (int i = 0; i < 8; ++i) m = fmaxf(m, fabsf(x[t][i]));
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            if (!isA) {
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
                m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
                if ((tid & 31) == 0) gmax[c][tid >> 5] = m;
            } else {
                const int S = f16_scale_exp(m);
                const float sc = pow2f(S);
#pragma unroll
                for (int t = 2 * c; t < 2 * c + 2; ++t)
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[t][i] *= sc;
                const int64_t gc = (int64_t)kb * 2 + c;
                if ((tid & 7) == 0 && gc < d.nch) scales[gc * ld_scale + r] = pow2f(-S);
            }
        }
        if (!isA) {
            __syncthreads();
#pragma unroll
            for (int c = 0; c < SPLIT_KT / 2; ++c) {
                float m = gmax[c][0];
#pragma unroll
                for (int w = 1; w < 8; ++w) m = fmaxf(m, gmax[c][w]);
                const int S = f16_scale_exp(m);
                const float sc = pow2f(S);
#pragma unroll
                for (int t = 2 * c; t < 2 * c + 2; ++t)
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[t][i] *= sc;
                const int64_t gc = (int64_t)kb * 2 + c;
                if (tid == 0 && gc < d.nch) scales[gc * ld_scale + rb] = pow2f(-S);
            }
        }
        // Planes: 16-byte chunk (tid % 8) of row r in k-tile kb * 4 + t, at
        // chunk (tid % 8) ^ (r % 8) of the row in its 128-row block.
#pragma unroll
        for (int t = 0; t < SPLIT_KT; ++t) {
            const int64_t ktile = (int64_t)kb * 4 + t;
            if (ktile >= d.kt) continue;
            uint32_t h[2][4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                const uint32_t q = f16x2_rn(x[t][i], x[t][i + 1]);
                h[0][i / 2] = q;
                h[1][i / 2] = f16x2_rn(x[t][i] - f16_lo_f32(q), x[t][i + 1] - f16_hi_f32(q));
            }
            unsigned char *blk = blocks + ((int64_t)(r / 128) * d.kt + ktile) * kGtcBlockBytes;
            const int off = (r % 128) * 128 + ((((tid & 7)) ^ (r & 7)) << 4);
#pragma unroll
            for (int pl2 = 0; pl2 < 2; ++pl2)
                *reinterpret_cast<uint4 *>(blk + pl2 * (kGtcBlockBytes / 2) + off) =
                    make_uint4(h[pl2][0], h[pl2][1], h[pl2][2], h[pl2][3]);
        }
    }
    pdl_trigger();
}

// Persistent GEMM over all tensor-core problems' 128 x 128 tiles: CTA b takes
// tiles b, b + gridDim.x, ... of the concatenated tile list.  The roles and
// the pipeline are those of the single-GEMM 3xF16 kernel (producer lane,
// MMA lane, four epilogue warps; stage, phase and chunk counters running on
// across tiles; two TMEM accumulators of 256 columns), with two 32 KB bulk
// copies per stage instead of tensor-map loads and each tile's problem
// found by binary search in the plan.
__global__ void __launch_bounds__(kGtcThreads, 1)
    gtc_gemm_kernel(const pt_gemm_problem_t *__restrict__ probs, int count, GtcPlan pl, int *err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_fail, s_issued, s_consumed;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    const uint32_t full0 = sbase + kGtcBarOffset;  // stages: blocks landed
    const uint32_t empty0 = full0 + 8 * kGtcStages;  // stages: MMAs done reading
    const uint32_t accf0 = empty0 + 8 * kGtcStages;  // 2: accumulator ready
    const uint32_t acce0 = accf0 + 16;               // 2: accumulator drained
    const uint32_t doneb = acce0 + 16;               // every issued MMA finished
    const uint32_t tslot = doneb + 8;
    const volatile uint32_t *tslot_ptr = reinterpret_cast<const volatile uint32_t *>(smem_raw + (tslot - raw));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kGtcStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);
        }
        mbar_init(doneb, 1);
        fence_mbarrier_init();
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;
    pdl_wait();  // the split kernel has completed
    const int total = pl.tile_prefix[count];
    bool epi_ok = true;

    if (warp == 4) {
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < total; t += gridDim.x) {
                const int p = gtc_find(pl.tile_prefix, count, t);
                const GtcDims d = gtc_dims(probs[p]);
                const int64_t lt = t - pl.tile_prefix[p];
                const unsigned char *reg = pl.regions + pl.off[p];
                const unsigned char *ab = reg + (lt / d.nt) * d.kt * kGtcBlockBytes;
                const unsigned char *bb = reg + gtc_a_bytes(d) + (lt % d.nt) * d.kt * kGtcBlockBytes;
                for (int64_t kt = 0; kt < d.kt; ++kt, ++g) {
                    const int s = g % kGtcStages, u = g / kGtcStages;
                    if (g >= kGtcStages && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)((u - 1) & 1), kWaitLimitNs)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + s * kGtcStageBytes;
                    mbar_arrive_expect_tx(full0 + 8 * s, (uint32_t)kGtcStageBytes);
                    bulk_load(st, ab + kt * kGtcBlockBytes, kGtcBlockBytes, full0 + 8 * s);
                    bulk_load(st + kGtcBlockBytes, bb + kt * kGtcBlockBytes, kGtcBlockBytes, full0 + 8 * s);
                }
            }
            s_issued = g;
        }
    } else if (warp == 5) {
        if (lane == 0) {
            int g = 0, c = 0, b = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < total; t += gridDim.x) {
                const GtcDims d = gtc_dims(probs[gtc_find(pl.tile_prefix, count, t)]);
                for (int64_t kt = 0; kt < d.kt; ++kt, ++g) {
                    const int s = g % kGtcStages, u = g / kGtcStages;
                    const bool first = (kt & 1) == 0;
                    if (first) {
                        b = c & 1;
                        if (c >= 2 && !mbar_wait_bounded(acce0 + 8 * b, (uint32_t)(((c >> 1) - 1) & 1), kWaitLimitNs)) {
                            s_fail = 1;
                            ok = false;
                            break;
                        }
                    }
                    if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)(u & 1), kWaitLimitNs)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * kGtcStageBytes;
                    const uint32_t dt = tmem + (uint32_t)(b * 256);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        // A0 [B0 | B1] into both halves, then A1 B0 into the right half.
                        const uint64_t a0 = kmajor_desc<128>(st) + (uint64_t)(2 * kk);
                        const uint64_t a1 = kmajor_desc<128>(st + kGtcBlockBytes / 2) + (uint64_t)(2 * kk);
                        const uint64_t b0 = kmajor_desc<128>(st + kGtcBlockBytes) + (uint64_t)(2 * kk);
                        tc_mma<kTcF16s>(dt, a0, b0, kGtcIdescW, (first && kk == 0) ? 0u : 1u);
                        tc_mma<kTcF16s>(dt + 128u, a1, b0, kGtcIdesc, 1u);
                    }
                    tc_commit(empty0 + 8 * s);
                    if ((kt & 1) == 1 || kt == d.kt - 1) {
                        tc_commit(accf0 + 8 * b);
                        ++c;
                    }
                }
            }
            tc_commit(doneb);
            s_consumed = g;
        }
    } else {
        // Epilogue warps: drain each chunk times its scales, then store the tile.
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        float racc[128];
        int c = 0;
        for (int t = blockIdx.x; epi_ok && t < total; t += gridDim.x) {
            const int p = gtc_find(pl.tile_prefix, count, t);
            const pt_gemm_problem_t &pr = probs[p];
            const GtcDims d = gtc_dims(pr);
            const int64_t lt = t - pl.tile_prefix[p];
            const int m0 = (int)(lt / d.nt) * 128, n0 = (int)(lt % d.nt) * 128;
            const unsigned char *reg = pl.regions + pl.off[p];
            const float *sa_arr = reinterpret_cast<const float *>(reg + gtc_a_bytes(d) + gtc_b_bytes(d));
            const float *sb_arr = reinterpret_cast<const float *>(reinterpret_cast<const unsigned char *>(sa_arr) +
                                                                  gtc_sa_bytes(d));
            const int64_t ld_sa = d.mt * 128, ld_sb = d.nt * 4;
            const int64_t srow = m0 + warp * 32 + lane, sgrp = n0 / 32;
#pragma unroll
            for (int j = 0; j < 128; ++j) racc[j] = 0.f;
            const int nch = (int)((d.kt + 1) / 2);
            float sa_next = sa_arr[srow], sb_next[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) sb_next[q] = sb_arr[sgrp + q];
            for (int ch = 0; ch < nch; ++ch) {
                const int b = c & 1;
                float sc[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) sc[q] = sa_next * sb_next[q];
                if (ch + 1 < nch) {
                    sa_next = sa_arr[(int64_t)(ch + 1) * ld_sa + srow];
#pragma unroll
                    for (int q = 0; q < 4; ++q) sb_next[q] = sb_arr[(int64_t)(ch + 1) * ld_sb + sgrp + q];
                }
                const bool ok = mbar_wait_bounded(accf0 + 8 * b, (uint32_t)((c >> 1) & 1), kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) {
                    epi_ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < 128; j += 32) {
                    uint32_t r[32], r2[32];
                    tmem_ld32x2(lane_base + (uint32_t)(b * 256 + j), lane_base + (uint32_t)(b * 256 + 128 + j), r, r2);
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        racc[j + q] = fmaf(__uint_as_float(r[q]) + __uint_as_float(r2[q]), sc[j / 32], racc[j + q]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8 * b);
                ++c;
            }
            if (!epi_ok) break;
            // Coalesced store through this warp's 32 x 36 staging buffer.
            const float alpha = pr.alpha, beta = pr.beta;
            float *C = pr.C;
            const int64_t ldc = pr.ldc;
            const int M = (int)pr.m, N = (int)pr.n;
            const bool vec4 = reinterpret_cast<uintptr_t>(C) % 16 == 0 && ldc % 4 == 0;
            float *stg = reinterpret_cast<float *>(smem_raw + (sbase - raw) + kGtcStgOffset) + warp * 32 * kGtcStgLd;
            const int rr = lane >> 3, cc = (lane & 7) * 4;
#pragma unroll
            for (int jb = 0; jb < 128; jb += 32) {
#pragma unroll
                for (int q = 0; q < 32; q += 4)
                    *reinterpret_cast<float4 *>(stg + lane * kGtcStgLd + q) =
                        make_float4(alpha * racc[jb + q], alpha * racc[jb + q + 1], alpha * racc[jb + q + 2],
                                    alpha * racc[jb + q + 3]);
                __syncwarp();
                const int col = n0 + jb + cc;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int rl = it * 4 + rr;
                    const int row = m0 + warp * 32 + rl;
                    float4 v = *reinterpret_cast<const float4 *>(stg + rl * kGtcStgLd + cc);
                    if (row < M && col < N) {
                        float *cp = C + (int64_t)row * ldc + col;
                        if (N - col >= 4 && vec4) {
                            if (beta != 0.f) {
                                const float4 o = *reinterpret_cast<const float4 *>(cp);
                                v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                            }
                            *reinterpret_cast<float4 *>(cp) = v;
                        } else {
                            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (col + e < N) cp[e] = (beta != 0.f) ? vv[e] + beta * cp[e] : vv[e];
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    if (!epi_ok) s_fail = 1;
    pdl_trigger();
    __syncthreads();
    if (tid == 0) {
        // No MMA may still write tensor memory when it is freed, and no bulk
        // copy may still be landing when the CTA exits.
        if (!mbar_wait_bounded(doneb, 0u, kWaitLimitNs)) s_fail = 1;
        if (s_fail) {
            if (err) atomicOr(err, 1);
            for (int q = s_consumed; q < s_issued; ++q)
                (void)mbar_wait_bounded(full0 + 8 * (q % kGtcStages), (uint32_t)((q / kGtcStages) & 1), kWaitLimitNs);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

std::atomic<uint64_t> g_gtc_attr{0};

}  // namespace

int grouped_tc_launch(const pt_gemm_problem_t *problems, const pt_gemm_problem_t *problems_dev, int count,
                      cudaStream_t st) {
    int64_t tiles = 0, units = 0, bytes = 0;
    for (int i = 0; i < count; ++i) {
        tiles += gtc_tiles(problems[i]);
        units += gtc_units(problems[i]);
        bytes += gtc_region_bytes(problems[i]);
    }
    if (tiles == 0) return PT_OK;
    if (tiles > 0x7fffffff || units > 0x7fffffff) return set_error(PT_EUNSUPPORTED, 1, "too many tensor-core tiles");
    const int64_t header = gtc_align256((int64_t)kSkHeaderBytes);
    void *ws = nullptr;
    int rc = stream_workspace(st, (size_t)(header + gtc_plan_bytes(count) + bytes), false, &ws);
    if (rc != PT_OK) return rc;
    const GtcPlan pl = gtc_plan_at(static_cast<unsigned char *>(ws) + header, count);
    const int dev = current_device();
    const uint64_t bit = 1ull << (dev & 63);
    if (!(g_gtc_attr.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(gtc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGtcSmem);
        if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        g_gtc_attr.fetch_or(bit, std::memory_order_acq_rel);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    int *errw = err_word(dev);
    gtc_plan_kernel<<<1, 256, 0, st>>>(problems_dev, count, pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "grouped plan kernel: %s", cudaGetErrorString(e));
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cudaLaunchAttribute attr[1];
    unsigned nattr = 0;
    add_pdl_attr(attr, nattr);
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    cfg.stream = st;
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(units, (int64_t)sms * 8), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    e = cudaLaunchKernelEx(&cfg, gtc_split_kernel, problems_dev, count, pl);
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "grouped split kernel: %s", cudaGetErrorString(e));
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(tiles, sms), 1, 1);
    cfg.blockDim = dim3(kGtcThreads, 1, 1);
    cfg.dynamicSmemBytes = kGtcSmem;
    e = cudaLaunchKernelEx(&cfg, gtc_gemm_kernel, problems_dev, count, pl, errw);
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "grouped tensor-core kernel: %s", cudaGetErrorString(e));
    return PT_OK;
}

}  // namespace pt
