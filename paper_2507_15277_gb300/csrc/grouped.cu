// Persistent grouped SGEMM: many independent problems in one launch (SIMT
// tiles; problems given the tensor-core tile run in grouped_tc.cu).
//
// Each problem carries a tile configuration chosen on the host by the runtime
// selector (pt_grouped_plan maps the variant the loaded manifest picks for
// that problem's shape onto the nearest of the kernel's tile shapes).  A
// fixed grid of CTAs (resident on every SM) walks the concatenated tile list
// of all problems with a static stride; every CTA first builds the prefix sum
// of the problems' tile counts in shared memory, then finds the problem of
// each of its tiles by binary search and runs that problem's configuration
// (the same CTA tile code as the per-GEMM SIMT variants, cp.async staging,
// packed FP32x2 FMA).  No atomics and no workspace: the schedule is a pure
// function of the descriptor array.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "common.h"
#include "grouped_tc.cuh"
#include "launch.cuh"

namespace pt {
namespace {

// Tile configurations (all 256 threads; M-major A, any layout).
using G0 = Simt<64, 64, 16, 16, 32, 4, 4, 1, 4, 3, 1, 0, 0, 1>;    // 64 x 64, 16-byte loads
using G1 = Simt<128, 64, 16, 32, 32, 8, 4, 1, 4, 3, 1, 0, 0, 1>;   // 128 x 64
using G2 = Simt<128, 128, 8, 32, 64, 8, 8, 1, 4, 3, 1, 0, 0, 1>;   // 128 x 128
using G3 = Simt<64, 64, 16, 16, 32, 4, 4, 1, 1, 3, 1, 0, 0, 1>;    // 64 x 64, 4-byte loads (any alignment)
constexpr int kThreads = 256;
constexpr int kSmem = cmax(cmax(G0::SMEM_BYTES, G1::SMEM_BYTES), cmax(G2::SMEM_BYTES, G3::SMEM_BYTES));
static_assert(G0::THREADS == kThreads && G1::THREADS == kThreads && G2::THREADS == kThreads &&
                  G3::THREADS == kThreads,
              "one block size");

__host__ __device__ inline void tile_dims(int tile, int *bm, int *bn) {
    switch (tile) {
        case 0: *bm = G0::BM; *bn = G0::BN; break;
        case 1: *bm = G1::BM; *bn = G1::BN; break;
        case 2: *bm = G2::BM; *bn = G2::BN; break;
        default: *bm = G3::BM; *bn = G3::BN; break;
    }
}

__device__ inline int tiles_of(const pt_gemm_problem_t &p) {
    if (p.m <= 0 || p.n <= 0 || p.tile < 0 || p.tile > 3) return 0;
    int bm, bn;
    tile_dims(p.tile, &bm, &bn);
    return (int)((p.m + bm - 1) / bm) * (int)((p.n + bn - 1) / bn);
}

__global__ void __launch_bounds__(kThreads, 2)
    grouped_sgemm_kernel(const pt_gemm_problem_t *__restrict__ probs, int count, int *err) {
    __shared__ int s_prefix[PT_GROUPED_MAX + 1];
    __shared__ int s_part[kThreads];
    const int tid = threadIdx.x;
    const int per = (count + kThreads - 1) / kThreads;
    int local = 0;
    for (int i = 0; i < per; ++i) {
        const int p = tid * per + i;
        if (p < count) {
            const int t = tiles_of(probs[p]);
            s_prefix[p + 1] = t;
            local += t;
        }
    }
    s_part[tid] = local;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int w = 0; w < kThreads; ++w) {
            const int v = s_part[w];
            s_part[w] = run;
            run += v;
        }
        s_prefix[0] = 0;
    }
    __syncthreads();
    int run = s_part[tid];
    for (int i = 0; i < per; ++i) {
        const int p = tid * per + i;
        if (p < count) {
            run += s_prefix[p + 1];
            s_prefix[p + 1] = run;
        }
    }
    __syncthreads();
    const int total = s_prefix[count];

    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = count - 1;  // last problem whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const pt_gemm_problem_t &pr = probs[lo];
        GemmArgs a;
        a.A = pr.A;
        a.B = pr.B;
        a.C = pr.C;
        a.lda = pr.lda;
        a.ldb = pr.ldb;
        a.ldc = pr.ldc;
        a.M = (int)pr.m;
        a.N = (int)pr.n;
        a.K = (int)pr.k;
        a.alpha = pr.alpha;
        a.beta = pr.beta;
        a.ta = (pr.transA == 'T' || pr.transA == 't' || pr.transA == 'C' || pr.transA == 'c') ? 1 : 0;
        a.tb = (pr.transB == 'T' || pr.transB == 't' || pr.transB == 'C' || pr.transB == 'c') ? 1 : 0;
        a.err = err;
        int bm, bn;
        tile_dims(pr.tile, &bm, &bn);
        const int local_t = t - s_prefix[lo];
        const int tiles_n = (a.N + bn - 1) / bn;
        const int m0 = (local_t / tiles_n) * bm, n0 = (local_t % tiles_n) * bn;
        switch (pr.tile) {
            case 0: simt_body<G0>(a, nullptr, nullptr, m0, n0, 0); break;
            case 1: simt_body<G1>(a, nullptr, nullptr, m0, n0, 0); break;
            case 2: simt_body<G2>(a, nullptr, nullptr, m0, n0, 0); break;
            default: simt_body<G3>(a, nullptr, nullptr, m0, n0, 0); break;
        }
    }
}

int check_problem(const pt_gemm_problem_t &p, int i) {
    if (p.m < 0 || p.n < 0 || p.k < 0 || p.m > 0x7fffffff || p.n > 0x7fffffff || p.k > 0x7fffffff)
        return set_error(PT_EINVAL, 1, "problem %d: extents out of range", i);
    const char ta = p.transA, tb = p.transB;
    const bool tA = ta == 'T' || ta == 't' || ta == 'C' || ta == 'c';
    const bool tB = tb == 'T' || tb == 't' || tb == 'C' || tb == 'c';
    if (!tA && ta != 'N' && ta != 'n') return set_error(PT_EINVAL, 1, "problem %d: bad transA", i);
    if (!tB && tb != 'N' && tb != 'n') return set_error(PT_EINVAL, 1, "problem %d: bad transB", i);
    const int64_t need_a = tA ? p.m : p.k, need_b = tB ? p.k : p.n;
    if (p.lda < std::max<int64_t>(1, need_a) || p.ldb < std::max<int64_t>(1, need_b) ||
        p.ldc < std::max<int64_t>(1, p.n))
        return set_error(PT_EINVAL, 1, "problem %d: leading dimension too small", i);
    if (p.m > 0 && p.n > 0) {
        if (!p.C) return set_error(PT_EINVAL, 1, "problem %d: C is NULL", i);
        if (p.k > 0 && (!p.A || !p.B)) return set_error(PT_EINVAL, 1, "problem %d: A or B is NULL", i);
        if (p.tile < 0 || p.tile > PT_GROUPED_TILE_TC)
            return set_error(PT_EINVAL, 1, "problem %d: tile %d (call pt_grouped_plan)", i, p.tile);
        if (p.tile == PT_GROUPED_TILE_TC && p.k == 0)
            return set_error(PT_EINVAL, 1, "problem %d: the tensor-core tile needs K > 0", i);
        if (p.tile < 3) {
            const bool al = (reinterpret_cast<uintptr_t>(p.C) % 16 == 0) && p.ldc % 4 == 0 &&
                            (p.k == 0 || ((reinterpret_cast<uintptr_t>(p.A) % 16 == 0) && p.lda % 4 == 0 &&
                                          (reinterpret_cast<uintptr_t>(p.B) % 16 == 0) && p.ldb % 4 == 0));
            if (!al) return set_error(PT_EINVAL, 1, "problem %d: tile %d needs 16-byte aligned operands", i, p.tile);
        }
    }
    return PT_OK;
}

std::atomic<uint64_t> g_grouped_attr{0};

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" {

int pt_grouped_plan(pt_gemm_problem_t *problems, int count) {
    clear_error();
    if (count < 0 || (count > 0 && !problems)) return set_error(PT_EINVAL, 1, "bad problem array");
    const VariantEntry *tab = variant_table();
    for (int i = 0; i < count; ++i) {
        pt_gemm_problem_t &p = problems[i];
        p.tile = 3;
        if (p.m <= 0 || p.n <= 0) continue;
        const bool aligned = (reinterpret_cast<uintptr_t>(p.C) % 16 == 0) && p.ldc % 4 == 0 &&
                             (reinterpret_cast<uintptr_t>(p.A) % 16 == 0) && p.lda % 4 == 0 &&
                             (reinterpret_cast<uintptr_t>(p.B) % 16 == 0) && p.ldb % 4 == 0;
        if (!aligned) continue;
        const int v = pt_selected_variant(p.transA, p.transB, p.m, p.n, p.k > 0 ? p.k : 1, p.A, p.lda, p.B, p.ldb,
                                          p.C, p.ldc);
        if (v < 0) {
            clear_error();
            p.tile = 0;
            continue;
        }
        const pt_variant_desc_t &d = tab[v].desc;
        const int area = d.bm * d.bn;
        if (d.kind != 0 && p.k > 0) p.tile = PT_GROUPED_TILE_TC;  // tensor-core pick: the 3xF16 tile
        else p.tile = area >= 128 * 128 ? 2 : (area >= 128 * 64 ? 1 : 0);
    }
    return PT_OK;
}

int pt_sgemm_grouped(const pt_gemm_problem_t *problems, const pt_gemm_problem_t *problems_dev, int count,
                     void *stream) {
    clear_error();
    if (count < 0 || count > PT_GROUPED_MAX) return set_error(PT_EINVAL, 3, "count must be in [0, %d]", PT_GROUPED_MAX);
    if (count == 0) return PT_OK;
    if (!problems) return set_error(PT_EINVAL, 1, "problems is NULL");
    if (!problems_dev) return set_error(PT_EINVAL, 2, "problems_dev is NULL");
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        const int rc = check_problem(problems[i], i);
        if (rc != PT_OK) return rc;
        if (problems[i].m > 0 && problems[i].n > 0 && problems[i].tile != PT_GROUPED_TILE_TC) {
            int bm, bn;
            tile_dims(problems[i].tile, &bm, &bn);
            tiles += ((problems[i].m + bm - 1) / bm) * ((problems[i].n + bn - 1) / bn);
        }
    }
    if (tiles > 0x7fffffff) return set_error(PT_EUNSUPPORTED, 1, "too many tiles");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Tensor-core problems: plan, split and one persistent tensor-core kernel.
    int rc = grouped_tc_launch(problems, problems_dev, count, st);
    if (rc != PT_OK) return rc;
    if (tiles == 0) return PT_OK;
    const int dev = current_device();
    const uint64_t bit = 1ull << (dev & 63);
    if (!(g_grouped_attr.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(grouped_sgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        g_grouped_attr.fetch_or(bit, std::memory_order_acq_rel);
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_sgemm_kernel, kThreads, kSmem);
    if (sms <= 0) sms = 1;
    if (per_sm <= 0) per_sm = 1;
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, tiles);
    grouped_sgemm_kernel<<<(unsigned)grid, kThreads, kSmem, st>>>(problems_dev, count, nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : set_error(PT_ECUDA, 0, "grouped kernel: %s", cudaGetErrorString(e));
}

}  // extern "C"
