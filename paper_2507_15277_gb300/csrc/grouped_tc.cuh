// Grouped 3xF16 tensor-core SGEMM: the problems whose grouped tile is
// PT_GROUPED_TILE_TC run on the tensor cores inside one persistent kernel.
//
// The split of every such problem writes its FP16 planes in a tiled layout
// that the GEMM reads with plain bulk copies, so no tensor map is needed per
// problem: for each 128-row tile and 64-value k-tile there is one 32 KB block,
// plane h0 (128 rows x 128 bytes) then plane h1, each row's eight 16-byte
// chunks already in the order the tensor core's 128-byte swizzle expects
// (chunk c of row r at position c ^ (r % 8)).  Rows past M (N) and values of
// k past K are zeros.  The scales are those of the single-GEMM 3xF16 versions:
// per 128-k chunk, one per row of op(A) and one per 32 columns of op(B).
//
// A small plan kernel turns the caller's descriptor array (device copy) into
// prefix sums of tiles, split units and workspace bytes, so the schedule is a
// pure function of that array and graph replays need no host work.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pt_sgemm.h"

namespace pt {

constexpr int kGtcBlockBytes = 32768;  // one 128-row x 64-k tile, both planes

__host__ __device__ inline bool gtc_is_tc(const pt_gemm_problem_t &p) {
    return p.tile == PT_GROUPED_TILE_TC && p.m > 0 && p.n > 0 && p.k > 0;
}

struct GtcDims {
    int64_t mt, nt, kt, nch;  // 128-row tiles of M and N, 64-k tiles, 128-k chunks
};

__host__ __device__ inline GtcDims gtc_dims(const pt_gemm_problem_t &p) {
    GtcDims d;
    d.mt = (p.m + 127) / 128;
    d.nt = (p.n + 127) / 128;
    d.kt = (p.k + 63) / 64;
    d.nch = (p.k + 127) / 128;
    return d;
}

__host__ __device__ inline int64_t gtc_align256(int64_t b) { return (b + 255) / 256 * 256; }

// Bytes of problem p's workspace region: A blocks, B blocks, A row scales
// [chunk][mt * 128], B group scales [chunk][nt * 4].
__host__ __device__ inline int64_t gtc_a_bytes(const GtcDims &d) { return d.mt * d.kt * kGtcBlockBytes; }
__host__ __device__ inline int64_t gtc_b_bytes(const GtcDims &d) { return d.nt * d.kt * kGtcBlockBytes; }
__host__ __device__ inline int64_t gtc_sa_bytes(const GtcDims &d) { return gtc_align256(d.nch * d.mt * 128 * 4); }
__host__ __device__ inline int64_t gtc_sb_bytes(const GtcDims &d) { return gtc_align256(d.nch * d.nt * 4 * 4); }
__host__ __device__ inline int64_t gtc_region_bytes(const pt_gemm_problem_t &p) {
    if (!gtc_is_tc(p)) return 0;
    const GtcDims d = gtc_dims(p);
    return gtc_a_bytes(d) + gtc_b_bytes(d) + gtc_sa_bytes(d) + gtc_sb_bytes(d);
}
// Output tiles (128 x 128) and split units (32 rows x 256 values of k, of A
// and of op(B)^T) of problem p.
__host__ __device__ inline int64_t gtc_tiles(const pt_gemm_problem_t &p) {
    if (!gtc_is_tc(p)) return 0;
    const GtcDims d = gtc_dims(p);
    return d.mt * d.nt;
}
__host__ __device__ inline int64_t gtc_units(const pt_gemm_problem_t &p) {
    if (!gtc_is_tc(p)) return 0;
    const GtcDims d = gtc_dims(p);
    return (d.mt * 4 + d.nt * 4) * ((d.kt + 3) / 4);
}

// Plan written by the plan kernel at the start of the grouped workspace:
// tile_prefix[count + 1], unit_prefix[count + 1] (int), off[count + 1]
// (int64, byte offset of each problem's region from the regions' base).
struct GtcPlan {
    int *tile_prefix;
    int *unit_prefix;
    int64_t *off;
    unsigned char *regions;
};

__host__ __device__ inline int64_t gtc_plan_bytes(int count) {
    return gtc_align256((int64_t)(count + 1) * 4) * 2 + gtc_align256((int64_t)(count + 1) * 8);
}

__host__ __device__ inline GtcPlan gtc_plan_at(unsigned char *base, int count) {
    GtcPlan pl;
    pl.tile_prefix = reinterpret_cast<int *>(base);
    pl.unit_prefix = reinterpret_cast<int *>(base + gtc_align256((int64_t)(count + 1) * 4));
    pl.off = reinterpret_cast<int64_t *>(base + 2 * gtc_align256((int64_t)(count + 1) * 4));
    pl.regions = base + gtc_plan_bytes(count);
    return pl;
}

// Launches the plan, split and GEMM kernels for the problems whose tile is
// PT_GROUPED_TILE_TC (none: nothing is launched).  `problems` is the
// validated host array, `problems_dev` its device copy.  Uses the stream's
// library workspace after the stream-K header.
int grouped_tc_launch(const pt_gemm_problem_t *problems, const pt_gemm_problem_t *problems_dev, int count,
                      cudaStream_t st);

}  // namespace pt
