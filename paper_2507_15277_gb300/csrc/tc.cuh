// Split-precision tensor-core SGEMM variants for sm_103a (tcgen05 + TMEM + TMA).
//
// FP32 operands are split into low-precision planes whose products the 5th-
// generation tensor cores compute exactly and accumulate in FP32 in tensor
// memory:
//   3xTF32:  x = hi + lo, hi = RN_tf32(x), lo = RN_tf32(x - hi);
//            a*b ~ hi_a*hi_b + hi_a*lo_b + lo_a*hi_b      (kind::tf32, 3 MMAs)
//   BF16x3:  x = b0 + b1 + b2, b0 = RN_bf16(x), b1 = RN_bf16(x - b0),
//            b2 = RN_bf16(x - b0 - b1);
//            a*b ~ sum of the six b_i*b_j with i + j <= 2 (kind::f16 with BF16, 6 MMAs)
//   3xF16:   x' = x * 2^S (S per 256 values of k and row of op(A), or group
//            of 32 columns of op(B), so that the largest |x'| there is in
//            [2^14, 2^15)), x' = h0 + h1 on the FP16 grid (11-bit
//            significands, as TF32); a'*b' ~ h0 h0 + h0 h1 + h1 h0 (kind::f16
//            with F16, 3 MMAs at the BF16 rate); each 256-k partial product is
//            multiplied by 2^-S_A * 2^-S_B when it is drained.
// The dropped terms are O(2^-22) (3xTF32, 3xF16) and O(2^-24) (BF16x3)
// relative to |a*b| (3xF16: relative to the largest |a| of the row's chunk
// times the largest |b| of the 32 columns' chunk), so the
// result is FP32-accurate; these variants join the FP32 SIMT family as
// further versions of the same operation.
//
// Pipeline (a persistent CTA per SM walks the 128 x BN output tiles;
// stream-K versions share the last waves' tiles in 128-k chunks; split-K
// versions: one tile per cluster):
//   a split kernel writes the planes K-major into the library workspace;
//   producer warp (one lane): TMA loads of every plane's tile (3-D tensor maps
//                  over [plane][row][k], 128/64/32-byte swizzle), full/empty
//                  mbarriers per stage; fused versions load the FP32 tile of
//                  one operand instead (2-D map over the operand itself);
//   converter warps (fused versions only): split that FP32 tile into the
//                  operand's three BF16 planes in the stage, in the layout a
//                  swizzled TMA load would give, then hand the stage to the
//                  MMA warp;
//   MMA warp (one lane): tcgen05.mma (cta_group::1, M = 128, A and B
//                  K-major from shared-memory descriptors) into one of two
//                  TMEM accumulators; every 128 values of k (a "chunk") the
//                  accumulator is committed and the other buffer is used.
//                  The products are paired along N: the B planes of a stage
//                  are adjacent in shared memory, so planes j and j+1 form one
//                  2*BN-row operand and A_i x [B_j | B_j+1] is a single
//                  N = 2*BN MMA whose left half accumulates A_i B_j and right
//                  half A_i B_j+1.  The remaining products go to the right
//                  half.  Each A tile is then read fewer times per k step
//                  (shared-memory bandwidth is the limit at N = BN); the two
//                  halves are summed in FP32 by the epilogue;
//   epilogue warps (4 per 128 columns): tcgen05.ld of their 32 TMEM lanes
//                  (= rows) after each chunk, both halves added into FP32
//                  registers with IEEE round-to-nearest ("promotion": the
//                  tensor core's own accumulation, which is not IEEE
//                  round-to-nearest, then spans only 128 products),
//                  alpha/beta, coalesced stores to C through a small
//                  per-warp staging buffer.
// Every mbarrier wait is bounded; tensor memory is always freed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ptx.cuh"
#include "simt.cuh"
#include "split.cuh"

namespace pt {

template <int KIND_, int BN_, int STAGES_, int SPLITK_ = 1, int SWZ_ = 128, int STREAMK_ = 0, int FUSE_ = 0,
          int PAIR_ = 0>
struct Tc {
    static constexpr int KIND = KIND_, BM = 128, BN = BN_, STAGES = STAGES_, SPLITK = SPLITK_;
    // Stream-K (SPLITK == 1 only): the grid's CTAs split tiles x chunks into
    // equal contiguous ranges, so no SM idles in a last partial wave of
    // tiles; a tile shared by several CTAs is finished by the CTA that owns
    // its last chunk, which adds the others' FP32 partial tiles.
    static constexpr int STREAMK = STREAMK_;
    static_assert(STREAMK == 0 || SPLITK == 1, "stream-K replaces split-K");
    // Fused split (BF16x3): the producer loads FP32 tiles of one operand
    // itself and four converter warps write its three planes into the stage,
    // so that operand never passes through the split kernel.  FUSE = 1: B
    // (stored K x N, N contiguous; pays for small M); FUSE = 2: A (stored
    // M x K, K contiguous; pays for small N); FUSE = 3: both, so a call is a
    // single launch (pays for small problems, whose time is mostly the fixed
    // cost of each launch).
    static constexpr int FUSE = FUSE_;
    static constexpr bool FUSEB = FUSE == 1 || FUSE == 3, FUSEA = FUSE == 2 || FUSE == 3;
    static_assert(FUSE == 0 || KIND_ == kTcBf16x3, "fused split is BF16x3 only");
    // Two-CTA pair (cta_group::2): a cluster (2,1,1) computes 256 x BN tiles
    // with M = 256 MMAs that its even CTA issues.  Each CTA loads its 128 rows
    // of A and half of the tile's BN rows of op(B)^T, so a stage holds 3/4
    // (BN = 128) or 2/3 (BN = 256) of the bytes of a one-CTA stage for the
    // same MMA work per SM, and more stages fit.  The products are not paired
    // along N (three N = BN MMAs per k step): the two halves of B sit in
    // different CTAs.  Stream-K pairs share chunks per CTA pair.
    static constexpr bool PAIR = PAIR_ != 0;
    static_assert(!PAIR || (SPLITK_ == 1 && FUSE_ == 0 && (BN_ == 128 || BN_ == 256) && KIND_ != kTcBf16x3),
                  "pair versions: unfused, 128 or 256 columns, three products");
    static constexpr int TILE_M = PAIR ? 256 : 128;  // rows of a scheduled tile
    // 256-column tiles (three-product kinds, one CTA or a pair): every
    // product is one N = 256 MMA into a single accumulator of 256 columns (no
    // left / right halves), so a k step is three MMAs for twice the output of
    // a 128-column tile's two (N = 256 + N = 128), and the two buffers still
    // fit tensor memory.
    static constexpr bool MERGED = BN_ == 256;
    static_assert(!MERGED || (KIND_ != kTcBf16x3 && FUSE_ == 0 && SPLITK_ == 1),
                  "256-column tiles: three-product kinds, unfused, no split-K");
    static constexpr int B_ROWS = PAIR ? BN_ / 2 : BN_;  // rows of op(B)^T a CTA loads per tile
    // Bytes of k per tile row = the TMA / MMA swizzle span (128, 64 or 32).
    // A narrower row makes the stage smaller, so more stages fit and the
    // producer refills a smaller part of the pipeline at a time.
    static constexpr int SWZ = SWZ_;
    static_assert(SWZ == 128 || SWZ == 64 || SWZ == 32, "swizzle span");
    // Split-K: SPLITK CTAs of a cluster (1,1,SPLITK) split the k-tiles; their
    // FP32 partial tiles are summed through distributed shared memory in
    // cluster-rank order (the pipeline's shared memory is reused for them).
    static constexpr int RED_LD = BN + 4;
    static constexpr bool SCALED = KIND == kTcF16s;       // chunk scales applied when draining
    static constexpr int ELEM = KIND == kTcTf32 ? 4 : 2;  // bytes per plane element
    static constexpr int P = KIND == kTcBf16x3 ? 3 : 2;   // planes per operand
    static constexpr int BK = SWZ / ELEM;                 // one swizzle row per tile row
    static constexpr int KSTEP = 32 / ELEM;               // K of one MMA instruction (32 bytes)
    static constexpr int NPROD = KIND == kTcBf16x3 ? 6 : 3;
    // MMA instructions per k step after pairing along N (see tc_op).
    static constexpr int NOPS = (PAIR || MERGED) ? 3 : (KIND == kTcBf16x3 ? 4 : 2);
    // Promotion: the tensor-core accumulator is restarted every CHUNK_KT
    // k-tiles (CHUNK_K values of k) and added into FP32 registers with IEEE
    // round-to-nearest, so the accumulation error grows with CHUNK_K, not K.
    // 3xF16 drains every 256 values of k (its scales' chunk): its MMAs run at
    // twice the rate per k of the other kinds, so a 128-k chunk would leave
    // the epilogue half the time per drain.
    static constexpr int CHUNK_K = SCALED ? 256 : 128;
    static constexpr int CHUNK_KT = CHUNK_K / BK;
    static constexpr int A_PLANE_BYTES = BM * SWZ;
    static constexpr int B_PLANE_BYTES = B_ROWS * SWZ;
    // FP32 tiles of the fused operands after the planes: A as [BM][BK] (at
    // F32A_OFFSET), then B as [BK][BN] (at F32B_OFFSET).
    static constexpr int F32A_BYTES = FUSEA ? BM * BK * 4 : 0, F32B_BYTES = FUSEB ? BK * BN * 4 : 0;
    static constexpr int F32_BYTES = F32A_BYTES + F32B_BYTES;
    static constexpr int F32A_OFFSET = P * (A_PLANE_BYTES + B_PLANE_BYTES), F32B_OFFSET = F32A_OFFSET + F32A_BYTES;
    static constexpr int STAGE_BYTES = P * (A_PLANE_BYTES + B_PLANE_BYTES) + F32_BYTES;
    // bytes the TMA loads deliver per stage
    // (pair versions: both CTAs' loads complete on the even CTA's barrier)
    static constexpr int LOAD_BYTES =
        (PAIR ? 2 : 1) * ((FUSEA ? F32A_BYTES : P * A_PLANE_BYTES) + (FUSEB ? F32B_BYTES : P * B_PLANE_BYTES));
    static constexpr int BAR_OFFSET = STAGES * STAGE_BYTES;
    // Barriers (full, empty per stage; converted per stage when FUSEB; two
    // accumulator-full, two accumulator-empty, MMA-done) and the TMEM address
    // slot.
    static constexpr int BAR_BYTES = 8 * ((FUSE ? 3 : 2) * STAGES + 6);

    // Accumulator buffer: 2*BN columns (left half, right half); two buffers.
    static constexpr int ACC_COLS = MERGED ? BN : 2 * BN;
    static constexpr int TMEM_COLS = 2 * ACC_COLS;
    // Epilogue warps: 4 per 128 columns (a warp reads its 32 TMEM lanes), each
    // thread owns one row and COLS columns; then one producer and one MMA warp.
    static constexpr int COL_GROUPS = BN >= 128 ? BN / 128 : 1;
    static constexpr int COLS = BN / COL_GROUPS;
    static constexpr int EPI_WARPS = 4 * COL_GROUPS;
    static constexpr int PRODUCER_WARP = EPI_WARPS, MMA_WARP = EPI_WARPS + 1;
    // Converter warps: four for 64-column tiles; two for 128-column tiles,
    // whose epilogue threads need the larger per-thread register budget of a
    // 256-thread CTA.
    static constexpr int CONV_WARP0 = EPI_WARPS + 2, CONV_WARPS = FUSE ? (BN >= 128 ? 2 : 4) : 0;
    static constexpr int THREADS = 32 * (EPI_WARPS + 2 + CONV_WARPS);
    // Fused versions: the epilogue warps convert too.  They drain the
    // accumulator only once per 128 values of k, so between drains they take
    // an equal share of every stage's conversion next to the converter warps.
    // Not in 64-column stream-K versions: with the stream-K epilogue the
    // conversion code no longer fits the registers of a 320-thread CTA.
    static constexpr bool EPI_CONV = FUSE != 0 && !(STREAMK != 0 && BN == 64);
    static constexpr int CONV_ALL_WARPS = FUSE ? (EPI_CONV ? EPI_WARPS : 0) + CONV_WARPS : 0;
    static constexpr int CONV_THREADS = 32 * CONV_ALL_WARPS;
    // Epilogue staging (when it fits): each epilogue warp transposes its 32
    // rows through a STG_ROWS x STG_LD float buffer, 32 columns at a time, so
    // that C is written in whole 128-byte row segments; 16 rows at a time
    // (two passes) where a 32-row buffer does not fit beside the pipeline.
    static constexpr int STG_LD = 36;
    static constexpr int STG_OFFSET = (BAR_OFFSET + BAR_BYTES + 15) / 16 * 16;
    static constexpr int STG_ROWS = STG_OFFSET + EPI_WARPS * 32 * STG_LD * 4 + 1024 <= 232448 ? 32 : 16;
    static constexpr int STG_WARP_FLOATS = STG_ROWS * STG_LD;
    static constexpr int STG_END = STG_OFFSET + EPI_WARPS * STG_WARP_FLOATS * 4;
    static constexpr bool STAGE_C = STG_END + 1024 <= 232448;
    // TMA-store staging (SPLITK == 1, beta = 0, C 16-byte aligned): per
    // epilogue warp TSTG_BUFS buffers holding one 32 x 32 FP32 box of C in the
    // 128-byte swizzled layout (1024-byte aligned), two where they fit, so the
    // warp fills one while the TMA engine still reads the other.  It shares
    // the region after the barriers with the padded staging buffers above (a
    // launch uses one of the two).
    static constexpr int TSTG_OFFSET = (BAR_OFFSET + BAR_BYTES + 1023) / 1024 * 1024;
    static constexpr int TSTG_BUFS = SPLITK_ != 1                                              ? 0
                                     : TSTG_OFFSET + EPI_WARPS * 2 * 4096 + 1024 <= 232448 ? 2
                                     : TSTG_OFFSET + EPI_WARPS * 4096 + 1024 <= 232448     ? 1
                                                                                           : 0;
    static constexpr int TSTG_END = TSTG_OFFSET + EPI_WARPS * TSTG_BUFS * 4096;
    static constexpr int STG_USED = STAGE_C ? STG_END : STG_OFFSET;
    static constexpr int SMEM_BYTES = (STG_USED > TSTG_END ? STG_USED : TSTG_END) + 1024;
    // Instruction descriptor: D = F32 (bits 4-5 = 1), A/B format (bits 7-9,
    // 10-12: TF32 = 2, BF16 = 1, F16 = 0), both K-major (bits 15, 16 = 0),
    // N >> 3 at bit 17, M >> 4 at bit 24.
    static constexpr uint32_t FMT = KIND == kTcTf32 ? 2u : (KIND == kTcBf16x3 ? 1u : 0u);
    static constexpr uint32_t IDESC =
        (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TILE_M >> 4) << 24);
    static constexpr uint32_t IDESC_W =
        (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)((2 * BN) >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    static_assert(BN == 32 || BN == 64 || BN == 128 || MERGED, "N of the MMA (2*BN <= 256, a multiple of 16)");
    static_assert(FUSE == 0 || BN >= 64, "fused versions use 64- or 128-column tiles");
    static_assert(SPLITK == 1 || BM * RED_LD * 4 <= BAR_OFFSET, "split-K partial tile fits the pipeline memory");
    static_assert(BM % SPLITK == 0, "split-K reduction slices rows");
    // Consecutive CTAs walk GROUP_M tile rows down before moving right, so a
    // wave's A and B panels stay in L2.
    // (256 x 256 pair tiles: 8 rows of pairs, about the square root of the
    // pairs in a wave, which minimises the A and B panels a wave reads.)
    static constexpr int GROUP_M = PAIR && !MERGED ? 4 : 8;
    static_assert(TMEM_COLS <= 512, "tensor memory columns");
    static_assert(EPI_WARPS <= 8, "stream-K flag slots per CTA");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// MMA q of a k step: A plane pa times B plane pb.  wide: N = 2*BN over the
// adjacent planes pb and pb+1 (left half of the accumulator += A_pa B_pb,
// right half += A_pa B_pb+1); otherwise N = BN into the right half.  The
// first MMA is wide, so the zeroing of a chunk's first k step covers both
// halves.
//   3xTF32, 3xF16: A0 [B0|B1] (hh, hl), A1 B0 (lh).
//   BF16x3: A0 [B0|B1], A1 [B0|B1], A0 B2, A2 B0  (the six b_i b_j, i+j <= 2).
template <int KIND>
__device__ __forceinline__ void tc_op(int q, int &pa, int &pb, bool &wide) {
    if constexpr (KIND != kTcBf16x3) {
        constexpr int a[2] = {0, 1}, b[2] = {0, 0};
        pa = a[q];
        pb = b[q];
        wide = q == 0;
    } else {
        constexpr int a[4] = {0, 1, 0, 2}, b[4] = {0, 0, 2, 0};
        pa = a[q];
        pb = b[q];
        wide = q < 2;
    }
}

// Shared-memory matrix descriptor of a K-major tile whose rows are one
// swizzle span (SWZ = 128, 64 or 32 bytes): start address >> 4 (bits 0-13),
// leading byte offset 16 B (unused for swizzled K-major layouts), stride byte
// offset 8 rows x SWZ bytes between 8-row groups (bits 32-45), descriptor
// version 1 (bit 46), layout type at bits 61-63 (2 = 128-byte swizzle,
// 4 = 64-byte, 6 = 32-byte swizzle).  Tile bases are 1024-byte aligned, so the
// base-offset field is 0.  Successive MMA K steps within a row advance the
// start address by 32 bytes.
template <int SWZ>
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
    constexpr uint64_t layout = SWZ == 128 ? 2 : (SWZ == 64 ? 4 : 6);
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)((8 * SWZ) >> 4) << 32) |
           ((uint64_t)1 << 46) | (layout << 61);
}

// TMA tile store of a 2-D box from shared memory (tracked per issuing
// thread in bulk groups), and the waits for those groups: `.read` until the
// shared memory of all but the newest N groups has been read, plain until
// their global writes are done.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

struct TcArgs {
    float *C;
    int64_t ldc;
    int M, N, K;
    float alpha, beta;
    int vec4;  // C and ldc allow 16-byte stores
    int tma_c;  // C is stored through mapC by the TMA engine (beta = 0, C and ldc 16-byte aligned)
    int *err;
    // Stream-K: words[0] = launches completed on this workspace (the epoch),
    // words[1] = CTAs of this launch that have finished, words[kSkFlags + 8b
    // + w] = epoch + 1 once epilogue warp w of CTA b has written its rows of
    // CTA b's partial tile (partials + b * BM * BN, row-major BM x BN).
    unsigned *sk_words;
    float *sk_partials;
    // 3xF16: 2^-S of chunk c (256 values of k) of row r of op(A) at
    // scale_a[c * ld_sa + r] (ld_sa >= round_up(M, 128)), and of the 32-column
    // group g of op(B) at scale_b[c * ld_sb + g] (ld_sb >= round_up(N, 128) / 32).
    const float *scale_a;
    const float *scale_b;
    int64_t ld_sa, ld_sb;
    // Stream-K finisher's wait for a contributor's flag: time limit (ns) and
    // the offset of the awaited value from epoch + 1 (0; 1 only under the
    // test hook pt_debug_streamk_wait, which makes the value one nobody writes).
    uint64_t sk_wait_ns;
    unsigned sk_wait_bias;
};

constexpr int kSkFlags = 32;                  // first flag word
constexpr int kSkMaxGrid = 2048;              // flag slots (CTAs)
constexpr int kSkFlagsPerCta = 8;             // one per epilogue warp (at most 8)
constexpr size_t kSkHeaderBytes = 4 * (kSkFlags + kSkFlagsPerCta * kSkMaxGrid);

// Work of one CTA as segments (tile t, chunks [c0, c1) of the tile's k range;
// a chunk is 128 values of k).  Tile mode: tiles t_first, t_first + t_step,
// ..., whole.  Stream-K: first ndp whole tiles in the same strided order
// (all but the last full wave of tiles, which keeps concurrently processed
// tiles close together in L2), then the chunk range [lo, hi) of the
// remaining tiles x chunks, which the CTAs share equally, visited tile by
// tile from the last to the first: the partial tile a CTA contributes to a
// later CTA's tile is written first and the tile it finishes comes last.
struct TcWork {
    int nch;
    int t_first, t_step, tiles;
    bool streamk;
    int ndp, sk_tile0;  // stream-K: whole tiles per CTA; first tile of the shared part
    int64_t lo, hi;     // stream-K: chunk range within the shared part
    // Stream-K share of unit `unit` of G (a unit is a CTA, or a CTA pair):
    // whole tiles for all but the last full wave, then the rest (one to two
    // waves' worth) cut into G equal contiguous chunk ranges.  nch and tiles
    // are set first.
    __host__ __device__ void streamk_init(int G, int unit) {
        const int full_waves = tiles / G;
        ndp = full_waves >= 2 ? full_waves - 1 : 0;
        sk_tile0 = ndp * G;
        const int64_t W = (int64_t)(tiles - sk_tile0) * nch;
        lo = (int64_t)unit * W / G;
        hi = ((int64_t)unit + 1) * W / G;
    }
    __host__ __device__ int count() const {
        if (streamk) return ndp + (hi > lo ? (int)((hi - 1) / nch - lo / nch + 1) : 0);
        return t_first < tiles ? (tiles - 1 - t_first) / t_step + 1 : 0;
    }
    __host__ __device__ void seg(int i, int &t, int &c0, int &c1) const {
        if (!streamk || i < ndp) {
            t = t_first + i * t_step;
            c0 = 0;
            c1 = nch;
            return;
        }
        const int u_tile = (int)((hi - 1) / nch) - (i - ndp);
        t = sk_tile0 + u_tile;
        const int64_t base = (int64_t)u_tile * nch;
        c0 = (int)((lo > base ? lo : base) - base);
        c1 = (int)((hi < base + nch ? hi : base + nch) - base);
    }
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Fused split: converting thread ct (0 <= ct < V::CONV_THREADS) writes its
// share of the stage's three BF16 planes of each fused operand from the FP32
// tile the producer loaded, K-major in the swizzled layout a TMA load would
// produce (16-byte chunk c of plane row r at chunk c ^ ((r * SWZ / 128) &
// (SWZ / 16 - 1))).  x = b0 + b1 + b2 with b0 = RN_bf16(x), b1 = RN_bf16(x - b0),
// b2 = RN_bf16(x - b0 - b1); both subtractions are exact.
template <class V>
__device__ __forceinline__ void tc_convert_stage(unsigned char *stp, int ct) {
    constexpr int BK = V::BK, BN = V::BN, P = V::P, KC = BK / 8, NCT = V::CONV_THREADS;
    if constexpr (V::FUSEB) {
        const float *bf = reinterpret_cast<const float *>(stp + V::F32B_OFFSET);
        unsigned char *bp = stp + P * V::A_PLANE_BYTES;
        // B: lanes take consecutive n of one k chunk (the FP32 tile is
        // [k][n]) and each writes one 16-byte chunk of every plane.
#pragma unroll 2
        for (int it = ct; it < BN * KC; it += NCT) {
            const int n = it % BN, kc = it / BN;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = bf[(kc * 8 + e) * BN + n];
            uint32_t b[3][4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float v0 = x[e], v1 = x[e + 1];
#pragma unroll
                for (int pl = 0; pl < 3; ++pl) {
                    const uint32_t q = bf16x2_rn(v0, v1);
                    b[pl][e / 2] = q;
                    v0 -= bf16_lo_f32(q);
                    v1 -= bf16_hi_f32(q);
                }
            }
            const int sw = (n * V::SWZ / 128) & (V::SWZ / 16 - 1);
            const int off = n * V::SWZ + ((kc ^ sw) << 4);
#pragma unroll
            for (int pl = 0; pl < 3; ++pl)
                *reinterpret_cast<uint4 *>(bp + pl * V::B_PLANE_BYTES + off) =
                    make_uint4(b[pl][0], b[pl][1], b[pl][2], b[pl][3]);
        }
    }
    if constexpr (V::FUSEA) {
        // A: consecutive lanes read consecutive 16-byte pieces of the [m][k]
        // tile (no bank conflicts); a piece is four k values, half of one
        // 16-byte plane chunk.
        const float *bf = reinterpret_cast<const float *>(stp + V::F32A_OFFSET);
        unsigned char *bp = stp;
        constexpr int HC = 2 * KC;  // pieces per row
#pragma unroll 2
        for (int it = ct; it < V::BM * HC; it += NCT) {
            const int n = it / HC, h = it % HC;
            const float4 x4 = *reinterpret_cast<const float4 *>(bf + n * BK + h * 4);
            const float x[4] = {x4.x, x4.y, x4.z, x4.w};
            uint32_t b[3][2];
#pragma unroll
            for (int e = 0; e < 4; e += 2) {
                float v0 = x[e], v1 = x[e + 1];
#pragma unroll
                for (int pl = 0; pl < 3; ++pl) {
                    const uint32_t q = bf16x2_rn(v0, v1);
                    b[pl][e / 2] = q;
                    v0 -= bf16_lo_f32(q);
                    v1 -= bf16_hi_f32(q);
                }
            }
            const int sw = (n * V::SWZ / 128) & (V::SWZ / 16 - 1);
            const int off = n * V::SWZ + (((h >> 1) ^ sw) << 4) + ((h & 1) << 3);
#pragma unroll
            for (int pl = 0; pl < 3; ++pl)
                *reinterpret_cast<uint2 *>(bp + pl * V::A_PLANE_BYTES + off) = make_uint2(b[pl][0], b[pl][1]);
        }
    }
    // Generic-proxy writes become visible to the tensor core's (async-proxy)
    // reads before the stage is handed over.
    fence_proxy_async_smem();
}

// Tile coordinates of 1-D tile index t: consecutive indices walk GROUP_M
// tile rows down before moving right (keeps a wave's panels in L2).
template <class V>
__device__ __forceinline__ void tc_tile_coords(int t, int tiles_m, int tiles_n, int &m0, int &n0) {
    const int per_group = V::GROUP_M * tiles_n;
    const int first_m = (t / per_group) * V::GROUP_M;
    const int gsize = tiles_m - first_m < V::GROUP_M ? tiles_m - first_m : V::GROUP_M;
    const int r = t % per_group;
    m0 = (first_m + r % gsize) * V::TILE_M;
    n0 = (r / gsize) * V::BN;
}

// This CTA's rows of tile t: pair versions split the 256 rows between the
// two CTAs of the cluster by rank.
template <class V>
__device__ __forceinline__ void tc_cta_coords(int t, int tiles_m, int tiles_n, uint32_t rank, int &m0, int &n0) {
    tc_tile_coords<V>(t, tiles_m, tiles_n, m0, n0);
    if constexpr (V::PAIR) m0 += (int)rank * V::BM;
}

// SPLITK == 1: persistent; CTA b computes tiles b, b + gridDim.x, ...  The
// stage / phase and chunk / buffer counters run on across tiles, so the
// producer and the MMA warp start the next tile while the epilogue warps are
// still storing the previous one.  SPLITK > 1: one tile per cluster of CTAs.
template <class V>
__global__ void __launch_bounds__(V::THREADS, 1)
    tc_sgemm_kernel(const TcArgs args, const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapC) {
    constexpr int STAGES = V::STAGES, BK = V::BK, BN = V::BN, P = V::P, CKT = V::CHUNK_KT, COLS = V::COLS;
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_fail, s_issued, s_consumed, s_peer_issued;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    const uint32_t full0 = sbase + V::BAR_OFFSET;  // STAGES: TMA landed
    const uint32_t empty0 = full0 + 8 * STAGES;    // STAGES: MMAs done reading
    const uint32_t conv0 = empty0 + 8 * STAGES;    // STAGES (FUSE): fused operand's planes written
    const uint32_t accf0 = conv0 + (V::FUSE ? 8 * STAGES : 0);  // 2: accumulator buffer ready
    const uint32_t acce0 = accf0 + 16;             // 2: accumulator buffer drained
    const uint32_t doneb = acce0 + 16;             // every issued MMA finished
    const uint32_t tslot = doneb + 8;
    const volatile uint32_t *tslot_ptr =
        reinterpret_cast<const volatile uint32_t *>(smem_raw + (tslot - raw));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_m = (args.M + V::TILE_M - 1) / V::TILE_M, tiles_n = (args.N + BN - 1) / BN;
    const int tiles = tiles_m * tiles_n;
    // Pair versions: the cluster (2,1,1) is the scheduling unit; rank 0 issues the MMAs.
    const uint32_t rank = V::PAIR ? cluster_ctarank() : 0u;
    const int t_first = V::PAIR ? (int)blockIdx.x / 2 : (int)blockIdx.x;
    // K range (k-tiles) of this CTA; the same for every tile.
    const int kt_total = (args.K + BK - 1) / BK;
    int kt0 = 0, nkt = kt_total;
    if constexpr (V::SPLITK > 1) {
        int per = (kt_total + V::SPLITK - 1) / V::SPLITK;
        // 3xF16: a CTA's k range starts on a 128-k chunk, so its chunks are
        // the split kernel's scale chunks.
        if constexpr (V::SCALED) per = (per + CKT - 1) / CKT * CKT;
        kt0 = (int)blockIdx.z * per;
        const int kt_end = kt0 + per < kt_total ? kt0 + per : kt_total;
        nkt = kt_end > kt0 ? kt_end - kt0 : 0;
    }
    const int nchunks = (nkt + CKT - 1) / CKT;
    TcWork work;
    work.nch = nchunks;
    work.t_first = t_first;
    work.t_step = V::SPLITK > 1 ? tiles : (V::PAIR ? (int)gridDim.x / 2 : (int)gridDim.x);  // split-K: one tile
    work.tiles = tiles;
    work.streamk = V::STREAMK != 0;
    // Stream-K: the scheduling unit is a CTA, or a CTA pair in pair versions
    // (both CTAs of a pair have the same work; each keeps its own
    // partial-tile slot, blockIdx.x).
    const int G = V::PAIR ? (int)gridDim.x / 2 : (int)gridDim.x;
    const int unit = t_first;
    work.streamk_init(G, unit);
    const int64_t W_sk = (int64_t)(tiles - work.sk_tile0) * nchunks;
    const int nseg = work.count();

    if (tid == 0) {
        prefetch_tensormap(&mapA);
        prefetch_tensormap(&mapB);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
            if (V::FUSE) mbar_init(conv0 + 8 * s, V::CONV_ALL_WARPS);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, (V::PAIR ? 2 : 1) * V::EPI_WARPS);  // pair: both CTAs' drains
        }
        mbar_init(doneb, 1);
        fence_mbarrier_init();
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        s_peer_issued = 0;
    }
    if (warp == 0) {
        if constexpr (V::PAIR) {
            tmem_alloc_pair(tslot, V::TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tslot, V::TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (V::PAIR) cluster_sync();  // the peer's barriers are initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *tslot_ptr;
    // The prologue above touches no global memory; from here on the previous
    // kernel of the stream (the split) must have completed.
    pdl_wait();

    const float alpha = args.alpha, beta = args.beta;
    float racc[COLS];
    bool epi_ok = true;

    if (warp == V::PRODUCER_WARP) {
        if (lane == 0) {
            int g = 0;  // k-tiles issued so far (all segments)
            bool ok = true;
            for (int i = 0; ok && i < nseg; ++i) {
                int t, c0, c1;
                work.seg(i, t, c0, c1);
                int m0, n0;
                tc_cta_coords<V>(t, tiles_m, tiles_n, rank, m0, n0);
                const int nb = n0 + (int)rank * V::B_ROWS;  // pair versions: this CTA's half of the B rows
                const int kt_end = c1 * CKT < nkt ? c1 * CKT : nkt;
                for (int kt = c0 * CKT; kt < kt_end; ++kt, ++g) {
                    const int s = g % STAGES, u = g / STAGES;
                    if (g >= STAGES && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)((u - 1) & 1), kWaitLimitNs)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + s * V::STAGE_BYTES;
                    if constexpr (V::PAIR) {
                        // Both CTAs' copies complete on the even CTA's barrier, which
                        // expects the bytes of both.
                        const uint32_t lead_full = mapa_shared(full0 + 8 * s, 0u);
                        if (rank == 0) mbar_arrive_expect_tx(full0 + 8 * s, (uint32_t)V::LOAD_BYTES);
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            tma_load_3d_pair(st + p * V::A_PLANE_BYTES, &mapA, lead_full, (kt0 + kt) * BK, m0, p);
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            tma_load_3d_pair(st + P * V::A_PLANE_BYTES + p * V::B_PLANE_BYTES, &mapB, lead_full,
                                             (kt0 + kt) * BK, nb, p);
                        continue;
                    } else {
                        mbar_arrive_expect_tx(full0 + 8 * s, (uint32_t)V::LOAD_BYTES);
                    }
                    if constexpr (V::FUSEA) {
                        // FP32 tile of A: BM rows, BK columns of k (2-D map over A itself).
                        tma_load_2d(st + V::F32A_OFFSET, &mapA, full0 + 8 * s, (kt0 + kt) * BK, m0);
                    } else {
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            tma_load_3d(st + p * V::A_PLANE_BYTES, &mapA, full0 + 8 * s, (kt0 + kt) * BK, m0, p);
                    }
                    if constexpr (V::FUSEB) {
                        // FP32 tile of B: BK rows of k, BN columns of n (2-D map over B itself).
                        tma_load_2d(st + V::F32B_OFFSET, &mapB, full0 + 8 * s, n0, (kt0 + kt) * BK);
                    } else {
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            tma_load_3d(st + P * V::A_PLANE_BYTES + p * V::B_PLANE_BYTES, &mapB, full0 + 8 * s,
                                        (kt0 + kt) * BK, n0, p);
                    }
                }
            }
            s_issued = g;
            // Every load of this CTA is issued: the next kernel of the stream
            // may be scheduled (on SMs this grid leaves free; it waits for this
            // grid to complete before it touches memory).
            pdl_trigger();
        }
    } else if (warp == V::MMA_WARP) {
        if (lane == 0 && rank == 0) {  // pair versions: the even CTA issues for both
            int g = 0, c = 0, b = 0;  // k-tiles consumed, chunks started (all segments)
            bool ok = true;
            for (int i = 0; ok && i < nseg; ++i) {
                int t, c0, c1;
                work.seg(i, t, c0, c1);
                const int kt_end = c1 * CKT < nkt ? c1 * CKT : nkt;
                for (int kt = c0 * CKT; kt < kt_end; ++kt, ++g) {
                    const int s = g % STAGES, u = g / STAGES;
                    const bool first = (kt % CKT) == 0;
                    if (first) {
                        b = c & 1;
                        // Buffer b was last used by chunk c - 2; wait until it is drained.
                        const uint32_t par = (uint32_t)(((c >> 1) - 1) & 1);
                        if (c >= 2 && !(V::PAIR ? mbar_wait_cluster_bounded(acce0 + 8 * b, par, kWaitLimitNs)
                                                : mbar_wait_bounded(acce0 + 8 * b, par, kWaitLimitNs))) {
                            s_fail = 1;
                            ok = false;
                            break;
                        }
                    }
                    if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)(u & 1), kWaitLimitNs) ||
                        (V::FUSE && !mbar_wait_bounded(conv0 + 8 * s, (uint32_t)(u & 1), kWaitLimitNs))) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * V::STAGE_BYTES;
                    const uint32_t dt = tmem + (uint32_t)(b * V::ACC_COLS);
                    if constexpr (V::PAIR) {
                        // A0 B0 into the left half; A0 B1 and A1 B0 into the right half
                        // (256-column pairs: all three into the one accumulator).
#pragma unroll
                        for (int kk = 0; kk < BK / V::KSTEP; ++kk) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                                const uint64_t ad =
                                    kmajor_desc<V::SWZ>(st + pa * V::A_PLANE_BYTES) + (uint64_t)(2 * kk);
                                const uint64_t bd =
                                    kmajor_desc<V::SWZ>(st + P * V::A_PLANE_BYTES + pb * V::B_PLANE_BYTES) +
                                    (uint64_t)(2 * kk);
                                const bool zero = first && kk == 0 && (V::MERGED ? q == 0 : q < 2);
                                tc_mma_pair<V::KIND>((V::MERGED || q == 0) ? dt : dt + (uint32_t)BN, ad, bd, V::IDESC,
                                                     zero ? 0u : 1u);
                            }
                        }
                        tc_commit_pair(empty0 + 8 * s);
                        if ((kt % CKT) == CKT - 1 || kt == kt_end - 1) {
                            tc_commit_pair(accf0 + 8 * b);
                            ++c;
                        }
                    } else if constexpr (V::MERGED) {
                        // A0 B0, A0 B1, A1 B0, each N = 256, into the same columns.
#pragma unroll
                        for (int kk = 0; kk < BK / V::KSTEP; ++kk) {
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                                const uint64_t ad =
                                    kmajor_desc<V::SWZ>(st + pa * V::A_PLANE_BYTES) + (uint64_t)(2 * kk);
                                const uint64_t bd =
                                    kmajor_desc<V::SWZ>(st + P * V::A_PLANE_BYTES + pb * V::B_PLANE_BYTES) +
                                    (uint64_t)(2 * kk);
                                tc_mma<V::KIND>(dt, ad, bd, V::IDESC, (first && kk == 0 && q == 0) ? 0u : 1u);
                            }
                        }
                        tc_commit(empty0 + 8 * s);
                        if ((kt % CKT) == CKT - 1 || kt == kt_end - 1) {
                            tc_commit(accf0 + 8 * b);
                            ++c;
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / V::KSTEP; ++kk) {
#pragma unroll
                            for (int q = 0; q < V::NOPS; ++q) {
                                int pa, pb;
                                bool wide;
                                tc_op<V::KIND>(q, pa, pb, wide);
                                const uint64_t ad =
                                    kmajor_desc<V::SWZ>(st + pa * V::A_PLANE_BYTES) + (uint64_t)(2 * kk);
                                const uint64_t bd =
                                    kmajor_desc<V::SWZ>(st + P * V::A_PLANE_BYTES + pb * V::B_PLANE_BYTES) +
                                    (uint64_t)(2 * kk);
                                tc_mma<V::KIND>(wide ? dt : dt + (uint32_t)BN, ad, bd, wide ? V::IDESC_W : V::IDESC,
                                                (first && kk == 0 && q == 0) ? 0u : 1u);
                            }
                        }
                        tc_commit(empty0 + 8 * s);  // stage s may be refilled once these MMAs finish
                        if ((kt % CKT) == CKT - 1 || kt == kt_end - 1) {
                            tc_commit(accf0 + 8 * b);  // chunk c complete
                            ++c;
                        }
                    }
                }
            }
            if constexpr (V::PAIR)
                tc_commit_pair(doneb);  // every MMA issued so far (also after a failure), in both CTAs
            else
                tc_commit(doneb);  // every MMA issued so far (also after a failure)
            s_consumed = g;
        }
    } else if (V::FUSE && warp >= V::CONV_WARP0) {
        // Converter warps: their share of every stage's conversion (the
        // epilogue warps take the rest).
        if constexpr (V::FUSE) {
            const int ct = (V::EPI_CONV ? 32 * V::EPI_WARPS : 0) + (tid - 32 * V::CONV_WARP0);
            int g = 0;
            bool ok = true;
            for (int i = 0; ok && i < nseg; ++i) {
                int t, c0, c1;
                work.seg(i, t, c0, c1);
                const int kt_end = c1 * CKT < nkt ? c1 * CKT : nkt;
                for (int kt = c0 * CKT; kt < kt_end; ++kt, ++g) {
                    const int s = g % STAGES, u = g / STAGES;
                    const bool landed = mbar_wait_bounded(full0 + 8 * s, (uint32_t)(u & 1), kWaitLimitNs);
                    if (!__all_sync(0xffffffffu, landed)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_convert_stage<V>(smem_raw + (sbase - raw) + s * V::STAGE_BYTES, ct);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(conv0 + 8 * s);
                }
            }
        }
    } else {
        // Epilogue warps: drain each chunk's accumulator into FP32 registers,
        // then store the tile (SPLITK == 1) or keep it for the reduction.
        // Fused versions (EPI_CONV): first convert this warp's share of chunk ch's
        // stages, then drain chunk ch - 1, so the conversions the MMAs wait
        // for never queue behind a drain; the drain only waits for MMAs of
        // stages converted earlier.
        const int sub = warp & 3, grp = warp >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(grp * COLS);
        int c = 0;  // chunks drained (all segments)
        int g = 0;  // k-tiles converted (fused versions)
        unsigned epoch1 = 0;  // stream-K: this launch's flag value
        int sblk = 0;         // C boxes handed to the TMA engine (TMA-store epilogue)
        if constexpr (V::STREAMK != 0) epoch1 = ld_acquire_u32(args.sk_words) + 1u;
        for (int i = 0; epi_ok && i < nseg; ++i) {
            int t, c0, c1;
            work.seg(i, t, c0, c1);
#pragma unroll
            for (int j = 0; j < COLS; ++j) racc[j] = 0.f;
            // 3xF16: this thread's row scale and its COLS / 32 column-group
            // scales for chunk ch, loaded one chunk ahead.
            constexpr int NG = V::SCALED ? COLS / 32 : 1;
            int64_t srow = 0, sgrp = 0;
            float sa_next = 1.f, sb_next[NG];
#pragma unroll
            for (int q = 0; q < NG; ++q) sb_next[q] = 1.f;
            if constexpr (V::SCALED) {
                int sm0, sn0;
                tc_cta_coords<V>(t, tiles_m, tiles_n, rank, sm0, sn0);
                srow = sm0 + sub * 32 + lane;
                sgrp = (sn0 + grp * COLS) / 32;
                if (!V::MERGED && c0 < c1) {
                    const int64_t gc = kt0 / CKT + c0;
                    sa_next = args.scale_a[gc * args.ld_sa + srow];
#pragma unroll
                    for (int q = 0; q < NG; ++q) sb_next[q] = args.scale_b[gc * args.ld_sb + sgrp + q];
                }
            }
            constexpr int DEFER = V::EPI_CONV ? 1 : 0;  // drains run one chunk behind the conversions
            for (int ch = c0; ch < c1 + DEFER; ++ch) {
                if constexpr (V::EPI_CONV) {
                    const int kt_end = c1 * CKT < nkt ? c1 * CKT : nkt;
                    const int k_hi = (ch + 1) * CKT < kt_end ? (ch + 1) * CKT : kt_end;
                    for (int kt = ch * CKT; ch < c1 && kt < k_hi; ++kt, ++g) {
                        const int s = g % STAGES, u = g / STAGES;
                        const bool landed = mbar_wait_bounded(full0 + 8 * s, (uint32_t)(u & 1), kWaitLimitNs);
                        if (!__all_sync(0xffffffffu, landed)) {
                            s_fail = 1;
                            epi_ok = false;
                            break;
                        }
                        tc_convert_stage<V>(smem_raw + (sbase - raw) + s * V::STAGE_BYTES, tid);
                        __syncwarp();
                        if (lane == 0) mbar_arrive(conv0 + 8 * s);
                    }
                    if (!epi_ok) break;
                    if (ch == c0) continue;
                }
                const int b = c & 1;
                float sc[NG];
#pragma unroll
                for (int q = 0; q < NG; ++q) sc[q] = 1.f;
                if constexpr (V::SCALED && V::MERGED) {
                    // 256-column tiles hold no scales across chunks (registers are
                    // short there); the loads overlap the wait for the accumulator.
                    const int64_t gc = kt0 / CKT + ch;
                    const float sa = args.scale_a[gc * args.ld_sa + srow];
#pragma unroll
                    for (int q = 0; q < NG; ++q) sc[q] = sa * args.scale_b[gc * args.ld_sb + sgrp + q];
                } else if constexpr (V::SCALED) {
                    // This chunk's scale per 32-column group; the next chunk's loads go out.
#pragma unroll
                    for (int q = 0; q < NG; ++q) sc[q] = sa_next * sb_next[q];
                    if (ch + 1 < c1) {
                        const int64_t gc = kt0 / CKT + ch + 1;
                        sa_next = args.scale_a[gc * args.ld_sa + srow];
#pragma unroll
                        for (int q = 0; q < NG; ++q) sb_next[q] = args.scale_b[gc * args.ld_sb + sgrp + q];
                    }
                }
                const bool ok = mbar_wait_bounded(accf0 + 8 * b, (uint32_t)((c >> 1) & 1), kWaitLimitNs);
                if (!__all_sync(0xffffffffu, ok)) {
                    epi_ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < COLS; j += 32) {
                    if constexpr (V::MERGED) {
                        // one accumulator: chunk sum (times the chunk's scales) into the
                        // registers, 16 columns per load (the 128 accumulator registers
                        // leave little room)
                        const float s32 = sc[V::SCALED ? j / 32 : 0];  // 1 for the unscaled kinds
#pragma unroll
                        for (int h = 0; h < 32; h += 16) {
                            uint32_t r16[16];
                            tmem_ld16(lane_base + (uint32_t)(b * V::ACC_COLS + j + h), r16);
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                racc[j + h + q] = fmaf(__uint_as_float(r16[q]), s32, racc[j + h + q]);
                        }
                    } else {
                        uint32_t r[32];
                        if constexpr (V::SCALED) {
                            // (left + right) * 2^-S_A * 2^-S_B (a power of two: exact),
                            // added into the FP32 registers with one rounding.
                            const float s32 = sc[j / 32];
                            uint32_t r2[32];
                            tmem_ld32x2(lane_base + (uint32_t)(b * V::ACC_COLS + j),
                                        lane_base + (uint32_t)(b * V::ACC_COLS + BN + j), r, r2);
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                racc[j + q] = fmaf(__uint_as_float(r[q]) + __uint_as_float(r2[q]), s32, racc[j + q]);
                        } else {
                            tmem_ld32(lane_base + (uint32_t)(b * V::ACC_COLS + j), r);
#pragma unroll
                            for (int q = 0; q < 32; ++q) racc[j + q] += __uint_as_float(r[q]);
                            tmem_ld32(lane_base + (uint32_t)(b * V::ACC_COLS + BN + j), r);
#pragma unroll
                            for (int q = 0; q < 32; ++q) racc[j + q] += __uint_as_float(r[q]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    // Pair versions: the even CTA's MMA warp waits for the drains of both CTAs.
                    if constexpr (V::PAIR)
                        mbar_arrive_cluster(mapa_shared(acce0 + 8 * b, 0u));
                    else
                        mbar_arrive(acce0 + 8 * b);
                }
                ++c;
            }
            if (V::STREAMK != 0 && epi_ok && c1 < nchunks) {
                // Contributor: this CTA's partial tile goes to the workspace;
                // each warp publishes its 32 rows with its own flag.
                // Lane-major layout: a warp writes 512 contiguous bytes per store.
                float4 *pw = reinterpret_cast<float4 *>(args.sk_partials) +
                             ((int64_t)blockIdx.x * V::EPI_WARPS + warp) * (COLS / 4) * 32 + lane;
#pragma unroll
                for (int q = 0; q < COLS; q += 4)
                    pw[(q / 4) * 32] = make_float4(racc[q], racc[q + 1], racc[q + 2], racc[q + 3]);
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release_u32(args.sk_words + kSkFlags + kSkFlagsPerCta * blockIdx.x + warp, epoch1);
                continue;
            }
            if (V::STREAMK != 0 && epi_ok && c0 > 0) {
                // Finisher: add the partial tiles of the earlier CTAs that
                // share this tile (nearest first), after their flags are set.
                // (pair versions: the same-rank CTA of each earlier pair)
                const int64_t tile_lo = (int64_t)(t - work.sk_tile0) * nchunks;
                for (int j = unit - 1; j >= 0; --j) {
                    const int64_t lo_j = (int64_t)j * W_sk / G, hi_j = ((int64_t)j + 1) * W_sk / G;
                    if (hi_j <= tile_lo) break;
                    if (lo_j == hi_j) continue;  // an empty range contributes nothing
                    const int slot = V::PAIR ? 2 * j + (int)rank : j;
                    const unsigned *flag = args.sk_words + kSkFlags + kSkFlagsPerCta * slot + warp;
                    const uint64_t t0 = globaltimer_ns();
                    bool ready = false;
                    while (!(ready = ld_acquire_u32(flag) == epoch1 + args.sk_wait_bias)) {
                        if (globaltimer_ns() - t0 > args.sk_wait_ns) break;
                    }
                    if (!__all_sync(0xffffffffu, ready)) {
                        epi_ok = false;
                        break;
                    }
                    const float4 *pr = reinterpret_cast<const float4 *>(args.sk_partials) +
                                       ((int64_t)slot * V::EPI_WARPS + warp) * (COLS / 4) * 32 + lane;
#pragma unroll
                    for (int q = 0; q < COLS; q += 4) {
                        const float4 v = pr[(q / 4) * 32];
                        racc[q] += v.x; racc[q + 1] += v.y; racc[q + 2] += v.z; racc[q + 3] += v.w;
                    }
                }
            }
            if (V::SPLITK == 1 && V::TSTG_BUFS > 0 && epi_ok && args.tma_c) {
                // Asynchronous store: the warp writes each 32 x 32 block (alpha
                // applied; row = lane, 16-byte chunk q of a row at chunk
                // q ^ (row & 7), the 128-byte swizzle of mapC) into a staging
                // box, and one lane hands the box to the TMA engine, which clips
                // rows and columns past M and N.  The warp goes on to its next
                // drain while C is written.
                int m0, n0;
                tc_cta_coords<V>(t, tiles_m, tiles_n, rank, m0, n0);
                constexpr int NB = V::TSTG_BUFS;
                float *tbox = reinterpret_cast<float *>(smem_raw + (sbase - raw) + V::TSTG_OFFSET) + warp * NB * 1024;
                const uint32_t tbox_s = sbase + V::TSTG_OFFSET + (uint32_t)(warp * NB * 4096);
                const float as = alpha;
#pragma unroll
                for (int jb = 0; jb < COLS; jb += 32, ++sblk) {
                    const int bi = sblk % NB;
                    // the box stored NB blocks ago has been read out of buffer bi
                    if (lane == 0) bulk_wait_read<NB - 1>();
                    __syncwarp();
                    float *row = tbox + bi * 1024 + lane * 32;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4 *>(row + ((q ^ (lane & 7)) << 2)) =
                            make_float4(as * racc[jb + 4 * q], as * racc[jb + 4 * q + 1], as * racc[jb + 4 * q + 2],
                                        as * racc[jb + 4 * q + 3]);
                    fence_proxy_async_smem();  // generic writes before the async proxy reads them
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&mapC, tbox_s + (uint32_t)(bi * 4096), n0 + grp * COLS + jb, m0 + sub * 32);
                        bulk_commit();
                    }
                }
            } else if (V::SPLITK == 1 && epi_ok && V::STAGE_C) {
                // Coalesced store: the warp's 32 x 32 blocks go through its
                // staging buffer (row = lane in, four rows of 32 columns per
                // instruction out), STG_ROWS rows per pass.
                int m0, n0;
                tc_cta_coords<V>(t, tiles_m, tiles_n, rank, m0, n0);
                float *stg = reinterpret_cast<float *>(smem_raw + (sbase - raw) + V::STG_OFFSET) +
                             warp * V::STG_WARP_FLOATS;
                const int rr = lane >> 3, cc = (lane & 7) * 4;
                const float as = alpha;
                constexpr int SR = V::STG_ROWS;
#pragma unroll
                for (int jb = 0; jb < COLS; jb += 32) {
#pragma unroll
                for (int h = 0; h < 32 / SR; ++h) {
                    if (lane / SR == h) {
#pragma unroll
                        for (int q = 0; q < 32; q += 4)
                            *reinterpret_cast<float4 *>(stg + (lane % SR) * V::STG_LD + q) =
                                make_float4(as * racc[jb + q], as * racc[jb + q + 1], as * racc[jb + q + 2],
                                            as * racc[jb + q + 3]);
                    }
                    __syncwarp();
                    const int col = n0 + grp * COLS + jb + cc;
#pragma unroll
                    for (int it = 0; it < SR / 4; ++it) {
                        const int r = it * 4 + rr;
                        const int row = m0 + sub * 32 + h * SR + r;
                        float4 v = *reinterpret_cast<const float4 *>(stg + r * V::STG_LD + cc);
                        if (row < args.M && col < args.N) {
                            float *cp = args.C + (int64_t)row * args.ldc + col;
                            if (args.N - col >= 4 && args.vec4) {
                                if (beta != 0.f) {
                                    const float4 o = *reinterpret_cast<const float4 *>(cp);
                                    v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                                }
                                *reinterpret_cast<float4 *>(cp) = v;
                            } else {
                                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (col + e < args.N) cp[e] = (beta != 0.f) ? vv[e] + beta * cp[e] : vv[e];
                            }
                        }
                    }
                    __syncwarp();
                }
                }
            } else if (V::SPLITK == 1 && epi_ok) {
                int m0, n0;
                tc_cta_coords<V>(t, tiles_m, tiles_n, rank, m0, n0);
                const int row = m0 + sub * 32 + lane;
                const int cbase = n0 + grp * COLS;
                if (row < args.M && cbase < args.N) {
                    float *cp = args.C + (int64_t)row * args.ldc + cbase;
                    const int ncol = args.N - cbase;
                    const float as = alpha;
                    if (ncol >= COLS && args.vec4) {
#pragma unroll
                        for (int q = 0; q < COLS; q += 4) {
                            float4 v = make_float4(as * racc[q], as * racc[q + 1], as * racc[q + 2],
                                                   as * racc[q + 3]);
                            if (beta != 0.f) {
                                const float4 o = *reinterpret_cast<const float4 *>(cp + q);
                                v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                            }
                            *reinterpret_cast<float4 *>(cp + q) = v;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < COLS; ++q) {
                            if (q < ncol) {
                                const float v = as * racc[q];
                                cp[q] = (beta != 0.f) ? v + beta * cp[q] : v;
                            }
                        }
                    }
                }
            }
        }
        // Every box handed to the TMA engine is written before the CTA goes on
        // (and before its shared memory can be released).
        if (V::TSTG_BUFS > 0 && args.tma_c && lane == 0) bulk_wait_all();
    }
    __syncthreads();
    if (!epi_ok) s_fail = 1;
    pdl_trigger();
    __syncthreads();
    const bool failed = s_fail != 0;
    if constexpr (V::STREAMK != 0) {
        // The last CTA to finish advances the epoch (every CTA has read it
        // before counting itself) and re-arms the counter.
        if (tid == 0) {
            __threadfence();
            const unsigned old = atomicAdd(args.sk_words + 1, 1u);
            if (old == gridDim.x - 1) {
                args.sk_words[1] = 0u;
                __threadfence();
                atomicAdd(args.sk_words, 1u);
            }
        }
    }

    if constexpr (V::SPLITK > 1) {
        // One tile per CTA: every MMA and TMA copy of this CTA has completed
        // (the last chunk was drained), so the pipeline memory can hold the
        // partial tile; CTA r of the cluster then sums rows
        // [r*BM/S, (r+1)*BM/S) over ranks 0..S-1 in order.
        int m0 = 0, n0 = 0;
        if (t_first < tiles) tc_tile_coords<V>(t_first, tiles_m, tiles_n, m0, n0);
        float *red = reinterpret_cast<float *>(smem_raw + (sbase - raw));
        if (warp < V::EPI_WARPS) {
            float *rrow = red + ((warp & 3) * 32 + lane) * V::RED_LD + (warp >> 2) * COLS;
            if (nchunks == 0) {
#pragma unroll
                for (int j = 0; j < COLS; ++j) racc[j] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < COLS; q += 4)
                *reinterpret_cast<float4 *>(rrow + q) = make_float4(racc[q], racc[q + 1], racc[q + 2], racc[q + 3]);
        }
        cluster_sync();
        const uint32_t rank = cluster_ctarank();
        constexpr int ROWS = V::BM / V::SPLITK, C4 = BN / 4;
        const uint32_t red_addr = smem_u32(red);
        for (int idx = tid; idx < ROWS * C4; idx += V::THREADS) {
            const int rl = (int)rank * ROWS + idx / C4, cl = (idx % C4) * 4;
            const int row = m0 + rl, col = n0 + cl;
            if (failed || t_first >= tiles || row >= args.M || col >= args.N) continue;
            const uint32_t a = red_addr + (uint32_t)(rl * V::RED_LD + cl) * 4u;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < V::SPLITK; ++q) {
                const float4 v = ld_dsmem_f4(mapa_shared(a, (uint32_t)q));
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            float *cp = args.C + (int64_t)row * args.ldc + col;
            const float r4[4] = {sum.x, sum.y, sum.z, sum.w};
            if (args.N - col >= 4 && args.vec4) {
                float4 o = make_float4(alpha * r4[0], alpha * r4[1], alpha * r4[2], alpha * r4[3]);
                if (beta != 0.f) {
                    const float4 cc = *reinterpret_cast<const float4 *>(cp);
                    o.x += beta * cc.x; o.y += beta * cc.y; o.z += beta * cc.z; o.w += beta * cc.w;
                }
                *reinterpret_cast<float4 *>(cp) = o;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (col + q < args.N) cp[q] = (beta != 0.f) ? alpha * r4[q] + beta * cp[q] : alpha * r4[q];
            }
        }
        cluster_sync();  // no CTA leaves while a peer may still read its tile
    }
    if constexpr (V::PAIR) {
        // The odd CTA's copies complete on the even CTA's barriers: the even CTA
        // learns how many stages its peer issued.
        if (rank == 1 && tid == 0) st_dsmem_u32(mapa_shared(smem_u32(&s_peer_issued), 0u), (uint32_t)s_issued);
        cluster_sync();
    }
    if (tid == 0) {
        // No MMA may still write tensor memory when it is freed, and no TMA
        // copy may still be landing when the CTA exits.
        if (!mbar_wait_bounded(doneb, 0u, kWaitLimitNs)) s_fail = 1;
        if (s_fail) {
            if (args.err) atomicOr(args.err, 1);
            const int issued = s_issued > s_peer_issued ? s_issued : s_peer_issued;
            if (rank == 0)
                for (int q = s_consumed; q < issued; ++q)
                    (void)mbar_wait_bounded(full0 + 8 * (q % STAGES), (uint32_t)((q / STAGES) & 1), kWaitLimitNs);
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (V::PAIR) cluster_sync();  // the odd CTA stays until the even one has waited
    if (warp == 0) {
        tc_fence_after();
        if constexpr (V::PAIR)
            tmem_dealloc_pair(tmem, V::TMEM_COLS);
        else
            tmem_dealloc(tmem, V::TMEM_COLS);
    }
}

}  // namespace pt
