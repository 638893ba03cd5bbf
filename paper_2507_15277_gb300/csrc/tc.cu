// Host side of the split-precision tensor-core variants: workspace for the
// split planes, tensor maps, launches, registry entries.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "launch.cuh"
#include "tc.cuh"

namespace pt {
namespace {

// ---- workspace: one buffer per (device, stream), grown on demand ----------------
std::mutex g_ws_mu;
std::map<std::pair<int, uintptr_t>, std::pair<void *, size_t>> g_ws;

int workspace(cudaStream_t st, size_t need, bool dry, void **out) {
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto &e = g_ws[{dev, reinterpret_cast<uintptr_t>(st)}];
    if (e.second >= need) {
        *out = e.first;
        return PT_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return set_error(PT_EUNSUPPORTED, 0, "cannot query the stream's capture state");
    }
    if (cs != cudaStreamCaptureStatusNone)
        return set_error(PT_EUNSUPPORTED, 0, "split workspace must grow while the stream is being captured");
    if (dry) return PT_OK;
    if (e.first) {
        cudaStreamSynchronize(st);
        cudaFree(e.first);
        e = {nullptr, 0};
    }
    size_t bytes = need + need / 4;
    bytes = (bytes + ((size_t)2 << 20) - 1) & ~(((size_t)2 << 20) - 1);
    void *p = nullptr;
    cudaError_t err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return set_error(PT_ECUDA, 0, "workspace allocation of %zu bytes: %s", bytes, cudaGetErrorString(err));
    }
    // The stream-K header (epoch, finished-CTA count, flags) starts at zero.
    err = cudaMemsetAsync(p, 0, kSkHeaderBytes, st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return set_error(PT_ECUDA, 0, "workspace initialisation: %s", cudaGetErrorString(err));
    }
    e = {p, bytes};
    *out = p;
    return PT_OK;
}

int make_map_3d(CUtensorMap *map, const void *base, CUtensorMapDataType dt, int elem, int64_t inner, int64_t rows,
                int64_t planes, int64_t pitch_bytes, int64_t plane_bytes, int box_inner, int box_rows, int swz) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled unavailable");
    (void)elem;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)pitch_bytes, (cuuint64_t)plane_bytes};
    cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swz == 32   ? CU_TENSOR_MAP_SWIZZLE_32B
                    : swz == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(PT_ECUDA, 0, "cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
    return PT_OK;
}

inline int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

// Number of SMs of device `dev` (cached).
int device_sms(int dev) {
    static std::atomic<int> sm_count[64];
    int sms = dev >= 0 && dev < 64 ? sm_count[dev].load(std::memory_order_relaxed) : 0;
    if (sms <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (dev >= 0 && dev < 64) sm_count[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// Pair versions: how many CTA pairs of this kernel can be resident at once
// (clusters of two need two free SMs of one GPC), so the persistent grid is
// a single wave.  Cached per device.
template <class V>
int max_pairs(int dev, int sms) {
    static std::atomic<int> cap[64];
    int c = dev < 64 ? cap[dev].load(std::memory_order_relaxed) : 0;
    if (c > 0) return c;
    c = std::max(1, sms / 2);
    if (cudaFuncSetAttribute(tc_sgemm_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, V::SMEM_BYTES) ==
        cudaSuccess) {
        cudaLaunchConfig_t cfg;
        std::memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(2 * c), 1, 1);
        cfg.blockDim = dim3(V::THREADS, 1, 1);
        cfg.dynamicSmemBytes = V::SMEM_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_sgemm_kernel<V>, &cfg) == cudaSuccess && n > 0)
            c = std::min(c, n);
        else
            (void)cudaGetLastError();
    } else {
        (void)cudaGetLastError();
    }
    if (dev < 64) cap[dev].store(c, std::memory_order_relaxed);
    return c;
}

template <class V>
int launch_tc(const GemmArgs &a, cudaStream_t st, bool dry) {
    const int64_t tiles = (((int64_t)a.M + V::TILE_M - 1) / V::TILE_M) * (((int64_t)a.N + V::BN - 1) / V::BN);
    if (tiles > 0x7fffffff || ((int64_t)a.M + 31) / 32 + ((int64_t)a.N + 31) / 32 > 65535)
        return set_error(PT_EUNSUPPORTED, 3, "shape too large for this variant's grid");
    // Row pitch: a multiple of 8 elements (16-byte aligned rows, whole
    // 8-column groups for the split kernel's vector stores).
    if (V::FUSEB && (a.tb || misaligned(a.B, 16) || a.ldb % 4 != 0))
        return set_error(PT_EUNSUPPORTED, 0, "fused-B variant needs B as K x N (transB = N), 16-byte aligned, ldb %% 4 == 0");
    if (V::FUSEA && (a.ta || misaligned(a.A, 16) || a.lda % 4 != 0))
        return set_error(PT_EUNSUPPORTED, 0, "fused-A variant needs A as M x K (transA = N), 16-byte aligned, lda %% 4 == 0");
    const int64_t pitch = ((int64_t)a.K + 7) / 8 * 8;
    const int64_t a_plane = V::FUSEA ? 0 : align256((int64_t)a.M * pitch * V::ELEM);
    const int64_t b_plane = V::FUSEB ? 0 : align256((int64_t)a.N * pitch * V::ELEM);
    const int dev = current_device();
    // Grid: SPLITK == 1 is persistent, one CTA per SM (shared memory allows
    // one); stream-K needs every CTA to hold at least one chunk.
    int64_t grid = tiles;
    if (V::SPLITK == 1) {
        const int sms = device_sms(dev);
        if (V::STREAMK) {
            // Scheduling units: CTAs, or CTA pairs (at most as many as fit at once).
            const int64_t nch = (((int64_t)a.K + V::BK - 1) / V::BK + V::CHUNK_KT - 1) / V::CHUNK_KT;
            const int64_t cap = V::PAIR ? std::min<int64_t>(max_pairs<V>(dev, sms), kSkMaxGrid / 2)
                                        : std::min<int64_t>(sms, kSkMaxGrid);
            int64_t units = std::max<int64_t>(1, std::min<int64_t>(cap, tiles * nch));
            // Between 3/4 of a wave and one wave of tiles, one unit per tile (the
            // schedule then has no shared tiles): splitting every tile over 1-1.3
            // units costs more in partial tiles than the idle SMs do.
            if (tiles <= cap && 4 * tiles >= 3 * cap) units = tiles;
            grid = (V::PAIR ? 2 : 1) * units;
        } else if (V::PAIR) {
            // Two CTAs per tile, at most as many pairs as fit on the device at once.
            grid = 2 * std::min<int64_t>(tiles, max_pairs<V>(dev, sms));
        } else if (grid > sms) {
            grid = sms;
        }
    }
    // Workspace: stream-K header, stream-K partial tiles, the planes, then
    // (3xF16) the chunk scales of op(A) rows, [chunk][round_up(M, 128)], and
    // of op(B) 32-column groups, [chunk][round_up(N, 128) / 32].
    const int64_t header = align256((int64_t)kSkHeaderBytes);
    const int64_t partials = V::STREAMK ? align256(grid * V::BM * V::BN * 4) : 0;
    const int64_t nchk = ((int64_t)a.K + V::CHUNK_K - 1) / V::CHUNK_K;
    // (every tile's rows and 32-column groups have a slot, also past M and N)
    constexpr int64_t NR = V::BN > 128 ? V::BN : 128;
    const int64_t ld_sa = ((int64_t)a.M + V::TILE_M - 1) / V::TILE_M * V::TILE_M,
                  ld_sb = ((int64_t)a.N + NR - 1) / NR * (NR / 32);
    const int64_t sa_bytes = V::SCALED ? align256(nchk * ld_sa * 4) : 0;
    const int64_t sb_bytes = V::SCALED ? align256(nchk * ld_sb * 4) : 0;
    const size_t need =
        (size_t)(header + partials) + (size_t)V::P * (size_t)(a_plane + b_plane) + (size_t)(sa_bytes + sb_bytes);
    void *ws = nullptr;
    int rc = workspace(st, need, dry, &ws);
    if (rc != PT_OK || dry) return rc;

    static std::atomic<uint64_t> attr_done{0};
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(tc_sgemm_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             V::SMEM_BYTES);
        if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        attr_done.fetch_or(bit, std::memory_order_acq_rel);
    }

    unsigned char *wA = static_cast<unsigned char *>(ws) + header + partials;
    unsigned char *wB = wA + V::P * a_plane;
    float *scA = reinterpret_cast<float *>(wB + V::P * b_plane);
    float *scB = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(scA) + sa_bytes);
    const int va = (!misaligned(a.A, 16) && a.lda % 4 == 0) ? 1 : 0;
    const int vb = (!misaligned(a.B, 16) && a.ldb % 4 == 0) ? 1 : 0;
    const SplitOperand oa{a.A, a.lda, a.ta, a.M, wA, a_plane, va, V::SCALED ? scA : nullptr, ld_sa};
    const SplitOperand ob{a.B, a.ldb, a.tb ? 0 : 1, a.N, wB, b_plane, vb, V::SCALED ? scB : nullptr, ld_sb};
    // Blocks with blockIdx.y < ya split the first operand, the rest the second.
    const int ya = V::FUSEA ? (a.N + 31) / 32 : (a.M + 31) / 32;
    const int yb = V::FUSE ? 0 : (a.N + 31) / 32;
    cudaLaunchConfig_t scfg;
    std::memset(&scfg, 0, sizeof(scfg));
    scfg.gridDim = dim3((unsigned)((pitch + SPLIT_K_PER_BLOCK - 1) / SPLIT_K_PER_BLOCK), (unsigned)(ya + yb), 1);
    scfg.blockDim = dim3(256, 1, 1);
    scfg.stream = st;
    cudaLaunchAttribute sattr[1];
    unsigned nsattr = 0;
    add_pdl_attr(sattr, nsattr);
    scfg.attrs = sattr;
    scfg.numAttrs = nsattr;
    cudaError_t e = cudaSuccess;
    if constexpr (V::FUSE != 3) {  // both operands fused: no split kernel at all
        e = V::FUSEA ? cudaLaunchKernelEx(&scfg, tc_split_kernel<V::KIND>, ob, ob, (int)a.K, pitch, ya)
                     : cudaLaunchKernelEx(&scfg, tc_split_kernel<V::KIND>, oa, ob, (int)a.K, pitch, ya);
    }
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "split kernel: %s", cudaGetErrorString(e));

    const CUtensorMapDataType dt = V::KIND == kTcTf32     ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : V::KIND == kTcBf16x3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUtensorMap mA, mB;
    if (V::FUSEA)
        rc = make_map_2d(&mA, a.A, a.K, a.M, a.lda, V::BK, V::BM, CU_TENSOR_MAP_SWIZZLE_NONE);
    else
        rc = make_map_3d(&mA, wA, dt, V::ELEM, a.K, a.M, V::P, pitch * V::ELEM, a_plane, V::BK, V::BM, V::SWZ);
    if (rc != PT_OK) return rc;
    if (V::FUSEB)
        rc = make_map_2d(&mB, a.B, a.N, a.K, a.ldb, V::BN, V::BK, CU_TENSOR_MAP_SWIZZLE_NONE);
    else
        rc = make_map_3d(&mB, wB, dt, V::ELEM, a.K, a.N, V::P, pitch * V::ELEM, b_plane, V::BK, V::B_ROWS, V::SWZ);
    if (rc != PT_OK) return rc;

    TcArgs t;
    t.C = a.C;
    t.ldc = a.ldc;
    t.M = a.M;
    t.N = a.N;
    t.K = a.K;
    t.alpha = a.alpha;
    t.beta = a.beta;
    t.vec4 = (!misaligned(a.C, 16) && a.ldc % 4 == 0) ? 1 : 0;
    // C through the TMA engine where the version has the staging boxes, C
    // need not be read (beta = 0), C and ldc are 16-byte aligned and the rows
    // end on a 16-byte boundary (N % 4 == 0: a store of a box that crosses N
    // wrote the rest of the row's last 16 bytes, past N); otherwise the
    // epilogue warps store C themselves.
    CUtensorMap mC = mA;  // unused unless tma_c
    t.tma_c = 0;
    if (V::TSTG_BUFS > 0 && a.beta == 0.f && t.vec4 && a.N % 4 == 0 && a.M > 0 && a.N > 0) {
        if (make_map_2d(&mC, a.C, a.N, a.M, a.ldc, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B) == PT_OK)
            t.tma_c = 1;
        else
            clear_error();
    }
    t.err = a.err;
    t.sk_words = static_cast<unsigned *>(ws);
    t.sk_partials = reinterpret_cast<float *>(static_cast<unsigned char *>(ws) + header);
    streamk_wait_settings(&t.sk_wait_ns, &t.sk_wait_bias);
    t.scale_a = V::SCALED ? scA : nullptr;
    t.scale_b = V::SCALED ? scB : nullptr;
    t.ld_sa = ld_sa;
    t.ld_sb = ld_sb;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid, 1, V::SPLITK);
    cfg.blockDim = dim3(V::THREADS, 1, 1);
    cfg.dynamicSmemBytes = V::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    unsigned nattr = 0;
    if (V::SPLITK > 1 || V::PAIR) {
        attr[nattr].id = cudaLaunchAttributeClusterDimension;
        attr[nattr].val.clusterDim.x = V::PAIR ? 2 : 1;
        attr[nattr].val.clusterDim.y = 1;
        attr[nattr].val.clusterDim.z = V::SPLITK;
        ++nattr;
    }
    add_pdl_attr(attr, nattr);
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    kernel_timer_mark(st, true);
    e = cudaLaunchKernelEx(&cfg, tc_sgemm_kernel<V>, t, mA, mB, mC);
    kernel_timer_mark(st, false);
    if (e != cudaSuccess) return set_error(PT_ECUDA, 0, "tensor-core kernel: %s", cudaGetErrorString(e));
    return PT_OK;
}

template <class V>
VariantEntry tc_entry(const char *name) {
    VariantEntry v;
    std::memset(&v.desc, 0, sizeof(v.desc));
    v.desc.bm = V::TILE_M;  // pair versions: the 256-row tile of a CTA pair
    v.desc.bn = V::BN;
    v.desc.bk = V::BK;
    v.desc.kl = 1;
    v.desc.vec = 1;
    v.desc.stages = V::STAGES;
    v.desc.splitk = V::SPLITK;
    v.desc.loader = PT_LOADER_TMA;
    v.desc.a_kmajor = 1;
    v.desc.threads = V::THREADS;
    v.desc.smem_bytes = V::SMEM_BYTES;
    // fused B: transB = N only; fused A: transA = N only; both: N N only
    v.desc.trans_mask = V::FUSE == 3 ? 1 : (V::FUSEB ? 5 : (V::FUSEA ? 3 : 15));
    v.desc.kind = V::KIND == kTcTf32 ? 1 : (V::KIND == kTcBf16x3 ? 2 : 3);
    v.desc.schedule = V::STREAMK ? PT_SCHED_STREAMK : (V::SPLITK > 1 ? PT_SCHED_TILE : PT_SCHED_PERSISTENT);
    std::strncpy(v.desc.name, name, sizeof(v.desc.name) - 1);
    v.launch = launch_tc<V>;
    return v;
}

// A persistent version that switches to its stream-K twin when the tiles
// make more than one wave and the last wave is less than 3/4 full (there the
// idle SMs of the last wave cost more than the shared tiles' partial sums);
// single-wave and near-whole-wave shapes keep one CTA per tile.  The
// descriptor is the persistent one's.
template <class Vdp, class Vsk>
int launch_tc_hybrid(const GemmArgs &a, cudaStream_t st, bool dry) {
    const int64_t tiles = (((int64_t)a.M + Vdp::TILE_M - 1) / Vdp::TILE_M) * (((int64_t)a.N + Vdp::BN - 1) / Vdp::BN);
    const int dev = current_device(), sms = device_sms(dev);
    const int64_t cap = Vdp::PAIR ? max_pairs<Vdp>(dev, sms) : sms;  // tiles in flight at once
    const int64_t tail = tiles % cap;
    const bool sk = tiles > cap && tail != 0 && 4 * tail < 3 * cap;
    return sk ? launch_tc<Vsk>(a, st, dry) : launch_tc<Vdp>(a, st, dry);
}

template <class Vdp, class Vsk>
VariantEntry tc_entry_hybrid(const char *name) {
    VariantEntry v = tc_entry<Vdp>(name);
    v.launch = launch_tc_hybrid<Vdp, Vsk>;
    return v;
}

}  // namespace

int stream_workspace(cudaStream_t st, size_t need, bool dry, void **out) { return workspace(st, need, dry, out); }

// The segments (tile, first chunk, end chunk) that stream-K unit `unit` of
// `units` processes, in the kernel's order, from the kernel's own partition
// code (TcWork); returns their number, writing at most `cap`.
int streamk_segments(int tiles, int nchunks, int units, int unit, int *out, int cap) {
    TcWork w;
    w.nch = nchunks;
    w.t_first = unit;
    w.t_step = units;
    w.tiles = tiles;
    w.streamk = true;
    w.streamk_init(units, unit);
    const int n = w.count();
    for (int i = 0; i < n && i < cap; ++i) w.seg(i, out[3 * i], out[3 * i + 1], out[3 * i + 2]);
    return n;
}

// Tensor-core variants appended to the registry after the SIMT family.
std::vector<VariantEntry> tc_variants() {
    return {
        tc_entry<Tc<kTcTf32, 128, 3>>("tc3xtf32_m128n128_p3"),
        tc_entry<Tc<kTcTf32, 128, 2>>("tc3xtf32_m128n128_p2"),
        tc_entry<Tc<kTcTf32, 64, 4>>("tc3xtf32_m128n64_p4"),
        tc_entry<Tc<kTcBf16x3, 128, 2>>("tcbf16x3_m128n128_p2"),
        tc_entry<Tc<kTcBf16x3, 64, 3>>("tcbf16x3_m128n64_p3"),
        tc_entry<Tc<kTcTf32, 128, 3, 2>>("tc3xtf32_m128n128_p3_sk2"),
        tc_entry<Tc<kTcTf32, 128, 3, 4>>("tc3xtf32_m128n128_p3_sk4"),
        tc_entry<Tc<kTcTf32, 64, 4, 2>>("tc3xtf32_m128n64_p4_sk2"),
        tc_entry<Tc<kTcTf32, 64, 4, 4>>("tc3xtf32_m128n64_p4_sk4"),
        tc_entry<Tc<kTcTf32, 64, 4, 8>>("tc3xtf32_m128n64_p4_sk8"),
        tc_entry<Tc<kTcBf16x3, 128, 2, 2>>("tcbf16x3_m128n128_p2_sk2"),
        tc_entry<Tc<kTcBf16x3, 128, 2, 4>>("tcbf16x3_m128n128_p2_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 2>>("tcbf16x3_m128n64_p3_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 4>>("tcbf16x3_m128n64_p3_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 8>>("tcbf16x3_m128n64_p3_sk8"),
        // 64-byte rows: half-size stages, twice the depth.
        tc_entry<Tc<kTcTf32, 128, 6, 1, 64>>("tc3xtf32_m128n128_p6_sw64"),
        tc_entry<Tc<kTcTf32, 64, 8, 1, 64>>("tc3xtf32_m128n64_p8_sw64"),
        tc_entry<Tc<kTcBf16x3, 128, 4, 1, 64>>("tcbf16x3_m128n128_p4_sw64"),
        tc_entry<Tc<kTcBf16x3, 64, 6, 1, 64>>("tcbf16x3_m128n64_p6_sw64"),
        tc_entry<Tc<kTcTf32, 128, 6, 2, 64>>("tc3xtf32_m128n128_p6_sw64_sk2"),
        tc_entry<Tc<kTcTf32, 128, 6, 4, 64>>("tc3xtf32_m128n128_p6_sw64_sk4"),
        tc_entry<Tc<kTcBf16x3, 128, 4, 2, 64>>("tcbf16x3_m128n128_p4_sw64_sk2"),
        tc_entry<Tc<kTcBf16x3, 128, 4, 4, 64>>("tcbf16x3_m128n128_p4_sw64_sk4"),
        // 32-byte rows: one MMA k step per stage, eight or twelve stages.
        tc_entry<Tc<kTcTf32, 128, 12, 1, 32>>("tc3xtf32_m128n128_p12_sw32"),
        tc_entry<Tc<kTcBf16x3, 128, 8, 1, 32>>("tcbf16x3_m128n128_p8_sw32"),
        // Stream-K: equal shares of tiles x chunks per SM.
        tc_entry<Tc<kTcBf16x3, 128, 2, 1, 128, 1>>("tcbf16x3_m128n128_p2_stk"),
        tc_entry<Tc<kTcBf16x3, 128, 4, 1, 64, 1>>("tcbf16x3_m128n128_p4_sw64_stk"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 1, 128, 1>>("tcbf16x3_m128n64_p3_stk"),
        tc_entry<Tc<kTcTf32, 128, 3, 1, 128, 1>>("tc3xtf32_m128n128_p3_stk"),
        tc_entry<Tc<kTcTf32, 64, 4, 1, 128, 1>>("tc3xtf32_m128n64_p4_stk"),
        // Fused B split (B converted inside the GEMM kernel; small M).
        tc_entry<Tc<kTcBf16x3, 64, 2, 1, 128, 0, 1>>("tcbf16x3_m128n64_p2_fb"),
        tc_entry<Tc<kTcBf16x3, 64, 2, 2, 128, 0, 1>>("tcbf16x3_m128n64_p2_fb_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 2, 4, 128, 0, 1>>("tcbf16x3_m128n64_p2_fb_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 2, 1, 128, 1, 1>>("tcbf16x3_m128n64_p2_fb_stk"),
        // Fused A split (A converted inside the GEMM kernel; small N).
        tc_entry<Tc<kTcBf16x3, 64, 3, 1, 64, 0, 2>>("tcbf16x3_m128n64_p3_sw64_fa"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 2, 64, 0, 2>>("tcbf16x3_m128n64_p3_sw64_fa_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 4, 64, 0, 2>>("tcbf16x3_m128n64_p3_sw64_fa_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 1, 64, 1, 2>>("tcbf16x3_m128n64_p3_sw64_fa_stk"),
        // Deeper fused pipelines (64-byte rows): more FP32 bytes in flight per SM
        // for the skinny, long-K shapes whose loads are latency-bound.
        tc_entry<Tc<kTcBf16x3, 64, 4, 1, 64, 0, 2>>("tcbf16x3_m128n64_p4_sw64_fa"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 2, 64, 0, 2>>("tcbf16x3_m128n64_p4_sw64_fa_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 4, 64, 0, 2>>("tcbf16x3_m128n64_p4_sw64_fa_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 5, 1, 64, 0, 1>>("tcbf16x3_m128n64_p5_sw64_fb"),
        tc_entry<Tc<kTcBf16x3, 64, 5, 2, 64, 0, 1>>("tcbf16x3_m128n64_p5_sw64_fb_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 5, 4, 64, 0, 1>>("tcbf16x3_m128n64_p5_sw64_fb_sk4"),
        // Fused 128-column tiles: with N (fused A) or M (fused B) at most 128
        // each FP32 element is converted once, and the tensor core reads the
        // other operand's planes once per 128 columns instead of per 64.
        tc_entry<Tc<kTcBf16x3, 128, 3, 1, 64, 0, 2>>("tcbf16x3_m128n128_p3_sw64_fa"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 2, 64, 0, 2>>("tcbf16x3_m128n128_p3_sw64_fa_sk2"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 4, 64, 0, 2>>("tcbf16x3_m128n128_p3_sw64_fa_sk4"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 1, 64, 1, 2>>("tcbf16x3_m128n128_p3_sw64_fa_stk"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 1, 64, 0, 1>>("tcbf16x3_m128n128_p3_sw64_fb"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 2, 64, 0, 1>>("tcbf16x3_m128n128_p3_sw64_fb_sk2"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 4, 64, 0, 1>>("tcbf16x3_m128n128_p3_sw64_fb_sk4"),
        tc_entry<Tc<kTcBf16x3, 128, 3, 1, 64, 1, 1>>("tcbf16x3_m128n128_p3_sw64_fb_stk"),
        // Both operands split inside the GEMM kernel: one launch per call,
        // for small problems whose time is mostly the fixed cost per launch.
        tc_entry<Tc<kTcBf16x3, 64, 3, 1, 64, 0, 3>>("tcbf16x3_m128n64_p3_sw64_fab"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 2, 64, 0, 3>>("tcbf16x3_m128n64_p3_sw64_fab_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 3, 4, 64, 0, 3>>("tcbf16x3_m128n64_p3_sw64_fab_sk4"),
        tc_entry<Tc<kTcBf16x3, 128, 2, 1, 64, 0, 3>>("tcbf16x3_m128n128_p2_sw64_fab"),
        tc_entry<Tc<kTcBf16x3, 128, 2, 4, 64, 0, 3>>("tcbf16x3_m128n128_p2_sw64_fab_sk4"),
        // 32-column tiles: twice the CTAs of 64-column ones on skinny,
        // long-K shapes (5-10 % faster there; more A re-reads elsewhere).
        tc_entry<Tc<kTcBf16x3, 32, 3, 4>>("tcbf16x3_m128n32_p3_sk4"),
        tc_entry<Tc<kTcBf16x3, 32, 3, 8>>("tcbf16x3_m128n32_p3_sk8"),
        // BF16x3 64-column tiles with room for the coalescing epilogue stage.
        tc_entry<Tc<kTcBf16x3, 64, 2>>("tcbf16x3_m128n64_p2"),
        tc_entry<Tc<kTcBf16x3, 64, 2, 4>>("tcbf16x3_m128n64_p2_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 1, 64>>("tcbf16x3_m128n64_p4_sw64"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 2, 64>>("tcbf16x3_m128n64_p4_sw64_sk2"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 4, 64>>("tcbf16x3_m128n64_p4_sw64_sk4"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 8, 64>>("tcbf16x3_m128n64_p4_sw64_sk8"),
        tc_entry<Tc<kTcBf16x3, 64, 4, 1, 64, 1>>("tcbf16x3_m128n64_p4_sw64_stk"),
        // Scaled 3xF16: 3xTF32's 22 significand bits in three MMAs at the
        // FP16 rate (half the tensor work of BF16x3, 4 bytes per element
        // of planes instead of 6).
        tc_entry<Tc<kTcF16s, 128, 3>>("tc3xf16_m128n128_p3"),
        tc_entry<Tc<kTcF16s, 128, 6, 1, 64>>("tc3xf16_m128n128_p6_sw64"),
        tc_entry<Tc<kTcF16s, 128, 3, 1, 128, 1>>("tc3xf16_m128n128_p3_stk"),
        tc_entry<Tc<kTcF16s, 128, 6, 1, 64, 1>>("tc3xf16_m128n128_p6_sw64_stk"),
        tc_entry<Tc<kTcF16s, 64, 4>>("tc3xf16_m128n64_p4"),
        tc_entry<Tc<kTcF16s, 64, 4, 1, 128, 1>>("tc3xf16_m128n64_p4_stk"),
        tc_entry<Tc<kTcF16s, 128, 3, 2>>("tc3xf16_m128n128_p3_sk2"),
        tc_entry<Tc<kTcF16s, 128, 3, 4>>("tc3xf16_m128n128_p3_sk4"),
        tc_entry<Tc<kTcF16s, 64, 4, 2>>("tc3xf16_m128n64_p4_sk2"),
        tc_entry<Tc<kTcF16s, 64, 4, 4>>("tc3xf16_m128n64_p4_sk4"),
        tc_entry<Tc<kTcF16s, 64, 4, 8>>("tc3xf16_m128n64_p4_sk8"),
        tc_entry<Tc<kTcF16s, 32, 5, 4>>("tc3xf16_m128n32_p5_sk4"),
        tc_entry<Tc<kTcF16s, 32, 5, 8>>("tc3xf16_m128n32_p5_sk8"),
        // CTA pairs (cta_group::2): 256 x 128 tiles, four 48 KB stages.
        tc_entry<Tc<kTcF16s, 128, 4, 1, 128, 0, 0, 1>>("tc3xf16_m256n128_p4_2sm"),
        tc_entry<Tc<kTcTf32, 128, 4, 1, 128, 0, 0, 1>>("tc3xtf32_m256n128_p4_2sm"),
        // 256-column tiles: three N = 256 MMAs per k step into one accumulator,
        // four 48 KB stages of 64-byte rows.
        tc_entry_hybrid<Tc<kTcF16s, 256, 4, 1, 64>, Tc<kTcF16s, 256, 4, 1, 64, 1>>("tc3xf16_m128n256_p4_sw64"),
        tc_entry<Tc<kTcF16s, 256, 4, 1, 64, 1>>("tc3xf16_m128n256_p4_sw64_stk"),
        // 256 x 256 pair tiles: each CTA loads its 128 rows of A and 128 of the
        // 256 rows of op(B)^T (32 KB stages of 64-byte rows); three N = 256
        // MMAs of M = 256 per k step into one accumulator; stream-K per pair
        // when the last wave of pairs is under 3/4 full.
        tc_entry_hybrid<Tc<kTcF16s, 256, 6, 1, 64, 0, 0, 1>, Tc<kTcF16s, 256, 6, 1, 64, 1, 0, 1>>(
            "tc3xf16_m256n256_p6_sw64_2sm"),
        tc_entry<Tc<kTcF16s, 256, 6, 1, 64, 1, 0, 1>>("tc3xf16_m256n256_p6_sw64_2sm_stk"),
        tc_entry_hybrid<Tc<kTcF16s, 256, 5, 1, 64, 0, 0, 1>, Tc<kTcF16s, 256, 5, 1, 64, 1, 0, 1>>(
            "tc3xf16_m256n256_p5_sw64_2sm"),
    };
}

void free_workspaces() {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto &kv : g_ws) {
        if (kv.second.first) {
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(kv.first.first);
            cudaDeviceSynchronize();
            cudaFree(kv.second.first);
            cudaSetDevice(cur);
        }
    }
    g_ws.clear();
}

}  // namespace pt
