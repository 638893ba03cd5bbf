// Data collection for portability tuning (the paper's Section V-D): every
// listed variant is run on every listed shape, screened against the reference
// kernel, timed, and appended to the timing table (CSV, one row per
// (shape, variant), flushed per row so the file doubles as the checkpoint).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "common.h"
#include "launch.cuh"

namespace pt {
namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), counter form: output i of
// the sequence seeded with `seed` is mix(seed + (i+1)*gamma).  Values map to
// uniform FP32 on [-1, 1) as 2*(x>>40)/2^24 - 1.
__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void fill_uniform_kernel(float *p, int64_t n, uint64_t seed, int64_t offset) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = splitmix_at(seed, (uint64_t)(offset + i));
        p[i] = 2.0f * ((float)(x >> 40) * 5.9604644775390625e-8f) - 1.0f;
    }
}

struct CmpOut {
    unsigned int max_diff;  // float bits of max |C - R| (non-negative floats order as uints)
    unsigned int max_abs;   // float bits of max |X| (for max-abs reductions)
    int nonfinite;
};

// max |C - R| over an M x N matrix (row pitch ldc / ldr) and a non-finite flag.
__global__ void compare_kernel(const float *C, int64_t ldc, const float *R, int64_t ldr, int M, int N, CmpOut *out) {
    float m = 0.f;
    int bad = 0;
    const int64_t total = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / N, c = i % N;
        const float x = C[r * ldc + c], y = R[r * ldr + c];
        if (!isfinite(x)) bad = 1;
        else m = fmaxf(m, fabsf(x - y));
    }
    for (int off = 16; off > 0; off >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out->max_diff, __float_as_uint(m));
        if (bad) atomicOr(&out->nonfinite, 1);
    }
}

__global__ void maxabs_kernel(const float *X, int64_t n, CmpOut *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(X[i]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&out->max_abs, __float_as_uint(m));
}

int cuda_fail(cudaError_t e, const char *what) {
    return set_error(PT_ECUDA, 0, "%s: %s", what, cudaGetErrorString(e));
}

// A sticky error (illegal address, ...) leaves the context unusable.
bool sticky(cudaError_t e) {
    return e == cudaErrorIllegalAddress || e == cudaErrorLaunchFailure || e == cudaErrorIllegalInstruction ||
           e == cudaErrorMisalignedAddress || e == cudaErrorHardwareStackError || e == cudaErrorInvalidPc ||
           e == cudaErrorAssert || e == cudaErrorLaunchTimeout || e == cudaErrorECCUncorrectable;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

double median_of(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

struct Buffers {
    char *pool = nullptr;
    size_t pool_bytes = 0;
    float *ref = nullptr;
    size_t ref_bytes = 0;
    CmpOut *cmp = nullptr;
    ~Buffers() {
        if (pool) cudaFree(pool);
        if (ref) cudaFree(ref);
        if (cmp) cudaFree(cmp);
    }
};

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" {

void pt_tune_default_opts(pt_tune_opts_t *o) {
    if (!o) return;
    o->warmup = 2;
    o->reps_min = 5;
    o->reps_max = 50;
    o->target_ms = 5.0;
    o->seed = 1;
    o->resume = 0;
    o->tol = 2e-6;
    o->pool_bytes = (int64_t)1 << 30;
    o->verbose = 0;
    o->fail_launch = 0;
}

int pt_tune(const pt_shape_t *shapes, int n_shapes, const int *ids, int n_ids, const pt_tune_opts_t *opts_in,
            const char *table_path) {
    clear_error();
    if (!shapes || n_shapes <= 0) return set_error(PT_EINVAL, 1, "no shapes");
    if (ids && n_ids <= 0) return set_error(PT_EINVAL, 4, "empty id list");
    if (!table_path) return set_error(PT_EINVAL, 6, "table_path is NULL");
    pt_tune_opts_t o;
    pt_tune_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.warmup < 0 || o.reps_min < 1 || o.reps_max < o.reps_min || !(o.target_ms > 0) || !(o.tol > 0) ||
        o.fail_launch < 0)
        return set_error(PT_EINVAL, 5, "invalid tuning options");
    std::vector<int> vids;
    if (ids) {
        for (int i = 0; i < n_ids; ++i) {
            if (ids[i] < 0 || ids[i] >= variant_table_size()) return set_error(PT_EINVAL, 3, "bad variant id %d", ids[i]);
            vids.push_back(ids[i]);
        }
    } else {
        for (int i = 0; i < variant_table_size(); ++i) vids.push_back(i);
    }
    for (int s = 0; s < n_shapes; ++s) {
        const pt_shape_t &sh = shapes[s];
        if (sh.m < 1 || sh.n < 1 || sh.k < 1 || sh.m > 0x7fffffff || sh.n > 0x7fffffff || sh.k > 0x7fffffff ||
            (sh.transA != 'N' && sh.transA != 'T') || (sh.transB != 'N' && sh.transB != 'T'))
            return set_error(PT_EINVAL, 1, "invalid shape %d", s);
    }

    // Resume: keep existing rows, skip their (shape, variant) pairs.
    std::set<std::pair<std::string, std::string>> done;
    bool have_header = false;
    if (o.resume) {
        FILE *f = std::fopen(table_path, "r");
        if (f) {
            std::fclose(f);
            Table t;
            int rc = read_table(table_path, &t);
            if (rc == PT_OK) {
                have_header = true;
                for (const auto &r : t.rows) {
                    char key[128];
                    std::snprintf(key, sizeof(key), "%lld,%lld,%lld,%c,%c", (long long)r.shape.m,
                                  (long long)r.shape.n, (long long)r.shape.k, r.shape.transA, r.shape.transB);
                    done.insert({key, r.variant});
                }
            } else if (rc != PT_EIO) {
                return rc;  // refuse to append to a malformed table
            }
        }
    }
    FILE *out = std::fopen(table_path, have_header ? "a" : "w");
    if (!out) return set_error(PT_EIO, 6, "cannot open '%s' for writing", table_path);
    if (!have_header) {
        std::fprintf(out, "%s\n", kTableHeader);
        std::fflush(out);
    }

    int rc = PT_OK;
    Buffers buf;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> ev(2 * (size_t)o.reps_max + 6);
    for (auto &e : ev) e = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (size_t i = 0; ce == cudaSuccess && i < ev.size(); ++i) ce = cudaEventCreate(&ev[i]);
    if (ce == cudaSuccess) ce = cudaMalloc(&buf.cmp, sizeof(CmpOut));
    if (ce != cudaSuccess) rc = cuda_fail(ce, "tuner setup");
    int64_t launches = 0;  // variant launches made (the fail_launch hook counts them)
    auto run = [&](const VariantEntry &ve, const GemmArgs &g) {
        if (++launches == o.fail_launch) return set_error(PT_ECUDA, 0, "launch %lld failed (injected)",
                                                          (long long)launches);
        return ve.launch(g, st, false);
    };

    for (int s = 0; rc == PT_OK && s < n_shapes; ++s) {
        const pt_shape_t &sh = shapes[s];
        const int M = (int)sh.m, N = (int)sh.n, K = (int)sh.k;
        const int ta = sh.transA == 'T', tb = sh.transB == 'T';
        const int64_t lda = ta ? M : K, ldb = tb ? K : N, ldc = N;
        const size_t bA = align256((size_t)M * K * 4), bB = align256((size_t)K * N * 4), bC = align256((size_t)M * N * 4);
        const size_t rep_bytes = bA + bB + bC;
        char key[128];
        std::snprintf(key, sizeof(key), "%d,%d,%d,%c,%c", M, N, K, sh.transA, sh.transB);
        bool all_done = true;
        for (int id : vids) all_done = all_done && done.count({key, variant_table()[id].desc.name});
        if (all_done) continue;

        // Pool of input replicas: consecutive launches read different
        // replicas, so inputs come from HBM rather than L2.
        const size_t want = std::max((size_t)std::max<int64_t>(o.pool_bytes, 0), rep_bytes);
        if (buf.pool_bytes < want) {
            if (buf.pool) cudaFree(buf.pool);
            buf.pool = nullptr;
            buf.pool_bytes = 0;
            ce = cudaMalloc(&buf.pool, want);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "pool allocation"); break; }
            buf.pool_bytes = want;
        }
        // Fresh U[-1,1) inputs for every shape: earlier shapes' outputs lie
        // where this shape's A and B replicas are.
        fill_uniform_kernel<<<4096, 256, 0, st>>>(reinterpret_cast<float *>(buf.pool), (int64_t)(buf.pool_bytes / 4),
                                                  o.seed, 0);
        const int nrep = (int)std::max<size_t>(1, buf.pool_bytes / rep_bytes);
        auto A_of = [&](int r) { return reinterpret_cast<const float *>(buf.pool + (size_t)r * rep_bytes); };
        auto B_of = [&](int r) { return reinterpret_cast<const float *>(buf.pool + (size_t)r * rep_bytes + bA); };
        auto C_of = [&](int r) { return reinterpret_cast<float *>(buf.pool + (size_t)r * rep_bytes + bA + bB); };
        if (buf.ref_bytes < (size_t)M * N * 4) {
            if (buf.ref) cudaFree(buf.ref);
            buf.ref = nullptr;
            buf.ref_bytes = 0;
            ce = cudaMalloc(&buf.ref, (size_t)M * N * 4);
            if (ce != cudaSuccess) { rc = cuda_fail(ce, "reference buffer"); break; }
            buf.ref_bytes = (size_t)M * N * 4;
        }
        // Reference result and input maxima on replica 0.
        rc = pt_sgemm_reference(sh.transA, sh.transB, M, N, K, 1.f, A_of(0), lda, B_of(0), ldb, 0.f, buf.ref, ldc, st);
        if (rc != PT_OK) break;
        CmpOut zero{0u, 0u, 0};
        cudaMemcpyAsync(buf.cmp, &zero, sizeof(zero), cudaMemcpyHostToDevice, st);
        maxabs_kernel<<<1024, 256, 0, st>>>(A_of(0), (int64_t)M * K, buf.cmp);
        CmpOut ma{};
        cudaMemcpyAsync(&ma, buf.cmp, sizeof(ma), cudaMemcpyDeviceToHost, st);
        ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "reference"); break; }
        cudaMemcpyAsync(buf.cmp, &zero, sizeof(zero), cudaMemcpyHostToDevice, st);
        maxabs_kernel<<<1024, 256, 0, st>>>(B_of(0), (int64_t)K * N, buf.cmp);
        CmpOut mb{};
        cudaMemcpyAsync(&mb, buf.cmp, sizeof(mb), cudaMemcpyDeviceToHost, st);
        ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc = cuda_fail(ce, "input maxima"); break; }
        float maxA, maxB;
        std::memcpy(&maxA, &ma.max_abs, 4);
        std::memcpy(&maxB, &mb.max_abs, 4);
        const double denom = (double)K * maxA * maxB;

        for (size_t vi = 0; rc == PT_OK && vi < vids.size(); ++vi) {
            const VariantEntry &ve = variant_table()[vids[vi]];
            if (done.count({key, ve.desc.name})) continue;
            TableRow row;
            row.shape_idx = s;
            row.shape = sh;
            row.variant = ve.desc.name;
            GemmArgs g;
            g.A = A_of(0); g.B = B_of(0); g.C = C_of(0);
            g.lda = lda; g.ldb = ldb; g.ldc = ldc;
            g.M = M; g.N = N; g.K = K;
            g.alpha = 1.f; g.beta = 0.f;
            g.ta = ta; g.tb = tb;
            g.err = nullptr;
            int lr = ve.launch(g, st, true);
            if (lr == PT_OK) {
                // Screening run on replica 0 with C poisoned (all-ones bits = NaN).
                cudaMemsetAsync(C_of(0), 0xFF, (size_t)M * N * 4, st);
                lr = run(ve, g);
                if (lr == PT_OK) {
                    cudaMemcpyAsync(buf.cmp, &zero, sizeof(zero), cudaMemcpyHostToDevice, st);
                    compare_kernel<<<1024, 256, 0, st>>>(C_of(0), ldc, buf.ref, ldc, M, N, buf.cmp);
                    CmpOut co{};
                    cudaMemcpyAsync(&co, buf.cmp, sizeof(co), cudaMemcpyDeviceToHost, st);
                    ce = cudaStreamSynchronize(st);
                    if (ce != cudaSuccess) {
                        lr = cuda_fail(ce, "screening run");
                        if (sticky(ce)) { rc = lr; }
                    } else {
                        float md;
                        std::memcpy(&md, &co.max_diff, 4);
                        row.max_err = co.nonfinite ? INFINITY : (denom > 0 ? md / denom : (md > 0 ? INFINITY : 0.0));
                        if (!(row.max_err <= o.tol)) lr = PT_EUNSUPPORTED;  // fails screening
                    }
                } else {
                    cudaGetLastError();
                }
            }
            row.status = lr;
            if (rc == PT_OK && lr == PT_OK) {
                int r = 1;
                auto launch_rep = [&]() {
                    GemmArgs h = g;
                    const int idx = r++ % nrep;
                    h.A = A_of(idx); h.B = B_of(idx); h.C = C_of(idx);
                    return run(ve, h);
                };
                int e2 = PT_OK;
                for (int w = 0; w < o.warmup && e2 == PT_OK; ++w) e2 = launch_rep();
                // Pilot timing to choose the repetition count.
                std::vector<double> pilot;
                for (int p = 0; p < 3 && e2 == PT_OK; ++p) {
                    cudaEventRecord(ev[0], st);
                    e2 = launch_rep();
                    cudaEventRecord(ev[1], st);
                    ce = cudaEventSynchronize(ev[1]);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, ev[0], ev[1]);
                    pilot.push_back(ms);
                }
                int reps = o.reps_min;
                if (e2 == PT_OK) {
                    const double est = std::max(1e-4, median_of(pilot));
                    reps = (int)std::min<double>(o.reps_max, std::max<double>(o.reps_min, std::ceil(o.target_ms / est)));
                }
                for (int q = 0; q < reps && e2 == PT_OK; ++q) {
                    cudaEventRecord(ev[2 * q], st);
                    e2 = launch_rep();
                    cudaEventRecord(ev[2 * q + 1], st);
                }
                ce = cudaStreamSynchronize(st);
                if (ce != cudaSuccess) {
                    e2 = cuda_fail(ce, "timed runs");
                    if (sticky(ce)) rc = e2;
                }
                if (e2 == PT_OK) {
                    std::vector<double> ts(reps);
                    double sum = 0;
                    for (int q = 0; q < reps; ++q) {
                        float ms = 0;
                        cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]);
                        ts[q] = ms;
                        sum += ms;
                    }
                    row.valid = 1;
                    row.reps = reps;
                    row.median_ms = median_of(ts);
                    row.mean_ms = sum / reps;
                    row.min_ms = *std::min_element(ts.begin(), ts.end());
                    const double flops = 2.0 * M * (double)N * K;
                    const double bytes = 4.0 * ((double)M * K + (double)K * N + (double)M * N);
                    row.tflops = flops / (row.median_ms * 1e-3) / 1e12;
                    row.gbs = bytes / (row.median_ms * 1e-3) / 1e9;
                } else {
                    row.status = e2;
                }
            }
            std::fprintf(out, "%s\n", format_row(row).c_str());
            std::fflush(out);
            if (o.verbose)
                std::fprintf(stderr, "[pt_tune] %s %s status=%d valid=%d median=%.4f ms err=%.3g\n", key,
                             row.variant.c_str(), row.status, row.valid, row.median_ms, row.max_err);
        }
    }
    std::fclose(out);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    if (st) cudaStreamDestroy(st);
    return rc;
}

}  // extern "C"
