// noalloc_reset.cu -- lp_solve_uniform_noalloc (and the library's cached
// memory pool) across a cudaDeviceReset.
//
// Built by tests/test_zz_no_alloc.py from this file and the library's own
// object files, so that this program and the library share one CUDA runtime
// and the reset below really ends the context the library's module lives in.
//
//  1. LPs of one size (some with b_i < 0, so phase I runs) are solved by
//     lp_batch_create + lp_batch_solve + lp_batch_results (the reference).
//  2. lp_solve_uniform_noalloc solves them; the results must be bit-identical.
//  3. cudaDeviceReset() ends the context: every allocation and the loaded
//     module (with its static scratch array) are gone.
//  4. The inputs are allocated and copied again, and lp_solve_uniform_noalloc
//     is called again in the new context: bit-identical again.
//  5. The regular path and lp_solve_host (host arrays, 3 ranges) run before
//     and after the reset too: the library keeps a stream-ordered memory pool
//     per device and context, and must not use the old context's pool in the
//     new one.
//
// Prints "noalloc reset ok" and exits 0 on success; any mismatch or error
// exits non-zero with a message.

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lpbatch.h"

namespace {

uint64_t g_state = 0x2545F4914F6CDD1Dull;
double uniform(double lo, double hi) {  // xorshift64*, plenty for test data
    g_state ^= g_state >> 12;
    g_state ^= g_state << 25;
    g_state ^= g_state >> 27;
    const uint64_t r = g_state * 0x2545F4914F6CDD1Dull;
    return lo + (hi - lo) * (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

struct Results {
    std::vector<int32_t> status, iters;
    std::vector<double> obj, x, y;
    Results(int N, int m, int n) : status(N), iters(N), obj(N), x((size_t)N * n), y((size_t)N * m) {}
};

struct DeviceData {
    double *A = nullptr, *b = nullptr, *c = nullptr, *obj = nullptr, *x = nullptr, *y = nullptr;
    int32_t *status = nullptr, *iters = nullptr;
};

#define CHECK_CUDA(call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            std::fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));             \
            return false;                                                                       \
        }                                                                                       \
    } while (0)

bool upload(DeviceData& d, const std::vector<double>& A, const std::vector<double>& b, const std::vector<double>& c,
            int N, int m, int n) {
    CHECK_CUDA(cudaMalloc(&d.A, A.size() * 8));
    CHECK_CUDA(cudaMalloc(&d.b, b.size() * 8));
    CHECK_CUDA(cudaMalloc(&d.c, c.size() * 8));
    CHECK_CUDA(cudaMalloc(&d.obj, (size_t)N * 8));
    CHECK_CUDA(cudaMalloc(&d.x, (size_t)N * n * 8));
    CHECK_CUDA(cudaMalloc(&d.y, (size_t)N * m * 8));
    CHECK_CUDA(cudaMalloc(&d.status, (size_t)N * 4));
    CHECK_CUDA(cudaMalloc(&d.iters, (size_t)N * 4));
    CHECK_CUDA(cudaMemcpy(d.A, A.data(), A.size() * 8, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d.b, b.data(), b.size() * 8, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d.c, c.data(), c.size() * 8, cudaMemcpyHostToDevice));
    return true;
}

bool noalloc_solve(const DeviceData& d, int N, int m, int n, Results& r) {
    // outputs poisoned first, so a call that writes nothing cannot pass
    CHECK_CUDA(cudaMemset(d.status, 0xFF, (size_t)N * 4));
    CHECK_CUDA(cudaMemset(d.obj, 0xFF, (size_t)N * 8));
    CHECK_CUDA(cudaMemset(d.x, 0xFF, (size_t)N * n * 8));
    CHECK_CUDA(cudaMemset(d.y, 0xFF, (size_t)N * m * 8));
    const lpb_err e = lp_solve_uniform_noalloc(N, m, n, d.A, d.b, d.c, d.status, d.iters, d.obj, d.x, d.y, nullptr,
                                               nullptr);
    if (e != LPB_OK) {
        std::fprintf(stderr, "lp_solve_uniform_noalloc: %s\n", lpb_strerror(e));
        return false;
    }
    CHECK_CUDA(cudaDeviceSynchronize());
    CHECK_CUDA(cudaMemcpy(r.status.data(), d.status, (size_t)N * 4, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(r.iters.data(), d.iters, (size_t)N * 4, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(r.obj.data(), d.obj, (size_t)N * 8, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(r.x.data(), d.x, (size_t)N * n * 8, cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(r.y.data(), d.y, (size_t)N * m * 8, cudaMemcpyDeviceToHost));
    return true;
}

bool regular_solve(const DeviceData& d, int N, int m, int n, size_t a_len, Results& r) {
    lp_batch* h = nullptr;
    lpb_err e = lp_batch_create(&h, N, std::vector<int32_t>(N, m).data(), std::vector<int32_t>(N, n).data(), nullptr,
                                d.A, (int64_t)a_len, nullptr, d.b, (int64_t)N * m, nullptr, d.c, (int64_t)N * n,
                                LPB_DEVICE, nullptr, nullptr);
    if (e == LPB_OK) e = lp_batch_solve(h, nullptr);
    if (e == LPB_OK)
        e = lp_batch_results(h, r.status.data(), r.iters.data(), r.obj.data(), r.x.data(), r.y.data(), LPB_HOST);
    if (h) lp_batch_destroy(h);
    if (e != LPB_OK) {
        std::fprintf(stderr, "regular path: %s (%s)\n", lpb_strerror(e), lpb_last_error());
        return false;
    }
    return true;
}

bool host_solve(const std::vector<double>& A, const std::vector<double>& b, const std::vector<double>& c, int N,
                int m, int n, Results& r) {
    const lpb_err e = lp_solve_host(N, std::vector<int32_t>(N, m).data(), std::vector<int32_t>(N, n).data(), nullptr,
                                    A.data(), (int64_t)A.size(), nullptr, b.data(), (int64_t)b.size(), nullptr,
                                    c.data(), (int64_t)c.size(), nullptr, 3, r.status.data(), r.iters.data(),
                                    r.obj.data(), r.x.data(), r.y.data());
    if (e != LPB_OK) {
        std::fprintf(stderr, "lp_solve_host: %s (%s)\n", lpb_strerror(e), lpb_last_error());
        return false;
    }
    return true;
}

bool same(const Results& a, const Results& b, const char* what) {
    const bool ok = a.status == b.status && a.iters == b.iters &&
                    std::memcmp(a.obj.data(), b.obj.data(), a.obj.size() * 8) == 0 &&
                    std::memcmp(a.x.data(), b.x.data(), a.x.size() * 8) == 0 &&
                    std::memcmp(a.y.data(), b.y.data(), a.y.size() * 8) == 0;
    if (!ok) std::fprintf(stderr, "%s: results differ from lp_batch_create + solve + results\n", what);
    return ok;
}

bool run() {
    const int N = 700, m = 30, n = 24;
    std::vector<double> A((size_t)N * m * n), b((size_t)N * m), c((size_t)N * n);
    for (double& v : A) v = uniform(-1.0, 1.0);
    for (int k = 0; k < N; ++k)
        for (int i = 0; i < m; ++i) b[(size_t)k * m + i] = (k % 4 == 0) ? uniform(-5.0, 10.0) : uniform(1.0, 10.0);
    for (double& v : c) v = uniform(-1.0, 1.0);

    DeviceData d;
    if (!upload(d, A, b, c, N, m, n)) return false;
    Results ref(N, m, n);
    if (!regular_solve(d, N, m, n, A.size(), ref)) return false;
    Results r0(N, m, n);
    if (!host_solve(A, b, c, N, m, n, r0) || !same(ref, r0, "lp_solve_host before the reset")) return false;
    int phase1 = 0, statuses[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < N; ++k) {
        phase1 += (k % 4 == 0);
        if (ref.status[k] >= 0 && ref.status[k] < 5) ++statuses[ref.status[k]];
    }

    Results r1(N, m, n);
    if (!noalloc_solve(d, N, m, n, r1) || !same(ref, r1, "before the reset")) return false;

    CHECK_CUDA(cudaDeviceReset());  // ends this process's context on the device

    DeviceData d2;
    if (!upload(d2, A, b, c, N, m, n)) return false;
    Results r2(N, m, n);
    if (!noalloc_solve(d2, N, m, n, r2) || !same(ref, r2, "after the reset")) return false;
    Results r3(N, m, n), r4(N, m, n);
    if (!regular_solve(d2, N, m, n, A.size(), r3) || !same(ref, r3, "regular path after the reset")) return false;
    if (!host_solve(A, b, c, N, m, n, r4) || !same(ref, r4, "lp_solve_host after the reset")) return false;
    std::printf("noalloc reset ok: %d LPs of %dx%d (%d with phase I; optimal %d, infeasible %d, unbounded %d)\n", N,
                m, n, phase1, statuses[0], statuses[1], statuses[2]);
    return true;
}

}  // namespace

int main() { return run() ? 0 : 1; }
