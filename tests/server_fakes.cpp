// Test-only fakes for running the serving runtime (csrc/server.cpp) on the CPU: the
// CUDA runtime calls it makes act on host memory, gm_solve / gm_info / gm_free act on
// fake operators that record every call (gm_solve_many records each operator), and
// gm_build_ex builds such operators.  A gate
// can hold a solve inside the worker so that a test can queue requests behind it
// (continuous batching) or try to evict an operator that is being served.  Every wait
// here has a time limit.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../include/gm.h"

namespace {

struct FakeOp {
    int n, tag, solve_rc;
    long long bytes;
};

std::mutex mu;
std::condition_variable cv;
bool gate_closed = false;
int blocked = 0;
std::vector<int> call_tag, call_batch, freed_tag;

}  // namespace

extern "C" {

// ---- CUDA runtime calls of the server, on host memory
cudaError_t cudaGetDevice(int *d) { *d = 0; return cudaSuccess; }
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned int) {
    *s = reinterpret_cast<cudaStream_t>(new char[1]);
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithPriority(cudaStream_t *s, unsigned int, int) {
    *s = reinterpret_cast<cudaStream_t>(new char[1]);
    return cudaSuccess;
}
cudaError_t cudaDeviceGetStreamPriorityRange(int *lo, int *hi) {
    *lo = 0;
    *hi = -5;
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) { delete[] reinterpret_cast<char *>(s); return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMalloc(void **p, size_t bytes) {
    *p = std::malloc(bytes);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p) { std::free(p); return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind, cudaStream_t) {
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }

// ---- the library calls the server makes, on fake operators
int gm_solve(gm_handle *h, const double *g, double *dudn, int batch, void *) {
    FakeOp *op = reinterpret_cast<FakeOp *>(h);
    {
        std::unique_lock<std::mutex> lk(mu);
        call_tag.push_back(op->tag);
        call_batch.push_back(batch);
        if (gate_closed) {
            ++blocked;
            cv.notify_all();
            cv.wait_for(lk, std::chrono::seconds(10), [] { return !gate_closed; });
            --blocked;
        }
    }
    if (op->solve_rc) return op->solve_rc;
    for (long long i = 0; i < 4LL * op->n * batch; ++i) dudn[i] = 1000.0 * op->tag + 2.0 * g[i];
    return GM_OK;
}

// The grouped solve: every operator enters the call log in order (one gate hold per
// call); the result is the first failing operator's code.
int gm_solve_many(int count, gm_handle *const *hs, const double *const *g, double *const *dudn, const int *batch,
                  void *) {
    {
        std::unique_lock<std::mutex> lk(mu);
        for (int i = 0; i < count; ++i) {
            call_tag.push_back(reinterpret_cast<FakeOp *>(hs[i])->tag);
            call_batch.push_back(batch[i]);
        }
        if (gate_closed) {
            ++blocked;
            cv.notify_all();
            cv.wait_for(lk, std::chrono::seconds(10), [] { return !gate_closed; });
            --blocked;
        }
    }
    int rc = GM_OK;
    for (int i = 0; i < count; ++i) {
        FakeOp *op = reinterpret_cast<FakeOp *>(hs[i]);
        if (op->solve_rc) {
            if (rc == GM_OK) rc = op->solve_rc;
            continue;
        }
        for (long long k = 0; k < 4LL * op->n * batch[i]; ++k) dudn[i][k] = 1000.0 * op->tag + 2.0 * g[i][k];
    }
    return rc;
}

void gm_opts_default(gm_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = GM_PREC_FP64;
}

// A build makes a fake operator tagged with its n (10 n bytes resident); n = 13 fails
// as a singular problem.  Builds enter the call log with batch -1.
int gm_build_ex(const gm_opts *, const double *, const double *, const double *, int n, int, double,
                gm_handle **out) {
    {
        std::lock_guard<std::mutex> lk(mu);
        call_tag.push_back(n);
        call_batch.push_back(-1);
    }
    if (n == 13) return GM_ESINGULAR;
    *out = reinterpret_cast<gm_handle *>(new FakeOp{n, n, 0, 10LL * n});
    return GM_OK;
}

int gm_info(gm_handle *h, gm_info_t *info) {
    FakeOp *op = reinterpret_cast<FakeOp *>(h);
    std::memset(info, 0, sizeof(*info));
    info->n = op->n;
    info->resident_bytes = op->bytes;
    return GM_OK;
}

void gm_free(gm_handle *h) {
    if (!h) return;
    FakeOp *op = reinterpret_cast<FakeOp *>(h);
    {
        std::lock_guard<std::mutex> lk(mu);
        freed_tag.push_back(op->tag);
    }
    delete op;
}

// ---- control from the tests
gm_handle *fake_op(int n, long long bytes, int tag, int solve_rc) {
    return reinterpret_cast<gm_handle *>(new FakeOp{n, tag, solve_rc, bytes});
}

void fake_reset(void) {
    std::lock_guard<std::mutex> lk(mu);
    gate_closed = false;
    call_tag.clear();
    call_batch.clear();
    freed_tag.clear();
    cv.notify_all();
}

void fake_gate(int closed) {
    std::lock_guard<std::mutex> lk(mu);
    gate_closed = closed != 0;
    cv.notify_all();
}

// 1 once a solve is held at the gate, 0 after timeout_ms without one.
int fake_wait_blocked(int timeout_ms) {
    std::unique_lock<std::mutex> lk(mu);
    return cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [] { return blocked > 0; }) ? 1 : 0;
}

// The recorded solves (operator tag, vectors) in call order; returns their number.
int fake_calls(int *tags, int *batches, int cap) {
    std::lock_guard<std::mutex> lk(mu);
    int k = 0;
    for (; k < (int)call_tag.size() && k < cap; ++k) {
        tags[k] = call_tag[k];
        batches[k] = call_batch[k];
    }
    return (int)call_tag.size();
}

int fake_freed(int *tags, int cap) {
    std::lock_guard<std::mutex> lk(mu);
    int k = 0;
    for (; k < (int)freed_tag.size() && k < cap; ++k) tags[k] = freed_tag[k];
    return (int)freed_tag.size();
}

}  // extern "C"
