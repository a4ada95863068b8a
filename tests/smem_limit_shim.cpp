// Test-only shim for csrc/smem_limit.h on the CPU.  The fake cudaFuncSetAttribute keeps
// each function's dynamic shared-memory limit (and refuses limits above 227 KB, as the
// device does); a fake launch fails when its request is above the limit in force, as a
// real launch would.  No GPU is involved.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include "../paper_1302_5995_gb300/csrc/smem_limit.h"

namespace {
std::mutex mu;
std::map<const void *, int> limit;
int n_set = 0;
const int kMaxSmem = 227 * 1024;
char fn_a, fn_b;  // two fake kernels

int launch(const void *fn, int bytes) {
    std::lock_guard<std::mutex> lk(mu);
    return bytes <= limit[fn] ? 0 : 1;
}
}  // namespace

extern "C" {
cudaError_t cudaGetDevice(int *d) {
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaFuncSetAttribute(const void *fn, cudaFuncAttribute attr, int v) {
    if (attr != cudaFuncAttributeMaxDynamicSharedMemorySize || v > kMaxSmem) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(mu);
    limit[fn] = v;
    ++n_set;
    return cudaSuccess;
}

// Two launches interleaved the way two host threads can run them: thread 1 prepares a
// launch of `big` bytes, thread 2 prepares one of `small` bytes, then thread 1 launches.
// raise = 0 prepares by setting the limit to the launch's own size, raise = 1 by
// raise_smem_limit.  Returns the number of failed launches (0, 1 or 2).
int shim_interleaved(int raise, int big, int small) {
    const void *fn = &fn_a;
    auto prep = [&](int bytes) {
        return raise ? (int)gm::raise_smem_limit(fn, (size_t)bytes)
                     : (int)cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    if (prep(big) || prep(small)) return -1;
    return launch(fn, big) + launch(fn, small);
}

// `threads` host threads, each preparing (by raise_smem_limit) and launching `iters`
// random requests on two functions; returns the failed launches.
int shim_stress(int threads, int iters, unsigned seed) {
    std::vector<std::thread> th;
    std::vector<int> fails(threads, 0);
    for (int t = 0; t < threads; ++t)
        th.emplace_back([&, t] {
            std::mt19937 rng(seed + 977u * t);
            std::uniform_int_distribution<int> size(0, 200 * 1024);
            for (int i = 0; i < iters; ++i) {
                const void *fn = (i + t) & 1 ? (const void *)&fn_a : (const void *)&fn_b;
                const int bytes = size(rng);
                if (gm::raise_smem_limit(fn, (size_t)bytes) != cudaSuccess) {
                    ++fails[t];
                    continue;
                }
                std::this_thread::yield();
                fails[t] += launch(fn, bytes);
            }
        });
    for (auto &x : th) x.join();
    int f = 0;
    for (int x : fails) f += x;
    return f;
}

// A request above the device's limit fails and leaves the limit where it was: returns
// the failed launches of the earlier size after the refusal (0 expected), -1 if the
// refusal did not happen.
int shim_too_large(void) {
    const void *fn = &fn_b;
    if (gm::raise_smem_limit(fn, 64 * 1024) != cudaSuccess) return -1;
    if (gm::raise_smem_limit(fn, (size_t)kMaxSmem + 1) == cudaSuccess) return -1;
    return launch(fn, 64 * 1024);
}

int shim_limit(int which) {
    std::lock_guard<std::mutex> lk(mu);
    return limit[which ? (const void *)&fn_b : (const void *)&fn_a];
}
int shim_sets(void) {
    std::lock_guard<std::mutex> lk(mu);
    return n_set;
}
}  // extern "C"
