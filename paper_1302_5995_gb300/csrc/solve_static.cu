// gm_solve_static: the DtN apply with no device allocation of any kind.
//
// gm_solve stages host Dirichlet data and host results through device buffers that it
// takes from the stream-ordered allocator.  Some callers cannot let a library allocate:
// a serving loop that must not touch the allocator once it runs, a host application
// whose device memory is owned by another runtime's pool, or code that may not call
// cudaMalloc at that point.  This entry point stages through one fixed array of device
// memory that is part of the library image instead, so it allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "gm_internal.h"
#include "kernels.h"
#include "mixed.h"

namespace {

// 2 Mi doubles = 16 MiB.  Every GPU that loads the library holds this array until the
// process exits.  All calls share it: calls that overlap on the GPU race on it.
constexpr size_t kStaticDoubles = size_t(2) << 20;
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device.
int scratch_on_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GM_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GM_ECUDA;
        }
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return GM_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gm_solve_static(gm_handle *h, const double *g, double *dudn, int batch, void *stream) {
    if (!h || batch < 0) return GM_EINVAL;
    if (batch == 0) return GM_OK;
    if (!g || !dudn) return GM_EINVAL;
    int n = 0;
    const double *T = gm::handle_dtn(h, &n);
    if (!T) return GM_EUNSUPPORTED;  // an HBS build has no dense T
    const size_t N = 4 * (size_t)n, elems = N * (size_t)batch;
    const bool gd = on_device(g), vd = on_device(dudn);
    if (gd && vd && gm::overlaps(g, dudn, elems)) return GM_EINVAL;  // the apply reads g while it writes dudn
    // a mixed-precision handle applies T by split products, like gm_solve: the digit
    // planes of g (split x batch x kpad bf16) and their exponents also come from the
    // array; every part starts on a 256-byte boundary
    const void *tdig = nullptr;
    const int *tex = nullptr;
    int split = 0;
    const bool mixed = gm::handle_split(h, &tdig, &tex, &split);
    auto up = [](size_t d) { return (d + 31) / 32 * 32; };
    const int kpad = gm::mx_kpad((int)N);
    const size_t g_at = 0, v_at = g_at + (gd ? 0 : up(elems)), dig_at = v_at + (vd ? 0 : up(elems));
    const size_t dig_doubles = mixed ? up((size_t)split * batch * kpad * 2 / 8 + 1) : 0;
    const size_t ex_at = dig_at + dig_doubles;
    const size_t need = ex_at + (mixed ? up((size_t)batch * sizeof(int) / 8 + 1) : 0);
    if (need > kStaticDoubles) return GM_ESCRATCH;
    double *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const double *dg = g;
    double *dv = dudn;
    if (!gd) {
        dg = scratch + g_at;
        if (cudaMemcpyAsync(scratch + g_at, g, elems * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) return GM_ECUDA;
    }
    if (!vd) dv = scratch + v_at;
    cudaError_t e;
    if (mixed)
        e = gm::mx_apply((const __nv_bfloat16 *)tdig, tex, dg, (__nv_bfloat16 *)(scratch + dig_at),
                         (int *)(scratch + ex_at), dv, (int)N, batch, split, s);
    else
        e = gm::launch_apply(T, dg, dv, (int)N, batch, s);
    if (e != cudaSuccess) return GM_ECUDA;
    if (!vd) {
        if (cudaMemcpyAsync(dudn, dv, elems * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GM_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GM_ECUDA;
    }
    return GM_OK;
}
