// Blocked Gauss-Jordan sweep with block-local pivoting (mixed precision).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "gm_internal.h"
#include "kernels.h"

#define BLK_NB 64

namespace gm {

struct BlkScratch {
    __nv_bfloat16 *x_dig = nullptr, *a11_dig = nullptr;  // [S][systems * 64][64]: rows of X0, A11
    int64_t inv_plane = 0;                                // systems * 64 * 64
    int *x_ex = nullptr, *a11_ex = nullptr;               // [systems * 64]
    float *pmag = nullptr;             // [systems][64]: |pivot| of the block elimination
    // digit planes of F and R, two sets used by alternate block steps (the update of one
    // step still reads its set while the next step's R kernel writes the other)
    __nv_bfloat16 *fdig[2] = {nullptr, nullptr};  // [S][sum rows][64]: rows of F
    int64_t fplane = 0;
    int *fex[2] = {nullptr, nullptr};
    __nv_bfloat16 *rdig[2] = {nullptr, nullptr};  // [S][sum cols][64]: columns of R
    int64_t cplane = 0;
    int *rex[2] = {nullptr, nullptr};
    // look-ahead (optional): the chain factor -> R -> the next block's update runs on s1
    // (high priority), the rest of each update on s2; events ev_r (R done), ev_rest
    // (the rest done) and ev_join (entry and exit of the sweep)
    cudaStream_t s1 = nullptr, s2 = nullptr;
    cudaEvent_t ev_r = nullptr, ev_rest = nullptr, ev_join = nullptr;
    int wait_limit = 1 << 22;  // polls of the tensor-core completion wait before GM_ETIMEOUT
    int rtile32_max = 96;      // R kernel: 32-column tiles while systems x 64-column tiles <= this
    int upd_tiles = 0;         // bulk update: 64-column tiles per CTA (0: one wave, < 0: one tile per CTA)
    int sms = 152;             // multiprocessors of the device
    // early-factor schedule (needs the look-ahead streams, s3 and the second factor set):
    // the chain is R of the next block's columns -> that block's pivot tile -> its factor;
    // the rest of R, the diagonal tile two blocks ahead and the next band on s3 (high
    // priority), the bulk of the update on s2
    bool early = false;
    bool a11first = false;  // look-ahead: only the next diagonal tile on the chain (needs s3, ev_next)
    cudaStream_t s3 = nullptr;
    cudaEvent_t ev_rr = nullptr, ev_next = nullptr, ev_rest2[2] = {nullptr, nullptr};
    __nv_bfloat16 *x_dig2 = nullptr, *a11_dig2 = nullptr;  // the factor's second output set
    int *x_ex2 = nullptr, *a11_ex2 = nullptr;
    float *pmag2 = nullptr;
};

size_t blk_factor_smem(int split);
size_t blk_rgemm_smem(int split);
cudaError_t blk_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                         float2 *ws, int split, BlkScratch &scr, Status *st, int stage, cudaStream_t s, KTimer &kt);

}  // namespace gm
