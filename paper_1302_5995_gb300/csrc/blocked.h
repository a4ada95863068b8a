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
    __nv_bfloat16 *fdig = nullptr;     // [S][sum rows][64]: rows of F
    int64_t fplane = 0;
    int *fex = nullptr;
    __nv_bfloat16 *adig = nullptr, *r0dig = nullptr, *edig = nullptr, *rdig = nullptr;  // [S][sum cols][64]
    int64_t cplane = 0;
    int *aex = nullptr, *r0ex = nullptr, *eex = nullptr, *rex = nullptr;
    float2 *r0 = nullptr;              // [sum cols][64]: first approximation of R
    cudaStream_t s2 = nullptr;         // optional second stream for the look-ahead update
    cudaEvent_t ev_r = nullptr, ev_rest = nullptr;
};

size_t blk_factor_smem(int split);
size_t blk_rgemm_smem(int split);
cudaError_t blk_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                         float2 *ws, int split, BlkScratch &scr, Status *st, int stage, cudaStream_t s, KTimer &kt);

}  // namespace gm
