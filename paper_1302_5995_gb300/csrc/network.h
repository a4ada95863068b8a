// Conductance networks (Section 6.1, Random Laplacian I and II): the square grid whose
// links carry conductivities sigma; the equation at node k is
//     (1/h^2) sum over its four links of sigma_l (u_k - u_l) = f_k,
// scaled like the five-point Laplacian (unit conductivities give the Laplace problem),
// and the datum at ghost k is the current sigma_k (g_k - u_k')/h through its link.
// The FP64 build runs on a table of five weights per node (centre, E, W, N, S), which
// the stencil lookups of the FP64 kernels take when their c pointer is null.
#pragma once
#include <cuda_runtime.h>

namespace gm {

// sx: n rows of n + 1 x-links, sx[i + (n+1) j] joins (i-1, j) and (i, j); sy: n + 1 rows
// of n y-links, sy[i + n j] joins (i, j-1) and (i, j) (the outermost links reach the
// ghosts).  Writes W (5 n^2 weights) and sig (4n ghost-link conductivities, ghost order).
cudaError_t launch_net_weights(const double *sx, const double *sy, int n, double *W, double *sig, cudaStream_t s);

// T[k + N c] *= sig[k] for k < N, c < ncols: the datum weights of a network's T and F.
cudaError_t launch_scale_rows(double *T, int N, int ncols, const double *sig, cudaStream_t s);

}  // namespace gm
