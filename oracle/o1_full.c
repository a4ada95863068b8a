/*
 * Oracle O1 -- the plain definition of the discrete Dirichlet-to-Neumann map.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links or calls this file; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * What it computes (Section 1.1 problem statement, Section 6 stencil): for each
 * Dirichlet vector g on the 4n ghost nodes, solve the full n^2 x n^2 five-point
 * system
 *     (1/h^2)[4u_k - u_n - u_s - u_w - u_e] + (1/h) b_k [u_e - u_w]
 *                                           + (1/h) c_k [u_n - u_s] + d_k u_k = f_k
 * with the ghost values moved to the right-hand side, then return the outward
 * one-sided flux (g_k - u_{k'})/h at every ghost k, where k' is its only interior
 * neighbour.  There is no nested dissection here: the whole matrix is factored by
 * banded Gaussian elimination with partial pivoting (bandwidth n below, 2n above
 * after pivoting fill), which is exact up to rounding.
 *
 * The body load f is zero except at a few listed nodes (Section 6.3: the solution
 * operator then has two terms, v = G g + F f_hat).  The same solve also serves the
 * Random Laplacian problems of Section 6.1, a square-grid network whose links carry
 * conductivities sigma: the equation at node k is
 *     (1/h^2) sum over its four links of sigma_l (u_k - u_l) = f_k,
 * and the datum at ghost k is the current sigma_k (g_k - u_{k'})/h through its link
 * (scaled like the flux, so unit conductivities give the Laplace operator).
 *
 * Grid: unknown (i, j), i, j = 0..n-1, flat index i + n*j, h = 1/(n+1).
 * Ghost order: counter-clockwise from the south-west corner (south x increasing,
 * east y increasing, north x decreasing, west y decreasing), n per side.
 * Network links: sx[i + (n+1) j] joins (i-1, j) and (i, j), i = 0..n; sy[i + n j] joins
 * (i, j-1) and (i, j), j = 0..n (the outermost ones reach the ghosts).
 *
 * Plain C, FP64, no BLAS.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Band storage: row r keeps columns r-KL .. r+KL+KU at offsets 0 .. W-1. */
typedef struct {
    int N, KL, KU, W;
    double *a;
    int *piv;
} band_t;

static double *bat(band_t *B, int r, int c) { return &B->a[(size_t)r * B->W + (c - r + B->KL)]; }

/* The equation's coefficients: the Section 6 PDE fields, or a conductance network. */
typedef struct {
    int n, net;
    const double *b, *c, *d;  /* PDE: n*n each */
    const double *sx, *sy;    /* network: n (n+1) each, layouts above */
} stencil_t;

/* Conductivity of the link from (i,j) in direction dir (1 east, 2 west, 3 north, 4 south). */
static double link(const stencil_t *S, int i, int j, int dir) {
    int n = S->n;
    switch (dir) {
    case 1: return S->sx[(i + 1) + (n + 1) * j];
    case 2: return S->sx[i + (n + 1) * j];
    case 3: return S->sy[i + n * (j + 1)];
    default: return S->sy[i + n * j];
    }
}

/* Stencil weight of the equation at node (i,j) on its neighbour in direction dir
 * (0 centre, 1 east, 2 west, 3 north, 4 south). */
static double weight(const stencil_t *S, int i, int j, int dir) {
    int n = S->n;
    double h = 1.0 / (n + 1), ih2 = 1.0 / (h * h);
    if (S->net) {
        if (dir) return -link(S, i, j, dir) * ih2;
        return (link(S, i, j, 1) + link(S, i, j, 2) + link(S, i, j, 3) + link(S, i, j, 4)) * ih2;
    }
    int k = i + n * j;
    switch (dir) {
    case 0: return 4.0 * ih2 + S->d[k];
    case 1: return -ih2 + S->b[k] / h;
    case 2: return -ih2 - S->b[k] / h;
    case 3: return -ih2 + S->c[k] / h;
    default: return -ih2 - S->c[k] / h;
    }
}

/* Ghost k -> its interior neighbour (i, j) and the direction from that neighbour to k. */
static void ghost_neighbour(int n, int k, int *i, int *j, int *dir) {
    int side = k / n, t = k % n;
    if (side == 0) { *i = t; *j = 0; *dir = 4; }                /* south ghost below (t,0) */
    else if (side == 1) { *i = n - 1; *j = t; *dir = 1; }       /* east ghost right of (n-1,t) */
    else if (side == 2) { *i = n - 1 - t; *j = n - 1; *dir = 3; } /* north ghost above */
    else { *i = 0; *j = n - 1 - t; *dir = 2; }                  /* west ghost left of (0, .) */
}

/* Assemble A (n^2 x n^2, band n) and factor it in place: partial pivoting within the band. */
static int factor(const stencil_t *S, band_t *B) {
    int n = S->n, N = n * n;
    B->N = N; B->KL = n; B->KU = n; B->W = 2 * n + n + 1;
    B->a = (double *)calloc((size_t)N * B->W, sizeof(double));
    B->piv = (int *)malloc(sizeof(int) * (size_t)N);
    if (!B->a || !B->piv) return -1;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int r = i + n * j;
            *bat(B, r, r) = weight(S, i, j, 0);
            if (i + 1 < n) *bat(B, r, r + 1) = weight(S, i, j, 1);
            if (i > 0) *bat(B, r, r - 1) = weight(S, i, j, 2);
            if (j + 1 < n) *bat(B, r, r + n) = weight(S, i, j, 3);
            if (j > 0) *bat(B, r, r - n) = weight(S, i, j, 4);
        }
    int KL = B->KL, UW = B->KL + B->KU; /* U's upper bandwidth after pivoting */
    for (int k = 0; k < N; ++k) {
        int last = k + KL < N - 1 ? k + KL : N - 1;
        int p = k;
        double best = fabs(*bat(B, k, k));
        for (int r = k + 1; r <= last; ++r) {
            double v = fabs(*bat(B, r, k));
            if (v > best) { best = v; p = r; }
        }
        B->piv[k] = p;
        if (best == 0.0) return -2;
        int cend = k + UW < N - 1 ? k + UW : N - 1;
        if (p != k)
            for (int cc = k; cc <= cend; ++cc) {
                /* row p holds columns up to p+UW >= cend; row k up to k+UW = cend */
                double t = *bat(B, k, cc); *bat(B, k, cc) = *bat(B, p, cc); *bat(B, p, cc) = t;
            }
        double piv = *bat(B, k, k);
        for (int r = k + 1; r <= last; ++r) {
            double l = *bat(B, r, k) / piv;
            *bat(B, r, k) = l;
            if (l != 0.0)
                for (int cc = k + 1; cc <= cend; ++cc) *bat(B, r, cc) -= l * *bat(B, k, cc);
        }
    }
    return 0;
}

static void solve(const band_t *B, double *x) {
    int N = B->N, KL = B->KL, UW = B->KL + B->KU;
    band_t *Bm = (band_t *)B;
    for (int k = 0; k < N; ++k) {
        int p = B->piv[k];
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
        int last = k + KL < N - 1 ? k + KL : N - 1;
        for (int r = k + 1; r <= last; ++r) x[r] -= *bat(Bm, r, k) * x[k];
    }
    for (int k = N - 1; k >= 0; --k) {
        int cend = k + UW < N - 1 ? k + UW : N - 1;
        double s = x[k];
        for (int cc = k + 1; cc <= cend; ++cc) s -= *bat(Bm, k, cc) * x[cc];
        x[k] = s / *bat(Bm, k, k);
    }
}

/* Ghost k's datum weight: 1 for the PDE (the flux), its link's conductivity for a network. */
static double ghost_scale(const stencil_t *S, int k) {
    int i, j, dir;
    if (!S->net) return 1.0;
    ghost_neighbour(S->n, k, &i, &j, &dir);
    return link(S, i, j, dir);
}

/*
 * V[:, v] = G-term + F-term for v < nvec: solve with Dirichlet data G[:, v] and body
 * loads Fl[m + nload v] at the nodes idx[m] (flat i + n j), then take each ghost's
 * datum.  G and V are 4n x nvec column-major; nload may be 0 (idx, Fl unused).
 */
static int apply(const stencil_t *S, int nvec, const double *G, int nload, const int *idx,
                 const double *Fl, double *V) {
    int n = S->n, N = n * n;
    for (int m = 0; m < nload; ++m)
        if (idx[m] < 0 || idx[m] >= N) return -3;
    band_t B;
    memset(&B, 0, sizeof B);
    int rc = factor(S, &B);
    if (rc) { free(B.a); free(B.piv); return rc; }
    double h = 1.0 / (n + 1);
    double *x = (double *)malloc(sizeof(double) * (size_t)N);
    if (!x) { free(B.a); free(B.piv); return -1; }
    for (int v = 0; v < nvec; ++v) {
        const double *g = G + (size_t)v * 4 * n;
        memset(x, 0, sizeof(double) * (size_t)N);
        for (int m = 0; m < nload; ++m) x[idx[m]] += Fl[(size_t)v * nload + m];
        for (int k = 0; k < 4 * n; ++k) {
            int i, j, dir;
            ghost_neighbour(n, k, &i, &j, &dir);
            x[i + n * j] -= weight(S, i, j, dir) * g[k];
        }
        solve(&B, x);
        for (int k = 0; k < 4 * n; ++k) {
            int i, j, dir;
            ghost_neighbour(n, k, &i, &j, &dir);
            V[(size_t)v * 4 * n + k] = ghost_scale(S, k) * (g[k] - x[i + n * j]) / h;
        }
    }
    free(x); free(B.a); free(B.piv);
    return 0;
}

static void assemble(const stencil_t *S, double *A) {
    int n = S->n, N = n * n;
    memset(A, 0, sizeof(double) * (size_t)N * N);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int r = i + n * j;
            A[(size_t)r * N + r] = weight(S, i, j, 0);
            if (i + 1 < n) A[(size_t)r * N + r + 1] = weight(S, i, j, 1);
            if (i > 0) A[(size_t)r * N + r - 1] = weight(S, i, j, 2);
            if (j + 1 < n) A[(size_t)r * N + r + n] = weight(S, i, j, 3);
            if (j > 0) A[(size_t)r * N + r - n] = weight(S, i, j, 4);
        }
}

/*
 * V[:, v] = DtN(G[:, v]) for v < nvec.  G and V are 4n x nvec, column-major (vector v
 * starts at v*4n).  b, c, d are n*n, flat index i + n*j.  Returns 0, or -1 (no memory),
 * -2 (an exactly zero pivot: the discrete problem is singular).
 */
int o1_dtn_apply(int n, const double *b, const double *c, const double *d, int nvec,
                 const double *G, double *V) {
    stencil_t S = {n, 0, b, c, d, NULL, NULL};
    return apply(&S, nvec, G, 0, NULL, NULL, V);
}

/* The same with body loads: V = G-term + F-term (Section 6.3); Fl is nload x nvec
 * column-major, idx the load nodes.  -3: a load index outside the grid. */
int o1_apply_loads(int n, const double *b, const double *c, const double *d, int nvec,
                   const double *G, int nload, const int *idx, const double *Fl, double *V) {
    stencil_t S = {n, 0, b, c, d, NULL, NULL};
    return apply(&S, nvec, G, nload, idx, Fl, V);
}

/* The conductance network (Section 6.1 Random Laplacian) with optional body loads. */
int o1_net_apply(int n, const double *sx, const double *sy, int nvec, const double *G, int nload,
                 const int *idx, const double *Fl, double *V) {
    stencil_t S = {n, 1, NULL, NULL, NULL, sx, sy};
    return apply(&S, nvec, G, nload, idx, Fl, V);
}

/* Dense A (n^2 x n^2, row-major) for the plain-definition pins on tiny grids. */
int o1_assemble_dense(int n, const double *b, const double *c, const double *d, double *A) {
    stencil_t S = {n, 0, b, c, d, NULL, NULL};
    assemble(&S, A);
    return 0;
}

int o1_net_assemble_dense(int n, const double *sx, const double *sy, double *A) {
    stencil_t S = {n, 1, NULL, NULL, NULL, sx, sy};
    assemble(&S, A);
    return 0;
}
