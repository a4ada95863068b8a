/*
 * gm.h -- C ABI of the GB300 builder/applier of discrete Dirichlet-to-Neumann maps.
 *
 * Problem (Section 1.1, eq. basic; stencil of Section 6):
 *     -Lap u + b u_x + c u_y + d u = 0 on the unit square,  u = g on its boundary,
 * discretised on an n x n grid of UNKNOWN nodes with h = 1/(n+1): node (i, j) sits at
 * ((i+1)h, (j+1)h) and has flat index i + n*j.  The equation at node k is
 *     (1/h^2)[4u_k - u_n - u_s - u_w - u_e] + (1/h) b_k [u_e - u_w]
 *                                          + (1/h) c_k [u_n - u_s] + d_k u_k = 0.
 * The Dirichlet data g lives on the 4n non-corner "ghost" nodes one step outside the
 * grid, ordered counter-clockwise from the south-west corner: south (x increasing),
 * east (y increasing), north (x decreasing), west (y decreasing), n per side.
 * The Neumann datum returned at ghost k is the outward one-sided flux
 *     (g_k - u_{k'})/h,  k' = the only unknown next to ghost k,
 * so the built operator is the dense 4n x 4n matrix T with  dudn = T g.
 *
 * Build (Sections 2-3): quad-tree of boxes whose edges are at most `leaf` (Section 2),
 * leaf Schur complements S = A_bb - A_bi A_ii^{-1} A_ib (Section 3.1, eq. def_schur_nd),
 * level-by-level pairwise merges (Section 3.2, eq. S_fromtwo_nd; four-child merge as
 * three pairwise merges, Section 3.3), and the root (Section 3.3 step 4):
 *     T = (I - P S_root^{-1} B)/h,
 * with B the ring nodes' weights on the ghosts (negated) and P the ghost-to-ring map.
 * Solve (Section 1.1): dudn = T g for a batch of Dirichlet vectors.
 *
 * Conventions for every entry point:
 *   - Arrays are FP64.  A pointer may be host memory or device memory of the current
 *     device; the library detects which (cudaPointerGetAttributes) and copies host
 *     data through the call's stream.
 *   - Matrices and vector batches are column-major: vector v of a batch of 4n-vectors
 *     starts at element v*4n.
 *   - Inputs are borrowed for the duration of the call only; outputs are caller-owned.
 *   - Return value: GM_OK (0) or a negative GM_E* code; gm_strerror() names it.
 *   - Handles are not thread-safe: one thread at a time per handle.
 *   - `stream` arguments are a cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef GM_H
#define GM_H

#ifdef __cplusplus
extern "C" {
#endif

#define GM_OK 0
#define GM_EINVAL (-1)       /* bad argument: sizes, NULL pointers, leaf < 3, ...      */
#define GM_ENOMEM (-2)       /* a device or pinned-host allocation failed               */
#define GM_ESINGULAR (-3)    /* an exactly zero / non-finite pivot: the Dirichlet
                                problem of some box (or of the whole grid) is singular;
                                gm_info().bad_stage names where                          */
#define GM_ETIMEOUT (-4)     /* a bounded device-side wait gave up                       */
#define GM_ECUDA (-5)        /* a CUDA runtime call failed                               */
#define GM_EUNSUPPORTED (-6) /* valid request the library does not support              */
#define GM_ESCRATCH (-7)     /* request larger than the fixed scratch of gm_solve_static */

#define GM_PREC_FP64 0  /* every step in FP64 */
#define GM_PREC_MIXED 1 /* double-float (FP32 pair) storage, FP32 pivot search, FP64 pivot
                           blocks, and every dense update as exact split products of
                           bf16 integer digits on the tensor cores                       */

typedef struct gm_handle gm_handle;

typedef struct gm_opts {
    int precision;    /* GM_PREC_FP64 (default) or GM_PREC_MIXED                        */
    int keep_levels;  /* nonzero: keep every intermediate Schur complement for
                         gm_get_schur() (costs the memory of all levels)                 */
    void *stream;     /* cudaStream_t for the build (NULL = legacy default stream)      */
    int panel_width;  /* pivot panel width of the partial-pivoting eliminations
                         (0 = default 16, the fastest measured)                        */
    int timing;       /* nonzero: time every kernel launch of the build with CUDA events
                         (per kernel family, reported by gm_info)                       */
    int split_digits; /* GM_PREC_MIXED: 7-bit digits per operand of the split products,
                         3..6 (0 = default 6); more digits = more accuracy, more work.
                         The automatic fallback (GM_PIVOT_AUTO) is calibrated for 6:
                         with fewer digits the digit truncation, amplified by the
                         problem's conditioning, is not checked.                     */
    int pivoting;     /* GM_PREC_MIXED: GM_PIVOT_AUTO (default), GM_PIVOT_BLOCK or
                         GM_PIVOT_PARTIAL (see below); GM_PREC_FP64 always uses partial  */
    int hbs_leaf;     /* tol > 0: node size m of the HBS trees (0 = default 64; 2..192) */
    int hbs_min_edge; /* tol > 0, FP64: pairwise merges whose shared edge has at least
                         this many nodes solve their interface system by HBS block
                         elimination (0 = default 128)                                  */
    int timing_mask;  /* with timing: time only the families whose bit is set
                         (bit GM_K_*; 0 = all)                                          */
    int background;   /* nonzero: every stream the build creates for itself takes the
                         lowest priority (a build beside latency-bound solves)          */
    int wait_limit;   /* polls of a bounded device-side wait (on the tensor cores'
                         completion or a bulk copy) before the build gives up with
                         GM_ETIMEOUT (0 = default 2^22, far beyond any normal wait; a
                         negative value gives up at the first wait, which tests the
                         path); a kernel that gives up still waits, for a fixed bound,
                         for its own copies and products in flight before it releases
                         its tensor memory and returns                                   */
    int graph;        /* nonzero (tol = 0, no keep_levels, no timing): the first build of
                         a plan runs as usual and records every launch of its build into a
                         CUDA graph, kept with its own buffers (coefficients, Schur
                         complements, workspaces, outputs) per plan and options; later
                         builds of the plan copy their coefficients in, replay the graph
                         and copy the operator out (at most 8 graphs are kept, least
                         recently used dropped)                                         */
    int autotune;     /* nonzero: the first build of a plan times a few launch shapes and
                         schedules (the R kernel's tile width, tiles per CTA of the bulk
                         update, the early-factor and A11-first schedules, the tcgen05
                         merge-update bound) and keeps the fastest for every later build
                         of that plan and options.  The environment variable GM_TUNE
                         (e.g. "early=1,upd_tiles=-1"; keys rtile32_max, tc_min_k, early,
                         a11, upd_tiles) forces a choice, for testing                    */
} gm_opts;

/* Pivoting of the mixed-precision dense eliminations.
 *   GM_PIVOT_PARTIAL: partial pivoting over all remaining rows, 16-column panels.
 *   GM_PIVOT_BLOCK:   64-column blocks; pivots are chosen among the rows of the block
 *                     (its 64 x 64 pivot block is inverted with partial pivoting).
 *   GM_PIVOT_AUTO:    a problem whose reaction term makes the operator indefinite
 *                     (d < -2 pi^2 everywhere, 2 pi^2 the smallest Dirichlet eigenvalue
 *                     of -Laplace on the unit square) is built in FP64 from the start;
 *                     the others
 *                     use block pivoting, with a check per problem: if a row below some
 *                     block held an entry more than 16x that block column's pivot (partial
 *                     pivoting would have chosen differently), or if the one refinement
 *                     step of a block solve contracted by less than 2^13 (an ill-
 *                     conditioned pivot block, as in indefinite Helmholtz problems), that
 *                     problem is built again in FP64.  Mixed-precision digit products lose
 *                     about as many digits as such problems amplify, so FP64 is the only
 *                     safe choice for them.  gm_info().pivot_fallback and .precision
 *                     report it.  On a batch only the flagged problems are rebuilt. */
#define GM_PIVOT_AUTO 0
#define GM_PIVOT_BLOCK 1
#define GM_PIVOT_PARTIAL 2

/* Kernel families reported by gm_info when gm_opts.timing is set. */
#define GM_K_LEAF 0        /* leaf elimination                                          */
#define GM_K_ASSEMBLE 1    /* gather [M | Z] of the merges, [S | B] of the root          */
#define GM_K_PANEL 2       /* pivot search and panel factorisation                      */
#define GM_K_PIVROWS 3     /* row interchanges + triangular solves of the pivot rows    */
#define GM_K_GJUPDATE 4    /* rank-nb update of all non-pivot rows                      */
#define GM_K_MERGEUPDATE 5 /* Schur update S_parent = C - Y X with ring scatter          */
#define GM_K_ROOT 6        /* T = (I - P X)/h                                            */
#define GM_K_NFAM 7

typedef struct gm_info_t {
    int n, leaf, levels;          /* grid size, leaf edge, number of tree levels L       */
    int precision;                /* precision mode the handle was built with            */
    long long dtn_bytes;          /* device bytes of the DtN matrix                      */
    long long peak_workspace;     /* largest device workspace the build held             */
    double min_pivot_ratio;       /* min |pivot| / (4/h^2) over all eliminations         */
    int bad_stage;                /* stage index of a GM_ESINGULAR failure, else -1      */
    int launches;                 /* kernels launched by the build                       */
    double kernel_ms[GM_K_NFAM];      /* device time per kernel family (timing builds)   */
    double kernel_flops[GM_K_NFAM];   /* algorithmic flops per family (always counted)   */
    int kernel_launches[GM_K_NFAM];   /* launches per family                             */
    int pivoting;                     /* pivoting actually used (GM_PIVOT_BLOCK/PARTIAL;
                                         PARTIAL for every FP64 build)                    */
    int pivot_fallback;               /* 1 if GM_PIVOT_AUTO rebuilt this problem in FP64 */
    double refine_ratio;              /* block pivoting: largest |X0 E| / |R| of the one
                                         refinement step of a block solve (0 otherwise)  */
    int hbs_levels;                   /* tol > 0: levels L of the root's HBS tree          */
    int hbs_max_rank;                 /* tol > 0: largest node rank                        */
    long long hbs_bytes;              /* tol > 0: device bytes of the HBS factors          */
    long long resident_bytes;         /* device bytes the handle holds after the build     */
    int hbs_merges;                   /* tol > 0: merges built by the accelerated merge   */
    int hbs_update_rank;              /* tol > 0: largest rank of their S13 / S24 blocks   */
    long long hbs_operator_bytes;     /* tol > 0: bytes of the root operator in HBS form
                                         (D, U, V, B at the node ranks; the paper's M(n)) */
    int load_rank;                    /* body loads: rank of F after
                                         gm_compress_load_operator (-1: F dense)         */
    int hbs_fallbacks;                /* tol > 0: merges and roots left to the dense
                                         elimination because an HBS form was not possible
                                         (a rank above the cap) or Algorithm 1's inverse
                                         failed its residual check (a relative residual
                                         above 1e-3 on random vectors)                    */
} gm_info_t;

/* Fill *opts with defaults (FP64, no kept levels, default stream). */
void gm_opts_default(gm_opts *opts);

/*
 * Build the DtN operator of the problem above (Sections 2-3).
 *   b, c, d : n*n coefficient values at the unknown nodes, flat index i + n*j.
 *   n       : grid of unknowns, n >= 2.
 *   leaf    : largest leaf-box edge (Section 2's N_leaf, as an edge): the tree has the
 *             smallest L with ceil(n / 2^L) <= leaf, 3 <= leaf (leaf >= n: one leaf).
 *             GM_EINVAL if the tree would hold a box narrower than 2 nodes (only
 *             possible for leaf = 3, when 1.5 < n / 2^L < 2): such a box has no ring.
 *             The leaf kernels keep a leaf's band in shared memory up to edge 17; a
 *             wider leaf's Schur complement is formed by eliminating its interior in
 *             nested-dissection order (the tree continues below the requested level
 *             with boxes of edge <= 16, whose splits are those of every level), the same
 *             S up to rounding.  gm_info().levels is the requested tree's L.
 *   tol     : 0 selects the all-dense build.  tol > 0 compresses the root Schur
 *             complement to HBS form at local relative tolerance tol (Section 4; node
 *             size gm_opts.hbs_leaf) and inverts it by Algorithm 1 (Section 5); the
 *             solve then applies Algorithm 2 instead of a dense T.  In FP64 builds the
 *             pairwise merges with a shared edge of at least gm_opts.hbs_min_edge nodes
 *             solve their interface system by the accelerated Step 1 (HBS inverses of
 *             S33 and of its Schur complement) and form the parent from the low-rank
 *             factors of S13 and S24 (Steps 2-3, eq. matmult); the merges of a stage run
 *             side by side on host threads.  A merge whose node ranks exceed the cap
 *             (480, the largest sample count of 512 less its oversampling of 32), or
 *             whose Algorithm 1 inverse fails its residual check (relative residual above
 *             1e-3 on four Gaussian vectors), is eliminated densely; so is a root whose
 *             inverse fails the check (gm_info.hbs_fallbacks counts them).
 *             GM_EUNSUPPORTED if a root node's rank exceeds the cap (the root does not
 *             compress enough; build with tol = 0).
 *   out     : receives a new handle that owns all device memory of the operator.
 * Blocks the calling thread until the build has finished on the device.  Temporaries
 * come from a stream-ordered memory pool the library keeps per device; it does not
 * return freed memory to the system (later builds reuse it), so the process holds the
 * largest build's workspace (peak_workspace) after the first build.
 */
int gm_build(const double *b, const double *c, const double *d, int n, int leaf, double tol,
             gm_handle **out);
int gm_build_ex(const gm_opts *opts, const double *b, const double *c, const double *d, int n,
                int leaf, double tol, gm_handle **out);

/* One problem of a batched build. */
typedef struct gm_problem {
    const double *b, *c, *d; /* n*n coefficients each (host or device), index i + n*j */
    int n, leaf;             /* as for gm_build                                      */
} gm_problem;

/*
 * Build `count` independent operators in one sweep (Section 3.3's level-by-level order
 * applied to all of them together): all leaves in one launch, then for each tree level,
 * counted from the root, one stage of horizontal and one of vertical pairwise merges over
 * every problem that has that level, then all roots in one batched elimination.
 * Problems may differ in n and leaf.  outs[p] receives problem p's handle (freed
 * separately).  keep_levels is not supported here (GM_EUNSUPPORTED).  On an error no
 * handle is returned.  The same opts apply to every problem.
 */
int gm_build_batch(int count, const gm_problem *probs, const gm_opts *opts, double tol,
                   gm_handle **outs);

/*
 * Solve stage (Section 1.1): dudn[:, v] = T g[:, v] for v < batch.
 *   g, dudn : 4n x batch, column-major, host or device.  They must not overlap
 *             (GM_EINVAL when both are device buffers that do).
 * With device pointers the call is asynchronous on `stream`; with a host pointer it
 * returns after the result has reached the host.
 */
int gm_solve(gm_handle *h, const double *g, double *dudn, int batch, void *stream);

/*
 * Solve stage for several operators in one call: dudn[i] = T_i g[i] for i < count, where
 * g[i] and dudn[i] are 4 n_i x batch[i] column-major DEVICE buffers of operator hs[i]
 * (the paper has no such call: it batches the vectors of a serving loop).  Dense
 * operators of the same precision share one apply launch over all their vectors (a
 * descriptor per operator); HBS operators run Algorithm 2 each.  Asynchronous on
 * `stream`.  GM_EINVAL for a NULL array, a NULL handle, a negative batch or a host
 * pointer.  Buffers must not overlap one another.
 */
int gm_solve_many(int count, gm_handle *const *hs, const double *const *g, double *const *dudn, const int *batch,
                  void *stream);

/* Copy the dense 4n x 4n DtN matrix (column-major) to T_out (host or device).  For an
 * HBS build (tol > 0) T is formed by applying the solve to the identity. */
int gm_get_dtn(gm_handle *h, double *T_out);

/*
 * Copy the Schur complement of the box [x0, x0+a) x [y0, y0+b) -- a leaf, a half-box
 * rectangle of a four-child merge, or a box of any level -- to S_out, an r x r
 * column-major matrix over the box's ring, r = 2a + 2b - 4, ring ordered
 * counter-clockwise from the box's south-west corner.  Needs keep_levels at build time
 * (else GM_EUNSUPPORTED); GM_EINVAL if no such box exists in the tree.
 */
int gm_get_schur(gm_handle *h, int x0, int y0, int a, int b, double *S_out);

/*
 * gm_solve_static -- gm_solve without any device allocation.  The paper has no
 * counterpart; it exists for callers that cannot let a library allocate device memory:
 * a serving loop that must not touch the allocator once it runs, or a host application
 * whose device memory belongs to another runtime's pool.
 *   Same arguments and result as gm_solve (a mixed-precision handle gets the same
 *   split-product apply).  Host g / dudn, and for a mixed-precision handle the digit
 *   planes of g (split x batch x kpad bf16, kpad = 4n rounded up to 16) and their batch
 *   exponents, are staged through one fixed 16 MiB array of device memory inside the
 *   library (2^21 doubles; every GPU that loads the library holds it until the process
 *   exits) instead of freshly allocated buffers; device g / dudn are used in place.
 *   Limit: the parts above, each rounded up to 256 bytes, at most 2^21 doubles in total,
 *   else GM_ESCRATCH and nothing is done.  GM_EINVAL if device g and dudn overlap.
 *   The first call on a device looks up the array's device address (once per device);
 *   make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents: calls that overlap
 *   on the GPU (other streams, other threads) race on it and must be serialised by the
 *   caller.
 *   Dense operators only: a handle built with tol > 0 returns GM_EUNSUPPORTED.
 */
int gm_solve_static(gm_handle *h, const double *g, double *dudn, int batch, void *stream);

/*
 * Body loads at fixed nodes (Section 6.3).  With a body load f_k added to the Section 6
 * equation at each of nbody listed unknowns, the boundary data become
 *     dudn = T g + F f_hat,   F: 4n x nbody,
 * T the DtN matrix of gm_build and F the map from the loads to the same one-sided
 * fluxes.  Every box carries, beside its Schur complement, a load map from the loads
 * inside it to its ring's right-hand side (leaf: Section 3.1's f_b - A_bi A_ii^{-1} f_i;
 * merge: Section 3.2's updated right-hand side, solved with the merge's interface
 * system as extra columns); the root gives F.
 *   gm_build_loads : body = nbody distinct flat indices i + n*j (a HOST array, read
 *                    during the call); column c of F belongs to body[c].  b, c, d, n,
 *                    leaf, opts as gm_build_ex.  FP64 only: GM_EUNSUPPORTED for a mixed
 *                    precision or keep_levels request.  GM_EINVAL for an empty, repeated
 *                    or out-of-grid list.  The handle also serves gm_solve (T g alone),
 *                    gm_get_dtn and gm_info (resident_bytes counts T and F).
 *   gm_solve_loads : dudn[:, v] = T g[:, v] + F f[:, v]; g, dudn 4n x batch, f nbody x
 *                    batch, column-major, host or device; pointer rules as gm_solve.
 *                    GM_EUNSUPPORTED for a handle built without loads.
 *   gm_get_load_operator : copy F (4n x nbody, column-major) to F_out, host or device.
 */
int gm_build_loads(const gm_opts *opts, const double *b, const double *c, const double *d, int n, int leaf,
                   const int *body, int nbody, gm_handle **out);
int gm_solve_loads(gm_handle *h, const double *g, const double *f, double *dudn, int batch, void *stream);
int gm_get_load_operator(gm_handle *h, double *F_out);
/*
 * The low-rank form of the load operator (Section 6.3: F, built uncompressed, is then
 * replaced by a low-rank approximation): F ~ L R with L (4n x k) an orthonormal basis of
 * the range of a Gaussian sample of F, truncated at the first |R_jj| <= tol |R_11| of its
 * pivoted QR, and R = L^T F (k x nbody).  The dense F is released; gm_solve_loads then
 * applies L (R f), gm_get_load_operator returns L R, gm_info reports k as load_rank and
 * resident_bytes the smaller footprint.  GM_EINVAL for tol <= 0; GM_EUNSUPPORTED for a
 * handle without loads or one already compressed.  Blocks until done.
 */
int gm_compress_load_operator(gm_handle *h, double tol);

/*
 * Conductance networks (Section 6.1, Random Laplacian I and II): the square grid whose
 * links carry conductivities sigma, each node's equation
 *     (1/h^2) sum over its four links of sigma_l (u_k - u_l) = f_k
 * (scaled like the five-point Laplacian: unit conductivities give the Laplace problem),
 * and the datum at ghost k the current sigma_k (g_k - u_k')/h through its link, so that T
 * is the network's symmetric response matrix with T 1 = 0.
 *   sx : n rows of n + 1 x-links, sx[i + (n+1) j] joins (i-1, j) and (i, j), i = 0..n
 *        (i = 0 and i = n reach the west and east ghosts);
 *   sy : n + 1 rows of n y-links, sy[i + n j] joins (i, j-1) and (i, j), j = 0..n;
 *        both host or device, read during the call.
 *   tol : 0 for the dense T; > 0 for the root in HBS form at that tolerance (as in
 *        gm_build; not with body loads: GM_EUNSUPPORTED).
 *   body, nbody : optional body loads (nbody = 0: none) as in gm_build_loads; the handle
 *        then also serves gm_solve_loads and gm_get_load_operator.
 * FP64 only (GM_EUNSUPPORTED for mixed precision, and for keep_levels or tol > 0 with
 * body loads); with keep_levels, gm_get_schur returns every box's Schur complement.
 */
int gm_build_net(const gm_opts *opts, const double *sx, const double *sy, int n, int leaf, double tol,
                 const int *body, int nbody, gm_handle **out);

int gm_info(gm_handle *h, gm_info_t *info);

/*
 * Serving (the solve stage under load; the paper has no serving layer).  A server owns
 * the operators added to it and keeps them resident within a device-memory budget.
 * Two worker threads: the solve worker, on a stream of the highest priority, takes every
 * pending solve request whose operator exists, groups the requests by operator and
 * applies them all in one gm_solve_many call (one launch per precision class over the
 * vectors of every operator taken: continuous batching across operators); the build
 * worker runs build requests one at a time on a stream of the lowest priority, so that
 * builds and solves overlap on the device.
 *   gm_server_create : budget_bytes for the resident operators (gm_info.resident_bytes);
 *                      batching = 0 serves every request by its own solve (the unbatched
 *                      baseline).  Uses the current device.
 *   gm_server_add    : takes ownership of h (freed on eviction or destroy) and returns
 *                      its id.  Least recently used operators not being served are
 *                      evicted to make room; GM_ENOMEM if it cannot fit.  On any error
 *                      the caller keeps h.
 *   gm_server_submit : queue dudn = T g for `batch` vectors (4n x batch column-major,
 *                      host or device); returns at once.  g and dudn must stay valid
 *                      until the request completes.  GM_EINVAL for an unknown operator.
 *   gm_server_submit_build : queue a build of the operator for b, c, d (arguments as
 *                      gm_build_ex; opts->stream and opts->background are set by the
 *                      server); returns at once with the request id and the id the
 *                      operator will have, for which solves may be submitted right away
 *                      (they wait in the queue until it is admitted).  The worker admits
 *                      the built operator like gm_server_add; the request's result is the
 *                      build's code, or GM_ENOMEM if it cannot fit (a solve queued for a
 *                      failed build then returns GM_EINVAL).  b, c, d must stay valid
 *                      until the request completes.
 *   gm_server_poll   : without blocking: *done = 1 and the request's result code once it
 *                      has completed, else *done = 0 and GM_OK; GM_EINVAL for an unknown id.
 *   gm_server_set_callback : cb(req_id, result code, user) is called on a worker thread
 *                      for every request that completes from then on (NULL: none), after
 *                      its result is visible to wait and poll, outside the server's lock
 *                      (cb may call the server); it should return quickly.  Returns after
 *                      any callback already running with the previous function has ended
 *                      (so `user` of that function may be released), except when called
 *                      from a callback.
 *   gm_server_wait   : block until request req_id has completed; returns its result code
 *                      (GM_EINVAL if its operator was evicted before it ran).
 *   gm_server_sync   : block until nothing is queued or running and no callback is
 *                      running (a callback calling it waits for everything but itself).
 *   gm_server_stats  : latency from submission to completion (p50/p99), vectors per
 *                      second from the first submission to the last completion, and the
 *                      number of (grouped) solve calls.
 * Thread-safe: any thread may submit, add, wait or read statistics.
 */
typedef struct gm_server gm_server;
typedef struct gm_server_stats_t {
    long long requests, vectors, solves, evictions;
    int resident_ops, pad;
    long long resident_bytes;
    double p50_ms, p99_ms, vectors_per_s;
} gm_server_stats_t;
int gm_server_create(long long budget_bytes, int batching, gm_server **out);
int gm_server_add(gm_server *s, gm_handle *h, int *op_id);
int gm_server_submit(gm_server *s, int op_id, const double *g, double *dudn, int batch, long long *req_id);
int gm_server_submit_build(gm_server *s, const gm_opts *opts, const double *b, const double *c, const double *d,
                           int n, int leaf, double tol, int *op_id, long long *req_id);
int gm_server_poll(gm_server *s, long long req_id, int *done);
typedef void (*gm_server_callback)(long long req_id, int result, void *user);
int gm_server_set_callback(gm_server *s, gm_server_callback cb, void *user);
int gm_server_wait(gm_server *s, long long req_id);
int gm_server_sync(gm_server *s);
int gm_server_stats(gm_server *s, gm_server_stats_t *st);
int gm_server_reset_stats(gm_server *s);
void gm_server_destroy(gm_server *s);

/* Failure injection for tests of the error paths (the paper has no counterpart): the
 * n-th device allocation the library makes from now on (n >= 1; any thread, any call)
 * fails as if the device were out of memory, so the call making it returns GM_ENOMEM
 * and releases what it holds.  n = 0 turns the injection off. */
void gm_debug_fail_alloc(long long n);

/* Release the handle and its device memory.  NULL is a no-op. */
void gm_free(gm_handle *h);

const char *gm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GM_H */
