/*
 * cascade_mg.h -- C ABI of the GB300 (sm_103a) cascading-smoother multigrid
 * library.
 *
 * The library solves A x = b for an operator given on a structured 2D/3D
 * grid of interior nodes (homogeneous Dirichlet boundary nodes eliminated),
 * with a geometric V-cycle (Algorithm 1) whose smoother is a cascading
 * smoother (Sec. 2): an ordered sequence of block-diagonal steps
 *     x_l = x_{l-1} - Lambda_l (A x_{l-1} - b),   l = 1..nu      (eq. fwda)
 * (multiplicative form: one step per colour, eq. fwdm), each Lambda_l the
 * block-diagonal minimiser of || (I - Lambda A) E_{l-1} ||_F (Sec. 2.1-2.2,
 * Algorithm 2), built on the prescaled operator W A W, W = diag(A_ii^-1/2)
 * (Sec. 2.3.1).
 *
 * Conventions for every entry point:
 *   - Return value: CS_OK (0) or a negative cs_status; on error
 *     cs_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread).  No C++ exception crosses this boundary.
 *   - Vectors are FP64, one value per interior node, node (ix,iy,iz) at index
 *     ix + nx*(iy + ny*iz) (x fastest).  Unless a call says otherwise they
 *     are DEVICE pointers owned by the caller.
 *   - Handles own all their device memory (allocated at setup); the cycle and
 *     solve calls allocate nothing.  A handle may be used by one host thread
 *     at a time.  A cascade refers to its hierarchy, which must outlive it.
 *   - Calls are asynchronous on the given stream (a cudaStream_t; NULL = the
 *     legacy default stream), except where a call returns host data (exports,
 *     cs_solve's info): those synchronise the stream before returning.
 */
#ifndef CASCADE_MG_H
#define CASCADE_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cs_status;
enum {
    CS_OK = 0,
    CS_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, non-positive diagonal) */
    CS_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    CS_ERR_NOMEM = -3,       /* device allocation failed */
    CS_ERR_SINGULAR = -4,    /* the coarsest-level matrix could not be factorised */
    CS_ERR_DIVERGED = -5,    /* residual became non-finite or grew > 1e3 x its start */
    CS_ERR_TIMEOUT = -6,     /* a bounded device-side wait expired */
    CS_ERR_UNSUPPORTED = -7, /* option not implemented for this operator */
    CS_ERR_NOTCONV = -8      /* maxit reached before the tolerance */
};

typedef void *cs_stream; /* cudaStream_t */
typedef struct cs_hierarchy cs_hierarchy;
typedef struct cs_cascade cs_cascade;
typedef struct cs_mlp cs_mlp;

/* ------------------------------------------------------------- operator */
/* A structured-grid operator in stencil form (Sec. 2: the block-partitioned
 * A x = b; Sec. 3.3.1: FD Poisson).  coeff[s*N + i] couples unknown i to the
 * node at i + off[s]; where that node lies outside the grid (a homogeneous
 * Dirichlet node) the coefficient multiplies a zero value and is ignored:
 * cs_setup_hierarchy stores it as zero.  Offsets are in {-1,0,1}^dim and (0,0,0) must be
 * present.  With periodic != 0 neighbours wrap around (accepted by
 * cs_setup_hierarchy only with max_levels == 1: used to check the setup
 * against the constant-coefficient coefficients of Table 1). */
typedef struct {
    int dim;           /* 2 or 3 */
    int n[3];          /* interior nodes per side; n[2] = 1 when dim == 2 */
    int nst;           /* stencil entries, 1..27 */
    int off[27][3];    /* (dx, dy, dz) of entry s */
    const double *coeff; /* [nst][N], N = n[0]*n[1]*n[2]; device, or host if coeff_on_host */
    int coeff_on_host; /* 1: coeff is a host pointer (copied during setup) */
    int periodic;
} cs_stencil;

/* ------------------------------------------------------------ hierarchy */
typedef struct {
    int coarse_max; /* stop coarsening when every side is <= coarse_max (default 4) */
    int max_levels; /* 0 = no limit */
    int block;      /* block edge in nodes: 1 = point blocks; 2 or 3 (2D), 2 (3D) = blocks of
                       block^dim nodes, partial at the upper edges (default 1) */
    int no_reuse;   /* 0 (default): coarse rows whose fine neighbourhood repeats the
                       grid-centre row's are computed once and copied (exact: bitwise the
                       same as computing each); 1: compute every row */
} cs_hierarchy_opts;

/* Geometric hierarchy (Sec. 2.4): coarse interior nodes are the fine nodes
 * with even 1-based index on every axis (so n -> floor(n/2)); interpolation
 * P is bilinear/trilinear on that node set and the coarse operator is the
 * Galerkin product A_2h = R A_h P with R = 2^-dim P^T (SM Sec. 4.1), a
 * 9-point (2D) / 27-point (3D) stencil.  The coarsest operator, when it has
 * at most 1024 unknowns, is factorised densely in FP64 for the bottom-level
 * direct solve (Algorithm 1); a larger coarsest level (max_levels cutting
 * the hierarchy short) is kept for cascade setups, and cycles on it return
 * CS_ERR_UNSUPPORTED.
 * A0: the finest operator (its coefficients are copied).  opts may be NULL
 * (defaults).  On success *out receives a handle that cs_destroy_hierarchy
 * frees.  Errors: CS_ERR_ARG (bad stencil), CS_ERR_NOMEM, CS_ERR_SINGULAR,
 * CS_ERR_CUDA, CS_ERR_UNSUPPORTED (block > 1). */
cs_status cs_setup_hierarchy(const cs_stencil *A0, const cs_hierarchy_opts *opts, cs_stream stream,
                             cs_hierarchy **out);

/* -------------------------------------------------------------- cascade */
enum { CS_ADDITIVE = 0, CS_MULTIPLICATIVE = 1 };
enum { CS_FP64 = 0, CS_FP32 = 1, CS_BF16 = 2 };

typedef struct {
    int kind;      /* CS_ADDITIVE (Sec. 2.1) or CS_MULTIPLICATIVE (Sec. 2.2, red-black) */
    int nu;        /* depth, 1..8 */
    int prescale;  /* 1: elliptic prescaling W = diag(A_ii^-1/2) (Sec. 2.3.1); 0: none */
    int alpha;     /* residual truncation (Algorithm 2): after each row update keep the alpha columns
                      of largest magnitude (ties: smaller column index), on block levels the alpha
                      column blocks of largest Frobenius norm over the block's rows (ties: smaller
                      block index); 0 = none.  Block levels take alpha <= 64 (or alpha at least the
                      column blocks in reach, which truncates nothing), else CS_ERR_UNSUPPORTED;
                      CS_ERR_UNSUPPORTED with a model */
    int lowp;      /* 1: also keep FP32 copies of the level operators and Lambda for
                      CS_FP32 cycles (iterative refinement); 2: FP32 and BF16 copies, the
                      latter for CS_BF16 cycles (BF16 storage, FP32 arithmetic; point-block
                      hierarchies only, else CS_ERR_UNSUPPORTED) */
    int no_reuse;  /* 0 (default): on structured levels with a region of identical
                      coefficient rows, rows whose whole setup dependency lies in that
                      region are computed once per colour and copied -- the stencil
                      repetition the paper's concluding remarks suggest caching; exact
                      (bitwise the same as computing each row); 1: compute every row */
    const cs_mlp *model; /* optional learned setup of the finest level (2D, blocks, additive):
                      Lambda of every block predicted from its operator window (see the
                      learned-setup section below); NULL: exact setup */
    double model_tol;    /* per block: keep the prediction of a full block when its level-1
                      Frobenius objective is <= (1 + model_tol) x that of the exact level-1
                      block (default 0.05); rejected and partial edge blocks take the exact
                      level-1 block at every cascade step; if no block is kept the exact
                      setup of the level runs (fallback) */
    int setup_precision; /* CS_FP64 (default): the Frobenius-norm setup of Algorithm 2 in FP64;
                      CS_FP32: the residual rows R = A E and the propagator rows E in FP32,
                      their inner products summed in FP64 over chunks of 8 terms and each
                      row's lambda = <E_i, R_i> / <R_i, R_i> divided in FP64 (Lambda agrees
                      with the FP64 setup to about 1e-5 relative; meant for FP32 cycles).
                      Block levels form their R and E rows the same way, their Gram and cross
                      products in FP32 over chunks of 8 and in FP64 across them, and solve the
                      block least squares in FP64 with the minimum-norm cutoff at 1e-5 tr(G), the
                      resolution of FP32 products (exactly singular Gram matrices occur from the
                      second step on 9-point levels).  CS_ERR_UNSUPPORTED with a model or with
                      alpha (the ranking of truncation would flip near ties).  With
                      sketch > 0: the sketch vectors Y and Z = A~ Y in FP32, the inner
                      products and lambda in FP64 */
    int sketch;          /* 0 (default): the exact setup.  s in 1..128: the sketched setup of the
                      concluding remarks (Sec. 4): step l minimises ||(I - Lambda A) E_{l-1} S||_F
                      for an N x s Rademacher sketch S of every level, carrying Y = E S
                      (Y_0 = S; per node lam~ = <Y_i, Z_i> / <Z_i, Z_i>, Z = A~ Y, then
                      Y_i -= lam~ Z_i; multiplicative colour by colour).  No residual
                      fill-in: two N x s arrays per level whatever the depth.  Point-block
                      hierarchies without alpha or model, else CS_ERR_UNSUPPORTED.  s = 1
                      is degenerate beyond step 1 (it leaves Y = 0 in exact arithmetic) */
    int sketch_exact_first; /* 1: the first step (multiplicative: its first colour, whose
                      residual is E_0 = I) solves the unsketched problem, then sketches */
    uint64_t sketch_seed;   /* S(i, t) of level l = sign of SplitMix64 (Steele, Lea and Flood
                      2014) output mix(seed + (c + 1) 0x9E3779B97F4A7C15), c = l 2^48 + i s + t:
                      +1 when its top bit is 0, else -1 */
} cs_cascade_opts;

/* Build the cascade (Lambda_l, l = 1..nu; multiplicative: Lambda_{l,k},
 * k = red, black) on every level that has a smoother (all but the
 * coarsest), by the per-block least-squares problems of Algorithm 2 / the
 * SM algorithm in FP64 on the device.  Red = nodes with an even 1-based
 * index sum.  Multiplicative steps read the residual E_{l,k-1} of the
 * previous colour (snapshot semantics, exact also where red-black is not a
 * graph colouring, e.g. on 27-point Galerkin levels).
 * Errors: CS_ERR_ARG (nu out of range, non-positive diagonal under
 * prescaling), CS_ERR_NOMEM, CS_ERR_UNSUPPORTED (alpha > 0, periodic wrap
 * that aliases the fill-in: side <= 2 * fill radius), CS_ERR_CUDA. */
cs_status cs_setup_cascade(cs_hierarchy *h, const cs_cascade_opts *opts, cs_stream stream,
                           cs_cascade **out);

/* --------------------------------------------------------------- cycles */
enum { CS_FF = 0, CS_RF = 1 };

typedef struct {
    int mu_pre;    /* applications of the cascade before the coarse correction */
    int mu_post;   /* ... and after */
    int order;     /* CS_RF: reverse pre-smoother, forward post (symmetric V, SM Sec. 3);
                      CS_FF: forward both (Sec. 2.4) */
    int precision; /* CS_FP64, CS_FP32 (needs lowp >= 1) or CS_BF16 (BF16 storage, FP32 arithmetic;
                      needs lowp = 2); the coarsest solve stays FP64 */
} cs_vcycle_opts;

/* One V-cycle (Algorithm 1) on the finest level: x <- V(x, b), i.e.
 * x + V0 (b - A x) with V0 the zero-initial-guess cycle.  b, x: device,
 * N doubles each; x is read and overwritten. */
cs_status cs_vcycle(const cs_hierarchy *h, cs_cascade *c, const cs_vcycle_opts *opts, const double *b,
                    double *x, cs_stream stream);

/* ---------------------------------------------------------- level steps */
/* One application of the depth-nu cascade on `level` (forward: eq. fwda /
 * fwdm; reverse != 0: the reverse application eq. fwdar / fwdmr, read as
 * Lambda_{nu-l+1}^T with the colour order reversed).  b, x: device vectors
 * of that level (N_level doubles); x is updated in place. */
cs_status cs_smooth(const cs_hierarchy *h, cs_cascade *c, int level, int reverse, const double *b,
                    double *x, cs_stream stream);

/* One cascade step on `level` (a single kernel launch):
 *     out = x - Lambda_{step+1[, colour]} (A x - b)
 * over every node (colour = -1, additive step of eq. fwda) or over the nodes
 * of one colour (colour = 0 red / 1 black, eq. fwdm; other nodes are copied
 * to out unless out == x).  precision CS_FP64: b, x, out are double
 * vectors; CS_FP32: float vectors (needs lowp).  out == x is allowed only
 * for a colour step on a 5/7-point level (red-black is then a graph
 * colouring); otherwise out must not alias x. */
cs_status cs_sweep(const cs_hierarchy *h, cs_cascade *c, int level, int step, int colour, int precision,
                   const void *b, const void *x, void *out, cs_stream stream);

/* One cascade step with nrhs right-hand sides (1..32), vectors stored
 * RHS-contiguous (value r of node i at [i*nrhs + r]):
 *     X_out = X - Lambda_{step+1[, colour]}^(T) (A X - B),  block by block,
 * the multi-RHS block product X_b -= Lambda_b R_b of n_b x nrhs tiles;
 * transpose != 0 applies Lambda^T (the reverse application).  precision
 * CS_FP64: double vectors; CS_FP32: float vectors (needs lowp).  Aliasing
 * rules as for cs_sweep. */
cs_status cs_sweep_rhs(const cs_hierarchy *h, cs_cascade *c, int level, int step, int colour, int transpose,
                       int precision, int nrhs, const void *b, const void *x, void *out, cs_stream stream);

/* rc = R (A x - b) on `level` (Algorithm 1's restricted residual; R =
 * 2^-dim P^T).  rc has N_{level+1} doubles. */
cs_status cs_residual_restrict(const cs_hierarchy *h, int level, const double *b, const double *x,
                               double *rc, cs_stream stream);

/* x <- x - P xc on `level` (Algorithm 1's interpolate-and-correct). */
cs_status cs_prolong_correct(const cs_hierarchy *h, int level, const double *xc, double *x,
                             cs_stream stream);

/* The transfers of a low-precision V-cycle (Algorithm 1's restricted
 * residual and interpolate-and-correct, R = 2^-dim P^T), run by the same
 * kernels the cycle launches: precision CS_FP32 takes float vectors and the
 * cascade's FP32 operator copy (needs lowp >= 1); CS_BF16 takes bfloat16
 * vectors and the BF16 operator copy (needs lowp = 2).  FP64 transfers are
 * cs_residual_restrict / cs_prolong_correct.
 *   b, x: device vectors of `level` (N_level values); rc: N_{level+1};
 *   xc: N_{level+1}; x is updated in place by the prolongation.
 * The FP32 restriction forms the fine residual in the cascade's own FP32
 * scratch vector of that level, so calls on one cascade must not overlap
 * on the GPU.  Errors: CS_ERR_ARG (null pointer, bad level, precision or
 * missing lowp copies). */
cs_status cs_residual_restrict_lowp(const cs_hierarchy *h, cs_cascade *c, int level, int precision,
                                    const void *b, const void *x, void *rc, cs_stream stream);
cs_status cs_prolong_correct_lowp(const cs_hierarchy *h, cs_cascade *c, int level, int precision,
                                  const void *xc, void *x, cs_stream stream);

/* x = A_c^-1 b on the coarsest level (bottom-level direct solve, FP64:
 * Cholesky when A_c is symmetric to 1e-14 of its largest entry, else LU
 * with partial pivoting; applied as the precomputed dense inverse). */
cs_status cs_coarse_solve(const cs_hierarchy *h, const double *b, double *x, cs_stream stream);

/* r = b - A x on `level`; if norm2 != NULL, *norm2 (HOST) receives ||r||_2
 * (the call then synchronises). */
cs_status cs_residual(const cs_hierarchy *h, int level, const double *b, const double *x, double *r,
                      double *norm2, cs_stream stream);

/* Allocation-free variant of cs_smooth (the paper has no counterpart: this is
 * an interface convenience, not a step of the method).
 *
 * For callers that cannot allocate device memory: code that runs inside a
 * host application or framework whose allocator already owns the whole GPU,
 * callers that must not risk the implicit device synchronisation a
 * cudaMalloc/cudaFree can cause, or callers that never create the handles of
 * cs_setup_hierarchy / cs_setup_cascade (which allocate).  The caller passes
 * the operator and Lambda directly; the ping-pong vector that cs_smooth takes
 * from its hierarchy comes from a fixed 16 MiB device array inside the
 * library (2,097,152 doubles), which every GPU that loads the library keeps
 * until the process exits.  No call allocates device memory or calls an
 * allocating library routine (but see the first call on a device below).
 *
 * Computes the same thing as cs_smooth: one application of the depth-nu
 * cascade (forward, or reverse when reverse != 0), x updated in place.
 *   dim, n:  grid (n[2] ignored in 2D); N = n[0]*n[1]*n[2] must be
 *            <= 2,097,152, else CS_ERR_ARG.
 *   box:     0: coeff holds a 5/7-point stencil in the order C,-x,+x,-y,+y[,-z,+z];
 *            1: a 9/27-point stencil, entry s at offset ((s%3)-1, (s/3%3)-1, (s/9)-1)
 *            (the layouts cs_query_level / cs_export_operator report);
 *            coefficients to nodes outside the grid are ignored.
 *   coeff:   device [nst][N];  lam: device [nu][N] (point-block Lambda_l, the
 *            multiplicative Lambda_{l,k} on the nodes of colour k, as
 *            cs_export_lambda returns);  b, x: device [N].
 *   kind:    CS_ADDITIVE or CS_MULTIPLICATIVE (red-black).
 * The first call on a device looks up the device address of the internal
 * array (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Under lazy module loading (the CUDA
 * default) that first call, or the first kernel launch, also loads the
 * library's device code on the device, which creates the array and the code
 * there and may synchronise: make one warm-up call per device outside any
 * capture and outside latency-critical regions.  coeff, lam, b and x must be
 * device memory of the current device (else CS_ERR_ARG), and the grid must
 * fit the node kernels' launch (ny <= 262,140, nz <= 65,535; else
 * CS_ERR_ARG).  All calls share the one array and leave
 * their last intermediate vector in it; every step overwrites all N entries
 * it later reads, so nothing needs clearing between calls.  Calls that
 * overlap on the GPU (other streams, other host threads) race on the array:
 * order them on one stream. */
cs_status cs_smooth_noalloc(int dim, const int *n, int box, const double *coeff, const double *lam, int nu,
                            int kind, int reverse, const double *b, double *x, cs_stream stream);

/* ---------------------------------------------------------------- solve */
enum { CS_STATIONARY = 0, CS_GMRES = 1, CS_REFINE = 2, CS_GMRES_RIGHT = 3, CS_PCG = 4 };

typedef struct {
    int method;      /* CS_STATIONARY: x <- V(x,b); CS_GMRES: left-preconditioned
                        restarted GMRES with V0 (Sec. 3.1); CS_REFINE: FP64 iterative
                        refinement x += V0(b - A x) with the cycle in cycle.precision;
                        CS_GMRES_RIGHT: restarted GMRES with V0 applied on the right,
                        in flexible form (Z_j = V0 v_j kept, x += Z y): it minimises the
                        true residual ||b - A x||, so it also stops on it where the
                        left form's preconditioned residual ||V0 r|| no longer bounds
                        ||r|| (high-contrast coefficients); one more N-vector per step;
                        CS_PCG: preconditioned conjugate gradients (general path only) */
    int restart;     /* GMRES restart length (default 30) */
    int maxit;       /* maximum V-cycle applications (default 100) */
    double tol;      /* stop when ||b - A x||_2 / ||b||_2 <= tol (default 1e-10) */
    cs_vcycle_opts cycle;
    int host_buffers; /* 1: b and x are HOST pointers; copies happen inside the call */
    double *hist;    /* optional host array: relative residual per iteration (true residual
                        for stationary/refine, preconditioned estimate ||V0 r||/||V0 b|| for
                        CS_GMRES, true-residual estimate ||r||/||b|| for CS_GMRES_RIGHT) */
    int hist_cap;
} cs_solve_opts;

typedef struct {
    int iterations;        /* V-cycle applications in the iteration (GMRES: Arnoldi steps) */
    int converged;         /* 1 if the tolerance was met */
    double final_rel_residual; /* ||b - A x||_2 / ||b||_2 in FP64 */
    int nhist;             /* entries written to opts->hist */
} cs_solve_info;

/* Solve A x = b from the given initial x (0 for the paper's convention).
 * Synchronises the stream before returning (info is host data).
 * Errors: CS_ERR_NOTCONV (maxit reached; x holds the last iterate),
 * CS_ERR_DIVERGED, CS_ERR_ARG, CS_ERR_CUDA. */
cs_status cs_solve(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *opts, const double *b,
                   double *x, cs_solve_info *info, cs_stream stream);

/* ------------------------------------------------------ many problems */
/* Set up nprob independent problems: cs_setup_hierarchy then
 * cs_setup_cascade for each, run concurrently from nthreads host threads
 * (<= 0: up to 16), each on its own stream.  The batched-solve form of the
 * method (many uneven problems at once); the paper sets up one problem at a
 * time.  A[p] may hold host or device coefficients (coeff_on_host).  The
 * handles are returned in h[p], c[p]; on any failure every handle is released,
 * all entries are NULL and the first failing problem's error is reported.
 * `stream` waits for all the work. */
cs_status cs_setup_many(int nprob, const cs_stencil *A, const cs_hierarchy_opts *hopts,
                        const cs_cascade_opts *copts, int nthreads, cs_stream stream, cs_hierarchy **h,
                        cs_cascade **c);

/* Batched solve: nprob independent 2D Dirichlet problems of any sizes, each
 * with its own red-black multiplicative cascade (point blocks, the same depth
 * nu for all: additive or red-black multiplicative, eq. fwda / fwdm; point
 * or 2x2-node blocks) and 1..32 right-hand sides, iterated together by
 * FP64 refinement x += V0(b - A x) or by GMRES preconditioned with V0
 * (Algorithm 1 V-cycles in opts.precision; FP64 residuals and Krylov
 * vectors) until every problem meets its tolerance.  The whole solve
 * is ONE persistent cooperative kernel launch (grid-wide barriers between its
 * stages), replayed from a CUDA graph.  Vectors of problem p are
 * [N_p][nrhs_p], right-hand sides contiguous per node: element (i, r) at
 * i * nrhs_p + r.  The paper solves one problem at a time; this is the
 * many-problem form of the same iteration. */
typedef struct cs_batch cs_batch;
typedef struct {
    int precision;   /* CS_FP32 (FP32 cycles inside FP64 refinement) or CS_FP64 */
    int order;       /* CS_RF or CS_FF, as for cs_vcycle */
    int mu_pre, mu_post;
    int autotune;    /* 1: time each (threads, tiles_per_cta) candidate on the batch and keep the fastest */
    int threads;     /* CTA size if not autotuned (default 256; 32..512, multiple of 32) */
    int tiles_per_cta; /* if not autotuned (default 2; 1..1024): each stage's work items (grid node x
                        right-hand side) are cut into about tiles_per_cta x CTAs tiles of equal work,
                        none smaller than the CTA size */
    int method;      /* CS_REFINE: x += V0(b - A x); CS_GMRES: left-preconditioned restarted GMRES
                        with M = V0 per right-hand side (classical Gram-Schmidt, projected a
                        second time when the first removes more than half of ||Z||^2 (DGKS);
                        Givens; inner steps stop on |g_{j+1}| <= tol ||M b||, restarts check
                        the FP64 true residual).  The Krylov vectors have the cycle precision:
                        with CS_FP32 a cycle also stops at |g_{j+1}| <= 1e-5 ||M r|| and the
                        restart refines in FP64 (GMRES-based iterative refinement);
                        CS_GMRES_RIGHT: the same with M applied on the right in flexible form
                        (Z_j = M V_j kept in the cycle precision, A Z_j formed with the FP64
                        operator, x += Z y in FP64), so |g_{j+1}| estimates ||b - A x|| and the
                        inner steps stop on |g_{j+1}| <= tol ||b|| (or 1e-5 ||r|| with CS_FP32):
                        the form that converges where the coefficients' contrast makes ||M r||
                        a poor measure of ||r||; restart more vectors of [N0][m] per problem */
    int restart;     /* GMRES restart length (default 30, at most 256) */
} cs_batch_opts;
typedef struct {
    int threads;
    int tiles_per_cta;
    float ms;        /* measured time of two iterations on the batch */
} cs_batch_tune;
/* Plan a batched solve over existing handles (not owned; they must outlive
 * the plan): validates them, allocates the multi-RHS level vectors and the
 * tile tables, and autotunes if asked.  Errors: CS_ERR_ARG (null, nrhs not in
 * 1..32, FP32 without lowp cascades, mixed nu, cascade kinds or block sizes),
 * CS_ERR_UNSUPPORTED (3D, periodic, blocks other than 1 or 2x2 nodes, no
 * coarsest factorisation). */
cs_status cs_batch_create(int nprob, cs_hierarchy *const *h, cs_cascade *const *c, const int *nrhs,
                          const cs_batch_opts *opts, cs_stream stream, cs_batch **out);
/* Solve all problems from the initial x[p] (device, [N_p][nrhs_p]) to
 * ||b - A x||_2 / ||b||_2 <= tol for every right-hand side (tol <= 0: 1e-10;
 * maxit <= 0: 100).  info[p] (host, optional): V-cycles applied, converged,
 * worst relative residual over the problem's right-hand sides.  Synchronises
 * the stream.  Errors: CS_ERR_NOTCONV / CS_ERR_DIVERGED if any problem did not
 * converge (the others are still solved), CS_ERR_ARG, CS_ERR_CUDA. */
cs_status cs_batch_solve(cs_batch *b, const double *const *bvec, double *const *x, double tol, int maxit,
                         cs_solve_info *info, cs_stream stream);
/* The configuration in use, the CTAs of the cooperative launch, and the
 * autotuner's measurements (up to cap entries; *ntuned = their count). */
cs_status cs_batch_config(const cs_batch *b, int *threads, int *tiles_per_cta, int *ctas, cs_batch_tune *tuned,
                          int cap, int *ntuned);
/* Force a configuration (e.g. to compare schedules); results do not depend on it. */
cs_status cs_batch_set_config(cs_batch *b, int threads, int tiles_per_cta, cs_stream stream);
int64_t cs_batch_bytes(const cs_batch *b);
void cs_batch_destroy(cs_batch *b);
/* One-shot form: plan (no autotuning), solve, release.  opts->cycle gives the
 * precision, order and mu; opts->method (CS_GMRES, else refinement) and
 * opts->restart the iteration; opts->tol and opts->maxit the stopping rule. */
cs_status cs_solve_batched(int nprob, cs_hierarchy *const *h, cs_cascade *const *c, const cs_solve_opts *opts,
                           const double *const *b, double *const *x, const int *nrhs, cs_solve_info *info,
                           cs_stream stream);

/* ------------------------------------------------------- learned setup */
/* A small MLP (nin -> nhid -> nhid -> nout, ReLU) that maps a block's operator
 * window to its prescaled Lambda~_1..nu blocks.  This learned form is not in
 * the paper; the exact Frobenius setup (Algorithm 2) stays the reference and
 * the fallback.  Weights are FP32 masters used in BF16 for every product,
 * with FP32 accumulation; parameters are [W1 (nhid x nin), b1, W2, b2, W3
 * (nout x nhid), b3], row-major.  max_batch: rows per forward/backward pass
 * (longer forward calls are chunked).  Weights are He-uniform from seed.
 * Every product of the forward and backward passes runs on the tensor cores
 * (cs_tc_gemm_bf16's kernel): the BF16 weights enter as they are, FP32
 * activations and gradients as BF16 pairs hi = bf16(x), lo = bf16(x - hi)
 * (products of two FP32 factors as a_hi b_hi + a_lo b_hi + a_hi b_lo), so
 * results agree with FP32 products of BF16 weights to about 2^-16.  A wait
 * of the GEMM kernel that expires makes the next call that synchronises
 * return CS_ERR_TIMEOUT. */
cs_status cs_mlp_create(int nin, int nhid, int nout, int max_batch, uint64_t seed, cs_mlp **out);
/* C[M x N] (FP32, row-major, DEVICE) = A[M x K] B[N x K]^T for DEVICE BF16
 * matrices A and B, row-major with K contiguous, FP32 accumulation: the
 * tcgen05 tensor-core GEMM of the learned setup (128 x 128 tiles, TMA-staged
 * 128 x 64 operand tiles with the 128-byte swizzle, the accumulator in tensor
 * memory).  K a multiple of 8 (16-byte rows), A and B 16-byte aligned, all
 * three on the current device.  Products with at least two tiles per SM run
 * persistent (one CTA per SM, two TMEM accumulators).  Synchronises the
 * stream.  Errors: CS_ERR_ARG (shapes, alignment, memory not of the current
 * device), CS_ERR_CUDA, CS_ERR_TIMEOUT (a bounded wait of the kernel expired;
 * the context stays usable). */
cs_status cs_tc_gemm_bf16(int M, int N, int K, const void *A, const void *B, float *C, cs_stream stream);
void cs_mlp_destroy(cs_mlp *m);
int64_t cs_mlp_nparam(const cs_mlp *m);
cs_status cs_mlp_get_params(const cs_mlp *m, float *host_params);
cs_status cs_mlp_set_params(cs_mlp *m, const float *host_params);
/* Y[batch x nout] = f(X[batch x nin]); X, Y device FP32, row-major. */
cs_status cs_mlp_forward(cs_mlp *m, int batch, const float *X, float *Y, cs_stream stream);
/* Mean-squared-error loss against T[batch x nout] (device) and its gradient
 * w.r.t. every parameter (host copy if grad_host != NULL); batch <= max_batch.
 * Synchronises. */
cs_status cs_mlp_gradients(cs_mlp *m, int batch, const float *X, const float *T, float *grad_host, float *loss,
                           cs_stream stream);
/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on that loss; *loss
 * (host, optional; then the call synchronises) receives the loss before the step. */
cs_status cs_mlp_train_step(cs_mlp *m, int batch, const float *X, const float *T, float lr, float *loss,
                            cs_stream stream);
/* Features of every block of a 2D block level into F [nblocks x bs^2 (bs+2)^2]
 * (device, FP32): for each block node its row of the prescaled operator
 * W A W over the (bs+2)^2-node window around the block. */
cs_status cs_block_features(const cs_hierarchy *h, int level, float *F, cs_stream stream);
/* Training targets from an exact additive cascade: prescaled blocks
 * W^-1 Lambda_l W^-1, l = 1..nu, into T [nblocks x nu bs^4] (device, FP32). */
cs_status cs_block_targets(const cs_cascade *c, int level, float *T, cs_stream stream);
/* After cs_setup_cascade with a model: *used = 1 if predicted blocks are in
 * use, 0 if the exact setup ran instead, -1 without a model; *ratio = level-1
 * Frobenius objective of the prediction (every block) / exact. */
cs_status cs_learned_status(const cs_cascade *c, int *used, double *ratio);
/* Per-block detail of the learned setup: blocks of the finest level, full
 * blocks, blocks whose prediction is in use; level-1 Frobenius objective of
 * the prediction and of the Lambda in use (predicted or exact level-1 block),
 * each over the exact one. */
cs_status cs_learned_stats(const cs_cascade *c, int64_t *blocks, int64_t *full_blocks, int64_t *predicted_blocks,
                           double *ratio_predicted, double *ratio_used);

/* ------------------------------------------ general sparse operators */
/* The method for an arbitrary block-partitioned A x = b (Sec. 2: the user
 * chooses the blocks; Sec. 2.4: the user chooses the transfers), with
 * index-driven kernels instead of stencils.  The user gives the finest
 * operator in CSR form, one interpolation P_l (N_l x N_{l+1}) per coarser
 * level, the restriction scale (R_l = rscale P_l^T; the V-cycle does not
 * depend on it) and optionally a block partition of the finest level
 * (point blocks elsewhere).  The coarse operators are Galerkin,
 * A_{l+1} = R_l A_l P_l, formed on the device.  The multiplicative cascade
 * colours every level's block graph (blocks adjacent when A couples them in
 * either direction) greedily in decreasing order of a pseudo-random
 * priority (ties: smaller block index), computed in parallel by
 * Jones-Plassmann rounds: block b of level l has priority
 * mix(seed + (c + 1) 0x9E3779B97F4A7C15) (SplitMix64, c = l 2^40 + b); the
 * colouring is a graph colouring, so colour steps run in place.  Setup
 * (Algorithm 2 / SM Algorithm), cycles and solves are FP64. */
typedef struct {
    int n, m;                /* rows, columns */
    const int64_t *rowptr;   /* [n + 1] */
    const int32_t *col;      /* [nnz], ascending within every row */
    const double *val;       /* [nnz] */
    int on_host;             /* 1: host arrays; 0: device arrays (both are copied) */
} cs_csr;

typedef struct cs_ghier cs_ghier;
typedef struct cs_gcascade cs_gcascade;

/* nP interpolations P[0..nP-1] (P[l]: N_l x N_{l+1}).  Blocks per level:
 * nblocks[l] > 0 with HOST arrays bptr[l] [nblocks[l] + 1] and bidx[l]
 * [bptr[l][nblocks[l]]]: 1..16 distinct nodes per block in the order given,
 * every node in at least one block.  A node in several blocks makes the
 * level's blocks overlapping (Sec. 3.6.2): the additive cascade averages
 * the blocks' rows and corrections at each node over its theta_i blocks,
 * and the colouring separates blocks that share a node, so a
 * multiplicative colour step writes each node once.  nblocks[l] = 0 (or
 * nblocks NULL) for point blocks.  field (HOST, [N_0], or NULL): 0 for a velocity or scalar unknown,
 * 1 for a pressure (constraint) unknown; a coarse unknown takes the field
 * of the fine unknowns its interpolation column reaches (two fields:
 * CS_ERR_ARG).  The coarsest level (at most 1024 unknowns) is factorised
 * densely.  Errors: CS_ERR_ARG (shapes, a node in no block or twice in one, block too large,
 * more than 64 colours, fields), CS_ERR_SINGULAR, CS_ERR_NOMEM, CS_ERR_CUDA. */
cs_status cs_gsetup_hierarchy(const cs_csr *A0, int nP, const cs_csr *P, double rscale, const int *nblocks,
                              const int *const *bptr, const int *const *bidx, const int *field,
                              uint64_t colour_seed, cs_stream stream, cs_ghier **out);
/* Prescaling W of the general path (Sec. 2.3): none; elliptic,
 * W = diag(A_ii^-1/2); Stokes (SM "Prescaling Stokes problems"): a velocity
 * unknown takes w_i = sqrt(||A_{i,:}||_1) / A_ii, the 1-norm over the
 * velocity columns (so the velocity diagonal of W A W is ||A_{i,:}||_1 /
 * A_ii), and the pressure weights make every row of diag(w_p) D diag(w_u)
 * of unit q-norm, q = 1 (the paper's choice for finite differences), 2 or
 * infinity (its choice for element methods). */
enum { CS_PRESCALE_NONE = 0, CS_PRESCALE_ELLIPTIC = 1, CS_PRESCALE_STOKES_L1 = 2, CS_PRESCALE_STOKES_L2 = 3,
       CS_PRESCALE_STOKES_LINF = 4 };
/* The cascade of every smoothing level: kind CS_ADDITIVE or
 * CS_MULTIPLICATIVE (greedy colours), depth nu (1..8), prescale a
 * CS_PRESCALE_* mode (Stokes modes need the fields).  spd = 1 projects
 * every block of Lambda~, as soon as it is solved and before the next
 * step uses it, onto the symmetric matrices between 0 and the block-Jacobi
 * block (A~_bb)^{-1}, nearest in the Frobenius norm weighted by A~_bb (the
 * plain positive semidefinite projection where A~_bb is not positive
 * definite), so that the cycle can precondition CS_PCG (SM "On
 * preconditioned conjugate gradient").  The residual rows E are kept per
 * block over the union of the block rows' columns (per node when blocks
 * overlap); their patterns are built on the host, their values on the
 * device.  Errors: CS_ERR_ARG (non-positive diagonal under prescaling, bad
 * kind / nu / mode / spd), CS_ERR_NOMEM, CS_ERR_CUDA. */
cs_status cs_gsetup_cascade(cs_ghier *h, int kind, int nu, int prescale, int spd, cs_stream stream,
                            cs_gcascade **out);
/* One cascade step (a single kernel launch on point-block levels):
 * out = x - Lambda_{step+1[, colour]} (A x - b) over every block (colour
 * = -1, additive) or over the blocks of one colour (multiplicative; out may
 * equal x, and with out != x the other blocks are copied). */
cs_status cs_gsweep(const cs_ghier *h, cs_gcascade *c, int level, int step, int colour, const double *b,
                    const double *x, double *out, cs_stream stream);
/* One application of the depth-nu cascade (forward, or reverse with the
 * transposed blocks in reverse step and colour order), x in place. */
cs_status cs_gsmooth(const cs_ghier *h, cs_gcascade *c, int level, int reverse, const double *b, double *x,
                     cs_stream stream);
/* x <- V(x, b) (Algorithm 1) with the cycle options of cs_vcycle (FP64). */
cs_status cs_gvcycle(const cs_ghier *h, cs_gcascade *c, const cs_vcycle_opts *opts, const double *b, double *x,
                     cs_stream stream);
/* Solve as cs_solve; methods CS_STATIONARY, CS_GMRES_RIGHT and CS_PCG
 * (conjugate gradients preconditioned by V(0, .); the iteration stops when
 * the recurrence residual reaches tol, the history holds those residuals
 * and final_rel_residual the true one; it needs a symmetric cycle, e.g. an
 * spd cascade with mu_pre = mu_post and the RF order); FP64 cycles; b, x
 * device vectors.  Errors as cs_solve. */
cs_status cs_gsolve(const cs_ghier *h, cs_gcascade *c, const cs_solve_opts *opts, const double *b, double *x,
                    cs_solve_info *info, cs_stream stream);
/* Level sizes: rows, stored entries, blocks, colours (HOST outputs, any may be NULL). */
cs_status cs_gquery_level(const cs_ghier *h, int level, int *n, int64_t *nnz, int *nblocks, int *ncolours);
int cs_gnlevels(const cs_ghier *h);
/* HOST copies: the level's CSR operator; the colour of every block; the
 * blocks (bptr [nblocks + 1], bidx [bptr[nblocks]]; bidx NULL: bptr only); Lambda as [nu][lamsize]
 * (block b's n_b x n_b matrix row-major at its offset, blocks in order;
 * Lambda_{l,k} on the blocks of colour k). */
cs_status cs_gexport_operator(const cs_ghier *h, int level, int64_t *rowptr, int32_t *col, double *val);
cs_status cs_gexport_colours(const cs_ghier *h, int level, int32_t *colour);
cs_status cs_gexport_blocks(const cs_ghier *h, int level, int32_t *bptr, int32_t *bidx);
int64_t cs_glamsize(const cs_gcascade *c, int level);
cs_status cs_gexport_lambda(const cs_gcascade *c, int level, double *host_lambda);
void cs_gdestroy_hierarchy(cs_ghier *h);
void cs_gdestroy_cascade(cs_gcascade *c);

/* -------------------------------------------------------------- queries */
typedef struct {
    int dim;
    int n[3];
    int64_t N;
    int nst;          /* stencil entries stored for this level */
    int off[27][3];   /* their offsets */
    int nlevels;      /* levels in the hierarchy */
    int block;        /* block edge in nodes */
    int64_t lamsize;  /* doubles of Lambda per cascade step (sum of n_b^2 over blocks) */
    int sym32;        /* 1: a 3D 27-point point-block level whose operator is symmetric (to 1e-12 of
                         the diagonals); FP32 cycles store its centre and 13 forward couplings and
                         take each backward coupling from the neighbour's row */
} cs_level_info;

cs_status cs_query_level(const cs_hierarchy *h, int level, cs_level_info *info);
/* Copy the level operator to HOST memory: [nst][N] doubles, offsets as in
 * cs_query_level (zero where the neighbour lies outside the grid). */
cs_status cs_export_operator(const cs_hierarchy *h, int level, double *host_coeff);
/* Red-black colour id of every node of `level` (0 = red) into HOST memory. */
cs_status cs_export_colours(const cs_hierarchy *h, int level, int8_t *host_colour);
/* Copy Lambda of `level` to HOST memory: [nu][lamsize] doubles.  Point blocks:
 * one value per node.  Blocks: for every block (x fastest over the block
 * grid) its n_b x n_b matrix, row-major over its nodes in ascending index
 * order.  The multiplicative Lambda_{l,k} occupy the blocks of colour k
 * (red = even 1-based block index sum). */
cs_status cs_export_lambda(const cs_cascade *c, int level, double *host_lambda);
/* Number of device bytes the handle holds. */
int64_t cs_hierarchy_bytes(const cs_hierarchy *h);
int64_t cs_cascade_bytes(const cs_cascade *c);

/* Kernel launches issued by this library in this process so far (a replay
 * of a captured cycle counts each of its kernels). */
int64_t cs_kernel_launches(void);
const char *cs_last_error(void);
void cs_destroy_hierarchy(cs_hierarchy *h);
void cs_destroy_cascade(cs_cascade *c);

#ifdef __cplusplus
}
#endif
#endif /* CASCADE_MG_H */
