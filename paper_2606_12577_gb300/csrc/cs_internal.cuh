// Internal declarations of the cascading-smoother multigrid library.
// Device data layout (HBM):
//   * every level stores its operator as structure-of-arrays stencil
//     coefficients A[s*N + i] (no index arrays: columns are implicit in the
//     structured grid); the canonical stencil of a level is either STAR
//     (2*dim+1 entries: C,-x,+x,-y,+y[,-z,+z]) or BOX (3^dim entries,
//     s = (dx+1) + 3(dy+1) + 9(dz+1));
//   * Lambda of a point-block cascade is one FP64 value per node per step,
//     lam[l*N + i]; FP32 copies sit beside it for low-precision cycles;
//   * vectors are contiguous N-arrays in natural (x fastest) order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cascade_mg.h"

namespace csx {

enum StencilKind { STAR = 0, BOX = 1 };

struct Grid {
    int dim;
    int nx, ny, nz;
    int64_t N;
};

struct Level {
    Grid g;
    int kind = STAR;
    int nst = 0;
    int off[27][3];
    double *A = nullptr;  // [nst][N]
    // work vectors (FP64): b (rhs), x (iterate), t (ping-pong)
    double *b = nullptr, *x = nullptr, *t = nullptr;
    // every row at boundary distance >= margin has a coefficient row equal
    // (bitwise) to the grid-centre row; NO_MARGIN: no such region is used
    int margin = NO_MARGIN;
    static constexpr int NO_MARGIN = 1 << 30;
    // block partition: blocks of bs^dim nodes (partial at the upper edges),
    // block (bx,by,bz) = nodes bs*b .. bs*b+bs-1 per axis; nmax = bs^dim.
    // Lambda of a block level is stored [nu][nblocks][nmax][nmax] over the
    // local positions lp = lx + bs (ly + bs lz); absent positions are zero.
    int bs = 1, nbx = 0, nby = 0, nbz = 0, nmax = 1;
    int64_t nblocks = 0;
    // a 3D 27-point point-block level whose operator is symmetric (to 1e-12
    // of the diagonals): its FP32 copies keep the centre and the 13 forward
    // couplings only, [14][N] (entry k = 27-point entry 13 + k); a backward
    // coupling is the forward one stored at the neighbour
    int sym32 = 0;
};

// entries per node of a level's FP32 operator copy
inline int64_t lo_nst(const Level &L) { return L.sym32 ? 14 : L.nst; }

struct LowLevel {   // FP32 state of one level (owned by a cascade)
    float *A = nullptr;    // [nst][N]
    float *lam = nullptr;  // [nu][N]
    float *b = nullptr, *x = nullptr, *t = nullptr;
};

struct LowLevel16 {  // BF16 storage of one level (FP32 arithmetic; owned by a cascade)
    __nv_bfloat16 *A = nullptr;    // [nst][N]
    __nv_bfloat16 *lam = nullptr;  // [nu][N]
    __nv_bfloat16 *b = nullptr, *x = nullptr, *t = nullptr;
};

}  // namespace csx

struct cs_hierarchy {
    int dim = 0;
    int nlev = 0;
    bool periodic = false;
    std::vector<csx::Level> lev;
    int cn = 0;                 // coarsest size
    double *cinv = nullptr;     // dense inverse of the coarsest operator, row-major
    double *fine_r = nullptr;   // FP64 residual scratch, finest level
    double *red = nullptr;      // reduction partials
    double *red_host = nullptr; // pinned host mirror of the reduction result
    double *hb = nullptr, *hx = nullptr; // device copies for host-buffer solves
    int64_t bytes = 0;
};

struct cs_cascade {
    cs_hierarchy *h = nullptr;
    int kind = CS_ADDITIVE;
    int nu = 1;
    int ncol = 1;
    int nlev = 0;               // smoothing levels
    bool lowp = false;
    std::vector<double *> lam;  // per level [nu][N]
    std::vector<csx::LowLevel> lo;
    std::vector<csx::LowLevel16> lo16;  // BF16 copies (lowp = 2, point-block hierarchies)
    float *fine_b32 = nullptr, *fine_x32 = nullptr;
    // captured zero-initial-guess V-cycles, keyed by (precision, order, mu)
    struct Graph {
        int prec, order, mu_pre, mu_post;
        cudaGraphExec_t exec;
        int64_t kernels;
    };
    std::vector<Graph> graphs;
    cudaStream_t capture_stream = nullptr;
    // GMRES workspace (lazily allocated at first GMRES solve)
    int gm_restart = 0;
    double *gm_V = nullptr, *gm_h = nullptr;
    double *gm_Z = nullptr;  // right-preconditioned GMRES: Z_j = M V_j
    int64_t bytes = 0;
    // learned setup of the finest level: 1 used (some blocks predicted), 0
    // fell back to the exact setup, -1 no model; level-1 Frobenius objectives
    // of the prediction and of the Lambda in use, over the exact one; block counts
    int learned_used = -1;
    double learned_ratio = 0.0, learned_ratio_used = 0.0;
    int64_t learned_blocks = 0, learned_full = 0, learned_accepted = 0;
};

namespace csx {

// error handling ----------------------------------------------------------
void set_error(const char *fmt, ...);
cs_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define CSX_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return csx::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)
// for functions that release their scratch at a `done:` label and return rc
#define CSX_CUDA_GOTO(call)                                             \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) { rc = csx::cuda_fail(_e, #call, __FILE__, __LINE__); goto done; } \
    } while (0)
#define CSX_TRY(...)                                                    \
    do {                                                                \
        cs_status _s = (__VA_ARGS__);                                   \
        if (_s != CS_OK) return _s;                                     \
    } while (0)

extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Device memory comes from a library-owned stream-ordered pool per device
// (cudaMallocFromPoolAsync / cudaFreeAsync) that keeps freed memory mapped,
// so repeated setups of multi-GB residual buffers cost no driver calls.
cs_status dalloc(void **p, size_t bytes, int64_t *acct, cudaStream_t s = 0);
void dfree(void *p, cudaStream_t s = 0);
template <typename T>
cs_status dalloc_t(T **p, size_t count, int64_t *acct, cudaStream_t s = 0) {
    return dalloc(reinterpret_cast<void **>(p), count * sizeof(T), acct, s);
}

inline Grid make_grid(int dim, int nx, int ny, int nz) {
    Grid g;
    g.dim = dim; g.nx = nx; g.ny = ny; g.nz = dim == 3 ? nz : 1;
    g.N = (int64_t)g.nx * g.ny * g.nz;
    return g;
}

// launch geometry: one thread per node, x fastest
constexpr int TBX = 64, TBY = 4;
inline dim3 node_grid(const Grid &g) {
    return dim3((unsigned)((g.nx + TBX - 1) / TBX), (unsigned)((g.ny + TBY - 1) / TBY), (unsigned)g.nz);
}
inline dim3 node_block() { return dim3(TBX, TBY, 1); }

// ---- stencil kernels (cs_stencil.cu)
// out = x - lam_l (A x - b) over all nodes (additive step), or over colour
// `colour` only (multiplicative step; other nodes copied when out != x).
template <typename T>
cs_status launch_sweep(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out,
                       int colour, bool x_is_zero, cudaStream_t s);
// rc = R (A x - b) (full weighting, 2^-dim P^T); with a fine-level scratch
// vector (FP32 / FP64) in two passes, else in one
template <typename T>
cs_status launch_residual_restrict(const Level &f, const Level &c, const T *A, const T *b, const T *x,
                                   T *rc, T *scratch, cudaStream_t s);
template <typename T>
cs_status launch_prolong_correct(const Level &f, const Level &c, const T *xc, const T *x, T *xo,
                                 cudaStream_t s);
// r = b - A x (FP64) with FP64 or FP32-stored coefficients; optional FP32
// copy of r and per-block partial sums of r^2 into red (nblocks entries;
// norm32: the block sums in FP32, enough for a convergence test).
cs_status launch_residual64(const Level &L, const double *A, const double *b, const double *x,
                            double *r, float *r32, double *red, int nred, cudaStream_t s, bool norm32 = false);
cs_status launch_coarse_solve(const cs_hierarchy *h, const double *b, double *x, cudaStream_t s);
cs_status launch_coarse_solve32(const cs_hierarchy *h, const float *b, float *x, cudaStream_t s);
cs_status launch_axpy_f32(int64_t N, const float *d, double *x, cudaStream_t s);  // x += d
cs_status launch_copy_d2f(int64_t N, const double *a, float *o, cudaStream_t s);
cs_status launch_copy_d2bf(int64_t N, const double *a, __nv_bfloat16 *o, cudaStream_t s);
cs_status launch_axpy_bf16(int64_t N, const __nv_bfloat16 *d, double *x, cudaStream_t s);  // x += d
cs_status launch_residual64_bf16(const Level &L, const double *A, const double *b, const double *x,
                                 __nv_bfloat16 *r16, cudaStream_t s);
cs_status launch_coarse_solve16(const cs_hierarchy *h, const __nv_bfloat16 *b, __nv_bfloat16 *x, cudaStream_t s);
// sum of red[0..nred) into red[nred] (one block, fixed order)
cs_status launch_finish_sum(double *red, int nred, cudaStream_t s);
cs_status launch_dot(int64_t N, const double *a, const double *b, double *red, int nred, cudaStream_t s);
cs_status launch_axpy_dev(int64_t N, const double *alpha, double sign, const double *x, double *y,
                          cudaStream_t s);  // y += sign * (*alpha) * x
cs_status launch_scale_dev(int64_t N, const double *num, double *y, const double *x, cudaStream_t s); // y = x / *num
cs_status launch_matvec64(const Level &L, const double *A, const double *x, double *y, cudaStream_t s);
cs_status launch_add64(int64_t N, const double *d, double *x, cudaStream_t s);  // x += d
cs_status launch_axpy_multi(int64_t N, int m, const double *alpha, const double *V, double *y, cudaStream_t s);
constexpr int NRED = 1024;  // partial sums of a reduction

// ---- setup kernels (cs_setup.cu)
cs_status galerkin_level(const Level &f, Level &c, bool reuse, cudaStream_t s);
cs_status level_margin(Level &L, bool periodic, cudaStream_t s);
// zeroes the coefficients of couplings to nodes outside a Dirichlet grid
cs_status drop_outside_couplings(const Level &L, cudaStream_t s);
// sets L.sym32 (3D 27-point point-block levels; synchronises the stream)
cs_status check_symmetric(Level &L, cudaStream_t s);
// the FP32 copy of a sym32 level's operator ([14][N])
cs_status launch_copy_box_sym32(const Level &L, float *o, cudaStream_t s);
cs_status coarse_factor(cs_hierarchy *h, cudaStream_t s);
// fp32: form the residual rows R and the error propagator E in FP32 (the
// row products summed in FP64 over chunks of 8); lambda is stored in FP64
cs_status cascade_setup_level(const cs_hierarchy *h, int l, int kind, int nu, int prescale, bool reuse, int alpha,
                              bool fp32, double *lam, cudaStream_t s, int64_t *peak_bytes);
cs_status cascade_setup_level_sketch(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int s,
                                     uint64_t seed, int exact_first, bool fp32, double *lam, cudaStream_t st);
cs_status cascade_setup_level_blocks(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int alpha, bool fp32, double *lam,
                                     cudaStream_t s);
cs_status learned_setup_level0(const cs_hierarchy *h, cs_cascade *c, cs_mlp *M, double tol, double *lam,
                               const double *lam_exact1, cudaStream_t s);
// block cascade step (bs > 1): out_b = x_b - Lambda_b^(T) (A x - b)_b over all
// blocks or the blocks of one colour
template <typename T>
cs_status launch_block_sweep(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out, int colour,
                             bool transpose, bool x_is_zero, cudaStream_t s);
template <>
cs_status launch_block_sweep<__nv_bfloat16>(const Level &, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                            const __nv_bfloat16 *, const __nv_bfloat16 *, __nv_bfloat16 *, int, bool,
                                            bool, cudaStream_t);
// the same with m right-hand sides, vectors RHS-contiguous (X[i*m + r], m <= 32)
template <typename T>
cs_status launch_block_sweep_m(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out, int m,
                               int colour, bool transpose, cudaStream_t s);

}  // namespace csx
