// Batched solve of many independent problems of uneven size, each with its
// own right-hand sides: the V-cycles (Algorithm 1) with multiplicative
// red-black cascade smoothing (eq. fwdm and its reverse), the FP64 residual
// and the update of every problem run in ONE persistent cooperative kernel
// per solve, launched from a CUDA graph.  Stages are separated by grid-wide
// barriers; the levels of all problems are aligned at the coarsest, so that
// level slot t of the batch holds level t - (D - nlev_p) of problem p
// (D = the largest level count) and every stage is one ragged sweep over the
// slot's levels.  Work is dealt out in tiles (a problem, a level, a contiguous
// range of its grid rows' nodes) of about equal work; the number of tiles per
// CTA and the CTA size are picked by a measuring autotuner.
//
// Data layout: vectors of problem p hold its m_p right-hand sides
// contiguously per node, v[i * m_p + r] (m_p <= 8); operators and Lambda are
// the problem's own level arrays (structure of arrays, FP32 or FP64).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cs_internal.cuh"

namespace cg = cooperative_groups;

namespace csx {

constexpr int BMAXLEV = 16;
constexpr int BMAXRHS = 32;
constexpr int BMAXRESTART = 256;
constexpr int RED_DOUBLES = 4 * 512;  // the kernel's shared reduction buffer

template <typename T>
struct BLevel {
    int nx, ny, kind, inplace;
    int64_t N;
    int bs, nbx, nmax;  // blocks of bs x bs nodes (1: point blocks), nbx per row, nmax = bs^2
    int64_t nblocks;
    const T *A;    // [nst][N]
    const T *lam;  // [nu][N] (points) or [nu][nblocks][nmax][nmax] (blocks)
    T *b, *x, *t;  // [N][m]
};

template <typename T>
struct BProb {
    int nlev, m, slot0, cn;
    const double *A64;   // finest operator, FP64
    const double *cinv;  // coarsest dense inverse, FP64 row-major
    T *Z;                // GMRES work vector [N0][m] (the cycle precision)
    T *V;                // GMRES basis: restart + 1 vectors of [N0][m]
    T *ZB;               // right-preconditioned GMRES: restart vectors Z_j = M V_j of [N0][m]
    BLevel<T> lev[BMAXLEV];
};

struct BTile {
    int p, l, i0, ni;
};

enum { OP_SWEEP = 0, OP_RESTRICT = 1, OP_COARSE = 2, OP_PROLONG = 3 };
// colour >= 0: a multiplicative colour step (in place on 5-point levels, else
// x -> t for parity 0 and t -> x for parity 1); colour < 0: an additive step
// from buffer src to dst (0: x, 1: t).  Restriction reads the fine level's
// buffer src; prolongation reads src and writes dst.  transpose: Lambda^T
// (the reversed smoother on block levels).
struct BStep {
    int op, slot, lv, colour, parity, src, dst, transpose;
};

struct BCtl {
    double tol;
    int maxit;
    int cnt[2];  // counts of the counting stages, alternating slots
};

enum { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_DIVERGED = 2, ST_MAXIT = 3 };

struct BArgs {
    const void *probs;
    int nprob;
    const BTile *tiles;      // tiles of slot t: [slot_tile[t], slot_tile[t + 1])
    const int *slot_tile;
    const BTile *btiles;     // block tiles (i0, ni in blocks) of slot t, for block-level sweeps
    const int *slot_btile;
    int dmax;
    const BTile *ftiles;     // finest-level tiles; problem p: [ftile_of[p], ftile_of[p + 1])
    const int *ftile_of;
    int nftiles;
    const BStep *steps;
    int nsteps;
    const double *const *b64;  // per problem, [N0][m]
    double *const *x64;
    double *part;   // [nftiles][BMAXRHS]
    double *nb;     // [nprob][BMAXRHS]
    double *rel;    // [nprob][BMAXRHS]
    double *rel0;   // [nprob]
    int *state;     // [nprob]
    int *iters;     // [nprob]
    int *work;      // [nprob]: the problem takes part in the cycle stages
    BCtl *ctl;
    // GMRES (restarted, left or right preconditioned; per problem and right-hand side q = p * BMAXRHS + r)
    int method, restart, hstride;
    double *H;      // [q][(restart + 1) * restart]
    double *cs, *sn, *y;  // [q][restart]
    double *g;      // [q][restart + 1]
    double *inv;    // [q]: 1 / ||Z|| of the last normalisation
    double *nmb;    // [q]: ||M b|| (left) or ||b|| (right): the scale of the GMRES stopping test
    int *jcols;     // [q]: Krylov columns built in this cycle
    int *frozen;    // [q]: no longer extending in this cycle
    // classical Gram-Schmidt: per-tile projection partials, problem p's
    // block at p2off[p], [tile of p][slot i < restart + 2][r < m_p]
    double *part2;
    const int64_t *p2off;
    int qtot;            // right-hand sides of all problems
    const int *qlist;    // [qtot]: q = p * BMAXRHS + r
    double *hsum;        // [q][restart + 2]: this pass's <Z, V_i> (slot j + 1: <Z, Z>)
    double *znorm2;      // [q]: ||Z||^2 after the first projection
    int *reorth;         // [q]: the step projects a second time
    double *beta;        // [q]: ||M r|| at the start of the GMRES cycle
    double itol;         // inner stop |g_{j+1}| <= itol beta (FP32 Krylov vectors), 0: none
};

__device__ __forceinline__ int bcolour(int ix, int iy) { return ((ix + 1) + (iy + 1)) & 1; }

template <int KIND>
__device__ __forceinline__ void boff(int s, int &dx, int &dy) {
    if (KIND == STAR) {
        dx = s == 1 ? -1 : s == 2 ? 1 : 0;
        dy = s == 3 ? -1 : s == 4 ? 1 : 0;
    } else {
        dx = s % 3 - 1;
        dy = s / 3 - 1;
    }
}

// (A v)_{i,r} at node i = (ix, iy), computed in T; neighbours outside
// contribute nothing
template <int KIND, typename T, typename TA, typename TV = T>
__device__ __forceinline__ T row_apply(int nx, int ny, int64_t N, const TA *__restrict__ A, const TV *v, int m, int r,
                                       int ix, int iy, int i) {
    constexpr int NST = KIND == STAR ? 5 : 9;
    T ax = T(0);
#pragma unroll
    for (int s = 0; s < NST; ++s) {
        int dx, dy;
        boff<KIND>(s, dx, dy);
        const bool in = (unsigned)(ix + dx) < (unsigned)nx && (unsigned)(iy + dy) < (unsigned)ny;
        const T a = (T)A[(int64_t)s * N + i];
        const int j = i + dx + nx * dy;
        ax = fma(a, in ? (T)v[(int64_t)j * m + r] : T(0), ax);
    }
    return ax;
}

// Work items of a tile: item (node, right-hand side r).  Thread t < U, U the
// largest multiple of m not above the CTA size, takes r = t % m for the
// nodes i0 + t / m + k U / m, so no index is divided per item and the m
// threads of a node are adjacent (its coefficient loads are one broadcast).
struct TileMap {
    int r, n0, step;
    bool on;
};
__device__ __forceinline__ TileMap tile_map(int m) {
    TileMap t;
    const int U = ((int)blockDim.x / m) * m;
    t.on = (int)threadIdx.x < U;
    t.r = (int)threadIdx.x % m;
    t.n0 = (int)threadIdx.x / m;
    t.step = U / m;
    return t;
}

// Deterministic CTA sums per right-hand side: red[t] holds thread t's sum;
// threads t and t + k m (same r) are combined by a fixed pairwise tree over
// the groups g = t / m; out[r] = the sum of right-hand side r.
__device__ __forceinline__ void cta_sum_by_rhs(double v, int m, double *red, double *out) {
    const int t = threadIdx.x;
    const int G = (int)blockDim.x / m, U = G * m;
    red[t] = t < U ? v : 0.0;
    __syncthreads();
    int P = 1;
    while (2 * P <= G) P *= 2;
    if (t < (G - P) * m) red[t] += red[t + P * m];  // fold the groups beyond the largest power of two
    __syncthreads();
    for (int h = P / 2; h > 0; h /= 2) {
        if (t < h * m) red[t] += red[t + h * m];
        __syncthreads();
    }
    if (t < m) out[t] = red[t];
    __syncthreads();
}

// The same tree for nv <= 4 sums at once (red holds 4 x blockDim.x values):
// out[u * ostride + r] = the sum of value u over right-hand side r.
__device__ __forceinline__ void cta_sum4_by_rhs(const double *v, int nv, int m, double *red, double *out,
                                                int ostride) {
    const int t = threadIdx.x, T = (int)blockDim.x;
    const int G = T / m, U = G * m;
#pragma unroll
    for (int u = 0; u < 4; ++u) red[u * T + t] = t < U && u < nv ? v[u] : 0.0;
    __syncthreads();
    int P = 1;
    while (2 * P <= G) P *= 2;
    if (t < (G - P) * m)
#pragma unroll
        for (int u = 0; u < 4; ++u) red[u * T + t] += red[u * T + t + P * m];
    __syncthreads();
    for (int h = P / 2; h > 0; h /= 2) {
        if (t < h * m)
#pragma unroll
            for (int u = 0; u < 4; ++u) red[u * T + t] += red[u * T + t + h * m];
        __syncthreads();
    }
    if (t < m)
        for (int u = 0; u < nv; ++u) out[u * ostride + t] = red[u * T + t];
    __syncthreads();
}

// ------------------------------------------------------------- stages
// (the level descriptors are read once per tile into registers: the item
// loops touch only plain pointers and sizes)
// Items are taken SW at a time, all loads before any store: in place (a
// graph colouring) the loads of a colour step read only entries of the other
// colour, which its stores never touch, so the order is free, and the SW
// independent load groups keep SW times more requests in flight per thread.
constexpr int SW = 4;
// Krylov dot products and norms: products are summed in the vector precision
// over up to KCH items, and those partial sums in FP64 (on this part FP64
// adds issue at 1/64 of the FP32 rate, so FP32 vectors keep them rare)
constexpr int KCH = 8;

// Red-black colour c = (ix + iy) mod 2 of the nodes of an nx-wide grid,
// enumerated in index order: colour_before counts the colour-c nodes with
// index below i; colour_node gives the g-th one.  With nx odd the colour is
// i mod 2; with nx even every row holds nx / 2 nodes of each colour, at the
// x-parity (c + iy) mod 2.
__device__ __forceinline__ int colour_before(int nx, int c, int i) {
    if (nx & 1) return (i + 1 - c) >> 1;
    const int iy = i / nx, ix = i - iy * nx;
    return iy * (nx >> 1) + ((ix + 1 - ((c + iy) & 1)) >> 1);
}
__device__ __forceinline__ void colour_node(int nx, int c, int g, int &i, int &ix, int &iy) {
    if (nx & 1) {
        i = 2 * g + c;
        iy = i / nx;
        ix = i - iy * nx;
    } else {
        const int h = nx >> 1;
        iy = g / h;
        ix = 2 * (g - iy * h) + ((c + iy) & 1);
        i = ix + iy * nx;
    }
}

// x_i - lambda_i ((A x)_i - b_i) for cnt nodes: the nodes g0 .. g0 + cnt - 1
// (COL false) or the colour-`colour` nodes of those ranks (COL true)
template <typename T, int KIND, bool COL>
__device__ __forceinline__ void relax_nodes(int nx, int ny, int64_t N, const T *__restrict__ A,
                                            const T *__restrict__ lam, const T *__restrict__ b, int m, int r,
                                            int g0, int cnt, int n0, int step, int colour, const T *src, T *dst) {
    for (int nn = n0; nn < cnt; nn += SW * step) {
        T val[SW];
        int64_t ee[SW];
        bool wr[SW];
#pragma unroll
        for (int u = 0; u < SW; ++u) {
            const int n = nn + u * step;
            wr[u] = false;
            ee[u] = 0;
            val[u] = T(0);
            if (n < cnt) {
                int i, ix, iy;
                if (COL) {
                    colour_node(nx, colour, g0 + n, i, ix, iy);
                } else {
                    i = g0 + n;
                    iy = i / nx;
                    ix = i - iy * nx;
                }
                const int64_t e = (int64_t)i * m + r;
                ee[u] = e;
                const T ax = row_apply<KIND, T, T>(nx, ny, N, A, src, m, r, ix, iy, i);
                const T res = ax - b[e];
                val[u] = src[e] - lam[i] * res;
                wr[u] = true;
            }
        }
#pragma unroll
        for (int u = 0; u < SW; ++u)
            if (wr[u]) dst[ee[u]] = val[u];
    }
}

// One cascade step over the tile's nodes [i0, i0 + ni).  A colour step
// (colour >= 0) deals out only the nodes of its colour, so no lane idles on
// the other colour; out of place it then copies the other colour's nodes.
template <typename T, int KIND>
__device__ __forceinline__ void sweep_tile(int nx, int ny, int64_t N, const T *__restrict__ A,
                                           const T *__restrict__ lam, const T *__restrict__ b, int m, int r, int i0,
                                           int ni, int n0, int step, int colour, const T *src, T *dst) {
    if (colour < 0) {
        relax_nodes<T, KIND, false>(nx, ny, N, A, lam, b, m, r, i0, ni, n0, step, -1, src, dst);
        return;
    }
    const int g0 = colour_before(nx, colour, i0);
    relax_nodes<T, KIND, true>(nx, ny, N, A, lam, b, m, r, g0, colour_before(nx, colour, i0 + ni) - g0, n0, step,
                               colour, src, dst);
    if (src != dst) {
        const int oc = colour ^ 1, h0 = colour_before(nx, oc, i0), hc = colour_before(nx, oc, i0 + ni) - h0;
#pragma unroll 4
        for (int nn = n0; nn < hc; nn += step) {
            int i, ix, iy;
            colour_node(nx, oc, h0 + nn, i, ix, iy);
            const int64_t e = (int64_t)i * m + r;
            dst[e] = src[e];
        }
    }
}

// Block step over a range of blocks (one thread per block and right-hand
// side): the residual rows of the block's present nodes, then
// x_b -= Lambda_b^(T) r_b (eq. fwda / fwdm with block Lambda).  Blocks of the
// other colour are copied when the step is not in place.
template <typename T, int KIND, int BS>
__device__ __forceinline__ void block_sweep_tile(int nx, int ny, int64_t N, int nbx, const T *__restrict__ A,
                                                 const T *__restrict__ lam, const T *__restrict__ b, int m, int r,
                                                 int b0, int nb, int n0, int step, int colour, int transpose,
                                                 const T *src, T *dst) {
    constexpr int NM = BS * BS;
    const bool copy = src != dst;
    for (int nn = n0; nn < nb; nn += step) {
        const int blk = b0 + nn;
        const int by = blk / nbx, bx = blk - by * nbx;
        int node[NM];
        bool pres[NM];
#pragma unroll
        for (int lp = 0; lp < NM; ++lp) {
            const int ix = BS * bx + lp % BS, iy = BS * by + lp / BS;
            pres[lp] = ix < nx && iy < ny;
            node[lp] = ix + nx * iy;
        }
        if (colour >= 0 && (((bx + 1) + (by + 1)) & 1) != colour) {
            if (copy)
#pragma unroll
                for (int lp = 0; lp < NM; ++lp)
                    if (pres[lp]) dst[(int64_t)node[lp] * m + r] = src[(int64_t)node[lp] * m + r];
            continue;
        }
        T res[NM], xv[NM];
#pragma unroll 1
        for (int lp = 0; lp < NM; ++lp) {
            res[lp] = T(0);
            xv[lp] = T(0);
            if (pres[lp]) {
                const int i = node[lp], iy = i / nx, ix = i - iy * nx;
                const int64_t e = (int64_t)i * m + r;
                res[lp] = row_apply<KIND, T, T>(nx, ny, N, A, src, m, r, ix, iy, i) - b[e];
                xv[lp] = src[e];
            }
        }
        const T *lb = lam + (int64_t)blk * (NM * NM);
#pragma unroll 1
        for (int lp = 0; lp < NM; ++lp) {
            if (!pres[lp]) continue;
            T acc = xv[lp];
#pragma unroll
            for (int q = 0; q < NM; ++q)
                acc = fma(-(transpose ? lb[q * NM + lp] : lb[lp * NM + q]), res[q], acc);
            dst[(int64_t)node[lp] * m + r] = acc;
        }
    }
}

// coarse node I of level l+1: b_c = 2^-2 sum_f P_{f,I} (A x - b)_f, x_c = 0
template <typename T, int KIND>
__device__ __forceinline__ void restrict_tile(int fnx, int fny, int64_t fN, const T *__restrict__ A,
                                              const T *__restrict__ xf, const T *__restrict__ bf, int cnx,
                                              T *__restrict__ bc, T *__restrict__ xc, int m, int r, int i0, int ni,
                                              int n0, int step) {
    for (int nn = n0; nn < ni; nn += step) {
        const int I = i0 + nn;
        const int cy = I / cnx, cx = I - cy * cnx;
        T acc = T(0);
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            const int fy = 2 * cy + 1 + dy;
            if (fy >= fny) continue;
#pragma unroll 1
            for (int dx = -1; dx <= 1; ++dx) {
                const int fx = 2 * cx + 1 + dx;
                if (fx >= fnx) continue;
                const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0));
                const int f = fx + fnx * fy;
                const T ax = row_apply<KIND, T, T>(fnx, fny, fN, A, xf, m, r, fx, fy, f);
                acc = fma(w, ax - bf[(int64_t)f * m + r], acc);
            }
        }
        bc[(int64_t)I * m + r] = acc * T(0.25);
        xc[(int64_t)I * m + r] = T(0);
    }
}

// 1D interpolation weights of fine node f from the coarse nodes (as in the
// single-problem prolongation): odd f sits on coarse (f-1)/2, even f takes
// half of coarse f/2-1 and f/2 where present.
__device__ __forceinline__ int bp1d(int f, int nc, int *c, float *w) {
    if (f & 1) {
        c[0] = (f - 1) >> 1;
        w[0] = 1.f;
        return 1;
    }
    int k = 0;
    const int lo = (f >> 1) - 1, hi = f >> 1;
    if (lo >= 0) { c[k] = lo; w[k] = 0.5f; ++k; }
    if (hi < nc) { c[k] = hi; w[k] = 0.5f; ++k; }
    return k;
}

template <typename T>
__device__ __forceinline__ void prolong_tile(int fnx, const T *xs, T *xf, int cnx, int cny,
                                             const T *__restrict__ xc, int m, int r, int i0, int ni, int n0,
                                             int step) {
    for (int nn = n0; nn < ni; nn += step) {
        const int f = i0 + nn;
        const int fy = f / fnx, fx = f - fy * fnx;
        int cxs[2], cys[2];
        float wx[2], wy[2];
        const int kx = bp1d(fx, cnx, cxs, wx), ky = bp1d(fy, cny, cys, wy);
        T acc = T(0);
        for (int bb = 0; bb < ky; ++bb)
            for (int a = 0; a < kx; ++a) {
                const T w = T(wx[a] * wy[bb] * 1.f);
                const int c = cxs[a] + cnx * cys[bb];
                acc = fma(w, xc[(int64_t)c * m + r], acc);
            }
        const int64_t e = (int64_t)f * m + r;
        xf[e] = xs[e] - acc;
    }
}

template <typename T>
__device__ void stage_step(const BArgs &a, const BProb<T> *P, const BStep st) {
    const int tslot = st.op == OP_RESTRICT ? st.slot + 1 : st.slot;
    const bool blocks = st.op == OP_SWEEP && a.btiles != nullptr;
    const BTile *tiles = blocks ? a.btiles : a.tiles;
    const int *slot_tile = blocks ? a.slot_btile : a.slot_tile;
    const int t0 = slot_tile[tslot], t1 = slot_tile[tslot + 1];
    for (int k = t0 + blockIdx.x; k < t1; k += gridDim.x) {
        const BTile tile = tiles[k];
        if (__ldcg(a.work + tile.p) == 0) continue;
        if (st.op == OP_RESTRICT && tile.l == 0) continue;  // this problem's finest level starts at the coarse slot
        const BProb<T> &pr = P[tile.p];
        const int m = pr.m;
        const TileMap tm = tile_map(m);
        if (!tm.on) continue;
        const int r = tm.r;
        if (st.op == OP_SWEEP) {
            const BLevel<T> L = pr.lev[tile.l];
            const T *src;
            T *dst;
            if (st.colour >= 0) {
                src = L.inplace || st.parity == 0 ? L.x : L.t;
                dst = L.inplace || st.parity == 1 ? L.x : L.t;
            } else {
                src = st.src ? L.t : L.x;
                dst = st.dst ? L.t : L.x;
            }
            if (blocks) {
                const T *lamb = L.lam + (int64_t)st.lv * L.nblocks * L.nmax * L.nmax;
                if (L.kind == STAR)  // 2x2-node blocks (the batch plan admits no others)
                    block_sweep_tile<T, STAR, 2>(L.nx, L.ny, L.N, L.nbx, L.A, lamb, L.b, m, r, tile.i0, tile.ni,
                                                 tm.n0, tm.step, st.colour, st.transpose, src, dst);
                else
                    block_sweep_tile<T, BOX, 2>(L.nx, L.ny, L.N, L.nbx, L.A, lamb, L.b, m, r, tile.i0, tile.ni, tm.n0,
                                                tm.step, st.colour, st.transpose, src, dst);
                continue;
            }
            const T *lam = L.lam + (int64_t)st.lv * L.N;
            if (L.kind == STAR)
                sweep_tile<T, STAR>(L.nx, L.ny, L.N, L.A, lam, L.b, m, r, tile.i0, tile.ni, tm.n0, tm.step, st.colour,
                                    src, dst);
            else
                sweep_tile<T, BOX>(L.nx, L.ny, L.N, L.A, lam, L.b, m, r, tile.i0, tile.ni, tm.n0, tm.step, st.colour,
                                   src, dst);
        } else if (st.op == OP_RESTRICT) {
            const BLevel<T> F = pr.lev[tile.l - 1], C = pr.lev[tile.l];
            const T *fx = st.src ? F.t : F.x;
            if (F.kind == STAR)
                restrict_tile<T, STAR>(F.nx, F.ny, F.N, F.A, fx, F.b, C.nx, C.b, C.x, m, r, tile.i0, tile.ni, tm.n0,
                                       tm.step);
            else
                restrict_tile<T, BOX>(F.nx, F.ny, F.N, F.A, fx, F.b, C.nx, C.b, C.x, m, r, tile.i0, tile.ni, tm.n0,
                                      tm.step);
        } else if (st.op == OP_COARSE) {
            const BLevel<T> L = pr.lev[tile.l];
            const int n = pr.cn;
            const double *__restrict__ cinv = pr.cinv;
            const T *__restrict__ lb = L.b;
            T *__restrict__ lx = L.x;
            for (int nn = tm.n0; nn < tile.ni; nn += tm.step) {
                const int i = tile.i0 + nn;
                double sacc = 0.0;
                for (int j = 0; j < n; ++j) sacc = fma(cinv[(int64_t)i * n + j], (double)lb[(int64_t)j * m + r], sacc);
                lx[(int64_t)i * m + r] = (T)sacc;
            }
        } else {  // OP_PROLONG
            const BLevel<T> F = pr.lev[tile.l], C = pr.lev[tile.l + 1];
            prolong_tile<T>(F.nx, st.src ? F.t : F.x, st.dst ? F.t : F.x, C.nx, C.ny, C.x, m, r, tile.i0, tile.ni,
                            tm.n0, tm.step);
        }
    }
}

// finest-level FP64 stages over the finest tiles.  Stages marked (A) run
// for every problem still iterating (state active); (W) ones only for
// problems with a right-hand side still extending its Krylov space in the
// current GMRES cycle (for the refinement method W = A).
enum {
    F_BNORM = 0,   // (A) partial sums of b^2
    F_ZEROX,       // (A) x = 0 for right-hand sides with b = 0
    F_RESID,       // (A) r = b - A x in FP64 -> cycle input (T), cycle output = 0; partial sums of r^2
    F_UPDATE,      // (A) x += cycle output (refinement)
    F_MB,          // (A) cycle input = b, output = 0 (for ||M b||)
    F_CONVZ,       // (W) Z = cycle output in FP64; partial sums of Z^2
    F_MATVEC,      // (W) cycle input = A V_j, output = 0
    F_PROJ,        // (W) partial sums of <Z, V_i>, i <= j (pass 0 also <Z, Z>) -> part2
    F_PAXPY,       // (W) Z -= sum_i hsum_i V_i, i <= j; partial sums of Z^2
    F_SCALEV,      // (W) V_j = Z / ||Z||
    F_XUPD,        // (A) x += sum_k y_k V_k (left) or sum_k y_k Z_k (right)
    F_VTOB,        // (W) right: cycle input = V_j, output = 0
    F_AZ           // (W) right: Z_j = cycle output (kept), Z = A Z_j in FP64
};

__device__ __forceinline__ bool fine_gate_all(int what) {
    return what == F_BNORM || what == F_ZEROX || what == F_RESID || what == F_UPDATE || what == F_MB ||
           what == F_XUPD;
}
__device__ __forceinline__ bool fine_reduces(int what) {
    return what == F_BNORM || what == F_RESID || what == F_CONVZ;
}

template <typename T>
__device__ void stage_fine(const BArgs &a, const BProb<T> *P, int what, int iarg, int jarg, double *red) {
    const bool gate_all = fine_gate_all(what), reduces = fine_reduces(what);
    for (int k = blockIdx.x; k < a.nftiles; k += gridDim.x) {
        const BTile tile = a.ftiles[k];
        const int p = tile.p;
        // uniform over the CTA: the flags change only in the per-problem stages
        if (gate_all ? __ldcg(a.state + p) != ST_ACTIVE : __ldcg(a.work + p) == 0) continue;
        const BProb<T> &pr = P[p];
        const BLevel<T> L = pr.lev[0];
        const int m = pr.m, nx = L.nx, ny = L.ny;
        const int64_t N = L.N, nm = N * m;
        const TileMap tm = tile_map(m);
        const int r = tm.r, q = p * BMAXRHS + r;
        const int i0 = tile.i0, ni = tile.ni, n0 = tm.n0, step = tm.step;
        const double *__restrict__ b = a.b64[p];
        double *__restrict__ x = a.x64[p];
        T *__restrict__ Z = pr.Z;
        const T *__restrict__ V = pr.V;
        T *__restrict__ lb = L.b;
        T *__restrict__ lx = L.x;
        if (what == F_PROJ) {
            // projections of Z on V_0..V_j (pass 0 adds <Z, Z> as slot j + 1),
            // four slots per sweep over the tile's items; products summed in
            // T over up to KCH items, those partial sums in FP64
            const int nsl = iarg == 0 ? jarg + 2 : jarg + 1;
            const bool on = tm.on && (iarg == 0 ? !a.frozen[q] : a.reorth[q] != 0);
            double *dst = a.part2 + a.p2off[p] + (int64_t)(k - a.ftile_of[p]) * (a.restart + 2) * m;
            for (int s0 = 0; s0 < nsl; s0 += 4) {
                double pacc[4] = {0.0, 0.0, 0.0, 0.0};
                const T *__restrict__ vs[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = s0 + u;
                    vs[u] = i <= jarg ? V + (int64_t)i * nm : Z;
                }
                const int nv = min(4, nsl - s0);
                if (on)
                    for (int nn = n0; nn < ni;) {
                        T c[4] = {T(0), T(0), T(0), T(0)};
                        for (int t = 0; t < KCH && nn < ni; ++t, nn += step) {
                            const int64_t e = (int64_t)(i0 + nn) * m + r;
                            const T z = Z[e];
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (u < nv) c[u] = fma(z, vs[u][e], c[u]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) pacc[u] += (double)c[u];
                    }
                cta_sum4_by_rhs(pacc, nv, m, red, dst + (int64_t)s0 * m, m);
            }
            continue;
        }
        if (what == F_PAXPY) {
            // Z -= sum_i h_i V_i in T (the coefficients staged in shared
            // memory as T, in chunks of slots that fit the reduction buffer:
            // one chunk up to restart 64 with 32 RHS), ||Z||^2 as in F_PROJ;
            // pass iarg: 0 -> every extending right-hand side, 1 -> those
            // reprojected
            T *hs = reinterpret_cast<T *>(red);
            const int cap = (int)((sizeof(double) * RED_DOUBLES) / sizeof(T)) / m;  // slots per chunk
            const bool act = tm.on && (iarg == 0 ? !a.frozen[q] : a.reorth[q] != 0);
            double acc = 0.0;
            for (int s0 = 0; s0 <= jarg; s0 += cap) {
                const int s1 = min(jarg + 1, s0 + cap);
                const bool last = s1 == jarg + 1;
                for (int t = threadIdx.x; t < (s1 - s0) * m; t += blockDim.x) {
                    const int i = t / m, rr = t - i * m;
                    hs[t] = (T)a.hsum[(int64_t)(p * BMAXRHS + rr) * (a.restart + 2) + s0 + i];
                }
                __syncthreads();
                if (act) {
                    for (int nn = n0; nn < ni;) {
                        T c = T(0);
                        for (int t = 0; t < KCH && nn < ni; ++t, nn += step) {
                            const int64_t e = (int64_t)(i0 + nn) * m + r;
                            T z = Z[e];
#pragma unroll 4
                            for (int i = s0; i < s1; ++i) z = fma(-hs[(i - s0) * m + r], V[(int64_t)i * nm + e], z);
                            Z[e] = z;
                            if (last) c = fma(z, z, c);
                        }
                        acc += (double)c;
                    }
                }
                __syncthreads();  // hs aliases the reduction buffer
            }
            cta_sum_by_rhs(acc, m, red, a.part + (int64_t)k * BMAXRHS);
            continue;
        }
        double acc = 0.0;
        if (tm.on) {
            if (what == F_BNORM) {
                for (int nn = n0; nn < ni; nn += step) {
                    const double v = b[(int64_t)(i0 + nn) * m + r];
                    acc = fma(v, v, acc);
                }
            } else if (what == F_ZEROX) {
                if (a.nb[q] == 0.0)
                    for (int nn = n0; nn < ni; nn += step) x[(int64_t)(i0 + nn) * m + r] = 0.0;
            } else if (what == F_RESID) {
                // the true residual: FP64 operator and arithmetic
                const double *__restrict__ A64 = pr.A64;
                const bool star = L.kind == STAR;
                for (int nn = n0; nn < ni; nn += step) {
                    const int i = i0 + nn;
                    const int iy = i / nx, ix = i - iy * nx;
                    const double ax = star ? row_apply<STAR, double, double>(nx, ny, N, A64, x, m, r, ix, iy, i)
                                           : row_apply<BOX, double, double>(nx, ny, N, A64, x, m, r, ix, iy, i);
                    const int64_t e = (int64_t)i * m + r;
                    const double v = b[e] - ax;
                    acc = fma(v, v, acc);
                    lb[e] = (T)v;
                    lx[e] = T(0);
                    if (a.method == CS_GMRES_RIGHT) Z[e] = (T)v;  // V_0 = r / ||r|| next
                }
            } else if (what == F_AZ) {
                // right preconditioning: keep Z_j = M V_j (the cycle output,
                // exact in T) and form the Krylov product A Z_j with the FP64
                // operator, as F_MATVEC does for the left form
                T *__restrict__ zj = pr.ZB + (int64_t)jarg * nm;
                const double *__restrict__ A64 = pr.A64;
                const bool star = L.kind == STAR;
                for (int nn = n0; nn < ni; nn += step) {
                    const int i = i0 + nn;
                    const int iy = i / nx, ix = i - iy * nx;
                    const double ax = star ? row_apply<STAR, double, double, T>(nx, ny, N, A64, lx, m, r, ix, iy, i)
                                           : row_apply<BOX, double, double, T>(nx, ny, N, A64, lx, m, r, ix, iy, i);
                    const int64_t e = (int64_t)i * m + r;
                    zj[e] = lx[e];
                    Z[e] = (T)ax;
                }
            } else if (what == F_VTOB) {
                const T *__restrict__ vj = V + (int64_t)jarg * nm;
                for (int nn = n0; nn < ni; nn += step) {
                    const int64_t e = (int64_t)(i0 + nn) * m + r;
                    lb[e] = vj[e];
                    lx[e] = T(0);
                }
            } else if (what == F_MATVEC) {
                // the Krylov product A V_j: the FP64 operator applied in FP64
                // to the basis vector's (exact) values.  The cycles' rounded
                // operator would perturb it by about u |A| |V_j|, which the
                // preconditioner amplifies by the operator's (Skeel)
                // condition number: too much for high-contrast coefficients.
                const T *__restrict__ vj = V + (int64_t)jarg * nm;
                const double *__restrict__ A64 = pr.A64;
                const bool star = L.kind == STAR;
                for (int nn = n0; nn < ni; nn += step) {
                    const int i = i0 + nn;
                    const int iy = i / nx, ix = i - iy * nx;
                    const double ax = star ? row_apply<STAR, double, double, T>(nx, ny, N, A64, vj, m, r, ix, iy, i)
                                           : row_apply<BOX, double, double, T>(nx, ny, N, A64, vj, m, r, ix, iy, i);
                    const int64_t e = (int64_t)i * m + r;
                    lb[e] = (T)ax;
                    lx[e] = T(0);
                }
            } else if (what == F_UPDATE) {
                for (int nn = n0; nn < ni; nn += step) {
                    const int64_t e = (int64_t)(i0 + nn) * m + r;
                    x[e] += (double)lx[e];
                }
            } else if (what == F_MB) {
                for (int nn = n0; nn < ni; nn += step) {
                    const int64_t e = (int64_t)(i0 + nn) * m + r;
                    lb[e] = (T)b[e];
                    lx[e] = T(0);
                }
            } else if (what == F_CONVZ) {
                for (int nn = n0; nn < ni;) {
                    T c = T(0);
                    for (int t = 0; t < KCH && nn < ni; ++t, nn += step) {
                        const int64_t e = (int64_t)(i0 + nn) * m + r;
                        const T z = lx[e];
                        Z[e] = z;
                        c = fma(z, z, c);
                    }
                    acc += (double)c;
                }
            } else if (what == F_SCALEV) {
                if (!a.frozen[q] || jarg == 0) {
                    T *__restrict__ Vj = pr.V + (int64_t)jarg * nm;
                    const T inv = (T)a.inv[q];
                    for (int nn = n0; nn < ni; nn += step) {
                        const int64_t e = (int64_t)(i0 + nn) * m + r;
                        Vj[e] = Z[e] * inv;
                    }
                }
            } else {  // F_XUPD: x += V y (left) or Z y (right) in FP64 (y can combine with heavy cancellation)
                const int nc = a.jcols[q];
                const double *__restrict__ y = a.y + (int64_t)q * a.restart;
                const T *__restrict__ basis = a.method == CS_GMRES_RIGHT ? pr.ZB : V;
                for (int nn = n0; nn < ni; nn += step) {
                    const int64_t e = (int64_t)(i0 + nn) * m + r;
                    double sx = x[e];
                    for (int kk = 0; kk < nc; ++kk) sx = fma(y[kk], (double)basis[(int64_t)kk * nm + e], sx);
                    x[e] = sx;
                }
            }
        }
        if (reduces) cta_sum_by_rhs(acc, m, red, a.part + (int64_t)k * BMAXRHS);
    }
}

// Per-problem stages (one thread per problem, its right-hand sides in turn):
// they sum the problem's tile partials in tile order and advance the small
// per-right-hand-side state.  Stages that count write ctl->cnt[ph] and clear
// ctl->cnt[ph ^ 1] (read before the barriers that precede this stage).
enum {
    P_NORMB = 0,  // ||b||
    P_NORM,       // true relative residuals: convergence, divergence, limit; counts active problems
    P_NMB,        // ||M b|| (GMRES stopping estimate scale)
    P_BETA,       // beta = ||M r|| (left) or ||r|| (right), g = beta e_1, V_0 scale; counts extending ones
    P_REORTH,     // ||Z||^2 after the first projection; reproject where it fell below half <Z, Z>; counts them
    P_GIVENS,     // H(j+1, j) = ||Z||, rotations, g, freeze; counts extending right-hand sides
    P_SOLVEY      // y = H^{-1} g (back substitution over the columns built)
};

template <typename T>
__device__ void stage_prob(const BArgs &a, const BProb<T> *P, int what, int iarg, int jarg, int ph, bool first,
                           double *wsum) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if ((what == P_NORM || what == P_BETA || what == P_GIVENS || what == P_REORTH) && gid == 0)
        a.ctl->cnt[ph ^ 1] = 0;
    const int R = a.restart;
    const int lane = threadIdx.x & 31;
    double *ws = wsum + (threadIdx.x >> 5) * BMAXRHS;
    const bool sums = what != P_SOLVEY;
    // one warp per problem: the lanes sum the problem's tile partials (lane
    // l takes tiles k0 + l, k0 + l + 32, ...; fixed shuffle tree), lane 0 then
    // advances the problem's state
    for (int p = gid >> 5; p < a.nprob; p += (gridDim.x * blockDim.x) >> 5) {
        if (a.state[p] != ST_ACTIVE) continue;  // warp-uniform
        if ((what == P_REORTH || what == P_GIVENS) && !a.work[p]) continue;
        const int m = P[p].m;
        const int q0 = p * BMAXRHS;
        if (sums) {
            const int k0 = a.ftile_of[p], k1 = a.ftile_of[p + 1];
            for (int r = 0; r < m; ++r) {
                double v = 0.0;
                for (int k = k0 + lane; k < k1; k += 32) v += __ldcg(a.part + (int64_t)k * BMAXRHS + r);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) ws[r] = v;
            }
        }
        __syncwarp();
        if (lane != 0) continue;
        auto tsum = [&](int r) { return ws[r]; };
        if (what == P_NORMB || what == P_NMB) {
            double *dst = what == P_NORMB ? a.nb : a.nmb;
            for (int r = 0; r < m; ++r) dst[q0 + r] = sqrt(tsum(r));
            if (what == P_NORMB && a.method == CS_GMRES_RIGHT)  // right: the test is on ||r|| / ||b||
                for (int r = 0; r < m; ++r) a.nmb[q0 + r] = a.nb[q0 + r];
        } else if (what == P_NORM) {
            double worst = 0.0;
            bool conv = true, bad = false;
            for (int r = 0; r < m; ++r) {
                const double nb = a.nb[q0 + r];
                const double rel = nb > 0.0 ? sqrt(tsum(r)) / nb : 0.0;
                a.rel[q0 + r] = rel;
                if (!(rel <= a.ctl->tol)) conv = false;
                if (!isfinite(rel)) bad = true;
                worst = fmax(worst, rel);
            }
            if (first) a.rel0[p] = worst;
            if (!first && a.method == CS_REFINE) a.iters[p] += 1;
            int st = ST_ACTIVE;
            if (conv) st = ST_CONVERGED;
            else if (bad || (a.method == CS_REFINE && worst > 1e3 * fmax(a.rel0[p], 1.0))) st = ST_DIVERGED;
            else if (a.iters[p] >= a.ctl->maxit) st = ST_MAXIT;
            a.state[p] = st;
            a.work[p] = st == ST_ACTIVE;
            if (st == ST_ACTIVE) atomicAdd(&a.ctl->cnt[ph], 1);
        } else if (what == P_BETA) {
            int ext = 0;
            for (int r = 0; r < m; ++r) {
                const int q = q0 + r;
                const double ss = tsum(r);
                const double beta = sqrt(ss);
                a.g[(int64_t)q * (R + 1)] = beta;
                a.beta[q] = beta;
                a.inv[q] = beta > 0.0 ? 1.0 / sqrt(ss) : 0.0;
                a.jcols[q] = 0;
                a.frozen[q] = !(beta > 0.0) || a.iters[p] >= a.ctl->maxit;
                ext += !a.frozen[q];
            }
            a.work[p] = ext > 0;
            if (ext) atomicAdd(&a.ctl->cnt[ph], ext);
        } else if (what == P_REORTH) {
            // DGKS criterion: a second projection when ||Z - V h|| < ||Z|| / sqrt(2)
            int nre = 0;
            for (int r = 0; r < m; ++r) {
                const int q = q0 + r;
                if (a.frozen[q]) {
                    a.reorth[q] = 0;
                    continue;
                }
                const double ss = tsum(r);
                a.znorm2[q] = ss;
                const int re = ss < 0.5 * a.hsum[(int64_t)q * (R + 2) + jarg + 1];
                a.reorth[q] = re;
                nre += re;
            }
            if (nre) atomicAdd(&a.ctl->cnt[ph], nre);
        } else if (what == P_GIVENS) {
            const int j = jarg;
            a.iters[p] += 1;
            const bool limit = a.iters[p] >= a.ctl->maxit;
            int ext = 0;
            for (int r = 0; r < m; ++r) {
                const int q = q0 + r;
                if (a.frozen[q]) continue;
                double *H = a.H + (int64_t)q * a.hstride;
                double *cs = a.cs + (int64_t)q * R, *sn = a.sn + (int64_t)q * R, *g = a.g + (int64_t)q * (R + 1);
                const double ss = a.reorth[q] ? tsum(r) : a.znorm2[q];  // ||Z||^2 after the last projection
                const double hn = sqrt(ss);
                a.inv[q] = hn > 0.0 ? 1.0 / sqrt(ss) : 0.0;
                H[(j + 1) * R + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double x0 = H[i * R + j], x1 = H[(i + 1) * R + j];
                    H[i * R + j] = cs[i] * x0 + sn[i] * x1;
                    H[(i + 1) * R + j] = -sn[i] * x0 + cs[i] * x1;
                }
                const double x0 = H[j * R + j], x1 = H[(j + 1) * R + j];
                const double d = sqrt(x0 * x0 + x1 * x1);
                cs[j] = d > 0 ? x0 / d : 1.0;
                sn[j] = d > 0 ? x1 / d : 0.0;
                H[j * R + j] = d;
                H[(j + 1) * R + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                a.jcols[q] = j + 1;
                if (fabs(g[j + 1]) <= a.ctl->tol * a.nmb[q] || fabs(g[j + 1]) <= a.itol * a.beta[q] || hn == 0.0 ||
                    limit || j + 1 >= R)
                    a.frozen[q] = 1;
                else ++ext;
            }
            a.work[p] = ext > 0;
            if (ext) atomicAdd(&a.ctl->cnt[ph], ext);
        } else {  // P_SOLVEY
            for (int r = 0; r < m; ++r) {
                const int q = q0 + r;
                const double *H = a.H + (int64_t)q * a.hstride, *g = a.g + (int64_t)q * (R + 1);
                double *y = a.y + (int64_t)q * R;
                const int nc = a.jcols[q];
                for (int i = nc - 1; i >= 0; --i) {
                    double sum = g[i];
                    for (int k = i + 1; k < nc; ++k) sum -= H[i * R + k] * y[k];
                    y[i] = sum / H[i * R + i];
                }
            }
        }
    }
}

// Sums of the projection partials over each problem's tiles, one warp per
// (slot i, right-hand side): hsum_i = <Z, V_i> (pass 0 also slot j + 1 =
// <Z, Z>); H(i, j) takes the first pass's value and adds the second's.
template <typename T>
__device__ void stage_hsum(const BArgs &a, const BProb<T> *P, int j, int pass) {
    const int R = a.restart, nsl = pass == 0 ? j + 2 : j + 1;
    const int lane = threadIdx.x & 31;
    const int64_t nitems = (int64_t)nsl * a.qtot;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nitems; w += nwarps) {
        const int qi = (int)(w % a.qtot), i = (int)(w / a.qtot);
        const int q = a.qlist[qi], p = q / BMAXRHS, r = q - p * BMAXRHS;
        // warp-uniform gates (flags written before the preceding barrier)
        if (__ldcg(a.state + p) != ST_ACTIVE || __ldcg(a.work + p) == 0) continue;
        if (pass == 0 ? __ldcg(a.frozen + q) != 0 : __ldcg(a.reorth + q) == 0) continue;
        const int m = P[p].m;
        const int k0 = a.ftile_of[p], k1 = a.ftile_of[p + 1];
        const int64_t ts = (int64_t)(R + 2) * m;
        const double *src = a.part2 + a.p2off[p] + (int64_t)i * m + r;
        double v = 0.0;
        for (int k = k0 + lane; k < k1; k += 32) v += __ldcg(src + (int64_t)(k - k0) * ts);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            a.hsum[(int64_t)q * (R + 2) + i] = v;
            if (i <= j) {
                double *h = a.H + (int64_t)q * a.hstride + i * R + j;
                *h = pass == 0 ? v : *h + v;
            }
        }
    }
}

// A grid-wide barrier between stages; the code names the stage it closes
// (1000 + 100 op + slot: cycle stages, 2000 + F_*: fine stages, 3000 + P_*:
// per-problem stages, 4000 + pass: projection sums, 5000: loop tests).
#define BSYNC(code) grid.sync()

template <typename T>
__device__ __forceinline__ void vcycle_stages(const BArgs &a, const BProb<T> *P, cg::grid_group &grid) {
    for (int s = 0; s < a.nsteps; ++s) {
        stage_step<T>(a, P, a.steps[s]);
        BSYNC(1000 + 100 * a.steps[s].op + a.steps[s].slot);
    }
}

// The whole solve: every CTA runs every stage and passes every grid barrier
// (no early exit anywhere).  Each loop ends for all CTAs at once: the count
// it tests was written before the barrier that precedes the test, and the
// counting stage that clears it again runs only after at least one more
// barrier (or only when the count is zero); every loop is bounded by the
// iteration limit in any case.
template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_batch_solve(BArgs a) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[RED_DOUBLES];
    __shared__ double wsum[16 * BMAXRHS];
    const BProb<T> *P = static_cast<const BProb<T> *>(a.probs);
    const int maxit = a.ctl->maxit;
    // counting stages write ctl->cnt[ph] after flipping ph and clear the other
    // slot; the loop tests read the slot written last
    int ph = 0;
    stage_fine<T>(a, P, F_BNORM, 0, 0, red);
    BSYNC(2000 + F_BNORM);
    stage_prob<T>(a, P, P_NORMB, 0, 0, ph, true, wsum);
    BSYNC(3000 + P_NORMB);
    stage_fine<T>(a, P, F_ZEROX, 0, 0, red);
    BSYNC(2000 + F_ZEROX);
    const bool gmres = a.method == CS_GMRES || a.method == CS_GMRES_RIGHT;
    const bool right = a.method == CS_GMRES_RIGHT;
    if (a.method == CS_GMRES) {  // ||M b|| per right-hand side
        stage_fine<T>(a, P, F_MB, 0, 0, red);
        BSYNC(2000 + F_MB);
        vcycle_stages<T>(a, P, grid);
        stage_fine<T>(a, P, F_CONVZ, 0, 0, red);
        BSYNC(2000 + F_CONVZ);
        stage_prob<T>(a, P, P_NMB, 0, 0, ph, true, wsum);
        BSYNC(3000 + P_NMB);
    }
    stage_fine<T>(a, P, F_RESID, 0, 0, red);
    BSYNC(2000 + F_RESID);
    ph ^= 1;
    stage_prob<T>(a, P, P_NORM, 0, 0, ph, true, wsum);
    BSYNC(3000 + P_NORM);
    if (!gmres) {
        for (int it = 0; it < maxit; ++it) {
            if (__ldcg(&a.ctl->cnt[ph]) == 0) break;  // active problems
            vcycle_stages<T>(a, P, grid);
            stage_fine<T>(a, P, F_UPDATE, 0, 0, red);
            BSYNC(2000 + F_UPDATE);
            stage_fine<T>(a, P, F_RESID, 0, 0, red);
            BSYNC(2000 + F_RESID);
            ph ^= 1;
            stage_prob<T>(a, P, P_NORM, 0, 0, ph, false, wsum);
            BSYNC(3000 + P_NORM);
        }
        return;
    }
    const int R = a.restart;
    for (int cyc = 0; cyc <= maxit; ++cyc) {
        if (__ldcg(&a.ctl->cnt[ph]) == 0) break;  // active problems
        if (!right) {
            vcycle_stages<T>(a, P, grid);  // M r (the cycle input is r from F_RESID)
            stage_fine<T>(a, P, F_CONVZ, 0, 0, red);
            BSYNC(2000 + F_CONVZ);
        } else {
            // right: Z = r and the partial sums of r^2 come from F_RESID.  P_BETA
            // clears the count slot every CTA has just tested; the barrier keeps
            // a fast CTA from clearing it before a slow one has read it
            BSYNC(5000);
        }
        ph ^= 1;
        stage_prob<T>(a, P, P_BETA, 0, 0, ph, false, wsum);
        BSYNC(3000 + P_BETA);
        stage_fine<T>(a, P, F_SCALEV, 0, 0, red);
        BSYNC(2000 + F_SCALEV);
        for (int j = 0; j < R; ++j) {
            if (__ldcg(&a.ctl->cnt[ph]) == 0) break;  // right-hand sides still extending
            if (right) {  // Z = A M V_j, M V_j kept
                stage_fine<T>(a, P, F_VTOB, 0, j, red);
                BSYNC(2000 + F_VTOB);
                vcycle_stages<T>(a, P, grid);
                stage_fine<T>(a, P, F_AZ, 0, j, red);
                BSYNC(2000 + F_AZ);
            } else {  // Z = M A V_j
                stage_fine<T>(a, P, F_MATVEC, 0, j, red);
                BSYNC(2000 + F_MATVEC);
                vcycle_stages<T>(a, P, grid);
                stage_fine<T>(a, P, F_CONVZ, 0, 0, red);
                BSYNC(2000 + F_CONVZ);
            }
            // classical Gram-Schmidt with a second projection where the
            // first cancelled more than half of ||Z|| (DGKS)
            stage_fine<T>(a, P, F_PROJ, 0, j, red);
            BSYNC(2000 + F_PROJ);
            stage_hsum<T>(a, P, j, 0);
            BSYNC(4000);
            stage_fine<T>(a, P, F_PAXPY, 0, j, red);
            BSYNC(2000 + F_PAXPY);
            ph ^= 1;
            stage_prob<T>(a, P, P_REORTH, 0, j, ph, false, wsum);
            BSYNC(3000 + P_REORTH);
            if (__ldcg(&a.ctl->cnt[ph]) != 0) {  // right-hand sides projected again
                stage_fine<T>(a, P, F_PROJ, 1, j, red);
                BSYNC(2000 + F_PROJ);
                stage_hsum<T>(a, P, j, 1);
                BSYNC(4001);
                stage_fine<T>(a, P, F_PAXPY, 1, j, red);
                BSYNC(2000 + F_PAXPY);
            }
            ph ^= 1;
            stage_prob<T>(a, P, P_GIVENS, 0, j, ph, false, wsum);
            BSYNC(3000 + P_GIVENS);
            stage_fine<T>(a, P, F_SCALEV, 0, j + 1, red);
            BSYNC(2000 + F_SCALEV);
        }
        // every problem still active solves its small systems and updates x
        // (work flags may have cleared: these stages are gated on the state)
        stage_prob<T>(a, P, P_SOLVEY, 0, 0, ph, false, wsum);
        BSYNC(3000 + P_SOLVEY);
        stage_fine<T>(a, P, F_XUPD, 0, 0, red);
        BSYNC(2000 + F_XUPD);
        stage_fine<T>(a, P, F_RESID, 0, 0, red);
        BSYNC(2000 + F_RESID);
        ph ^= 1;
        stage_prob<T>(a, P, P_NORM, 0, 0, ph, false, wsum);
        BSYNC(3000 + P_NORM);
    }
}

}  // namespace csx

using namespace csx;


struct cs_batch {
    int nprob = 0, dmax = 0, precision = CS_FP32, order = CS_RF, mu_pre = 1, mu_post = 1, nu = 1;
    int kind = CS_MULTIPLICATIVE, bs = 1;
    int dev = 0;
    std::vector<int> m, nlev, slot0;
    std::vector<int64_t> nfine;
    std::vector<std::vector<int>> nx, ny;  // per problem per level
    void *probs = nullptr;
    size_t probs_bytes = 0;
    std::vector<unsigned char> hprobs;
    void *vec = nullptr;  // all multi-RHS level vectors
    BTile *tiles = nullptr, *ftiles = nullptr, *btiles = nullptr;
    int *slot_btile = nullptr;
    int *slot_tile = nullptr, *ftile_of = nullptr;
    int ntiles = 0, nftiles = 0;
    BStep *steps = nullptr;
    int nsteps = 0;
    double *part = nullptr, *nb = nullptr, *rel = nullptr, *rel0 = nullptr;
    int *state = nullptr, *iters = nullptr, *work = nullptr;
    BCtl *ctl = nullptr;
    int method = CS_REFINE, restart = 0;
    void *gm = nullptr;   // GMRES basis and work vectors of all problems
    void *gsm = nullptr;  // GMRES per-right-hand-side small state
    double *H = nullptr, *gcs = nullptr, *gsn = nullptr, *gy = nullptr, *gg = nullptr, *ginv = nullptr,
           *gnmb = nullptr;
    int *jcols = nullptr, *frozen = nullptr;
    double *part2 = nullptr, *hsum = nullptr, *znorm2 = nullptr, *gbeta = nullptr;
    int64_t *p2off = nullptr;
    int *qlist = nullptr, *reorth = nullptr;
    int qtot = 0;
    const double **bptr = nullptr;
    double **xptr = nullptr;
    // pinned host staging
    void *hstage = nullptr;
    size_t hstage_bytes = 0;
    int threads = 256, tiles_per_cta = 2, ctas = 0;
    std::vector<cs_batch_tune> tuned;
    cudaGraphExec_t graph = nullptr;
    bool graph_ok = true;
    double *tune_b = nullptr, *tune_x = nullptr;
    int64_t bytes = 0;
};

namespace {

template <typename T>
void *kernel_ptr() {
    return reinterpret_cast<void *>(&k_batch_solve<T>);
}

void *kernel_of(const cs_batch *B) {
    return B->precision == CS_FP32 ? kernel_ptr<float>() : kernel_ptr<double>();
}

// Work tiles of about equal work (grid nodes x right-hand sides): every
// slot's items, the finest levels' items and (block cascades) every slot's
// block items are cut into about tiles_per_cta x CTAs tiles, but no tile
// holds fewer items than a CTA has threads.  A problem's tiles are ranges of
// its own nodes (or blocks), so a tile's node count is its item share over
// the problem's right-hand side count.  Few large tiles per CTA keep each
// stage's serial chain of tile start-up latencies short; equal work per tile
// keeps the CTAs arriving at the stage barrier together.
cs_status build_tiles(cs_batch *B, int tiles_per_cta, cudaStream_t s) {
    const int64_t want = std::max<int64_t>(1, (int64_t)B->ctas * tiles_per_cta);
    auto tile_items = [&](int64_t items) { return std::max<int64_t>(B->threads, (items + want - 1) / want); };
    auto cut = [](std::vector<BTile> &out, int p, int l, int64_t n, int64_t per) {
        for (int64_t i0 = 0; i0 < n; i0 += per) out.push_back({p, l, (int)i0, (int)std::min<int64_t>(per, n - i0)});
    };
    std::vector<BTile> tl;
    std::vector<int> st(B->dmax + 1, 0);
    for (int t = 0; t < B->dmax; ++t) {
        st[t] = (int)tl.size();
        int64_t items = 0;
        for (int p = 0; p < B->nprob; ++p) {
            const int l = t - B->slot0[p];
            if (l >= 0) items += (int64_t)B->nx[p][l] * B->ny[p][l] * B->m[p];
        }
        const int64_t ti = tile_items(items);
        for (int p = 0; p < B->nprob; ++p) {
            const int l = t - B->slot0[p];
            if (l < 0) continue;
            cut(tl, p, l, (int64_t)B->nx[p][l] * B->ny[p][l], (ti + B->m[p] - 1) / B->m[p]);
        }
    }
    st[B->dmax] = (int)tl.size();
    std::vector<BTile> ft;
    std::vector<int> fo(B->nprob + 1, 0);
    {
        int64_t items = 0;
        for (int p = 0; p < B->nprob; ++p) items += B->nfine[p] * B->m[p];
        const int64_t ti = tile_items(items);
        for (int p = 0; p < B->nprob; ++p) {
            fo[p] = (int)ft.size();
            cut(ft, p, 0, B->nfine[p], (ti + B->m[p] - 1) / B->m[p]);
        }
    }
    fo[B->nprob] = (int)ft.size();
    // block tiles (block-level sweeps: one item per block and right-hand side)
    std::vector<BTile> bt;
    std::vector<int> sb(B->dmax + 1, 0);
    if (B->bs > 1) {
        auto nblk = [&](int p, int l) {
            return (int64_t)((B->nx[p][l] + B->bs - 1) / B->bs) * ((B->ny[p][l] + B->bs - 1) / B->bs);
        };
        for (int t = 0; t < B->dmax; ++t) {
            sb[t] = (int)bt.size();
            int64_t items = 0;
            for (int p = 0; p < B->nprob; ++p) {
                const int l = t - B->slot0[p];
                if (l >= 0) items += nblk(p, l) * B->m[p];
            }
            const int64_t ti = tile_items(items);
            for (int p = 0; p < B->nprob; ++p) {
                const int l = t - B->slot0[p];
                if (l < 0) continue;
                cut(bt, p, l, nblk(p, l), (ti + B->m[p] - 1) / B->m[p]);
            }
        }
        sb[B->dmax] = (int)bt.size();
    }
    // a captured graph holds the old table pointers
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    dfree(B->tiles, s); dfree(B->ftiles, s); dfree(B->slot_tile, s); dfree(B->ftile_of, s); dfree(B->part, s);
    dfree(B->btiles, s); dfree(B->slot_btile, s); dfree(B->part2, s); dfree(B->p2off, s);
    B->tiles = nullptr; B->ftiles = nullptr; B->slot_tile = nullptr; B->ftile_of = nullptr; B->part = nullptr;
    B->btiles = nullptr; B->slot_btile = nullptr; B->part2 = nullptr; B->p2off = nullptr;
    if (B->method != CS_REFINE) {  // projection partials: (restart + 2) slots x m_p per finest tile
        std::vector<int64_t> po(B->nprob + 1, 0);
        for (int p = 0; p < B->nprob; ++p)
            po[p + 1] = po[p] + (int64_t)(fo[p + 1] - fo[p]) * (B->restart + 2) * B->m[p];
        CSX_TRY(dalloc_t(&B->p2off, po.size(), nullptr, s));
        CSX_TRY(dalloc_t(&B->part2, (size_t)std::max<int64_t>(1, po[B->nprob]), nullptr, s));
        CSX_CUDA(cudaMemcpyAsync(B->p2off, po.data(), po.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        CSX_CUDA(cudaStreamSynchronize(s));
    }
    if (B->bs > 1) {
        CSX_TRY(dalloc_t(&B->btiles, bt.size(), nullptr, s));
        CSX_TRY(dalloc_t(&B->slot_btile, sb.size(), nullptr, s));
        CSX_CUDA(cudaMemcpyAsync(B->btiles, bt.data(), bt.size() * sizeof(BTile), cudaMemcpyHostToDevice, s));
        CSX_CUDA(cudaMemcpyAsync(B->slot_btile, sb.data(), sb.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    CSX_TRY(dalloc_t(&B->tiles, tl.size(), nullptr, s));
    CSX_TRY(dalloc_t(&B->ftiles, ft.size(), nullptr, s));
    CSX_TRY(dalloc_t(&B->slot_tile, st.size(), nullptr, s));
    CSX_TRY(dalloc_t(&B->ftile_of, fo.size(), nullptr, s));
    CSX_TRY(dalloc_t(&B->part, ft.size() * BMAXRHS, nullptr, s));
    CSX_CUDA(cudaMemcpyAsync(B->tiles, tl.data(), tl.size() * sizeof(BTile), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(B->ftiles, ft.data(), ft.size() * sizeof(BTile), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(B->slot_tile, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(B->ftile_of, fo.data(), fo.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    B->ntiles = (int)tl.size();
    B->nftiles = (int)ft.size();
    B->tiles_per_cta = tiles_per_cta;
    return CS_OK;
}

BArgs args_of(const cs_batch *B) {
    BArgs a;
    a.probs = B->probs;
    a.nprob = B->nprob;
    a.tiles = B->tiles;
    a.slot_tile = B->slot_tile;
    a.btiles = B->btiles;
    a.slot_btile = B->slot_btile;
    a.dmax = B->dmax;
    a.ftiles = B->ftiles;
    a.ftile_of = B->ftile_of;
    a.nftiles = B->nftiles;
    a.steps = B->steps;
    a.nsteps = B->nsteps;
    a.b64 = B->bptr;
    a.x64 = B->xptr;
    a.part = B->part;
    a.nb = B->nb;
    a.rel = B->rel;
    a.rel0 = B->rel0;
    a.state = B->state;
    a.iters = B->iters;
    a.work = B->work;
    a.ctl = B->ctl;
    a.method = B->method;
    a.restart = B->restart;
    a.hstride = (B->restart + 1) * B->restart;
    a.H = B->H;
    a.cs = B->gcs;
    a.sn = B->gsn;
    a.y = B->gy;
    a.g = B->gg;
    a.inv = B->ginv;
    a.nmb = B->gnmb;
    a.jcols = B->jcols;
    a.frozen = B->frozen;
    a.part2 = B->part2;
    a.p2off = B->p2off;
    a.qtot = B->qtot;
    a.qlist = B->qlist;
    a.hsum = B->hsum;
    a.znorm2 = B->znorm2;
    a.reorth = B->reorth;
    a.beta = B->gbeta;
    // FP32 Krylov vectors resolve about 1e-6 of ||M r||: a GMRES cycle stops
    // at 1e-5 and the restart's FP64 residual refines (GMRES-IR)
    a.itol = B->precision == CS_FP32 ? 1e-5 : 0.0;
    return a;
}

// CTAs that can be co-resident (a cooperative launch needs all of them)
cs_status coresident(const cs_batch *B, int threads, int *ctas) {
    int nsm = 0, per = 0;
    CSX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->dev));
    CSX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel_of(B), threads, 0));
    if (per < 1) {
        set_error("batched solve kernel cannot run %d threads per CTA", threads);
        return CS_ERR_UNSUPPORTED;
    }
    *ctas = per * nsm;
    return CS_OK;
}

cs_status launch(cs_batch *B, cudaStream_t s) {
    BArgs a = args_of(B);
    void *params[] = {&a};
    CSX_CUDA(cudaLaunchCooperativeKernel(kernel_of(B), dim3((unsigned)B->ctas), dim3((unsigned)B->threads), params, 0,
                                         s));
    count_launch();
    return CS_OK;
}

// per-solve control: tolerance, iteration limit, zeroed counters and states
cs_status reset_control(cs_batch *B, double tol, int maxit, cudaStream_t s) {
    BCtl c;
    c.tol = tol;
    c.maxit = maxit;
    c.cnt[0] = c.cnt[1] = 0;
    std::memcpy(B->hstage, &c, sizeof(c));
    CSX_CUDA(cudaMemcpyAsync(B->ctl, B->hstage, sizeof(c), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemsetAsync(B->state, 0, sizeof(int) * B->nprob, s));
    CSX_CUDA(cudaMemsetAsync(B->iters, 0, sizeof(int) * B->nprob, s));
    CSX_CUDA(cudaMemsetAsync(B->work, 1, sizeof(int) * B->nprob, s));  // nonzero: every problem takes part
    return CS_OK;
}

cs_status set_pointers(cs_batch *B, const double *const *b, double *const *x, cudaStream_t s) {
    char *h = static_cast<char *>(B->hstage) + 64;
    std::memcpy(h, b, sizeof(double *) * B->nprob);
    std::memcpy(h + sizeof(double *) * B->nprob, x, sizeof(double *) * B->nprob);
    CSX_CUDA(cudaMemcpyAsync(B->bptr, h, sizeof(double *) * B->nprob, cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(B->xptr, h + sizeof(double *) * B->nprob, sizeof(double *) * B->nprob,
                             cudaMemcpyHostToDevice, s));
    return CS_OK;
}

// the kernel, captured once per configuration into a graph; if capturing a
// cooperative launch is refused, it is launched directly
cs_status run(cs_batch *B, cudaStream_t s) {
    if (!B->graph && B->graph_ok) {
        cudaStream_t cs = nullptr;
        CSX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            BArgs a = args_of(B);
            void *params[] = {&a};
            cudaError_t le = cudaLaunchCooperativeKernel(kernel_of(B), dim3((unsigned)B->ctas),
                                                         dim3((unsigned)B->threads), params, 0, cs);
            e = cudaStreamEndCapture(cs, &g);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            B->graph = nullptr;
            B->graph_ok = false;
        }
    }
    if (B->graph) {
        CSX_CUDA(cudaGraphLaunch(B->graph, s));
        count_launch();
        return CS_OK;
    }
    return launch(B, s);
}

void build_steps(const cs_batch *B, std::vector<BStep> &out) {
    // The buffer holding a level's iterate is the same for every problem at a
    // slot: multiplicative steps come in colour pairs that end in x; additive
    // steps flip between x and t, and the prolongation writes the buffer from
    // which the post-smoothing steps end in x (the single-problem rule).
    const bool rf = B->order == CS_RF, mult = B->kind == CS_MULTIPLICATIVE;
    std::vector<int> pre_cur(B->dmax, 0);
    for (int t = 0; t + 1 < B->dmax; ++t) {
        int cur = 0;
        for (int mu = 0; mu < B->mu_pre; ++mu)
            for (int step = 0; step < B->nu; ++step) {
                const int lv = rf ? B->nu - 1 - step : step;
                if (mult) {
                    for (int kk = 0; kk < 2; ++kk) out.push_back({OP_SWEEP, t, lv, rf ? 1 - kk : kk, kk, 0, 0, rf});
                } else {
                    out.push_back({OP_SWEEP, t, lv, -1, 0, cur, 1 - cur, rf});
                    cur ^= 1;
                }
            }
        out.push_back({OP_RESTRICT, t, 0, 0, 0, cur, 0, 0});
        pre_cur[t] = cur;
    }
    out.push_back({OP_COARSE, B->dmax - 1, 0, 0, 0, 0, 0, 0});
    const int post_flips = mult ? 0 : B->mu_post * B->nu;
    for (int t = B->dmax - 2; t >= 0; --t) {
        int cur = post_flips % 2 == 0 ? 0 : 1;
        out.push_back({OP_PROLONG, t, 0, 0, 0, pre_cur[t], cur, 0});
        for (int mu = 0; mu < B->mu_post; ++mu)
            for (int step = 0; step < B->nu; ++step) {
                if (mult) {
                    for (int kk = 0; kk < 2; ++kk) out.push_back({OP_SWEEP, t, step, kk, kk, 0, 0, 0});
                } else {
                    out.push_back({OP_SWEEP, t, step, -1, 0, cur, 1 - cur, 0});
                    cur ^= 1;
                }
            }
    }
}

template <typename T>
cs_status fill_probs(cs_batch *B, cs_hierarchy *const *h, cs_cascade *const *c, T *vec, T *gm) {
    B->probs_bytes = sizeof(BProb<T>) * B->nprob;
    B->hprobs.assign(B->probs_bytes, 0);
    BProb<T> *hp = reinterpret_cast<BProb<T> *>(B->hprobs.data());
    T *v = vec;
    for (int p = 0; p < B->nprob; ++p) {
        BProb<T> &q = hp[p];
        q.nlev = h[p]->nlev;
        q.m = B->m[p];
        q.slot0 = B->slot0[p];
        q.cn = h[p]->cn;
        q.A64 = h[p]->lev[0].A;
        q.cinv = h[p]->cinv;
        q.Z = nullptr;
        q.V = nullptr;
        q.ZB = nullptr;
        if (gm) {
            const int64_t n0 = h[p]->lev[0].g.N * B->m[p];
            q.Z = gm;
            q.V = gm + n0;
            gm += (int64_t)(B->restart + 2) * n0;
            if (B->method == CS_GMRES_RIGHT) {
                q.ZB = gm;
                gm += (int64_t)B->restart * n0;
            }
        }
        for (int l = 0; l < q.nlev; ++l) {
            const Level &L = h[p]->lev[l];
            BLevel<T> &d = q.lev[l];
            d.nx = L.g.nx;
            d.ny = L.g.ny;
            d.kind = L.kind;
            // red-black (of nodes or of blocks) is a graph colouring of the 5-point stencil only
            d.inplace = B->kind == CS_MULTIPLICATIVE && L.kind == STAR ? 1 : 0;
            d.N = L.g.N;
            d.bs = L.bs;
            d.nbx = L.nbx;
            d.nmax = L.nmax;
            d.nblocks = L.nblocks;
            if (sizeof(T) == sizeof(float)) {
                d.A = reinterpret_cast<const T *>(c[p]->lo[l].A);
                d.lam = l < c[p]->nlev ? reinterpret_cast<const T *>(c[p]->lo[l].lam) : nullptr;
            } else {
                d.A = reinterpret_cast<const T *>(L.A);
                d.lam = l < c[p]->nlev ? reinterpret_cast<const T *>(c[p]->lam[l]) : nullptr;
            }
            const int64_t n = L.g.N * q.m;
            d.b = v; v += n;
            d.x = v; v += n;
            d.t = v; v += n;
        }
    }
    return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_batch_create(int nprob, cs_hierarchy *const *h, cs_cascade *const *c, const int *nrhs,
                          const cs_batch_opts *o, cs_stream stream, cs_batch **out) {
    if (!out || !h || !c || !nrhs || !o || nprob < 1) { set_error("null argument or empty batch"); return CS_ERR_ARG; }
    *out = nullptr;
    if (o->precision != CS_FP32 && o->precision != CS_FP64) { set_error("bad precision"); return CS_ERR_ARG; }
    if (o->order != CS_RF && o->order != CS_FF) { set_error("bad order"); return CS_ERR_ARG; }
    if (o->method != CS_REFINE && o->method != CS_GMRES && o->method != CS_GMRES_RIGHT) {
        set_error("batched method must be CS_REFINE, CS_GMRES or CS_GMRES_RIGHT");
        return CS_ERR_ARG;
    }
    if (o->method != CS_REFINE && (o->restart < 0 || o->restart > BMAXRESTART)) {
        set_error("GMRES restart must be in 1..%d", BMAXRESTART);
        return CS_ERR_ARG;
    }
    if (o->mu_pre < 0 || o->mu_post < 0 || o->mu_pre + o->mu_post < 1 || o->mu_pre > 16 || o->mu_post > 16) {
        set_error("bad smoothing counts");
        return CS_ERR_ARG;
    }
    int nu = -1;
    for (int p = 0; p < nprob; ++p) {
        const cs_hierarchy *hp = h[p];
        const cs_cascade *cp = c[p];
        if (!hp || !cp || cp->h != hp) { set_error("problem %d: missing or mismatched handles", p); return CS_ERR_ARG; }
        if (nrhs[p] < 1 || nrhs[p] > BMAXRHS) { set_error("problem %d: nrhs must be in 1..%d", p, BMAXRHS); return CS_ERR_ARG; }
        if (hp->dim != 2 || hp->periodic) { set_error("problem %d: the batched solver takes 2D Dirichlet grids", p); return CS_ERR_UNSUPPORTED; }
        if (cp->kind != c[0]->kind) { set_error("all problems of a batch need the same cascade kind"); return CS_ERR_ARG; }
        if (hp->nlev < 2 || hp->nlev > BMAXLEV || !hp->cinv) { set_error("problem %d: need 2..%d levels and a coarsest factorisation", p, BMAXLEV); return CS_ERR_UNSUPPORTED; }
        for (int l = 0; l < hp->nlev; ++l)
            if (hp->lev[l].bs != h[0]->lev[0].bs) { set_error("all problems of a batch need the same block size"); return CS_ERR_ARG; }
        if (hp->lev[0].bs > 2) { set_error("problem %d: the batched solver takes point blocks or 2x2-node blocks", p); return CS_ERR_UNSUPPORTED; }
        if (o->precision == CS_FP32 && !cp->lowp) { set_error("problem %d: FP32 cycles need a cascade built with lowp", p); return CS_ERR_ARG; }
        if (nu < 0) nu = cp->nu;
        if (cp->nu != nu) { set_error("all problems of a batch need the same cascade depth"); return CS_ERR_ARG; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cs_batch *B = new cs_batch();
    cs_status rc = CS_OK;
    B->nprob = nprob;
    B->precision = o->precision;
    B->order = o->order;
    B->mu_pre = o->mu_pre;
    B->mu_post = o->mu_post;
    B->nu = nu;
    B->kind = c[0]->kind;
    B->bs = h[0]->lev[0].bs;
    B->method = o->method;
    B->restart = o->restart > 0 ? o->restart : 30;
    cudaGetDevice(&B->dev);
    B->m.assign(nrhs, nrhs + nprob);
    B->nlev.resize(nprob);
    B->slot0.resize(nprob);
    B->nfine.resize(nprob);
    B->nx.resize(nprob);
    B->ny.resize(nprob);
    int64_t nvec = 0;
    for (int p = 0; p < nprob; ++p) {
        B->nlev[p] = h[p]->nlev;
        B->dmax = std::max(B->dmax, h[p]->nlev);
        B->nfine[p] = h[p]->lev[0].g.N;
        for (int l = 0; l < h[p]->nlev; ++l) {
            B->nx[p].push_back(h[p]->lev[l].g.nx);
            B->ny[p].push_back(h[p]->lev[l].g.ny);
            nvec += 3 * h[p]->lev[l].g.N * nrhs[p];
        }
    }
    for (int p = 0; p < nprob; ++p) B->slot0[p] = B->dmax - B->nlev[p];
    const size_t esz = o->precision == CS_FP32 ? sizeof(float) : sizeof(double);
    std::vector<BStep> steps;
    build_steps(B, steps);
    B->nsteps = (int)steps.size();
    int64_t nfine_rhs = 0;
    for (int p = 0; p < nprob; ++p) nfine_rhs += B->nfine[p] * B->m[p];
    if ((rc = dalloc(&B->vec, (size_t)nvec * esz, &B->bytes, s)) != CS_OK) goto fail;
    if (B->method != CS_REFINE) {
        // basis (restart + 1 vectors) and Z per problem, in the cycle precision, [N0][m] each;
        // right preconditioning keeps restart more (Z_j = M V_j)
        const size_t nv = (size_t)(B->restart + 2) + (B->method == CS_GMRES_RIGHT ? (size_t)B->restart : 0);
        if ((rc = dalloc(&B->gm, nv * nfine_rhs * esz, &B->bytes, s)) != CS_OK)
            goto fail;
        const size_t nq = (size_t)nprob * BMAXRHS, R = (size_t)B->restart;
        const size_t nd = nq * ((R + 1) * R + 3 * R + (R + 1) + 2 + (R + 2) + 2);
        if ((rc = dalloc(&B->gsm, nd * sizeof(double) + 3 * nq * sizeof(int), &B->bytes, s)) != CS_OK) goto fail;
        double *d = static_cast<double *>(B->gsm);
        B->H = d; d += nq * (R + 1) * R;
        B->gcs = d; d += nq * R;
        B->gsn = d; d += nq * R;
        B->gy = d; d += nq * R;
        B->gg = d; d += nq * (R + 1);
        B->ginv = d; d += nq;
        B->gnmb = d; d += nq;
        B->hsum = d; d += nq * (R + 2);
        B->znorm2 = d; d += nq;
        B->gbeta = d; d += nq;
        B->jcols = reinterpret_cast<int *>(d);
        B->frozen = B->jcols + nq;
        B->reorth = B->frozen + nq;
        // every right-hand side of every problem, for the projection sums
        std::vector<int> ql;
        for (int p = 0; p < nprob; ++p)
            for (int r = 0; r < B->m[p]; ++r) ql.push_back(p * BMAXRHS + r);
        B->qtot = (int)ql.size();
        if ((rc = dalloc_t(&B->qlist, ql.size(), &B->bytes, s)) != CS_OK) goto fail;
        if (cudaMemcpyAsync(B->qlist, ql.data(), ql.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch create", __FILE__, __LINE__);
            goto fail;
        }
    }
    if (o->precision == CS_FP32)
        rc = fill_probs<float>(B, h, c, static_cast<float *>(B->vec), static_cast<float *>(B->gm));
    else rc = fill_probs<double>(B, h, c, static_cast<double *>(B->vec), static_cast<double *>(B->gm));
    if (rc != CS_OK) goto fail;
    if ((rc = dalloc(&B->probs, B->probs_bytes, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->steps, steps.size(), &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->nb, (size_t)nprob * BMAXRHS, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->rel, (size_t)nprob * BMAXRHS, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->rel0, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->state, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->iters, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->work, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->ctl, 1, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->bptr, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&B->xptr, (size_t)nprob, &B->bytes, s)) != CS_OK) goto fail;
    B->hstage_bytes = 64 + 2 * sizeof(double *) * nprob + sizeof(double) * nprob * (BMAXRHS + 1) + sizeof(int) * 2 * nprob;
    {
        cudaError_t e = cudaMallocHost(&B->hstage, B->hstage_bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->probs, B->hprobs.data(), B->probs_bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->steps, steps.data(), steps.size() * sizeof(BStep), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "batch create", __FILE__, __LINE__); goto fail; }
    }
    {
        int threads = o->threads > 0 ? o->threads : 256;
        int tile = o->tiles_per_cta > 0 ? o->tiles_per_cta : 2;
        if (o->autotune) {
            // time each candidate on the batch itself: two cycles from x = 0
            // with b = 1 (tol 0: exactly two iterations), best of three
            if ((rc = dalloc_t(&B->tune_b, (size_t)nfine_rhs, nullptr, s)) != CS_OK) goto fail;
            if ((rc = dalloc_t(&B->tune_x, (size_t)nfine_rhs, nullptr, s)) != CS_OK) goto fail;
            std::vector<double> ones((size_t)std::min<int64_t>(nfine_rhs, 1 << 20), 1.0);
            for (int64_t o0 = 0; o0 < nfine_rhs; o0 += (int64_t)ones.size()) {
                const int64_t n = std::min<int64_t>((int64_t)ones.size(), nfine_rhs - o0);
                if (cudaMemcpyAsync(B->tune_b + o0, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess) {
                    rc = cuda_fail(cudaGetLastError(), "autotune input", __FILE__, __LINE__);
                    goto fail;
                }
            }
            std::vector<const double *> bp(nprob);
            std::vector<double *> xp(nprob);
            int64_t off = 0;
            for (int p = 0; p < nprob; ++p) {
                bp[p] = B->tune_b + off;
                xp[p] = B->tune_x + off;
                off += B->nfine[p] * B->m[p];
            }
            const int cand_threads[] = {128, 256, 512};
            const int cand_tile[] = {1, 2, 4};
            float best = 1e30f;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int ct : cand_threads)
                for (int tt : cand_tile) {
                    int ctas = 0;
                    if (coresident(B, ct, &ctas) != CS_OK) continue;
                    B->threads = ct;
                    B->ctas = ctas;
                    if ((rc = build_tiles(B, tt, s)) != CS_OK) break;
                    float ms_best = 1e30f;
                    for (int rep = 0; rep < 3 && rc == CS_OK; ++rep) {
                        if (cudaMemsetAsync(B->tune_x, 0, sizeof(double) * nfine_rhs, s) != cudaSuccess) {
                            rc = cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__);
                            break;
                        }
                        if ((rc = set_pointers(B, bp.data(), xp.data(), s)) != CS_OK) break;
                        if ((rc = reset_control(B, 0.0, 2, s)) != CS_OK) break;
                        cudaEventRecord(e0, s);
                        if ((rc = launch(B, s)) != CS_OK) break;
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) {
                            rc = cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__);
                            break;
                        }
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        ms_best = std::min(ms_best, ms);
                    }
                    if (rc != CS_OK) break;
                    B->tuned.push_back({ct, tt, ms_best});
                    if (ms_best < best) {
                        best = ms_best;
                        threads = ct;
                        tile = tt;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            dfree(B->tune_b, s);
            dfree(B->tune_x, s);
            B->tune_b = B->tune_x = nullptr;
            if (rc != CS_OK) goto fail;
        }
        if ((rc = coresident(B, threads, &B->ctas)) != CS_OK) goto fail;
        B->threads = threads;
        if ((rc = build_tiles(B, tile, s)) != CS_OK) goto fail;
    }
    *out = B;
    return CS_OK;
fail:
    cs_batch_destroy(B);
    return rc;
}

cs_status cs_batch_solve(cs_batch *B, const double *const *b, double *const *x, double tol, int maxit,
                         cs_solve_info *info, cs_stream stream) {
    if (!B || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    for (int p = 0; p < B->nprob; ++p)
        if (!b[p] || !x[p]) { set_error("problem %d: null vector", p); return CS_ERR_ARG; }
    if (tol <= 0) tol = 1e-10;
    if (maxit <= 0) maxit = 100;
    cudaStream_t s = (cudaStream_t)stream;
    CSX_TRY(set_pointers(B, b, x, s));
    CSX_TRY(reset_control(B, tol, maxit, s));
    CSX_TRY(run(B, s));
    const int np = B->nprob;
    char *h = static_cast<char *>(B->hstage) + 64 + 2 * sizeof(double *) * np;
    double *hrel = reinterpret_cast<double *>(h);
    int *hst = reinterpret_cast<int *>(hrel + (size_t)np * BMAXRHS);
    int *hit = hst + np;
    CSX_CUDA(cudaMemcpyAsync(hrel, B->rel, sizeof(double) * np * BMAXRHS, cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaMemcpyAsync(hst, B->state, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaMemcpyAsync(hit, B->iters, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    cs_status rc = CS_OK;
    int ndiv = 0, nnc = 0;
    for (int p = 0; p < np; ++p) {
        double worst = 0.0;
        for (int r = 0; r < B->m[p]; ++r) worst = std::max(worst, hrel[(size_t)p * BMAXRHS + r]);
        if (info) info[p] = {hit[p], hst[p] == ST_CONVERGED ? 1 : 0, worst, 0};
        if (hst[p] == ST_DIVERGED) ++ndiv;
        else if (hst[p] != ST_CONVERGED) ++nnc;
    }
    if (ndiv) {
        set_error("%d of %d problems diverged", ndiv, np);
        rc = CS_ERR_DIVERGED;
    } else if (nnc) {
        set_error("%d of %d problems not converged after %d iterations", nnc, np, maxit);
        rc = CS_ERR_NOTCONV;
    }
    return rc;
}

cs_status cs_batch_config(const cs_batch *B, int *threads, int *tiles_per_cta, int *ctas, cs_batch_tune *tuned,
                          int cap, int *ntuned) {
    if (!B) { set_error("null argument"); return CS_ERR_ARG; }
    if (threads) *threads = B->threads;
    if (tiles_per_cta) *tiles_per_cta = B->tiles_per_cta;
    if (ctas) *ctas = B->ctas;
    if (ntuned) *ntuned = (int)B->tuned.size();
    if (tuned)
        for (int k = 0; k < cap && k < (int)B->tuned.size(); ++k) tuned[k] = B->tuned[k];
    return CS_OK;
}

cs_status cs_batch_set_config(cs_batch *B, int threads, int tiles_per_cta, cs_stream stream) {
    if (!B || threads < 32 || threads > 512 || (threads & 31) || tiles_per_cta < 1 || tiles_per_cta > 1024) {
        set_error("bad batch configuration");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int ctas = 0;
    CSX_TRY(coresident(B, threads, &ctas));
    B->threads = threads;
    B->ctas = ctas;
    CSX_TRY(build_tiles(B, tiles_per_cta, s));
    return CS_OK;
}

int64_t cs_batch_bytes(const cs_batch *B) { return B ? B->bytes : 0; }

void cs_batch_destroy(cs_batch *B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    dfree(B->vec); dfree(B->probs); dfree(B->tiles); dfree(B->ftiles); dfree(B->slot_tile); dfree(B->ftile_of);
    dfree(B->btiles); dfree(B->slot_btile);
    dfree(B->steps); dfree(B->part); dfree(B->nb); dfree(B->rel); dfree(B->rel0); dfree(B->state); dfree(B->iters);
    dfree(B->ctl); dfree(B->bptr); dfree(B->xptr); dfree(B->tune_b); dfree(B->tune_x); dfree(B->work);
    dfree(B->gm); dfree(B->gsm); dfree(B->part2); dfree(B->p2off); dfree(B->qlist);
    if (B->hstage) cudaFreeHost(B->hstage);
    delete B;
}

cs_status cs_solve_batched(int nprob, cs_hierarchy *const *h, cs_cascade *const *c, const cs_solve_opts *o,
                           const double *const *b, double *const *x, const int *nrhs, cs_solve_info *info,
                           cs_stream stream) {
    if (!o) { set_error("null argument"); return CS_ERR_ARG; }
    cs_batch_opts bo{};
    bo.precision = o->cycle.precision;
    bo.order = o->cycle.order;
    bo.mu_pre = o->cycle.mu_pre;
    bo.mu_post = o->cycle.mu_post;
    bo.autotune = 0;
    bo.method = (o->method == CS_GMRES || o->method == CS_GMRES_RIGHT) ? o->method : CS_REFINE;
    bo.restart = o->restart;
    cs_batch *B = nullptr;
    CSX_TRY(cs_batch_create(nprob, h, c, nrhs, &bo, stream, &B));
    cs_status rc = cs_batch_solve(B, b, x, o->tol, o->maxit, info, stream);
    cs_batch_destroy(B);
    return rc;
}

}  // extern "C"
