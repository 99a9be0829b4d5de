// Setup kernels: Galerkin coarse operators (Sec. 2.4, SM Sec. 4.1), the
// bottom-level dense factorisation (Algorithm 1), and the cascade setup of
// Algorithm 2 / the SM multicoloured algorithm for point blocks.
//
// Cascade setup on a structured grid.  The residual E_l of the prescaled
// operator A~ = W A W has, in every row i, entries only at column offsets
// o in a set O_l that grows by the stencil S at every step (E_0 = I:
// O_0 = {0}; O_{next} = O + S).  E is stored as structure-of-arrays
// E[o*N + i] (no column indices).  One thread owns one row i and computes,
// in FP64,
//     R_i[o'] = sum_s A~_s(i) E_{i+s}[o' - s]                 ((A E)_{i,:})
//     lambda~_i = <E_i, R_i> / <R_i, R_i>       (least squares, Algorithm 2)
//     E'_i = E_i - lambda~_i R_i                            (residual update)
//     Lambda_i = w_i lambda~_i w_i                                (unscale)
// The pairs (o', s) -> index of o'-s in O are a host-built table read
// uniformly by a warp.  Additive: all rows read E_{l-1} and write E_l
// (separate buffers).  Multiplicative: the rows of colour k update from the
// state after colour k-1; other rows are carried over (snapshot semantics of
// E_{l,k} = (I - Lambda_{l,k} A) E_{l,k-1}).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <tuple>

#include "cs_internal.cuh"

namespace csx {

template <int DIM, int KIND>
struct StenS {
    static constexpr int NST = KIND == STAR ? 2 * DIM + 1 : (DIM == 3 ? 27 : 9);
    static __host__ __device__ __forceinline__ void off(int s, int &dx, int &dy, int &dz) {
        if (KIND == STAR) {
            dx = dy = dz = 0;
            if (s == 1) dx = -1;
            else if (s == 2) dx = 1;
            else if (s == 3) dy = -1;
            else if (s == 4) dy = 1;
            else if (s == 5) dz = -1;
            else if (s == 6) dz = 1;
        } else {
            dx = s % 3 - 1;
            dy = (s / 3) % 3 - 1;
            dz = DIM == 3 ? s / 9 - 1 : 0;
        }
    }
};

// ------------------------------------------------- repeated-row detection
// Sec. 4 (concluding remarks) notes that on structured meshes with uniform
// coefficients the smoother construction is the same almost everywhere and
// can be cached.  We use that exactly: if every row at boundary distance
// >= m has the same coefficient row as the grid-centre row, then any
// quantity that depends only on rows within radius r of row i is identical
// for all rows at distance >= m + r (for the multiplicative form: identical
// among rows of one colour).  Such "deep" rows are computed once, in a
// representative row, and copied; the result is bitwise the same as
// computing every row.
__device__ __forceinline__ int bdist(const Grid &g, int ix, int iy, int iz) {
    int d = min(min(ix, g.nx - 1 - ix), min(iy, g.ny - 1 - iy));
    if (g.dim == 3) d = min(d, min(iz, g.nz - 1 - iz));
    return d;
}
__device__ __forceinline__ int rb_colour(const Grid &g, int ix, int iy, int iz) {
    return ((ix + 1) + (iy + 1) + (g.dim == 3 ? iz + 1 : 0)) & 1;
}
static int bdist_host(const Grid &g, int ix, int iy, int iz) {
    int d = std::min(std::min(ix, g.nx - 1 - ix), std::min(iy, g.ny - 1 - iy));
    if (g.dim == 3) d = std::min(d, std::min(iz, g.nz - 1 - iz));
    return d;
}

// The rows a reuse-enabled kernel computes: the grid minus an inner box of
// deep rows (lo..hi inclusive per axis), enumerated densely so that warps
// hold only rows with work, followed by nrep representative rows.
struct RowSet {
    int on;
    int lo[3], hi[3];
    int64_t nshell;
    int nrep;
    int rep[2][3];
};

static int64_t rowset_shell_count(const Grid &g, const int *lo, const int *hi) {
    const int64_t nxi = hi[0] - lo[0] + 1, nyi = hi[1] - lo[1] + 1;
    const int64_t nzi = g.dim == 3 ? hi[2] - lo[2] + 1 : 1;
    return g.N - nxi * nyi * nzi;
}

// coordinates of the t-th row of the set; false past its end
__device__ __forceinline__ bool rowset_coord(const RowSet &rs, const Grid &g, int64_t t, int &ix, int &iy, int &iz) {
    if (t >= rs.nshell) {
        const int r = (int)(t - rs.nshell);
        if (r >= rs.nrep) return false;
        ix = rs.rep[r][0]; iy = rs.rep[r][1]; iz = rs.rep[r][2];
        return true;
    }
    const int nxi = rs.hi[0] - rs.lo[0] + 1, nyi = rs.hi[1] - rs.lo[1] + 1;
    const int nxo = g.nx - nxi, nyo = g.ny - nyi;
    int zlo = 0, nzi = 1;
    if (g.dim == 3) {  // whole outer z-planes first
        nzi = rs.hi[2] - rs.lo[2] + 1;
        zlo = rs.lo[2];
        const int64_t plane = (int64_t)g.nx * g.ny;
        const int64_t pz = (int64_t)(g.nz - nzi) * plane;
        if (t < pz) {
            const int k = (int)(t / plane);
            const int64_t rem = t - (int64_t)k * plane;
            iz = k < rs.lo[2] ? k : k + nzi;
            iy = (int)(rem / g.nx);
            ix = (int)(rem - (int64_t)iy * g.nx);
            return true;
        }
        t -= pz;
    }
    const int64_t pery = (int64_t)nyo * g.nx;  // outer y-rows of the inner z-range
    const int64_t py = (int64_t)nzi * pery;
    if (t < py) {
        const int zz = (int)(t / pery);
        const int64_t rem = t - (int64_t)zz * pery;
        const int k = (int)(rem / g.nx);
        iz = zlo + zz;
        iy = k < rs.lo[1] ? k : k + nyi;
        ix = (int)(rem - (int64_t)k * g.nx);
        return true;
    }
    t -= py;  // outer x-columns of the inner y- and z-range
    const int64_t perz = (int64_t)nyi * nxo;
    const int zz = (int)(t / perz);
    const int64_t rem = t - (int64_t)zz * perz;
    const int yy = (int)(rem / nxo);
    const int k = (int)(rem - (int64_t)yy * nxo);
    iz = zlo + zz;
    iy = rs.lo[1] + yy;
    ix = k < rs.lo[0] ? k : k + nxi;
    return true;
}

// maxd = max boundary distance of the rows whose coefficients differ from
// row `ref` (bitwise); -1 if none
__global__ void k_const_margin(Grid g, int nst, const double *__restrict__ A, int64_t ref, int *maxd) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    bool eq = true;
    for (int s = 0; s < nst; ++s)
        eq = eq && __double_as_longlong(A[(int64_t)s * g.N + i]) == __double_as_longlong(A[(int64_t)s * g.N + ref]);
    if (!eq) atomicMax(maxd, bdist(g, ix, iy, iz));
}

// Homogeneous Dirichlet elimination: a coupling to a node outside the grid
// multiplies a zero boundary value, so its coefficient is dropped once, on
// the copy of the fine operator; the Galerkin product and the margin scan
// then see only couplings inside the grid.
template <int DIM, int KIND>
__global__ void k_drop_outside(Grid g, double *__restrict__ A) {
    using S = StenS<DIM, KIND>;
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
#pragma unroll
    for (int s = 0; s < S::NST; ++s) {
        int dx, dy, dz;
        S::off(s, dx, dy, dz);
        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        const bool in = jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny && (DIM == 2 || (jz >= 0 && jz < g.nz));
        if (!in) A[(int64_t)s * g.N + i] = 0.0;
    }
}

cs_status drop_outside_couplings(const Level &L, cudaStream_t s) {
    const dim3 gr = node_grid(L.g), bl = node_block();
    if (L.g.dim == 2) {
        if (L.kind == STAR) k_drop_outside<2, STAR><<<gr, bl, 0, s>>>(L.g, L.A);
        else k_drop_outside<2, BOX><<<gr, bl, 0, s>>>(L.g, L.A);
    } else {
        if (L.kind == STAR) k_drop_outside<3, STAR><<<gr, bl, 0, s>>>(L.g, L.A);
        else k_drop_outside<3, BOX><<<gr, bl, 0, s>>>(L.g, L.A);
    }
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

// Symmetry of a 3D 27-point operator: every forward coupling A_{i,i+o}
// (entries 14..26) against the backward one stored at the neighbour,
// A_{i+o,i} (entry 26 - s there), within 1e-12 of the two diagonals.
__global__ void k_sym_check(Grid g, const double *__restrict__ A, int *asym) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t N = g.N, i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    const double di = fabs(A[13 * N + i]);
    for (int s = 14; s < 27; ++s) {
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny || jz < 0 || jz >= g.nz) continue;
        const int64_t j = jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz);
        const double f = A[(int64_t)s * N + i], bk = A[(int64_t)(26 - s) * N + j];
        if (!(fabs(f - bk) <= 1e-12 * (di + fabs(A[13 * N + j])))) atomicExch(asym, 1);
    }
}

cs_status check_symmetric(Level &L, cudaStream_t s) {
    L.sym32 = 0;
    if (L.g.dim != 3 || L.kind != BOX || L.bs != 1) return CS_OK;
    int *d = nullptr, asym = 1;
    CSX_TRY(dalloc_t(&d, 1, nullptr, s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_sym_check<<<node_grid(L.g), node_block(), 0, s>>>(L.g, L.A, d);
        count_launch();
        e = cudaMemcpyAsync(&asym, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "symmetry check", __FILE__, __LINE__);
    L.sym32 = asym ? 0 : 1;
    return CS_OK;
}

cs_status level_margin(Level &L, bool periodic, cudaStream_t s) {
    const Grid &g = L.g;
    const int64_t ref = g.nx / 2 + (int64_t)g.nx * (g.ny / 2 + (int64_t)g.ny * (g.nz / 2));
    int *d = nullptr;
    CSX_TRY(dalloc_t(&d, 1, nullptr, s));
    int init = -1, maxd = 0;
    cudaError_t e = cudaMemcpyAsync(d, &init, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_const_margin<<<node_grid(g), node_block(), 0, s>>>(g, L.nst, L.A, ref, d);
        count_launch();
        e = cudaMemcpyAsync(&maxd, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "level margin", __FILE__, __LINE__);
    if (periodic) L.margin = maxd < 0 ? 0 : Level::NO_MARGIN;
    else {
        L.margin = maxd + 1;
        if (bdist_host(g, g.nx / 2, g.ny / 2, g.nz / 2) < L.margin) L.margin = Level::NO_MARGIN;
    }
    return CS_OK;
}

// ------------------------------------------------------------ Galerkin RAP
// 1D interpolation weight between fine node 2J+1+u and coarse node J:
// 1 at u = 0, 1/2 at u = +-1, else 0.
__host__ __device__ constexpr double pw(int u) { return u == 0 ? 1.0 : ((u == 1 || u == -1) ? 0.5 : 0.0); }

// Ac_{I, I+dJ} = 2^-dim sum_{f,j} P_{f,I} A_{f,j} P_{j,I+dJ}, stored as a BOX
// stencil (dJ in {-1,0,1}^dim).  With f = 2I+1+d and j = f+s, A_s(f) enters
// entry dJ with weight prod_k pw(d_k) pw(d_k + s_k - 2 dJ_k); per axis
// u = d_k + s_k in [-2, 2] selects one coarse neighbour (u even) or two with
// weight 1/2 (u odd).  The 3^dim accumulators of a thread live in shared
// memory (registers would need dynamic indexing).  Couplings to nodes
// outside the grid carry zero coefficients (dropped when the fine operator
// is copied in, and zero by construction on Galerkin levels); fine nodes
// beyond the upper edge are skipped; entries whose coarse neighbour lies
// outside are set to zero.
template <int DIM, int KIND>
__global__ void __launch_bounds__(TBX *TBY) k_galerkin(Grid gf, Grid gc, const double *__restrict__ Af,
                                                        double *__restrict__ Ac, RowSet rs) {
    using S = StenS<DIM, KIND>;
    constexpr int NC = DIM == 3 ? 27 : 9;
    extern __shared__ double acc_sm[];  // [NC][TBX*TBY]
    const int tid = threadIdx.x + TBX * threadIdx.y;
    double *acc = acc_sm + tid;
#pragma unroll
    for (int t = 0; t < NC; ++t) acc[t * TBX * TBY] = 0.0;
    int cx, cy, cz;
    if (rs.on) {  // only coarse rows outside the deep box (plus the representative)
        if (!rowset_coord(rs, gc, (int64_t)blockIdx.x * (TBX * TBY) + tid, cx, cy, cz)) return;
    } else {
        cx = blockIdx.x * TBX + threadIdx.x; cy = blockIdx.y * TBY + threadIdx.y; cz = blockIdx.z;
        if (cx >= gc.nx || cy >= gc.ny) return;
    }
    const int64_t ci = cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz);
    for (int e = 0; e < NC; ++e) {
        const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = DIM == 3 ? e / 9 - 1 : 0;
        const int fx = 2 * cx + 1 + ex, fy = 2 * cy + 1 + ey, fz = DIM == 3 ? 2 * cz + 1 + ez : 0;
        if (fx >= gf.nx || fy >= gf.ny || (DIM == 3 && fz >= gf.nz)) continue;
        const int64_t fi = fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz);
        const double wr = pw(ex) * pw(ey) * pw(ez);
#pragma unroll
        for (int s = 0; s < S::NST; ++s) {
            int dx, dy, dz;
            S::off(s, dx, dy, dz);
            const double a = wr * Af[(int64_t)s * gf.N + fi];
            // per axis: target offsets j0 (weight w0) and, for odd u, j0+1
            const int ux = ex + dx, uy = ey + dy, uz = ez + dz;
            const int jx0 = (ux - 1) >> 1, jy0 = (uy - 1) >> 1, jz0 = (uz - 1) >> 1;  // floor((u-1)/2)
            const int nxj = (ux & 1) ? 2 : 1, nyj = (uy & 1) ? 2 : 1, nzj = DIM == 3 ? ((uz & 1) ? 2 : 1) : 1;
            const int bx = (ux & 1) ? jx0 : ux >> 1, by = (uy & 1) ? jy0 : uy >> 1, bz = (uz & 1) ? jz0 : uz >> 1;
            const double wx = (ux & 1) ? 0.5 : 1.0, wy = (uy & 1) ? 0.5 : 1.0, wz = (DIM == 3 && (uz & 1)) ? 0.5 : 1.0;
            const double awx = a * wx * wy * wz;
            for (int kz = 0; kz < nzj; ++kz)
                for (int ky = 0; ky < nyj; ++ky)
                    for (int kx = 0; kx < nxj; ++kx) {
                        const int t = (bx + kx + 1) + 3 * (by + ky + 1) + (DIM == 3 ? 9 * (bz + kz + 1) : 0);
                        acc[t * TBX * TBY] += awx;
                    }
        }
    }
    const double sc = DIM == 3 ? 0.125 : 0.25;
#pragma unroll
    for (int t = 0; t < NC; ++t) {
        const int jx = cx + t % 3 - 1, jy = cy + (t / 3) % 3 - 1, jz = DIM == 3 ? cz + t / 9 - 1 : 0;
        const bool in = jx >= 0 && jx < gc.nx && jy >= 0 && jy < gc.ny && (DIM == 2 || (jz >= 0 && jz < gc.nz));
        Ac[(int64_t)t * gc.N + ci] = in ? sc * acc[t * TBX * TBY] : 0.0;
    }
}

// The same product for levels of up to 16^3 coarse rows, one warp per
// (coarse row, stencil entry t) with the 3^dim fine neighbours e of the
// row's fine node on its lanes: each lane sums its neighbour's contributions
// to t over the fine stencil entries, and a fixed shuffle tree adds the
// lanes.  The row-per-thread kernel runs a row's 3^dim x nst contributions as
// one chain of dependent loads; on these levels that chain, not the data,
// set the launch time (about 0.4-0.5 ms per level from 16^3 down, against
// 28-300 us here).  On 32^3 and 64^3 levels the warps cost more than the
// chains (1.2 and 4.9 ms against 0.53 and 0.57 ms).  The summation order
// differs from the row-per-thread kernel's, so a level always takes the
// same kernel whether its deep rows are copied or not.
constexpr int64_t GALERKIN_WARP_MAX_ROWS = 16 * 16 * 16;
template <int DIM, int KIND>
__global__ void __launch_bounds__(256) k_galerkin_w(Grid gf, Grid gc, const double *__restrict__ Af,
                                                    double *__restrict__ Ac, RowSet rs, int64_t nrows) {
    using S = StenS<DIM, KIND>;
    constexpr int NC = DIM == 3 ? 27 : 9;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t row = w / NC;
    const int t = (int)(w - row * NC);
    if (row >= nrows) return;  // warp-uniform
    int cx, cy, cz;
    if (rs.on) {
        if (!rowset_coord(rs, gc, row, cx, cy, cz)) return;
    } else {
        cx = (int)(row % gc.nx);
        cy = (int)((row / gc.nx) % gc.ny);
        cz = (int)(row / ((int64_t)gc.nx * gc.ny));
    }
    const int64_t ci = cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz);
    const int tx = t % 3 - 1, ty = (t / 3) % 3 - 1, tz = DIM == 3 ? t / 9 - 1 : 0;
    const int jx = cx + tx, jy = cy + ty, jz = cz + tz;
    if (!(jx >= 0 && jx < gc.nx && jy >= 0 && jy < gc.ny && (DIM == 2 || (jz >= 0 && jz < gc.nz)))) {
        if (lane == 0) Ac[(int64_t)t * gc.N + ci] = 0.0;
        return;
    }
    double part = 0.0;
    if (lane < NC) {
        const int e = lane;
        const int ex = e % 3 - 1, ey = (e / 3) % 3 - 1, ez = DIM == 3 ? e / 9 - 1 : 0;
        const int fx = 2 * cx + 1 + ex, fy = 2 * cy + 1 + ey, fz = DIM == 3 ? 2 * cz + 1 + ez : 0;
        if (fx < gf.nx && fy < gf.ny && (DIM == 2 || fz < gf.nz)) {
            const int64_t fi = fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz);
            const double wr = pw(ex) * pw(ey) * pw(ez);
            // axis offset u = d + s reaches target offset tt: weight 1 (u even, tt = u / 2) or
            // 1/2 (u odd, tt one of the two coarse nodes around it); else 0
            auto wt = [](int u, int tt) {
                if (u & 1) {
                    const int j0 = (u - 1) >> 1;
                    return (tt == j0 || tt == j0 + 1) ? 0.5 : 0.0;
                }
                return tt == (u >> 1) ? 1.0 : 0.0;
            };
#pragma unroll
            for (int s2 = 0; s2 < S::NST; ++s2) {
                int dx, dy, dz;
                S::off(s2, dx, dy, dz);
                const double wx = wt(ex + dx, tx), wy = wt(ey + dy, ty), wz = DIM == 3 ? wt(ez + dz, tz) : 1.0;
                if (wx != 0.0 && wy != 0.0 && wz != 0.0) part += wr * Af[(int64_t)s2 * gf.N + fi] * wx * wy * wz;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if (lane == 0) Ac[(int64_t)t * gc.N + ci] = (DIM == 3 ? 0.125 : 0.25) * part;
}

// rows inside the deep box take the representative row's values
__global__ void k_copy_deep(Grid g, int nv, double *__restrict__ V, RowSet rs, int colour) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    if (ix < rs.lo[0] || ix > rs.hi[0] || iy < rs.lo[1] || iy > rs.hi[1]) return;
    if (g.dim == 3 && (iz < rs.lo[2] || iz > rs.hi[2])) return;
    const int c = rb_colour(g, ix, iy, iz);
    if (colour >= 0 && c != colour) return;
    const int r = rs.nrep == 2 ? c : 0;  // representative of this row's colour
    const int64_t ri = rs.rep[r][0] + (int64_t)g.nx * (rs.rep[r][1] + (int64_t)g.ny * rs.rep[r][2]);
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    if (i == ri) return;
    for (int t = 0; t < nv; ++t) V[(int64_t)t * g.N + i] = V[(int64_t)t * g.N + ri];
}

cs_status galerkin_level(const Level &f, Level &c, bool reuse, cudaStream_t s) {
    dim3 gr = node_grid(c.g), bl = node_block();
    // fine rows at distance >= margin repeat the centre row; a coarse row I is
    // deep when its fine neighbourhood (radius 1 around 2I+1) lies there and
    // all its coarse neighbours exist: per axis lo <= I <= hi with
    // 2I >= margin, 2I + 2 <= nf - 1 - margin, and 1 <= I <= nc - 2
    RowSet rs{};
    if (reuse && f.margin < Level::NO_MARGIN) {
        const int nf[3] = {f.g.nx, f.g.ny, f.g.nz}, nc[3] = {c.g.nx, c.g.ny, c.g.nz};
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            if (d == 2 && c.g.dim == 2) { rs.lo[2] = rs.hi[2] = 0; continue; }
            rs.lo[d] = std::max(1, (f.margin + 1) / 2);
            rs.hi[d] = std::min(nc[d] - 2, (nf[d] - 3 - f.margin) / 2);
            const int cc = nc[d] / 2;
            if (rs.lo[d] > cc || rs.hi[d] < cc) ok = false;  // the centre must be deep
        }
        if (ok) {
            rs.on = 1;
            rs.nrep = 1;
            rs.rep[0][0] = c.g.nx / 2; rs.rep[0][1] = c.g.ny / 2; rs.rep[0][2] = c.g.dim == 3 ? c.g.nz / 2 : 0;
            rs.nshell = rowset_shell_count(c.g, rs.lo, rs.hi);
            gr = dim3((unsigned)((rs.nshell + rs.nrep + TBX * TBY - 1) / (TBX * TBY)), 1, 1);
            bl = dim3(TBX * TBY, 1, 1);
        }
    }
    if (c.g.N <= GALERKIN_WARP_MAX_ROWS) {  // by level size, so that reuse does not change the kernel
        const int64_t nrows = rs.on ? rs.nshell + rs.nrep : c.g.N;
        const int nc = c.g.dim == 3 ? 27 : 9;
        const unsigned nb = (unsigned)((nrows * nc * 32 + 255) / 256);
        if (f.g.dim == 2) {
            if (f.kind == STAR) k_galerkin_w<2, STAR><<<nb, 256, 0, s>>>(f.g, c.g, f.A, c.A, rs, nrows);
            else k_galerkin_w<2, BOX><<<nb, 256, 0, s>>>(f.g, c.g, f.A, c.A, rs, nrows);
        } else {
            if (f.kind == STAR) k_galerkin_w<3, STAR><<<nb, 256, 0, s>>>(f.g, c.g, f.A, c.A, rs, nrows);
            else k_galerkin_w<3, BOX><<<nb, 256, 0, s>>>(f.g, c.g, f.A, c.A, rs, nrows);
        }
        CSX_CUDA(cudaGetLastError());
        count_launch();
        if (rs.on) {
            k_copy_deep<<<node_grid(c.g), node_block(), 0, s>>>(c.g, c.nst, c.A, rs, -1);
            CSX_CUDA(cudaGetLastError());
            count_launch();
        }
        return CS_OK;
    }
    const size_t sm2 = sizeof(double) * 9 * TBX * TBY, sm3 = sizeof(double) * 27 * TBX * TBY;
    if (f.g.dim == 2) {
        if (f.kind == STAR) k_galerkin<2, STAR><<<gr, bl, sm2, s>>>(f.g, c.g, f.A, c.A, rs);
        else k_galerkin<2, BOX><<<gr, bl, sm2, s>>>(f.g, c.g, f.A, c.A, rs);
    } else {
        // 27 x 256 doubles = 54 KB exceeds the default 48 KB (set per call: the attribute is per device)
        CSX_CUDA(cudaFuncSetAttribute(k_galerkin<3, STAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
        CSX_CUDA(cudaFuncSetAttribute(k_galerkin<3, BOX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
        if (f.kind == STAR) k_galerkin<3, STAR><<<gr, bl, sm3, s>>>(f.g, c.g, f.A, c.A, rs);
        else k_galerkin<3, BOX><<<gr, bl, sm3, s>>>(f.g, c.g, f.A, c.A, rs);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    if (rs.on) {
        k_copy_deep<<<node_grid(c.g), node_block(), 0, s>>>(c.g, c.nst, c.A, rs, -1);
        CSX_CUDA(cudaGetLastError());
        count_launch();
    }
    return CS_OK;
}

// ------------------------------------------------- coarsest factorisation
__global__ void k_assemble_dense(Grid g, int nst, const int *__restrict__ offs, const double *__restrict__ A,
                                 double *__restrict__ M) {
    int64_t n = g.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((int64_t)g.nx * g.ny));
        for (int j = 0; j < n; ++j) M[i * n + j] = 0.0;
        for (int s = 0; s < nst; ++s) {
            int jx = ix + offs[3 * s], jy = iy + offs[3 * s + 1], jz = iz + offs[3 * s + 2];
            if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny || jz < 0 || jz >= g.nz) continue;
            int64_t j = jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz);
            M[i * n + j] += A[(int64_t)s * n + i];
        }
    }
}

// Single-CTA dense factorisation and inverse (Algorithm 1's bottom-level
// direct solve): Cholesky when M is symmetric to 1e-14 of its largest entry
// and every pivot is positive, else LU with partial pivoting (the Cholesky
// loop reads only the lower triangle, so it would solve another matrix when
// M is not symmetric).  Launched with 256 threads.  status[0] = 0 ok,
// 1 singular.
__global__ void k_factor_inverse(int n, double *M, double *W, double *Inv, int *piv, int *status) {
    __shared__ int bad;
    __shared__ int spd;
    __shared__ double red_max[256], red_asym[256];
    int tid = threadIdx.x, nt = blockDim.x;
    double amax = 0.0, asym = 0.0;
    for (int64_t t = tid; t < (int64_t)n * n; t += nt) {
        W[t] = M[t];
        int i = (int)(t / n), j = (int)(t % n);
        amax = fmax(amax, fabs(M[t]));
        asym = fmax(asym, fabs(M[t] - M[(int64_t)j * n + i]));
    }
    red_max[tid] = amax;
    red_asym[tid] = asym;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (tid < w) {
            red_max[tid] = fmax(red_max[tid], red_max[tid + w]);
            red_asym[tid] = fmax(red_asym[tid], red_asym[tid + w]);
        }
        __syncthreads();
    }
    if (tid == 0) { bad = 0; spd = red_asym[0] <= 1e-14 * red_max[0]; }
    __syncthreads();
    for (int k = 0; k < n && spd; ++k) {  // right-looking Cholesky on W (lower)
        if (tid == 0) {
            double d = W[(int64_t)k * n + k];
            if (!(d > 0.0)) spd = 0;
            else W[(int64_t)k * n + k] = sqrt(d);
        }
        __syncthreads();
        if (!spd) break;
        double dk = W[(int64_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) W[(int64_t)i * n + k] /= dk;
        __syncthreads();
        for (int64_t t = tid; t < (int64_t)(n - k - 1) * (n - k - 1); t += nt) {
            int i = k + 1 + (int)(t / (n - k - 1)), j = k + 1 + (int)(t % (n - k - 1));
            if (j <= i) W[(int64_t)i * n + j] -= W[(int64_t)i * n + k] * W[(int64_t)j * n + k];
        }
        __syncthreads();
    }
    __syncthreads();
    if (spd) {
        for (int c = tid; c < n; c += nt) {  // column c of the inverse: L L^T y = e_c
            for (int i = 0; i < n; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) s -= W[(int64_t)i * n + k] * Inv[(int64_t)k * n + c];
                Inv[(int64_t)i * n + c] = s / W[(int64_t)i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = Inv[(int64_t)i * n + c];
                for (int k = i + 1; k < n; ++k) s -= W[(int64_t)k * n + i] * Inv[(int64_t)k * n + c];
                Inv[(int64_t)i * n + c] = s / W[(int64_t)i * n + i];
            }
        }
        if (tid == 0) status[0] = 0;
        return;
    }
    // LU with partial pivoting
    for (int64_t t = tid; t < (int64_t)n * n; t += nt) W[t] = M[t];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            int p = k;
            double best = fabs(W[(int64_t)k * n + k]);
            for (int i = k + 1; i < n; ++i)
                if (fabs(W[(int64_t)i * n + k]) > best) { best = fabs(W[(int64_t)i * n + k]); p = i; }
            piv[k] = p;
            if (best == 0.0) bad = 1;
        }
        __syncthreads();
        if (bad) break;
        int p = piv[k];
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                double t = W[(int64_t)k * n + j];
                W[(int64_t)k * n + j] = W[(int64_t)p * n + j];
                W[(int64_t)p * n + j] = t;
            }
        __syncthreads();
        double dk = W[(int64_t)k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) W[(int64_t)i * n + k] /= dk;
        __syncthreads();
        for (int64_t t = tid; t < (int64_t)(n - k - 1) * (n - k - 1); t += nt) {
            int i = k + 1 + (int)(t / (n - k - 1)), j = k + 1 + (int)(t % (n - k - 1));
            W[(int64_t)i * n + j] -= W[(int64_t)i * n + k] * W[(int64_t)k * n + j];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) status[0] = 1;
        return;
    }
    for (int c = tid; c < n; c += nt) {
        for (int i = 0; i < n; ++i) Inv[(int64_t)i * n + c] = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k) {
            int p = piv[k];
            if (p != k) {
                double t = Inv[(int64_t)k * n + c];
                Inv[(int64_t)k * n + c] = Inv[(int64_t)p * n + c];
                Inv[(int64_t)p * n + c] = t;
            }
        }
        for (int i = 0; i < n; ++i) {
            double s = Inv[(int64_t)i * n + c];
            for (int k = 0; k < i; ++k) s -= W[(int64_t)i * n + k] * Inv[(int64_t)k * n + c];
            Inv[(int64_t)i * n + c] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = Inv[(int64_t)i * n + c];
            for (int k = i + 1; k < n; ++k) s -= W[(int64_t)i * n + k] * Inv[(int64_t)k * n + c];
            Inv[(int64_t)i * n + c] = s / W[(int64_t)i * n + i];
        }
    }
    if (tid == 0) status[0] = 0;
}

cs_status coarse_factor(cs_hierarchy *h, cudaStream_t s) {
    const Level &L = h->lev[h->nlev - 1];
    int n = (int)L.g.N;
    h->cn = n;
    double *M = nullptr, *W = nullptr;
    int *piv = nullptr, *st = nullptr, *offs = nullptr;
    CSX_TRY(dalloc_t(&h->cinv, (size_t)n * n, &h->bytes, s));
    cs_status rc = CS_OK;
    int offh[81];
    for (int t = 0; t < L.nst; ++t)
        for (int d = 0; d < 3; ++d) offh[3 * t + d] = L.off[t][d];
    int sth = 0;
    if ((rc = dalloc_t(&M, (size_t)n * n, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&W, (size_t)n * n, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&piv, (size_t)n + 1, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&st, 1, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&offs, 81, nullptr, s)) != CS_OK) goto done;
    if (cudaMemcpyAsync(offs, offh, sizeof(int) * 3 * L.nst, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "copy offsets", __FILE__, __LINE__);
        goto done;
    }
    k_assemble_dense<<<64, 256, 0, s>>>(L.g, L.nst, offs, L.A, M);
    k_factor_inverse<<<1, 256, 0, s>>>(n, M, W, h->cinv, piv, st);
    count_launch(2);
    if (cudaMemcpyAsync(&sth, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "coarse factorisation", __FILE__, __LINE__);
        goto done;
    }
    if (sth != 0) {
        set_error("coarsest-level matrix (%d x %d) is singular", n, n);
        rc = CS_ERR_SINGULAR;
    }
done:
    dfree(M, s); dfree(W, s); dfree(piv, s); dfree(st, s); dfree(offs, s);
    return rc;
}

// ------------------------------------------------------------ cascade setup
// w_i = A_ii^{-1/2}; A~_s(i) = w_i A_s(i) w_{i+s}; bad[0] set if A_ii <= 0
template <int DIM, int KIND>
__global__ void k_prescale(Grid g, int periodic, int prescale, const double *__restrict__ A, double *__restrict__ w,
                           double *__restrict__ At, int *bad) {
    using S = StenS<DIM, KIND>;
    const int C = KIND == STAR ? 0 : (DIM == 3 ? 13 : 4);
    int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    double d = A[(int64_t)C * g.N + i];
    if (prescale && !(d > 0.0)) atomicExch(bad, 1);
    w[i] = prescale ? 1.0 / sqrt(d) : 1.0;
    (void)periodic;
    (void)At;
}

template <int DIM, int KIND, typename W = double>
__global__ void k_scale_op(Grid g, int periodic, const double *__restrict__ A, const double *__restrict__ w,
                           W *__restrict__ At) {
    using S = StenS<DIM, KIND>;
    int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    double wi = w[i];
#pragma unroll
    for (int s = 0; s < S::NST; ++s) {
        int dx, dy, dz;
        S::off(s, dx, dy, dz);
        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        bool in;
        if (periodic) {
            jx = (jx + g.nx) % g.nx; jy = (jy + g.ny) % g.ny; jz = DIM == 3 ? (jz + g.nz) % g.nz : 0;
            in = true;
        } else {
            in = jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny && (DIM == 2 || (jz >= 0 && jz < g.nz));
        }
        double v = 0.0;
        if (in) v = wi * A[(int64_t)s * g.N + i] * w[jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz)];
        At[(int64_t)s * g.N + i] = (W)v;
    }
}

template <typename W>
__global__ void k_fill(int64_t n, W *p, W v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// Reuse of repeated rows in a setup step (see "repeated-row detection"):
// rows at boundary distance >= d_now are deep after this step, rows at
// distance >= d_prev were deep before it (their E_cur rows are stored only
// in the representatives rep0 / rep1 of red / black).
struct Reuse {
    int on;
    int d_now, d_prev;
    int rep0, rep1;
};

// One setup step (l, k) over rows and a chunk of output offsets o'.
// For every o' the host supplies the list of valid pairs (s, c) -- stencil
// entry s and index c in O_cur of o' - off(s) -- packed as (s << 24) | c in
// pairs[pstart[o'] .. pstart[o'+1]), plus cur_of[o'] (index of o' in O_cur or
// -1).  Only valid pairs issue an FP64 FMA (on GB300 the FP64 pipe is the
// bound of this kernel).  The row's prescaled coefficients and neighbour
// indices sit in shared memory so that s can be a run-time index; a
// neighbour outside the grid carries a zero coefficient and is read at the
// row itself.  nchunks == 1: the thread finishes the row (lambda, residual
// update); otherwise partial <E_i,R_i>, <R_i,R_i> go to part[q*N + i] and
// k_setup_finish completes the row.  LAST: the final step of the cascade,
// where E_nu is not needed -- R is neither stored nor used to update E.
template <int DIM, int KIND, bool LAST, typename W = double>
__global__ void __launch_bounds__(TBX *TBY) k_setup_rows(Grid g, int periodic, const W *__restrict__ At,
                                                          const double *__restrict__ w, const W *__restrict__ Ecur,
                                                          W *__restrict__ Enxt, int nnxt, int chunk, int nchunks,
                                                          const int *__restrict__ pstart,
                                                          const unsigned *__restrict__ pairs,
                                                          const int *__restrict__ cur_of, int colour,
                                                          double *__restrict__ lam, double2 *__restrict__ part,
                                                          Reuse ru, RowSet rs) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    constexpr int NT = TBX * TBY;
    extern __shared__ double sm_setup[];
    W *sa = reinterpret_cast<W *>(sm_setup);                 // [NST][NT]
    int *snb = reinterpret_cast<int *>(sa + NST * NT);       // [NST][NT]
    const int tid = threadIdx.x + TBX * threadIdx.y;
    int ix, iy, iz, q;
    if (rs.on) {  // shell rows and representatives only, packed densely
        q = blockIdx.y;
        if (!rowset_coord(rs, g, (int64_t)blockIdx.x * NT + tid, ix, iy, iz)) return;
    } else {
        ix = blockIdx.x * TBX + threadIdx.x; iy = blockIdx.y * TBY + threadIdx.y;
        iz = (int)(blockIdx.z % (unsigned)g.nz); q = (int)(blockIdx.z / (unsigned)g.nz);
        if (ix >= g.nx || iy >= g.ny) return;
    }
    const int64_t N = g.N;
    const int i = ix + g.nx * (iy + g.ny * iz);
    const int o0 = q * chunk, o1 = min(nnxt, o0 + chunk);
    const int cme = rb_colour(g, ix, iy, iz);
    const bool active = colour < 0 || cme == colour;
    const int dist = periodic ? (1 << 30) : bdist(g, ix, iy, iz);
    const int repme = cme ? ru.rep1 : ru.rep0;
    if (ru.on && dist >= ru.d_now && i != repme) return;  // deep row: copied from its representative
    const int iread = (ru.on && dist >= ru.d_prev) ? repme : i;  // where this row's E_cur is stored
    if (!active) {
        if (!LAST)
            for (int o = o0; o < o1; ++o) {
                int c = __ldg(cur_of + o);
                Enxt[(int64_t)o * N + i] = c >= 0 ? Ecur[(int64_t)c * N + iread] : W(0);
            }
        return;
    }
#pragma unroll
    for (int s = 0; s < NST; ++s) {
        int dx, dy, dz;
        S::off(s, dx, dy, dz);
        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        bool in;
        if (periodic) {
            jx = (jx + g.nx) % g.nx; jy = (jy + g.ny) % g.ny; jz = DIM == 3 ? (jz + g.nz) % g.nz : 0;
            in = true;
        } else {
            in = jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny && (DIM == 2 || (jz >= 0 && jz < g.nz));
        }
        int j = in ? jx + g.nx * (jy + g.ny * jz) : iread;
        if (in && ru.on && (periodic || bdist(g, jx, jy, jz) >= ru.d_prev))
            j = rb_colour(g, jx, jy, jz) ? ru.rep1 : ru.rep0;
        snb[s * NT + tid] = j;
        sa[s * NT + tid] = in ? At[(int64_t)s * N + i] : W(0);
    }
    // <E_i, R_i> and <R_i, R_i>: in FP64, or (W = float) in FP32 over
    // chunks of 8 offsets whose sums are added in FP64
    constexpr bool CH = sizeof(W) < sizeof(double);
    double num = 0.0, den = 0.0;
    W cnum = W(0), cden = W(0);
    int p = __ldg(pstart + o0);
    for (int o = o0; o < o1; ++o) {
        const int pe = __ldg(pstart + o + 1);
        W r = W(0);
        for (; p < pe; ++p) {
            const unsigned u = __ldg(pairs + p);
            const int s = (int)(u >> 24), c = (int)(u & 0xffffffu);
            r = fma(sa[s * NT + tid], Ecur[(int64_t)c * N + snb[s * NT + tid]], r);
        }
        const int c0 = __ldg(cur_of + o);
        if (CH) {
            if (c0 >= 0) cnum = fma(Ecur[(int64_t)c0 * N + iread], r, cnum);
            cden = fma(r, r, cden);
            if (((o - o0) & 7) == 7) {
                num += (double)cnum;
                den += (double)cden;
                cnum = W(0);
                cden = W(0);
            }
        } else {
            if (c0 >= 0) num = fma((double)Ecur[(int64_t)c0 * N + iread], (double)r, num);
            den = fma((double)r, (double)r, den);
        }
        if (!LAST) Enxt[(int64_t)o * N + i] = r;
    }
    if (CH) {
        num += (double)cnum;
        den += (double)cden;
    }
    if (nchunks > 1) {
        part[(int64_t)q * N + i] = make_double2(num, den);
        return;
    }
    // normal equations of the 1 x 1 least-squares problem; a zero row R_i
    // (pivot <= 1e-14 tr(G) = 0) gives the minimum-norm solution 0
    const double lt = den > 0.0 ? num / den : 0.0;
    if (!LAST) {
        const W ltw = (W)lt;
        for (int o = o0; o < o1; ++o) {
            const int c0 = __ldg(cur_of + o);
            const W e = c0 >= 0 ? Ecur[(int64_t)c0 * N + iread] : W(0);
            Enxt[(int64_t)o * N + i] = e - ltw * Enxt[(int64_t)o * N + i];
        }
    }
    const double wi = w[i];
    lam[i] = wi * lt * wi;
}

// Completes rows processed in several chunks: sums the partial inner
// products in chunk order, forms lambda and (unless LAST) updates this
// chunk's entries of E.
template <int DIM, bool LAST, typename W = double>
__global__ void __launch_bounds__(TBX *TBY) k_setup_finish(Grid g, const double *__restrict__ w,
                                                            const W *__restrict__ Ecur, W *__restrict__ Enxt,
                                                            int nnxt, int chunk, int nchunks,
                                                            const int *__restrict__ cur_of, int colour,
                                                            double *__restrict__ lam, const double2 *__restrict__ part,
                                                            int periodic, Reuse ru, RowSet rs) {
    int ix, iy, iz, q;
    if (rs.on) {
        q = blockIdx.y;
        if (!rowset_coord(rs, g, (int64_t)blockIdx.x * (TBX * TBY) + threadIdx.x + TBX * threadIdx.y, ix, iy, iz))
            return;
    } else {
        ix = blockIdx.x * TBX + threadIdx.x; iy = blockIdx.y * TBY + threadIdx.y;
        iz = (int)(blockIdx.z % (unsigned)g.nz); q = (int)(blockIdx.z / (unsigned)g.nz);
        if (ix >= g.nx || iy >= g.ny) return;
    }
    const int cme = rb_colour(g, ix, iy, iz);
    const bool active = colour < 0 || cme == colour;
    if (!active) return;
    const int64_t N = g.N;
    const int i = ix + g.nx * (iy + g.ny * iz);
    const int dist = periodic ? (1 << 30) : bdist(g, ix, iy, iz);
    const int repme = cme ? ru.rep1 : ru.rep0;
    if (ru.on && dist >= ru.d_now && i != repme) return;
    const int iread = (ru.on && dist >= ru.d_prev) ? repme : i;
    double num = 0.0, den = 0.0;
    for (int t = 0; t < nchunks; ++t) {
        double2 p = part[(int64_t)t * N + i];
        num += p.x;
        den += p.y;
    }
    const double lt = den > 0.0 ? num / den : 0.0;
    if (q == 0) lam[i] = w[i] * lt * w[i];
    if (LAST) return;
    const W ltw = (W)lt;
    const int o0 = q * chunk, o1 = min(nnxt, o0 + chunk);
    for (int o = o0; o < o1; ++o) {
        const int c0 = __ldg(cur_of + o);
        const W e = c0 >= 0 ? Ecur[(int64_t)c0 * N + iread] : W(0);
        Enxt[(int64_t)o * N + i] = e - ltw * Enxt[(int64_t)o * N + i];
    }
}


template <int DIM, int KIND, bool LAST, typename W>
static cs_status launch_setup_rows(const Grid &g, int periodic, const W *At, const double *w,
                                   const W *Ecur, W *Enxt, int nn, int chunk, int nchunks,
                                   const int *pstart, const unsigned *pairs, const int *cur_of, int colour,
                                   double *lam, double2 *part, const Reuse &ru, const RowSet &rs, cudaStream_t s) {
    dim3 gr = node_grid(g), bl = node_block();
    gr.z *= nchunks;
    if (rs.on) {
        gr = dim3((unsigned)((rs.nshell + rs.nrep + TBX * TBY - 1) / (TBX * TBY)), (unsigned)nchunks, 1);
        bl = dim3(TBX * TBY, 1, 1);
    }
    const size_t smem = (size_t)StenS<DIM, KIND>::NST * TBX * TBY * (sizeof(W) + sizeof(int));
    // up to 27 x 256 x 12 B = 81 KB: above the default 48 KB (set per call: the attribute is per device)
    CSX_CUDA(cudaFuncSetAttribute(k_setup_rows<DIM, KIND, LAST, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_setup_rows<DIM, KIND, LAST, W><<<gr, bl, smem, s>>>(g, periodic, At, w, Ecur, Enxt, nn, chunk, nchunks,
                                                          pstart, pairs, cur_of, colour, lam, part, ru, rs);
    count_launch();
    if (nchunks > 1) {
        k_setup_finish<DIM, LAST, W><<<gr, bl, 0, s>>>(g, w, Ecur, Enxt, nn, chunk, nchunks, cur_of, colour, lam,
                                                       part, periodic, ru, rs);
        count_launch();
    }
    if (rs.on) {  // deep rows of the active colour take their representative's lambda
        k_copy_deep<<<node_grid(g), node_block(), 0, s>>>(g, 1, lam, rs, colour);
        count_launch();
    }
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

struct Off3 {
    int x, y, z;
    bool operator<(const Off3 &o) const { return std::tie(z, y, x) < std::tie(o.z, o.y, o.x); }
    bool operator==(const Off3 &o) const { return x == o.x && y == o.y && z == o.z; }
};

// Truncation of the updated rows (Algorithm 2, optional step): a row of the
// step's colour keeps the alpha columns of largest |E_ij| -- ties go to the
// smaller column index -- and the others are set to zero.  Candidates are the
// row's offsets whose column lies in the grid (wrapped on periodic grids).
// The alpha-th largest (value, column) pair is found by alpha passes of
// "largest after the previous one", then one pass zeroes what ranks below it.
template <int DIM, typename W = double>
__global__ void __launch_bounds__(TBX *TBY) k_truncate_rows(Grid g, int periodic, int nn, const int *__restrict__ off,
                                                             W *__restrict__ E, int alpha, int colour) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    if (colour >= 0 && (((ix + 1) + (iy + 1) + (DIM == 3 ? iz + 1 : 0)) & 1) != colour) return;
    const int64_t N = g.N;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    auto column = [&](int o, int64_t &j) {
        int jx = ix + off[3 * o], jy = iy + off[3 * o + 1], jz = DIM == 3 ? iz + off[3 * o + 2] : 0;
        if (periodic) {
            jx = ((jx % g.nx) + g.nx) % g.nx;
            jy = ((jy % g.ny) + g.ny) % g.ny;
            jz = DIM == 3 ? ((jz % g.nz) + g.nz) % g.nz : 0;
        } else if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny || (DIM == 3 && (jz < 0 || jz >= g.nz))) {
            return false;
        }
        j = jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz);
        return true;
    };
    double tn = INFINITY;  // threshold pair (tn, tc): the last one selected
    int64_t tc = -1;
    bool full = true;  // alpha pairs found
    for (int a = 0; a < alpha; ++a) {
        double bn = -1.0;
        int64_t bc = 0;
        for (int o = 0; o < nn; ++o) {
            int64_t j;
            if (!column(o, j)) continue;
            const double v = (double)E[(int64_t)o * N + i], n = v * v;
            const bool after = n < tn || (n == tn && j > tc);
            if (after && (n > bn || (n == bn && j < bc))) { bn = n; bc = j; }
        }
        if (bn < 0.0) { full = false; break; }
        tn = bn;
        tc = bc;
    }
    if (!full) return;  // no more candidates than alpha: all kept
    for (int o = 0; o < nn; ++o) {
        int64_t j;
        if (!column(o, j)) continue;
        const double v = (double)E[(int64_t)o * N + i], n = v * v;
        if (!(n > tn || (n == tn && j <= tc))) E[(int64_t)o * N + i] = 0.0;
    }
}

template <int DIM, int KIND, typename W>
static cs_status setup_level_t(const cs_hierarchy *h, int l, int kind, int nu, int prescale, bool reuse, int alpha,
                               double *lam, cudaStream_t s, int64_t *peak) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    const Level &L = h->lev[l];
    const Grid g = L.g;
    const int64_t N = g.N;
    const int ncol = kind == CS_MULTIPLICATIVE ? 2 : 1;
    dim3 gr = node_grid(g), bl = node_block();
    double *w = nullptr;
    W *At = nullptr, *Ecur = nullptr, *Enxt = nullptr;
    int *bad = nullptr, *pstart = nullptr, *cur_of = nullptr, *offs = nullptr;
    unsigned *pairs = nullptr;
    double2 *part = nullptr;
    cs_status rc = CS_OK;
    int badh = 0;
    std::vector<Off3> Ocur{{0, 0, 0}};
    int64_t live = 0, pk = 0;
    auto track = [&](int64_t d) { live += d; pk = std::max(pk, live); };
    Reuse ru{0, 0, 0, 0, 0};

    if ((rc = dalloc_t(&w, N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&At, (size_t)NST * N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&bad, 1, nullptr, s)) != CS_OK) goto done;
    track((int64_t)NST * N * sizeof(W) + N * 8);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); goto done; }
    k_prescale<DIM, KIND><<<gr, bl, 0, s>>>(g, h->periodic, prescale, L.A, w, static_cast<double *>(nullptr), bad);
    count_launch();
    if (cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "prescale", __FILE__, __LINE__);
        goto done;
    }
    if (badh) {
        set_error("level %d: non-positive diagonal entry; elliptic prescaling needs A_ii > 0", l);
        rc = CS_ERR_ARG;
        goto done;
    }
    k_scale_op<DIM, KIND, W><<<gr, bl, 0, s>>>(g, h->periodic, L.A, w, At);
    count_launch();
    if ((rc = dalloc_t(&Ecur, N, nullptr, s)) != CS_OK) goto done;
    track(N * (int64_t)sizeof(W));
    k_fill<W><<<1216, 256, 0, s>>>(N, Ecur, W(1));
    count_launch();

    // representatives: the grid centre and its +x neighbour (the other colour)
    {
        const int cx = g.nx / 2, cy = g.ny / 2, cz = DIM == 3 ? g.nz / 2 : 0;
        const int ci = cx + g.nx * (cy + g.ny * cz);
        const int cc = ((cx + 1) + (cy + 1) + (DIM == 3 ? cz + 1 : 0)) & 1;
        const int steps = nu * ncol;
        const bool deep_enough = h->periodic ? true : bdist_host(g, cx, cy, cz) - 1 >= L.margin + steps;
        if (reuse && L.margin < Level::NO_MARGIN && deep_enough && cx + 1 < g.nx) {
            ru.on = 1;
            if (ncol == 1) {  // additive: all deep rows repeat one row, whatever their colour
                ru.rep0 = ru.rep1 = ci;
            } else {
                ru.rep0 = cc == 0 ? ci : ci + 1;
                ru.rep1 = cc == 0 ? ci + 1 : ci;
            }
        }
    }
    for (int lev = 0; lev < nu; ++lev) {
        for (int k = 0; k < ncol; ++k) {
            const int t = lev * ncol + k + 1;  // flattened step number
            ru.d_now = L.margin + t;
            ru.d_prev = L.margin + t - 1;
            RowSet rs{};
            if (ru.on) {
                rs.on = 1;
                const int nn3[3] = {g.nx, g.ny, g.nz};
                for (int d = 0; d < 3; ++d) {
                    if (d == 2 && DIM == 2) { rs.lo[2] = rs.hi[2] = 0; continue; }
                    rs.lo[d] = h->periodic ? 0 : ru.d_now;
                    rs.hi[d] = h->periodic ? nn3[d] - 1 : nn3[d] - 1 - ru.d_now;
                }
                rs.nshell = rowset_shell_count(g, rs.lo, rs.hi);
                rs.nrep = ncol;
                for (int c = 0; c < ncol; ++c) {
                    const int ri = c == 0 ? ru.rep0 : ru.rep1;
                    rs.rep[c][0] = ri % g.nx;
                    rs.rep[c][1] = (ri / g.nx) % g.ny;
                    rs.rep[c][2] = ri / (g.nx * g.ny);
                }
            }
            // O_next = O_cur + S
            std::vector<Off3> On;
            for (const Off3 &o : Ocur)
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    On.push_back({o.x + dx, o.y + dy, o.z + dz});
                }
            std::sort(On.begin(), On.end());
            On.erase(std::unique(On.begin(), On.end()), On.end());
            if (h->periodic) {
                int rx = 0, ry = 0, rz = 0;
                for (const Off3 &o : On) { rx = std::max(rx, std::abs(o.x)); ry = std::max(ry, std::abs(o.y)); rz = std::max(rz, std::abs(o.z)); }
                if (2 * rx >= g.nx || 2 * ry >= g.ny || (DIM == 3 && 2 * rz >= g.nz)) {
                    set_error("periodic grid too small for the fill-in of this cascade (side must exceed twice the fill radius)");
                    rc = CS_ERR_UNSUPPORTED;
                    goto done;
                }
            }
            std::map<Off3, int> idx;
            for (size_t t = 0; t < Ocur.size(); ++t) idx[Ocur[t]] = (int)t;
            const int nn = (int)On.size();
            std::vector<int> hps(nn + 1, 0), hc(nn);
            std::vector<unsigned> hpairs;
            for (int o = 0; o < nn; ++o) {
                auto it = idx.find(On[o]);
                hc[o] = it == idx.end() ? -1 : it->second;
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    auto jt = idx.find({On[o].x - dx, On[o].y - dy, On[o].z - dz});
                    if (jt != idx.end()) hpairs.push_back(((unsigned)t << 24) | (unsigned)jt->second);
                }
                hps[o + 1] = (int)hpairs.size();
            }
            const bool last = lev == nu - 1 && k == ncol - 1;
            // parallelism for small levels: split each row's offsets into chunks
            int nchunks = (int)std::min<int64_t>((524288 + N - 1) / N, (nn + 3) / 4);
            nchunks = std::max(1, std::min(nchunks, 65535 / std::max(1, g.nz)));
            const int chunk = (nn + nchunks - 1) / nchunks;
            nchunks = (nn + chunk - 1) / chunk;
            dfree(pstart, s); dfree(cur_of, s); dfree(pairs, s); dfree(part, s);
            pstart = nullptr; cur_of = nullptr; pairs = nullptr; part = nullptr;
            if ((rc = dalloc_t(&pstart, hps.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&cur_of, hc.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&pairs, hpairs.size(), nullptr, s)) != CS_OK) goto done;
            if (nchunks > 1 && (rc = dalloc_t(&part, (size_t)nchunks * N, nullptr, s)) != CS_OK) goto done;
            if (cudaMemcpyAsync(pstart, hps.data(), hps.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(cur_of, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(pairs, hpairs.data(), hpairs.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "copy setup tables", __FILE__, __LINE__);
                goto done;
            }
            if (!last) {
                if ((rc = dalloc_t(&Enxt, (size_t)nn * N, nullptr, s)) != CS_OK) goto done;
                track((int64_t)nn * N * (int64_t)sizeof(W));
            }
            {
                const int colour = ncol == 2 ? k : -1;
                double *lam_l = lam + (int64_t)lev * N;
                rc = last ? launch_setup_rows<DIM, KIND, true, W>(g, h->periodic, At, w, Ecur, Enxt, nn, chunk, nchunks,
                                                               pstart, pairs, cur_of, colour, lam_l, part, ru, rs, s)
                          : launch_setup_rows<DIM, KIND, false, W>(g, h->periodic, At, w, Ecur, Enxt, nn, chunk, nchunks,
                                                                pstart, pairs, cur_of, colour, lam_l, part, ru, rs, s);
                if (rc != CS_OK) goto done;
            }
            if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "k_setup_rows", __FILE__, __LINE__); goto done; }
            if (alpha > 0 && !last) {
                std::vector<int> ho(3 * (size_t)nn);
                for (int o = 0; o < nn; ++o) { ho[3 * o] = On[o].x; ho[3 * o + 1] = On[o].y; ho[3 * o + 2] = On[o].z; }
                dfree(offs, s);
                offs = nullptr;
                if ((rc = dalloc_t(&offs, ho.size(), nullptr, s)) != CS_OK) goto done;
                if (cudaMemcpyAsync(offs, ho.data(), ho.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                    rc = cuda_fail(cudaGetLastError(), "copy offsets", __FILE__, __LINE__);
                    goto done;
                }
                k_truncate_rows<DIM, W><<<gr, bl, 0, s>>>(g, h->periodic, nn, offs, Enxt, alpha, ncol == 2 ? k : -1);
                count_launch();
                if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "k_truncate_rows", __FILE__, __LINE__); goto done; }
            }
            dfree(Ecur, s);
            track(-(int64_t)Ocur.size() * N * (int64_t)sizeof(W));
            Ecur = Enxt;
            Enxt = nullptr;
            Ocur.swap(On);
        }
    }
done:
    dfree(w, s); dfree(At, s); dfree(Ecur, s); dfree(Enxt, s); dfree(bad, s); dfree(pstart, s); dfree(cur_of, s);
    dfree(pairs, s); dfree(part, s); dfree(offs, s);
    if (peak) *peak = std::max(*peak, pk);
    return rc;
}

template <typename W>
static cs_status setup_level_w(const cs_hierarchy *h, int l, int kind, int nu, int prescale, bool reuse, int alpha,
                               double *lam, cudaStream_t s, int64_t *peak) {
    const Level &L = h->lev[l];
    if (L.g.dim == 2) {
        if (L.kind == STAR) return setup_level_t<2, STAR, W>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak);
        return setup_level_t<2, BOX, W>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak);
    }
    if (L.kind == STAR) return setup_level_t<3, STAR, W>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak);
    return setup_level_t<3, BOX, W>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak);
}

cs_status cascade_setup_level(const cs_hierarchy *h, int l, int kind, int nu, int prescale, bool reuse, int alpha,
                              bool fp32, double *lam, cudaStream_t s, int64_t *peak) {
    // with truncation every row is computed (the repeated-row shortcut keeps deep rows unwritten)
    if (alpha > 0) reuse = false;
    return fp32 ? setup_level_w<float>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak)
                : setup_level_w<double>(h, l, kind, nu, prescale, reuse, alpha, lam, s, peak);
}


// ------------------------------------------------------ block cascade setup
// Blocks of bs^dim nodes (Algorithm 2 with n_b > 1).  E rows keep their
// column offsets relative to their own node.  For block b with nodes p at
// local displacement delta_p from the block anchor, the entry of row p at
// column node_p + o sits at offset o, so with Delta_pq = delta_p - delta_q
//   G_pq = sum_o R_p[o] R_q[o + Delta_pq],   C_pq = sum_o E_p[o] R_q[o + Delta_pq],
//   Lam~_b = C G^{-1} (normal equations; minimum-norm C G^+ if a Cholesky
//   pivot <= 1e-14 tr G),  E'_p[o] = E_p[o] - sum_q Lam~_pq R_q[o + Delta_pq].
// R lives on O_R = O_cur + S; the update spreads each row over the block, so
// O_next = O_R + D with D the displacements {-(bs-1)..bs-1}^dim.

// R rows of the nodes of active blocks (one thread per node), in W
// (FP64, or FP32 for the FP32 setup products)
template <int DIM, int KIND, typename W = double>
__global__ void __launch_bounds__(TBX *TBY) k_block_R(Grid g, int periodic, const W *__restrict__ At,
                                                       const W *__restrict__ Ecur, W *__restrict__ Rbuf,
                                                       int nR, const int *__restrict__ pstart,
                                                       const unsigned *__restrict__ pairs, int bs, int colour) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    constexpr int NT = TBX * TBY;
    extern __shared__ double sm_blk[];
    W *sa = reinterpret_cast<W *>(sm_blk);
    int *snb = reinterpret_cast<int *>(sa + NST * NT);
    const int tid = threadIdx.x + TBX * threadIdx.y;
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    if (colour >= 0) {
        const int bc = ((ix / bs + 1) + (iy / bs + 1) + (DIM == 3 ? iz / bs + 1 : 0)) & 1;
        if (bc != colour) return;
    }
    const int64_t N = g.N;
    const int i = ix + g.nx * (iy + g.ny * iz);
#pragma unroll
    for (int s = 0; s < NST; ++s) {
        int dx, dy, dz;
        S::off(s, dx, dy, dz);
        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        bool in;
        if (periodic) {
            jx = (jx + g.nx) % g.nx; jy = (jy + g.ny) % g.ny; jz = DIM == 3 ? (jz + g.nz) % g.nz : 0;
            in = true;
        } else {
            in = jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny && (DIM == 2 || (jz >= 0 && jz < g.nz));
        }
        snb[s * NT + tid] = in ? jx + g.nx * (jy + g.ny * jz) : i;
        sa[s * NT + tid] = in ? At[(int64_t)s * N + i] : W(0);
    }
    int p = __ldg(pstart);
    for (int o = 0; o < nR; ++o) {
        const int pe = __ldg(pstart + o + 1);
        W r = W(0);
        for (; p < pe; ++p) {
            const unsigned u = __ldg(pairs + p);
            const int s = (int)(u >> 24), c = (int)(u & 0xffffffu);
            r = fma(sa[s * NT + tid], Ecur[(int64_t)c * N + snb[s * NT + tid]], r);
        }
        Rbuf[(int64_t)o * N + i] = r;
    }
}

// Nodes of block b (x fastest inside the block; absent nodes past the upper
// grid edges skipped): global index, position in the padded bs^d layout and
// local coordinates.  Returns the count; *colour receives the block's
// red-black colour (parity of the 1-based block coordinates).
template <int DIM, int NMAX>
__device__ __forceinline__ int block_nodes(const Grid &g, int bs, int nbx, int nby, int64_t b, int *node, int *lpos,
                                           int (*dl)[3], int *colour) {
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
    int np = 0;
    for (int lp = 0; lp < NMAX; ++lp) {
        const int lx = lp % bs, ly = (lp / bs) % bs, lz = DIM == 3 ? lp / (bs * bs) : 0;
        if (DIM == 2 && lp >= bs * bs) break;
        const int ix = bs * bx + lx, iy = bs * by + ly, iz = DIM == 3 ? bs * bz + lz : 0;
        if (ix >= g.nx || iy >= g.ny || (DIM == 3 && iz >= g.nz)) continue;
        node[np] = ix + g.nx * (iy + g.ny * iz);
        lpos[np] = lp;
        if (dl) { dl[np][0] = lx; dl[np][1] = ly; dl[np][2] = lz; }
        ++np;
    }
    *colour = ((bx + 1) + (by + 1) + (DIM == 3 ? bz + 1 : 0)) & 1;
    return np;
}

// Index of the displacement between block nodes p and q in the (2 bs - 1)^d
// displacement list (lexicographic, x fastest).
template <int DIM>
__device__ __forceinline__ int block_sidx(const int (*dl)[3], int p, int q, int bs) {
    const int side = 2 * bs - 1;
    const int ex = dl[p][0] - dl[q][0] + bs - 1, ey = dl[p][1] - dl[q][1] + bs - 1;
    const int ez = DIM == 3 ? dl[p][2] - dl[q][2] + bs - 1 : 0;
    return ex + side * (ey + side * ez);
}

// Gram and cross products of one block per warp (Algorithm 2, the block
// least-squares data): G = R_i R_i^T and C = E_i R_i^T over the prescaled
// block rows R_i = (A~ E)_i.  Lanes split the offsets of each product,
// warp-shuffle sums in a fixed order.  Output layout: entry e of block b at
// GC[e * nblocks + b], e = p NMAX + q for G (q >= p only) and NMAX^2 + p NMAX
// + q for C, so that the thread-per-block solve reads it coalesced.
template <int DIM, int NMAX, typename W = double>
__global__ void __launch_bounds__(128) k_block_gram(Grid g, int bs, int nbx, int nby, int64_t nblocks,
                                                     const W *__restrict__ Ecur, const W *__restrict__ Rbuf,
                                                     int nR, const int *__restrict__ curR,
                                                     const int *__restrict__ shiftR, int colour,
                                                     double *__restrict__ GC) {
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * (int64_t)4 + (threadIdx.x >> 5);
    if (b >= nblocks) return;
    int node[NMAX], lpos[NMAX], dl[NMAX][3], bc;
    const int np = block_nodes<DIM, NMAX>(g, bs, nbx, nby, b, node, lpos, dl, &bc);
    if (colour >= 0 && bc != colour) return;
    const int64_t N = g.N;
    for (int p = 0; p < np; ++p)
        for (int q = 0; q < np; ++q) {
            const int *sh = shiftR + (int64_t)block_sidx<DIM>(dl, p, q, bs) * nR;
            // FP64: the lane's products accumulated in FP64; FP32: in FP32 over
            // chunks of 8 terms, the chunks added in FP64
            double gg = 0.0, cc = 0.0;
            W gw = W(0), cw = W(0);
            int nt = 0;
            for (int o = lane; o < nR; o += 32) {
                const int t = __ldg(sh + o);
                if (t < 0) continue;
                const W rq = Rbuf[(int64_t)t * N + node[q]];
                const int c0 = __ldg(curR + o);
                if constexpr (sizeof(W) == sizeof(double)) {
                    if (q >= p) gg = fma(Rbuf[(int64_t)o * N + node[p]], rq, gg);
                    if (c0 >= 0) cc = fma(Ecur[(int64_t)c0 * N + node[p]], rq, cc);
                } else {
                    if (q >= p) gw = fma(Rbuf[(int64_t)o * N + node[p]], rq, gw);
                    if (c0 >= 0) cw = fma(Ecur[(int64_t)c0 * N + node[p]], rq, cw);
                    if (++nt == 8) {
                        gg += (double)gw;
                        cc += (double)cw;
                        gw = W(0);
                        cw = W(0);
                        nt = 0;
                    }
                }
            }
            if constexpr (sizeof(W) != sizeof(double)) {
                gg += (double)gw;
                cc += (double)cw;
            }
            for (int off = 16; off > 0; off >>= 1) {
                gg += __shfl_xor_sync(0xffffffffu, gg, off);
                cc += __shfl_xor_sync(0xffffffffu, cc, off);
            }
            if (lane == 0) {
                if (q >= p) GC[(int64_t)(p * NMAX + q) * nblocks + b] = gg;
                GC[(int64_t)(NMAX * NMAX + p * NMAX + q) * nblocks + b] = cc;
            }
        }
}

// Packed upper-triangle slot of the symmetric entry (i, j).
template <int NMAX>
__device__ __forceinline__ int pk(int i, int j) {
    if (i > j) { const int t = i; i = j; j = t; }
    return i * NMAX - (i * (i - 1)) / 2 + (j - i);
}

// Least squares Lam~ = C G^{-1} of one block per thread: Cholesky of G with
// pivot threshold rtol tr(G) (rtol = 1e-14; 1e-5 for FP32 setup products);
// otherwise the minimum-norm solution C G^+ from a cyclic Jacobi
// eigendecomposition of G (eigenvalues <= rtol tr(G) dropped).  A 3x3-node block whose centre node has its whole 9-point
// stencil inside the block has an exactly singular G from the second cascade
// level on (the level-1 step annihilates that row of A E), so the Jacobi
// path is common, not exceptional.  One block per thread keeps every lane of
// each FP64 instruction busy, which is what bounds this kernel: the
// symmetric matrix (packed) and the eigenvectors sit in shared memory, entry
// e of thread t at [e * 64 + t].  The sweeps stop once the off-diagonal mass
// reaches rounding level (<= 1e-30 of the Frobenius mass, or no longer
// decreasing).  Writes Lam~ (entry p NMAX + q of block b at Lt[e * nblocks +
// b]) and the unscaled Lambda_ii = W_i Lam~ W_i into lam.
template <int DIM, int NMAX>
__global__ void __launch_bounds__(64) k_block_ls(Grid g, int bs, int nbx, int nby, int64_t nblocks,
                                                  const double *__restrict__ w, int colour,
                                                  const double *__restrict__ GC, double *__restrict__ Lt,
                                                  double *__restrict__ lam, double rtol) {
    constexpr int NP = NMAX * (NMAX + 1) / 2;
    extern __shared__ double sm_ls[];
    const int tid = threadIdx.x;
    double *A = sm_ls + tid;              // packed symmetric, stride 64
    double *Q = sm_ls + NP * 64 + tid;    // NMAX x NMAX, stride 64
    const int64_t b = blockIdx.x * (int64_t)64 + tid;
    if (b >= nblocks) return;
    int node[NMAX], lpos[NMAX], bc;
    const int n = block_nodes<DIM, NMAX>(g, bs, nbx, nby, b, node, lpos, nullptr, &bc);
    if (colour >= 0 && bc != colour) return;
    auto Gat = [&](int i, int j) { return GC[(int64_t)(i * NMAX + j) * nblocks + b]; };  // i <= j
    auto Cat = [&](int p, int m) { return GC[(int64_t)(NMAX * NMAX + p * NMAX + m) * nblocks + b]; };
    auto out = [&](int p, int q, double v) {
        Lt[(int64_t)(p * NMAX + q) * nblocks + b] = v;
        lam[b * (NMAX * NMAX) + lpos[p] * NMAX + lpos[q]] = w[node[p]] * v * w[node[q]];
    };
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += Gat(i, i);
    const double tol = rtol * tr;
    bool ok = tr > 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) A[64 * pk<NMAX>(i, j)] = Gat(i, j);
    // Cholesky in place: L(i, j), i >= j, in the slot of (j, i)
    for (int j = 0; j < n && ok; ++j) {
        double d = A[64 * pk<NMAX>(j, j)];
        for (int k = 0; k < j; ++k) d -= A[64 * pk<NMAX>(j, k)] * A[64 * pk<NMAX>(j, k)];
        if (!(d > tol)) { ok = false; break; }
        d = sqrt(d);
        A[64 * pk<NMAX>(j, j)] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = A[64 * pk<NMAX>(i, j)];
            for (int k = 0; k < j; ++k) v -= A[64 * pk<NMAX>(i, k)] * A[64 * pk<NMAX>(j, k)];
            A[64 * pk<NMAX>(i, j)] = v / d;
        }
    }
    if (ok) {
        for (int p = 0; p < n; ++p) {  // row p of C G^{-1}: G y = C_p^T by two triangular solves
            double y[NMAX];
#pragma unroll
            for (int i = 0; i < NMAX; ++i) {
                if (i >= n) break;
                double v = Cat(p, i);
#pragma unroll
                for (int k = 0; k < i; ++k) v -= A[64 * pk<NMAX>(i, k)] * y[k];
                y[i] = v / A[64 * pk<NMAX>(i, i)];
            }
#pragma unroll
            for (int i = NMAX - 1; i >= 0; --i) {
                if (i >= n) continue;
                double v = y[i];
#pragma unroll
                for (int k = i + 1; k < NMAX; ++k)
                    if (k < n) v -= A[64 * pk<NMAX>(k, i)] * y[k];
                y[i] = v / A[64 * pk<NMAX>(i, i)];
            }
#pragma unroll
            for (int q = 0; q < NMAX; ++q)
                if (q < n) out(p, q, y[q]);
        }
        return;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (j >= i) A[64 * pk<NMAX>(i, j)] = Gat(i, j);
            Q[64 * (i * NMAX + j)] = i == j ? 1.0 : 0.0;
        }
    double frob = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) frob += A[64 * pk<NMAX>(i, j)] * A[64 * pk<NMAX>(i, j)];
    double prev = frob;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[64 * pk<NMAX>(i, j)] * A[64 * pk<NMAX>(i, j)];
        if (off < 1e-300 || off <= 1e-30 * frob || (sweep > 0 && off >= prev)) break;
        prev = off;
        for (int a = 0; a < n; ++a)
            for (int c = a + 1; c < n; ++c) {
                const double apq = A[64 * pk<NMAX>(a, c)];
                if (apq == 0.0) continue;
                const double th = (A[64 * pk<NMAX>(c, c)] - A[64 * pk<NMAX>(a, a)]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {
                    if (k != a && k != c) {
                        const double x0 = A[64 * pk<NMAX>(k, a)], x1 = A[64 * pk<NMAX>(k, c)];
                        A[64 * pk<NMAX>(k, a)] = cs * x0 - sn * x1;
                        A[64 * pk<NMAX>(k, c)] = sn * x0 + cs * x1;
                    }
                    const double q0 = Q[64 * (k * NMAX + a)], q1 = Q[64 * (k * NMAX + c)];
                    Q[64 * (k * NMAX + a)] = cs * q0 - sn * q1;
                    Q[64 * (k * NMAX + c)] = sn * q0 + cs * q1;
                }
                A[64 * pk<NMAX>(a, a)] -= t * apq;
                A[64 * pk<NMAX>(c, c)] += t * apq;
                A[64 * pk<NMAX>(a, c)] = 0.0;
            }
    }
    double ev[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) ev[k] = k < n ? A[64 * pk<NMAX>(k, k)] : 0.0;
    for (int p = 0; p < n; ++p) {  // row p of C G^+ = C Q diag(1/ev, ev > tol) Q^T
        double cq[NMAX];
#pragma unroll
        for (int k = 0; k < NMAX; ++k) cq[k] = 0.0;
        for (int m = 0; m < n; ++m) {
            const double cpm = Cat(p, m);
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k < n) cq[k] += cpm * Q[64 * (m * NMAX + k)];
        }
        for (int q = 0; q < n; ++q) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k < n && ev[k] > tol) v += cq[k] * Q[64 * (q * NMAX + k)] / ev[k];
            out(p, q, v);
        }
    }
}

// The same least squares with one warp per block, for levels with too few
// blocks to fill the GPU one block per thread (there the serial FP64 chain of
// a single thread, not the FP64 throughput, sets the time).  G, C (full, row
// stride NMAX) are read only; Lt receives the n x n result; A, Q (NMAX^2) and
// ev (NMAX) are per-warp shared workspace.  Lanes split the rows of each
// elimination step, the right-hand sides of the triangular solves, the index
// k of each plane rotation and the entries of C G^+; every lane evaluates the
// scalar recurrences itself, so the rotations are those of the serial
// algorithm (two-sided, as written for a full matrix).
template <int NMAX>
__device__ void block_lstsq_warp(const double *G, const double *C, int n, double *Lt, double *A, double *Q,
                                 double *ev, int lane, double rtol) {
    double tr = 0.0;
    for (int k = 0; k < n; ++k) tr += G[k * NMAX + k];
    const double tol = rtol * tr;
    bool ok = tr > 0.0;
    for (int k = lane; k < NMAX * NMAX; k += 32) A[k] = G[k];
    __syncwarp();
    for (int j = 0; j < n && ok; ++j) {
        double d = A[j * NMAX + j];
        for (int k = 0; k < j; ++k) d -= A[j * NMAX + k] * A[j * NMAX + k];
        if (!(d > tol)) { ok = false; break; }
        d = sqrt(d);
        const int i = j + 1 + lane;
        double v = 0.0;
        if (i < n) {
            v = A[i * NMAX + j];
            for (int k = 0; k < j; ++k) v -= A[i * NMAX + k] * A[j * NMAX + k];
        }
        __syncwarp();
        if (i < n) A[i * NMAX + j] = v / d;
        if (lane == 0) A[j * NMAX + j] = d;
        __syncwarp();
    }
    __syncwarp();
    if (ok) {
        if (lane < n) {  // row `lane` of C G^{-1}: G y = C_p^T by two triangular solves
            double *y = Lt + lane * NMAX;
            for (int i = 0; i < n; ++i) {
                double v = C[lane * NMAX + i];
                for (int k = 0; k < i; ++k) v -= A[i * NMAX + k] * y[k];
                y[i] = v / A[i * NMAX + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double v = y[i];
                for (int k = i + 1; k < n; ++k) v -= A[k * NMAX + i] * y[k];
                y[i] = v / A[i * NMAX + i];
            }
        }
        __syncwarp();
        return;
    }
    for (int k = lane; k < NMAX * NMAX; k += 32) {
        const int r = k / NMAX, c = k % NMAX;
        A[k] = r < n && c < n ? G[k] : 0.0;
        Q[k] = r == c ? 1.0 : 0.0;
    }
    __syncwarp();
    double frob = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) frob += A[i * NMAX + j] * A[i * NMAX + j];
    double prev = frob;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i * NMAX + j] * A[i * NMAX + j];
        if (off < 1e-300 || off <= 1e-30 * frob || (sweep > 0 && off >= prev)) break;
        prev = off;
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b) {
                const double apq = A[a * NMAX + b];
                if (apq == 0.0) continue;
                const double th = (A[b * NMAX + b] - A[a * NMAX + a]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                __syncwarp();
                if (lane < n) {
                    const double x0 = A[lane * NMAX + a], x1 = A[lane * NMAX + b];
                    A[lane * NMAX + a] = cs * x0 - sn * x1;
                    A[lane * NMAX + b] = sn * x0 + cs * x1;
                }
                __syncwarp();
                if (lane < n) {
                    const double x0 = A[a * NMAX + lane], x1 = A[b * NMAX + lane];
                    A[a * NMAX + lane] = cs * x0 - sn * x1;
                    A[b * NMAX + lane] = sn * x0 + cs * x1;
                    const double q0 = Q[lane * NMAX + a], q1 = Q[lane * NMAX + b];
                    Q[lane * NMAX + a] = cs * q0 - sn * q1;
                    Q[lane * NMAX + b] = sn * q0 + cs * q1;
                }
                __syncwarp();
            }
    }
    if (lane < n) ev[lane] = A[lane * NMAX + lane];
    __syncwarp();
    for (int k = lane; k < n * n; k += 32) {  // (C Q)_{p,k} into A
        const int p = k / n, kk = k % n;
        double cq = 0.0;
        for (int m = 0; m < n; ++m) cq += C[p * NMAX + m] * Q[m * NMAX + kk];
        A[p * NMAX + kk] = cq;
    }
    __syncwarp();
    for (int k = lane; k < n * n; k += 32) {  // G^+ = Q diag(1/ev, ev > tol) Q^T
        const int p = k / n, q = k % n;
        double v = 0.0;
        for (int kk = 0; kk < n; ++kk)
            if (ev[kk] > tol) v += A[p * NMAX + kk] * Q[q * NMAX + kk] / ev[kk];
        Lt[p * NMAX + q] = v;
    }
    __syncwarp();
}

// Block counts below which the least squares run one warp per block.
constexpr int64_t kLsThreadMin = 4096;

template <int DIM, int NMAX>
__global__ void __launch_bounds__(128) k_block_ls_warp(Grid g, int bs, int nbx, int nby, int64_t nblocks,
                                                        const double *__restrict__ w, int colour,
                                                        const double *__restrict__ GC, double *__restrict__ Lt,
                                                        double *__restrict__ lam, double rtol) {
    __shared__ double sG[4][NMAX * NMAX], sC[4][NMAX * NMAX], sL[4][NMAX * NMAX], sA[4][NMAX * NMAX],
        sQ[4][NMAX * NMAX], sEv[4][NMAX];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * (int64_t)4 + wib;
    if (b >= nblocks) return;
    int node[NMAX], lpos[NMAX], bc;
    const int np = block_nodes<DIM, NMAX>(g, bs, nbx, nby, b, node, lpos, nullptr, &bc);
    if (colour >= 0 && bc != colour) return;
    for (int e = lane; e < NMAX * NMAX; e += 32) {
        const int p = e / NMAX, q = e % NMAX;
        const bool in = p < np && q < np;
        sG[wib][e] = in ? GC[(int64_t)(p <= q ? e : q * NMAX + p) * nblocks + b] : 0.0;
        sC[wib][e] = in ? GC[(int64_t)(NMAX * NMAX + e) * nblocks + b] : 0.0;
    }
    __syncwarp();
    block_lstsq_warp<NMAX>(sG[wib], sC[wib], np, sL[wib], sA[wib], sQ[wib], sEv[wib], lane, rtol);
    for (int e = lane; e < np * np; e += 32) {
        const int p = e / np, q = e % np;
        const double v = sL[wib][p * NMAX + q];
        Lt[(int64_t)(p * NMAX + q) * nblocks + b] = v;
        lam[b * (NMAX * NMAX) + lpos[p] * NMAX + lpos[q]] = w[node[p]] * v * w[node[q]];
    }
}

// E update of one block per warp (Algorithm 2): new rows E_i - Lam~_ii R_i
// over the next offset set; blocks of the other colour carry their rows
// over unchanged.
template <int DIM, int NMAX, typename W = double>
__global__ void __launch_bounds__(128) k_block_update(Grid g, int bs, int nbx, int nby, int64_t nblocks,
                                                       const W *__restrict__ Ecur,
                                                       const W *__restrict__ Rbuf, W *__restrict__ Enxt,
                                                       int nN, const int *__restrict__ curN,
                                                       const int *__restrict__ shiftN, int colour,
                                                       const double *__restrict__ Lt) {
    __shared__ double sLt[4][NMAX * NMAX];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * (int64_t)4 + wib;
    if (b >= nblocks) return;
    int node[NMAX], lpos[NMAX], dl[NMAX][3], bc;
    const int np = block_nodes<DIM, NMAX>(g, bs, nbx, nby, b, node, lpos, dl, &bc);
    const int64_t N = g.N;
    if (colour >= 0 && bc != colour) {
        for (int k = 0; k < np; ++k)
            for (int o = lane; o < nN; o += 32) {
                const int c = __ldg(curN + o);
                Enxt[(int64_t)o * N + node[k]] = c >= 0 ? Ecur[(int64_t)c * N + node[k]] : W(0);
            }
        return;
    }
    double *L = sLt[wib];
    for (int e = lane; e < NMAX * NMAX; e += 32) {
        const int p = e / NMAX, q = e % NMAX;
        L[e] = p < np && q < np ? Lt[(int64_t)e * nblocks + b] : 0.0;
    }
    __syncwarp();
    for (int p = 0; p < np; ++p)
        for (int o = lane; o < nN; o += 32) {
            const int c0 = __ldg(curN + o);
            W v = c0 >= 0 ? Ecur[(int64_t)c0 * N + node[p]] : W(0);
            for (int q = 0; q < np; ++q) {
                const int t = __ldg(shiftN + (int64_t)block_sidx<DIM>(dl, p, q, bs) * nN + o);
                if (t >= 0) v = fma((W)-L[p * NMAX + q], Rbuf[(int64_t)t * N + node[q]], v);
            }
            Enxt[(int64_t)o * N + node[p]] = v;
        }
}

// Truncation of the updated block rows (Algorithm 2's optional step, for
// blocks): block b's rows keep the alpha column blocks of largest Frobenius
// norm over the block's rows -- ties go to the smaller block index -- and
// the others are set to zero.  Candidates are the blocks within reach of the
// offsets (radius R) that hold an in-grid column of one of the rows; a
// column block's squared norm adds, over its nodes in ascending index and
// per node over the block's rows in ascending index, the squared entries
// (unfused).  With no more candidates than alpha the rows are kept.  One
// warp per block: lanes over candidates, alpha rounds of a warp arg-max,
// then lanes over offsets zero what was not selected.  offidx maps an offset
// (ox, oy, oz), |o| <= R per axis, to its index in the step's offsets, or -1.
// err is set when the candidates exceed 32 TR_KC or alpha exceeds 64.
constexpr int TR_KC = 32;  // candidates per lane
template <int DIM, int NMAX, typename W = double>
__global__ void __launch_bounds__(128) k_block_truncate(Grid g, int bs, int nbx, int nby, int nbz, int64_t nblocks,
                                                         W *__restrict__ E, int nN, const int *__restrict__ off,
                                                         const int *__restrict__ offidx, int R, int alpha,
                                                         int colour, int *err) {
    __shared__ int ssel[4][64];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * (int64_t)4 + wib;
    if (b >= nblocks) return;
    int node[NMAX], lpos[NMAX], bc;
    const int np = block_nodes<DIM, NMAX>(g, bs, nbx, nby, b, node, lpos, nullptr, &bc);
    if (colour >= 0 && bc != colour) return;
    const int64_t N = g.N;
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
    auto lo = [&](int c) { return bs * c - R >= 0 ? (bs * c - R) / bs : 0; };  // floor, clamped at 0
    const int cx0 = lo(bx), cy0 = lo(by), cz0 = DIM == 3 ? lo(bz) : 0;
    const int cx1 = min(nbx - 1, (bs * bx + bs - 1 + R) / bs), cy1 = min(nby - 1, (bs * by + bs - 1 + R) / bs);
    const int cz1 = DIM == 3 ? min(nbz - 1, (bs * bz + bs - 1 + R) / bs) : 0;
    const int ncx = cx1 - cx0 + 1, ncy = cy1 - cy0 + 1, ncz = cz1 - cz0 + 1;
    const int ncand = ncx * ncy * ncz;
    if (ncand > 32 * TR_KC || alpha > 64) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    const int side = 2 * R + 1;
    double nrm[TR_KC];
    bool pres[TR_KC], sel[TR_KC];
#pragma unroll
    for (int k = 0; k < TR_KC; ++k) {
        nrm[k] = 0.0;
        pres[k] = false;
        sel[k] = false;
        const int c = lane + 32 * k;
        if (c >= ncand) continue;
        const int qx = cx0 + c % ncx, qy = cy0 + (c / ncx) % ncy, qz = cz0 + c / (ncx * ncy);
        double acc = 0.0;
        bool any = false;
        for (int jz = (DIM == 3 ? bs * qz : 0); jz < (DIM == 3 ? min(g.nz, bs * qz + bs) : 1); ++jz)
            for (int jy = bs * qy; jy < min(g.ny, bs * qy + bs); ++jy)
                for (int jx = bs * qx; jx < min(g.nx, bs * qx + bs); ++jx)
                    for (int p = 0; p < np; ++p) {
                        const int ix = node[p] % g.nx, iy = (node[p] / g.nx) % g.ny, iz = node[p] / (g.nx * g.ny);
                        const int ox = jx - ix, oy = jy - iy, oz = jz - iz;
                        if (abs(ox) > R || abs(oy) > R || abs(oz) > R) continue;
                        const int t = __ldg(offidx + (ox + R) + side * ((oy + R) + side * (DIM == 3 ? oz + R : 0)));
                        if (t < 0) continue;
                        const double v = (double)E[(int64_t)t * N + node[p]];
                        acc = __dadd_rn(acc, __dmul_rn(v, v));
                        any = true;
                    }
        nrm[k] = acc;
        pres[k] = any;
    }
    int npres = 0;
#pragma unroll
    for (int k = 0; k < TR_KC; ++k) npres += pres[k] ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) npres += __shfl_xor_sync(0xffffffffu, npres, o);
    if (npres <= alpha) return;  // every candidate kept
    for (int a = 0; a < alpha; ++a) {
        double bn = -1.0;
        int bcand = 1 << 30;
#pragma unroll
        for (int k = 0; k < TR_KC; ++k) {
            const int c = lane + 32 * k;
            if (!pres[k] || sel[k]) continue;
            if (nrm[k] > bn || (nrm[k] == bn && c < bcand)) { bn = nrm[k]; bcand = c; }
        }
        for (int o = 16; o > 0; o >>= 1) {  // arg-max: larger norm, then the smaller candidate (block index)
            const double on = __shfl_xor_sync(0xffffffffu, bn, o);
            const int oc = __shfl_xor_sync(0xffffffffu, bcand, o);
            if (on > bn || (on == bn && oc < bcand)) { bn = on; bcand = oc; }
        }
#pragma unroll
        for (int k = 0; k < TR_KC; ++k)
            if (lane + 32 * k == bcand) sel[k] = true;
        if (lane == 0) ssel[wib][a] = bcand;
    }
    __syncwarp();
    for (int p = 0; p < np; ++p) {
        const int ix = node[p] % g.nx, iy = (node[p] / g.nx) % g.ny, iz = node[p] / (g.nx * g.ny);
        for (int t = lane; t < nN; t += 32) {
            const int jx = ix + __ldg(off + 3 * t), jy = iy + __ldg(off + 3 * t + 1);
            const int jz = DIM == 3 ? iz + __ldg(off + 3 * t + 2) : 0;
            if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny || (DIM == 3 && (jz < 0 || jz >= g.nz))) continue;
            const int c = (jx / bs - cx0) + ncx * ((jy / bs - cy0) + ncy * (DIM == 3 ? jz / bs - cz0 : 0));
            bool keep = false;
            for (int a = 0; a < alpha; ++a) keep = keep || ssel[wib][a] == c;
            if (!keep) E[(int64_t)t * N + node[p]] = W(0);
        }
    }
}

template <int DIM, int KIND, typename W>
static cs_status setup_blocks_t(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int alpha, double *lam,
                                cudaStream_t s) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    const Level &L = h->lev[l];
    const Grid g = L.g;
    const int64_t N = g.N;
    const int bs = L.bs, ncol = kind == CS_MULTIPLICATIVE ? 2 : 1;
    const int nmax = L.nmax;
    dim3 gr = node_grid(g), bl = node_block();
    double *w = nullptr, *GC = nullptr, *Ltb = nullptr;
    W *At = nullptr, *Ecur = nullptr, *Enxt = nullptr, *Rbuf = nullptr;  // the products' precision
    int *bad = nullptr, *pstart = nullptr, *curR = nullptr, *shiftR = nullptr, *curN = nullptr, *shiftN = nullptr;
    int *toff = nullptr, *tidx = nullptr, *terr = nullptr;  // truncation: offsets, offset lookup, error flag
    unsigned *pairs = nullptr;
    cs_status rc = CS_OK;
    int badh = 0;
    std::vector<Off3> Ocur{{0, 0, 0}};
    std::vector<Off3> D;
    const size_t smem = (size_t)NST * TBX * TBY * (sizeof(W) + sizeof(int));
    if (alpha > 0) {
        if ((rc = dalloc_t(&terr, 1, nullptr, s)) != CS_OK) goto done;
        CSX_CUDA_GOTO(cudaMemsetAsync(terr, 0, sizeof(int), s));
    }
    for (int dz = (DIM == 3 ? -(bs - 1) : 0); dz <= (DIM == 3 ? bs - 1 : 0); ++dz)
        for (int dy = -(bs - 1); dy <= bs - 1; ++dy)
            for (int dx = -(bs - 1); dx <= bs - 1; ++dx) D.push_back({dx, dy, dz});  // lexicographic = sidx order

    if ((rc = dalloc_t(&w, N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&At, (size_t)NST * N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&bad, 1, nullptr, s)) != CS_OK) goto done;
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(lam, 0, sizeof(double) * (size_t)nu * L.nblocks * nmax * nmax, s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
        goto done;
    }
    k_prescale<DIM, KIND><<<gr, bl, 0, s>>>(g, h->periodic, prescale, L.A, w, nullptr, bad);
    count_launch();
    if (cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "prescale", __FILE__, __LINE__);
        goto done;
    }
    if (badh) {
        set_error("level %d: non-positive diagonal entry; elliptic prescaling needs A_ii > 0", l);
        rc = CS_ERR_ARG;
        goto done;
    }
    k_scale_op<DIM, KIND, W><<<gr, bl, 0, s>>>(g, h->periodic, L.A, w, At);
    count_launch();
    if ((rc = dalloc_t(&Ecur, N, nullptr, s)) != CS_OK) goto done;
    // Gram/cross products and Lam~ of every block, entry-major (coalesced for the per-thread solve)
    if ((rc = dalloc_t(&GC, (size_t)2 * nmax * nmax * L.nblocks, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&Ltb, (size_t)nmax * nmax * L.nblocks, nullptr, s)) != CS_OK) goto done;
    k_fill<<<1216, 256, 0, s>>>(N, Ecur, W(1));
    count_launch();
    CSX_CUDA_GOTO(cudaFuncSetAttribute(k_block_R<DIM, KIND, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int lev = 0; lev < nu; ++lev) {
        for (int k = 0; k < ncol; ++k) {
            const bool last = lev == nu - 1 && k == ncol - 1;
            std::vector<Off3> OR, ON;
            for (const Off3 &o : Ocur)
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    OR.push_back({o.x + dx, o.y + dy, o.z + dz});
                }
            std::sort(OR.begin(), OR.end());
            OR.erase(std::unique(OR.begin(), OR.end()), OR.end());
            for (const Off3 &o : OR)
                for (const Off3 &d : D) ON.push_back({o.x + d.x, o.y + d.y, o.z + d.z});
            std::sort(ON.begin(), ON.end());
            ON.erase(std::unique(ON.begin(), ON.end()), ON.end());
            if (h->periodic) {
                int rx = 0, ry = 0, rz = 0;
                for (const Off3 &o : ON) { rx = std::max(rx, std::abs(o.x)); ry = std::max(ry, std::abs(o.y)); rz = std::max(rz, std::abs(o.z)); }
                if (2 * rx >= g.nx || 2 * ry >= g.ny || (DIM == 3 && 2 * rz >= g.nz)) {
                    set_error("periodic grid too small for the fill-in of this cascade (side must exceed twice the fill radius)");
                    rc = CS_ERR_UNSUPPORTED;
                    goto done;
                }
            }
            std::map<Off3, int> icur, iR;
            for (size_t t = 0; t < Ocur.size(); ++t) icur[Ocur[t]] = (int)t;
            for (size_t t = 0; t < OR.size(); ++t) iR[OR[t]] = (int)t;
            const int nR = (int)OR.size(), nN = (int)ON.size();
            std::vector<int> hps(nR + 1, 0), hcurR(nR), hshR((size_t)D.size() * nR), hcurN(nN), hshN((size_t)D.size() * nN);
            std::vector<unsigned> hpairs;
            for (int o = 0; o < nR; ++o) {
                auto it = icur.find(OR[o]);
                hcurR[o] = it == icur.end() ? -1 : it->second;
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    auto jt = icur.find({OR[o].x - dx, OR[o].y - dy, OR[o].z - dz});
                    if (jt != icur.end()) hpairs.push_back(((unsigned)t << 24) | (unsigned)jt->second);
                }
                hps[o + 1] = (int)hpairs.size();
                for (size_t d = 0; d < D.size(); ++d) {
                    auto jt = iR.find({OR[o].x + D[d].x, OR[o].y + D[d].y, OR[o].z + D[d].z});
                    hshR[d * nR + o] = jt == iR.end() ? -1 : jt->second;
                }
            }
            for (int o = 0; o < nN; ++o) {
                auto it = icur.find(ON[o]);
                hcurN[o] = it == icur.end() ? -1 : it->second;
                for (size_t d = 0; d < D.size(); ++d) {
                    auto jt = iR.find({ON[o].x + D[d].x, ON[o].y + D[d].y, ON[o].z + D[d].z});
                    hshN[d * nN + o] = jt == iR.end() ? -1 : jt->second;
                }
            }
            dfree(pstart, s); dfree(pairs, s); dfree(curR, s); dfree(shiftR, s); dfree(curN, s); dfree(shiftN, s);
            pstart = nullptr; pairs = nullptr; curR = nullptr; shiftR = nullptr; curN = nullptr; shiftN = nullptr;
            if ((rc = dalloc_t(&pstart, hps.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&pairs, std::max<size_t>(1, hpairs.size()), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&curR, hcurR.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&shiftR, hshR.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&curN, hcurN.size(), nullptr, s)) != CS_OK) goto done;
            if ((rc = dalloc_t(&shiftN, hshN.size(), nullptr, s)) != CS_OK) goto done;
            if (cudaMemcpyAsync(pstart, hps.data(), hps.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(pairs, hpairs.data(), hpairs.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(curR, hcurR.data(), hcurR.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(shiftR, hshR.data(), hshR.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(curN, hcurN.data(), hcurN.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(shiftN, hshN.data(), hshN.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "copy block setup tables", __FILE__, __LINE__);
                goto done;
            }
            if ((rc = dalloc_t(&Rbuf, (size_t)nR * N, nullptr, s)) != CS_OK) goto done;
            if (!last && (rc = dalloc_t(&Enxt, (size_t)nN * N, nullptr, s)) != CS_OK) goto done;
            int tR = 0;
            for (const Off3 &o : ON) tR = std::max({tR, std::abs(o.x), std::abs(o.y), std::abs(o.z)});
            // at most (2 ceil(R / bs) + 2)^d column blocks are in reach: alpha at
            // least that truncates nothing
            const int reach = 2 * ((tR + bs - 1) / bs) + 2;
            const bool trunc = alpha > 0 && !last && (int64_t)alpha < (int64_t)reach * reach * (DIM == 3 ? reach : 1);
            if (trunc) {  // the new offsets and their dense lookup over [-R, R]^d
                const int side = 2 * tR + 1;
                std::vector<int> ho(3 * (size_t)nN), hidx((size_t)side * side * (DIM == 3 ? side : 1), -1);
                for (int o = 0; o < nN; ++o) {
                    ho[3 * o] = ON[o].x; ho[3 * o + 1] = ON[o].y; ho[3 * o + 2] = ON[o].z;
                    hidx[(ON[o].x + tR) + side * ((ON[o].y + tR) + side * (DIM == 3 ? ON[o].z + tR : 0))] = o;
                }
                dfree(toff, s); dfree(tidx, s);
                toff = nullptr; tidx = nullptr;
                if ((rc = dalloc_t(&toff, ho.size(), nullptr, s)) != CS_OK) goto done;
                if ((rc = dalloc_t(&tidx, hidx.size(), nullptr, s)) != CS_OK) goto done;
                CSX_CUDA_GOTO(cudaMemcpyAsync(toff, ho.data(), sizeof(int) * ho.size(), cudaMemcpyHostToDevice, s));
                CSX_CUDA_GOTO(cudaMemcpyAsync(tidx, hidx.data(), sizeof(int) * hidx.size(), cudaMemcpyHostToDevice, s));
                CSX_CUDA_GOTO(cudaStreamSynchronize(s));  // the host tables go out of scope
            }
            {
                const int colour = ncol == 2 ? k : -1;
                k_block_R<DIM, KIND, W><<<gr, bl, smem, s>>>(g, h->periodic, At, Ecur, Rbuf, nR, pstart, pairs, bs, colour);
                count_launch();
                const unsigned nwarp = (unsigned)((L.nblocks + 3) / 4), nthr = (unsigned)((L.nblocks + 63) / 64);
                // the minimum-norm cutoff: 1e-14 tr(G) with FP64 products; FP32 products resolve
                // G only to ~1e-6 of its trace, so an exact null direction (3x3 blocks of
                // 9-point operators, some 2x2 blocks of them from the second step on) is dropped
                // below 1e-5 tr(G)
                const double ls_rtol = sizeof(W) == sizeof(double) ? 1e-14 : 1e-5;
                double *lam_l = lam + (int64_t)lev * L.nblocks * nmax * nmax;
#define CSX_BLOCK_STEPS(NM)                                                                                         \
    {                                                                                                               \
        const size_t lsm = (size_t)64 * (NM * (NM + 1) / 2 + NM * NM) * sizeof(double);                          \
        k_block_gram<DIM, NM, W><<<nwarp, 128, 0, s>>>(g, bs, L.nbx, L.nby, L.nblocks, Ecur, Rbuf, nR, curR,    \
                                                        shiftR, \
                                                     colour, GC);                                                   \
        if (L.nblocks >= kLsThreadMin) {                                                                            \
            CSX_CUDA_GOTO(cudaFuncSetAttribute(k_block_ls<DIM, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                               (int)lsm));                                                          \
            k_block_ls<DIM, NM><<<nthr, 64, lsm, s>>>(g, bs, L.nbx, L.nby, L.nblocks, w, colour, GC, Ltb, lam_l,  \
                                                     ls_rtol);                                                      \
        } else {                                                                                                    \
            k_block_ls_warp<DIM, NM><<<nwarp, 128, 0, s>>>(g, bs, L.nbx, L.nby, L.nblocks, w, colour, GC, Ltb,    \
                                                           lam_l, ls_rtol);                                         \
        }                                                                                                           \
        count_launch(2);                                                                                            \
        if (!last) {                                                                                                \
            k_block_update<DIM, NM, W><<<nwarp, 128, 0, s>>>(g, bs, L.nbx, L.nby, L.nblocks, Ecur, Rbuf, Enxt, nN,\
                                                          curN, shiftN, colour, Ltb);                               \
            count_launch();                                                                                         \
            if (trunc) {                                                                                            \
                k_block_truncate<DIM, NM, W><<<nwarp, 128, 0, s>>>(g, bs, L.nbx, L.nby, L.nbz, L.nblocks, Enxt, nN, \
                                                                toff, tidx, tR, alpha, colour, terr);              \
                count_launch();                                                                                     \
            }                                                                                                       \
        }                                                                                                           \
    }
                if (nmax == 4) CSX_BLOCK_STEPS(4)
                else if (nmax == 8) CSX_BLOCK_STEPS(8)
                else if (nmax == 9) CSX_BLOCK_STEPS(9)
                else { set_error("blocks of %d nodes are not supported (4, 8 or 9)", nmax); rc = CS_ERR_UNSUPPORTED; goto done; }
#undef CSX_BLOCK_STEPS
            }
            if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "block setup", __FILE__, __LINE__); goto done; }
            if (trunc) {
                int th = 0;
                CSX_CUDA_GOTO(cudaMemcpyAsync(&th, terr, sizeof(int), cudaMemcpyDeviceToHost, s));
                CSX_CUDA_GOTO(cudaStreamSynchronize(s));
                if (th) {
                    set_error("level %d: truncation needs alpha <= 64 and at most %d column blocks in reach", l,
                              32 * TR_KC);
                    rc = CS_ERR_UNSUPPORTED;
                    goto done;
                }
            }
            dfree(Ecur, s);
            dfree(Rbuf, s);
            Rbuf = nullptr;
            Ecur = Enxt;
            Enxt = nullptr;
            Ocur.swap(ON);
        }
    }
done:
    dfree(w, s); dfree(At, s); dfree(Ecur, s); dfree(Enxt, s); dfree(Rbuf, s); dfree(bad, s); dfree(pstart, s);
    dfree(GC, s); dfree(Ltb, s);
    dfree(pairs, s); dfree(curR, s); dfree(shiftR, s); dfree(curN, s); dfree(shiftN, s);
    dfree(toff, s); dfree(tidx, s); dfree(terr, s);
    return rc;
}

cs_status cascade_setup_level_blocks(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int alpha, bool fp32, double *lam,
                                     cudaStream_t s) {
    const Level &L = h->lev[l];
    if (L.g.dim == 2) {
        if (L.kind == STAR)
            return fp32 ? setup_blocks_t<2, STAR, float>(h, l, kind, nu, prescale, alpha, lam, s)
                        : setup_blocks_t<2, STAR, double>(h, l, kind, nu, prescale, alpha, lam, s);
        return fp32 ? setup_blocks_t<2, BOX, float>(h, l, kind, nu, prescale, alpha, lam, s)
                    : setup_blocks_t<2, BOX, double>(h, l, kind, nu, prescale, alpha, lam, s);
    }
    if (L.kind == STAR)
        return fp32 ? setup_blocks_t<3, STAR, float>(h, l, kind, nu, prescale, alpha, lam, s)
                    : setup_blocks_t<3, STAR, double>(h, l, kind, nu, prescale, alpha, lam, s);
    return fp32 ? setup_blocks_t<3, BOX, float>(h, l, kind, nu, prescale, alpha, lam, s)
                : setup_blocks_t<3, BOX, double>(h, l, kind, nu, prescale, alpha, lam, s);
}

}  // namespace csx
