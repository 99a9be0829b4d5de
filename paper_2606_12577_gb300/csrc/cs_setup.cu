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
// outside the grid are zero coefficients; fine nodes beyond the upper edge
// are skipped; entries whose coarse neighbour lies outside are set to zero.
template <int DIM, int KIND>
__global__ void __launch_bounds__(TBX *TBY) k_galerkin(Grid gf, Grid gc, const double *__restrict__ Af,
                                                        double *__restrict__ Ac) {
    using S = StenS<DIM, KIND>;
    constexpr int NC = DIM == 3 ? 27 : 9;
    extern __shared__ double acc_sm[];  // [NC][TBX*TBY]
    const int tid = threadIdx.x + TBX * threadIdx.y;
    double *acc = acc_sm + tid;
#pragma unroll
    for (int t = 0; t < NC; ++t) acc[t * TBX * TBY] = 0.0;
    const int cx = blockIdx.x * TBX + threadIdx.x, cy = blockIdx.y * TBY + threadIdx.y, cz = blockIdx.z;
    if (cx >= gc.nx || cy >= gc.ny) return;
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
    const int64_t ci = cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz);
    const double sc = DIM == 3 ? 0.125 : 0.25;
#pragma unroll
    for (int t = 0; t < NC; ++t) {
        const int jx = cx + t % 3 - 1, jy = cy + (t / 3) % 3 - 1, jz = DIM == 3 ? cz + t / 9 - 1 : 0;
        const bool in = jx >= 0 && jx < gc.nx && jy >= 0 && jy < gc.ny && (DIM == 2 || (jz >= 0 && jz < gc.nz));
        Ac[(int64_t)t * gc.N + ci] = in ? sc * acc[t * TBX * TBY] : 0.0;
    }
}

cs_status galerkin_level(const Level &f, Level &c, cudaStream_t s) {
    dim3 gr = node_grid(c.g), bl = node_block();
    const size_t sm2 = sizeof(double) * 9 * TBX * TBY, sm3 = sizeof(double) * 27 * TBX * TBY;
    if (f.g.dim == 2) {
        if (f.kind == STAR) k_galerkin<2, STAR><<<gr, bl, sm2, s>>>(f.g, c.g, f.A, c.A);
        else k_galerkin<2, BOX><<<gr, bl, sm2, s>>>(f.g, c.g, f.A, c.A);
    } else {
        static bool attr = false;  // 27 x 256 doubles = 54 KB exceeds the default 48 KB
        if (!attr) {
            CSX_CUDA(cudaFuncSetAttribute(k_galerkin<3, STAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
            CSX_CUDA(cudaFuncSetAttribute(k_galerkin<3, BOX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
            attr = true;
        }
        if (f.kind == STAR) k_galerkin<3, STAR><<<gr, bl, sm3, s>>>(f.g, c.g, f.A, c.A);
        else k_galerkin<3, BOX><<<gr, bl, sm3, s>>>(f.g, c.g, f.A, c.A);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
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

// Single-CTA dense factorisation and inverse: Cholesky (SPD), else LU with
// partial pivoting.  status[0] = 0 ok, 1 singular.
__global__ void k_factor_inverse(int n, double *M, double *W, double *Inv, int *piv, int *status) {
    __shared__ int bad;
    __shared__ int spd;
    int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t t = tid; t < (int64_t)n * n; t += nt) W[t] = M[t];
    if (tid == 0) { bad = 0; spd = 1; }
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
    CSX_TRY(dalloc_t(&h->cinv, (size_t)n * n, &h->bytes));
    cs_status rc = CS_OK;
    int offh[81];
    for (int t = 0; t < L.nst; ++t)
        for (int d = 0; d < 3; ++d) offh[3 * t + d] = L.off[t][d];
    int sth = 0;
    if ((rc = dalloc_t(&M, (size_t)n * n, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&W, (size_t)n * n, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&piv, (size_t)n + 1, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&st, 1, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&offs, 81, nullptr)) != CS_OK) goto done;
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
    cudaFree(M); cudaFree(W); cudaFree(piv); cudaFree(st); cudaFree(offs);
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

template <int DIM, int KIND>
__global__ void k_scale_op(Grid g, int periodic, const double *__restrict__ A, const double *__restrict__ w,
                           double *__restrict__ At) {
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
        At[(int64_t)s * g.N + i] = v;
    }
}

__global__ void k_fill(int64_t n, double *p, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// One setup step (l, k) over rows and a chunk of output offsets o'.
// Per o' the host supplies (uniform across a warp): mask[o'] with bit s set
// when o' - off(s) is in O_cur, its index cidx[o'*NST + s], and cur_of[o']
// (index of o' in O_cur or -1).  Neighbours outside the grid carry a zero
// prescaled coefficient, so they are read at the row itself (no branch).
// nchunks == 1: the thread finishes the row (lambda, residual update);
// otherwise partial <E_i,R_i>, <R_i,R_i> go to part[q*N + i] and
// k_setup_finish completes the row.  LAST: the final step of the cascade,
// where E_nu is not needed -- R is neither stored nor used to update E.
template <int DIM, int KIND, bool LAST>
__global__ void __launch_bounds__(TBX *TBY) k_setup_rows(Grid g, int periodic, const double *__restrict__ At,
                                                          const double *__restrict__ w, const double *__restrict__ Ecur,
                                                          double *__restrict__ Enxt, int nnxt, int chunk, int nchunks,
                                                          const unsigned *__restrict__ mask, const int *__restrict__ cidx,
                                                          const int *__restrict__ cur_of, int colour,
                                                          double *__restrict__ lam, double2 *__restrict__ part) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y;
    const int iz = (int)(blockIdx.z % (unsigned)g.nz), q = (int)(blockIdx.z / (unsigned)g.nz);
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t N = g.N;
    const int i = ix + g.nx * (iy + g.ny * iz);
    const int o0 = q * chunk, o1 = min(nnxt, o0 + chunk);
    const bool active = colour < 0 || ((((ix + 1) + (iy + 1) + (DIM == 3 ? iz + 1 : 0)) & 1) == colour);
    if (!active) {
        if (!LAST)
            for (int o = o0; o < o1; ++o) {
                int c = __ldg(cur_of + o);
                Enxt[(int64_t)o * N + i] = c >= 0 ? Ecur[(int64_t)c * N + i] : 0.0;
            }
        return;
    }
    double a[NST];
    int nb[NST];
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
        nb[s] = in ? jx + g.nx * (jy + g.ny * jz) : i;
        a[s] = in ? At[(int64_t)s * N + i] : 0.0;
    }
    double num = 0.0, den = 0.0;
    for (int o = o0; o < o1; ++o) {
        const unsigned m = __ldg(mask + o);
        const int *co = cidx + o * NST;
        double r = 0.0;
#pragma unroll
        for (int s = 0; s < NST; ++s)
            if (m & (1u << s)) r = fma(a[s], Ecur[(int64_t)__ldg(co + s) * N + nb[s]], r);
        const int c0 = __ldg(cur_of + o);
        if (c0 >= 0) num = fma(Ecur[(int64_t)c0 * N + i], r, num);
        den = fma(r, r, den);
        if (!LAST) Enxt[(int64_t)o * N + i] = r;
    }
    if (nchunks > 1) {
        part[(int64_t)q * N + i] = make_double2(num, den);
        return;
    }
    // normal equations of the 1 x 1 least-squares problem; a zero row R_i
    // (pivot <= 1e-14 tr(G) = 0) gives the minimum-norm solution 0
    const double lt = den > 0.0 ? num / den : 0.0;
    if (!LAST)
        for (int o = o0; o < o1; ++o) {
            const int c0 = __ldg(cur_of + o);
            const double e = c0 >= 0 ? Ecur[(int64_t)c0 * N + i] : 0.0;
            Enxt[(int64_t)o * N + i] = e - lt * Enxt[(int64_t)o * N + i];
        }
    const double wi = w[i];
    lam[i] = wi * lt * wi;
}

// Completes rows processed in several chunks: sums the partial inner
// products in chunk order, forms lambda and (unless LAST) updates this
// chunk's entries of E.
template <int DIM, bool LAST>
__global__ void __launch_bounds__(TBX *TBY) k_setup_finish(Grid g, const double *__restrict__ w,
                                                            const double *__restrict__ Ecur, double *__restrict__ Enxt,
                                                            int nnxt, int chunk, int nchunks,
                                                            const int *__restrict__ cur_of, int colour,
                                                            double *__restrict__ lam, const double2 *__restrict__ part) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y;
    const int iz = (int)(blockIdx.z % (unsigned)g.nz), q = (int)(blockIdx.z / (unsigned)g.nz);
    if (ix >= g.nx || iy >= g.ny) return;
    const bool active = colour < 0 || ((((ix + 1) + (iy + 1) + (DIM == 3 ? iz + 1 : 0)) & 1) == colour);
    if (!active) return;
    const int64_t N = g.N;
    const int i = ix + g.nx * (iy + g.ny * iz);
    double num = 0.0, den = 0.0;
    for (int t = 0; t < nchunks; ++t) {
        double2 p = part[(int64_t)t * N + i];
        num += p.x;
        den += p.y;
    }
    const double lt = den > 0.0 ? num / den : 0.0;
    if (q == 0) lam[i] = w[i] * lt * w[i];
    if (LAST) return;
    const int o0 = q * chunk, o1 = min(nnxt, o0 + chunk);
    for (int o = o0; o < o1; ++o) {
        const int c0 = __ldg(cur_of + o);
        const double e = c0 >= 0 ? Ecur[(int64_t)c0 * N + i] : 0.0;
        Enxt[(int64_t)o * N + i] = e - lt * Enxt[(int64_t)o * N + i];
    }
}

template <int DIM, int KIND, bool LAST>
static void launch_setup_rows(const Grid &g, int periodic, const double *At, const double *w, const double *Ecur,
                              double *Enxt, int nn, int chunk, int nchunks, const unsigned *mask, const int *cidx,
                              const int *cur_of, int colour, double *lam, double2 *part, cudaStream_t s) {
    dim3 gr = node_grid(g), bl = node_block();
    gr.z *= nchunks;
    k_setup_rows<DIM, KIND, LAST><<<gr, bl, 0, s>>>(g, periodic, At, w, Ecur, Enxt, nn, chunk, nchunks, mask, cidx,
                                                    cur_of, colour, lam, part);
    count_launch();
    if (nchunks > 1) {
        k_setup_finish<DIM, LAST><<<gr, bl, 0, s>>>(g, w, Ecur, Enxt, nn, chunk, nchunks, cur_of, colour, lam, part);
        count_launch();
    }
}

struct Off3 {
    int x, y, z;
    bool operator<(const Off3 &o) const { return std::tie(z, y, x) < std::tie(o.z, o.y, o.x); }
    bool operator==(const Off3 &o) const { return x == o.x && y == o.y && z == o.z; }
};

template <int DIM, int KIND>
static cs_status setup_level_t(const cs_hierarchy *h, int l, int kind, int nu, int prescale, double *lam,
                               cudaStream_t s, int64_t *peak) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    const Level &L = h->lev[l];
    const Grid g = L.g;
    const int64_t N = g.N;
    const int ncol = kind == CS_MULTIPLICATIVE ? 2 : 1;
    dim3 gr = node_grid(g), bl = node_block();
    double *w = nullptr, *At = nullptr, *Ecur = nullptr, *Enxt = nullptr;
    int *bad = nullptr, *cidx = nullptr, *cur_of = nullptr;
    unsigned *mask = nullptr;
    double2 *part = nullptr;
    cs_status rc = CS_OK;
    int badh = 0;
    std::vector<Off3> Ocur{{0, 0, 0}};
    int64_t live = 0, pk = 0;
    auto track = [&](int64_t d) { live += d; pk = std::max(pk, live); };

    if ((rc = dalloc_t(&w, N, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&At, (size_t)NST * N, nullptr)) != CS_OK) goto done;
    if ((rc = dalloc_t(&bad, 1, nullptr)) != CS_OK) goto done;
    track((int64_t)(NST + 1) * N * 8);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); goto done; }
    k_prescale<DIM, KIND><<<gr, bl, 0, s>>>(g, h->periodic, prescale, L.A, w, At, bad);
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
    k_scale_op<DIM, KIND><<<gr, bl, 0, s>>>(g, h->periodic, L.A, w, At);
    count_launch();
    if ((rc = dalloc_t(&Ecur, N, nullptr)) != CS_OK) goto done;
    track(N * 8);
    k_fill<<<1216, 256, 0, s>>>(N, Ecur, 1.0);
    count_launch();

    for (int lev = 0; lev < nu; ++lev) {
        for (int k = 0; k < ncol; ++k) {
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
            std::vector<int> hci((size_t)nn * NST, 0), hc(nn);
            std::vector<unsigned> hm(nn, 0u);
            for (int o = 0; o < nn; ++o) {
                auto it = idx.find(On[o]);
                hc[o] = it == idx.end() ? -1 : it->second;
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    auto jt = idx.find({On[o].x - dx, On[o].y - dy, On[o].z - dz});
                    if (jt != idx.end()) {
                        hm[o] |= 1u << t;
                        hci[(size_t)o * NST + t] = jt->second;
                    }
                }
            }
            const bool last = lev == nu - 1 && k == ncol - 1;
            // parallelism for small levels: split each row's offsets into chunks
            int nchunks = (int)std::min<int64_t>((524288 + N - 1) / N, (nn + 3) / 4);
            nchunks = std::max(1, std::min(nchunks, 65535 / std::max(1, g.nz)));
            const int chunk = (nn + nchunks - 1) / nchunks;
            nchunks = (nn + chunk - 1) / chunk;
            cudaFree(cidx); cudaFree(cur_of); cudaFree(mask); cudaFree(part);
            cidx = nullptr; cur_of = nullptr; mask = nullptr; part = nullptr;
            if ((rc = dalloc_t(&cidx, hci.size(), nullptr)) != CS_OK) goto done;
            if ((rc = dalloc_t(&cur_of, hc.size(), nullptr)) != CS_OK) goto done;
            if ((rc = dalloc_t(&mask, hm.size(), nullptr)) != CS_OK) goto done;
            if (nchunks > 1 && (rc = dalloc_t(&part, (size_t)nchunks * N, nullptr)) != CS_OK) goto done;
            if (cudaMemcpyAsync(cidx, hci.data(), hci.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(cur_of, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(mask, hm.data(), hm.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "copy setup tables", __FILE__, __LINE__);
                goto done;
            }
            if (!last) {
                if ((rc = dalloc_t(&Enxt, (size_t)nn * N, nullptr)) != CS_OK) goto done;
                track((int64_t)nn * N * 8);
            }
            {
                const int colour = ncol == 2 ? k : -1;
                double *lam_l = lam + (int64_t)lev * N;
                if (last)
                    launch_setup_rows<DIM, KIND, true>(g, h->periodic, At, w, Ecur, Enxt, nn, chunk, nchunks, mask,
                                                       cidx, cur_of, colour, lam_l, part, s);
                else
                    launch_setup_rows<DIM, KIND, false>(g, h->periodic, At, w, Ecur, Enxt, nn, chunk, nchunks, mask,
                                                        cidx, cur_of, colour, lam_l, part, s);
            }
            if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "k_setup_rows", __FILE__, __LINE__); goto done; }
            // the host tables are rebuilt next step: wait for their copies
            if (cudaStreamSynchronize(s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "setup step", __FILE__, __LINE__); goto done; }
            cudaFree(Ecur);
            track(-(int64_t)Ocur.size() * N * 8);
            Ecur = Enxt;
            Enxt = nullptr;
            Ocur.swap(On);
        }
    }
done:
    cudaFree(w); cudaFree(At); cudaFree(Ecur); cudaFree(Enxt); cudaFree(bad); cudaFree(cidx); cudaFree(cur_of);
    cudaFree(mask); cudaFree(part);
    if (peak) *peak = std::max(*peak, pk);
    return rc;
}

cs_status cascade_setup_level(const cs_hierarchy *h, int l, int kind, int nu, int prescale, double *lam,
                              cudaStream_t s, int64_t *peak) {
    const Level &L = h->lev[l];
    if (L.g.dim == 2) {
        if (L.kind == STAR) return setup_level_t<2, STAR>(h, l, kind, nu, prescale, lam, s, peak);
        return setup_level_t<2, BOX>(h, l, kind, nu, prescale, lam, s, peak);
    }
    if (L.kind == STAR) return setup_level_t<3, STAR>(h, l, kind, nu, prescale, lam, s, peak);
    return setup_level_t<3, BOX>(h, l, kind, nu, prescale, lam, s, peak);
}

}  // namespace csx
