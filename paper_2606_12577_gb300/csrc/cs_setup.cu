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
__device__ __forceinline__ int p1d_s(int f, int nc, int *c, double *w) {
    if (f & 1) { c[0] = (f - 1) >> 1; w[0] = 1.0; return 1; }
    int k = 0, lo = (f >> 1) - 1, hi = f >> 1;
    if (lo >= 0) { c[k] = lo; w[k] = 0.5; ++k; }
    if (hi < nc) { c[k] = hi; w[k] = 0.5; ++k; }
    return k;
}

// Ac_{I, I+dJ} = 2^-dim sum_{i,j} P_{i,I} A_{i,j} P_{j,I+dJ}; the result is
// stored as a BOX stencil (dJ in {-1,0,1}^dim).
template <int DIM, int KIND>
__global__ void k_galerkin(Grid gf, Grid gc, const double *__restrict__ Af, double *__restrict__ Ac) {
    using S = StenS<DIM, KIND>;
    constexpr int NC = DIM == 3 ? 27 : 9;
    int cx = blockIdx.x * TBX + threadIdx.x, cy = blockIdx.y * TBY + threadIdx.y, cz = blockIdx.z;
    if (cx >= gc.nx || cy >= gc.ny) return;
    double acc[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) acc[t] = 0.0;
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    for (int ez = zlo; ez <= zhi; ++ez) {
        int fz = DIM == 3 ? 2 * cz + 1 + ez : 0;
        if (DIM == 3 && fz >= gf.nz) continue;
        for (int ey = -1; ey <= 1; ++ey) {
            int fy = 2 * cy + 1 + ey;
            if (fy >= gf.ny) continue;
            for (int ex = -1; ex <= 1; ++ex) {
                int fx = 2 * cx + 1 + ex;
                if (fx >= gf.nx) continue;
                double wr = (ex ? 0.5 : 1.0) * (ey ? 0.5 : 1.0) * (ez ? 0.5 : 1.0);
                int64_t fi = fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz);
                for (int s = 0; s < S::NST; ++s) {
                    int dx, dy, dz;
                    S::off(s, dx, dy, dz);
                    int jx = fx + dx, jy = fy + dy, jz = fz + dz;
                    if (jx < 0 || jx >= gf.nx || jy < 0 || jy >= gf.ny) continue;
                    if (DIM == 3 && (jz < 0 || jz >= gf.nz)) continue;
                    double a = wr * Af[(int64_t)s * gf.N + fi];
                    int Jx[2], Jy[2], Jz[2];
                    double wx[2], wy[2], wz[2];
                    int kx = p1d_s(jx, gc.nx, Jx, wx), ky = p1d_s(jy, gc.ny, Jy, wy), kz = 1;
                    Jz[0] = cz; wz[0] = 1.0;
                    if (DIM == 3) kz = p1d_s(jz, gc.nz, Jz, wz);
                    for (int c = 0; c < kz; ++c)
                        for (int b = 0; b < ky; ++b)
                            for (int q = 0; q < kx; ++q) {
                                int t = (Jx[q] - cx + 1) + 3 * (Jy[b] - cy + 1) + (DIM == 3 ? 9 * (Jz[c] - cz + 1) : 0);
                                acc[t] += a * wx[q] * wy[b] * wz[c];
                            }
                }
            }
        }
    }
    int64_t ci = cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz);
    const double sc = DIM == 3 ? 0.125 : 0.25;
#pragma unroll
    for (int t = 0; t < NC; ++t) Ac[(int64_t)t * gc.N + ci] = sc * acc[t];
}

cs_status galerkin_level(const Level &f, Level &c, cudaStream_t s) {
    dim3 gr = node_grid(c.g), bl = node_block();
    if (f.g.dim == 2) {
        if (f.kind == STAR) k_galerkin<2, STAR><<<gr, bl, 0, s>>>(f.g, c.g, f.A, c.A);
        else k_galerkin<2, BOX><<<gr, bl, 0, s>>>(f.g, c.g, f.A, c.A);
    } else {
        if (f.kind == STAR) k_galerkin<3, STAR><<<gr, bl, 0, s>>>(f.g, c.g, f.A, c.A);
        else k_galerkin<3, BOX><<<gr, bl, 0, s>>>(f.g, c.g, f.A, c.A);
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

// One setup step (l, k): see the file header.  pairs[o'*NST + s] is the
// index in O_cur of o' - offset(s), or -1; cur_of[o'] is the index of o' in
// O_cur or -1.
template <int DIM, int KIND>
__global__ void __launch_bounds__(TBX *TBY) k_setup_step(Grid g, int periodic, const double *__restrict__ At,
                                                          const double *__restrict__ w, const double *__restrict__ Ecur,
                                                          double *__restrict__ Enxt, int nnxt,
                                                          const int *__restrict__ pairs, const int *__restrict__ cur_of,
                                                          int colour, double *__restrict__ lam) {
    using S = StenS<DIM, KIND>;
    constexpr int NST = S::NST;
    int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t N = g.N;
    int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    bool active = colour < 0 || ((((ix + 1) + (iy + 1) + (DIM == 3 ? iz + 1 : 0)) & 1) == colour);
    if (!active) {
        for (int o = 0; o < nnxt; ++o) {
            int c = __ldg(cur_of + o);
            Enxt[(int64_t)o * N + i] = c >= 0 ? Ecur[(int64_t)c * N + i] : 0.0;
        }
        return;
    }
    double a[NST];
    int64_t nb[NST];
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
        nb[s] = in ? jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz) : -1;
        a[s] = At[(int64_t)s * N + i];
    }
    double num = 0.0, den = 0.0;
    for (int o = 0; o < nnxt; ++o) {
        double r = 0.0;
#pragma unroll
        for (int s = 0; s < NST; ++s) {
            int c = __ldg(pairs + o * NST + s);
            if (c >= 0 && nb[s] >= 0) r = fma(a[s], Ecur[(int64_t)c * N + nb[s]], r);
        }
        int c0 = __ldg(cur_of + o);
        double e = c0 >= 0 ? Ecur[(int64_t)c0 * N + i] : 0.0;
        num = fma(e, r, num);
        den = fma(r, r, den);
        Enxt[(int64_t)o * N + i] = r;
    }
    // normal equations of the 1 x 1 least-squares problem; a zero row R_i
    // (pivot <= 1e-14 tr(G) = 0) gives the minimum-norm solution 0
    double lt = den > 0.0 ? num / den : 0.0;
    for (int o = 0; o < nnxt; ++o) {
        int c0 = __ldg(cur_of + o);
        double e = c0 >= 0 ? Ecur[(int64_t)c0 * N + i] : 0.0;
        Enxt[(int64_t)o * N + i] = e - lt * Enxt[(int64_t)o * N + i];
    }
    double wi = w[i];
    lam[i] = wi * lt * wi;
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
    int *bad = nullptr, *pairs = nullptr, *cur_of = nullptr;
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
            std::vector<int> hp(On.size() * NST), hc(On.size());
            for (size_t o = 0; o < On.size(); ++o) {
                auto it = idx.find(On[o]);
                hc[o] = it == idx.end() ? -1 : it->second;
                for (int t = 0; t < NST; ++t) {
                    int dx, dy, dz;
                    S::off(t, dx, dy, dz);
                    auto jt = idx.find({On[o].x - dx, On[o].y - dy, On[o].z - dz});
                    hp[o * NST + t] = jt == idx.end() ? -1 : jt->second;
                }
            }
            int nn = (int)On.size();
            cudaFree(pairs); cudaFree(cur_of);
            pairs = nullptr; cur_of = nullptr;
            if ((rc = dalloc_t(&pairs, hp.size(), nullptr)) != CS_OK) goto done;
            if ((rc = dalloc_t(&cur_of, hc.size(), nullptr)) != CS_OK) goto done;
            if (cudaMemcpyAsync(pairs, hp.data(), hp.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(cur_of, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "copy setup tables", __FILE__, __LINE__);
                goto done;
            }
            if ((rc = dalloc_t(&Enxt, (size_t)nn * N, nullptr)) != CS_OK) goto done;
            track((int64_t)nn * N * 8);
            k_setup_step<DIM, KIND><<<gr, bl, 0, s>>>(g, h->periodic, At, w, Ecur, Enxt, nn, pairs, cur_of,
                                                      ncol == 2 ? k : -1, lam + (int64_t)lev * N);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "k_setup_step", __FILE__, __LINE__); goto done; }
            // the host tables are rewritten next step: wait for the copies
            if (cudaStreamSynchronize(s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "setup step", __FILE__, __LINE__); goto done; }
            cudaFree(Ecur);
            track(-(int64_t)Ocur.size() * N * 8);
            Ecur = Enxt;
            Enxt = nullptr;
            Ocur.swap(On);
        }
    }
done:
    cudaFree(w); cudaFree(At); cudaFree(Ecur); cudaFree(Enxt); cudaFree(bad); cudaFree(pairs); cudaFree(cur_of);
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
