// Stencil kernels of the V-cycle: cascade sweeps (eq. fwda / fwdm and their
// reverse forms), the restricted residual and the interpolated correction of
// Algorithm 1, the bottom-level solve, and FP64 reductions.
//
// One thread per node; x fastest across a warp so that every coefficient
// array A[s][.] is streamed with coalesced loads, and the neighbour reads of
// x hit L1/L2.  These kernels are HBM-bound in FP32 (bytes per node per
// additive step: nst*sizeof(T) + 4*sizeof(T) for A, Lambda, b, x read, x
// written).
#include <algorithm>
#include <type_traits>
#include <cstdint>
#include <cstdio>

#include <cuda_bf16.h>

#include "cs_internal.cuh"

namespace csx {

// canonical stencil offsets -------------------------------------------------
template <int DIM, int KIND>
struct Sten {
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

// Arithmetic type of a storage type: FP64 and FP32 compute in their own
// type, BF16 storage computes in FP32 (FP32 accumulation).
template <typename T> struct AccT { using type = T; };
template <> struct AccT<__nv_bfloat16> { using type = float; };
template <typename T>
__device__ __forceinline__ typename AccT<T>::type ld(T v) { return v; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T st(typename AccT<T>::type v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 st<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T>
__device__ __forceinline__ T zero() { return st<T>(typename AccT<T>::type(0)); }

__device__ __forceinline__ int node_colour(int dim, int ix, int iy, int iz) {
    return ((ix + 1) + (iy + 1) + (dim == 3 ? iz + 1 : 0)) & 1;
}

// (A x)_i at node (ix,iy,iz); neighbours outside the grid contribute nothing
template <int DIM, int KIND, typename T>
__device__ __forceinline__ typename AccT<T>::type apply_row(const Grid &g, const T *__restrict__ A, const T *x, int ix,
                                                            int iy, int iz, int64_t i) {
    using S = Sten<DIM, KIND>;
    using C = typename AccT<T>::type;
    C ax = C(0);
#pragma unroll
    for (int s = 0; s < S::NST; ++s) {
        int dx, dy, dz;
        S::off(s, dx, dy, dz);
        bool in = (unsigned)(ix + dx) < (unsigned)g.nx && (unsigned)(iy + dy) < (unsigned)g.ny &&
                  (DIM == 2 || (unsigned)(iz + dz) < (unsigned)g.nz);
        C a = ld<T>(A[(int64_t)s * g.N + i]);
        C xv = in ? ld<T>(x[i + dx + (int64_t)g.nx * (dy + (int64_t)g.ny * dz)]) : C(0);
        ax = fma(a, xv, ax);
    }
    return ax;
}

// Cascade step: out_i = x_i - lam_i ((A x)_i - b_i).
// COL < 0: every node (additive step, out != x).
// COL >= 0: only nodes of colour `colour`; the others keep x (copied when
// out != x, i.e. snapshot semantics for non-graph colourings).
template <int DIM, int KIND, typename T, bool COLOURED>
__global__ void __launch_bounds__(TBX *TBY) k_sweep(Grid g, const T *__restrict__ A, const T *__restrict__ lam,
                                                     const T *__restrict__ b, const T *x, T *out, int colour,
                                                     int xzero) {
    int ix = blockIdx.x * TBX + threadIdx.x;
    int iy = blockIdx.y * TBY + threadIdx.y;
    int iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    if (COLOURED) {
        if (node_colour(DIM, ix, iy, iz) != colour) {
            if (xzero) out[i] = zero<T>();
            else if (out != x) out[i] = x[i];
            return;
        }
    }
    using C = typename AccT<T>::type;
    C r;
    C xi;
    if (xzero) {
        r = -ld<T>(b[i]);
        xi = C(0);
    } else {
        r = apply_row<DIM, KIND, T>(g, A, x, ix, iy, iz, i) - ld<T>(b[i]);
        xi = ld<T>(x[i]);
    }
    out[i] = st<T>(xi - ld<T>(lam[i]) * r);
}

// ---- 3D 27-point levels with symmetric FP32 storage (Level::sym32):
// Af[k][i] holds entry 13 + k of row i (centre and forward couplings); the
// backward entry s < 13 of row i is the forward entry 26 - s of the
// neighbour j = i + off(s).  Same summation order as apply_row, so only the
// (mirrored) coefficient values can differ from the full copy's.
__device__ __forceinline__ float apply_row_box_sym(const Grid &g, const float *__restrict__ Af, const float *x,
                                                   int ix, int iy, int iz, int64_t i) {
    float ax = 0.f;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        const bool in = (unsigned)(ix + dx) < (unsigned)g.nx && (unsigned)(iy + dy) < (unsigned)g.ny &&
                        (unsigned)(iz + dz) < (unsigned)g.nz;
        const int64_t j = i + dx + (int64_t)g.nx * (dy + (int64_t)g.ny * dz);
        float a = 0.f, xv = 0.f;
        if (s >= 13) a = Af[(int64_t)(s - 13) * g.N + i];
        else if (in) a = Af[(int64_t)(13 - s) * g.N + j];
        if (in) xv = x[j];
        ax = fmaf(a, xv, ax);
    }
    return ax;
}

template <bool COLOURED>
__global__ void __launch_bounds__(TBX *TBY) k_sweep_sym(Grid g, const float *__restrict__ Af,
                                                         const float *__restrict__ lam, const float *__restrict__ b,
                                                         const float *x, float *out, int colour, int xzero) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    if (COLOURED) {
        if (node_colour(3, ix, iy, iz) != colour) {
            if (xzero) out[i] = 0.f;
            else if (out != x) out[i] = x[i];
            return;
        }
    }
    float r, xi;
    if (xzero) {
        r = -b[i];
        xi = 0.f;
    } else {
        r = apply_row_box_sym(g, Af, x, ix, iy, iz, i) - b[i];
        xi = x[i];
    }
    out[i] = xi - lam[i] * r;
}

__global__ void k_d2f_box_sym(int64_t N, const double *__restrict__ A, float *__restrict__ o) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 14 * N; t += (int64_t)gridDim.x * blockDim.x)
        o[t] = (float)A[13 * N + t];
}

cs_status launch_copy_box_sym32(const Level &L, float *o, cudaStream_t s) {
    if (!L.sym32) {
        set_error("internal: symmetric FP32 copy of a level without symmetric storage");
        return CS_ERR_ARG;
    }
    k_d2f_box_sym<<<1216, 256, 0, s>>>(L.g.N, L.A, o);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

// ---- BF16 storage, 3D 7-point additive steps: two x-adjacent nodes per
// thread, every array read as bf16x2 pairs (nx even keeps the pairs 4-byte
// aligned).  With one 2-byte load per array and node the BF16 step issues as
// many requests as the FP32 one for half the bytes and stays request-bound;
// pairs halve the requests.  Per node the arithmetic is k_sweep's, in the
// same order.
__global__ void __launch_bounds__(TBX *TBY) k_sweep_bf16x2(Grid g, const __nv_bfloat16 *__restrict__ A,
                                                            const __nv_bfloat16 *__restrict__ lam,
                                                            const __nv_bfloat16 *__restrict__ b,
                                                            const __nv_bfloat16 *__restrict__ x,
                                                            __nv_bfloat16 *__restrict__ out, int xzero) {
    const int ix = 2 * (blockIdx.x * TBX + threadIdx.x), iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t N = g.N, i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz), sy = g.nx, sz = (int64_t)g.nx * g.ny;
    auto pair = [](const __nv_bfloat16 *p) { return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p)); };
    const float2 bb = pair(b + i), ll = pair(lam + i);
    float2 res;
    if (xzero) {
        res.x = 0.f - ll.x * (-bb.x);  // x = 0: 0 - lam (0 - b)
        res.y = 0.f - ll.y * (-bb.y);
    } else {
        const float2 xc = pair(x + i);
        const float xm = ix > 0 ? __bfloat162float(x[i - 1]) : 0.f;
        const float xp = ix + 2 < g.nx ? __bfloat162float(x[i + 2]) : 0.f;
        const float2 ym = iy > 0 ? pair(x + i - sy) : make_float2(0.f, 0.f);
        const float2 yp = iy + 1 < g.ny ? pair(x + i + sy) : make_float2(0.f, 0.f);
        const float2 zm = iz > 0 ? pair(x + i - sz) : make_float2(0.f, 0.f);
        const float2 zp = iz + 1 < g.nz ? pair(x + i + sz) : make_float2(0.f, 0.f);
        // neighbours in k_sweep's order: centre, -x, +x, -y, +y, -z, +z
        const float n0[7] = {xc.x, xm, xc.y, ym.x, yp.x, zm.x, zp.x};
        const float n1[7] = {xc.y, xc.x, xp, ym.y, yp.y, zm.y, zp.y};
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < 7; ++s2) {
            const float2 a = pair(A + (int64_t)s2 * N + i);
            a0 = fmaf(a.x, n0[s2], a0);
            a1 = fmaf(a.y, n1[s2], a1);
        }
        const float r0 = a0 - bb.x, r1 = a1 - bb.y;
        res.x = xc.x - ll.x * r0;
        res.y = xc.y - ll.y * r1;
    }
    *reinterpret_cast<__nv_bfloat162 *>(out + i) = __floats2bfloat162_rn(res.x, res.y);
}

// ---- FP32, 3D 7-point additive steps: two x-adjacent nodes per thread with
// float2 loads (nx even keeps the pairs 8-byte aligned): half the load
// requests of k_sweep for the same bytes.  Per node the arithmetic is
// k_sweep's, in the same order.
__global__ void __launch_bounds__(TBX *TBY) k_sweep_f32x2(Grid g, const float *__restrict__ A,
                                                           const float *__restrict__ lam, const float *__restrict__ b,
                                                           const float *__restrict__ x, float *__restrict__ out,
                                                           int xzero) {
    const int ix = 2 * (blockIdx.x * TBX + threadIdx.x), iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t N = g.N, i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz), sy = g.nx, sz = (int64_t)g.nx * g.ny;
    auto pair = [](const float *p) { return *reinterpret_cast<const float2 *>(p); };
    const float2 bb = pair(b + i), ll = pair(lam + i);
    float2 res;
    if (xzero) {
        res.x = 0.f - ll.x * (-bb.x);  // x = 0: 0 - lam (0 - b)
        res.y = 0.f - ll.y * (-bb.y);
    } else {
        const float2 xc = pair(x + i);
        const float xm = ix > 0 ? x[i - 1] : 0.f;
        const float xp = ix + 2 < g.nx ? x[i + 2] : 0.f;
        const float2 ym = iy > 0 ? pair(x + i - sy) : make_float2(0.f, 0.f);
        const float2 yp = iy + 1 < g.ny ? pair(x + i + sy) : make_float2(0.f, 0.f);
        const float2 zm = iz > 0 ? pair(x + i - sz) : make_float2(0.f, 0.f);
        const float2 zp = iz + 1 < g.nz ? pair(x + i + sz) : make_float2(0.f, 0.f);
        // neighbours in k_sweep's order: centre, -x, +x, -y, +y, -z, +z
        const float n0[7] = {xc.x, xm, xc.y, ym.x, yp.x, zm.x, zp.x};
        const float n1[7] = {xc.y, xc.x, xp, ym.y, yp.y, zm.y, zp.y};
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < 7; ++s2) {
            const float2 a = pair(A + (int64_t)s2 * N + i);
            a0 = fmaf(a.x, n0[s2], a0);
            a1 = fmaf(a.y, n1[s2], a1);
        }
        const float r0 = a0 - bb.x, r1 = a1 - bb.y;
        res.x = xc.x - ll.x * r0;
        res.y = xc.y - ll.y * r1;
    }
    *reinterpret_cast<float2 *>(out + i) = res;
}

template <typename T, bool COLOURED>
static cs_status sweep_dispatch(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out,
                                int colour, bool xzero, cudaStream_t s) {
    dim3 gr = node_grid(L.g), bl = node_block();
    int xz = xzero ? 1 : 0;
    // the paired kernels load two values at once: every array must be aligned
    // to two elements (caller-given vectors may be views at an odd offset)
    auto pairs_aligned = [&](size_t bytes) {
        const uintptr_t m = (uintptr_t)A | (uintptr_t)lam | (uintptr_t)b | (uintptr_t)x | (uintptr_t)out;
        return (m % bytes) == 0;
    };
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if (!COLOURED && L.g.dim == 3 && L.kind == STAR && L.g.nx % 2 == 0 && out != x && pairs_aligned(4)) {
            const dim3 g2((unsigned)((L.g.nx / 2 + TBX - 1) / TBX), gr.y, gr.z);
            k_sweep_bf16x2<<<g2, bl, 0, s>>>(L.g, A, lam, b, x, out, xz);
            CSX_CUDA(cudaGetLastError());
            count_launch();
            return CS_OK;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (!COLOURED && L.g.dim == 3 && L.kind == STAR && L.g.nx % 2 == 0 && out != x && pairs_aligned(8)) {
            const dim3 g2((unsigned)((L.g.nx / 2 + TBX - 1) / TBX), gr.y, gr.z);
            k_sweep_f32x2<<<g2, bl, 0, s>>>(L.g, A, lam, b, x, out, xz);
            CSX_CUDA(cudaGetLastError());
            count_launch();
            return CS_OK;
        }
        if (L.sym32) {  // FP32 operators of these levels are stored symmetric
            k_sweep_sym<COLOURED><<<gr, bl, 0, s>>>(L.g, A, lam, b, x, out, colour, xz);
            CSX_CUDA(cudaGetLastError());
            count_launch();
            return CS_OK;
        }
    }
    if (L.g.dim == 2) {
        if (L.kind == STAR) k_sweep<2, STAR, T, COLOURED><<<gr, bl, 0, s>>>(L.g, A, lam, b, x, out, colour, xz);
        else k_sweep<2, BOX, T, COLOURED><<<gr, bl, 0, s>>>(L.g, A, lam, b, x, out, colour, xz);
    } else {
        if (L.kind == STAR) k_sweep<3, STAR, T, COLOURED><<<gr, bl, 0, s>>>(L.g, A, lam, b, x, out, colour, xz);
        else k_sweep<3, BOX, T, COLOURED><<<gr, bl, 0, s>>>(L.g, A, lam, b, x, out, colour, xz);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

template <typename T>
cs_status launch_sweep(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out, int colour,
                       bool x_is_zero, cudaStream_t s) {
    if (colour < 0) return sweep_dispatch<T, false>(L, A, lam, b, x, out, -1, x_is_zero, s);
    return sweep_dispatch<T, true>(L, A, lam, b, x, out, colour, x_is_zero, s);
}
template cs_status launch_sweep<double>(const Level &, const double *, const double *, const double *,
                                        const double *, double *, int, bool, cudaStream_t);
template cs_status launch_sweep<float>(const Level &, const float *, const float *, const float *, const float *,
                                       float *, int, bool, cudaStream_t);
template cs_status launch_sweep<__nv_bfloat16>(const Level &, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                               const __nv_bfloat16 *, const __nv_bfloat16 *, __nv_bfloat16 *, int, bool,
                                               cudaStream_t);

// ------------------------------------------------------------ block steps
// Nodes of block (bx,by,bz): bs*b + l per axis, local position
// lp = lx + bs (ly + bs lz); partial blocks at the upper edges skip absent
// positions.  Lambda_b is nmax x nmax over local positions.
template <int DIM, int NMAX>
__device__ __forceinline__ int block_nodes(const Grid &g, int bs, int bx, int by, int bz, int *node, int *lpos,
                                           int (*co)[3]) {
    int np = 0;
    for (int lp = 0; lp < NMAX; ++lp) {
        const int lx = lp % bs, ly = (lp / bs) % bs, lz = DIM == 3 ? lp / (bs * bs) : 0;
        if (DIM == 2 && lp >= bs * bs) break;
        const int ix = bs * bx + lx, iy = bs * by + ly, iz = DIM == 3 ? bs * bz + lz : 0;
        if (ix >= g.nx || iy >= g.ny || (DIM == 3 && iz >= g.nz)) continue;
        node[np] = ix + g.nx * (iy + g.ny * iz);
        lpos[np] = lp;
        co[np][0] = ix; co[np][1] = iy; co[np][2] = iz;
        ++np;
    }
    return np;
}

// out_b = x_b - Lambda_b^(T) ((A x)_b - b_b), one thread per block
template <int DIM, int KIND, typename T, int NMAX, bool COLOURED>
__global__ void k_block_sweep(Grid g, int bs, int nbx, int nby, int64_t nblocks, const T *__restrict__ A,
                              const T *__restrict__ lam, const T *__restrict__ b, const T *x, T *out, int colour,
                              int transpose, int xzero) {
    const int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (blk >= nblocks) return;
    const int bx = (int)(blk % nbx), by = (int)((blk / nbx) % nby), bz = (int)(blk / ((int64_t)nbx * nby));
    int node[NMAX], lpos[NMAX], co[NMAX][3];
    const int np = block_nodes<DIM, NMAX>(g, bs, bx, by, bz, node, lpos, co);
    if (COLOURED && ((((bx + 1) + (by + 1) + (DIM == 3 ? bz + 1 : 0)) & 1) != colour)) {
        for (int p = 0; p < np; ++p) {
            if (xzero) out[node[p]] = T(0);
            else if (out != x) out[node[p]] = x[node[p]];
        }
        return;
    }
    T r[NMAX];
    for (int p = 0; p < np; ++p)
        r[p] = (xzero ? T(0) : apply_row<DIM, KIND, T>(g, A, x, co[p][0], co[p][1], co[p][2], node[p])) - b[node[p]];
    const T *lb = lam + blk * (NMAX * NMAX);
    T xo[NMAX];
    for (int p = 0; p < np; ++p) {
        T acc = xzero ? T(0) : x[node[p]];
        for (int q = 0; q < np; ++q)
            acc = fma(-(transpose ? lb[lpos[q] * NMAX + lpos[p]] : lb[lpos[p] * NMAX + lpos[q]]), r[q], acc);
        xo[p] = acc;
    }
    for (int p = 0; p < np; ++p) out[node[p]] = xo[p];
}

template <typename T>
cs_status launch_block_sweep(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out, int colour,
                             bool transpose, bool xzero, cudaStream_t s) {
    const int threads = 128;
    const unsigned nblk = (unsigned)((L.nblocks + threads - 1) / threads);
    const int tr = transpose ? 1 : 0, xz = xzero ? 1 : 0;
#define CSX_BSW(DIM, KIND, NM)                                                                                   \
    if (colour < 0)                                                                                              \
        k_block_sweep<DIM, KIND, T, NM, false><<<nblk, threads, 0, s>>>(L.g, L.bs, L.nbx, L.nby, L.nblocks, A, lam, \
                                                                         b, x, out, colour, tr, xz);              \
    else                                                                                                         \
        k_block_sweep<DIM, KIND, T, NM, true><<<nblk, threads, 0, s>>>(L.g, L.bs, L.nbx, L.nby, L.nblocks, A, lam, \
                                                                        b, x, out, colour, tr, xz);
    if (L.g.dim == 2) {
        if (L.nmax <= 4) { if (L.kind == STAR) { CSX_BSW(2, STAR, 4) } else { CSX_BSW(2, BOX, 4) } }
        else { if (L.kind == STAR) { CSX_BSW(2, STAR, 9) } else { CSX_BSW(2, BOX, 9) } }
    } else {
        if (L.kind == STAR) { CSX_BSW(3, STAR, 8) } else { CSX_BSW(3, BOX, 8) }
    }
#undef CSX_BSW
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
template cs_status launch_block_sweep<double>(const Level &, const double *, const double *, const double *,
                                              const double *, double *, int, bool, bool, cudaStream_t);
template cs_status launch_block_sweep<float>(const Level &, const float *, const float *, const float *, const float *,
                                             float *, int, bool, bool, cudaStream_t);
// BF16 storage is implemented for point-block levels only
template <>
cs_status launch_block_sweep<__nv_bfloat16>(const Level &, const __nv_bfloat16 *, const __nv_bfloat16 *,
                                            const __nv_bfloat16 *, const __nv_bfloat16 *, __nv_bfloat16 *, int, bool,
                                            bool, cudaStream_t) {
    set_error("BF16 cycles are implemented for point-block levels only");
    return CS_ERR_UNSUPPORTED;
}

// The multi-RHS block step X_b <- X_b - Lambda_b^(T) (A X - B)_b.  One warp
// per node of a block (lane r = right-hand side r, so every load of X and B
// is a contiguous row of m values); the residual rows of a block meet in
// shared memory and, after one barrier, each warp forms its node's row of the
// n_b x m block product.  Per RHS and unknown this is nst + n_b FMAs against
// (nst + n_b + 3 m) words moved: HBM-bound, so plain FMAs, no tensor cores.
// BPC blocks adjacent in x share a CTA of 32 * NMAX * BPC threads; the grid
// spans the block grid (x tiles of BPC, y, z), so no index division is needed.
template <int DIM, int KIND, typename T, int BS, int BPC>
__global__ void __launch_bounds__(32 * (DIM == 3 ? BS * BS * BS : BS * BS) * BPC)
    k_block_sweep_m(Grid g, int nbx, const T *__restrict__ A, const T *__restrict__ lam, const T *__restrict__ B,
                    const T *X, T *out, int m, int colour, int transpose) {
    using S = Sten<DIM, KIND>;
    constexpr int NMAX = DIM == 3 ? BS * BS * BS : BS * BS;
    __shared__ T rsm[BPC][NMAX][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bl = warp / NMAX, lp = warp % NMAX;  // compile-time divisors
    const int bx = blockIdx.x * BPC + bl, by = blockIdx.y, bz = blockIdx.z;
    const int lx = lp % BS, ly = (lp / BS) % BS, lz = DIM == 3 ? lp / (BS * BS) : 0;
    const int ix = BS * bx + lx, iy = BS * by + ly, iz = DIM == 3 ? BS * bz + lz : 0;
    const bool present = bx < nbx && ix < g.nx && iy < g.ny && (DIM == 2 || iz < g.nz);
    const bool active = colour < 0 || ((((bx + 1) + (by + 1) + (DIM == 3 ? bz + 1 : 0)) & 1) == colour);
    const bool work = present && lane < m;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    T r = T(0);
    if (work && active) {
        T ax = T(0);
#pragma unroll
        for (int s = 0; s < S::NST; ++s) {
            int dx, dy, dz;
            S::off(s, dx, dy, dz);
            const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
            const bool in = (unsigned)jx < (unsigned)g.nx && (unsigned)jy < (unsigned)g.ny &&
                            (DIM == 2 || (unsigned)jz < (unsigned)g.nz);
            const int64_t j = i + dx + (int64_t)g.nx * (dy + (int64_t)g.ny * dz);
            ax = fma(A[(int64_t)s * g.N + i], in ? X[j * m + lane] : T(0), ax);
        }
        r = ax - B[i * m + lane];
    }
    rsm[bl][lp][lane] = r;  // absent nodes contribute zero (their Lambda entries are zero too)
    __syncthreads();
    if (!work) return;
    if (!active) {
        if (out != X) out[i * m + lane] = X[i * m + lane];
        return;
    }
    const int64_t blk = bx + (int64_t)nbx * (by + (int64_t)gridDim.y * bz);
    const T *lb = lam + blk * (NMAX * NMAX);
    T acc = X[i * m + lane];
#pragma unroll
    for (int q = 0; q < NMAX; ++q)
        acc = fma(-(transpose ? lb[q * NMAX + lp] : lb[lp * NMAX + q]), rsm[bl][q][lane], acc);
    out[i * m + lane] = acc;
}

// The same block step in FP32 with four right-hand sides per lane (float4),
// for m = 4 LPN right-hand sides and blocks of NMAX nodes with NMAX LPN
// dividing 32: a warp holds 32 / (NMAX LPN) whole blocks, lane l takes node
// (l / LPN) % NMAX of its block and right-hand sides 4 (l % LPN) .. +3.  Every
// load of a step (coefficients, the x neighbourhood, b and the Lambda row) is
// issued before the first use, the block's residuals meet through warp
// shuffles (no CTA barrier), and warps stride over the blocks.  Per RHS and
// node the arithmetic and its order are those of k_block_sweep_m.
template <int DIM, int KIND, int BS, int LPN>
__global__ void __launch_bounds__(256) k_block_sweep_m4(Grid g, int nbx, int nby, int64_t nblocks,
                                                        const float *__restrict__ A, const float *__restrict__ lam,
                                                        const float4 *__restrict__ B, const float4 *X, float4 *out,
                                                        int colour, int transpose) {
    using S = Sten<DIM, KIND>;
    constexpr int NMAX = DIM == 3 ? BS * BS * BS : BS * BS;
    constexpr int G = NMAX * LPN;  // lanes per block
    constexpr int BPW = 32 / G;    // blocks per warp
    const int lane = threadIdx.x & 31;
    const int gsub = lane / G, lp = (lane % G) / LPN, rg = lane % LPN;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lx = lp % BS, ly = (lp / BS) % BS, lz = DIM == 3 ? lp / (BS * BS) : 0;
    // block and node indices fit in 31 bits (the hierarchy checks N < 2^31): 32-bit index arithmetic
    for (int64_t w = warp0; w * BPW < nblocks; w += nwarps) {
        const int blk = (int)(w * BPW) + gsub;
        const bool valid = blk < nblocks;
        int bx = 0, by = 0, bz = 0;
        if (valid) {
            const int q = blk / nbx;
            bx = blk - q * nbx;
            if (DIM == 3) {
                bz = q / nby;
                by = q - bz * nby;
            } else {
                by = q;
            }
        }
        const int ix = BS * bx + lx, iy = BS * by + ly, iz = DIM == 3 ? BS * bz + lz : 0;
        const bool present = valid && ix < g.nx && iy < g.ny && (DIM == 2 || iz < g.nz);
        const bool active = colour < 0 || ((((bx + 1) + (by + 1) + (DIM == 3 ? bz + 1 : 0)) & 1) == colour);
        const int i = ix + g.nx * (iy + g.ny * iz);
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f), xo = r;
        float lrow[NMAX];
        if (present && active) {
            const float *lb = lam + (int64_t)blk * (NMAX * NMAX);
#pragma unroll
            for (int q = 0; q < NMAX; ++q) lrow[q] = transpose ? lb[q * NMAX + lp] : lb[lp * NMAX + q];
            float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int s = 0; s < S::NST; ++s) {
                int dx, dy, dz;
                S::off(s, dx, dy, dz);
                const bool in = (unsigned)(ix + dx) < (unsigned)g.nx && (unsigned)(iy + dy) < (unsigned)g.ny &&
                                (DIM == 2 || (unsigned)(iz + dz) < (unsigned)g.nz);
                const int j = i + dx + g.nx * (dy + g.ny * dz);
                const float a = A[(int64_t)s * g.N + i];
                const float4 xv = in ? X[(int64_t)j * LPN + rg] : make_float4(0.f, 0.f, 0.f, 0.f);
                if (dx == 0 && dy == 0 && dz == 0) xo = xv;
                ax.x = fmaf(a, xv.x, ax.x);
                ax.y = fmaf(a, xv.y, ax.y);
                ax.z = fmaf(a, xv.z, ax.z);
                ax.w = fmaf(a, xv.w, ax.w);
            }
            const float4 bv = B[(int64_t)i * LPN + rg];
            r = make_float4(ax.x - bv.x, ax.y - bv.y, ax.z - bv.z, ax.w - bv.w);
        } else if (present) {
            xo = X[(int64_t)i * LPN + rg];
        }
        // residuals of the block's nodes (absent nodes: 0, their Lambda entries are 0 too)
        float4 acc = xo;
        const int base = gsub * G + rg;
#pragma unroll
        for (int q = 0; q < NMAX; ++q) {
            const float rx = __shfl_sync(0xffffffffu, r.x, base + q * LPN);
            const float ry = __shfl_sync(0xffffffffu, r.y, base + q * LPN);
            const float rz = __shfl_sync(0xffffffffu, r.z, base + q * LPN);
            const float rw = __shfl_sync(0xffffffffu, r.w, base + q * LPN);
            if (present && active) {
                acc.x = fmaf(-lrow[q], rx, acc.x);
                acc.y = fmaf(-lrow[q], ry, acc.y);
                acc.z = fmaf(-lrow[q], rz, acc.z);
                acc.w = fmaf(-lrow[q], rw, acc.w);
            }
        }
        if (present && (active || out != X)) out[(int64_t)i * LPN + rg] = acc;
    }
}

template <typename T>
cs_status launch_block_sweep_m(const Level &L, const T *A, const T *lam, const T *b, const T *x, T *out, int m,
                               int colour, bool transpose, cudaStream_t s) {
    const int tr = transpose ? 1 : 0;
    if (sizeof(T) == sizeof(float) && m % 4 == 0 && L.bs == 2 && L.nmax * (m / 4) <= 32 &&
        32 % (L.nmax * (m / 4)) == 0 && ((uintptr_t)b | (uintptr_t)x | (uintptr_t)out) % 16 == 0) {
        const int lpn = m / 4, bpw = 32 / (L.nmax * lpn);
        const int64_t warps = (L.nblocks + bpw - 1) / bpw;
        int dev = 0, nsm = 0;
        CSX_CUDA(cudaGetDevice(&dev));
        CSX_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const float *Af = reinterpret_cast<const float *>(A), *lf = reinterpret_cast<const float *>(lam);
        const float4 *b4 = reinterpret_cast<const float4 *>(b), *x4 = reinterpret_cast<const float4 *>(x);
        float4 *o4 = reinterpret_cast<float4 *>(out);
        // one wave: as many CTAs as can be resident, so that no partial wave trails the strided loop
#define CSX_BSM4_LAUNCH(DIM, KIND, LPN)                                                                          \
    do {                                                                                                         \
        int per = 0;                                                                                             \
        CSX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_block_sweep_m4<DIM, KIND, 2, LPN>, 256, 0)); \
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8,                 \
                                                                               (int64_t)nsm * std::max(per, 1))); \
        k_block_sweep_m4<DIM, KIND, 2, LPN><<<grid, 256, 0, s>>>(L.g, L.nbx, L.nby, L.nblocks, Af, lf, b4, x4, o4,  \
                                                                 colour, tr);                                    \
    } while (0)
#define CSX_BSM4(DIM, LPN)                                                                                       \
    do {                                                                                                         \
        if (L.kind == STAR) CSX_BSM4_LAUNCH(DIM, STAR, LPN);                                                     \
        else CSX_BSM4_LAUNCH(DIM, BOX, LPN);                                                                     \
    } while (0)
        if (L.g.dim == 2) {
            if (lpn == 1) CSX_BSM4(2, 1);
            else if (lpn == 2) CSX_BSM4(2, 2);
            else if (lpn == 4) CSX_BSM4(2, 4);
            else CSX_BSM4(2, 8);
        } else {
            if (lpn == 1) CSX_BSM4(3, 1);
            else if (lpn == 2) CSX_BSM4(3, 2);
            else CSX_BSM4(3, 4);
        }
#undef CSX_BSM4
#undef CSX_BSM4_LAUNCH
        CSX_CUDA(cudaGetLastError());
        count_launch();
        return CS_OK;
    }
#define CSX_BSM(DIM, KIND, BS, BPC)                                                                              \
    k_block_sweep_m<DIM, KIND, T, BS, BPC>                                                                       \
        <<<dim3((unsigned)((L.nbx + BPC - 1) / BPC), (unsigned)L.nby, (unsigned)L.nbz),                          \
           32 * (DIM == 3 ? BS * BS * BS : BS * BS) * BPC, 0, s>>>(L.g, L.nbx, A, lam, b, x, out, m, colour, tr);
    if (L.g.dim == 2) {
        if (L.bs == 1) { if (L.kind == STAR) { CSX_BSM(2, STAR, 1, 8) } else { CSX_BSM(2, BOX, 1, 8) } }
        else if (L.bs == 2) { if (L.kind == STAR) { CSX_BSM(2, STAR, 2, 2) } else { CSX_BSM(2, BOX, 2, 2) } }
        else { if (L.kind == STAR) { CSX_BSM(2, STAR, 3, 1) } else { CSX_BSM(2, BOX, 3, 1) } }
    } else {
        if (L.bs == 1) { if (L.kind == STAR) { CSX_BSM(3, STAR, 1, 8) } else { CSX_BSM(3, BOX, 1, 8) } }
        else { if (L.kind == STAR) { CSX_BSM(3, STAR, 2, 1) } else { CSX_BSM(3, BOX, 2, 1) } }
    }
#undef CSX_BSM
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
template cs_status launch_block_sweep_m<double>(const Level &, const double *, const double *, const double *,
                                                const double *, double *, int, int, bool, cudaStream_t);
template cs_status launch_block_sweep_m<float>(const Level &, const float *, const float *, const float *,
                                               const float *, float *, int, int, bool, cudaStream_t);

// rc_I = 2^-dim sum_f P_{f,I} (A x - b)_f.  Coarse node I sits on fine node
// 2I+1 (0-based); its fine neighbours 2I+1+d (d in {-1,0,1}) carry weight
// 1/2 per nonzero component of d (bilinear / trilinear interpolation).
template <int DIM, int KIND, typename T>
__global__ void __launch_bounds__(TBX *TBY) k_res_restrict(Grid gf, Grid gc, const T *__restrict__ A,
                                                            const T *__restrict__ b, const T *__restrict__ x,
                                                            T *__restrict__ rc) {
    int cx = blockIdx.x * TBX + threadIdx.x;
    int cy = blockIdx.y * TBY + threadIdx.y;
    int cz = blockIdx.z;
    if (cx >= gc.nx || cy >= gc.ny) return;
    using C = typename AccT<T>::type;
    C acc = C(0);
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int fz = DIM == 3 ? 2 * cz + 1 + dz : 0;
        if (DIM == 3 && fz >= gf.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int fy = 2 * cy + 1 + dy;
            if (fy >= gf.ny) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                int fx = 2 * cx + 1 + dx;
                if (fx >= gf.nx) continue;
                C w = C((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
                int64_t f = fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz);
                C r = apply_row<DIM, KIND, T>(gf, A, x, fx, fy, fz, f) - ld<T>(b[f]);
                acc = fma(w, r, acc);
            }
        }
    }
    rc[cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz)] = st<T>(acc * C(DIM == 3 ? 0.125 : 0.25));
}

// Two-pass form of the same restriction for FP32 / FP64 storage: every fine
// residual (A x - b)_f once into a fine-level scratch vector, then each
// coarse node gathers its 3^dim window from it in the one-pass kernel's
// order.  The one-pass kernel recomputes a fine residual for each of the up
// to 2^dim coarse nodes whose window holds it; on 256^3 it ran at a third of
// the fine level's bandwidth.
template <int DIM, int KIND, typename T>
__global__ void __launch_bounds__(TBX *TBY) k_fine_residual(Grid g, const T *__restrict__ A, const T *__restrict__ b,
                                                             const T *__restrict__ x, T *__restrict__ r) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    r[i] = apply_row<DIM, KIND, T>(g, A, x, ix, iy, iz, i) - b[i];
}

__global__ void __launch_bounds__(TBX *TBY) k_fine_residual_sym(Grid g, const float *__restrict__ Af,
                                                                 const float *__restrict__ b,
                                                                 const float *__restrict__ x, float *__restrict__ r) {
    const int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    const int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    r[i] = apply_row_box_sym(g, Af, x, ix, iy, iz, i) - b[i];
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TBX *TBY) k_restrict_gather(Grid gf, Grid gc, const T *__restrict__ r,
                                                               T *__restrict__ rc) {
    const int cx = blockIdx.x * TBX + threadIdx.x, cy = blockIdx.y * TBY + threadIdx.y, cz = blockIdx.z;
    if (cx >= gc.nx || cy >= gc.ny) return;
    T acc = T(0);
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int fz = DIM == 3 ? 2 * cz + 1 + dz : 0;
        if (DIM == 3 && fz >= gf.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int fy = 2 * cy + 1 + dy;
            if (fy >= gf.ny) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int fx = 2 * cx + 1 + dx;
                if (fx >= gf.nx) continue;
                const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
                acc = fma(w, r[fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz)], acc);
            }
        }
    }
    rc[cx + (int64_t)gc.nx * (cy + (int64_t)gc.ny * cz)] = acc * T(DIM == 3 ? 0.125 : 0.25);
}

template <typename T>
cs_status launch_residual_restrict(const Level &f, const Level &c, const T *A, const T *b, const T *x, T *rc,
                                   T *scratch, cudaStream_t s) {
    dim3 gr = node_grid(c.g), bl = node_block();
    if (std::is_same<T, float>::value && f.sym32 && !scratch) {
        set_error("internal: the restriction from a symmetric FP32 level needs a scratch vector");
        return CS_ERR_ARG;
    }
    if constexpr (std::is_same<T, float>::value || std::is_same<T, double>::value) {
        if (scratch) {
            const dim3 gf = node_grid(f.g);
            if (std::is_same<T, float>::value && f.sym32) {
                k_fine_residual_sym<<<gf, bl, 0, s>>>(f.g, (const float *)A, (const float *)b, (const float *)x,
                                                      (float *)scratch);
                k_restrict_gather<3, T><<<gr, bl, 0, s>>>(f.g, c.g, scratch, rc);
            } else if (f.g.dim == 2) {
                if (f.kind == STAR) k_fine_residual<2, STAR, T><<<gf, bl, 0, s>>>(f.g, A, b, x, scratch);
                else k_fine_residual<2, BOX, T><<<gf, bl, 0, s>>>(f.g, A, b, x, scratch);
                k_restrict_gather<2, T><<<gr, bl, 0, s>>>(f.g, c.g, scratch, rc);
            } else {
                if (f.kind == STAR) k_fine_residual<3, STAR, T><<<gf, bl, 0, s>>>(f.g, A, b, x, scratch);
                else k_fine_residual<3, BOX, T><<<gf, bl, 0, s>>>(f.g, A, b, x, scratch);
                k_restrict_gather<3, T><<<gr, bl, 0, s>>>(f.g, c.g, scratch, rc);
            }
            CSX_CUDA(cudaGetLastError());
            count_launch(2);
            return CS_OK;
        }
    }
    if (f.g.dim == 2) {
        if (f.kind == STAR) k_res_restrict<2, STAR, T><<<gr, bl, 0, s>>>(f.g, c.g, A, b, x, rc);
        else k_res_restrict<2, BOX, T><<<gr, bl, 0, s>>>(f.g, c.g, A, b, x, rc);
    } else {
        if (f.kind == STAR) k_res_restrict<3, STAR, T><<<gr, bl, 0, s>>>(f.g, c.g, A, b, x, rc);
        else k_res_restrict<3, BOX, T><<<gr, bl, 0, s>>>(f.g, c.g, A, b, x, rc);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
template cs_status launch_residual_restrict<double>(const Level &, const Level &, const double *, const double *,
                                                    const double *, double *, double *, cudaStream_t);
template cs_status launch_residual_restrict<float>(const Level &, const Level &, const float *, const float *,
                                                   const float *, float *, float *, cudaStream_t);
template cs_status launch_residual_restrict<__nv_bfloat16>(const Level &, const Level &, const __nv_bfloat16 *,
                                                           const __nv_bfloat16 *, const __nv_bfloat16 *,
                                                           __nv_bfloat16 *, __nv_bfloat16 *, cudaStream_t);

// 1D interpolation weights of fine node f (0-based) from coarse nodes: an
// odd f coincides with coarse (f-1)/2; an even f takes half of coarse f/2-1
// and f/2 (those inside the coarse grid).
__device__ __forceinline__ int p1d(int f, int nc, int *c, float *w) {
    if (f & 1) {
        c[0] = (f - 1) >> 1; w[0] = 1.f;
        return 1;
    }
    int k = 0, lo = (f >> 1) - 1, hi = f >> 1;
    if (lo >= 0) { c[k] = lo; w[k] = 0.5f; ++k; }
    if (hi < nc) { c[k] = hi; w[k] = 0.5f; ++k; }
    return k;
}

// xo_f = x_f - sum_I P_{f,I} xc_I, one thread per coarse cell: cell j of an
// axis holds the fine nodes 2j (between coarse nodes j - 1 and j, weights
// 1/2, a node outside the grid dropped) and 2j + 1 (on coarse node j, weight
// 1).  The thread loads the cell's up to 2^d coarse corners once, all at
// once, and forms each of its up to 2^d fine nodes with the products in the
// order of the per-node definition (z outer, then y, then x; weight
// wx wy wz rounded once), so every fine value is the one a per-node loop
// gives.  A per-node thread issued its up to 2^d coarse reads one after the
// other and was latency bound.
template <int DIM, typename T>
__global__ void __launch_bounds__(TBX *TBY) k_prolong(Grid gf, Grid gc, const T *__restrict__ xc, const T *x,
                                                       T *xo) {
    using C = typename AccT<T>::type;
    const int jx = blockIdx.x * TBX + threadIdx.x, jy = blockIdx.y * TBY + threadIdx.y, jz = blockIdx.z;
    if (2 * jx >= gf.nx || 2 * jy >= gf.ny) return;
    // corner d of an axis: coarse node j - 1 (d = 0) or j (d = 1)
    const int cx[2] = {jx - 1, jx}, cy[2] = {jy - 1, jy}, cz[2] = {DIM == 3 ? jz - 1 : 0, DIM == 3 ? jz : 0};
    auto okx = [&](int d) { return cx[d] >= 0 && cx[d] < gc.nx; };
    auto oky = [&](int d) { return cy[d] >= 0 && cy[d] < gc.ny; };
    auto okz = [&](int d) { return DIM == 3 ? (cz[d] >= 0 && cz[d] < gc.nz) : d == 1; };
    C v[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx)
                v[dz][dy][dx] = (okx(dx) && oky(dy) && okz(dz))
                                    ? ld<T>(xc[cx[dx] + (int64_t)gc.nx * (cy[dy] + (int64_t)gc.ny * cz[dz])])
                                    : C(0);
    // fine node e of an axis (0: 2j, 1: 2j + 1) takes corner d when
    // e == 1 ? d == 1 : the corner is inside the grid, with weight 1 or 1/2;
    // the corners run in ascending d, as in the per-node definition
#pragma unroll
    for (int ez = 0; ez < (DIM == 3 ? 2 : 1); ++ez) {
        const int fz = DIM == 3 ? 2 * jz + ez : jz;
        if (fz >= gf.nz) continue;
#pragma unroll
        for (int ey = 0; ey < 2; ++ey) {
            const int fy = 2 * jy + ey;
            if (fy >= gf.ny) continue;
#pragma unroll
            for (int ex = 0; ex < 2; ++ex) {
                const int fx = 2 * jx + ex;
                if (fx >= gf.nx) continue;
                C acc = C(0);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const bool uz = DIM == 3 ? (ez == 1 ? dz == 1 : okz(dz)) : dz == 1;
                    const float wz = (DIM == 3 && ez == 0) ? 0.5f : 1.f;
                    if (!uz) continue;
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const bool uy = ey == 1 ? dy == 1 : oky(dy);
                        const float wy = ey == 0 ? 0.5f : 1.f;
                        if (!uy) continue;
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const bool ux = ex == 1 ? dx == 1 : okx(dx);
                            const float wx = ex == 0 ? 0.5f : 1.f;
                            if (!ux) continue;
                            acc = fma(C(wx * wy * wz), v[dz][dy][dx], acc);
                        }
                    }
                }
                const int64_t f = fx + (int64_t)gf.nx * (fy + (int64_t)gf.ny * fz);
                xo[f] = st<T>(ld<T>(x[f]) - acc);
            }
        }
    }
}

template <typename T>
cs_status launch_prolong_correct(const Level &f, const Level &c, const T *xc, const T *x, T *xo, cudaStream_t s) {
    const int cxn = (f.g.nx + 1) / 2, cyn = (f.g.ny + 1) / 2, czn = f.g.dim == 3 ? (f.g.nz + 1) / 2 : f.g.nz;
    dim3 gr((unsigned)((cxn + TBX - 1) / TBX), (unsigned)((cyn + TBY - 1) / TBY), (unsigned)czn), bl = node_block();
    if (f.g.dim == 2) k_prolong<2, T><<<gr, bl, 0, s>>>(f.g, c.g, xc, x, xo);
    else k_prolong<3, T><<<gr, bl, 0, s>>>(f.g, c.g, xc, x, xo);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
template cs_status launch_prolong_correct<double>(const Level &, const Level &, const double *, const double *,
                                                  double *, cudaStream_t);
template cs_status launch_prolong_correct<float>(const Level &, const Level &, const float *, const float *,
                                                 float *, cudaStream_t);
template cs_status launch_prolong_correct<__nv_bfloat16>(const Level &, const Level &, const __nv_bfloat16 *,
                                                         const __nv_bfloat16 *, __nv_bfloat16 *, cudaStream_t);

// block-wide deterministic sum (fixed tree order)
__device__ __forceinline__ double block_sum(double v, double *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
    int warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sm[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

__device__ __forceinline__ float block_sum_f(float v, float *sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
    int warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (warp == 0) {
        t = lane < nw ? sm[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// r = b - A x in FP64; per-block partial sums of r^2 into red[block id],
// summed in FP64 or (N32: for a convergence test only, where the FP64 adds
// of the block tree would cost as much as the residual) in FP32
template <int DIM, int KIND, typename TL = float, bool N32 = false>
__global__ void __launch_bounds__(TBX *TBY) k_residual64(Grid g, const double *__restrict__ A,
                                                          const double *__restrict__ b, const double *__restrict__ x,
                                                          double *__restrict__ r, TL *__restrict__ r32,
                                                          double *__restrict__ red) {
    __shared__ double sm[32];
    __shared__ float smf[32];
    int ix = blockIdx.x * TBX + threadIdx.x;
    int iy = blockIdx.y * TBY + threadIdx.y;
    int iz = blockIdx.z;
    double v = 0.0;
    if (ix < g.nx && iy < g.ny) {
        int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
        v = b[i] - apply_row<DIM, KIND, double>(g, A, x, ix, iy, iz, i);
        if (r) r[i] = v;
        if (r32) r32[i] = st<TL>((typename AccT<TL>::type)v);
    }
    if (red) {
        double t;
        if (N32) {
            const float vf = (float)v;
            t = (double)block_sum_f(vf * vf, smf);
        } else {
            t = block_sum(v * v, sm);
        }
        if (threadIdx.x == 0 && threadIdx.y == 0)
            red[blockIdx.x + gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = t;
    }
}

cs_status launch_residual64(const Level &L, const double *A, const double *b, const double *x, double *r,
                            float *r32, double *red, int nred, cudaStream_t s, bool norm32) {
    dim3 gr = node_grid(L.g), bl = node_block();
    if (red && (int64_t)gr.x * gr.y * gr.z != nred) {
        set_error("internal: reduction size mismatch");
        return CS_ERR_ARG;
    }
    if (norm32) {
        if (L.g.dim == 2) {
            if (L.kind == STAR) k_residual64<2, STAR, float, true><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
            else k_residual64<2, BOX, float, true><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
        } else {
            if (L.kind == STAR) k_residual64<3, STAR, float, true><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
            else k_residual64<3, BOX, float, true><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
        }
    } else if (L.g.dim == 2) {
        if (L.kind == STAR) k_residual64<2, STAR><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
        else k_residual64<2, BOX><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
    } else {
        if (L.kind == STAR) k_residual64<3, STAR><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
        else k_residual64<3, BOX><<<gr, bl, 0, s>>>(L.g, A, b, x, r, r32, red);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

__global__ void k_finish_sum(double *red, int n) {
    __shared__ double sm[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += red[i];
    double t = block_sum(v, sm);
    if (threadIdx.x == 0) red[n] = t;
}
cs_status launch_finish_sum(double *red, int nred, cudaStream_t s) {
    k_finish_sum<<<1, 1024, 0, s>>>(red, nred);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

__global__ void k_dot(int64_t N, const double *__restrict__ a, const double *__restrict__ b, double *red) {
    __shared__ double sm[32];
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        v = fma(a[i], b[i], v);
    double t = block_sum(v, sm);
    if (threadIdx.x == 0) red[blockIdx.x] = t;
}
cs_status launch_dot(int64_t N, const double *a, const double *b, double *red, int nred, cudaStream_t s) {
    k_dot<<<nred, 256, 0, s>>>(N, a, b, red);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return launch_finish_sum(red, nred, s);
}

__global__ void k_axpy_dev(int64_t N, const double *alpha, double sign, const double *__restrict__ x,
                           double *__restrict__ y) {
    double a = sign * *alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}
cs_status launch_axpy_dev(int64_t N, const double *alpha, double sign, const double *x, double *y, cudaStream_t s) {
    k_axpy_dev<<<1216, 256, 0, s>>>(N, alpha, sign, x, y);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
__global__ void k_scale_dev(int64_t N, const double *num, double *y, const double *__restrict__ x) {
    double inv = 1.0 / sqrt(*num);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * inv;
}
// y = x / sqrt(*num)
cs_status launch_scale_dev(int64_t N, const double *num, double *y, const double *x, cudaStream_t s) {
    k_scale_dev<<<1216, 256, 0, s>>>(N, num, y, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

// r = b - A x in FP64, stored in BF16 for the cycle (no reduction)
cs_status launch_residual64_bf16(const Level &L, const double *A, const double *b, const double *x,
                                 __nv_bfloat16 *r16, cudaStream_t s) {
    dim3 gr = node_grid(L.g), bl = node_block();
    if (L.g.dim == 2) {
        if (L.kind == STAR) k_residual64<2, STAR, __nv_bfloat16><<<gr, bl, 0, s>>>(L.g, A, b, x, nullptr, r16, nullptr);
        else k_residual64<2, BOX, __nv_bfloat16><<<gr, bl, 0, s>>>(L.g, A, b, x, nullptr, r16, nullptr);
    } else {
        if (L.kind == STAR) k_residual64<3, STAR, __nv_bfloat16><<<gr, bl, 0, s>>>(L.g, A, b, x, nullptr, r16, nullptr);
        else k_residual64<3, BOX, __nv_bfloat16><<<gr, bl, 0, s>>>(L.g, A, b, x, nullptr, r16, nullptr);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
__global__ void k_axpy_bf16(int64_t N, const __nv_bfloat16 *__restrict__ d, double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)__bfloat162float(d[i]);
}
cs_status launch_axpy_bf16(int64_t N, const __nv_bfloat16 *d, double *x, cudaStream_t s) {
    k_axpy_bf16<<<1216, 256, 0, s>>>(N, d, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
__global__ void k_d2bf(int64_t N, const double *__restrict__ a, __nv_bfloat16 *__restrict__ o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = __double2bfloat16(a[i]);
}
cs_status launch_copy_d2bf(int64_t N, const double *a, __nv_bfloat16 *o, cudaStream_t s) {
    k_d2bf<<<1216, 256, 0, s>>>(N, a, o);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

__global__ void k_axpy_f32(int64_t N, const float *__restrict__ d, double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}
cs_status launch_axpy_f32(int64_t N, const float *d, double *x, cudaStream_t s) {
    k_axpy_f32<<<1216, 256, 0, s>>>(N, d, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
__global__ void k_d2f(int64_t N, const double *__restrict__ a, float *__restrict__ o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}
cs_status launch_copy_d2f(int64_t N, const double *a, float *o, cudaStream_t s) {
    k_d2f<<<1216, 256, 0, s>>>(N, a, o);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

// y = A x (FP64)
template <int DIM, int KIND>
__global__ void __launch_bounds__(TBX *TBY) k_matvec64(Grid g, const double *__restrict__ A,
                                                        const double *__restrict__ x, double *__restrict__ y) {
    int ix = blockIdx.x * TBX + threadIdx.x, iy = blockIdx.y * TBY + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    int64_t i = ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
    y[i] = apply_row<DIM, KIND, double>(g, A, x, ix, iy, iz, i);
}
cs_status launch_matvec64(const Level &L, const double *A, const double *x, double *y, cudaStream_t s) {
    dim3 gr = node_grid(L.g), bl = node_block();
    if (L.g.dim == 2) {
        if (L.kind == STAR) k_matvec64<2, STAR><<<gr, bl, 0, s>>>(L.g, A, x, y);
        else k_matvec64<2, BOX><<<gr, bl, 0, s>>>(L.g, A, x, y);
    } else {
        if (L.kind == STAR) k_matvec64<3, STAR><<<gr, bl, 0, s>>>(L.g, A, x, y);
        else k_matvec64<3, BOX><<<gr, bl, 0, s>>>(L.g, A, x, y);
    }
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

__global__ void k_add64(int64_t N, const double *__restrict__ d, double *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}
cs_status launch_add64(int64_t N, const double *d, double *x, cudaStream_t s) {
    k_add64<<<1216, 256, 0, s>>>(N, d, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

// y += alpha_host * x with alpha from device memory slot
__global__ void k_axpy_vec(int64_t N, int m, const double *__restrict__ alpha, const double *__restrict__ V,
                           double *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double s = y[i];
        for (int k = 0; k < m; ++k) s = fma(alpha[k], V[(int64_t)k * N + i], s);
        y[i] = s;
    }
}
// y += sum_k alpha[k] V[k]  (alpha: device array of m values)
cs_status launch_axpy_multi(int64_t N, int m, const double *alpha, const double *V, double *y, cudaStream_t s) {
    k_axpy_vec<<<1216, 256, 0, s>>>(N, m, alpha, V, y);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

// x = Cinv b (bottom-level direct solve with the inverse formed at setup):
// one warp per row, FP64
template <typename T>
__global__ void k_coarse_solve(int n, const double *__restrict__ Cinv, const T *__restrict__ b, T *__restrict__ x) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(Cinv[(int64_t)warp * n + j], (double)ld<T>(b[j]), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[warp] = st<T>((typename AccT<T>::type)s);
}
cs_status launch_coarse_solve(const cs_hierarchy *h, const double *b, double *x, cudaStream_t s) {
    int threads = 256, blocks = (h->cn * 32 + threads - 1) / threads;
    k_coarse_solve<double><<<blocks, threads, 0, s>>>(h->cn, h->cinv, b, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
cs_status launch_coarse_solve32(const cs_hierarchy *h, const float *b, float *x, cudaStream_t s) {
    int threads = 256, blocks = (h->cn * 32 + threads - 1) / threads;
    k_coarse_solve<float><<<blocks, threads, 0, s>>>(h->cn, h->cinv, b, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}
cs_status launch_coarse_solve16(const cs_hierarchy *h, const __nv_bfloat16 *b, __nv_bfloat16 *x, cudaStream_t s) {
    int threads = 256, blocks = (h->cn * 32 + threads - 1) / threads;
    k_coarse_solve<__nv_bfloat16><<<blocks, threads, 0, s>>>(h->cn, h->cinv, b, x);
    CSX_CUDA(cudaGetLastError());
    count_launch();
    return CS_OK;
}

}  // namespace csx
