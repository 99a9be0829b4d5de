// Sketched cascade setup (the reformulation of the paper's concluding
// remarks, Sec. 4): step l minimises ||(I - Lambda A~) E_{l-1} S||_F over
// point-block Lambda instead of ||(I - Lambda A~) E_{l-1}||_F.  With
// Y = E_{l-1} S carried along (Y_0 = S), every node i solves the 1 x 1
// normal equations of min ||Y_i - lam Z_i|| with Z = A~ Y,
//     lam~_i = <Y_i, Z_i> / <Z_i, Z_i>   (0 when Z_i = 0),
// and Y_i <- Y_i - lam~_i Z_i; multiplicative: colour by colour, every colour
// reading the state after the previous one.  A~ = W A W with
// W = diag(A_ii^-1/2) (Sec. 2.3.1) and Lambda = W Lambda~ W.  No residual
// fill-in: the memory is two N x s arrays whatever the depth.
//
// S is Rademacher: entry (i, t) of level l is the sign of the SplitMix64
// output (Steele, Lea and Flood 2014) at counter c = l 2^48 + i s + t of
// the stream seeded with the given seed, i.e. of mix(seed + (c + 1) g).
//
// Layout: Y[i * s + t] (the s entries of a node contiguous).  One warp per
// node, its lanes over t (s <= 128: up to 4 entries per lane): the stencil
// neighbours' rows are read as 32 consecutive values per warp, and the two
// inner products are warp sums in FP64.  T = double (the exact arithmetic
// of the method) or float (Y and Z in FP32, the inner products and lambda
// in FP64).
#include "cs_internal.cuh"

namespace csx {

__device__ __forceinline__ uint64_t sk_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_sketch_init(int64_t N, int s, uint64_t seed, int l, T *__restrict__ Y) {
    const int64_t total = N * s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = ((uint64_t)l << 48) + (uint64_t)e;  // e = i s + t
        const uint64_t z = sk_mix(seed + (c + 1) * 0x9E3779B97F4A7C15ULL);
        Y[e] = (z >> 63) ? T(-1) : T(1);
    }
}

// w_i = A_ii^-1/2 (1 without prescaling); bad = 1 when a diagonal is <= 0
__global__ void k_sketch_w(int64_t N, const double *__restrict__ diag, int prescale, double *__restrict__ w,
                           int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[i];
        if (prescale && !(d > 0.0)) atomicExch(bad, 1);
        w[i] = prescale ? 1.0 / sqrt(d) : 1.0;
    }
}

struct SkOff {
    int d[27][3];
};

// One sketched step (colour < 0: every node; else the nodes of that
// red-black colour, the others copied) from Y to Yn; lam (FP64, [N]) gets
// the unscaled lambda of the updated nodes.  exact: this step solves the
// unsketched problem (E = I): lam~ = A~_ii / sum_j A~_ij^2.
template <int SPL, typename T>
__global__ void __launch_bounds__(256) k_sketch_step(Grid g, int nst, SkOff off, int centre,
                                                     const double *__restrict__ A, const double *__restrict__ w,
                                                     const T *__restrict__ Y, T *__restrict__ Yn, int s, int colour,
                                                     int exact, double *__restrict__ lam) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < g.N; i += nwarps) {
        const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((int64_t)g.nx * g.ny));
        const bool upd = colour < 0 || ((((ix + 1) + (iy + 1) + (g.dim == 3 ? iz + 1 : 0)) & 1) == colour);
        if (!upd) {  // the other colour keeps its state
#pragma unroll
            for (int u = 0; u < SPL; ++u) {
                const int t = lane + 32 * u;
                if (t < s) Yn[i * s + t] = Y[i * s + t];
            }
            continue;
        }
        const double wi = w[i];
        T z[SPL];
#pragma unroll
        for (int u = 0; u < SPL; ++u) z[u] = T(0);
        double rowsq = 0.0, aii = 0.0;
        for (int k = 0; k < nst; ++k) {
            const int jx = ix + off.d[k][0], jy = iy + off.d[k][1], jz = iz + off.d[k][2];
            if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny || jz < 0 || jz >= g.nz) continue;
            const int64_t j = jx + (int64_t)g.nx * (jy + (int64_t)g.ny * jz);
            const double at = wi * A[(int64_t)k * g.N + i] * w[j];  // A~_ij
            if (exact) {
                rowsq = fma(at, at, rowsq);
                if (k == centre) aii = at;
            }
            const T a = (T)at;
#pragma unroll
            for (int u = 0; u < SPL; ++u) {
                const int t = lane + 32 * u;
                if (t < s) z[u] = fma(a, Y[j * s + t], z[u]);
            }
        }
        // <Z, Z> and <Y, Z>: each lane's columns in T, the lanes combined in
        // FP64; with FP32 vectors the products and the update stay off the
        // FP64 pipe (GB300 issues FP64 at a small fraction of the FP32 rate)
        T gl = T(0), cl = T(0);
#pragma unroll
        for (int u = 0; u < SPL; ++u) {
            const int t = lane + 32 * u;
            if (t < s) {
                const T yv = Y[i * s + t];
                gl = fma(z[u], z[u], gl);
                cl = fma(yv, z[u], cl);
            }
        }
        double gz = (double)gl, cz = (double)cl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
            cz += __shfl_xor_sync(0xffffffffu, cz, o);
        }
        const double G = exact ? rowsq : gz, C = exact ? aii : cz;
        const double lt = G > 0.0 ? C / G : 0.0;
        const T ltt = (T)lt;
#pragma unroll
        for (int u = 0; u < SPL; ++u) {
            const int t = lane + 32 * u;
            if (t < s) Yn[i * s + t] = fma(-ltt, z[u], Y[i * s + t]);
        }
        if (lane == 0) lam[i] = wi * lt * wi;
    }
}

template <typename T>
static cs_status sketch_level_t(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int s, uint64_t seed,
                                int exact_first, double *lam, cudaStream_t st) {
    const Level &L = h->lev[l];
    const int64_t N = L.g.N;
    const int centre = L.kind == STAR ? 0 : (L.g.dim == 3 ? 13 : 4);
    SkOff off;
    for (int k = 0; k < 27; ++k)
        for (int d = 0; d < 3; ++d) off.d[k][d] = k < L.nst ? L.off[k][d] : 0;
    double *w = nullptr;
    T *Y = nullptr, *Yn = nullptr;
    int *bad = nullptr;
    int badh = 0;
    cs_status rc = CS_OK;
    const int ncol = kind == CS_MULTIPLICATIVE ? 2 : 1;
    const int spl = (s + 31) / 32;
    const int threads = 256;
    const int64_t want = (N * 32 + threads - 1) / threads;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 32));
    if ((rc = dalloc_t(&w, (size_t)N, nullptr, st)) != CS_OK) goto done;
    if ((rc = dalloc_t(&Y, (size_t)N * s, nullptr, st)) != CS_OK) goto done;
    if ((rc = dalloc_t(&Yn, (size_t)N * s, nullptr, st)) != CS_OK) goto done;
    if ((rc = dalloc_t(&bad, 1, nullptr, st)) != CS_OK) goto done;
    CSX_CUDA_GOTO(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_sketch_w<<<std::min<int64_t>(1216, (N + 255) / 256), 256, 0, st>>>(N, L.A + (int64_t)centre * N, prescale, w, bad);
    k_sketch_init<T><<<1216, 256, 0, st>>>(N, s, seed, l, Y);
    count_launch(2);
    CSX_CUDA_GOTO(cudaGetLastError());
    for (int step = 0; step < nu; ++step)
        for (int k = 0; k < ncol; ++k) {
            const int colour = ncol == 2 ? k : -1;
            const int exact = exact_first && step == 0 && k == 0;
            double *lst = lam + (int64_t)step * N;
            if (spl == 1)
                k_sketch_step<1, T><<<blocks, threads, 0, st>>>(L.g, L.nst, off, centre, L.A, w, Y, Yn, s, colour, exact, lst);
            else if (spl == 2)
                k_sketch_step<2, T><<<blocks, threads, 0, st>>>(L.g, L.nst, off, centre, L.A, w, Y, Yn, s, colour, exact, lst);
            else
                k_sketch_step<4, T><<<blocks, threads, 0, st>>>(L.g, L.nst, off, centre, L.A, w, Y, Yn, s, colour, exact, lst);
            count_launch();
            CSX_CUDA_GOTO(cudaGetLastError());
            std::swap(Y, Yn);
        }
    CSX_CUDA_GOTO(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSX_CUDA_GOTO(cudaStreamSynchronize(st));
    if (badh) {
        set_error("level %d: a non-positive diagonal entry under elliptic prescaling", l);
        rc = CS_ERR_ARG;
    }
done:
    dfree(w, st); dfree(Y, st); dfree(Yn, st); dfree(bad, st);
    return rc;
}

cs_status cascade_setup_level_sketch(const cs_hierarchy *h, int l, int kind, int nu, int prescale, int s,
                                     uint64_t seed, int exact_first, bool fp32, double *lam, cudaStream_t st) {
    const Level &L = h->lev[l];
    if (L.bs != 1) {
        set_error("the sketched setup is implemented for point blocks");
        return CS_ERR_UNSUPPORTED;
    }
    if (s < 1 || s > 128) {
        set_error("sketch size must be in 1..128");
        return CS_ERR_ARG;
    }
    if (h->periodic) {
        set_error("the sketched setup takes Dirichlet hierarchies");
        return CS_ERR_UNSUPPORTED;
    }
    // multiplicative: every node of a colour gets its lambda in its own step's
    // array; the other colour's entries of that array stay zero
    CSX_CUDA(cudaMemsetAsync(lam, 0, sizeof(double) * (size_t)nu * L.g.N, st));
    return fp32 ? sketch_level_t<float>(h, l, kind, nu, prescale, s, seed, exact_first, lam, st)
                : sketch_level_t<double>(h, l, kind, nu, prescale, s, seed, exact_first, lam, st);
}

}  // namespace csx
