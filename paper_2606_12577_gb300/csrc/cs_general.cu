// The method for a general block-partitioned sparse A x = b: the user's
// operator (CSR), transfers and block partition (Sec. 2, Sec. 2.4), with
// index-driven kernels in place of the structured stencil kernels.
//
//   hierarchy  Galerkin A_{l+1} = rscale P_l^T A_l P_l by two sparse
//              products: their patterns on the host, their values on the
//              device (one warp per output row, the contributions of a row
//              summed in the order of the left factor's entries with
//              unfused multiplies and adds, as the oracle's Gustavson loop);
//              greedy colouring of each level's block graph by
//              Jones-Plassmann rounds; dense FP64 factorisation of the
//              coarsest operator.
//   cascade    Algorithm 2 / the SM algorithm with the residual rows E kept
//              per block over the union of the block rows' columns: the
//              patterns on the host, the values on the device (one warp per
//              block: R_b = (A~ E)_{b,:}, G = R_b R_b^T, C = E_b R_b^T,
//              Lambda~ = C G^{-1} or C G^+, E_b <- E_b - Lambda~ R_b).
//   cycles     CSR residuals and transfers, the cascade steps (one thread
//              per row on point-block levels, one warp per block
//              otherwise), the coarsest solve as a dense inverse mat-vec,
//              stationary and right-preconditioned flexible GMRES solves.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "cs_internal.cuh"

namespace csx {

__global__ void k_factor_inverse(int n, double *M, double *W, double *Inv, int *piv, int *status);  // cs_setup.cu

constexpr int GMAXBLK = 16;     // nodes per block
constexpr int GMAXCOL = 64;     // colours per level
constexpr int GMAXCOARSE = 1024;

struct GCsr {
    int n = 0, m = 0;
    int64_t nnz = 0;
    int64_t *rp = nullptr;  // device
    int *ci = nullptr;
    double *v = nullptr;
    std::vector<int64_t> hrp;  // host pattern
    std::vector<int> hci;
};

struct GLevel {
    GCsr A, P, R;  // P, R: transfers to the next coarser level
    int nb = 0, nbmax = 1;
    int ident = 0;  // the blocks are the points in order (block b = node b)
    std::vector<int> hfield;      // per unknown: 0 velocity / scalar, 1 pressure
    int *field = nullptr;
    // overlapping blocks (a node in several blocks): node -> blocks holding it,
    // ascending (nptr [N + 1], nblk / nloc [M]: block and position in it)
    int overlap = 0;
    std::vector<int> hnptr, hnblk, hnloc;
    int *nptr = nullptr, *nblk = nullptr, *nloc = nullptr;
    double *dpool = nullptr;  // per (block, row) corrections of the overlapping additive step
    std::vector<int> hbptr, hbidx, hcol;  // block partition and colour per block
    int *bptr = nullptr, *bidx = nullptr;
    int ncol = 1;
    std::vector<int> colstart;  // [ncol + 1] offsets into cblocks
    int *cblocks = nullptr;     // blocks sorted by colour, ascending within a colour
    double *b = nullptr, *x = nullptr, *t = nullptr, *r = nullptr;
};

}  // namespace csx

struct cs_ghier {
    int nlev = 0;
    std::vector<csx::GLevel> lev;
    double rscale = 1.0;
    int cn = 0;
    double *cinv = nullptr;
    double *red = nullptr, *red_host = nullptr;
    int64_t bytes = 0;
};

struct cs_gcascade {
    const cs_ghier *h = nullptr;
    int kind = CS_ADDITIVE, nu = 1, nlev = 0;
    std::vector<double *> lam;
    std::vector<std::vector<int64_t>> hlamoff;
    std::vector<int64_t *> lamoff;
    std::vector<int64_t> lamsize;
    int gm_restart = 0;
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_h = nullptr;
    double *cg = nullptr;  // PCG vectors r, z, p, q
    int64_t bytes = 0;
};

namespace csx {

static void gcsr_free(GCsr &A) {
    dfree(A.rp); dfree(A.ci); dfree(A.v);
    A.rp = nullptr; A.ci = nullptr; A.v = nullptr;
}

// Copy a user CSR matrix (host or device arrays) to the device and keep its
// pattern on the host; checks shapes, monotone row pointers, column range
// and ascending columns within every row.
static cs_status gcsr_in(const cs_csr &U, GCsr &A, int64_t *acct, cudaStream_t s) {
    if (U.n < 1 || U.m < 1 || !U.rowptr || !U.col || !U.val) { set_error("CSR: empty shape or null array"); return CS_ERR_ARG; }
    A.n = U.n; A.m = U.m;
    A.hrp.resize((size_t)U.n + 1);
    if (U.on_host) std::memcpy(A.hrp.data(), U.rowptr, sizeof(int64_t) * ((size_t)U.n + 1));
    else CSX_CUDA(cudaMemcpy(A.hrp.data(), U.rowptr, sizeof(int64_t) * ((size_t)U.n + 1), cudaMemcpyDeviceToHost));
    if (A.hrp[0] != 0) { set_error("CSR: rowptr[0] must be 0"); return CS_ERR_ARG; }
    for (int i = 0; i < U.n; ++i)
        if (A.hrp[i + 1] < A.hrp[i]) { set_error("CSR: rowptr decreases at row %d", i); return CS_ERR_ARG; }
    A.nnz = A.hrp[U.n];
    A.hci.resize((size_t)std::max<int64_t>(A.nnz, 1));
    if (U.on_host) std::memcpy(A.hci.data(), U.col, sizeof(int) * (size_t)A.nnz);
    else CSX_CUDA(cudaMemcpy(A.hci.data(), U.col, sizeof(int) * (size_t)A.nnz, cudaMemcpyDeviceToHost));
    for (int i = 0; i < U.n; ++i)
        for (int64_t p = A.hrp[i]; p < A.hrp[i + 1]; ++p) {
            if (A.hci[p] < 0 || A.hci[p] >= U.m) { set_error("CSR: column out of range in row %d", i); return CS_ERR_ARG; }
            if (p > A.hrp[i] && A.hci[p] <= A.hci[p - 1]) { set_error("CSR: columns not ascending in row %d", i); return CS_ERR_ARG; }
        }
    const cudaMemcpyKind k = U.on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CSX_TRY(dalloc_t(&A.rp, (size_t)U.n + 1, acct, s));
    CSX_TRY(dalloc_t(&A.ci, (size_t)std::max<int64_t>(A.nnz, 1), acct, s));
    CSX_TRY(dalloc_t(&A.v, (size_t)std::max<int64_t>(A.nnz, 1), acct, s));
    CSX_CUDA(cudaMemcpyAsync(A.rp, U.rowptr, sizeof(int64_t) * ((size_t)U.n + 1), k, s));
    CSX_CUDA(cudaMemcpyAsync(A.ci, U.col, sizeof(int) * (size_t)A.nnz, k, s));
    CSX_CUDA(cudaMemcpyAsync(A.v, U.val, sizeof(double) * (size_t)A.nnz, k, s));
    return CS_OK;
}

static cs_status gcsr_upload_pattern(GCsr &C, int64_t *acct, cudaStream_t s) {
    C.nnz = C.hrp[C.n];
    CSX_TRY(dalloc_t(&C.rp, (size_t)C.n + 1, acct, s));
    CSX_TRY(dalloc_t(&C.ci, (size_t)std::max<int64_t>(C.nnz, 1), acct, s));
    CSX_TRY(dalloc_t(&C.v, (size_t)std::max<int64_t>(C.nnz, 1), acct, s));
    CSX_CUDA(cudaMemcpyAsync(C.rp, C.hrp.data(), sizeof(int64_t) * ((size_t)C.n + 1), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(C.ci, C.hci.data(), sizeof(int) * (size_t)C.nnz, cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaStreamSynchronize(s));  // the host pattern may be resized by the caller afterwards
    return CS_OK;
}

__device__ __forceinline__ int64_t gfind(const int *__restrict__ c, int64_t lo, int64_t hi, int key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (c[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// C = scale (A B) on C's pattern: one warp per row; the row's entries are
// zeroed, then every entry (k, a) of A's row adds a * B(k, j) to C(i, j),
// the lanes over B's row k (distinct columns), in the order of A's entries.
__global__ void k_gspgemm(int n, const int64_t *__restrict__ arp, const int *__restrict__ aci,
                          const double *__restrict__ av, const int64_t *__restrict__ brp,
                          const int *__restrict__ bci, const double *__restrict__ bv,
                          const int64_t *__restrict__ crp, const int *__restrict__ cci, double *cv, double scale) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int64_t c0 = crp[i], c1 = crp[i + 1];
        for (int64_t q = c0 + lane; q < c1; q += 32) cv[q] = 0.0;
        __syncwarp();
        for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
            const int k = aci[p];
            const double a = av[p];
            for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
                const int64_t pos = gfind(cci, c0, c1, bci[q]);
                cv[pos] = __dadd_rn(cv[pos], __dmul_rn(a, bv[q]));
            }
            __syncwarp();
        }
        if (scale != 1.0)
            for (int64_t q = c0 + lane; q < c1; q += 32) cv[q] = __dmul_rn(scale, cv[q]);
    }
}

// Host symbolic work in parallel: fn(t, lo, hi) over T contiguous ranges
// of [0, n) (T host threads, at most 16); callers write per-range parts and
// join them in range order, so results do not depend on T.
template <class F>
static int gpar_ranges(int64_t n, F &&fn) {
    const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(hw, 16), (n + 8191) / 8192));
    if (T == 1) {
        fn(0, (int64_t)0, n);
        return 1;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)T);
    for (int t = 0; t < T; ++t) th.emplace_back([&fn, t, T, n] { fn(t, n * t / T, n * (t + 1) / T); });
    for (std::thread &x : th) x.join();
    return T;
}

// the pattern of A B (sorted rows), host
static void gspgemm_pattern(const GCsr &A, const GCsr &B, GCsr &C) {
    C.n = A.n; C.m = B.m;
    C.hrp.assign((size_t)A.n + 1, 0);
    std::vector<std::vector<int>> part(16);
    const int T = gpar_ranges(A.n, [&](int t, int64_t lo, int64_t hi) {
        std::vector<int> mark((size_t)B.m, -1), row;
        std::vector<int> &out = part[t];
        for (int64_t i = lo; i < hi; ++i) {
            row.clear();
            for (int64_t p = A.hrp[i]; p < A.hrp[i + 1]; ++p) {
                const int k = A.hci[p];
                for (int64_t q = B.hrp[k]; q < B.hrp[k + 1]; ++q)
                    if (mark[B.hci[q]] != (int)i) { mark[B.hci[q]] = (int)i; row.push_back(B.hci[q]); }
            }
            std::sort(row.begin(), row.end());
            out.insert(out.end(), row.begin(), row.end());
            C.hrp[i + 1] = (int64_t)row.size();
        }
    });
    for (int i = 0; i < A.n; ++i) C.hrp[i + 1] += C.hrp[i];
    C.hci.clear();
    C.hci.reserve((size_t)C.hrp[A.n]);
    for (int t = 0; t < T; ++t) C.hci.insert(C.hci.end(), part[t].begin(), part[t].end());
}

static unsigned gwarp_blocks(int64_t items) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items * 32 + 255) / 256, 152 * 16));
}

static cs_status gspgemm(const GCsr &A, const GCsr &B, double scale, GCsr &C, int64_t *acct, cudaStream_t s) {
    gspgemm_pattern(A, B, C);
    CSX_TRY(gcsr_upload_pattern(C, acct, s));
    k_gspgemm<<<gwarp_blocks(A.n), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, B.rp, B.ci, B.v, C.rp, C.ci, C.v, scale);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

__global__ void k_ggather(int64_t n, const int64_t *__restrict__ map, const double *__restrict__ src,
                          double *__restrict__ dst, double scale) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = scale == 1.0 ? src[map[q]] : __dmul_rn(scale, src[map[q]]);
}

// T = scale P^T: rows of T filled in ascending order of P's rows (so every
// row of T has ascending columns), the values gathered on the device
static cs_status gtranspose(const GCsr &P, double scale, GCsr &T, int64_t *acct, cudaStream_t s) {
    T.n = P.m; T.m = P.n;
    T.hrp.assign((size_t)T.n + 1, 0);
    for (int64_t p = 0; p < P.nnz; ++p) T.hrp[P.hci[p] + 1]++;
    for (int j = 0; j < T.n; ++j) T.hrp[j + 1] += T.hrp[j];
    std::vector<int64_t> fill(T.hrp.begin(), T.hrp.end() - 1), map((size_t)std::max<int64_t>(P.nnz, 1));
    T.hci.assign((size_t)std::max<int64_t>(P.nnz, 1), 0);
    for (int i = 0; i < P.n; ++i)
        for (int64_t p = P.hrp[i]; p < P.hrp[i + 1]; ++p) {
            const int64_t q = fill[P.hci[p]]++;
            T.hci[q] = i;
            map[q] = p;
        }
    CSX_TRY(gcsr_upload_pattern(T, acct, s));
    int64_t *dmap = nullptr;
    CSX_TRY(dalloc_t(&dmap, map.size(), nullptr, s));
    CSX_CUDA(cudaMemcpyAsync(dmap, map.data(), sizeof(int64_t) * map.size(), cudaMemcpyHostToDevice, s));
    k_ggather<<<1216, 256, 0, s>>>(P.nnz, dmap, P.v, T.v, scale);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    CSX_CUDA(cudaStreamSynchronize(s));
    dfree(dmap, s);
    return CS_OK;
}

}  // namespace csx

namespace csx {

// ---------------------------------------------------------- colouring
__device__ __forceinline__ uint64_t gmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_gprio(int nb, uint64_t seed, int l, uint64_t *__restrict__ prio, int *__restrict__ col) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const uint64_t c = ((uint64_t)l << 40) + (uint64_t)b;
        prio[b] = gmix(seed + (c + 1) * 0x9E3779B97F4A7C15ULL);
        col[b] = -1;
    }
}

// One Jones-Plassmann round: an uncoloured block whose uncoloured
// neighbours all rank below it (lower priority, or equal priority and a
// larger index) takes the smallest colour none of its coloured neighbours
// holds.  Reads the colours of the previous round (cin), writes cout; the
// blocks coloured in one round are pairwise non-adjacent, and a block's
// colour depends only on its higher-ranked neighbours, all coloured before
// it: the result is the sequential greedy colouring in rank order.
__global__ void k_gjpl(int nb, const int *__restrict__ gp, const int *__restrict__ gi,
                       const uint64_t *__restrict__ prio, const int *__restrict__ cin, int *__restrict__ cout,
                       int *left, int *over) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int c = cin[b];
        if (c < 0) {
            bool top = true;
            unsigned long long used = 0ull;
            const uint64_t pb = prio[b];
            for (int q = gp[b]; q < gp[b + 1]; ++q) {
                const int u = gi[q];
                const int cu = cin[u];
                if (cu < 0) {
                    if (prio[u] > pb || (prio[u] == pb && u < b)) { top = false; break; }
                } else if (cu < 64) {
                    used |= 1ull << cu;
                }
            }
            if (top) {
                c = __ffsll((long long)~used) - 1;  // lowest free colour
                if (c < 0 || c >= GMAXCOL) { atomicExch(over, 1); c = GMAXCOL - 1; }
            } else {
                atomicAdd(left, 1);
            }
        }
        cout[b] = c;
    }
}

static void gnode_blocks(GLevel &L) {
    const int N = L.A.n, nb = L.nb, M = L.hbptr[nb];
    L.hnptr.assign((size_t)N + 1, 0);
    L.hnblk.assign((size_t)M, 0);
    L.hnloc.assign((size_t)M, 0);
    for (int p = 0; p < M; ++p) L.hnptr[L.hbidx[p] + 1]++;
    for (int i = 0; i < N; ++i) L.hnptr[i + 1] += L.hnptr[i];
    std::vector<int> fill(L.hnptr.begin(), L.hnptr.end() - 1);
    for (int b = 0; b < nb; ++b)
        for (int p = L.hbptr[b]; p < L.hbptr[b + 1]; ++p) {
            const int q = fill[L.hbidx[p]]++;
            L.hnblk[q] = b;
            L.hnloc[q] = p - L.hbptr[b];
        }
}

static cs_status gcolour(GLevel &L, int l, uint64_t seed, cudaStream_t s) {
    const int nb = L.nb;
    // symmetrised block graph without duplicates: blocks b and c touch when a
    // row of b couples to a node of c or they share a node.  The directed
    // lists (b -> c) are built in parallel, then merged with their reverse.
    std::vector<std::vector<int>> out((size_t)nb);
    gpar_ranges(nb, [&](int, int64_t lo, int64_t hi) {
        for (int64_t b = lo; b < hi; ++b) {
            std::vector<int> &ob = out[b];
            for (int p = L.hbptr[b]; p < L.hbptr[b + 1]; ++p) {
                const int i = L.hbidx[p];
                for (int64_t q = L.A.hrp[i] - 1; q < L.A.hrp[i + 1]; ++q) {
                    const int j = q < L.A.hrp[i] ? i : L.A.hci[q];
                    for (int u = L.hnptr[j]; u < L.hnptr[j + 1]; ++u)
                        if (L.hnblk[u] != b) ob.push_back(L.hnblk[u]);
                }
            }
            std::sort(ob.begin(), ob.end());
            ob.erase(std::unique(ob.begin(), ob.end()), ob.end());
        }
    });
    std::vector<int> rp((size_t)nb + 1, 0);
    for (int b = 0; b < nb; ++b)
        for (int c : out[b]) rp[c + 1]++;
    for (int b = 0; b < nb; ++b) rp[b + 1] += rp[b];
    std::vector<int> rin((size_t)rp[nb]), fillr(rp.begin(), rp.end() - 1);
    for (int b = 0; b < nb; ++b)
        for (int c : out[b]) rin[fillr[c]++] = b;  // reverse edges, ascending b per c
    std::vector<int> gp((size_t)nb + 1, 0), gi;
    std::vector<std::vector<int>> part(16);
    std::vector<int> deg((size_t)nb);
    const int T = gpar_ranges(nb, [&](int t, int64_t lo, int64_t hi) {
        std::vector<int> &pt = part[t];
        for (int64_t b = lo; b < hi; ++b) {  // union of two ascending lists
            const std::vector<int> &ob = out[b];
            size_t x = 0;
            int y = rp[b];
            const size_t s0 = pt.size();
            while (x < ob.size() || y < rp[b + 1]) {
                int v;
                if (y >= rp[b + 1] || (x < ob.size() && ob[x] < rin[y])) v = ob[x++];
                else if (x >= ob.size() || rin[y] < ob[x]) v = rin[y++];
                else { v = ob[x++]; ++y; }
                pt.push_back(v);
            }
            deg[b] = (int)(pt.size() - s0);
        }
    });
    for (int b = 0; b < nb; ++b) gp[b + 1] = gp[b] + deg[b];
    gi.reserve((size_t)gp[nb]);
    for (int t = 0; t < T; ++t) gi.insert(gi.end(), part[t].begin(), part[t].end());
    if (gi.empty()) gi.push_back(0);
    int *dgp = nullptr, *dgi = nullptr, *ca = nullptr, *cb = nullptr, *cnt = nullptr;
    uint64_t *prio = nullptr;
    cs_status rc = CS_OK;
    int hcnt[2] = {0, 0};
    if ((rc = dalloc_t(&dgp, gp.size(), nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&dgi, gi.size(), nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&ca, (size_t)nb, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&cb, (size_t)nb, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&prio, (size_t)nb, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&cnt, 2, nullptr, s)) != CS_OK) goto done;
    CSX_CUDA_GOTO(cudaMemcpyAsync(dgp, gp.data(), sizeof(int) * gp.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA_GOTO(cudaMemcpyAsync(dgi, gi.data(), sizeof(int) * gi.size(), cudaMemcpyHostToDevice, s));
    k_gprio<<<std::max(1, std::min(1216, (nb + 255) / 256)), 256, 0, s>>>(nb, seed, l, prio, ca);
    count_launch();
    for (int round = 0; round <= nb; ++round) {  // every round colours the top-ranked uncoloured block at least
        CSX_CUDA_GOTO(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s));
        k_gjpl<<<std::max(1, std::min(1216, (nb + 255) / 256)), 256, 0, s>>>(nb, dgp, dgi, prio, ca, cb, cnt,
                                                                               cnt + 1);
        count_launch();
        CSX_CUDA_GOTO(cudaGetLastError());
        std::swap(ca, cb);
        CSX_CUDA_GOTO(cudaMemcpyAsync(hcnt, cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CSX_CUDA_GOTO(cudaStreamSynchronize(s));
        if (hcnt[0] == 0) break;
    }
    if (hcnt[1]) {
        set_error("level %d: the greedy colouring needs more than %d colours", l, GMAXCOL);
        rc = CS_ERR_ARG;
        goto done;
    }
    L.hcol.resize((size_t)nb);
    CSX_CUDA_GOTO(cudaMemcpy(L.hcol.data(), ca, sizeof(int) * (size_t)nb, cudaMemcpyDeviceToHost));
done:
    dfree(dgp, s); dfree(dgi, s); dfree(ca, s); dfree(cb, s); dfree(prio, s); dfree(cnt, s);
    return rc;
}

// blocks of each colour, ascending within a colour; device copies of the
// partition
static cs_status gblock_tables(GLevel &L, int64_t *acct, cudaStream_t s) {
    L.ncol = 0;
    for (int c : L.hcol) L.ncol = std::max(L.ncol, c + 1);
    L.colstart.assign((size_t)L.ncol + 1, 0);
    for (int c : L.hcol) L.colstart[c + 1]++;
    for (int k = 0; k < L.ncol; ++k) L.colstart[k + 1] += L.colstart[k];
    std::vector<int> fill(L.colstart.begin(), L.colstart.end() - 1), cbl((size_t)L.nb);
    for (int b = 0; b < L.nb; ++b) cbl[fill[L.hcol[b]]++] = b;
    L.nbmax = 1;
    for (int b = 0; b < L.nb; ++b) L.nbmax = std::max(L.nbmax, L.hbptr[b + 1] - L.hbptr[b]);
    L.ident = L.nb == L.A.n && (int)L.hbidx.size() == L.A.n;
    for (int i = 0; i < L.A.n && L.ident; ++i) L.ident = L.hbidx[i] == i;
    CSX_TRY(dalloc_t(&L.cblocks, (size_t)L.nb, acct, s));
    CSX_TRY(dalloc_t(&L.bptr, (size_t)L.nb + 1, acct, s));
    CSX_TRY(dalloc_t(&L.bidx, L.hbidx.size(), acct, s));
    CSX_TRY(dalloc_t(&L.nptr, L.hnptr.size(), acct, s));
    CSX_TRY(dalloc_t(&L.nblk, L.hnblk.size(), acct, s));
    CSX_TRY(dalloc_t(&L.nloc, L.hnloc.size(), acct, s));
    if (L.overlap) CSX_TRY(dalloc_t(&L.dpool, L.hbidx.size(), acct, s));
    CSX_CUDA(cudaMemcpyAsync(L.nptr, L.hnptr.data(), sizeof(int) * L.hnptr.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(L.nblk, L.hnblk.data(), sizeof(int) * L.hnblk.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(L.nloc, L.hnloc.data(), sizeof(int) * L.hnloc.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(L.cblocks, cbl.data(), sizeof(int) * cbl.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(L.bptr, L.hbptr.data(), sizeof(int) * L.hbptr.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(L.bidx, L.hbidx.data(), sizeof(int) * L.hbidx.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    return CS_OK;
}

__global__ void k_gdense(int n, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                         const double *__restrict__ v, double *__restrict__ M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int j = 0; j < n; ++j) M[(int64_t)i * n + j] = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) M[(int64_t)i * n + ci[p]] += v[p];
    }
}

static cs_status gcoarse_factor(cs_ghier *h, cudaStream_t s) {
    const GCsr &A = h->lev[h->nlev - 1].A;
    const int n = A.n;
    if (n > GMAXCOARSE) {
        set_error("the coarsest level has %d unknowns (at most %d are factorised densely)", n, GMAXCOARSE);
        return CS_ERR_ARG;
    }
    h->cn = n;
    double *M = nullptr, *W = nullptr;
    int *piv = nullptr, *st = nullptr;
    int sth = 0;
    cs_status rc = CS_OK;
    if ((rc = dalloc_t(&h->cinv, (size_t)n * n, &h->bytes, s)) != CS_OK) return rc;
    if ((rc = dalloc_t(&M, (size_t)n * n, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&W, (size_t)n * n, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&piv, (size_t)n + 1, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&st, 1, nullptr, s)) != CS_OK) goto done;
    k_gdense<<<std::max(1, (n + 127) / 128), 128, 0, s>>>(n, A.rp, A.ci, A.v, M);
    k_factor_inverse<<<1, 256, 0, s>>>(n, M, W, h->cinv, piv, st);
    count_launch(2);
    CSX_CUDA_GOTO(cudaGetLastError());
    CSX_CUDA_GOTO(cudaMemcpyAsync(&sth, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSX_CUDA_GOTO(cudaStreamSynchronize(s));
    if (sth) {
        set_error("coarsest-level matrix (%d x %d) is singular", n, n);
        rc = CS_ERR_SINGULAR;
    }
done:
    dfree(M, s); dfree(W, s); dfree(piv, s); dfree(st, s);
    return rc;
}

}  // namespace csx

using namespace csx;

extern "C" {

void cs_gdestroy_hierarchy(cs_ghier *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (GLevel &L : h->lev) {
        gcsr_free(L.A); gcsr_free(L.P); gcsr_free(L.R);
        dfree(L.bptr); dfree(L.bidx); dfree(L.cblocks); dfree(L.field);
        dfree(L.nptr); dfree(L.nblk); dfree(L.nloc); dfree(L.dpool);
        dfree(L.b); dfree(L.x); dfree(L.t); dfree(L.r);
    }
    dfree(h->cinv); dfree(h->red);
    if (h->red_host) cudaFreeHost(h->red_host);
    delete h;
}

cs_status cs_gsetup_hierarchy(const cs_csr *A0, int nP, const cs_csr *P, double rscale, const int *nblocks,
                              const int *const *bptr, const int *const *bidx, const int *field,
                              uint64_t colour_seed, cs_stream stream, cs_ghier **out) {
    if (!A0 || !out || nP < 0 || (nP > 0 && !P)) { set_error("null argument"); return CS_ERR_ARG; }
    *out = nullptr;
    if (A0->n != A0->m) { set_error("A0 must be square"); return CS_ERR_ARG; }
    if (nP + 1 > 24) { set_error("at most 24 levels"); return CS_ERR_ARG; }
    if (!(rscale > 0.0)) { set_error("rscale must be positive"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cs_ghier *h = new cs_ghier();
    h->rscale = rscale;
    h->nlev = nP + 1;
    h->lev.resize((size_t)h->nlev);
    cs_status rc = CS_OK;
    if ((rc = gcsr_in(*A0, h->lev[0].A, &h->bytes, s)) != CS_OK) goto fail;
    for (int l = 0; l < nP; ++l) {
        GLevel &F = h->lev[l], &Cc = h->lev[l + 1];
        if (P[l].n != F.A.n) { set_error("P[%d] has %d rows, level %d has %d unknowns", l, P[l].n, l, F.A.n); rc = CS_ERR_ARG; goto fail; }
        if ((rc = gcsr_in(P[l], F.P, &h->bytes, s)) != CS_OK) goto fail;
        GCsr AP, Pt;
        rc = gspgemm(F.A, F.P, 1.0, AP, nullptr, s);
        if (rc == CS_OK) rc = gtranspose(F.P, 1.0, Pt, nullptr, s);
        if (rc == CS_OK) rc = gspgemm(Pt, AP, rscale, Cc.A, &h->bytes, s);
        if (rc == CS_OK) rc = gtranspose(F.P, rscale, F.R, &h->bytes, s);
        cudaStreamSynchronize(s);
        gcsr_free(AP); gcsr_free(Pt);
        if (rc != CS_OK) goto fail;
    }
    if (field) {  // fields: the user's on level 0, the coarse ones through the interpolations
        h->lev[0].hfield.assign(field, field + h->lev[0].A.n);
        for (int f : h->lev[0].hfield)
            if (f != 0 && f != 1) { set_error("field values must be 0 or 1"); rc = CS_ERR_ARG; goto fail; }
        for (int l = 0; l + 1 < h->nlev; ++l) {
            const GCsr &Pl = h->lev[l].P;
            std::vector<int> &fc = h->lev[l + 1].hfield;
            fc.assign((size_t)Pl.m, -1);
            for (int i = 0; i < Pl.n; ++i)
                for (int64_t p = Pl.hrp[i]; p < Pl.hrp[i + 1]; ++p) {
                    int &f = fc[Pl.hci[p]];
                    if (f >= 0 && f != h->lev[l].hfield[i]) {
                        set_error("P[%d] maps coarse unknown %d to fine unknowns of two fields", l, Pl.hci[p]);
                        rc = CS_ERR_ARG;
                        goto fail;
                    }
                    f = h->lev[l].hfield[i];
                }
            for (int &f : fc) f = f < 0 ? 0 : f;
        }
        for (int l = 0; l < h->nlev; ++l) {
            GLevel &L = h->lev[l];
            if ((rc = dalloc_t(&L.field, L.hfield.size(), &h->bytes, s)) != CS_OK) goto fail;
            if (cudaMemcpyAsync(L.field, L.hfield.data(), sizeof(int) * L.hfield.size(), cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "copy fields", __FILE__, __LINE__);
                goto fail;
            }
        }
    }
    for (int l = 0; l < h->nlev; ++l) {
        GLevel &L = h->lev[l];
        const int N = L.A.n;
        const int nbl = nblocks ? nblocks[l] : 0;
        if (nbl > 0) {
            const int *bp = bptr ? bptr[l] : nullptr, *bi = bidx ? bidx[l] : nullptr;
            if (!bp || !bi || bp[0] != 0) { set_error("level %d blocks: bad bptr", l); rc = CS_ERR_ARG; goto fail; }
            // every node in at least one block and in no block twice; a node
            // in several blocks makes the level's blocks overlapping
            std::vector<int> cnt((size_t)N, 0), last((size_t)N, -1);
            for (int b = 0; b < nbl; ++b) {
                const int nbk = bp[b + 1] - bp[b];
                if (nbk < 1 || nbk > GMAXBLK) { set_error("level %d block %d has %d nodes (1..%d)", l, b, nbk, GMAXBLK); rc = CS_ERR_ARG; goto fail; }
            }
            if (bp[nbl] > (int64_t)N * GMAXBLK) { set_error("level %d blocks: bad bptr", l); rc = CS_ERR_ARG; goto fail; }
            for (int b = 0; b < nbl; ++b)
                for (int p = bp[b]; p < bp[b + 1]; ++p) {
                    const int i = bi[p];
                    if (i < 0 || i >= N || last[i] == b) { set_error("level %d block %d: node out of range or repeated", l, b); rc = CS_ERR_ARG; goto fail; }
                    last[i] = b;
                    L.overlap |= cnt[i]++ > 0;
                }
            for (int i = 0; i < N; ++i)
                if (!cnt[i]) { set_error("level %d: node %d is in no block", l, i); rc = CS_ERR_ARG; goto fail; }
            L.nb = nbl;
            L.hbptr.assign(bp, bp + nbl + 1);
            L.hbidx.assign(bi, bi + bp[nbl]);
        } else {
            L.nb = N;
            L.hbptr.resize((size_t)N + 1);
            L.hbidx.resize((size_t)N);
            for (int i = 0; i <= N; ++i) L.hbptr[i] = i;
            for (int i = 0; i < N; ++i) L.hbidx[i] = i;
        }
        gnode_blocks(L);
        if ((rc = gcolour(L, l, colour_seed, s)) != CS_OK) goto fail;
        if ((rc = gblock_tables(L, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.b, (size_t)N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.x, (size_t)N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.t, (size_t)N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.r, (size_t)N, &h->bytes, s)) != CS_OK) goto fail;
    }
    if ((rc = gcoarse_factor(h, s)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&h->red, NRED + 8, &h->bytes, s)) != CS_OK) goto fail;
    if (cudaMallocHost(&h->red_host, sizeof(double) * (NRED + 8)) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "pinned reduction buffer", __FILE__, __LINE__);
        goto fail;
    }
    *out = h;
    return CS_OK;
fail:
    cudaStreamSynchronize(s);
    cs_gdestroy_hierarchy(h);
    return rc;
}

int cs_gnlevels(const cs_ghier *h) { return h ? h->nlev : 0; }

cs_status cs_gquery_level(const cs_ghier *h, int level, int *n, int64_t *nnz, int *nblocks, int *ncolours) {
    if (!h) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const GLevel &L = h->lev[level];
    if (n) *n = L.A.n;
    if (nnz) *nnz = L.A.nnz;
    if (nblocks) *nblocks = L.nb;
    if (ncolours) *ncolours = L.ncol;
    return CS_OK;
}

cs_status cs_gexport_operator(const cs_ghier *h, int level, int64_t *rowptr, int32_t *col, double *val) {
    if (!h || !rowptr || !col || !val) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const GLevel &L = h->lev[level];
    CSX_CUDA(cudaDeviceSynchronize());
    std::memcpy(rowptr, L.A.hrp.data(), sizeof(int64_t) * ((size_t)L.A.n + 1));
    std::memcpy(col, L.A.hci.data(), sizeof(int) * (size_t)L.A.nnz);
    CSX_CUDA(cudaMemcpy(val, L.A.v, sizeof(double) * (size_t)L.A.nnz, cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_gexport_colours(const cs_ghier *h, int level, int32_t *colour) {
    if (!h || !colour) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const GLevel &L = h->lev[level];
    std::memcpy(colour, L.hcol.data(), sizeof(int) * (size_t)L.nb);
    return CS_OK;
}

cs_status cs_gexport_blocks(const cs_ghier *h, int level, int32_t *bptr, int32_t *bidx) {
    if (!h || !bptr) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const GLevel &L = h->lev[level];
    std::memcpy(bptr, L.hbptr.data(), sizeof(int) * L.hbptr.size());
    if (bidx) std::memcpy(bidx, L.hbidx.data(), sizeof(int) * L.hbidx.size());
    return CS_OK;
}

}  // extern "C"

namespace csx {

// ------------------------------------------------------------ cascade setup
// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix a, one
// thread: a is left diagonal (the eigenvalues), q holds the eigenvectors in
// its columns; sweeps until the squared off-diagonal mass is below 1e-300,
// 100 at most.
__device__ void gjacobi(int n, double *a, double *q) {
    for (int i = 0; i < n * n; ++i) q[i] = 0.0;
    for (int i = 0; i < n; ++i) q[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p)
            for (int r = p + 1; r < n; ++r) {
                const double apr = a[p * n + r];
                if (apr == 0.0) continue;
                const double th = (a[r * n + r] - a[p * n + p]) / (2.0 * apr);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = a[k * n + p], akr = a[k * n + r];
                    a[k * n + p] = c * akp - s * akr;
                    a[k * n + r] = s * akp + c * akr;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a[p * n + k], ark = a[r * n + k];
                    a[p * n + k] = c * apk - s * ark;
                    a[r * n + k] = s * apk + c * ark;
                }
                for (int k = 0; k < n; ++k) {
                    const double qkp = q[k * n + p], qkr = q[k * n + r];
                    q[k * n + p] = c * qkp - s * qkr;
                    q[k * n + r] = s * qkp + c * qkr;
                }
            }
    }
}

// Lambda~ (n x n) = C G^{-1} for a symmetric positive semidefinite G, one
// thread: Cholesky when every pivot exceeds 1e-14 tr(G); otherwise the
// minimum-norm solution C G^+, eigenvalues at or below 1e-14 tr(G) taken as
// zero, from a cyclic Jacobi eigendecomposition (sweeps until the squared
// off-diagonal mass is below 1e-300, 100 at most).  G is destroyed.
__device__ void gls_small(int n, double *G, const double *C, double *L, double *Q) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += G[i * n + i];
    const double tol = 1e-14 * tr;
    bool ok = tr > 0.0;
    for (int i = 0; i < n * n; ++i) Q[i] = G[i];
    for (int j = 0; j < n && ok; ++j) {  // Q <- lower Cholesky factor
        double d = Q[j * n + j];
        for (int k = 0; k < j; ++k) d -= Q[j * n + k] * Q[j * n + k];
        if (!(d > tol)) { ok = false; break; }
        d = sqrt(d);
        Q[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = Q[i * n + j];
            for (int k = 0; k < j; ++k) s -= Q[i * n + k] * Q[j * n + k];
            Q[i * n + j] = s / d;
        }
    }
    if (ok) {
        for (int p = 0; p < n; ++p) {  // row p of Lambda: solve Q Q^T y = C_p
            double y[GMAXBLK];
            for (int i = 0; i < n; ++i) {
                double s = C[p * n + i];
                for (int k = 0; k < i; ++k) s -= Q[i * n + k] * y[k];
                y[i] = s / Q[i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = y[i];
                for (int k = i + 1; k < n; ++k) s -= Q[k * n + i] * y[k];
                y[i] = s / Q[i * n + i];
            }
            for (int i = 0; i < n; ++i) L[p * n + i] = y[i];
        }
        return;
    }
    gjacobi(n, G, Q);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) {
                const double ev = G[k * n + k];
                if (!(ev > tol)) continue;
                double cq = 0.0;
                for (int m = 0; m < n; ++m) cq += C[p * n + m] * Q[m * n + k];
                acc += cq * Q[q * n + k] / ev;
            }
            L[p * n + q] = acc;
        }
}

// Scratch doubles one thread needs for gproject_spd (and the block of A~).
constexpr int GSPD_SCR = 7 * GMAXBLK * GMAXBLK + 2 * GMAXBLK;

// The SPD projection of one block of Lambda~ (SM "On preconditioned
// conjugate gradient"), one thread, L (n x n) in place.  D = A~_bb, the
// block's diagonal block of the prescaled operator.  When D is positive
// definite: with D = U diag(d) U^T, Dh = D^{1/2}, Di = D^{-1/2}, the
// symmetric part S of L is mapped to M = Dh S Dh = Q diag(m) Q^T and back
// as Di Q diag(min(max(m, 0), 1)) Q^T Di: the D-weighted Frobenius-nearest
// matrix between 0 and the block-Jacobi block D^{-1}.  Otherwise the
// nearest positive semidefinite matrix (S with its negative eigenvalues
// set to zero).
__device__ void gproject_spd(int n, double *L, const double *D, double *scr) {
    const int nn = n * n;
    double *S = scr, *Q = S + nn, *U = Q + nn, *T = U + nn, *Dh = T + nn, *Di = Dh + nn, *dv = Di + nn;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) S[p * n + q] = 0.5 * (L[p * n + q] + L[q * n + p]);
    for (int e = 0; e < nn; ++e) T[e] = D[e];
    gjacobi(n, T, U);
    bool pd = true;
    for (int k = 0; k < n; ++k) {
        dv[k] = T[k * n + k];
        pd = pd && dv[k] > 0.0;
    }
    if (pd) {
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double sq = sqrt(dv[k]);
                    a += U[p * n + k] * sq * U[q * n + k];
                    b += U[p * n + k] / sq * U[q * n + k];
                }
                Dh[p * n + q] = a;
                Di[p * n + q] = b;
            }
        for (int p = 0; p < n; ++p)  // T = Dh S Dh
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int r = 0; r < n; ++r)
                    for (int t = 0; t < n; ++t) a += Dh[p * n + r] * S[r * n + t] * Dh[t * n + q];
                T[p * n + q] = a;
            }
        gjacobi(n, T, Q);
        for (int p = 0; p < n; ++p)  // S = Q diag(clip(m)) Q^T
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int k = 0; k < n; ++k) a += Q[p * n + k] * fmin(fmax(T[k * n + k], 0.0), 1.0) * Q[q * n + k];
                S[p * n + q] = a;
            }
        for (int p = 0; p < n; ++p)  // L = Di S Di
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int r = 0; r < n; ++r)
                    for (int t = 0; t < n; ++t) a += Di[p * n + r] * S[r * n + t] * Di[t * n + q];
                L[p * n + q] = a;
            }
    } else {
        for (int e = 0; e < nn; ++e) T[e] = S[e];
        gjacobi(n, T, Q);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double ev = T[k * n + k];
                    if (ev > 0.0) a += Q[p * n + k] * ev * Q[q * n + k];
                }
                L[p * n + q] = a;
            }
    }
}

// The prescaling W (Sec. 2.3; SM "Prescaling Stokes problems"):
// mode CS_PRESCALE_NONE: 1; CS_PRESCALE_ELLIPTIC: A_ii^{-1/2};
// Stokes (q = 1, 2, infinity): a velocity / scalar unknown (field 0) takes
// sqrt(||A_{i,:}||_1) / A_ii over the field-0 columns (pass 0), a pressure
// unknown (field 1) the inverse q-norm of its field-0 columns scaled by
// their weights (pass 1, after pass 0).  bad = 1 when a weight is undefined.
__global__ void k_gprescale(int n, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const int *__restrict__ field, int mode, int pass,
                            double *__restrict__ w, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int fi = field ? field[i] : 0;
        if (pass == 0) {
            double d = 0.0, l1 = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                if (ci[p] == i) d += v[p];
                if (!field || field[ci[p]] == 0) l1 += fabs(v[p]);
            }
            if (mode == CS_PRESCALE_NONE) {
                w[i] = 1.0;
            } else if (mode == CS_PRESCALE_ELLIPTIC) {
                if (!(d > 0.0)) atomicExch(bad, 1);
                w[i] = 1.0 / sqrt(d);
            } else if (fi == 0) {
                if (!(d > 0.0) || !(l1 > 0.0)) atomicExch(bad, 1);
                w[i] = sqrt(l1) / d;
            }
        } else if (mode >= CS_PRESCALE_STOKES_L1 && fi == 1) {
            double nrm = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                if (field[ci[p]] != 0) continue;
                const double a = fabs(v[p]) * w[ci[p]];
                if (mode == CS_PRESCALE_STOKES_L1) nrm += a;
                else if (mode == CS_PRESCALE_STOKES_L2) nrm += a * a;
                else nrm = fmax(nrm, a);
            }
            if (mode == CS_PRESCALE_STOKES_L2) nrm = sqrt(nrm);
            if (!(nrm > 0.0)) atomicExch(bad, 1);
            w[i] = 1.0 / nrm;
        }
    }
}
__global__ void k_gscale_op(int n, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const double *__restrict__ w, double *__restrict__ at) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) at[p] = __dmul_rn(__dmul_rn(w[i], v[p]), w[ci[p]]);
}

// The residual rows of one cascade step in group-row storage: group c holds
// cols[coff[c] .. + u[c]) (ascending) and values [n_c][u[c]] at voff[c];
// ident[c]: the group's rows are still the identity rows (E_0).  The groups
// are the blocks of a partition (n_c = the block's nodes), or the nodes
// (n_c = 1) when blocks overlap; grp[j] / gloc[j] give node j's group and
// row in it.
struct GEView {
    const int64_t *coff, *voff;
    const int *u, *cols;
    const char *ident;
    const double *vals;
};

constexpr int GSETUP_WARPS = 4;

// One step for the listed blocks: R_b = (A~ E)_{b,:} over the new pattern,
// E_b mapped into it, G = R_b R_b^T, C = E_b R_b^T, Lambda~_b (projected
// when spd_scr is given: GSPD_SCR doubles per warp of the grid), the new
// rows E_b - Lambda~_b R_b (block-row storage at nvoff[b]), and the
// unscaled Lambda_b = W_b Lambda~_b W_b.
__global__ void __launch_bounds__(32 * GSETUP_WARPS) k_gsetup_step(
    int nupd, const int *__restrict__ upd, const int *__restrict__ bptr, const int *__restrict__ bidx,
    const int *__restrict__ grp, const int *__restrict__ gloc, const int64_t *__restrict__ arp,
    const int *__restrict__ aci, const double *__restrict__ at, GEView E, const int64_t *__restrict__ ncoff,
    const int64_t *__restrict__ nvoff, const int *__restrict__ nu, const int *__restrict__ ncols,
    double *__restrict__ nvals, double *__restrict__ Rpool, const int64_t *__restrict__ lamoff,
    const double *__restrict__ w, double *__restrict__ lam, double *__restrict__ spd_scr) {
    __shared__ double sh[GSETUP_WARPS][4][GMAXBLK * GMAXBLK];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    double *G = sh[wl][0], *Cm = sh[wl][1], *Lt = sh[wl][2], *Q = sh[wl][3];
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < nupd; k += nw) {
        const int b = upd[k];
        const int n = bptr[b + 1] - bptr[b];
        const int *rows = bidx + bptr[b];
        const int u = nu[b];
        const int *U = ncols + ncoff[b];
        double *Rb = Rpool + nvoff[b], *Eb = nvals + nvoff[b];
        for (int e = lane; e < n * u; e += 32) { Rb[e] = 0.0; Eb[e] = 0.0; }
        __syncwarp();
        for (int p = 0; p < n; ++p) {
            const int row = rows[p];
            for (int64_t q = arp[row]; q < arp[row + 1]; ++q) {
                const int j = aci[q];
                const double a = at[q];
                const int c = grp[j];
                if (E.ident[c]) {
                    if (lane == 0) {
                        const int64_t pos = gfind(U, 0, u, j);
                        Rb[p * u + pos] = __dadd_rn(Rb[p * u + pos], a);
                    }
                } else {
                    const int uc = E.u[c];
                    const int *Uc = E.cols + E.coff[c];
                    const double *Ec = E.vals + E.voff[c] + (int64_t)gloc[j] * uc;
                    for (int t = lane; t < uc; t += 32) {
                        const int64_t pos = gfind(U, 0, u, Uc[t]);
                        Rb[p * u + pos] = __dadd_rn(Rb[p * u + pos], __dmul_rn(a, Ec[t]));
                    }
                }
                __syncwarp();
            }
        }
        for (int p = 0; p < n; ++p) {  // the block's own rows of E
            const int r = rows[p], g = grp[r];
            if (E.ident[g]) {
                if (lane == 0) Eb[p * u + gfind(U, 0, u, r)] = 1.0;
            } else {
                const int ug = E.u[g];
                const int *Ug = E.cols + E.coff[g];
                const double *Eo = E.vals + E.voff[g] + (int64_t)gloc[r] * ug;
                for (int t = lane; t < ug; t += 32) Eb[p * u + gfind(U, 0, u, Ug[t])] = Eo[t];
            }
        }
        __syncwarp();
        for (int pq = 0; pq < n * n; ++pq) {
            const int p = pq / n, q = pq - p * n;
            double g = 0.0, cc = 0.0;
            for (int t = lane; t < u; t += 32) {
                g = fma(Rb[p * u + t], Rb[q * u + t], g);
                cc = fma(Eb[p * u + t], Rb[q * u + t], cc);
            }
            for (int o = 16; o > 0; o >>= 1) {
                g += __shfl_xor_sync(0xffffffffu, g, o);
                cc += __shfl_xor_sync(0xffffffffu, cc, o);
            }
            if (lane == 0) { G[pq] = g; Cm[pq] = cc; }
        }
        __syncwarp();
        if (lane == 0) {
            gls_small(n, G, Cm, Lt, Q);
            if (spd_scr) {  // D = A~_bb in G, then the projection of Lt
                double *scr = spd_scr + (int64_t)w0 * GSPD_SCR;
                for (int e = 0; e < n * n; ++e) G[e] = 0.0;
                for (int p = 0; p < n; ++p)
                    for (int64_t q = arp[rows[p]]; q < arp[rows[p] + 1]; ++q)
                        for (int t = 0; t < n; ++t)
                            if (aci[q] == rows[t]) G[p * n + t] += at[q];
                gproject_spd(n, Lt, G, scr);
            }
        }
        __syncwarp();
        for (int t = lane; t < u; t += 32)
            for (int p = 0; p < n; ++p) {
                double sacc = Eb[p * u + t];
                for (int q = 0; q < n; ++q) sacc = __dsub_rn(sacc, __dmul_rn(Lt[p * n + q], Rb[q * u + t]));
                Eb[p * u + t] = sacc;
            }
        for (int pq = lane; pq < n * n; pq += 32) {
            const int p = pq / n, q = pq - p * n;
            lam[lamoff[b] + pq] = __dmul_rn(Lt[pq], __dmul_rn(w[rows[p]], w[rows[q]]));
        }
        __syncwarp();
    }
}

// blocks that keep their rows in this step: values copied to the new pool
__global__ void k_gsetup_copy(int ncp, const int *__restrict__ cp, const int *__restrict__ bptr, GEView E,
                              const int64_t *__restrict__ nvoff, double *__restrict__ nvals) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < ncp; k += nw) {
        const int b = cp[k];
        if (E.ident[b]) continue;
        const int64_t cnt = (int64_t)(bptr[b + 1] - bptr[b]) * E.u[b];
        for (int64_t e = lane; e < cnt; e += 32) nvals[nvoff[b] + e] = E.vals[E.voff[b] + e];
    }
}

// Overlapping blocks, node rows after a step (Sec. 3.6.2): node i's new row
// sums, in ascending block order over the union of their columns, the rows
// fptr[i] .. fptr[i+1] of the updated blocks holding it (block fblk, row
// floc, block-row storage B), divided by their count when average is set
// (the additive form: diag(theta)^{-1} Theta^T); a node no updated block
// holds keeps its row of E.  One warp per node.
__global__ void k_gfuse(int N, const int *__restrict__ fptr, const int *__restrict__ fblk,
                        const int *__restrict__ floc, GEView B, GEView E, const int64_t *__restrict__ ncoff,
                        const int64_t *__restrict__ nvoff, const int *__restrict__ nu,
                        const int *__restrict__ ncols, double *__restrict__ nvals, int average) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < N; i += nw) {
        const int c0 = fptr[i], c1 = fptr[i + 1], uo = nu[i];
        double *out = nvals + nvoff[i];
        if (c0 == c1) {
            if (!E.ident[i])
                for (int t = lane; t < uo; t += 32) out[t] = E.vals[E.voff[i] + t];
            continue;
        }
        const int *Uo = ncols + ncoff[i];
        for (int t = lane; t < uo; t += 32) out[t] = 0.0;
        __syncwarp();
        for (int c = c0; c < c1; ++c) {
            const int b = fblk[c], ub = B.u[b];
            const int *Ub = B.cols + B.coff[b];
            const double *src = B.vals + B.voff[b] + (int64_t)floc[c] * ub;
            for (int t = lane; t < ub; t += 32) {
                const int64_t pos = gfind(Uo, 0, uo, Ub[t]);
                out[pos] = __dadd_rn(out[pos], src[t]);
            }
            __syncwarp();
        }
        if (average) {
            const double th = (double)(c1 - c0);
            for (int t = lane; t < uo; t += 32) out[t] = out[t] / th;
        }
        __syncwarp();
    }
}

}  // namespace csx

namespace csx {

struct GEHost {  // host side of a step's residual rows (patterns) and the device arrays
    std::vector<int> u;
    std::vector<int64_t> coff, voff;
    std::vector<int> cols;
    std::vector<char> ident;
    int64_t nvals = 0;
    int64_t *dcoff = nullptr, *dvoff = nullptr;
    int *du = nullptr, *dcols = nullptr;
    char *dident = nullptr;
    double *dvals = nullptr;
    void release(cudaStream_t s) {
        dfree(dcoff, s); dfree(dvoff, s); dfree(du, s); dfree(dcols, s); dfree(dident, s); dfree(dvals, s);
        dcoff = dvoff = nullptr; du = dcols = nullptr; dident = nullptr; dvals = nullptr;
    }
    GEView view() const { return GEView{dcoff, dvoff, du, dcols, dident, dvals}; }
};

static cs_status gehost_upload(GEHost &E, cudaStream_t s) {
    const size_t nb = E.u.size();
    CSX_TRY(dalloc_t(&E.dcoff, nb, nullptr, s));
    CSX_TRY(dalloc_t(&E.dvoff, nb, nullptr, s));
    CSX_TRY(dalloc_t(&E.du, nb, nullptr, s));
    CSX_TRY(dalloc_t(&E.dcols, std::max<size_t>(E.cols.size(), 1), nullptr, s));
    CSX_TRY(dalloc_t(&E.dident, nb, nullptr, s));
    CSX_TRY(dalloc_t(&E.dvals, (size_t)std::max<int64_t>(E.nvals, 1), nullptr, s));
    CSX_CUDA(cudaMemcpyAsync(E.dcoff, E.coff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(E.dvoff, E.voff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(E.du, E.u.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    if (!E.cols.empty())
        CSX_CUDA(cudaMemcpyAsync(E.dcols, E.cols.data(), sizeof(int) * E.cols.size(), cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaMemcpyAsync(E.dident, E.ident.data(), nb, cudaMemcpyHostToDevice, s));
    CSX_CUDA(cudaStreamSynchronize(s));  // the host vectors may change afterwards
    return CS_OK;
}

// Column pattern of block b's new rows: the union of the columns of its rows
// of A~ E and of its own rows of E, ascending.
static void gblock_pattern(const GLevel &L, int b, const GEHost &E, const std::vector<int> &grp,
                           std::vector<int> &mark, int stamp, std::vector<int> &row) {
    row.clear();
    auto add = [&](int c) { if (mark[c] != stamp) { mark[c] = stamp; row.push_back(c); } };
    auto add_row = [&](int j) {
        const int g = grp[j];
        if (E.ident[g]) add(j);
        else for (int t = 0; t < E.u[g]; ++t) add(E.cols[E.coff[g] + t]);
    };
    for (int p = L.hbptr[b]; p < L.hbptr[b + 1]; ++p) {
        const int r = L.hbidx[p];
        for (int64_t q = L.A.hrp[r]; q < L.A.hrp[r + 1]; ++q) add_row(L.A.hci[q]);
        add_row(r);
    }
    std::sort(row.begin(), row.end());
}

static cs_status gsetup_level(const cs_ghier *h, int l, int kind, int nu, int prescale, int spd, double *lam,
                              const int64_t *dlamoff, int64_t lamsize, cudaStream_t s) {
    const GLevel &L = h->lev[l];
    const int N = L.A.n, nb = L.nb;
    const bool over = L.overlap != 0;
    const int ng = over ? N : nb;  // row groups of E: the blocks, or the nodes when blocks overlap
    std::vector<int> grp((size_t)N), gloc((size_t)N, 0);
    if (over) {
        for (int i = 0; i < N; ++i) grp[i] = i;
    } else {
        for (int b = 0; b < nb; ++b)
            for (int p = L.hbptr[b]; p < L.hbptr[b + 1]; ++p) { grp[L.hbidx[p]] = b; gloc[L.hbidx[p]] = p - L.hbptr[b]; }
    }
    double *w = nullptr, *at = nullptr, *R = nullptr, *scr = nullptr;
    int *dgrp = nullptr, *dgloc = nullptr, *bad = nullptr, *dlist = nullptr;
    int *dfp = nullptr, *dfb = nullptr, *dfl = nullptr;
    int badh = 0;
    GEHost E, En, B;
    cs_status rc = CS_OK;
    // per host thread: column marks (allocated on first use) and stamps
    std::vector<std::vector<int>> marks(16);
    std::vector<int> stamps(16, 0);
    const int ncol = kind == CS_MULTIPLICATIVE ? L.ncol : 1;
    const unsigned spd_grid = 152 * 4;
    if ((rc = dalloc_t(&w, (size_t)N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&at, (size_t)std::max<int64_t>(L.A.nnz, 1), nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&dgrp, (size_t)N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&dgloc, (size_t)N, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&bad, 1, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&dlist, (size_t)nb, nullptr, s)) != CS_OK) goto done;
    if (spd && (rc = dalloc_t(&scr, (size_t)spd_grid * GSETUP_WARPS * GSPD_SCR, nullptr, s)) != CS_OK) goto done;
    if (over) {
        if ((rc = dalloc_t(&dfp, (size_t)N + 1, nullptr, s)) != CS_OK) goto done;
        if ((rc = dalloc_t(&dfb, L.hnblk.size(), nullptr, s)) != CS_OK) goto done;
        if ((rc = dalloc_t(&dfl, L.hnloc.size(), nullptr, s)) != CS_OK) goto done;
    }
    CSX_CUDA_GOTO(cudaMemsetAsync(bad, 0, sizeof(int), s));
    CSX_CUDA_GOTO(cudaMemcpyAsync(dgrp, grp.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s));
    CSX_CUDA_GOTO(cudaMemcpyAsync(dgloc, gloc.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s));
    CSX_CUDA_GOTO(cudaMemsetAsync(lam, 0, sizeof(double) * (size_t)nu * lamsize, s));
    for (int pass = 0; pass < 2; ++pass)
        k_gprescale<<<std::max(1, std::min(1216, (N + 255) / 256)), 256, 0, s>>>(N, L.A.rp, L.A.ci, L.A.v, L.field,
                                                                                   prescale, pass, w, bad);
    k_gscale_op<<<std::max(1, std::min(1216, (N + 255) / 256)), 256, 0, s>>>(N, L.A.rp, L.A.ci, L.A.v, w, at);
    count_launch(3);
    CSX_CUDA_GOTO(cudaGetLastError());
    CSX_CUDA_GOTO(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSX_CUDA_GOTO(cudaStreamSynchronize(s));
    if (badh) {
        set_error("level %d: a prescaling weight is undefined (non-positive diagonal or norm)", l);
        rc = CS_ERR_ARG;
        goto done;
    }
    // E_0 = I: identity rows, no storage
    E.u.assign((size_t)ng, 0);
    E.coff.assign((size_t)ng, 0);
    E.voff.assign((size_t)ng, 0);
    E.ident.assign((size_t)ng, 1);
    if ((rc = gehost_upload(E, s)) != CS_OK) goto done;
    for (int step = 0; step < nu; ++step)
        for (int k = 0; k < ncol; ++k) {
            std::vector<char> upd((size_t)nb, 0);
            std::vector<int> ulist, clist;
            for (int b = 0; b < nb; ++b) {
                upd[b] = kind != CS_MULTIPLICATIVE || L.hcol[b] == k;
                (upd[b] ? ulist : clist).push_back(b);
            }
            // the updated blocks' new rows in block-row storage: the new E
            // itself for a partition (the other blocks keep their rows), a
            // staging pool fused into node rows when blocks overlap
            GEHost &P = over ? B : En;
            P.u.assign((size_t)nb, 0);
            P.coff.assign((size_t)nb, 0);
            P.voff.assign((size_t)nb, 0);
            P.ident.assign((size_t)nb, 0);
            P.cols.clear();
            P.nvals = 0;
            {
                std::vector<std::vector<int>> part(16);
                const int T = gpar_ranges(nb, [&](int t, int64_t lo, int64_t hi) {
                    if (marks[t].empty()) marks[t].assign((size_t)N, -1);
                    std::vector<int> rw;
                    for (int64_t b = lo; b < hi; ++b) {
                        if (upd[b]) {
                            gblock_pattern(L, (int)b, E, grp, marks[t], ++stamps[t], rw);
                            P.u[b] = (int)rw.size();
                            part[t].insert(part[t].end(), rw.begin(), rw.end());
                        } else if (!over) {
                            P.ident[b] = E.ident[b];
                            P.u[b] = E.u[b];
                            part[t].insert(part[t].end(), E.cols.begin() + E.coff[b],
                                           E.cols.begin() + E.coff[b] + E.u[b]);
                        }
                    }
                });
                int64_t nc = 0;
                for (int b = 0; b < nb; ++b) {
                    P.coff[b] = nc;
                    P.voff[b] = P.nvals;
                    nc += P.u[b];
                    P.nvals += (int64_t)(L.hbptr[b + 1] - L.hbptr[b]) * P.u[b];
                }
                P.cols.reserve((size_t)nc);
                for (int t = 0; t < T; ++t) P.cols.insert(P.cols.end(), part[t].begin(), part[t].end());
            }
            if ((rc = gehost_upload(P, s)) != CS_OK) goto done;
            std::vector<int> fp, fb, fl;
            if (over) {  // node rows: the union of the patterns of the updated blocks holding the node
                fp.assign((size_t)N + 1, 0);
                En.u.assign((size_t)N, 0);
                En.coff.assign((size_t)N, 0);
                En.voff.assign((size_t)N, 0);
                En.ident.assign((size_t)N, 0);
                En.cols.clear();
                En.nvals = 0;
                std::vector<std::vector<int>> pcols(16), pfb(16), pfl(16);
                std::vector<int> ncontrib((size_t)N, 0);
                const int T = gpar_ranges(N, [&](int t, int64_t lo, int64_t hi) {
                    if (marks[t].empty()) marks[t].assign((size_t)N, -1);
                    std::vector<int> &mk = marks[t];
                    std::vector<int> rw;
                    for (int64_t i = lo; i < hi; ++i) {
                        const int st = ++stamps[t];
                        rw.clear();
                        for (int u = L.hnptr[i]; u < L.hnptr[i + 1]; ++u) {
                            const int b = L.hnblk[u];
                            if (!upd[b]) continue;
                            pfb[t].push_back(b);
                            pfl[t].push_back(L.hnloc[u]);
                            ++ncontrib[i];
                            for (int q = 0; q < P.u[b]; ++q) {
                                const int c = P.cols[P.coff[b] + q];
                                if (mk[c] != st) { mk[c] = st; rw.push_back(c); }
                            }
                        }
                        if (!ncontrib[i]) {
                            En.ident[i] = E.ident[i];
                            En.u[i] = E.u[i];
                            pcols[t].insert(pcols[t].end(), E.cols.begin() + E.coff[i],
                                            E.cols.begin() + E.coff[i] + E.u[i]);
                        } else {
                            std::sort(rw.begin(), rw.end());
                            En.u[i] = (int)rw.size();
                            pcols[t].insert(pcols[t].end(), rw.begin(), rw.end());
                        }
                    }
                });
                int64_t nc = 0;
                for (int i = 0; i < N; ++i) {
                    fp[i + 1] = fp[i] + ncontrib[i];
                    En.coff[i] = nc;
                    En.voff[i] = En.nvals;
                    nc += En.u[i];
                    En.nvals += En.u[i];
                }
                En.cols.reserve((size_t)nc);
                for (int t = 0; t < T; ++t) {
                    En.cols.insert(En.cols.end(), pcols[t].begin(), pcols[t].end());
                    fb.insert(fb.end(), pfb[t].begin(), pfb[t].end());
                    fl.insert(fl.end(), pfl[t].begin(), pfl[t].end());
                }
                if ((rc = gehost_upload(En, s)) != CS_OK) goto done;
                CSX_CUDA_GOTO(cudaMemcpyAsync(dfp, fp.data(), sizeof(int) * fp.size(), cudaMemcpyHostToDevice, s));
                if (!fb.empty()) {
                    CSX_CUDA_GOTO(cudaMemcpyAsync(dfb, fb.data(), sizeof(int) * fb.size(), cudaMemcpyHostToDevice, s));
                    CSX_CUDA_GOTO(cudaMemcpyAsync(dfl, fl.data(), sizeof(int) * fl.size(), cudaMemcpyHostToDevice, s));
                }
            }
            if ((rc = dalloc_t(&R, (size_t)std::max<int64_t>(P.nvals, 1), nullptr, s)) != CS_OK) goto done;
            std::vector<int> lists(ulist);
            lists.insert(lists.end(), clist.begin(), clist.end());
            CSX_CUDA_GOTO(cudaMemcpyAsync(dlist, lists.data(), sizeof(int) * (size_t)nb, cudaMemcpyHostToDevice, s));
            if (!ulist.empty()) {
                const unsigned grid = spd ? std::min(gwarp_blocks((int64_t)ulist.size()) * 2, spd_grid)
                                          : gwarp_blocks((int64_t)ulist.size()) * 2;
                k_gsetup_step<<<grid, 32 * GSETUP_WARPS, 0, s>>>(
                    (int)ulist.size(), dlist, L.bptr, L.bidx, dgrp, dgloc, L.A.rp, L.A.ci, at, E.view(), P.dcoff,
                    P.dvoff, P.du, P.dcols, P.dvals, R, dlamoff, w, lam + (int64_t)step * lamsize, scr);
                count_launch();
            }
            if (over) {
                k_gfuse<<<gwarp_blocks(N), 256, 0, s>>>(N, dfp, dfb, dfl, P.view(), E.view(), En.dcoff, En.dvoff,
                                                         En.du, En.dcols, En.dvals, kind == CS_ADDITIVE ? 1 : 0);
                count_launch();
            } else if (!clist.empty()) {
                k_gsetup_copy<<<gwarp_blocks((int64_t)clist.size()), 256, 0, s>>>(
                    (int)clist.size(), dlist + ulist.size(), L.bptr, E.view(), En.dvoff, En.dvals);
                count_launch();
            }
            CSX_CUDA_GOTO(cudaGetLastError());
            CSX_CUDA_GOTO(cudaStreamSynchronize(s));
            dfree(R, s);
            R = nullptr;
            B.release(s);
            E.release(s);
            std::swap(E, En);
        }
done:
    E.release(s);
    En.release(s);
    B.release(s);
    dfree(R, s); dfree(w, s); dfree(at, s); dfree(dgrp, s); dfree(dgloc, s); dfree(bad, s); dfree(dlist, s);
    dfree(scr, s); dfree(dfp, s); dfree(dfb, s); dfree(dfl, s);
    return rc;
}

}  // namespace csx

extern "C" {

void cs_gdestroy_cascade(cs_gcascade *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (double *p : c->lam) dfree(p);
    for (int64_t *p : c->lamoff) dfree(p);
    dfree(c->gm_V); dfree(c->gm_Z); dfree(c->gm_h); dfree(c->cg);
    delete c;
}

cs_status cs_gsetup_cascade(cs_ghier *h, int kind, int nu, int prescale, int spd, cs_stream stream,
                            cs_gcascade **out) {
    if (!h || !out) { set_error("null argument"); return CS_ERR_ARG; }
    *out = nullptr;
    if (kind != CS_ADDITIVE && kind != CS_MULTIPLICATIVE) { set_error("bad cascade kind"); return CS_ERR_ARG; }
    if (nu < 1 || nu > 8) { set_error("nu must be in 1..8"); return CS_ERR_ARG; }
    if (prescale < CS_PRESCALE_NONE || prescale > CS_PRESCALE_STOKES_LINF) { set_error("bad prescaling mode"); return CS_ERR_ARG; }
    if (spd != 0 && spd != 1) { set_error("spd must be 0 or 1"); return CS_ERR_ARG; }
    if (prescale >= CS_PRESCALE_STOKES_L1 && h->lev[0].hfield.empty()) {
        set_error("Stokes prescaling needs the fields of the unknowns");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cs_gcascade *c = new cs_gcascade();
    c->h = h;
    c->kind = kind;
    c->nu = nu;
    c->nlev = h->nlev > 1 ? h->nlev - 1 : 1;
    c->lam.assign((size_t)c->nlev, nullptr);
    c->lamoff.assign((size_t)c->nlev, nullptr);
    c->hlamoff.resize((size_t)c->nlev);
    c->lamsize.assign((size_t)c->nlev, 0);
    cs_status rc = CS_OK;
    for (int l = 0; l < c->nlev && rc == CS_OK; ++l) {
        const GLevel &L = h->lev[l];
        std::vector<int64_t> &off = c->hlamoff[l];
        off.assign((size_t)L.nb + 1, 0);
        for (int b = 0; b < L.nb; ++b) {
            const int64_t n = L.hbptr[b + 1] - L.hbptr[b];
            off[b + 1] = off[b] + n * n;
        }
        c->lamsize[l] = off[L.nb];
        if ((rc = dalloc_t(&c->lamoff[l], off.size(), &c->bytes, s)) != CS_OK) break;
        if ((rc = dalloc_t(&c->lam[l], (size_t)nu * c->lamsize[l], &c->bytes, s)) != CS_OK) break;
        if (cudaMemcpyAsync(c->lamoff[l], off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "copy block offsets", __FILE__, __LINE__);
            break;
        }
        rc = gsetup_level(h, l, kind, nu, prescale, spd, c->lam[l], c->lamoff[l], c->lamsize[l], s);
    }
    if (rc != CS_OK) {
        cudaStreamSynchronize(s);
        cs_gdestroy_cascade(c);
        return rc;
    }
    *out = c;
    return CS_OK;
}

int64_t cs_glamsize(const cs_gcascade *c, int level) {
    return (c && level >= 0 && level < c->nlev) ? c->lamsize[level] : 0;
}

cs_status cs_gexport_lambda(const cs_gcascade *c, int level, double *host) {
    if (!c || !host) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("level %d has no smoother", level); return CS_ERR_ARG; }
    CSX_CUDA(cudaDeviceSynchronize());
    CSX_CUDA(cudaMemcpy(host, c->lam[level], sizeof(double) * (size_t)c->nu * c->lamsize[level],
                        cudaMemcpyDeviceToHost));
    return CS_OK;
}

}  // extern "C"

namespace csx {

// ---------------------------------------------------------------- cycles
// point blocks: out_i = x_i - lam_b (A x - b)_i for the selected blocks
// (sel == nullptr: blocks 0..n-1), one thread per block; ident: block b is
// node b (no partition tables read)
__global__ void k_gsweep_point(int n, const int *__restrict__ sel, const int *__restrict__ bptr,
                               const int *__restrict__ bidx, const int64_t *__restrict__ rp,
                               const int *__restrict__ ci, const double *__restrict__ v,
                               const double *__restrict__ lam, const int64_t *__restrict__ lamoff,
                               const double *__restrict__ bv, const double *x, double *out, int ident) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int blkid = sel ? sel[k] : k;
        const int i = ident ? blkid : bidx[bptr[blkid]];
        double r = -bv[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) r = fma(v[p], x[ci[p]], r);
        out[i] = fma(-lam[ident ? (int64_t)blkid : lamoff[blkid]], r, x[i]);
    }
}

// blocks: one warp per selected block, lane p holds row p's residual;
// x_p - sum_q Lambda_pq r_q (Lambda^T with transpose)
__global__ void k_gsweep_block(int n, const int *__restrict__ sel, const int *__restrict__ bptr,
                               const int *__restrict__ bidx, const int64_t *__restrict__ rp,
                               const int *__restrict__ ci, const double *__restrict__ v,
                               const double *__restrict__ lam, const int64_t *__restrict__ lamoff,
                               const double *__restrict__ bv, const double *x, double *out, int transpose) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < n; k += nw) {
        const int blkid = sel ? sel[k] : (int)k;
        const int b0 = bptr[blkid], nbk = bptr[blkid + 1] - b0;
        const double *Lb = lam + lamoff[blkid];
        double r = 0.0, xi = 0.0;
        int i = 0;
        if (lane < nbk) {
            i = bidx[b0 + lane];
            r = -bv[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) r = fma(v[p], x[ci[p]], r);
            xi = x[i];
        }
        double acc = 0.0;
        for (int q = 0; q < nbk; ++q) {
            const double rq = __shfl_sync(0xffffffffu, r, q);
            if (lane < nbk) acc = fma(transpose ? Lb[q * nbk + lane] : Lb[lane * nbk + q], rq, acc);
        }
        if (lane < nbk) out[i] = xi - acc;
    }
}

// Overlapping additive blocks (Sec. 3.6.2), first half: d_(b,p) =
// sum_q Lambda_b[p][q] r_(rows_b[q]) (Lambda^T with transpose) for every
// block, r = A x - b given; one warp per block, lane p for row p.
__global__ void k_gblock_corr(int nb, const int *__restrict__ bptr, const int *__restrict__ bidx,
                              const double *__restrict__ lam, const int64_t *__restrict__ lamoff,
                              const double *__restrict__ r, double *__restrict__ d, int transpose) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = w0; b < nb; b += nw) {
        const int b0 = bptr[b], nbk = bptr[b + 1] - b0;
        const double *Lb = lam + lamoff[b];
        const double rl = lane < nbk ? r[bidx[b0 + lane]] : 0.0;
        double acc = 0.0;
        for (int q = 0; q < nbk; ++q) {
            const double rq = __shfl_sync(0xffffffffu, rl, q);
            if (lane < nbk) acc = fma(transpose ? Lb[q * nbk + lane] : Lb[lane * nbk + q], rq, acc);
        }
        if (lane < nbk) d[b0 + lane] = acc;
    }
}
// second half: out_i = x_i - (sum over the blocks holding i of d) / theta_i
__global__ void k_gnode_avg(int N, const int *__restrict__ nptr, const int *__restrict__ nblk,
                            const int *__restrict__ nloc, const int *__restrict__ bptr, const double *__restrict__ d,
                            const double *__restrict__ x, double *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double sacc = 0.0;
        for (int u = nptr[i]; u < nptr[i + 1]; ++u) sacc += d[bptr[nblk[u]] + nloc[u]];
        out[i] = x[i] - sacc / (double)(nptr[i + 1] - nptr[i]);
    }
}

// PCG vector updates: x += alpha p, r -= alpha q; and p = z + beta p
__global__ void k_gcg_update(int64_t n, double alpha, const double *__restrict__ p, const double *__restrict__ q,
                             double *__restrict__ x, double *__restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}
__global__ void k_gcg_dir(int64_t n, double beta, const double *__restrict__ z, double *__restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// r = A x - b (sign = 1) or b - A x (sign = -1)
__global__ void k_gresid(int n, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                         const double *__restrict__ v, const double *__restrict__ bv, const double *__restrict__ x,
                         double *__restrict__ r, double sign) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = -bv[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s = fma(v[p], x[ci[p]], s);
        r[i] = sign * s;
    }
}
// y = M v (sub = 0) or y -= M v (sub = 1)
__global__ void k_gspmv(int n, const int64_t *__restrict__ rp, const int *__restrict__ ci,
                        const double *__restrict__ v, const double *__restrict__ xv, double *__restrict__ y,
                        int sub) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s = fma(v[p], xv[ci[p]], s);
        y[i] = sub ? y[i] - s : s;
    }
}
__global__ void k_gdense_mv(int n, const double *__restrict__ M, const double *__restrict__ bv,
                            double *__restrict__ x) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s = fma(M[(int64_t)i * n + j], bv[j], s);
        x[i] = s;
    }
}

static unsigned grows(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// one cascade step on a level: colour < 0 every block, else the blocks of
// that colour (in place when out == x; otherwise x is copied to out first)
static cs_status gstep(const cs_ghier *h, const cs_gcascade *c, int l, int step, int colour, const double *b,
                       const double *x, double *out, bool transpose, cudaStream_t s) {
    const GLevel &L = h->lev[l];
    const double *lam = c->lam[l] + (int64_t)step * c->lamsize[l];
    int n = L.nb;
    const int *sel = nullptr;
    if (colour >= 0) {
        n = L.colstart[colour + 1] - L.colstart[colour];
        sel = L.cblocks + L.colstart[colour];
        if (out != x) CSX_CUDA(cudaMemcpyAsync(out, x, sizeof(double) * L.A.n, cudaMemcpyDeviceToDevice, s));
    }
    if (n == 0) return CS_OK;
    if (L.overlap && c->kind == CS_ADDITIVE) {  // x - diag(theta)^{-1} Theta^T Lambda Theta (A x - b)
        k_gresid<<<grows(L.A.n), 256, 0, s>>>(L.A.n, L.A.rp, L.A.ci, L.A.v, b, x, L.r, 1.0);
        k_gblock_corr<<<gwarp_blocks(L.nb), 256, 0, s>>>(L.nb, L.bptr, L.bidx, lam, c->lamoff[l], L.r, L.dpool,
                                                          transpose ? 1 : 0);
        k_gnode_avg<<<grows(L.A.n), 256, 0, s>>>(L.A.n, L.nptr, L.nblk, L.nloc, L.bptr, L.dpool, x, out);
        count_launch(3);
        CSX_CUDA(cudaGetLastError());
        return CS_OK;
    }
    if (L.nbmax == 1)
        k_gsweep_point<<<grows(n), 256, 0, s>>>(n, sel, L.bptr, L.bidx, L.A.rp, L.A.ci, L.A.v, lam, c->lamoff[l], b,
                                                 x, out, L.ident);
    else
        k_gsweep_block<<<gwarp_blocks(n), 256, 0, s>>>(n, sel, L.bptr, L.bidx, L.A.rp, L.A.ci, L.A.v, lam,
                                                        c->lamoff[l], b, x, out, transpose ? 1 : 0);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

// one application of the cascade on level l, x in place (L.t as the
// additive ping-pong buffer)
static cs_status gsmooth(const cs_ghier *h, const cs_gcascade *c, int l, bool reverse, const double *b, double *x,
                         cudaStream_t s) {
    const GLevel &L = h->lev[l];
    const int ncol = c->kind == CS_MULTIPLICATIVE ? L.ncol : 1;
    double *cur = x, *oth = L.t;
    for (int st = 0; st < c->nu; ++st) {
        const int lv = reverse ? c->nu - 1 - st : st;
        for (int kk = 0; kk < ncol; ++kk) {
            if (c->kind == CS_MULTIPLICATIVE) {
                const int k = reverse ? ncol - 1 - kk : kk;
                CSX_TRY(gstep(h, c, l, lv, k, b, cur, cur, reverse, s));  // a graph colouring: in place
            } else {
                CSX_TRY(gstep(h, c, l, lv, -1, b, cur, oth, reverse, s));
                std::swap(cur, oth);
            }
        }
    }
    if (cur != x) CSX_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * L.A.n, cudaMemcpyDeviceToDevice, s));
    return CS_OK;
}

// Algorithm 1 from level l: x <- V(x, b)
static cs_status gvcycle_rec(const cs_ghier *h, const cs_gcascade *c, int l, const cs_vcycle_opts &o,
                             const double *b, double *x, cudaStream_t s) {
    if (l == h->nlev - 1) {
        k_gdense_mv<<<std::max(1, (h->cn + 127) / 128), 128, 0, s>>>(h->cn, h->cinv, b, x);
        count_launch();
        CSX_CUDA(cudaGetLastError());
        return CS_OK;
    }
    const GLevel &L = h->lev[l], &C = h->lev[l + 1];
    for (int m = 0; m < o.mu_pre; ++m) CSX_TRY(gsmooth(h, c, l, o.order == CS_RF, b, x, s));
    k_gresid<<<grows(L.A.n), 256, 0, s>>>(L.A.n, L.A.rp, L.A.ci, L.A.v, b, x, L.r, 1.0);
    k_gspmv<<<grows(C.A.n), 256, 0, s>>>(C.A.n, L.R.rp, L.R.ci, L.R.v, L.r, C.b, 0);
    count_launch(2);
    CSX_CUDA(cudaMemsetAsync(C.x, 0, sizeof(double) * C.A.n, s));
    CSX_TRY(gvcycle_rec(h, c, l + 1, o, C.b, C.x, s));
    k_gspmv<<<grows(L.A.n), 256, 0, s>>>(L.A.n, L.P.rp, L.P.ci, L.P.v, C.x, x, 1);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    for (int m = 0; m < o.mu_post; ++m) CSX_TRY(gsmooth(h, c, l, false, b, x, s));
    return CS_OK;
}

static cs_status gcheck(const cs_ghier *h, const cs_gcascade *c, int level) {
    if (!h || !c || c->h != h) { set_error("null or mismatched handles"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("level %d has no smoother", level); return CS_ERR_ARG; }
    return CS_OK;
}

static cs_status gdot(const cs_ghier *h, int64_t n, const double *a, const double *b, double *out, cudaStream_t s) {
    CSX_TRY(launch_dot(n, a, b, h->red, NRED, s));
    CSX_CUDA(cudaMemcpyAsync(h->red_host, h->red + NRED, sizeof(double), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    *out = h->red_host[0];
    return CS_OK;
}

static cs_status gnorm(const cs_ghier *h, int64_t n, const double *a, double *out, cudaStream_t s) {
    CSX_TRY(launch_dot(n, a, a, h->red, NRED, s));
    CSX_CUDA(cudaMemcpyAsync(h->red_host, h->red + NRED, sizeof(double), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(h->red_host[0]);
    return CS_OK;
}

}  // namespace csx

extern "C" {

cs_status cs_gsweep(const cs_ghier *h, cs_gcascade *c, int level, int step, int colour, const double *b,
                    const double *x, double *out, cs_stream stream) {
    CSX_TRY(gcheck(h, c, level));
    if (!b || !x || !out) { set_error("null argument"); return CS_ERR_ARG; }
    if (step < 0 || step >= c->nu) { set_error("step out of range"); return CS_ERR_ARG; }
    const GLevel &L = h->lev[level];
    if (c->kind == CS_MULTIPLICATIVE ? (colour < 0 || colour >= L.ncol) : colour != -1) {
        set_error("colour does not match the cascade kind (level %d has %d colours)", level, L.ncol);
        return CS_ERR_ARG;
    }
    if (out == x && colour < 0) { set_error("out may alias x only for a colour step"); return CS_ERR_ARG; }
    return gstep(h, c, level, step, colour, b, x, out, false, (cudaStream_t)stream);
}

cs_status cs_gsmooth(const cs_ghier *h, cs_gcascade *c, int level, int reverse, const double *b, double *x,
                     cs_stream stream) {
    CSX_TRY(gcheck(h, c, level));
    if (!b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    return gsmooth(h, c, level, reverse != 0, b, x, (cudaStream_t)stream);
}

cs_status cs_gvcycle(const cs_ghier *h, cs_gcascade *c, const cs_vcycle_opts *o, const double *b, double *x,
                     cs_stream stream) {
    CSX_TRY(gcheck(h, c, 0));
    if (!o || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (o->precision != CS_FP64) { set_error("the general path cycles in FP64"); return CS_ERR_ARG; }
    if (o->mu_pre < 0 || o->mu_post < 0 || o->mu_pre + o->mu_post < 1) { set_error("bad smoothing counts"); return CS_ERR_ARG; }
    return gvcycle_rec(h, c, 0, *o, b, x, (cudaStream_t)stream);
}

// Stationary x <- V(x, b); right-preconditioned restarted GMRES in its
// flexible form (Z_j = V0 v_j kept, x += Z y; modified Gram-Schmidt,
// Givens rotations; the Hessenberg problem on the host); or preconditioned
// conjugate gradients with M = V(0, .) (SM "On preconditioned conjugate
// gradient"), stopping on the recurrence residual and reporting the true
// one.
cs_status cs_gsolve(const cs_ghier *h, cs_gcascade *c, const cs_solve_opts *o_in, const double *b, double *x,
                    cs_solve_info *info, cs_stream stream) {
    CSX_TRY(gcheck(h, c, 0));
    if (!o_in || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    cs_solve_opts o = *o_in;
    if (o.maxit <= 0) o.maxit = 100;
    if (o.tol <= 0) o.tol = 1e-10;
    if (o.restart <= 0) o.restart = 30;
    if (o.method != CS_STATIONARY && o.method != CS_GMRES_RIGHT && o.method != CS_PCG) {
        set_error("the general path solves with CS_STATIONARY, CS_GMRES_RIGHT or CS_PCG");
        return CS_ERR_ARG;
    }
    if (o.cycle.precision != CS_FP64 || o.host_buffers) { set_error("the general path takes FP64 device vectors"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const GLevel &L = h->lev[0];
    const int64_t N = L.A.n;
    cs_solve_info inf{0, 0, 0.0, 0};
    double nb = 0.0, rel = 1.0;
    cs_status rc = CS_OK;
    CSX_TRY(gnorm(h, N, b, &nb, s));
    if (nb == 0.0) {
        CSX_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
        CSX_CUDA(cudaStreamSynchronize(s));
        inf.converged = 1;
        if (info) *info = inf;
        return CS_OK;
    }
    auto residual = [&](double *r) -> cs_status {  // r = b - A x, returns ||r|| / ||b|| in rel
        k_gresid<<<grows(N), 256, 0, s>>>((int)N, L.A.rp, L.A.ci, L.A.v, b, x, r, -1.0);
        count_launch();
        CSX_CUDA(cudaGetLastError());
        double nr = 0.0;
        CSX_TRY(gnorm(h, N, r, &nr, s));
        rel = nr / nb;
        return CS_OK;
    };
    if (o.method == CS_PCG) {
        if (!c->cg) CSX_TRY(dalloc_t(&c->cg, (size_t)4 * N, &c->bytes, s));
        double *r = c->cg, *z = r + N, *p = z + N, *q = p + N;
        const unsigned g = grows(N);
        double rz = 0.0, pq = 0.0;
        CSX_TRY(residual(r));
        const double rel0 = rel;
        if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
        CSX_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * N, s));
        CSX_TRY(gvcycle_rec(h, c, 0, o.cycle, r, z, s));
        CSX_TRY(gdot(h, N, r, z, &rz, s));
        CSX_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        while (rel > o.tol && inf.iterations < o.maxit) {
            k_gspmv<<<g, 256, 0, s>>>((int)N, L.A.rp, L.A.ci, L.A.v, p, q, 0);
            count_launch();
            CSX_TRY(gdot(h, N, p, q, &pq, s));
            k_gcg_update<<<g, 256, 0, s>>>(N, rz / pq, p, q, x, r);
            count_launch();
            CSX_CUDA(cudaGetLastError());
            ++inf.iterations;
            double nr = 0.0;
            CSX_TRY(gnorm(h, N, r, &nr, s));
            rel = nr / nb;
            if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
            if (!std::isfinite(rel) || rel > 1e3 * std::max(rel0, 1.0)) {
                set_error("PCG diverged (relative residual %g)", rel);
                rc = CS_ERR_DIVERGED;
                break;
            }
            if (!(rel > o.tol)) break;
            CSX_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * N, s));
            CSX_TRY(gvcycle_rec(h, c, 0, o.cycle, r, z, s));
            double rz1 = 0.0;
            CSX_TRY(gdot(h, N, r, z, &rz1, s));
            k_gcg_dir<<<g, 256, 0, s>>>(N, rz1 / rz, z, p);
            count_launch();
            rz = rz1;
        }
        if (rc == CS_OK) CSX_TRY(residual(L.r));  // the true residual decides
    } else if (o.method == CS_STATIONARY) {
        CSX_TRY(residual(L.r));
        const double rel0 = rel;
        if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
        while (rel > o.tol && inf.iterations < o.maxit) {
            CSX_TRY(gvcycle_rec(h, c, 0, o.cycle, b, x, s));
            ++inf.iterations;
            CSX_TRY(residual(L.r));
            if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
            if (!std::isfinite(rel) || rel > 1e3 * std::max(rel0, 1.0)) {
                set_error("iteration diverged (relative residual %g)", rel);
                rc = CS_ERR_DIVERGED;
                break;
            }
        }
    } else {
        const int m = o.restart;
        if (c->gm_restart < m) {
            dfree(c->gm_V, s); dfree(c->gm_Z, s); dfree(c->gm_h, s);
            c->gm_V = c->gm_Z = c->gm_h = nullptr;
            CSX_TRY(dalloc_t(&c->gm_V, (size_t)(m + 2) * N, &c->bytes, s));
            CSX_TRY(dalloc_t(&c->gm_Z, (size_t)m * N, &c->bytes, s));
            CSX_TRY(dalloc_t(&c->gm_h, (size_t)(m + 2) * 2, &c->bytes, s));
            c->gm_restart = m;
        }
        double *V = c->gm_V, *Z = c->gm_Z, *hd = c->gm_h, *r = c->gm_V + (int64_t)(m + 1) * N;
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hh(m + 2);
        auto dot_to = [&](const double *a, const double *bb, double *dst) -> cs_status {
            CSX_TRY(launch_dot(N, a, bb, h->red, NRED, s));
            CSX_CUDA(cudaMemcpyAsync(dst, h->red + NRED, sizeof(double), cudaMemcpyDeviceToDevice, s));
            return CS_OK;
        };
        for (;;) {
            CSX_TRY(residual(r));
            if (!std::isfinite(rel)) { set_error("GMRES diverged"); rc = CS_ERR_DIVERGED; break; }
            if (inf.nhist == 0 && o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
            if (rel <= o.tol || inf.iterations >= o.maxit) break;
            CSX_TRY(dot_to(r, r, hd));
            CSX_TRY(launch_scale_dev(N, hd, V, r, s));
            CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double), cudaMemcpyDeviceToHost, s));
            CSX_CUDA(cudaStreamSynchronize(s));
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = std::sqrt(hh[0]);
            int j;
            for (j = 0; j < m && inf.iterations < o.maxit; ++j) {
                double *zj = Z + (int64_t)j * N, *w = V + (int64_t)(j + 1) * N;
                CSX_CUDA(cudaMemsetAsync(zj, 0, sizeof(double) * N, s));
                CSX_TRY(gvcycle_rec(h, c, 0, o.cycle, V + (int64_t)j * N, zj, s));
                ++inf.iterations;
                k_gspmv<<<grows(N), 256, 0, s>>>((int)N, L.A.rp, L.A.ci, L.A.v, zj, w, 0);
                count_launch();
                for (int i = 0; i <= j; ++i) {
                    CSX_TRY(dot_to(w, V + (int64_t)i * N, hd + i));
                    CSX_TRY(launch_axpy_dev(N, hd + i, -1.0, V + (int64_t)i * N, w, s));
                }
                CSX_TRY(dot_to(w, w, hd + j + 1));
                CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
                CSX_CUDA(cudaStreamSynchronize(s));
                const double hn = std::sqrt(hh[j + 1]);
                if (hn > 0.0) CSX_TRY(launch_scale_dev(N, hd + j + 1, w, w, s));
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i];
                H[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
                }
                const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
                const double d = std::sqrt(a * a + bb * bb);
                cs[j] = d > 0 ? a / d : 1.0;
                sn[j] = d > 0 ? bb / d : 0.0;
                H[(size_t)j * m + j] = d;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = std::fabs(g[j + 1]) / nb;
                if (std::fabs(g[j + 1]) <= o.tol * nb || hn == 0.0) { ++j; break; }
            }
            for (int i = j - 1; i >= 0; --i) {
                double sum = g[i];
                for (int k = i + 1; k < j; ++k) sum -= H[(size_t)i * m + k] * y[k];
                y[i] = sum / H[(size_t)i * m + i];
            }
            CSX_CUDA(cudaMemcpyAsync(hd, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
            CSX_TRY(launch_axpy_multi(N, j, hd, Z, x, s));
            CSX_CUDA(cudaStreamSynchronize(s));
        }
    }
    inf.final_rel_residual = rel;
    inf.converged = rel <= o.tol;
    if (rc == CS_OK && !inf.converged) {
        set_error("not converged after %d iterations (relative residual %g)", inf.iterations, rel);
        rc = CS_ERR_NOTCONV;
    }
    if (info) *info = inf;
    return rc;
}

}  // extern "C"
