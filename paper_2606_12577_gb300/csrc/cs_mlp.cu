// Learned cascade setup: a 3-layer MLP that maps a block's local operator
// neighbourhood to its prescaled Lambda~_1..nu blocks, with hand-written
// forward, backward and Adam kernels, plus the feature / target extraction
// from a hierarchy and an exact cascade.
//
// Network: in -> hid (ReLU) -> hid (ReLU) -> out, Y = H2 W3^T + b3.
// Weights are kept as FP32 masters and rounded to BF16 for every product
// (BF16 weights, FP32 accumulation); biases, activations and gradients FP32.
// Every product runs on the tensor cores (cs_tcgemm.cu): BF16 weights enter
// as they are, FP32 activations and gradients as BF16 hi + lo pairs along K.
// Layout: activations row-major [batch][width]; W_l row-major [out][in].
//
// Features of a block of bs x bs nodes (2D): for each block node p its row
// of the prescaled operator W A W restricted to the (bs+2)^2-node window
// around the block, at window position (lx + dx + 1) + (bs+2)(ly + dy + 1);
// targets: the prescaled blocks Lambda~_l = W^-1 Lambda_l W^-1 of the exact
// cascade, l = 1..nu, each bs^2 x bs^2 row-major (absent nodes zero).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "cs_internal.cuh"
#include "cs_tcgemm.cuh"

struct cs_mlp {
    int nin = 0, nhid = 0, nout = 0, max_batch = 0;
    int64_t nparam = 0;
    float *p = nullptr;          // FP32 master parameters: W1 b1 W2 b2 W3 b3
    float *g = nullptr;          // gradients (same layout as p)
    float *m = nullptr, *v = nullptr;  // Adam moments
    float *z1 = nullptr, *z2 = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr;  // activations
    float *d1 = nullptr, *d2 = nullptr, *dy = nullptr;  // backward buffers
    float *loss = nullptr;       // device scalar
    float *loss_host = nullptr;  // pinned
    int64_t step = 0;
    int64_t bytes = 0;
    // offsets into p / g
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;
    // tensor-core operands (K contiguous, K padded to 64 per segment): the
    // forward pass, the input gradients, and the weight gradients (K = batch)
    int kin = 0, khid = 0, kout = 0, kb = 0;
    csx::TcOperand tX, tW1, tH1, tW2, tH2, tW3, tDY, tW3T, tD2, tW2T;
    csx::TcOperand tDYT, tH2T, tD2T, tH1T, tD1T, tXT;
    float *part = nullptr;  // split-K partials
    int64_t part_cap = 0;
    int *err = nullptr;     // bounded-wait expiry flag of the GEMM kernel
};

namespace csx {

static int64_t round64(int64_t n) { return (n + 63) / 64 * 64; }

// h = relu(z) already fused; backward: d <- d * (z > 0)
__global__ void k_relu_grad(int64_t n, const float *__restrict__ z, float *__restrict__ d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(z[i] > 0.f)) d[i] = 0.f;
}

// column sums of d [rows x cols] into db (deterministic: one CTA per column)
__global__ void k_colsum(int rows, int cols, const float *__restrict__ d, float *__restrict__ db) {
    __shared__ float sm[256];
    const int c = blockIdx.x;
    float v = 0.f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) v += d[(int64_t)r * cols + c];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = sm[0];
}

// MSE loss over n values and dY = 2 (Y - T) / n; per-CTA partial sums of
// squared errors then one CTA sums them in order.
__global__ void k_mse(int64_t n, const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                      float *__restrict__ part) {
    __shared__ float sm[256];
    float v = 0.f;
    const float sc = 2.f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        v = fmaf(e, e, v);
        dy[i] = sc * e;
    }
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_mse_finish(int nparts, int64_t n, const float *__restrict__ part, float *__restrict__ loss) {
    __shared__ float sm[256];
    float v = 0.f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = sm[0] / (float)n;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// the BF16 weights (round to nearest even of the FP32 masters) as the
// tensor-core operands W_l (forward) and W_l^T (input gradients), each
// entering two K segments so that it meets both halves of the activations'
// hi + lo pairs
static cs_status refresh_bf16(cs_mlp *M, cudaStream_t s) {
    CSX_TRY(tc_pack(M->tW1, M->nhid, M->nin, M->kin, "hh", M->p + M->oW1, M->nin, false, s));
    CSX_TRY(tc_pack(M->tW2, M->nhid, M->nhid, M->khid, "hh", M->p + M->oW2, M->nhid, false, s));
    CSX_TRY(tc_pack(M->tW3, M->nout, M->nhid, M->khid, "hh", M->p + M->oW3, M->nhid, false, s));
    CSX_TRY(tc_pack(M->tW3T, M->nhid, M->nout, M->kout, "hh", M->p + M->oW3, M->nhid, true, s));
    CSX_TRY(tc_pack(M->tW2T, M->nhid, M->nhid, M->khid, "hh", M->p + M->oW2, M->nhid, true, s));
    return CS_OK;
}

static cs_status mlp_gemm(cs_mlp *M, const TcOperand &A, const TcOperand &B, int m, int n, int64_t k, float *C,
                          int ldc, const float *bias, bool relu, float *Z, cudaStream_t s) {
    return tc_gemm(A, B, m, n, k, C, ldc, bias, relu, Z, M->part, M->part_cap, M->err, s);
}

// the GEMM kernel's bounded waits: CS_ERR_TIMEOUT once one expired
static cs_status mlp_check(cs_mlp *M, cudaStream_t s) {
    int h = 0;
    CSX_CUDA(cudaMemcpyAsync(&h, M->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    if (h) {
        set_error("a tensor-core GEMM wait expired");
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}

static cs_status forward(cs_mlp *M, int B, const float *X, cudaStream_t s) {
    CSX_TRY(tc_pack(M->tX, B, M->nin, M->kin, "hl", X, M->nin, false, s));
    CSX_TRY(mlp_gemm(M, M->tX, M->tW1, B, M->nhid, 2 * M->kin, M->h1, M->nhid, M->p + M->ob1, true, M->z1, s));
    CSX_TRY(tc_pack(M->tH1, B, M->nhid, M->khid, "hl", M->h1, M->nhid, false, s));
    CSX_TRY(mlp_gemm(M, M->tH1, M->tW2, B, M->nhid, 2 * M->khid, M->h2, M->nhid, M->p + M->ob2, true, M->z2, s));
    CSX_TRY(tc_pack(M->tH2, B, M->nhid, M->khid, "hl", M->h2, M->nhid, false, s));
    CSX_TRY(mlp_gemm(M, M->tH2, M->tW3, B, M->nout, 2 * M->khid, M->y, M->nout, M->p + M->ob3, false, nullptr, s));
    return CS_OK;
}

// gradients of the mean squared error of the current forward pass w.r.t.
// every parameter, into M->g; the loss into M->loss (device)
static cs_status backward(cs_mlp *M, int B, const float *X, const float *T, cudaStream_t s) {
    const int64_t ny = (int64_t)B * M->nout;
    const int nparts = 256;
    float *part = M->d2;  // scratch: nparts floats (d2 is rewritten below)
    k_mse<<<nparts, 256, 0, s>>>(ny, M->y, T, M->dy, part);
    k_mse_finish<<<1, 256, 0, s>>>(nparts, ny, part, M->loss);
    count_launch(2);
    // weight gradients contract over the batch: both factors FP32, as
    // three K segments (a_hi b_hi + a_lo b_hi + a_hi b_lo)
    const int kseg = (int)round64(B);
    // layer 3: dW3 = dY^T H2, db3 = colsum(dY), dH2 = dY W3
    CSX_TRY(tc_pack(M->tDYT, M->nout, B, kseg, "hlh", M->dy, M->nout, true, s));
    CSX_TRY(tc_pack(M->tH2T, M->nhid, B, kseg, "hhl", M->h2, M->nhid, true, s));
    CSX_TRY(mlp_gemm(M, M->tDYT, M->tH2T, M->nout, M->nhid, 3 * kseg, M->g + M->oW3, M->nhid, nullptr, false, nullptr,
                     s));
    k_colsum<<<M->nout, 256, 0, s>>>(B, M->nout, M->dy, M->g + M->ob3);
    count_launch();
    CSX_TRY(tc_pack(M->tDY, B, M->nout, M->kout, "hl", M->dy, M->nout, false, s));
    CSX_TRY(mlp_gemm(M, M->tDY, M->tW3T, B, M->nhid, 2 * M->kout, M->d2, M->nhid, nullptr, false, nullptr, s));
    k_relu_grad<<<1024, 256, 0, s>>>((int64_t)B * M->nhid, M->z2, M->d2);
    count_launch();
    // layer 2
    CSX_TRY(tc_pack(M->tD2T, M->nhid, B, kseg, "hlh", M->d2, M->nhid, true, s));
    CSX_TRY(tc_pack(M->tH1T, M->nhid, B, kseg, "hhl", M->h1, M->nhid, true, s));
    CSX_TRY(mlp_gemm(M, M->tD2T, M->tH1T, M->nhid, M->nhid, 3 * kseg, M->g + M->oW2, M->nhid, nullptr, false,
                     nullptr, s));
    k_colsum<<<M->nhid, 256, 0, s>>>(B, M->nhid, M->d2, M->g + M->ob2);
    count_launch();
    CSX_TRY(tc_pack(M->tD2, B, M->nhid, M->khid, "hl", M->d2, M->nhid, false, s));
    CSX_TRY(mlp_gemm(M, M->tD2, M->tW2T, B, M->nhid, 2 * M->khid, M->d1, M->nhid, nullptr, false, nullptr, s));
    k_relu_grad<<<1024, 256, 0, s>>>((int64_t)B * M->nhid, M->z1, M->d1);
    count_launch();
    // layer 1
    CSX_TRY(tc_pack(M->tD1T, M->nhid, B, kseg, "hlh", M->d1, M->nhid, true, s));
    CSX_TRY(tc_pack(M->tXT, M->nin, B, kseg, "hhl", X, M->nin, true, s));
    CSX_TRY(mlp_gemm(M, M->tD1T, M->tXT, M->nhid, M->nin, 3 * kseg, M->g + M->oW1, M->nin, nullptr, false, nullptr,
                     s));
    k_colsum<<<M->nhid, 256, 0, s>>>(B, M->nhid, M->d1, M->g + M->ob1);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014) for the weight initialisation
static uint64_t splitmix(uint64_t &st) {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------ features and targets
// one thread per block of the finest level
__global__ void k_block_features(Grid g, int bs, int nbx, int64_t nblocks, int kind, const double *__restrict__ A,
                                 float *__restrict__ F) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = (int)(b % nbx), by = (int)(b / nbx);
    const int win = bs + 2, nf = bs * bs * win * win;
    float *f = F + b * nf;
    for (int t = 0; t < nf; ++t) f[t] = 0.f;
    const int C = kind == STAR ? 0 : 4;
    const int nst = kind == STAR ? 5 : 9;
    for (int p = 0; p < bs * bs; ++p) {
        const int lx = p % bs, ly = p / bs;
        const int ix = bs * bx + lx, iy = bs * by + ly;
        if (ix >= g.nx || iy >= g.ny) continue;
        const int64_t i = ix + (int64_t)g.nx * iy;
        const double wi = 1.0 / sqrt(A[(int64_t)C * g.N + i]);
        for (int s = 0; s < nst; ++s) {
            int dx, dy;
            if (kind == STAR) {
                dx = s == 1 ? -1 : (s == 2 ? 1 : 0);
                dy = s == 3 ? -1 : (s == 4 ? 1 : 0);
            } else {
                dx = s % 3 - 1;
                dy = s / 3 - 1;
            }
            const int jx = ix + dx, jy = iy + dy;
            if (jx < 0 || jx >= g.nx || jy < 0 || jy >= g.ny) continue;
            const int64_t j = jx + (int64_t)g.nx * jy;
            const double wj = 1.0 / sqrt(A[(int64_t)C * g.N + j]);
            f[p * win * win + (lx + dx + 1) + win * (ly + dy + 1)] = (float)(wi * A[(int64_t)s * g.N + i] * wj);
        }
    }
}

// prescaled Lambda~ = Lambda / (w_p w_q) = Lambda sqrt(A_pp A_qq), per step
__global__ void k_block_targets(Grid g, int bs, int nbx, int64_t nblocks, int nu, int kind,
                                const double *__restrict__ A, const double *__restrict__ lam,
                                float *__restrict__ T) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = (int)(b % nbx), by = (int)(b / nbx);
    const int nm = bs * bs, C = kind == STAR ? 0 : 4;
    float *t = T + b * (int64_t)nu * nm * nm;
    for (int l = 0; l < nu; ++l)
        for (int p = 0; p < nm; ++p)
            for (int q = 0; q < nm; ++q) {
                const int px = bs * bx + p % bs, py = bs * by + p / bs, qx = bs * bx + q % bs, qy = bs * by + q / bs;
                float v = 0.f;
                if (px < g.nx && py < g.ny && qx < g.nx && qy < g.ny) {
                    const double dp = A[(int64_t)C * g.N + px + (int64_t)g.nx * py];
                    const double dq = A[(int64_t)C * g.N + qx + (int64_t)g.nx * qy];
                    v = (float)(lam[((int64_t)l * nblocks + b) * nm * nm + p * nm + q] * sqrt(dp * dq));
                }
                t[((int64_t)l * nm + p) * nm + q] = v;
            }
}

// predicted prescaled blocks -> unscaled Lambda (FP64), absent nodes zero
__global__ void k_block_unscale(Grid g, int bs, int nbx, int64_t nblocks, int nu, int kind,
                                const double *__restrict__ A, const float *__restrict__ Y, double *__restrict__ lam) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = (int)(b % nbx), by = (int)(b / nbx);
    const int nm = bs * bs, C = kind == STAR ? 0 : 4;
    const float *y = Y + b * (int64_t)nu * nm * nm;
    for (int l = 0; l < nu; ++l)
        for (int p = 0; p < nm; ++p)
            for (int q = 0; q < nm; ++q) {
                const int px = bs * bx + p % bs, py = bs * by + p / bs, qx = bs * bx + q % bs, qy = bs * by + q / bs;
                double v = 0.0;
                if (px < g.nx && py < g.ny && qx < g.nx && qy < g.ny) {
                    const double dp = A[(int64_t)C * g.N + px + (int64_t)g.nx * py];
                    const double dq = A[(int64_t)C * g.N + qx + (int64_t)g.nx * qy];
                    v = (double)y[((int64_t)l * nm + p) * nm + q] / sqrt(dp * dq);
                }
                lam[((int64_t)l * nblocks + b) * nm * nm + p * nm + q] = v;
            }
}

// Frobenius objective of a level-1 block smoother on the prescaled operator:
// obj_b = || E_0 rows - Lam~_b (A~ E_0) rows ||_F^2 = || I_b - Lam~_b A~_{b,:} ||_F^2
// (E_0 = I); part[b] receives it for Lam~ from `lam` (unscaled, step 0).
__global__ void k_level1_objective(Grid g, int bs, int nbx, int64_t nblocks, int kind, const double *__restrict__ A,
                                   const double *__restrict__ lam, double *__restrict__ obj) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = (int)(b % nbx), by = (int)(b / nbx);
    const int nm = bs * bs, C = kind == STAR ? 0 : 4, nst = kind == STAR ? 5 : 9;
    const int win = bs + 2;
    double total = 0.0;
    // columns of the block row: the (bs+2)^2 window; entry (p, col) of A~_{b,:}
    for (int p = 0; p < nm; ++p) {
        const int px = bs * bx + p % bs, py = bs * by + p / bs;
        if (px >= g.nx || py >= g.ny) continue;
        for (int cw = 0; cw < win * win; ++cw) {
            const int cx = bs * bx - 1 + cw % win, cy = bs * by - 1 + cw / win;
            if (cx < 0 || cx >= g.nx || cy < 0 || cy >= g.ny) continue;
            const double dc = A[(int64_t)C * g.N + cx + (int64_t)g.nx * cy];
            double v = (cx == px && cy == py) ? 1.0 : 0.0;
            for (int q = 0; q < nm; ++q) {
                const int qx = bs * bx + q % bs, qy = bs * by + q / bs;
                if (qx >= g.nx || qy >= g.ny) continue;
                const int dx = cx - qx, dy = cy - qy;
                if (dx < -1 || dx > 1 || dy < -1 || dy > 1) continue;
                int s = -1;
                if (kind == STAR) {
                    if (dx == 0 && dy == 0) s = 0;
                    else if (dy == 0) s = dx < 0 ? 1 : 2;
                    else if (dx == 0) s = dy < 0 ? 3 : 4;
                } else {
                    s = (dx + 1) + 3 * (dy + 1);
                }
                if (s < 0 || s >= nst) continue;
                const double dq = A[(int64_t)C * g.N + qx + (int64_t)g.nx * qy];
                const double dp = A[(int64_t)C * g.N + px + (int64_t)g.nx * py];
                // prescaled Lam~_pq = Lam_pq sqrt(dp dq); A~_qc = A_qc / sqrt(dq dc)
                const double lt = lam[b * nm * nm + p * nm + q] * sqrt(dp * dq);
                v -= lt * A[(int64_t)s * g.N + qx + (int64_t)g.nx * qy] / sqrt(dq * dc);
            }
            total += v * v;
        }
    }
    obj[b] = total;
}

}  // namespace csx

using namespace csx;

extern "C" {

cs_status cs_mlp_create(int nin, int nhid, int nout, int max_batch, uint64_t seed, cs_mlp **out) {
    if (!out || nin < 1 || nhid < 1 || nout < 1 || max_batch < 1) { set_error("bad MLP shape"); return CS_ERR_ARG; }
    *out = nullptr;
    cs_mlp *M = new cs_mlp();
    M->nin = nin; M->nhid = nhid; M->nout = nout; M->max_batch = max_batch;
    M->oW1 = 0; M->ob1 = M->oW1 + (int64_t)nhid * nin;
    M->oW2 = M->ob1 + nhid; M->ob2 = M->oW2 + (int64_t)nhid * nhid;
    M->oW3 = M->ob2 + nhid; M->ob3 = M->oW3 + (int64_t)nout * nhid;
    M->nparam = M->ob3 + nout;
    cudaStream_t s = 0;
    cs_status rc = CS_OK;
    const int64_t B = max_batch;
    // He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases
    std::vector<float> h((size_t)M->nparam, 0.f);
    uint64_t st = seed;
    auto fill = [&](int64_t off, int64_t n, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int64_t i = 0; i < n; ++i) h[off + i] = (float)(-a + 2.0 * a * ((splitmix(st) >> 11) * 0x1.0p-53));
    };
    fill(M->oW1, (int64_t)nhid * nin, nin);
    fill(M->oW2, (int64_t)nhid * nhid, nhid);
    fill(M->oW3, (int64_t)nout * nhid, nhid);
    if ((rc = dalloc_t(&M->p, M->nparam, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->g, M->nparam, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->m, M->nparam, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->v, M->nparam, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->z1, B * nhid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->z2, B * nhid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->h1, B * nhid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->h2, B * nhid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->d1, B * nhid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->d2, std::max<int64_t>(B * nhid, 256), &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->y, B * nout, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->dy, B * nout, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->loss, 4, &M->bytes)) != CS_OK) goto fail;
    if (cudaMallocHost(&M->loss_host, sizeof(float) * 4) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "cudaMallocHost", __FILE__, __LINE__); goto fail; }
    M->kin = (int)round64(nin);
    M->khid = (int)round64(nhid);
    M->kout = (int)round64(nout);
    M->kb = (int)round64(B);
    if ((rc = tc_operand_init(M->tX, B, 2 * M->kin, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tW1, nhid, 2 * M->kin, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tH1, B, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tW2, nhid, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tH2, B, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tW3, nout, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tDY, B, 2 * M->kout, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tW3T, nhid, 2 * M->kout, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tD2, B, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tW2T, nhid, 2 * M->khid, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tDYT, nout, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tH2T, nhid, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tD2T, nhid, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tH1T, nhid, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tD1T, nhid, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    if ((rc = tc_operand_init(M->tXT, nin, 3 * M->kb, &M->bytes)) != CS_OK) goto fail;
    M->part_cap = (int64_t)4 << 20;
    if ((rc = dalloc_t(&M->part, (size_t)M->part_cap, &M->bytes)) != CS_OK) goto fail;
    if ((rc = dalloc_t(&M->err, 1, &M->bytes)) != CS_OK) goto fail;
    if (cudaMemset(M->err, 0, sizeof(int)) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "MLP init", __FILE__, __LINE__); goto fail; }
    if (cudaMemcpy(M->p, h.data(), sizeof(float) * M->nparam, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(M->m, 0, sizeof(float) * M->nparam) != cudaSuccess ||
        cudaMemset(M->v, 0, sizeof(float) * M->nparam) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "MLP init", __FILE__, __LINE__);
        goto fail;
    }
    if ((rc = refresh_bf16(M, s)) != CS_OK) goto fail;
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "MLP init", __FILE__, __LINE__); goto fail; }
    *out = M;
    return CS_OK;
fail:
    cs_mlp_destroy(M);
    return rc;
}

void cs_mlp_destroy(cs_mlp *M) {
    if (!M) return;
    dfree(M->p); dfree(M->g); dfree(M->m); dfree(M->v);
    dfree(M->z1); dfree(M->z2); dfree(M->h1); dfree(M->h2); dfree(M->d1); dfree(M->d2); dfree(M->y); dfree(M->dy);
    dfree(M->loss);
    for (csx::TcOperand *o : {&M->tX, &M->tW1, &M->tH1, &M->tW2, &M->tH2, &M->tW3, &M->tDY, &M->tW3T, &M->tD2,
                              &M->tW2T, &M->tDYT, &M->tH2T, &M->tD2T, &M->tH1T, &M->tD1T, &M->tXT})
        dfree(o->p);
    dfree(M->part); dfree(M->err);
    if (M->loss_host) cudaFreeHost(M->loss_host);
    delete M;
}

int64_t cs_mlp_nparam(const cs_mlp *M) { return M ? M->nparam : 0; }

cs_status cs_mlp_get_params(const cs_mlp *M, float *host) {
    if (!M || !host) { set_error("null argument"); return CS_ERR_ARG; }
    CSX_CUDA(cudaDeviceSynchronize());
    CSX_CUDA(cudaMemcpy(host, M->p, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_mlp_set_params(cs_mlp *M, const float *host) {
    if (!M || !host) { set_error("null argument"); return CS_ERR_ARG; }
    CSX_CUDA(cudaMemcpy(M->p, host, sizeof(float) * M->nparam, cudaMemcpyHostToDevice));
    CSX_TRY(refresh_bf16(M, 0));
    CSX_CUDA(cudaDeviceSynchronize());
    return CS_OK;
}

cs_status cs_mlp_forward(cs_mlp *M, int batch, const float *X, float *Y, cs_stream stream) {
    if (!M || !X || !Y) { set_error("null argument"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    for (int b0 = 0; b0 < batch; b0 += M->max_batch) {
        const int B = std::min(M->max_batch, batch - b0);
        CSX_TRY(forward(M, B, X + (int64_t)b0 * M->nin, s));
        CSX_CUDA(cudaMemcpyAsync(Y + (int64_t)b0 * M->nout, M->y, sizeof(float) * B * M->nout,
                                 cudaMemcpyDeviceToDevice, s));
    }
    return mlp_check(M, s);
}

cs_status cs_mlp_gradients(cs_mlp *M, int batch, const float *X, const float *T, float *grad_host, float *loss,
                           cs_stream stream) {
    if (!M || !X || !T) { set_error("null argument"); return CS_ERR_ARG; }
    if (batch < 1 || batch > M->max_batch) { set_error("batch must be in 1..max_batch"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    CSX_TRY(forward(M, batch, X, s));
    CSX_TRY(backward(M, batch, X, T, s));
    CSX_CUDA(cudaMemcpyAsync(M->loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CSX_TRY(mlp_check(M, s));
    if (loss) *loss = M->loss_host[0];
    if (grad_host) CSX_CUDA(cudaMemcpy(grad_host, M->g, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_mlp_train_step(cs_mlp *M, int batch, const float *X, const float *T, float lr, float *loss,
                            cs_stream stream) {
    if (!M || !X || !T) { set_error("null argument"); return CS_ERR_ARG; }
    if (batch < 1 || batch > M->max_batch) { set_error("batch must be in 1..max_batch"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    CSX_TRY(forward(M, batch, X, s));
    CSX_TRY(backward(M, batch, X, T, s));
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    k_adam<<<512, 256, 0, s>>>(M->nparam, M->p, M->g, M->m, M->v, lr, b1, b2, eps, c1, c2);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    CSX_TRY(refresh_bf16(M, s));
    if (loss) {
        CSX_CUDA(cudaMemcpyAsync(M->loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        CSX_TRY(mlp_check(M, s));
        *loss = M->loss_host[0];
    }
    return CS_OK;
}

cs_status cs_block_features(const cs_hierarchy *h, int level, float *F, cs_stream stream) {
    if (!h || !F) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev || h->lev[level].g.dim != 2 || h->lev[level].bs < 2) {
        set_error("block features need a 2D level with blocks");
        return CS_ERR_UNSUPPORTED;
    }
    const Level &L = h->lev[level];
    k_block_features<<<(unsigned)((L.nblocks + 127) / 128), 128, 0, (cudaStream_t)stream>>>(L.g, L.bs, L.nbx, L.nblocks,
                                                                                          L.kind, L.A, F);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

cs_status cs_block_targets(const cs_cascade *c, int level, float *T, cs_stream stream) {
    if (!c || !T) { set_error("null argument"); return CS_ERR_ARG; }
    const cs_hierarchy *h = c->h;
    if (level < 0 || level >= c->nlev || h->lev[level].g.dim != 2 || h->lev[level].bs < 2 || c->kind != CS_ADDITIVE) {
        set_error("block targets need an additive cascade on a 2D level with blocks");
        return CS_ERR_UNSUPPORTED;
    }
    const Level &L = h->lev[level];
    k_block_targets<<<(unsigned)((L.nblocks + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        L.g, L.bs, L.nbx, L.nblocks, c->nu, L.kind, L.A, c->lam[level], T);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // extern "C"

namespace csx {

// Per block: the prediction stays when the block is full (all bs^2 nodes
// inside the grid) and its level-1 objective is within (1 + tol) of the exact
// one; otherwise every cascade step of the block takes the exact level-1
// block.  flag[b] = 1 for a kept prediction.
__global__ void k_block_accept(Grid g, int bs, int nbx, int64_t nblocks, int nu, double tol,
                               const double *__restrict__ obj, const double *__restrict__ lam_exact1,
                               double *__restrict__ lam, int *__restrict__ flag) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = (int)(b % nbx), by = (int)(b / nbx);
    const int nm2 = bs * bs * bs * bs;
    const bool full = bs * bx + bs <= g.nx && bs * by + bs <= g.ny;
    const double op = obj[b], oe = obj[nblocks + b];
    const bool ok = full && isfinite(op) && op <= (1.0 + tol) * oe;
    flag[b] = ok ? 1 : 0;
    if (ok) return;
    for (int l = 0; l < nu; ++l)
        for (int e = 0; e < nm2; ++e) lam[((int64_t)l * nblocks + b) * nm2 + e] = lam_exact1[b * nm2 + e];
}

// Learned setup of the finest level (see cs_cascade_opts.model): features,
// MLP inference and unscaling for every block, then the per-block check of
// the level-1 Frobenius objective against the exact level-1 blocks (which
// cost one least-squares problem each); rejected and partial blocks take the
// exact level-1 block at every step.  Records the counts and objective
// ratios in c.
cs_status learned_setup_level0(const cs_hierarchy *h, cs_cascade *c, cs_mlp *M, double tol, double *lam,
                               const double *lam_exact1, cudaStream_t s) {
    const Level &L = h->lev[0];
    const int nm = L.bs * L.bs, win = L.bs + 2;
    if (M->nin != nm * win * win || M->nout != c->nu * nm * nm) {
        set_error("model shape (%d -> %d) does not match %dx%d blocks with nu = %d", M->nin, M->nout, L.bs, L.bs, c->nu);
        return CS_ERR_ARG;
    }
    float *F = nullptr, *Y = nullptr;
    double *obj = nullptr;
    int *flag = nullptr;
    cs_status rc = CS_OK;
    std::vector<double> op, oe;
    std::vector<int> fl;
    const unsigned nb = (unsigned)((L.nblocks + 127) / 128);
    if ((rc = dalloc_t(&F, (size_t)L.nblocks * M->nin, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&Y, (size_t)L.nblocks * M->nout, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&obj, (size_t)2 * L.nblocks, nullptr, s)) != CS_OK) goto done;
    if ((rc = dalloc_t(&flag, (size_t)L.nblocks, nullptr, s)) != CS_OK) goto done;
    k_block_features<<<nb, 128, 0, s>>>(L.g, L.bs, L.nbx, L.nblocks, L.kind, L.A, F);
    count_launch();
    if ((rc = cs_mlp_forward(M, (int)L.nblocks, F, Y, s)) != CS_OK) goto done;
    k_block_unscale<<<nb, 128, 0, s>>>(L.g, L.bs, L.nbx, L.nblocks, c->nu, L.kind, L.A, Y, lam);
    k_level1_objective<<<nb, 128, 0, s>>>(L.g, L.bs, L.nbx, L.nblocks, L.kind, L.A, lam, obj);
    k_level1_objective<<<nb, 128, 0, s>>>(L.g, L.bs, L.nbx, L.nblocks, L.kind, L.A, lam_exact1, obj + L.nblocks);
    k_block_accept<<<nb, 128, 0, s>>>(L.g, L.bs, L.nbx, L.nblocks, c->nu, tol, obj, lam_exact1, lam, flag);
    count_launch(4);
    op.resize(L.nblocks);
    oe.resize(L.nblocks);
    fl.resize(L.nblocks);
    if (cudaMemcpyAsync(op.data(), obj, sizeof(double) * L.nblocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(oe.data(), obj + L.nblocks, sizeof(double) * L.nblocks, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(fl.data(), flag, sizeof(int) * L.nblocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "learned setup", __FILE__, __LINE__);
        goto done;
    }
    {
        double sp = 0.0, se = 0.0, su = 0.0;
        int64_t nacc = 0, nfull = 0;
        for (int64_t b = 0; b < L.nblocks; ++b) {
            const int bx = (int)(b % L.nbx), by = (int)(b / L.nbx);
            nfull += L.bs * bx + L.bs <= L.g.nx && L.bs * by + L.bs <= L.g.ny;
            sp += op[b];
            se += oe[b];
            su += fl[b] ? op[b] : oe[b];
            nacc += fl[b];
        }
        c->learned_ratio = se > 0 ? sp / se : 1.0;
        c->learned_ratio_used = se > 0 ? su / se : 1.0;
        c->learned_blocks = L.nblocks;
        c->learned_full = nfull;
        c->learned_accepted = nacc;
    }
done:
    dfree(F, s); dfree(Y, s); dfree(obj, s); dfree(flag, s);
    return rc;
}

}  // namespace csx
