// Dense BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the
// learned-setup network: C[M x N] (FP32) = A[M x K] B[N x K]^T with A and B
// BF16, K contiguous (row-major A and B, "TN"), FP32 accumulation in tensor
// memory.
//
// One CTA computes a 128 x BN tile of C, BN = 128, or 256 when N > 128 (grid
// x: N tiles, y: M tiles, z: K splits).  Operand boxes of 128 rows x 64 BF16
// (128 B per row) are staged by TMA into shared memory with the 128-byte
// swizzle, four stages deep; one thread issues the TMA copies and the
// tcgen05.mma instructions (M = 128, N = BN, K = 16 each) and commits each
// stage back to its "empty" barrier; the accumulator lives in BN TMEM
// columns; the four warps read it back with
// tcgen05.ld (warp w owns TMEM lanes 32w .. 32w + 31, i.e. rows of C) for the
// epilogue (bias, pre-activation copy, ReLU) or for a split-K partial.
//
// Every wait on an mbarrier is bounded: on expiry the kernel raises *err,
// stops issuing, waits (bounded again) for its copies in flight, frees its
// TMEM and returns; the host reports CS_ERR_TIMEOUT.
//
// FP32 operands enter as BF16 pairs (hi = bf16(x), lo = bf16(x - hi)) laid
// side by side along K, so that one GEMM over the concatenated K forms
// a_hi b_hi + a_lo b_hi + a_hi b_lo: the products of FP32 values to about
// 2^-16 relative (the bf16x3 scheme of Henry, Tang and Heinecke 2019), while
// BF16 weights enter once per segment unsplit.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "cs_internal.cuh"
#include "cs_tcgemm.cuh"

namespace csx {

namespace {

constexpr int TC_BM = 128, TC_BK = 64;  // tile rows; BK: BF16 elements per 128-byte row
constexpr int TC_STAGES = 4;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;  // 16 KB: one 128-row operand box
// dynamic shared memory for a tile of BN columns: per stage one A box and
// BN / 128 B boxes, plus alignment and slack
template <int BN>
constexpr int tc_smem() {
    return TC_STAGES * TC_TILE_BYTES * (1 + BN / 128) + 1024 + 8192;
}
constexpr long long TC_SPIN = 1ll << 24;  // try_wait rounds before a wait is declared expired

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor of a K-major tile with the 128-byte
// swizzle: 8-row core groups 1024 B apart (stride byte offset), the leading
// byte offset unused for this layout (1), descriptor version 1 (bits 46-48),
// swizzle mode 2 (128 B) in bits 61-63
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28
template <int BN>
constexpr uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// C (+ bias, ReLU, pre-activation copy Z) = A B^T over the K blocks
// [z kps, min(nkb, (z + 1) kps)) of this CTA's split, or, with partial set,
// the split's raw sum into C + z M N (row stride N).  BN = 128 or 256 columns
// per tile: the B tile is BN / 128 stacked 128-row boxes, one MMA of N = BN
// per 16-wide K step, BN TMEM columns.
template <int BN>
__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap ma,
                                                    const __grid_constant__ CUtensorMap mb, TcArgs a) {
    constexpr int NB = BN / 128;                         // B boxes per stage
    constexpr int BTILE = NB * TC_TILE_BYTES;            // B bytes per stage
    constexpr uint32_t IDESC = tc_idesc<BN>();
    extern __shared__ uint8_t tc_smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    __shared__ float stile[4][32][33];  // per warp: a 32 x 32 chunk of C, padded against bank conflicts
    const uint32_t raw = smem_u32(tc_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // the 128-byte swizzle wants 1024-byte aligned tiles
    const uint32_t sA = base, sB = base + TC_STAGES * TC_TILE_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * TC_BM;
    const int kb0 = blockIdx.z * a.kps;
    const int nk = min(a.nkb, kb0 + a.kps) - kb0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&done), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // warp 0 is the issuing warp: lane 0 runs the copy / product loop and the
    // other lanes park at __syncwarp (a spinning lane of the same warp would
    // share its issue slots and stall the loop); warps 1-3 wait on "done"
    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0, consumed = 0;
        auto load = [&](int k) {
            const int s = k % TC_STAGES;
            const uint32_t fb = smem_u32(&full[s]);
            mbar_expect_tx(fb, TC_TILE_BYTES + BTILE);
            tma_load_2d(sA + s * TC_TILE_BYTES, &ma, (kb0 + k) * TC_BK, m0, fb);
#pragma unroll
            for (int h = 0; h < NB; ++h)  // 128-row boxes stacked: 8-row groups stay 1024 B apart
                tma_load_2d(sB + s * BTILE + h * TC_TILE_BYTES, &mb, (kb0 + k) * TC_BK, n0 + 128 * h, fb);
        };
        for (int k = 0; k < nk && k < TC_STAGES; ++k) {
            load(k);
            ++issued;
        }
        for (int k = 0; k < nk; ++k) {
            const int s = k % TC_STAGES;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(k / TC_STAGES) & 1u)) { ok = false; break; }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j)  // K = 16 per instruction: 32 bytes along the swizzled row
                mma_bf16(tmem, sw128_desc(sA + s * TC_TILE_BYTES + 32 * j), sw128_desc(sB + s * BTILE + 32 * j),
                         IDESC, (k > 0 || j > 0) ? 1u : 0u);
            mma_commit(smem_u32(&empty[s]));
            // refill the stage of the previous K block once its products are done
            if (k >= 1 && k - 1 + TC_STAGES < nk) {
                const int sp = (k - 1) % TC_STAGES;
                if (!mbar_wait(smem_u32(&empty[sp]), (uint32_t)((k - 1) / TC_STAGES) & 1u)) { ok = false; break; }
                load(k - 1 + TC_STAGES);
                ++issued;
            }
        }
        mma_commit(smem_u32(&done));  // arrives once every product issued above has completed
        if (!ok) {
            atomicExch(a.err, 1);
            failed = 1;
            for (int k = consumed; k < issued; ++k)  // copies still in flight land before the CTA exits
                mbar_wait(smem_u32(&full[k % TC_STAGES]), (uint32_t)(k / TC_STAGES) & 1u);
        }
    }
    if (warp == 0) __syncwarp();
    const bool got = mbar_wait(smem_u32(&done), 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int all_ok = __syncthreads_and(got ? 1 : 0);
    if (!all_ok && threadIdx.x == 0) atomicExch(a.err, 1);
    if (all_ok && !failed && nk > 0) {
        // each 32 x 32 chunk goes through shared memory, so that every row of
        // it leaves as one 128-byte segment (lane = column)
        float(*tile)[33] = stile[warp];
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) tile[lane][i] = v[i];
            __syncwarp();
            const int n = n0 + c + lane;
            const float bn = (!a.partial && a.bias && n < a.N) ? a.bias[n] : 0.f;
            for (int r = 0; r < 32; ++r) {
                const int row = m0 + warp * 32 + r;
                if (row >= a.M || n >= a.N) continue;
                float x = tile[r][lane];
                if (a.partial) {
                    a.C[((int64_t)blockIdx.z * a.M + row) * a.N + n] = x;
                } else {
                    if (a.bias) x += bn;
                    if (a.Z) a.Z[(int64_t)row * a.ldc + n] = x;
                    if (a.relu) x = fmaxf(x, 0.f);
                    a.C[(int64_t)row * a.ldc + n] = x;
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// Persistent form for large products (no K split): one CTA per SM walks the
// 128 x BN tiles in a grid-stride loop, in groups of 16 M blocks with the M
// block fastest inside a group (the tiles in flight share their A and B panels
// in L2), with three roles.  Warp 0 lane 0 streams the operand boxes of every
// (tile, K block) through the 4-stage ring; warp 1 lane 0 issues the MMAs
// into one of two TMEM accumulators (2 BN columns) and commits each stage
// to its "empty" barrier and each finished tile to its accumulator's "full"
// barrier; warps 2-5 read a finished accumulator back (warp w owns TMEM
// lanes 32 (w mod 4) ..), apply the epilogue and release the accumulator, so
// the epilogue of one tile overlaps the products of the next.  Every wait is
// bounded: on expiry *err is raised and the role stops, and all roles reach
// the final barrier.
// tile t -> (M block, N block) in groups of TC_GROUP M blocks
constexpr int TC_GROUP = 16;
__device__ __forceinline__ void tc_tile(int t, int tn, int tm, int &mb, int &nb) {
    const int per = TC_GROUP * tn, grp = t / per, first = grp * TC_GROUP;
    const int gsize = min(TC_GROUP, tm - first), r = t - grp * per;
    mb = first + r % gsize;
    nb = r / gsize;
}

template <int BN>
__global__ void __launch_bounds__(192, 1) k_tc_gemm_persistent(const __grid_constant__ CUtensorMap ma,
                                                               const __grid_constant__ CUtensorMap mb, TcArgs a,
                                                               int tn, int ntiles) {
    constexpr int NB = BN / 128;
    constexpr int BTILE = NB * TC_TILE_BYTES;
    constexpr uint32_t IDESC = tc_idesc<BN>();
    extern __shared__ uint8_t tc_smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ float stile[4][32][33];  // per epilogue warp: a 32 x 32 chunk, padded against bank conflicts
    const uint32_t raw = smem_u32(tc_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base, sB = base + TC_STAGES * TC_TILE_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int c = 0; c < 2; ++c) {
            mbar_init(smem_u32(&tfull[c]), 1);
            mbar_init(smem_u32(&tempty[c]), 4);  // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int nkb = a.nkb;
    if (warp == 0) {
        if (lane == 0) {  // producer
            int64_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int mbk, nbk;
                tc_tile(t, tn, ntiles / tn, mbk, nbk);
                const int m0 = mbk * TC_BM, n0 = nbk * BN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % TC_STAGES);
                    if (it >= TC_STAGES &&
                        !mbar_wait(smem_u32(&empty[s]), (uint32_t)((it / TC_STAGES - 1) & 1))) { ok = false; break; }
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, TC_TILE_BYTES + BTILE);
                    tma_load_2d(sA + s * TC_TILE_BYTES, &ma, kb * TC_BK, m0, fb);
#pragma unroll
                    for (int h = 0; h < NB; ++h)
                        tma_load_2d(sB + s * BTILE + h * TC_TILE_BYTES, &mb, kb * TC_BK, n0 + 128 * h, fb);
                }
            }
            if (!ok) atomicExch(a.err, 1);
            // the copies of the last stages land before the CTA exits
            for (int64_t k = std::max<int64_t>(0, it - TC_STAGES); k < it; ++k)
                mbar_wait(smem_u32(&full[k % TC_STAGES]), (uint32_t)((k / TC_STAGES) & 1));
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issue
            int64_t it = 0;
            int tc = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
                const int c = tc & 1;
                if (tc >= 2 && !mbar_wait(smem_u32(&tempty[c]), (uint32_t)(((tc >> 1) - 1) & 1))) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(c * BN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % TC_STAGES);
                    if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / TC_STAGES) & 1))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < TC_BK / 16; ++j)
                        mma_bf16(acc, sw128_desc(sA + s * TC_TILE_BYTES + 32 * j), sw128_desc(sB + s * BTILE + 32 * j),
                                 IDESC, (kb > 0 || j > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[s]));
                }
                mma_commit(smem_u32(&tfull[c]));
            }
            if (!ok) atomicExch(a.err, 1);
            // every product issued has completed before the accumulators are freed
            mma_commit(smem_u32(&done));
            if (!mbar_wait(smem_u32(&done), 0u)) atomicExch(a.err, 1);
        }
        __syncwarp();
    } else {  // epilogue warps 2..5
        const int quad = warp & 3;
        int tc = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
            const int c = tc & 1;
            const bool got = mbar_wait(smem_u32(&tfull[c]), (uint32_t)((tc >> 1) & 1));
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicExch(a.err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int mbk, nbk;
            tc_tile(t, tn, ntiles / tn, mbk, nbk);
            const int m0 = mbk * TC_BM, n0 = nbk * BN;
            float(*tile)[33] = stile[warp - 2];
            for (int cc = 0; cc < BN; cc += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * BN + cc), v);
#pragma unroll
                for (int i = 0; i < 32; ++i) tile[lane][i] = v[i];  // lane = row of the chunk
                __syncwarp();
                const int n = n0 + cc + lane;  // lane = column: every row goes out as one 128-byte segment
                const float bn = (a.bias && n < a.N) ? a.bias[n] : 0.f;
                for (int r = 0; r < 32; ++r) {
                    const int row = m0 + quad * 32 + r;
                    if (row >= a.M || n >= a.N) continue;
                    float x = tile[r][lane];
                    if (a.bias) x += bn;
                    if (a.Z) a.Z[(int64_t)row * a.ldc + n] = x;
                    if (a.relu) x = fmaxf(x, 0.f);
                    a.C[(int64_t)row * a.ldc + n] = x;
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[c])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
    }
}

// sum of the split partials in split order, then the epilogue
__global__ void k_tc_reduce(int M, int N, int splits, const float *__restrict__ P, float *__restrict__ C, int ldc,
                            const float *__restrict__ bias, int relu, float *__restrict__ Z) {
    const int64_t MN = (int64_t)M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / N;
        const int n = (int)(e - m * N);
        float x = 0.f;
        for (int z = 0; z < splits; ++z) x += P[z * MN + e];
        if (bias) x += bias[n];
        if (Z) Z[m * ldc + n] = x;
        if (relu) x = fmaxf(x, 0.f);
        C[m * ldc + n] = x;
    }
}

// dst[r kw + g kseg + k] = part_g(src(r, k)) for r < R, segment g < nseg,
// k < kseg (zero for k >= K); src(r, k) = trans ? src[k ld + r] : src[r ld + k];
// part code 0: hi = bf16(x), 1: lo = bf16(x - hi)
__global__ void k_tc_pack(int64_t R, int K, int kseg, int nseg, uint32_t codes, const float *__restrict__ src,
                          int64_t ld, int trans, __nv_bfloat16 *__restrict__ dst, int64_t kw) {
    const int64_t total = R * kseg;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r, k;
        if (trans) {  // r fastest: the source reads are coalesced
            k = e / R;
            r = e - k * R;
        } else {
            r = e / kseg;
            k = e - r * kseg;
        }
        const float x = k < K ? (trans ? src[k * ld + r] : src[r * ld + k]) : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        for (int g = 0; g < nseg; ++g) dst[r * kw + (int64_t)g * kseg + k] = ((codes >> (2 * g)) & 3u) ? lo : hi;
    }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

template <int BN>
void tc_launch(const TcOperand &A, const TcOperand &B, const TcArgs &a, int tn, int tm, int splits, cudaStream_t s) {
    const int ntiles = tn * tm;
    if (splits == 1 && ntiles >= 2 * 152)  // enough tiles that a CTA per SM overlaps its epilogues
        k_tc_gemm_persistent<BN><<<152, 192, tc_smem<BN>(), s>>>(A.map, B.map, a, tn, ntiles);
    else
        k_tc_gemm<BN><<<dim3(tn, tm, splits), 128, tc_smem<BN>(), s>>>(A.map, B.map, a);
}
}  // namespace

cs_status tc_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int64_t rows, int64_t kw) {
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return CS_ERR_CUDA;
    }
    if (((uintptr_t)ptr & 15) || kw % 8 || rows < 1 || kw < 1) {
        set_error("tensor-core operand: base not 16-byte aligned or K width not a multiple of 8");
        return CS_ERR_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)kw, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kw * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
    const cuuint32_t es[2] = {1, 1};
    std::memset(map, 0, sizeof(*map));
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)ptr, dims, strides, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return CS_ERR_CUDA;
    }
    return CS_OK;
}

cs_status tc_operand_init(TcOperand &op, int64_t rows, int64_t kw, int64_t *acct) {
    op.rows = rows;
    op.kw = kw;
    CSX_TRY(dalloc_t(&op.p, (size_t)(rows * kw), acct));
    CSX_CUDA(cudaMemset(op.p, 0, sizeof(__nv_bfloat16) * (size_t)(rows * kw)));
    return tc_map(&op.map, op.p, rows, kw);
}

cs_status tc_pack(TcOperand &op, int64_t R, int K, int kseg, const char *parts, const float *src, int64_t ld,
                  bool trans, cudaStream_t s) {
    const int nseg = (int)std::strlen(parts);
    if (R > op.rows || (int64_t)nseg * kseg > op.kw || kseg % TC_BK || K > kseg) {
        set_error("tensor-core operand too small for the pack");
        return CS_ERR_ARG;
    }
    uint32_t codes = 0;
    for (int g = 0; g < nseg; ++g) codes |= (parts[g] == 'l' ? 1u : 0u) << (2 * g);
    const int64_t total = R * kseg;
    k_tc_pack<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16)), 256, 0, s>>>(
        R, K, kseg, nseg, codes, src, ld, trans ? 1 : 0, op.p, op.kw);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    return CS_OK;
}

cs_status tc_gemm(const TcOperand &A, const TcOperand &B, int M, int N, int64_t K, float *C, int ldc,
                  const float *bias, bool relu, float *Z, float *partial, int64_t partial_cap, int *err,
                  cudaStream_t s) {
    if (M < 1 || N < 1 || K < 1 || M > A.rows || N > B.rows || K > A.kw || K > B.kw) {
        set_error("tensor-core GEMM: shape exceeds its operands");
        return CS_ERR_ARG;
    }
    std::call_once(g_attr_once, [] {
        g_attr_err = cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<128>());
        if (g_attr_err == cudaSuccess)
            g_attr_err =
                cudaFuncSetAttribute(k_tc_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<256>());
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(k_tc_gemm_persistent<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              tc_smem<128>());
        if (g_attr_err == cudaSuccess)
            g_attr_err = cudaFuncSetAttribute(k_tc_gemm_persistent<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              tc_smem<256>());
    });
    CSX_CUDA(g_attr_err);
    const int bn = N > 128 ? 256 : 128;  // one MMA of N = 256 per K step when the columns need it
    const int nkb = (int)((K + TC_BK - 1) / TC_BK);
    const int tn = (N + bn - 1) / bn, tm = (M + TC_BM - 1) / TC_BM;
    int splits = tn * tm >= 76 ? 1 : std::min(nkb, (152 + tn * tm - 1) / (tn * tm));
    int kps = (nkb + splits - 1) / splits;
    splits = (nkb + kps - 1) / kps;  // every split gets at least one K block
    if (splits > 1 && (!partial || (int64_t)splits * M * N > partial_cap)) {
        splits = 1;
        kps = nkb;
    }
    TcArgs a;
    a.M = M; a.N = N; a.nkb = nkb; a.kps = kps;
    a.partial = splits > 1;
    a.C = splits > 1 ? partial : C;
    a.ldc = ldc;
    a.bias = bias; a.relu = relu ? 1 : 0; a.Z = Z;
    a.err = err;
    if (bn == 256) tc_launch<256>(A, B, a, tn, tm, splits, s);
    else tc_launch<128>(A, B, a, tn, tm, splits, s);
    count_launch();
    CSX_CUDA(cudaGetLastError());
    if (splits > 1) {
        const int64_t MN = (int64_t)M * N;
        k_tc_reduce<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((MN + 255) / 256, 152 * 8)), 256, 0, s>>>(
            M, N, splits, partial, C, ldc, bias, relu ? 1 : 0, Z);
        count_launch();
        CSX_CUDA(cudaGetLastError());
    }
    return CS_OK;
}

}  // namespace csx

extern "C" {

cs_status cs_tc_gemm_bf16(int M, int N, int K, const void *A, const void *B, float *C, cs_stream stream) {
    using namespace csx;
    if (M < 1 || N < 1 || K < 8 || K % 8 || !A || !B || !C) {
        set_error("cs_tc_gemm_bf16: M, N >= 1, K a positive multiple of 8, non-null operands");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    CSX_CUDA(cudaGetDevice(&dev));
    const void *ptrs[3] = {A, B, C};
    const char *names[3] = {"A", "B", "C"};
    for (int k = 0; k < 3; ++k) {  // the operands must be memory of the current device
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptrs[k]) != cudaSuccess) {
            cudaGetLastError();
            set_error("cs_tc_gemm_bf16: %s is not a CUDA device pointer", names[k]);
            return CS_ERR_ARG;
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
            set_error("cs_tc_gemm_bf16: %s must be device memory of the current device %d", names[k], dev);
            return CS_ERR_ARG;
        }
    }
    // one wait-expiry flag per device, allocated on first use there
    static int *errs[64] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= 64) { set_error("device ordinal %d unsupported", dev); return CS_ERR_UNSUPPORTED; }
    int *err = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!errs[dev]) CSX_CUDA(cudaMalloc(&errs[dev], sizeof(int)));
        err = errs[dev];
    }
    TcOperand a, b;
    a.p = (__nv_bfloat16 *)A; a.rows = M; a.kw = K;
    b.p = (__nv_bfloat16 *)B; b.rows = N; b.kw = K;
    CSX_TRY(tc_map(&a.map, a.p, M, K));
    CSX_TRY(tc_map(&b.map, b.p, N, K));
    CSX_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    CSX_TRY(tc_gemm(a, b, M, N, K, C, N, nullptr, false, nullptr, nullptr, 0, err, s));
    int h = 0;
    CSX_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    if (h) {
        set_error("a tensor-core GEMM wait expired");
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}

}  // extern "C"
