// Tensor-core (tcgen05) BF16 GEMM C = A B^T used by the learned-setup
// network; see cs_tcgemm.cu.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "cs_internal.cuh"

namespace csx {

struct TcArgs {
    int M, N, nkb, kps;  // rows and columns of C, 64-wide K blocks in all, K blocks per split
    float *C;            // C (row stride ldc), or the split partials [split][M][N]
    int ldc;
    const float *bias;   // [N] or null
    int relu;
    float *Z;            // pre-activation copy (row stride ldc) or null
    int partial;
    int *err;            // set to 1 when a bounded wait expires
};

// A BF16 operand in HBM, K contiguous: rows x kw (kw a multiple of 8), with
// its TMA tensor map (128 x 64 boxes, 128-byte swizzle, zero fill outside).
struct TcOperand {
    __nv_bfloat16 *p = nullptr;
    int64_t rows = 0, kw = 0;
    CUtensorMap map;
};

cs_status tc_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int64_t rows, int64_t kw);
// allocate (zeroed) and describe a rows x kw operand
cs_status tc_operand_init(TcOperand &op, int64_t rows, int64_t kw, int64_t *acct);
// pack R rows of an FP32 matrix as K-segments of kseg columns (K valid, the
// rest zero): parts[g] = 'h' (bf16(x)) or 'l' (bf16(x - bf16(x))) for
// segment g; trans: element (r, k) is src[k ld + r], else src[r ld + k]
cs_status tc_pack(TcOperand &op, int64_t R, int K, int kseg, const char *parts, const float *src, int64_t ld,
                  bool trans, cudaStream_t s);
// C[M x N] (+ bias, ReLU, Z) = A[M x K] B[N x K]^T on the tensor cores,
// split along K when the tile grid is small (partials in partial[0 ..
// partial_cap), reduced in split order)
cs_status tc_gemm(const TcOperand &A, const TcOperand &B, int M, int N, int64_t K, float *C, int ldc,
                  const float *bias, bool relu, float *Z, float *partial, int64_t partial_cap, int *err,
                  cudaStream_t s);

}  // namespace csx
