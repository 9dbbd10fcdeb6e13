// tcgen05 tensor-core GEMM for sm_103a (internal):  C[M x N] (+)= A[M x K] * B[N x K]^T
//
// A and B are K-major (row-major with K contiguous) in bf16 or fp32-as-tf32, K padded to a multiple
// of the 128-byte k-block. Tiles of 128 x 256 are accumulated in TMEM (256 FP32 columns) by
// tcgen05.mma issued from one thread; operands are staged by TMA (cp.async.bulk.tensor, 128-byte
// swizzle) through a 4-stage mbarrier pipeline; four epilogue warps read TMEM with tcgen05.ld and
// write FP32 rows. blockIdx.z splits K (partial results at C + z * split_stride).
#pragma once
#include "gfcc_internal.cuh"

namespace gfcc {

enum class TcKind { BF16 = 0, TF32 = 1 };

struct TcOperand {
  const void* ptr = nullptr;   // device, row-major
  long long rows = 0;          // logical rows (TMA zero-fills beyond)
  long long k_pad = 0;         // K extent in elements (multiple of the k-block)
  long long ld = 0;            // row stride in elements (0: k_pad); multiple of the k-block
  TcOperand() = default;
  TcOperand(const void* p, long long r, long long k, long long l = 0) : ptr(p), rows(r), k_pad(k), ld(l ? l : k) {}
};

// Launch C = A B^T (beta = 0) or C += A B^T (beta = 1). C is FP32 row-major with leading dimension
// ldc; rows >= M and columns >= N are not written. ksplit > 1 splits K into equal k-block ranges and
// writes partial tiles to C + z * split_stride (beta must be 0 then).
void tc_gemm(TcKind kind, const TcOperand& A, const TcOperand& B, float* C, long long ldc, long long M,
             long long N, int beta, int ksplit, long long split_stride, int* err_dev, cudaStream_t s,
             int prof_class = 0);

// k-block (elements) of a kind: 64 bf16 or 32 tf32 = 128 bytes
inline int tc_kblock(TcKind k) { return k == TcKind::BF16 ? 64 : 32; }
inline int tc_pad_k(TcKind k, long long K) { int b = tc_kblock(k); return (int)((K + b - 1) / b * b); }

}  // namespace gfcc
