// tcgen05 tensor-core GEMM for sm_103a (internal):  C[M x N] (+)= A[M x K] * B[N x K]^T
//
// A and B are K-major (row-major with K contiguous) in bf16 or fp32-as-tf32, K padded to a multiple
// of the 128-byte k-block. A persistent grid (at most one CTA per SM) walks the 128 x 256 output
// tiles (x K splits); each tile is accumulated in TMEM by tcgen05.mma issued from one thread, with
// two 256-column accumulators so that the epilogue of one tile overlaps the MMAs of the next;
// operands are staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) through a 4-stage mbarrier
// pipeline; the epilogue warps read TMEM with tcgen05.ld and write FP32 rows. K splits write
// partial results at C + z * split_stride.
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
// prof_class / k_alg: profiling class of the launch and the unpadded K for its algorithmic flop count
// (0: the padded K).
void tc_gemm(TcKind kind, const TcOperand& A, const TcOperand& B, float* C, long long ldc, long long M,
             long long N, int beta, int ksplit, long long split_stride, int* err_dev, cudaStream_t s,
             int prof_class = 0, long long k_alg = 0);

// Exact integer GEMM for the Ozaki slices: A and B bf16 holding integers of magnitude <= 64, so
// that 2048 products sum exactly in FP32. P[z][m][n] (int32, row stride ldp, split z at
// P + z * split_stride) = sum over the k-blocks of split z of A[m][k] B[n][k]; the K range is cut
// into at most zs equal splits of at most TC_EXACT_MAX_KB k-blocks (255 exact FP32 accumulations of
// 32 k-blocks, |sum| < 255 * 2^23 < 2^31). Rows >= M and columns >= N are not written. Returns the
// number of splits written (<= zs; P must hold zs splits).
constexpr int TC_EXACT_MAX_KB = 255 * 32;
int tc_gemm_exact(const TcOperand& A, const TcOperand& B, int* P, long long ldp, long long M, long long N, int zs,
                   long long split_stride, int* err_dev, cudaStream_t s, int prof_class = 0);
// number of K splits for tc_gemm_exact: about one wave of work units, within the int32 bound
int tc_exact_splits(long long M, long long N, long long k_pad);

// k-block (elements) of a kind: 64 bf16 or 32 tf32 = 128 bytes
inline int tc_kblock(TcKind k) { return k == TcKind::BF16 ? 64 : 32; }
inline int tc_pad_k(TcKind k, long long K) { int b = tc_kblock(k); return (int)((K + b - 1) / b * b); }

}  // namespace gfcc
