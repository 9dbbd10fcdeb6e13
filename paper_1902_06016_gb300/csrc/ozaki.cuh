// FP64-accurate GEMM on the bf16 tensor cores by exact integer slicing (internal).
//
// Each row r of an FP64 operand is scaled by a power of two and written as
//   x = 2^(e_r - 6) * sum_{i<S} a_i 2^(-7 i),   a_i integers with |a_i| <= 64,
// so every a_i is exact in bf16 and every product a_i b_j is an integer of magnitude <= 2^12.
// A K-chunk of at most 2048 such products sums to an integer below 2^23, which the FP32 tensor-core
// accumulator holds exactly. The slice pairs with i + j = d ("diagonal" d) are one GEMM with the
// slices concatenated along K (A slices in order 0..d, B slices in order d..0); its K-chunks are
// accumulated exactly inside the GEMM kernel in int32 (each chunk's FP32 sum is an exact integer),
// the per-split int32 sums are added in 64-bit integers and weighted by 2^(-7d) in FP64, and the total
// is scaled by 2^(e_A + e_B - 12). With S = 6 slices the representation keeps 41 bits of each row (relative to its
// largest element) and the dropped pairs (i + j >= S) weigh at most 2^-42 of the leading term: the
// result is accurate to about 2^-40 of sum_k |a_mk||b_nk|, far below what FP32 or TF32 give.
// (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012).)
#pragma once
#include "gfcc_internal.cuh"

namespace gfcc {

constexpr int OZ_SLICES = 6;       // residual sigma: 41 bits per row
constexpr int OZ_SLICES_MAX = 8;   // 55 bits per row: as accurate as an FP64 GEMM

struct SlicedRows {
  DBuf<uint8_t> slices;   // bf16 [rows][ns][kp] (order 0..ns-1, or reversed)
  DBuf<int> expo;         // [rows]
  long long rows = 0;
  long long kp = 0;       // padded K (multiple of 64)
  int ns = OZ_SLICES;
  bool reversed = false;
};

// Allocate out for rows x K (padded to 64) and slice all rows of the FP64 matrix X (row stride ldx)
// into ns slices.
void oz_slice(const double* X, long long ldx, long long rows, long long K, bool reversed, SlicedRows& out,
              cudaStream_t s, int ns = OZ_SLICES);
// Slice nrows rows of X into rows [row0, row0 + nrows) of an already allocated out (same kp).
void oz_slice_into(const double* X, long long ldx, long long nrows, long long K, SlicedRows& out, long long row0,
                   cudaStream_t s);

// out[m][n] = beta * out[m][n] + sum_k A[m][k] B[n][k] for m < M, n < N (out row stride ldo), with
// A = sliced rows (normal order) and B = sliced rows (reversed order), same kp.
struct OzWork {
  DBuf<int> islabs;   // int32 split sums of one diagonal of a column chunk
  DBuf<double> acc;   // FP64 sum of the diagonals so far
  DBuf<int> err;
};
void oz_gemm(const SlicedRows& A, const SlicedRows& B, long long M, long long N, double* out, long long ldo,
             double beta, OzWork& w, cudaStream_t s);

// Complex GEMM C = alpha op(A) op(B) + beta C (strided, see ZGemmDesc) evaluated as one real
// exact-slice GEMM: K interleaves (re, im) and the N axis stacks the real and imaginary parts.
void zgemm_oz(const ZGemmDesc& g, int ns, cudaStream_t s);
// multiply-adds above which zgemm() uses zgemm_oz (GFCC_OZ_MIN_MACS overrides)
double oz_min_macs();
// bytes of int32 split sums up to which all diagonals of an exact product are kept side by side and
// summed into the output in one pass (default 4 GiB; GFCC_OZ_SLAB_BYTES overrides, so that tests can
// run the per-diagonal FP64 accumulation over column chunks at small sizes)
double oz_slab_bytes();

}  // namespace gfcc
