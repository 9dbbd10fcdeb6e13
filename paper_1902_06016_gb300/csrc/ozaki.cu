// Exact-slice FP64 GEMM on the tensor cores (see ozaki.cuh).
#include "ozaki.cuh"
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

namespace gfcc {
namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// one block per row (grid-stride): row exponent from the largest |x|, then S integer slices
__global__ void __launch_bounds__(256) slice_kernel(const double* __restrict__ X, long long ldx, long long rows,
                                                    long long K, long long kp, int reversed, int ns,
                                                    __nv_bfloat16* __restrict__ out, int* __restrict__ expo) {
  __shared__ double red[256];
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double* x = X + r * ldx;
    double mx = 0.0;
    for (long long k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(x[k]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
      __syncthreads();
    }
    int e = 0;
    if (red[0] > 0.0) frexp(red[0], &e);   // max < 2^e
    __syncthreads();
    if (threadIdx.x == 0) expo[r] = e;
    __nv_bfloat16* o = out + r * (long long)ns * kp;
    for (long long k = threadIdx.x; k < kp; k += blockDim.x) {
      double v = k < K ? ldexp(x[k], 6 - e) : 0.0;   // |v| < 64
#pragma unroll
      for (int i = 0; i < OZ_SLICES_MAX; ++i) {
        if (i < ns) {
          double a = rint(v);
          v = (v - a) * 128.0;
          const int slot = reversed ? ns - 1 - i : i;
          o[(long long)slot * kp + k] = __float2bfloat16_rn((float)a);
        }
      }
    }
  }
}

// acc[t] (+)= scale * sum_z part[z*stride + t]: the int32 split sums of one diagonal, added exactly
// in 64-bit integers, then weighted and accumulated in FP64
__global__ void accumulate_kernel(const int* __restrict__ part, int zs, long long stride, long long total,
                                  double scale, int first, double* __restrict__ acc) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long sum = 0;
    for (int z = 0; z < zs; ++z) sum += part[z * stride + t];
    acc[t] = first ? scale * (double)sum : acc[t] + scale * (double)sum;
  }
}

// out[m*ldo + n] = beta * out + 2^(ea[m] + eb[n] - 12) * acc[m*N + n]
__global__ void finalize_kernel(const double* __restrict__ acc, const int* __restrict__ ea, const int* __restrict__ eb,
                                long long M, long long N, double* __restrict__ out, long long ldo, double beta) {
  const long long total = M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long m = t / N, n = t % N;
    double v = ldexp(acc[t], ea[m] + eb[n] - 12);
    double* p = out + m * ldo + n;
    *p = (beta == 0.0) ? v : beta * (*p) + v;
  }
}

// A'[m][2k + r] = (re, im) of op(A)(m, k), conj applied
__global__ void zgather_a_kernel(const cplx* __restrict__ A, long long sam, long long sak, int conjA, long long M,
                                 long long K, double* __restrict__ out) {
  const long long total = M * K;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long m = t / K, k = t % K;
    const cplx a = A[m * sam + k * sak];
    out[m * 2 * K + 2 * k] = a.x;
    out[m * 2 * K + 2 * k + 1] = conjA ? -a.y : a.y;
  }
}
// B'[n][2k + r]: rows n < N give the real part of the product (Br, -Bi), rows N + n the imaginary
// part (Bi, Br), with B(k, n) conjugated first when asked
__global__ void zgather_b_kernel(const cplx* __restrict__ B, long long sbk, long long sbn, int conjB, long long K,
                                 long long N, double* __restrict__ out) {
  const long long total = N * K;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long n = t / K, k = t % K;
    cplx b = B[k * sbk + n * sbn];
    if (conjB) b.y = -b.y;
    out[n * 2 * K + 2 * k] = b.x;
    out[n * 2 * K + 2 * k + 1] = -b.y;
    out[(N + n) * 2 * K + 2 * k] = b.y;
    out[(N + n) * 2 * K + 2 * k + 1] = b.x;
  }
}
// C(m, n) = alpha (T[m][n] + i T[m][N + n]) + beta C(m, n)
__global__ void zscatter_kernel(const double* __restrict__ T, long long M, long long N, cplx* __restrict__ C,
                                long long scm, long long scn, cplx alpha, cplx beta) {
  const long long total = M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long m = t / N, n = t % N;
    const cplx v = make_cuDoubleComplex(T[m * 2 * N + n], T[m * 2 * N + N + n]);
    cplx* p = C + m * scm + n * scn;
    cplx r = cuCmul(alpha, v);
    if (beta.x != 0.0 || beta.y != 0.0) r = cuCadd(r, cuCmul(beta, *p));
    *p = r;
  }
}

}  // namespace

double oz_min_macs() {
  double v = 1e9;
  if (const char* env = getenv("GFCC_OZ_MIN_MACS")) v = atof(env);
  return v;
}

void zgemm_oz(const ZGemmDesc& g, int ns, cudaStream_t s) {
  const long long M = g.M, N = g.N, K = g.K;
  GFCC_CHECK(g.batch == 1, GFCC_ERR_ARG, "zgemm_oz: no batches");
  DBuf<double> Ar, Br, T;
  Ar.alloc(M * 2 * K);
  Br.alloc(2 * N * 2 * K);
  zgather_a_kernel<<<grid_for(M * K), 256, 0, s>>>(g.A, g.sam, g.sak, g.conjA ? 1 : 0, M, K, Ar.p);
  GFCC_LAUNCH_CHECK();
  zgather_b_kernel<<<grid_for(N * K), 256, 0, s>>>(g.B, g.sbk, g.sbn, g.conjB ? 1 : 0, K, N, Br.p);
  GFCC_LAUNCH_CHECK();
  SlicedRows sa, sb;
  oz_slice(Ar.p, 2 * K, M, 2 * K, false, sa, s, ns);
  oz_slice(Br.p, 2 * K, 2 * N, 2 * K, true, sb, s, ns);
  GFCC_CUDA(cudaStreamSynchronize(s));
  Ar.release();
  Br.release();
  T.alloc(M * 2 * N);
  OzWork w;
  oz_gemm(sa, sb, M, 2 * N, T.p, 2 * N, 0.0, w, s);
  zscatter_kernel<<<grid_for(M * N), 256, 0, s>>>(T.p, M, N, g.C, g.scm, g.scn, g.alpha, g.beta);
  GFCC_LAUNCH_CHECK();
  int herr = 0;
  GFCC_CUDA(cudaMemcpyAsync(&herr, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  GFCC_CHECK(herr == 0, GFCC_ERR_CUDA, "zgemm_oz: tensor-core pipeline wait timed out");
}

void oz_slice_into(const double* X, long long ldx, long long nrows, long long K, SlicedRows& out, long long row0,
                   cudaStream_t s) {
  GFCC_CHECK(row0 >= 0 && row0 + nrows <= out.rows && K <= out.kp, GFCC_ERR_ARG, "oz_slice_into: out of range");
  if (nrows == 0) return;
  const int grid = (int)std::min<long long>(nrows, 152LL * 16);
  slice_kernel<<<grid, 256, 0, s>>>(X, ldx, nrows, K, out.kp, out.reversed ? 1 : 0, out.ns,
                                    reinterpret_cast<__nv_bfloat16*>(out.slices.p) + row0 * out.ns * out.kp,
                                    out.expo.p + row0);
  GFCC_LAUNCH_CHECK();
}

void oz_slice(const double* X, long long ldx, long long rows, long long K, bool reversed, SlicedRows& out,
              cudaStream_t s, int ns) {
  GFCC_CHECK(ns >= 2 && ns <= OZ_SLICES_MAX, GFCC_ERR_ARG, "oz_slice: 2..8 slices");
  out.rows = rows;
  out.kp = tc_pad_k(TcKind::BF16, K);
  out.ns = ns;
  out.reversed = reversed;
  out.slices.alloc(sizeof(__nv_bfloat16) * std::max<long long>(rows, 1) * ns * out.kp);
  out.expo.alloc(std::max<long long>(rows, 1));
  oz_slice_into(X, ldx, rows, K, out, 0, s);
}

void oz_gemm(const SlicedRows& A, const SlicedRows& B, long long M, long long N, double* out, long long ldo,
             double beta, OzWork& w, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  GFCC_CHECK(!A.reversed && B.reversed && A.kp == B.kp && A.ns == B.ns, GFCC_ERR_ARG,
             "oz_gemm: operand slicing mismatch");
  GFCC_CHECK(A.rows >= M && B.rows >= N, GFCC_ERR_ARG, "oz_gemm: operand rows");
  const int ns = A.ns;
  const long long kp = A.kp, ld = (long long)ns * kp;
  // int32 split sums of the largest diagonal, with N processed in column chunks to bound memory
  const int max_splits = tc_exact_splits(M, N, (long long)ns * kp);
  const long long slab_budget = 2LL << 30;   // bytes of int32 split sums at a time
  long long nc = std::max<long long>(1, slab_budget / (4LL * M * max_splits));
  nc = std::min<long long>(N, std::max<long long>(256, nc / 256 * 256));
  w.islabs.alloc((size_t)max_splits * M * nc);
  w.acc.alloc((size_t)M * nc);
  if (w.err.n == 0) { w.err.alloc(1); w.err.zero(s); }
  const __nv_bfloat16* As = reinterpret_cast<const __nv_bfloat16*>(A.slices.p);
  const __nv_bfloat16* Bs = reinterpret_cast<const __nv_bfloat16*>(B.slices.p);
  for (long long n0 = 0; n0 < N; n0 += nc) {
    const long long nn = std::min(nc, N - n0);
    for (int d = 0; d < ns; ++d) {
      // diagonal d: A slices 0..d against B slices d..0, concatenated along K
      const long long kd = (long long)(d + 1) * kp;
      const int zs = std::min(tc_exact_splits(M, nn, kd), max_splits);
      TcOperand a(As, M, kd, ld);
      TcOperand b(Bs + (long long)n0 * ld + (long long)(ns - 1 - d) * kp, nn, kd, ld);
      const int zeff = tc_gemm_exact(a, b, w.islabs.p, nn, M, nn, zs, M * nn, w.err.p, s, PROF_TC_SLICE);
      accumulate_kernel<<<grid_for(M * nn), 256, 0, s>>>(w.islabs.p, zeff, M * nn, M * nn, ldexp(1.0, -7 * d),
                                                          d == 0 ? 1 : 0, w.acc.p);
      GFCC_LAUNCH_CHECK();
    }
    finalize_kernel<<<grid_for(M * nn), 256, 0, s>>>(w.acc.p, A.expo.p, B.expo.p + n0, M, nn, out + n0, ldo, beta);
    GFCC_LAUNCH_CHECK();
  }
}

}  // namespace gfcc
