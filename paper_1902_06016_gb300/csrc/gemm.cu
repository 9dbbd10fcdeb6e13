// FP64 SIMT GEMMs with arbitrary element strides (real and complex).
//
// GB300's FP64 pipe is narrow, so these kernels are FP64-ALU bound for every shape used here;
// the tiling (64x64 output tile, 16-deep K slab, 4x4 register micro-tile, double-buffered shared
// memory) keeps the DFMA pipe fed. They serve the one-time H-bar build, the FP64 residual sigma and
// the FP64 projections of the reduced model.
#include "gfcc_internal.cuh"

namespace gfcc {
namespace {

constexpr int BM = 64, BN = 64;

template <typename T> struct Ops;
template <> struct Ops<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __device__ static double cj(double a, bool) { return a; }
};
template <> struct Ops<cplx> {
  __device__ static cplx zero() { return make_cuDoubleComplex(0.0, 0.0); }
  __device__ static cplx fma(cplx a, cplx b, cplx c) {
    return make_cuDoubleComplex(::fma(a.x, b.x, ::fma(-a.y, b.y, c.x)), ::fma(a.x, b.y, ::fma(a.y, b.x, c.y)));
  }
  __device__ static cplx cj(cplx a, bool c) { return c ? make_cuDoubleComplex(a.x, -a.y) : a; }
};

__device__ inline double scal_mul(double a, double b) { return a * b; }
__device__ inline cplx scal_mul(cplx a, cplx b) { return cuCmul(a, b); }
__device__ inline double scal_add(double a, double b) { return a + b; }
__device__ inline cplx scal_add(cplx a, cplx b) { return cuCadd(a, b); }
__device__ inline bool is_zero(double a) { return a == 0.0; }
__device__ inline bool is_zero(cplx a) { return a.x == 0.0 && a.y == 0.0; }

template <typename T>
struct Args {
  int M, N, K;
  const T* A; long long sam, sak, bsa; bool conjA;
  const T* B; long long sbk, sbn, bsb; bool conjB;
  T* C; long long scm, scn, bsc;
  T alpha, beta;
};

// 256 threads: thread (tx, ty) in a 16x16 grid owns rows ty + 16*i and columns tx + 16*j.
template <typename T, int BK>
__global__ void __launch_bounds__(256) gemm_kernel(Args<T> g) {
  constexpr int LPT = BM * BK / 256;   // tile elements loaded per thread
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long long bz = blockIdx.z;
  const T* A = g.A + bz * g.bsa;
  const T* B = g.B + bz * g.bsb;
  T* C = g.C + bz * g.bsc;
  const bool a_k_fast = (g.sak == 1);
  const bool b_n_fast = (g.sbn == 1);

  T ra[LPT], rb[LPT];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LPT; ++r) {
      int idx = tid + 256 * r;
      int mm, kk;
      if (a_k_fast) { kk = idx % BK; mm = idx / BK; } else { mm = idx % BM; kk = idx / BM; }
      int gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < g.M && gk < g.K) ? Ops<T>::cj(A[gm * g.sam + gk * g.sak], g.conjA) : Ops<T>::zero();
      int nn, kb;
      if (b_n_fast) { nn = idx % BN; kb = idx / BN; } else { kb = idx % BK; nn = idx / BK; }
      int gn = n0 + nn, gkb = k0 + kb;
      rb[r] = (gn < g.N && gkb < g.K) ? Ops<T>::cj(B[gkb * g.sbk + gn * g.sbn], g.conjB) : Ops<T>::zero();
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LPT; ++r) {
      int idx = tid + 256 * r;
      int mm, kk;
      if (a_k_fast) { kk = idx % BK; mm = idx / BK; } else { mm = idx % BM; kk = idx / BM; }
      As[buf][kk][mm] = ra[r];
      int nn, kb;
      if (b_n_fast) { nn = idx % BN; kb = idx / BN; } else { kb = idx % BK; nn = idx / BK; }
      Bs[buf][kb][nn] = rb[r];
    }
  };

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Ops<T>::zero();

  const int nk = (g.K + BK - 1) / BK;
  if (nk > 0) {
    load_tiles(0);
    store_tiles(0);
  }
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_tiles((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Ops<T>::fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < nk) store_tiles(buf ^ 1);
    __syncthreads();
  }
  const bool beta0 = is_zero(g.beta);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      T* cp = C + gm * g.scm + gn * g.scn;
      T val = scal_mul(g.alpha, acc[i][j]);
      if (!beta0) val = scal_add(val, scal_mul(g.beta, *cp));
      *cp = val;
    }
  }
}

template <typename T>
void launch(const Args<T>& a, int batch, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || batch <= 0) return;
  GFCC_CHECK(batch <= 65535, GFCC_ERR_ARG, "gemm batch too large");
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, batch);
  GFCC_CHECK(grid.y <= 65535, GFCC_ERR_ARG, "gemm M too large");
  constexpr int BK = sizeof(T) == 8 ? 16 : 8;   // 33 KB of static shared memory either way
  gemm_kernel<T, BK><<<grid, 256, 0, s>>>(a);
  GFCC_LAUNCH_CHECK();
}

}  // namespace

void dgemm(const GemmDesc& d, cudaStream_t s) {
  Args<double> a{d.M, d.N, d.K, d.A, d.sam, d.sak, d.bsa, false, d.B, d.sbk, d.sbn, d.bsb, false,
                 d.C, d.scm, d.scn, d.bsc, d.alpha, d.beta};
  launch(a, d.batch, s);
}

void zgemm(const ZGemmDesc& d, cudaStream_t s) {
  Args<cplx> a{d.M, d.N, d.K, d.A, d.sam, d.sak, d.bsa, d.conjA, d.B, d.sbk, d.sbn, d.bsb, d.conjB,
               d.C, d.scm, d.scn, d.bsc, d.alpha, d.beta};
  launch(a, d.batch, s);
}

void dgemm_rm(int M, int N, int K, double alpha, const double* A, int lda, bool transA,
              const double* B, int ldb, bool transB, double beta, double* C, int ldc, cudaStream_t s) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.sam = transA ? 1 : lda; g.sak = transA ? lda : 1;
  g.B = B; g.sbk = transB ? 1 : ldb; g.sbn = transB ? ldb : 1;
  g.C = C; g.scm = ldc; g.scn = 1;
  g.alpha = alpha; g.beta = beta;
  dgemm(g, s);
}

}  // namespace gfcc
