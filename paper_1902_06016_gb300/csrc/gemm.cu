// FP64 SIMT GEMMs with arbitrary element strides (real and complex).
//
// GB300's FP64 pipe is narrow, so these kernels are FP64-ALU bound for every shape used here;
// the tiling (64x64 output tile, 16-deep K slab, 4x4 register micro-tile, double-buffered shared
// memory) keeps the DFMA pipe fed. They serve the one-time H-bar build, the FP64 residual sigma and
// the FP64 projections of the reduced model.
#include "gfcc_internal.cuh"
#include "ozaki.cuh"

#include <algorithm>

namespace gfcc {
namespace {

constexpr int BM = 64, BN = 64;

template <typename T> struct Ops;
template <> struct Ops<double> {
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __device__ static double cj(double a, bool) { return a; }
};
template <> struct Ops<cplx> {
  __host__ __device__ static cplx zero() { return make_cuDoubleComplex(0.0, 0.0); }
  __host__ __device__ static cplx one() { return make_cuDoubleComplex(1.0, 0.0); }
  __device__ static cplx fma(cplx a, cplx b, cplx c) {
    return make_cuDoubleComplex(::fma(a.x, b.x, ::fma(-a.y, b.y, c.x)), ::fma(a.x, b.y, ::fma(a.y, b.x, c.y)));
  }
  __device__ static cplx cj(cplx a, bool c) { return c ? make_cuDoubleComplex(a.x, -a.y) : a; }
};

__device__ inline double scal_mul(double a, double b) { return a * b; }
__device__ inline cplx scal_mul(cplx a, cplx b) { return cuCmul(a, b); }
__device__ inline double scal_add(double a, double b) { return a + b; }
__device__ inline cplx scal_add(cplx a, cplx b) { return cuCadd(a, b); }
__host__ __device__ inline bool is_zero(double a) { return a == 0.0; }
__host__ __device__ inline bool is_zero(cplx a) { return a.x == 0.0 && a.y == 0.0; }

template <typename T>
struct Args {
  int M, N, K;
  const T* A; long long sam, sak, bsa; bool conjA;
  const T* B; long long sbk, sbn, bsb; bool conjB;
  T* C; long long scm, scn, bsc;
  T alpha, beta;
  int ksplit = 1, kchunk = 0;   // split-K: blockIdx.z = batch * ksplit + split, partials in C
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
  const long long bz = blockIdx.z / g.ksplit;
  const int split = blockIdx.z % g.ksplit;
  const int kbeg = split * g.kchunk;
  const int kend = g.ksplit > 1 ? min(g.K, kbeg + g.kchunk) : g.K;
  const T* A = g.A + bz * g.bsa + (long long)kbeg * g.sak;
  const T* B = g.B + bz * g.bsb + (long long)kbeg * g.sbk;
  T* C = g.C + bz * g.bsc + (g.ksplit > 1 ? (long long)split * g.M * g.N : 0LL);
  const int Kloc = max(0, kend - kbeg);
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
      ra[r] = (gm < g.M && gk < Kloc) ? Ops<T>::cj(A[gm * g.sam + gk * g.sak], g.conjA) : Ops<T>::zero();
      int nn, kb;
      if (b_n_fast) { nn = idx % BN; kb = idx / BN; } else { kb = idx % BK; nn = idx / BK; }
      int gn = n0 + nn, gkb = k0 + kb;
      rb[r] = (gn < g.N && gkb < Kloc) ? Ops<T>::cj(B[gkb * g.sbk + gn * g.sbn], g.conjB) : Ops<T>::zero();
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

  const int nk = (Kloc + BK - 1) / BK;
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

// C = alpha * sum_split P[split] + beta * C  (P packed [batch][ksplit][M][N])
template <typename T>
__global__ void splitk_reduce_kernel(const T* __restrict__ P, int ksplit, int M, int N, int batch, T* C, long long scm,
                                     long long scn, long long bsc, T alpha, T beta) {
  const long long per = (long long)M * N;
  const long long total = per * batch;
  const bool beta0 = is_zero(beta);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, r = t % per;
    const int m = (int)(r / N), n = (int)(r % N);
    T sum = Ops<T>::zero();
    for (int k = 0; k < ksplit; ++k) sum = scal_add(sum, P[(b * ksplit + k) * per + r]);
    T* cp = C + b * bsc + m * scm + n * scn;
    T v = scal_mul(alpha, sum);
    if (!beta0) v = scal_add(v, scal_mul(beta, *cp));
    *cp = v;
  }
}

// Matrix-vector shapes (M == 1; N == 1 is mapped onto it by exchanging the operands): out[n] =
// sum_k opA[k] opB[k][n] over this block's K range, one HBM pass over B instead of 64x64 tiles that
// would be 1/64 occupied. Threads run along whichever B index is contiguous: along n (one thread per
// n) or along k (one warp per n, shuffle-reduced). With ksplit > 1 the sums are partials [z][n].
template <typename T>
__device__ __forceinline__ void gemv_store(const Args<T>& g, long long bz, int split, int n, T acc) {
  if (g.ksplit > 1) {
    g.C[(bz * g.ksplit + split) * (long long)g.N + n] = acc;
    return;
  }
  T* cp = g.C + bz * g.bsc + n * g.scn;
  T v = scal_mul(g.alpha, acc);
  if (!is_zero(g.beta)) v = scal_add(v, scal_mul(g.beta, *cp));
  *cp = v;
}
template <typename T>
__global__ void __launch_bounds__(256) gemv_n_kernel(Args<T> g) {
  const int n = blockIdx.x * 256 + threadIdx.x;
  const long long bz = blockIdx.z / g.ksplit;
  const int split = blockIdx.z % g.ksplit;
  const int kbeg = split * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  if (n >= g.N) return;
  const T* A = g.A + bz * g.bsa;
  const T* B = g.B + bz * g.bsb + n * g.sbn;
  T acc = Ops<T>::zero();
#pragma unroll 4
  for (int k = kbeg; k < kend; ++k)
    acc = Ops<T>::fma(Ops<T>::cj(A[k * g.sak], g.conjA), Ops<T>::cj(B[k * g.sbk], g.conjB), acc);
  gemv_store(g, bz, split, n, acc);
}
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ cplx shfl_down(cplx v, int o) {
  return make_cuDoubleComplex(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}
template <typename T>
__global__ void __launch_bounds__(256) gemv_k_kernel(Args<T> g) {
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const long long bz = blockIdx.z / g.ksplit;
  const int split = blockIdx.z % g.ksplit;
  const int kbeg = split * g.kchunk, kend = min(g.K, kbeg + g.kchunk);
  if (n >= g.N) return;   // whole warps leave together
  const T* A = g.A + bz * g.bsa;
  const T* B = g.B + bz * g.bsb + n * g.sbn;
  T acc = Ops<T>::zero();
  for (int k = kbeg + lane; k < kend; k += 32)
    acc = Ops<T>::fma(Ops<T>::cj(A[k * g.sak], g.conjA), Ops<T>::cj(B[k * g.sbk], g.conjB), acc);
  for (int o = 16; o > 0; o >>= 1) acc = scal_add(acc, shfl_down(acc, o));
  if (lane == 0) gemv_store(g, bz, split, n, acc);
}

template <typename T>
void launch_gemv(Args<T> a, int batch, cudaStream_t s) {
  ProfScope prof(PROF_F64_GEMM, (sizeof(T) == 8 ? 2.0 : 8.0) * (double)a.M * (double)a.N * (double)a.K * batch, s);
  if (a.M != 1) {   // N == 1: C^T = op(B)^T op(A)^T, a row vector times a matrix
    std::swap(a.M, a.N);
    std::swap(a.A, a.B);
    std::swap(a.sam, a.sbn);
    std::swap(a.sak, a.sbk);
    std::swap(a.bsa, a.bsb);
    std::swap(a.conjA, a.conjB);
    std::swap(a.scm, a.scn);
  }
  const bool along_n = a.sbn <= a.sbk;
  const long long bx = along_n ? (a.N + 255) / 256 : (a.N + 7) / 8;
  GFCC_CHECK(bx <= 0x7fffffffLL, GFCC_ERR_ARG, "gemv N too large");
  const long long per_split = bx * batch;
  int ksplit = (int)std::max<long long>(1, std::min<long long>((4 * 152 + per_split - 1) / per_split, a.K / 64));
  ksplit = std::max(1, std::min(ksplit, 65535 / std::max(batch, 1)));
  const int kchunk = (a.K + ksplit - 1) / ksplit;
  ksplit = (a.K + kchunk - 1) / kchunk;
  GFCC_CHECK((long long)batch * ksplit <= 65535, GFCC_ERR_ARG, "gemv batch too large");
  const dim3 grid((unsigned)bx, 1, (unsigned)(batch * ksplit));
  Args<T> p = a;
  p.ksplit = ksplit;
  p.kchunk = kchunk;
  DBuf<T> part;
  if (ksplit > 1) {
    part.alloc((long long)a.N * ksplit * batch);
    p.C = part.p;
  }
  if (along_n) gemv_n_kernel<T><<<grid, 256, 0, s>>>(p);
  else gemv_k_kernel<T><<<grid, 256, 0, s>>>(p);
  GFCC_LAUNCH_CHECK();
  if (ksplit == 1) return;
  const long long total = (long long)a.N * batch;
  const int rgrid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
  // partials [batch][ksplit][1][N]; C row 0, column n at C + n scn
  splitk_reduce_kernel<T><<<rgrid, 256, 0, s>>>(part.p, ksplit, 1, a.N, batch, a.C, a.scm, a.scn, a.bsc, a.alpha,
                                                a.beta);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(s));   // the partial buffer is released on return
}

template <typename T>
void launch(Args<T> a, int batch, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || batch <= 0) return;
  if (a.M == 1 || a.N == 1) {
    launch_gemv(a, batch, s);
    return;
  }
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, batch);
  GFCC_CHECK(grid.y <= 65535, GFCC_ERR_ARG, "gemm M too large");
  constexpr int BK = sizeof(T) == 8 ? 16 : 8;   // 33 KB of static shared memory either way
  ProfScope prof(PROF_F64_GEMM, (sizeof(T) == 8 ? 2.0 : 8.0) * (double)a.M * (double)a.N * (double)a.K * batch, s);
  // too few tiles to fill 152 SMs and a long K: split K, then reduce the partial tiles
  const long long tiles = (long long)grid.x * grid.y * batch;
  int ksplit = 1;
  if (tiles < 2 * 152 && a.K >= 1024) {
    ksplit = (int)std::min<long long>((2 * 152 + tiles - 1) / tiles, a.K / 256);
    ksplit = std::max(1, std::min(ksplit, 65535 / std::max(batch, 1)));
  }
  GFCC_CHECK((long long)batch * ksplit <= 65535, GFCC_ERR_ARG, "gemm batch too large");
  if (ksplit == 1) {
    gemm_kernel<T, BK><<<grid, 256, 0, s>>>(a);
    GFCC_LAUNCH_CHECK();
    return;
  }
  const int kchunk = ((a.K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
  ksplit = (a.K + kchunk - 1) / kchunk;
  const long long per = (long long)a.M * a.N;
  DBuf<T> part;
  part.alloc(per * ksplit * batch);
  Args<T> p = a;
  p.C = part.p;
  p.scm = a.N;
  p.scn = 1;
  p.bsc = per * ksplit;
  p.alpha = Ops<T>::one();
  p.beta = Ops<T>::zero();
  p.ksplit = ksplit;
  p.kchunk = kchunk;
  // partial z = batch * ksplit + split lands at part + (batch * ksplit + split) * per
  p.bsc = per * ksplit;
  grid.z = batch * ksplit;
  gemm_kernel<T, BK><<<grid, 256, 0, s>>>(p);
  GFCC_LAUNCH_CHECK();
  const long long total = per * batch;
  const int rgrid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
  splitk_reduce_kernel<T><<<rgrid, 256, 0, s>>>(part.p, ksplit, a.M, a.N, batch, a.C, a.scm, a.scn, a.bsc, a.alpha,
                                                a.beta);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(s));   // the partial buffer is released on return
}

}  // namespace

void dgemm(const GemmDesc& d, cudaStream_t s) {
  Args<double> a{d.M, d.N, d.K, d.A, d.sam, d.sak, d.bsa, false, d.B, d.sbk, d.sbn, d.bsb, false,
                 d.C, d.scm, d.scn, d.bsc, d.alpha, d.beta};
  launch(a, d.batch, s);
}

void zgemm(const ZGemmDesc& d, cudaStream_t s) {
  // large complex products (the subspace projections of the reduced model) go to the exact-slice
  // tensor-core GEMM with 7 slices (48 bits per row)
  if (d.batch == 1 && (double)d.M * (double)d.N * (double)d.K >= oz_min_macs() && d.M >= 16 && d.N >= 1 &&
      (double)d.K >= 256) {
    zgemm_oz(d, 7, s);
    return;
  }
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
