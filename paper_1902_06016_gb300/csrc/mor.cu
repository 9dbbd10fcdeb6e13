// Model-order reduction of the MIMO system (Eqs. gfcclineqn and model) on the GPU, FP64.
//
// * Subspace: S holds orthonormalised solutions X_p(w_k). New columns lose their components along
//   the current S by block classical Gram-Schmidt (two passes), then within the block panel by panel:
//   Cholesky QR twice for well-conditioned panels, otherwise column by column (two passes); a column is
//   kept when its norm after the passes is >= drop_tol times its norm before, else dropped.
//   Orthonormality is in the complex inner product, so the projections written S^T in Eq. model are
//   applied as S^H.
// * Z = M S comes for free: every solved column satisfies M x = b - (w - i eta) x - r with the FP64
//   residual r of the solver, and every linear combination applied to S is applied to Z as well.
// * Reduced model: Hhat = S^H Z, bhat = S^H b, chat = c^T S, updated incrementally.
// * Evaluation at many frequencies: Hhat is reduced once to upper Hessenberg form by Householder
//   reflections (applied alongside to bhat, chat and the residual coefficients); each frequency is
//   then an O(m^2) shifted Hessenberg solve (one CTA per frequency, partial pivoting between adjacent
//   rows). Ghat_pq = chat_q^T yhat_p for all frequencies is one complex GEMM, and A = -(1/pi) sum_p
//   Im Ghat_pp.
// * Residual estimate for refinement: the columns of [B, S, Z] are kept as coefficients in an
//   orthonormal basis Q of their span (extended with every new block), so that the residual
//   r = (w - i eta) S y + Z y - b has the coefficient vector (w - i eta) R_S y + R_Z y - R_B e_p and
//   ||r|| is its 2-norm, without the cancellation of a Gram-matrix formula; the coefficients of all
//   frequencies are two complex GEMMs.
#include "gfcc_internal.cuh"
#include "ozaki.cuh"

#include <algorithm>
#include <cmath>

namespace gfcc {
namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

__device__ __forceinline__ cplx cz() { return make_cuDoubleComplex(0.0, 0.0); }

// dst[nu][off + k] = src[nu][cols[k]]
__global__ void append_cols_kernel(const cplx* __restrict__ src, int lds, const int* __restrict__ cols, int nk,
                                   cplx* __restrict__ dst, int ldd, int off, long long D) {
  long long total = D * nk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int k = (int)(t % nk);
    long long nu = t / nk;
    dst[nu * ldd + off + k] = src[nu * lds + cols[k]];
  }
}

// ---- Householder reduction to Hessenberg form (column-major matrices) ---------------------------
// v = x - alpha e1 with alpha = -e^{i arg x0} ||x||, tau = 2 / ||v||^2; stores v in vbuf[0..len), tau in *tau
__global__ void house_kernel(const cplx* __restrict__ x, int len, cplx* __restrict__ v, double* __restrict__ tau) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) s += x[i].x * x[i].x + x[i].y * x[i].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  double nx = sqrt(red[0]);
  cplx x0 = x[0];
  double a0 = cuCabs(x0);
  cplx ph = a0 > 0.0 ? make_cuDoubleComplex(x0.x / a0, x0.y / a0) : make_cuDoubleComplex(1.0, 0.0);
  cplx alpha = make_cuDoubleComplex(-ph.x * nx, -ph.y * nx);
  for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = x[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    v[0] = cuCsub(x0, alpha);
    double vn2 = red[0] - (x0.x * x0.x + x0.y * x0.y) + (v[0].x * v[0].x + v[0].y * v[0].y);
    *tau = (nx > 0.0 && vn2 > 0.0) ? 2.0 / vn2 : 0.0;
  }
}
// A reflection H = I - tau v v^H applied to several column-major matrices at once (one launch per side
// and Householder step):
//   left:  A[r0+i][col] -= tau v[i] (sum_k conj(v[k]) A[r0+k][col]) on the columns of A (from c0a) and B
//   right: w[row] = sum_k A[row][c0+k] v[k]; A[row][c0+k] -= tau w[row] conj(v[k]) on up to four matrices
struct RightMats {
  cplx* p[4];
  long long ld[4];
  int rows[4];
  int n;
};
__global__ void house_left2_kernel(cplx* __restrict__ A, long long lda, int c0a, int na, cplx* __restrict__ B,
                                   long long ldb, int nbc, int r0, int len, const cplx* __restrict__ v,
                                   const double* __restrict__ tau) {
  __shared__ cplx red[256];
  const bool inA = (int)blockIdx.x < na;
  cplx* a = inA ? A + (long long)(c0a + blockIdx.x) * lda + r0 : B + (long long)(blockIdx.x - na) * ldb + r0;
  (void)nbc;
  cplx sdot = cz();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const cplx vv = v[i], aa = a[i];
    sdot.x += vv.x * aa.x + vv.y * aa.y;
    sdot.y += vv.x * aa.y - vv.y * aa.x;
  }
  red[threadIdx.x] = sdot;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) { red[threadIdx.x].x += red[threadIdx.x + w].x; red[threadIdx.x].y += red[threadIdx.x + w].y; }
    __syncthreads();
  }
  const cplx wsum = red[0];
  const double t = *tau;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const cplx d = cuCmul(v[i], wsum);
    a[i].x -= t * d.x;
    a[i].y -= t * d.y;
  }
}
// w[k][row] = sum_j A_k[row][c0 + j] v[j] for every matrix k and row (w rows stacked, matrix k at woff[k])
// w[row] = sum_j A[row][c0 + j] v[j] over the rows of all right-side matrices: a block takes a tile of 32
// rows (lanes, coalesced along the column-major rows) and its 8 warps split the reflector's length, so
// that short and long reflectors alike keep many warps in flight; the warps' sums meet in shared memory
__global__ void __launch_bounds__(256) house_right_w4_kernel(RightMats m, int c0, int len, const cplx* __restrict__ v,
                                                             cplx* __restrict__ w) {
  __shared__ cplx red[8][32];
  int t = blockIdx.x, k = 0, off = 0;
  while (k < m.n) {   // tile t -> matrix k (tiles do not cross matrices)
    const int nt = (m.rows[k] + 31) / 32;
    if (t < nt) break;
    t -= nt;
    off += m.rows[k];
    ++k;
  }
  if (k >= m.n) return;   // uniform for the whole block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = t * 32 + lane;
  const bool ok = row < m.rows[k];
  const cplx* A = m.p[k];
  cplx sum = cz();
  if (ok)
    for (int j = wid; j < len; j += 8) sum = cuCadd(sum, cuCmul(A[(long long)(c0 + j) * m.ld[k] + row], v[j]));
  red[wid][lane] = sum;
  __syncthreads();
  if (wid == 0 && ok) {
    cplx r = red[0][lane];
    for (int q = 1; q < 8; ++q) r = cuCadd(r, red[q][lane]);
    w[off + row] = r;
  }
}
// A_k[row][c0 + j] -= tau w[k][row] conj(v[j])
__global__ void house_right_update4_kernel(RightMats m, int c0, int len, const cplx* __restrict__ v,
                                           const cplx* __restrict__ w, const double* __restrict__ tau, long long total) {
  const double t = *tau;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    int k = 0, off = 0;
    while (k < m.n && r >= (long long)m.rows[k] * len) { r -= (long long)m.rows[k] * len; off += m.rows[k]; ++k; }
    if (k >= m.n) return;
    const int row = (int)(r % m.rows[k]), j = (int)(r / m.rows[k]);
    const cplx d = cuCmul(w[off + row], cuConj(v[j]));
    cplx* p = m.p[k] + (long long)(c0 + j) * m.ld[k] + row;
    p->x -= t * d.x;
    p->y -= t * d.y;
  }
}

// Y[r0 + i][n] -= tau v[i] sum_k conj(v[k]) Y[r0 + k][n] for every column n < N (Y row-major, ld ldy)
__global__ void house_rows_kernel(cplx* __restrict__ Y, long long ldy, long long N, int r0, int len,
                                  const cplx* __restrict__ v, const double* __restrict__ tau) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  cplx sdot = cz();
  for (int k = 0; k < len; ++k) {
    const cplx vv = v[k], yy = Y[(long long)(r0 + k) * ldy + n];
    sdot.x += vv.x * yy.x + vv.y * yy.y;
    sdot.y += vv.x * yy.y - vv.y * yy.x;
  }
  const double t = *tau;
  for (int k = 0; k < len; ++k) {
    const cplx d = cuCmul(v[k], sdot);
    Y[(long long)(r0 + k) * ldy + n].x -= t * d.x;
    Y[(long long)(r0 + k) * ldy + n].y -= t * d.y;
  }
}

// ---- per-frequency shifted Hessenberg solve --------------------------------------------------------
struct EvalArgs {
  int m, np, nw;
  const cplx* H;      // m x m col-major (ld m), upper Hessenberg
  const cplx* bw;     // m x np col-major (ld m)
  const double* omegas;
  double eta;
  cplx* scratch;      // per CTA: U (m(m+1)/2) | rows (2m)
  long long scratch_per_cta;
  cplx* Y;            // solutions: Y[k * ldy + w * np + p] = yhat_p(w)[k]
  long long ldy;
  int* singular;
  int rhs_in_Y = 0;   // 1: the right-hand sides are already in Y (per frequency), solved in place
};

__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }

// ---- double-float arithmetic (value = h + l, two FP32 numbers) ------------------------------------
// GB300 issues FP32 operations at many times its FP64 rate, so the O(m^2 np) back substitution runs
// on pairs of floats (about 48 significant bits; Dekker 1971, Knuth's two-sum). The explicitly
// rounded intrinsics keep the compiler from contracting the error-free transformations.
struct df2 {
  float h, l;
};
__device__ __forceinline__ df2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(float h, float l) { return (double)h + (double)l; }
// c + a1 b1 + a2 b2 (all double-float): the leading products exactly (fma), the rest in FP32
__device__ __forceinline__ df2 df_dot2(df2 c, df2 a1, df2 b1, df2 a2, df2 b2) {
  const float p1 = __fmul_rn(a1.h, b1.h), p2 = __fmul_rn(a2.h, b2.h);
  const float e1 = __fmaf_rn(a1.h, b1.h, -p1), e2 = __fmaf_rn(a2.h, b2.h, -p2);
  float cross = __fmul_rn(a2.l, b2.h);
  cross = __fmaf_rn(a2.h, b2.l, cross);
  cross = __fmaf_rn(a1.l, b1.h, cross);
  cross = __fmaf_rn(a1.h, b1.l, cross);
  const df2 s1 = two_sum(c.h, p1);
  const df2 s2 = two_sum(s1.h, p2);
  float low = __fadd_rn(c.l, e1);
  low = __fadd_rn(low, e2);
  low = __fadd_rn(low, cross);
  low = __fadd_rn(low, s1.l);
  low = __fadd_rn(low, s2.l);
  return fast_two_sum(s2.h, low);
}
// complex double-float in a float4 (re.h, re.l, im.h, im.l)
__device__ __forceinline__ float4 dfc_from(cplx z) {
  const df2 r = df_from(z.x), i = df_from(z.y);
  return make_float4(r.h, r.l, i.h, i.l);
}
__device__ __forceinline__ cplx dfc_to(float4 v) { return make_cuDoubleComplex(df_to(v.x, v.y), df_to(v.z, v.w)); }
// c - u y
__device__ __forceinline__ float4 dfc_sub_mul(float4 c, float4 u, float4 y) {
  const df2 cr{c.x, c.y}, ci{c.z, c.w};
  const df2 nur{-u.x, -u.y}, ui{u.z, u.w}, nui{-u.z, -u.w};
  const df2 yr{y.x, y.y}, yi{y.z, y.w};
  const df2 r = df_dot2(cr, nur, yr, ui, yi);     // cr - ur yr + ui yi
  const df2 i = df_dot2(ci, nur, yi, nui, yr);    // ci - ur yi - ui yr
  return make_float4(r.h, r.l, i.h, i.l);
}

// One CTA per frequency (grid-stride): LU of (w - i eta + H) with partial pivoting between adjacent
// rows (the only pivots a Hessenberg matrix needs), applied to the np right-hand sides, in FP64 (O(m^2
// + m np) work); then the back substitution (O(m^2 np)) in double-float, P right-hand sides at a time
// held in shared memory, with U stored column by column. Everything after the solves (Ghat, A,
// residual norms) is a GEMM over all frequencies at once and runs outside this kernel.
// Scratch per CTA (16-byte units): U (m(m+1)/2, double-float, column j at j(j+1)/2) | two FP64 rows
// (2m) | the FP64 diagonal of U (m). Dynamic shared memory: m P double-float complex values.
template <int P>
__global__ void __launch_bounds__(256) eval_solve_kernel(EvalArgs a) {
  static_assert(256 % P == 0, "P divides the block");
  extern __shared__ float4 Rs[];   // [m][P]
  const int m = a.m, np = a.np;
  float4* Ud = reinterpret_cast<float4*>(a.scratch + blockIdx.x * a.scratch_per_cta);
  cplx* rowA = reinterpret_cast<cplx*>(Ud + (long long)m * (m + 1) / 2);
  cplx* rowB = rowA + m;
  cplx* dU = rowB + m;
  const long long ldr = a.ldy;
  __shared__ int s_swap;
  __shared__ cplx s_l;
  for (int w = blockIdx.x; w < a.nw; w += gridDim.x) {
    const cplx sig = make_cuDoubleComplex(a.omegas[w], -a.eta);
    cplx* R = a.Y + (long long)w * np;   // R[k * ldr + p]
    if (!a.rhs_in_Y) {
      for (long long t = threadIdx.x; t < (long long)m * np; t += blockDim.x) {
        int k = (int)(t / np), p = (int)(t % np);
        R[k * ldr + p] = a.bw[k + (long long)p * m];
      }
    }
    for (int col = threadIdx.x; col < m; col += blockDim.x) {
      cplx h = a.H[(long long)col * m + 0];
      if (col == 0) h = cuCadd(h, sig);
      rowA[col] = h;
    }
    __syncthreads();
    cplx* cur = rowA;
    cplx* nxt = rowB;
    for (int j = 0; j < m; ++j) {
      if (j + 1 < m) {
        for (int col = j + threadIdx.x; col < m; col += blockDim.x) {
          cplx h = a.H[(long long)col * m + (j + 1)];
          if (col == j + 1) h = cuCadd(h, sig);
          nxt[col] = h;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_swap = (j + 1 < m && cabs2(nxt[j]) > cabs2(cur[j])) ? 1 : 0;
      }
      __syncthreads();
      if (s_swap) {
        cplx* tmp = cur; cur = nxt; nxt = tmp;
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
          cplx t0 = R[j * ldr + p];
          R[j * ldr + p] = R[(j + 1) * ldr + p];
          R[(j + 1) * ldr + p] = t0;
        }
      }
      __syncthreads();
      // row j of U: U(j, col) at column col's offset col(col+1)/2 + j
      for (int col = j + threadIdx.x; col < m; col += blockDim.x)
        Ud[(long long)col * (col + 1) / 2 + j] = dfc_from(cur[col]);
      if (threadIdx.x == 0) dU[j] = cur[j];
      if (j + 1 < m) {
        if (threadIdx.x == 0) {
          cplx piv = cur[j];
          if (piv.x == 0.0 && piv.y == 0.0) { atomicExch(a.singular, 1); s_l = cz(); }
          else s_l = cuCdiv(nxt[j], piv);
        }
        __syncthreads();
        const cplx l = s_l;
        for (int col = j + 1 + threadIdx.x; col < m; col += blockDim.x) nxt[col] = cuCsub(nxt[col], cuCmul(l, cur[col]));
        for (int p = threadIdx.x; p < np; p += blockDim.x)
          R[(j + 1) * ldr + p] = cuCsub(R[(j + 1) * ldr + p], cuCmul(l, R[j * ldr + p]));
        __syncthreads();
        cplx* tmp = cur; cur = nxt; nxt = tmp;
      }
    }
    __syncthreads();
    // back substitution, column oriented, P right-hand sides at a time: y_j = R_j / U_jj (FP64);
    // R_i -= U_ij y_j for i < j (double-float)
    const int p = threadIdx.x % P, i0 = threadIdx.x / P;
    constexpr int ISTEP = 256 / P;
    for (int pc0 = 0; pc0 < np; pc0 += P) {
      const int pn = min(P, np - pc0);
      for (int t = threadIdx.x; t < m * P; t += blockDim.x) {
        const int i = t / P, pp = t % P;
        Rs[t] = pp < pn ? dfc_from(R[i * ldr + pc0 + pp]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      for (int j = m - 1; j >= 0; --j) {
        if (threadIdx.x < pn) {
          const cplx d = dU[j];
          const cplx y = (d.x == 0.0 && d.y == 0.0) ? cz() : cuCdiv(dfc_to(Rs[j * P + threadIdx.x]), d);
          Rs[j * P + threadIdx.x] = dfc_from(y);
        }
        __syncthreads();
        if (p < pn) {
          const float4 yj = Rs[j * P + p];
          const float4* Uc = Ud + (long long)j * (j + 1) / 2;
          for (int i = i0; i < j; i += ISTEP) Rs[i * P + p] = dfc_sub_mul(Rs[i * P + p], Uc[i], yj);
        }
        __syncthreads();
      }
      for (int t = threadIdx.x; t < m * P; t += blockDim.x) {
        const int i = t / P, pp = t % P;
        if (pp < pn) R[i * ldr + pc0 + pp] = dfc_to(Rs[t]);
      }
      __syncthreads();
    }
  }
}

// scratch per CTA of eval_solve_kernel (16-byte units)
long long eval_scratch_per_cta(int m) { return (long long)m * (m + 1) / 2 + 3LL * m + 64; }

// CTAs per SM of the evaluation solves: the steps of one solve are a chain of barriers and memory
// round trips, so several solves share each SM
constexpr int EVAL_CTAS_PER_SM = 4;
// launch with the widest right-hand-side chunk whose double-float block lets EVAL_CTAS_PER_SM CTAs
// share an SM (narrower chunks, down to one column, for large models)
void launch_eval_solve(const EvalArgs& ea, int grid, cudaStream_t s) {
  const size_t cap = std::max<size_t>(200 * 1024 / EVAL_CTAS_PER_SM, sizeof(float4) * (size_t)ea.m);
  GFCC_CHECK(cap <= 200 * 1024, GFCC_ERR_ARG, "reduced model too large for the evaluation kernel");
  auto go = [&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    const size_t bytes = sizeof(float4) * (size_t)ea.m * P;
    static bool attr[64] = {};   // per instantiation, once per device (attributes live in each context)
    int dev = 0;
    GFCC_CUDA(cudaGetDevice(&dev));
    GFCC_CHECK(dev >= 0 && dev < 64, GFCC_ERR_ARG, "device ordinal above 63");
    if (!attr[dev]) {
      GFCC_CUDA(cudaFuncSetAttribute(eval_solve_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr[dev] = true;
    }
    eval_solve_kernel<P><<<grid, 256, bytes, s>>>(ea);
  };
  const size_t row = sizeof(float4) * (size_t)ea.m;
  if (row * 16 <= cap) go(std::integral_constant<int, 16>{});
  else if (row * 8 <= cap) go(std::integral_constant<int, 8>{});
  else if (row * 4 <= cap) go(std::integral_constant<int, 4>{});
  else if (row * 2 <= cap) go(std::integral_constant<int, 2>{});
  else go(std::integral_constant<int, 1>{});
  GFCC_LAUNCH_CHECK();
}

// A[w] = -(1/pi) sum_p Im G[w][p][qidx[p]] (p with a matching q only)
__global__ void spectral_from_G_kernel(const cplx* __restrict__ G, int nw, int np, int nq, const int* __restrict__ qidx,
                                       double* __restrict__ A) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double acc = 0.0;
  for (int p = 0; p < np; ++p) {
    const int qi = qidx[p];
    if (qi >= 0) acc += G[((long long)w * np + p) * nq + qi].y;
  }
  A[w] = -acc / 3.14159265358979323846;
}

// Ys[k][w np + p] = (w - i eta) Y[k][w np + p]
__global__ void shift_scale_kernel(const cplx* __restrict__ Y, long long ldy, int m, int np, int nw,
                                   const double* __restrict__ omegas, double eta, cplx* __restrict__ Ys) {
  const long long total = (long long)m * nw * np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t / ((long long)nw * np), n = t % ((long long)nw * np);
    const int w = (int)(n / np);
    Ys[k * ldy + n] = cuCmul(make_cuDoubleComplex(omegas[w], -eta), Y[k * ldy + n]);
  }
}

// res[w np + p] = || C[:, w np + p] - RB[:, p] || / bn[p]   (C row-major [qn][ldc])
__global__ void resnorm_kernel(const cplx* __restrict__ C, long long ldc, int qn, const cplx* __restrict__ RB,
                               int np, int nw, const double* __restrict__ bn, double* __restrict__ res) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= (long long)nw * np) return;
  const int p = (int)(n % np);
  double s = 0.0;
  for (int r = 0; r < qn; ++r) {
    const cplx d = cuCsub(C[(long long)r * ldc + n], RB[r + (long long)p * qn]);
    s += d.x * d.x + d.y * d.y;
  }
  res[n] = sqrt(s) / bn[p];
}
__global__ void rowmax_kernel(const double* __restrict__ res, int np, int nw, double* __restrict__ out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double mx = 0.0;
  for (int p = 0; p < np; ++p) mx = fmax(mx, res[(long long)w * np + p]);
  out[w] = mx;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
namespace {

// reallocate a batch-minor [rows][old_cap] block as [rows][new_cap] keeping ncols columns
void regrow_rows(DBuf<cplx>& b, long long rows, int old_cap, int new_cap, int ncols, cudaStream_t s) {
  DBuf<cplx> nb2;
  nb2.alloc(rows * new_cap);
  nb2.zero(s);
  if (ncols > 0)
    GFCC_CUDA(cudaMemcpy2DAsync(nb2.p, sizeof(cplx) * new_cap, b.p, sizeof(cplx) * old_cap, sizeof(cplx) * ncols, rows,
                                cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  std::swap(b.p, nb2.p);
  std::swap(b.n, nb2.n);
}
// reallocate a col-major [old_ld x ...] matrix as [new_ld x alloc_cols] keeping nrows x ncols
void regrow_cm(DBuf<cplx>& b, int old_ld, int new_ld, int alloc_cols, int nrows, int ncols, cudaStream_t s) {
  DBuf<cplx> nb2;
  nb2.alloc((long long)new_ld * std::max(alloc_cols, 1));
  nb2.zero(s);
  if (nrows > 0 && ncols > 0)
    GFCC_CUDA(cudaMemcpy2DAsync(nb2.p, sizeof(cplx) * new_ld, b.p, sizeof(cplx) * old_ld, sizeof(cplx) * nrows, ncols,
                                cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  std::swap(b.p, nb2.p);
  std::swap(b.n, nb2.n);
}

// FP64 arithmetic runs on a narrow pipe on this GPU: every product of the orthonormalisation above a
// small size goes to the exact-slice tensor-core GEMM (7 slices, 48 bits per row). Fewer slices are
// not enough: the residual basis resolves the solver-residual directions of Z = M S, about 1e-8 of
// the columns' norms, and 41-bit products perturb them enough to spoil the refinement estimates.
// The coefficients of the first Gram-Schmidt pass are the exception (ns = 5, 34 bits): the reconstruction
// y = Q (C1 + C2) + y'' holds for whatever C1 the first update subtracts, and the second pass, whose
// coefficients and both updates keep 7 slices, removes what a less accurate C1 leaves along Q. The
// second-pass and panel Gram products need the 7 slices even for the residual basis: with 5 the
// refinement no longer converged (the model grew to the size limit).
void fp64_accurate_zgemm(const ZGemmDesc& g, cudaStream_t s, int ns = 7) {
  if ((double)g.M * (double)g.N * (double)g.K >= (double)(1 << 22) && g.batch == 1) zgemm_oz(g, ns, s);
  else zgemm(g, s);
}

// ---- panel kernels: column-wise CGS2 inside a panel of at most PB columns -----------------------
constexpr int PB = 32;            // panel width (one lane per panel column)
constexpr int PTY = 8;            // warps per block, each sweeping its own rows

// out[c] (partial[chunk][c]) = sum_{nu in chunk} |Y[nu][c]|^2 for c < nc; block (32, PTY)
__global__ void colnorms_partial_kernel(const cplx* __restrict__ Y, int nc, long long D, long long rows,
                                        double* __restrict__ partial) {
  __shared__ double red[PTY][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const long long r0 = blockIdx.y * rows, r1 = min(D, r0 + rows);
  double acc = 0.0;
  if (c < nc)
    for (long long nu = r0 + threadIdx.y; nu < r1; nu += PTY) {
      const cplx a = Y[nu * nc + c];
      acc += a.x * a.x + a.y * a.y;
    }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && c < nc) {
    double t = 0.0;
    for (int k = 0; k < PTY; ++k) t += red[k][threadIdx.x];
    partial[(long long)blockIdx.y * nc + c] = t;
  }
}
__global__ void colnorms_reduce_kernel(const double* __restrict__ partial, int nchunk, int nc, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double t = 0.0;
  for (int k = 0; k < nchunk; ++k) t += partial[(long long)k * nc + c];
  out[c] = sqrt(t);
}

// partial[chunk][i] = sum_{nu in chunk} conj(Y[nu][c0 + i]) Y[nu][j] for i < n (n < PB); block (32, PTY)
__global__ void pdot_kernel(const cplx* __restrict__ Y, int nc, long long D, int c0, int n, int j, long long rows,
                            cplx* __restrict__ partial) {
  __shared__ cplx red[PTY][32];
  const int i = threadIdx.x;
  const long long r0 = blockIdx.y * rows, r1 = min(D, r0 + rows);
  cplx acc = cz();
  if (i < n)
#pragma unroll 4
    for (long long nu = r0 + threadIdx.y; nu < r1; nu += PTY) {
      const cplx a = Y[nu * nc + c0 + i], b = Y[nu * nc + j];
      acc.x += a.x * b.x + a.y * b.y;
      acc.y += a.x * b.y - a.y * b.x;
    }
  red[threadIdx.y][i] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    cplx t = cz();
    for (int k = 0; k < PTY; ++k) { t.x += red[k][i].x; t.y += red[k][i].y; }
    partial[(long long)blockIdx.y * PB + i] = t;
  }
}
// h[i] = sum_chunk partial[chunk][i]; T[c0 + i][j] += h[i] (T col-major, ld ldt) when T is non-null
// (block (32, PTY))
__global__ void preduce_kernel(const cplx* __restrict__ partial, int nchunk, int n, cplx* __restrict__ h,
                               cplx* __restrict__ T, int ldt, int c0, int j) {
  __shared__ cplx red[PTY][32];
  const int i = threadIdx.x;
  cplx t = cz();
  if (i < n)
    for (int k = threadIdx.y; k < nchunk; k += PTY) {
      t.x += partial[(long long)k * PB + i].x;
      t.y += partial[(long long)k * PB + i].y;
    }
  red[threadIdx.y][i] = t;
  __syncthreads();
  if (threadIdx.y == 0 && i < n) {
    for (int k = 1; k < PTY; ++k) { t.x += red[k][i].x; t.y += red[k][i].y; }
    h[i] = t;
    if (T) { T[c0 + i + (long long)j * ldt].x += t.x; T[c0 + i + (long long)j * ldt].y += t.y; }
  }
}
// Y[nu][j] -= sum_{i<n} Y[nu][c0 + i] h[i] (and MY alike); then, for mode 0, the partial dot products
// of the updated column with the panel columns (as pdot_kernel) or, for mode 1, partial[chunk][0].x =
// sum |Y[nu][j]|^2. Lane i holds panel column c0 + i; each warp takes PU rows per step (independent
// shuffle reductions in flight), block (32, PTY).
constexpr int PU = 4;
__global__ void pupdate_kernel(cplx* __restrict__ Y, cplx* __restrict__ MY, int nc, long long D, int c0, int n,
                               int j, long long rows, const cplx* __restrict__ h, int mode,
                               cplx* __restrict__ partial) {
  __shared__ cplx red[PTY][32];
  const int i = threadIdx.x;
  const long long r0 = blockIdx.y * rows, r1 = min(D, r0 + rows);
  const cplx hi = i < n ? h[i] : cz();
  cplx acc = cz();
  for (long long base = r0 + (long long)threadIdx.y * PU; base < r1; base += (long long)PTY * PU) {
    cplx a[PU], y[PU];
    double sx[PU], sy[PU];
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      const long long nu = base + u;
      const bool in = nu < r1;
      a[u] = (in && i < n) ? Y[nu * nc + c0 + i] : cz();
      y[u] = in ? Y[nu * nc + j] : cz();   // read by every lane before lane 0 writes it (the shuffles order them)
      sx[u] = a[u].x * hi.x - a[u].y * hi.y;
      sy[u] = a[u].x * hi.y + a[u].y * hi.x;
    }
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        sx[u] += __shfl_xor_sync(0xffffffffu, sx[u], off);
        sy[u] += __shfl_xor_sync(0xffffffffu, sy[u], off);
      }
    }
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      y[u].x -= sx[u];
      y[u].y -= sy[u];
      if (i == 0 && base + u < r1) Y[(base + u) * nc + j] = y[u];
    }
    if (MY) {
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        const long long nu = base + u;
        const cplx b = (nu < r1 && i < n) ? MY[nu * nc + c0 + i] : cz();
        sx[u] = b.x * hi.x - b.y * hi.y;
        sy[u] = b.x * hi.y + b.y * hi.x;
      }
      for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          sx[u] += __shfl_xor_sync(0xffffffffu, sx[u], off);
          sy[u] += __shfl_xor_sync(0xffffffffu, sy[u], off);
        }
      }
      if (i == 0) {
#pragma unroll
        for (int u = 0; u < PU; ++u)
          if (base + u < r1) { MY[(base + u) * nc + j].x -= sx[u]; MY[(base + u) * nc + j].y -= sy[u]; }
      }
    }
#pragma unroll
    for (int u = 0; u < PU; ++u) {
      if (mode == 0) {
        acc.x += a[u].x * y[u].x + a[u].y * y[u].y;
        acc.y += a[u].x * y[u].y - a[u].y * y[u].x;
      } else if (i == 0) {
        acc.x += y[u].x * y[u].x + y[u].y * y[u].y;
      }
    }
  }
  red[threadIdx.y][i] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && (mode == 0 ? i < n : i == 0)) {
    cplx t = cz();
    for (int k = 0; k < PTY; ++k) { t.x += red[k][i].x; t.y += red[k][i].y; }
    partial[(long long)blockIdx.y * PB + i] = t;
  }
}
// n1 = sqrt(sum_chunk partial[chunk][0].x); keep column j when n0[j] > 0 and n1 >= drop_tol n0[j];
// scale[j] = keep ? 1 / n1 : 0; T[j][j] = n1 when kept
__global__ void pfinish_kernel(const cplx* __restrict__ partial, int nchunk, const double* __restrict__ n0, int j,
                               double drop_tol, double* __restrict__ scale, int* __restrict__ keep,
                               cplx* __restrict__ T, int ldt) {
  __shared__ double red[256];
  double t = 0.0;
  for (int k = threadIdx.x; k < nchunk; k += blockDim.x) t += partial[(long long)k * PB].x;
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double n1 = sqrt(red[0]);
    const bool k = n0[j] > 0.0 && n1 >= drop_tol * n0[j];
    scale[j] = k ? 1.0 / n1 : 0.0;
    keep[j] = k ? 1 : 0;
    if (T && k) T[j + (long long)j * ldt] = make_cuDoubleComplex(n1, 0.0);
  }
}
__global__ void pscale_kernel(cplx* __restrict__ Y, cplx* __restrict__ MY, int nc, long long D, int j,
                              const double* __restrict__ scale) {
  const double sc = scale[j];
  for (long long nu = blockIdx.x * (long long)blockDim.x + threadIdx.x; nu < D; nu += (long long)gridDim.x * blockDim.x) {
    Y[nu * nc + j].x *= sc; Y[nu * nc + j].y *= sc;
    if (MY) { MY[nu * nc + j].x *= sc; MY[nu * nc + j].y *= sc; }
  }
}
// T[i][c0 + j] += Cf[i][j] for i < rows, j < pb (Cf row-major [rows][pb], T col-major ld ldt)
__global__ void add_block_kernel(cplx* __restrict__ T, int ldt, int c0, const cplx* __restrict__ Cf, int rows, int pb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * pb) return;
  const int i = t / pb, j = t % pb;
  T[i + (long long)(c0 + j) * ldt].x += Cf[t].x;
  T[i + (long long)(c0 + j) * ldt].y += Cf[t].y;
}

// Complex Cholesky G = R^H R of a Hermitian positive definite n x n matrix (row-major); returns false
// when a pivot is not positive.
bool cholesky_upper(const std::vector<cplx>& G, int n, std::vector<cplx>& R) {
  R.assign((size_t)n * n, make_cuDoubleComplex(0.0, 0.0));
  for (int j = 0; j < n; ++j) {
    double d = G[(size_t)j * n + j].x;
    for (int i = 0; i < j; ++i) d -= R[(size_t)i * n + j].x * R[(size_t)i * n + j].x + R[(size_t)i * n + j].y * R[(size_t)i * n + j].y;
    if (!(d > 0.0)) return false;
    const double rjj = std::sqrt(d);
    R[(size_t)j * n + j] = make_cuDoubleComplex(rjj, 0.0);
    for (int k = j + 1; k < n; ++k) {
      cplx t = G[(size_t)j * n + k];
      for (int i = 0; i < j; ++i) t = cuCsub(t, cuCmul(cuConj(R[(size_t)i * n + j]), R[(size_t)i * n + k]));
      R[(size_t)j * n + k] = make_cuDoubleComplex(t.x / rjj, t.y / rjj);
    }
  }
  return true;
}
// inverse of an upper triangular n x n matrix (row-major)
std::vector<cplx> inverse_upper(const std::vector<cplx>& R, int n) {
  std::vector<cplx> X((size_t)n * n, make_cuDoubleComplex(0.0, 0.0));
  for (int j = n - 1; j >= 0; --j) {
    X[(size_t)j * n + j] = cuCdiv(make_cuDoubleComplex(1.0, 0.0), R[(size_t)j * n + j]);
    for (int k = j + 1; k < n; ++k) {
      cplx t = make_cuDoubleComplex(0.0, 0.0);
      for (int i = j + 1; i <= k; ++i) t = cuCadd(t, cuCmul(R[(size_t)j * n + i], X[(size_t)i * n + k]));
      X[(size_t)j * n + k] = cuCmul(cuCsub(make_cuDoubleComplex(0.0, 0.0), t), X[(size_t)j * n + j]);
    }
  }
  return X;
}

// Panel of pb columns Y[:, c0:c0+pb] (already orthogonal to every earlier column): Cholesky QR twice
// (Y = Q R2 R1 with the Gram matrices formed by FP64-accurate GEMMs). In exact arithmetic this is the
// column-by-column Gram-Schmidt of the panel (the same Q and R with a positive diagonal). It is taken
// only when the panel is well conditioned: every first-pass pivot R1_jj at least 1e-5 of its column's
// norm (a bound on the conditioning of the column-scaled panel, which is what Cholesky QR's accuracy
// depends on) and at least 10 drop_tol of the column's norm before any projection (n0), so that two
// passes give orthonormality to rounding and no column is within a factor 10 of the drop threshold;
// otherwise the caller runs the column-by-column passes. Writes T[c0:c0+pb, c0:c0+pb] = R2 R1 and keep = 1.
// Z[nu][j] <- sum_{k <= j} Z[nu][k] X[k][j] for the pb (<= 32) columns of a panel: X upper
// triangular, double-float, row-major pb x pb. One warp per row, in place; each lane forms one output
// column in double-float (the row's entries are split once by their own lanes and broadcast).
__global__ void __launch_bounds__(256) panel_apply_kernel(cplx* __restrict__ Z, int nc, int pb, long long D,
                                                          const float4* __restrict__ Xdf) {
  __shared__ float4 xs[32 * 32];
  for (int t = threadIdx.x; t < pb * pb; t += blockDim.x) xs[t] = Xdf[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long nu = blockIdx.x * 8LL + warp; nu < D; nu += gridDim.x * 8LL) {
    cplx* row = Z + nu * nc;
    const float4 zk = lane < pb ? dfc_from(row[lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
    df2 ar{0.f, 0.f}, ai{0.f, 0.f};
    for (int k = 0; k < pb; ++k) {
      const float zrh = __shfl_sync(0xffffffffu, zk.x, k), zrl = __shfl_sync(0xffffffffu, zk.y, k);
      const float zih = __shfl_sync(0xffffffffu, zk.z, k), zil = __shfl_sync(0xffffffffu, zk.w, k);
      if (lane >= k && lane < pb) {
        const float4 x = xs[k * pb + lane];
        const df2 zr{zrh, zrl}, zi{zih, zil}, nzi{-zih, -zil}, xr{x.x, x.y}, xi{x.z, x.w};
        ar = df_dot2(ar, zr, xr, nzi, xi);   // re += zr xr - zi xi
        ai = df_dot2(ai, zr, xi, zi, xr);    // im += zr xi + zi xr
      }
    }
    if (lane < pb) row[lane] = make_cuDoubleComplex(df_to(ar.h, ar.l), df_to(ai.h, ai.l));
  }
}

struct PanelWork {
  DBuf<cplx> Gd;
  DBuf<float4> Rdf;
};
bool panel_cholqr2(gfcc_ctx* c, cplx* Y, cplx* MY, int nc, long long D, int c0, int pb, const double* n0,
                   cplx* T, int* keep_dev, PanelWork& pw) {
  cudaStream_t s = c->stream;
  std::vector<cplx> G((size_t)pb * pb), R1, R2;
  DBuf<cplx>& Gd = pw.Gd;
  DBuf<float4>& Rdf = pw.Rdf;
  Gd.alloc((long long)pb * pb);
  Rdf.alloc((long long)pb * pb);
  auto gram = [&]() {
    ZGemmDesc g;
    g.M = pb; g.N = pb; g.K = (int)D;
    g.A = Y + c0; g.sam = 1; g.sak = nc; g.conjA = true;
    g.B = Y + c0; g.sbk = nc; g.sbn = 1;
    g.C = Gd.p; g.scm = pb; g.scn = 1;
    g.work = zgemm_work(c);
    fp64_accurate_zgemm(g, s);
    GFCC_CUDA(cudaMemcpyAsync(G.data(), Gd.p, sizeof(cplx) * pb * pb, cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < pb; ++i) {   // exact Hermitian symmetry and a real diagonal
      G[(size_t)i * pb + i].y = 0.0;
      for (int k = i + 1; k < pb; ++k) G[(size_t)k * pb + i] = cuConj(G[(size_t)i * pb + k]);
    }
  };
  auto apply = [&](const std::vector<cplx>& R) {   // Y (and MY) <- Y R^{-1}, in double-float
    GFCC_CHECK(pb <= 32, GFCC_ERR_ARG, "panel wider than a warp");
    std::vector<cplx> X = inverse_upper(R, pb);
    std::vector<float4> Xf((size_t)pb * pb);
    for (size_t t = 0; t < Xf.size(); ++t) {   // the same split as on the device: h = fl(x), l = fl(x - h)
      const float rh = (float)X[t].x, ih = (float)X[t].y;
      Xf[t] = make_float4(rh, (float)(X[t].x - (double)rh), ih, (float)(X[t].y - (double)ih));
    }
    GFCC_CUDA(cudaMemcpyAsync(Rdf.p, Xf.data(), sizeof(float4) * pb * pb, cudaMemcpyHostToDevice, s));
    const int grid = (int)std::min<long long>((D + 7) / 8, 152LL * 16);
    for (cplx* Z : {Y, MY}) {
      if (!Z) continue;
      panel_apply_kernel<<<grid, 256, 0, s>>>(Z + c0, nc, pb, D, Rdf.p);
      GFCC_LAUNCH_CHECK();
    }
    GFCC_CUDA(cudaStreamSynchronize(s));   // Xf is host memory of this scope
  };
  gram();
  if (!cholesky_upper(G, pb, R1)) return false;
  for (int j = 0; j < pb; ++j) {   // pivot relative to the column's own norm (scale-invariant test)
    const double r = R1[(size_t)j * pb + j].x;
    if (!(r >= 1e-5 * std::sqrt(G[(size_t)j * pb + j].x)) || !(r >= 10.0 * c->opts.drop_tol * n0[j])) return false;
  }
  apply(R1);
  gram();
  if (!cholesky_upper(G, pb, R2)) return false;   // cannot happen after a well-conditioned first pass
  apply(R2);
  if (T) {   // T block = R2 R1 (upper triangular), column-major in T (ld nc)
    std::vector<cplx> Tb((size_t)pb * pb, make_cuDoubleComplex(0.0, 0.0));
    for (int i = 0; i < pb; ++i)
      for (int k = i; k < pb; ++k) {
        cplx t = make_cuDoubleComplex(0.0, 0.0);
        for (int l = i; l <= k; ++l) t = cuCadd(t, cuCmul(R2[(size_t)i * pb + l], R1[(size_t)l * pb + k]));
        Tb[(size_t)k * pb + i] = t;   // column k, row i
      }
    GFCC_CUDA(cudaMemcpy2DAsync(T + c0 + (long long)c0 * nc, sizeof(cplx) * nc, Tb.data(), sizeof(cplx) * pb,
                                sizeof(cplx) * pb, pb, cudaMemcpyHostToDevice, s));
  }
  std::vector<int> ones(pb, 1);
  GFCC_CUDA(cudaMemcpyAsync(keep_dev + c0, ones.data(), sizeof(int) * pb, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  return true;
}

// Orthonormalise the nc columns of Y ([D][nc] batch-minor) against the n_cur columns of the basis
// Bs ([D][cap]) and against each other, column by column in order: each column loses its components
// along all earlier columns by classical Gram-Schmidt applied twice, and is kept when its norm after
// that is >= drop_tol times its norm before, else zeroed. The same linear operations are applied to
// MY when it is non-null (MBs being the matching block of Bs). Cold (device, n_cur x nc col-major,
// ld n_cur) and T (device, nc x nc col-major) receive the coefficients
// y_j = Bs Cold[:, j] + sum_i T[i, j] ynew_i when the pointers are non-null. Returns the kept columns.
//
// Blocking (the same projections in exact arithmetic, since the subspaces are mutually orthogonal):
// two passes of block CGS against Bs; then panels of PB columns, each projected twice against the
// finished earlier panels by two GEMMs per pass, and finally column by column inside the panel, whose
// PB columns stay resident in L2. The keep decisions are taken on the device.
std::vector<int> ortho_block(gfcc_ctx* c, const cplx* Bs, int cap, int n_cur, cplx* Y, cplx* MY, const cplx* MBs,
                             int nc, cplx* Cold, cplx* T) {
  if (nc <= 0) return {};
  cudaStream_t s = c->stream;
  const long long D = c->D;
  // one chunk of rows per block: one wave of two PTY-warp blocks per SM (pupdate_kernel's registers)
  const long long rows = std::max<long long>(64, (D + 152 * 2 - 1) / (152 * 2));
  const int nchunk = (int)((D + rows - 1) / rows);
  DBuf<double> n0, scale, npart;
  DBuf<int> keep;
  n0.alloc(nc);
  scale.alloc(nc);
  keep.alloc(nc);
  npart.alloc((long long)nchunk * nc);
  colnorms_partial_kernel<<<dim3((nc + 31) / 32, nchunk), dim3(32, PTY), 0, s>>>(Y, nc, D, rows, npart.p);
  GFCC_LAUNCH_CHECK();
  colnorms_reduce_kernel<<<(nc + 127) / 128, 128, 0, s>>>(npart.p, nchunk, nc, n0.p);
  GFCC_LAUNCH_CHECK();
  if (T) GFCC_CUDA(cudaMemsetAsync(T, 0, sizeof(cplx) * nc * nc, s));
  DBuf<cplx> Cf;
  Cf.alloc((long long)std::max(std::max(n_cur, nc), 1) * std::max(nc, 1));
  auto block_cgs = [&](const cplx* Pb, int ldp, int np_, const cplx* MPb, int col0, int ncols, bool to_cold) {
    // two passes: Cf (row-major [np_][ncols]) = Pb^H Y[:, col0:col0+ncols]; Y[:, col0:...] -= Pb Cf.
    // Pb and MPb do not change between the passes: their slices as left operands of the updates are
    // made once.
    void* cache_p = zgemm_slice_cache(c, 0);
    void* cache_m = zgemm_slice_cache(c, 1);
    zgemm_slice_cache_reset(cache_p);
    zgemm_slice_cache_reset(cache_m);
    for (int pass = 0; pass < 2; ++pass) {
      ZGemmDesc g;
      g.M = np_; g.N = ncols; g.K = (int)D;
      g.A = Pb; g.sam = 1; g.sak = ldp; g.conjA = true;
      g.B = Y + col0; g.sbk = nc; g.sbn = 1;
      g.C = Cf.p; g.scm = ncols; g.scn = 1;
      g.work = zgemm_work(c);
      {
        ProfScope pg(PROF_ORTHO_GRAM, 0.0, s);
        fp64_accurate_zgemm(g, s, pass == 0 ? 5 : 7);
      }
      ZGemmDesc u;
      u.M = (int)D; u.N = ncols; u.K = np_;
      u.A = Pb; u.sam = ldp; u.sak = 1;
      u.B = Cf.p; u.sbk = ncols; u.sbn = 1;
      u.C = Y + col0; u.scm = nc; u.scn = 1;
      u.alpha = make_cuDoubleComplex(-1.0, 0.0); u.beta = make_cuDoubleComplex(1.0, 0.0);
      u.work = zgemm_work(c);
      u.a_cache = cache_p;
      {
        ProfScope pu(PROF_ORTHO_UPDATE, 0.0, s);
        fp64_accurate_zgemm(u, s);
        if (MY) { u.A = MPb; u.C = MY + col0; u.a_cache = cache_m; fp64_accurate_zgemm(u, s); }
      }
      if (to_cold) {
        if (Cold) {   // Cold (col-major, ld n_cur) += Cf (row-major [n_cur][nc])
          int dims[3] = {np_, ncols, 2};
          int pm[3] = {1, 0, 2};
          permute(reinterpret_cast<const double*>(Cf.p), dims, 3, pm, reinterpret_cast<double*>(Cold), 1.0, 1.0, s);
        }
      } else if (T) {
        add_block_kernel<<<(np_ * ncols + 255) / 256, 256, 0, s>>>(T, nc, col0, Cf.p, np_, ncols);
        GFCC_LAUNCH_CHECK();
      }
    }
  };
  if (n_cur > 0) {
    if (Cold) GFCC_CUDA(cudaMemsetAsync(Cold, 0, sizeof(cplx) * n_cur * nc, s));
    block_cgs(Bs, cap, n_cur, MBs, 0, nc, true);
  }
  DBuf<cplx> partial, h;
  partial.alloc((long long)nchunk * PB);
  h.alloc(PB);
  const dim3 pgrid(1, nchunk), pblock(32, PTY);
  PanelWork pwork;
  std::vector<double> hn0(nc);
  GFCC_CUDA(cudaMemcpyAsync(hn0.data(), n0.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  for (int c0 = 0; c0 < nc; c0 += PB) {
    const int pb = std::min(PB, nc - c0);
    if (c0 > 0) block_cgs(Y, nc, c0, MY, c0, pb, false);
    ProfScope pp(PROF_MOR_PANEL, 0.0, s);
    bool done;
    {
      ProfScope pq(PROF_ORTHO_CHOLQR, 0.0, s);
      done = panel_cholqr2(c, Y, MY, nc, D, c0, pb, hn0.data() + c0, T, keep.p, pwork);
    }
    if (done) continue;
    for (int j = c0; j < c0 + pb; ++j) {
      const int n = j - c0;
      if (n > 0) {
        pdot_kernel<<<pgrid, pblock, 0, s>>>(Y, nc, D, c0, n, j, rows, partial.p);
        GFCC_LAUNCH_CHECK();
        preduce_kernel<<<1, pblock, 0, s>>>(partial.p, nchunk, n, h.p, T, nc, c0, j);
        GFCC_LAUNCH_CHECK();
        pupdate_kernel<<<pgrid, pblock, 0, s>>>(Y, MY, nc, D, c0, n, j, rows, h.p, 0, partial.p);
        GFCC_LAUNCH_CHECK();
        preduce_kernel<<<1, pblock, 0, s>>>(partial.p, nchunk, n, h.p, T, nc, c0, j);
        GFCC_LAUNCH_CHECK();
      }
      pupdate_kernel<<<pgrid, pblock, 0, s>>>(Y, MY, nc, D, c0, n, j, rows, h.p, 1, partial.p);
      GFCC_LAUNCH_CHECK();
      pfinish_kernel<<<1, 256, 0, s>>>(partial.p, nchunk, n0.p, j, c->opts.drop_tol, scale.p, keep.p, T, nc);
      GFCC_LAUNCH_CHECK();
      pscale_kernel<<<grid_for(D), 256, 0, s>>>(Y, MY, nc, D, j, scale.p);
      GFCC_LAUNCH_CHECK();
    }
  }
  zgemm_work_check(c);
  std::vector<int> hk(nc);
  GFCC_CUDA(cudaMemcpyAsync(hk.data(), keep.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  std::vector<int> kept;
  for (int j = 0; j < nc; ++j)
    if (hk[j]) kept.push_back(j);
  return kept;
}

}  // namespace

// New column capacity of a model buffer that must hold `need` columns: doubling (few regrowths), unless the
// doubled buffers (bytes_per_col per column) would take more than half of the free device memory, in
// which case it grows to what is needed, rounded up to `quantum` (the old buffer is still held while the
// columns are copied, and large models at the biggest sizes are limited by memory, not by regrowths).
static int grown_capacity(gfcc_ctx* c, int cap_now, int need, int quantum, double bytes_per_col) {
  int cap = std::max(need, std::max(quantum, 2 * cap_now));
  size_t freeb = device_free_bytes();
  if (freeb == 0) return cap;
  if ((double)cap * bytes_per_col > 0.5 * (double)freeb) {
    // memory is short: give back the scratch buffers first (they regrow on demand), then size exactly
    release_scratch(c);
    freeb = device_free_bytes();
    if ((double)cap * bytes_per_col > 0.5 * (double)freeb)
      cap = std::max(need, ((need + quantum - 1) / quantum) * quantum);
  }
  return cap;
}

void release_scratch(gfcc_ctx* c) {
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  release_sigma_batch_buffers(c);
  c->ws.ut.release();
  c->ws.ct.release();
  c->ws.xe.release();
  c->ws.nb_cap = 0;
  zgemm_work_check(c);
  zgemm_work_free(c);
  GFCC_CUDA(cudaStreamSynchronize(c->stream));   // the frees have reached the pool before memory is measured
}

static void grow_model(gfcc_ctx* c, int need) {
  MorState& ms = c->mor;
  if (need <= ms.m_cap) return;
  const int np = (int)ms.porb.size(), nq = (int)ms.qorb.size();
  const int cap = grown_capacity(c, ms.m_cap, need, 64, 2.0 * (double)c->D * sizeof(cplx));   // S and Z
  cudaStream_t s = c->stream;
  regrow_rows(ms.S, c->D, ms.m_cap, cap, ms.m, s);
  regrow_rows(ms.Z, c->D, ms.m_cap, cap, ms.m, s);
  regrow_cm(ms.Hh, ms.m_cap, cap, cap, ms.m, ms.m, s);
  regrow_cm(ms.bh, ms.m_cap, cap, np, ms.m, np, s);
  regrow_cm(ms.ch, nq, nq, cap, nq, ms.m, s);
  regrow_cm(ms.RS, ms.q_cap, ms.q_cap, cap, ms.qn, ms.m, s);
  regrow_cm(ms.RZ, ms.q_cap, ms.q_cap, cap, ms.qn, ms.m, s);
  ms.m_cap = cap;
}

static void grow_basis(gfcc_ctx* c, int need) {
  MorState& ms = c->mor;
  if (need <= ms.q_cap) return;
  const int np = (int)ms.porb.size();
  const int cap = grown_capacity(c, ms.q_cap, need, 128, (double)c->D * sizeof(cplx));
  cudaStream_t s = c->stream;
  regrow_rows(ms.Q, c->D, ms.q_cap, cap, ms.qn, s);
  regrow_cm(ms.RS, ms.q_cap, cap, std::max(ms.m_cap, 1), ms.qn, ms.m, s);
  regrow_cm(ms.RZ, ms.q_cap, cap, std::max(ms.m_cap, 1), ms.qn, ms.m, s);
  regrow_cm(ms.RB, ms.q_cap, cap, np, ms.qn, np, s);
  ms.q_cap = cap;
}

// Append the kept columns of Ynew ([D][nc], destroyed) to Q and return, col-major [qn_new x nc], the
// coefficients of the ORIGINAL columns of Ynew in the enlarged basis (host memory).
static std::vector<cplx> basis_append(gfcc_ctx* c, cplx* Ynew, int nc) {
  MorState& ms = c->mor;
  cudaStream_t s = c->stream;
  ProfScope prof(PROF_MOR_BASIS, 0.0, s);
  const long long D = c->D;
  const int qn0 = ms.qn;
  DBuf<cplx> Cold, T;
  Cold.alloc((long long)std::max(qn0, 1) * nc);
  T.alloc((long long)nc * nc);
  std::vector<int> kept = ortho_block(c, ms.Q.p, ms.q_cap, qn0, Ynew, nullptr, nullptr, nc,
                                      qn0 > 0 ? Cold.p : nullptr, T.p);
  const int acc = (int)kept.size();
  grow_basis(c, qn0 + acc);
  if (acc > 0) {
    DBuf<int> dk;
    dk.alloc(acc);
    GFCC_CUDA(cudaMemcpyAsync(dk.p, kept.data(), sizeof(int) * acc, cudaMemcpyHostToDevice, s));
    append_cols_kernel<<<grid_for(D * acc), 256, 0, s>>>(Ynew, nc, dk.p, acc, ms.Q.p, ms.q_cap, qn0, D);
    GFCC_LAUNCH_CHECK();
    GFCC_CUDA(cudaStreamSynchronize(s));
  }
  const int qn1 = qn0 + acc;
  ms.qn = qn1;
  std::vector<cplx> hC((size_t)std::max(qn0, 1) * nc), hT((size_t)nc * nc);
  if (qn0 > 0) GFCC_CUDA(cudaMemcpyAsync(hC.data(), Cold.p, sizeof(cplx) * qn0 * nc, cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaMemcpyAsync(hT.data(), T.p, sizeof(cplx) * nc * nc, cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  std::vector<cplx> out((size_t)qn1 * nc, make_cuDoubleComplex(0.0, 0.0));
  for (int j = 0; j < nc; ++j) {
    for (int i = 0; i < qn0; ++i) out[(size_t)j * qn1 + i] = hC[(size_t)j * qn0 + i];
    for (int r = 0; r < acc; ++r) out[(size_t)j * qn1 + qn0 + r] = hT[(size_t)j * nc + kept[r]];
  }
  return out;
}

// write coefficient columns (host, col-major [rows x ncols]) into a device col-major matrix
static void put_cols(DBuf<cplx>& R, int ld, int col0, const std::vector<cplx>& h, int rows, int hcol0, int ncols,
                     cudaStream_t s) {
  if (ncols <= 0 || rows <= 0) return;
  GFCC_CUDA(cudaMemcpy2DAsync(R.p + (long long)col0 * ld, sizeof(cplx) * ld, h.data() + (size_t)hcol0 * rows,
                              sizeof(cplx) * rows, sizeof(cplx) * rows, ncols, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
}

void mor_init_basis(gfcc_ctx* c) {
  MorState& ms = c->mor;
  ++ms.version;
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int np = (int)ms.porb.size();
  DBuf<cplx> Bc;
  DBuf<int> rows;
  Bc.alloc(D * np);
  rows.alloc(np);
  GFCC_CUDA(cudaMemcpyAsync(rows.p, ms.porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
  gather_rows_real_to_cplx(c->bvec.p, (int)D, rows.p, np, (int)D, Bc.p, np, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
  std::vector<cplx> coef = basis_append(c, Bc.p, np);
  grow_basis(c, ms.qn);
  put_cols(ms.RB, ms.q_cap, 0, coef, ms.qn, 0, np, s);
}

void mor_append(gfcc_ctx* c, const cplx* Xin, const cplx* MXin, int nc) {
  MorState& ms = c->mor;
  ++ms.version;   // the model changes: its cached Hessenberg form is stale
  cudaStream_t s = c->stream;
  ProfScope prof(PROF_MOR_ORTHO, 0.0, s);
  const long long D = c->D;
  const int np = (int)ms.porb.size(), nq = (int)ms.qorb.size();
  if (nc == 0) return;
  DBuf<cplx> Y, MY;
  Y.alloc(D * nc);
  MY.alloc(D * nc);
  GFCC_CUDA(cudaMemcpyAsync(Y.p, Xin, sizeof(cplx) * D * nc, cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(MY.p, MXin, sizeof(cplx) * D * nc, cudaMemcpyDeviceToDevice, s));
  std::vector<int> kept = ortho_block(c, ms.S.p, ms.m_cap, ms.m, Y.p, MY.p, ms.Z.p, nc, nullptr, nullptr);
  const int acc = (int)kept.size();
  if (acc == 0) return;
  const int m0 = ms.m, m1 = ms.m + acc;
  grow_model(c, m1);
  const int cap = ms.m_cap;
  DBuf<cplx> SZ;   // [S_new | Z_new] for the residual basis
  SZ.alloc(D * 2 * acc);
  {
    DBuf<int> dk, di;
    dk.alloc(acc);
    di.alloc(acc);
    std::vector<int> iota(acc);
    for (int k = 0; k < acc; ++k) iota[k] = k;
    GFCC_CUDA(cudaMemcpyAsync(dk.p, kept.data(), sizeof(int) * acc, cudaMemcpyHostToDevice, s));
    append_cols_kernel<<<grid_for(D * acc), 256, 0, s>>>(Y.p, nc, dk.p, acc, ms.S.p, cap, m0, D);
    GFCC_LAUNCH_CHECK();
    append_cols_kernel<<<grid_for(D * acc), 256, 0, s>>>(MY.p, nc, dk.p, acc, ms.Z.p, cap, m0, D);
    GFCC_LAUNCH_CHECK();
    append_cols_kernel<<<grid_for(D * acc), 256, 0, s>>>(Y.p, nc, dk.p, acc, SZ.p, 2 * acc, 0, D);
    GFCC_LAUNCH_CHECK();
    append_cols_kernel<<<grid_for(D * acc), 256, 0, s>>>(MY.p, nc, dk.p, acc, SZ.p, 2 * acc, acc, D);
    GFCC_LAUNCH_CHECK();
    GFCC_CUDA(cudaStreamSynchronize(s));
  }
  auto proj = [&](const cplx* Lp, int l0, int nl, const cplx* Rp, int r0, int nr, long long ldr_rows,
                  cplx* Cp, long long scm, long long scn) {
    // C(i, j) = sum_nu conj(L[nu][l0+i]) R[nu][r0+j]
    ZGemmDesc g;
    g.M = nl; g.N = nr; g.K = (int)D;
    g.A = Lp + l0; g.sam = 1; g.sak = cap; g.conjA = true;
    g.B = Rp + r0; g.sbk = ldr_rows; g.sbn = 1;
    g.C = Cp; g.scm = scm; g.scn = scn;
    g.work = zgemm_work(c);
    zgemm(g, s);
  };
  // Hhat[0:m1, m0:m1] = S^H Z_new ; Hhat[m0:m1, 0:m0] = S_new^H Z_old
  proj(ms.S.p, 0, m1, ms.Z.p, m0, acc, cap, ms.Hh.p + (long long)m0 * cap, 1, cap);
  if (m0 > 0) proj(ms.S.p, m0, acc, ms.Z.p, 0, m0, cap, ms.Hh.p + m0, 1, cap);
  DBuf<cplx> Bc, Cc;
  Bc.alloc(D * np);
  Cc.alloc(D * nq);
  {
    DBuf<int> rows_p, rows_q;
    rows_p.alloc(np); rows_q.alloc(nq);
    GFCC_CUDA(cudaMemcpyAsync(rows_p.p, ms.porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    GFCC_CUDA(cudaMemcpyAsync(rows_q.p, ms.qorb.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    gather_rows_real_to_cplx(c->bvec.p, (int)D, rows_p.p, np, (int)D, Bc.p, np, s);
    gather_rows_real_to_cplx(c->cvec.p, (int)D, rows_q.p, nq, (int)D, Cc.p, nq, s);
    GFCC_CUDA(cudaStreamSynchronize(s));
  }
  proj(ms.S.p, m0, acc, Bc.p, 0, np, np, ms.bh.p + m0, 1, cap);
  {  // chat[q][m0+i] = sum_nu Cc[nu][q] S[nu][m0+i]
    ZGemmDesc g;
    g.M = nq; g.N = acc; g.K = (int)D;
    g.A = Cc.p; g.sam = 1; g.sak = nq;
    g.B = ms.S.p + m0; g.sbk = cap; g.sbn = 1;
    g.C = ms.ch.p + (long long)m0 * nq; g.scm = 1; g.scn = nq;
    g.work = zgemm_work(c);
    zgemm(g, s);
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
  ms.m = m1;
  // residual basis: coefficients of S_new and Z_new in Q
  std::vector<cplx> coef = basis_append(c, SZ.p, 2 * acc);
  grow_basis(c, ms.qn);
  grow_model(c, m1);
  put_cols(ms.RS, ms.q_cap, m0, coef, ms.qn, 0, acc, s);
  put_cols(ms.RZ, ms.q_cap, m0, coef, ms.qn, acc, acc, s);
  zgemm_work_check(c);
}

// Hessenberg form of the current reduced model, computed once per model version and reused by every
// evaluation and extrapolation: Householder reflections H_j = I - tau_j v_j v_j^H (j = 0..m-3),
// H = P^H Hhat P with P = H_0 H_1 ...; the left reflections go to bhat, the right ones to chat and
// (want_res) to the residual coefficient matrices.
static void hessenberg(gfcc_ctx* c, bool want_res) {
  MorState& ms = c->mor;
  if (ms.hess_version == ms.version && (!want_res || (ms.hess_res && ms.hess_qn == ms.qn))) return;
  cudaStream_t s = c->stream;
  ProfScope prof_h(PROF_EVAL_HESS, 0.0, s);
  const int m = ms.m, np = (int)ms.porb.size(), nq = (int)ms.qorb.size(), cap = ms.m_cap, qn = ms.qn;
  ms.hH.alloc((long long)m * m); ms.hb.alloc((long long)m * np); ms.hc.alloc((long long)nq * m);
  ms.hV.alloc((long long)m * m); ms.htau.alloc(m);
  cplx *Hw = ms.hH.p, *bw = ms.hb.p, *cw = ms.hc.p;
  GFCC_CUDA(cudaMemcpy2DAsync(Hw, sizeof(cplx) * m, ms.Hh.p, sizeof(cplx) * cap, sizeof(cplx) * m, m,
                              cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpy2DAsync(bw, sizeof(cplx) * m, ms.bh.p, sizeof(cplx) * cap, sizeof(cplx) * m, np,
                              cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(cw, ms.ch.p, sizeof(cplx) * nq * m, cudaMemcpyDeviceToDevice, s));
  cplx *A1 = nullptr, *A2 = nullptr;
  if (want_res) {
    ms.hA1.alloc((long long)qn * m); ms.hA2.alloc((long long)qn * m); ms.hRB.alloc((long long)qn * np);
    A1 = ms.hA1.p; A2 = ms.hA2.p;
    GFCC_CUDA(cudaMemcpy2DAsync(A1, sizeof(cplx) * qn, ms.RS.p, sizeof(cplx) * ms.q_cap, sizeof(cplx) * qn, m,
                                cudaMemcpyDeviceToDevice, s));
    GFCC_CUDA(cudaMemcpy2DAsync(A2, sizeof(cplx) * qn, ms.RZ.p, sizeof(cplx) * ms.q_cap, sizeof(cplx) * qn, m,
                                cudaMemcpyDeviceToDevice, s));
    GFCC_CUDA(cudaMemcpy2DAsync(ms.hRB.p, sizeof(cplx) * qn, ms.RB.p, sizeof(cplx) * ms.q_cap, sizeof(cplx) * qn, np,
                                cudaMemcpyDeviceToDevice, s));
  }
  DBuf<cplx> wv;
  wv.alloc((long long)m + nq + 2LL * qn + 1);
  RightMats rm;
  rm.n = 0;
  auto add = [&](cplx* p, long long ld, int rows) {
    if (rows > 0) { rm.p[rm.n] = p; rm.ld[rm.n] = ld; rm.rows[rm.n] = rows; ++rm.n; }
  };
  add(Hw, m, m);
  add(cw, nq, nq);
  if (want_res) { add(A1, qn, qn); add(A2, qn, qn); }
  long long rows_all = 0, tiles_all = 0;
  for (int k = 0; k < rm.n; ++k) {
    rows_all += rm.rows[k];
    tiles_all += (rm.rows[k] + 31) / 32;
  }
  for (int j = 0; j + 2 < m; ++j) {
    const int len = m - j - 1;
    cplx* v = ms.hV.p + (long long)j * m;
    double* tau = ms.htau.p + j;
    house_kernel<<<1, 256, 0, s>>>(Hw + (long long)j * m + j + 1, len, v, tau);
    GFCC_LAUNCH_CHECK();
    // left: columns j.. of H and all np columns of bhat
    house_left2_kernel<<<(m - j) + np, 256, 0, s>>>(Hw, m, j, m - j, bw, m, np, j + 1, len, v, tau);
    GFCC_LAUNCH_CHECK();
    // right: H, chat and the residual coefficient matrices
    house_right_w4_kernel<<<(unsigned)tiles_all, 256, 0, s>>>(rm, j + 1, len, v, wv.p);
    GFCC_LAUNCH_CHECK();
    house_right_update4_kernel<<<grid_for(rows_all * len), 256, 0, s>>>(rm, j + 1, len, v, wv.p, tau,
                                                                        rows_all * len);
    GFCC_LAUNCH_CHECK();
  }
  GFCC_CUDA(cudaStreamSynchronize(s));   // wv is released on return
  ms.hess_version = ms.version;
  ms.hess_res = want_res;
  ms.hess_qn = qn;
}

void mor_eval(gfcc_ctx* c, const double* omegas_host, int nw, cplx* G_dev, double* A_dev, double* maxres_dev,
              cplx* dG_dev) {
  MorState& ms = c->mor;
  cudaStream_t s = c->stream;
  ProfScope prof(PROF_MOR_EVAL, 0.0, s);
  const int m = ms.m, np = (int)ms.porb.size(), nq = (int)ms.qorb.size(), qn = ms.qn;
  GFCC_CHECK(m > 0, GFCC_ERR_STATE, "mor_eval: empty reduced model");
  const bool want_res = maxres_dev != nullptr;
  hessenberg(c, want_res);
  const cplx *Hw = ms.hH.p, *bw = ms.hb.p, *cw = ms.hc.p;
  const cplx *A1 = ms.hA1.p, *A2 = ms.hA2.p, *RBw = ms.hRB.p;
  DBuf<double> dbn;
  std::vector<int> qidx(np, -1);
  for (int p = 0; p < np; ++p)
    for (int q = 0; q < nq; ++q)
      if (ms.qorb[q] == ms.porb[p]) { qidx[p] = q; break; }
  DBuf<int> dq, dsing;
  DBuf<double> dom;
  dq.alloc(np); dsing.alloc(1); dom.alloc(nw); dbn.alloc(np);
  dsing.zero(s);
  GFCC_CUDA(cudaMemcpyAsync(dq.p, qidx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(dom.p, omegas_host, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(dbn.p, ms.bnorm.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
  // frequencies in batches: solutions Y [m][nb np] of a batch (about 2 GB at most), then Ghat = chat^T Y
  // and the residual coefficients (w - i eta) RS Y + RZ Y - RB as complex GEMMs over the whole batch
  const long long per = eval_scratch_per_cta(m);
  const long long bw_max = std::max<long long>(1, (2LL << 30) / ((long long)m * np * (long long)sizeof(cplx)));
  const int nbw = (int)std::min<long long>(nw, bw_max);
  const int ncta = (int)std::min<long long>(nbw, (long long)EVAL_CTAS_PER_SM * 152);
  DBuf<cplx> scratch, Y, Ys, Cr, Gt, Yd;
  DBuf<double> rcol;
  scratch.alloc(per * ncta);
  Y.alloc((long long)m * nbw * np);
  const bool want_G = G_dev != nullptr || A_dev != nullptr;
  if (want_G && !G_dev) Gt.alloc((long long)nbw * np * nq);
  if (dG_dev) Yd.alloc((long long)m * nbw * np);
  if (want_res) {
    Ys.alloc((long long)m * nbw * np);
    Cr.alloc((long long)qn * nbw * np);
    rcol.alloc((long long)nbw * np);
  }
  for (int w0 = 0; w0 < nw; w0 += nbw) {
    const int nb = std::min(nbw, nw - w0);
    const long long ldy = (long long)nb * np;
    EvalArgs ea;
    ea.m = m; ea.np = np; ea.nw = nb;
    ea.H = Hw; ea.bw = bw;
    ea.omegas = dom.p + w0; ea.eta = ms.eta;
    ea.scratch = scratch.p; ea.scratch_per_cta = per;
    ea.Y = Y.p; ea.ldy = ldy; ea.singular = dsing.p;
    {
      ProfScope ps(PROF_EVAL_SOLVE, 0.0, s);
      launch_eval_solve(ea, std::min(ncta, nb), s);
    }
    if (want_G) {   // G(q, n) = sum_k cw[q][k] Y[k][n], stored at Gb[n nq + q]
      cplx* Gb = G_dev ? G_dev + (long long)w0 * np * nq : Gt.p;
      ZGemmDesc g;
      g.M = nq; g.N = (int)ldy; g.K = m;
      g.A = cw; g.sam = 1; g.sak = nq;
      g.B = Y.p; g.sbk = ldy; g.sbn = 1;
      g.C = Gb; g.scm = 1; g.scn = nq;
      g.work = zgemm_work(c);
      zgemm(g, s);
      if (A_dev) {
        spectral_from_G_kernel<<<(nb + 127) / 128, 128, 0, s>>>(Gb, nb, np, nq, dq.p, A_dev + w0);
        GFCC_LAUNCH_CHECK();
      }
    }
    if (dG_dev) {   // dGhat/dw = -chat^T (w - i eta + H)^{-2} bhat: a second solve with y as right side
      GFCC_CUDA(cudaMemcpyAsync(Yd.p, Y.p, sizeof(cplx) * m * ldy, cudaMemcpyDeviceToDevice, s));
      EvalArgs eb = ea;
      eb.Y = Yd.p;
      eb.rhs_in_Y = 1;
      launch_eval_solve(eb, std::min(ncta, nb), s);
      ZGemmDesc g;
      g.M = nq; g.N = (int)ldy; g.K = m;
      g.A = cw; g.sam = 1; g.sak = nq;
      g.B = Yd.p; g.sbk = ldy; g.sbn = 1;
      g.C = dG_dev + (long long)w0 * np * nq; g.scm = 1; g.scn = nq;
      g.alpha = make_cuDoubleComplex(-1.0, 0.0);
      g.work = zgemm_work(c);
      zgemm(g, s);
    }
    if (want_res) {   // coefficients of r = (w - i eta) S y + Z y - b in the orthonormal residual basis
      shift_scale_kernel<<<grid_for((long long)m * ldy), 256, 0, s>>>(Y.p, ldy, m, np, nb, dom.p + w0, ms.eta, Ys.p);
      GFCC_LAUNCH_CHECK();
      ZGemmDesc g;
      g.M = qn; g.N = (int)ldy; g.K = m;
      g.A = A1; g.sam = 1; g.sak = qn;
      g.B = Ys.p; g.sbk = ldy; g.sbn = 1;
      g.C = Cr.p; g.scm = ldy; g.scn = 1;
      g.work = zgemm_work(c);
      zgemm(g, s);
      g.A = A2; g.B = Y.p; g.beta = make_cuDoubleComplex(1.0, 0.0);
      g.work = zgemm_work(c);
      zgemm(g, s);
      resnorm_kernel<<<(unsigned)((ldy + 255) / 256), 256, 0, s>>>(Cr.p, ldy, qn, RBw, np, nb, dbn.p, rcol.p);
      GFCC_LAUNCH_CHECK();
      rowmax_kernel<<<(nb + 127) / 128, 128, 0, s>>>(rcol.p, np, nb, maxres_dev + w0);
      GFCC_LAUNCH_CHECK();
    }
  }
  int hs = 0;
  GFCC_CUDA(cudaMemcpyAsync(&hs, dsing.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  GFCC_CHECK(hs == 0, GFCC_ERR_NONFINITE, "mor_eval: singular reduced system at a requested frequency");
  zgemm_work_check(c);
}

// Initial guesses for new frequencies: x0_p(w) = S yhat_p(w) with (w - i eta + Hhat) yhat_p = bhat_p.
// Hhat is reduced to Hessenberg form H = P^H Hhat P by Householder reflections (recorded), each
// frequency is the shifted Hessenberg solve of eval_solve_kernel, yhat = P y_H applies the reflections
// in reverse order, and X0 = S yhat is one complex GEMM. X0: [D][nw np] batch-minor (column w np + p).
void mor_extrapolate(gfcc_ctx* c, const double* omegas_host, int nw, cplx* X0) {
  MorState& ms = c->mor;
  cudaStream_t s = c->stream;
  const int m = ms.m, np = (int)ms.porb.size(), cap = ms.m_cap;
  GFCC_CHECK(m > 0, GFCC_ERR_STATE, "mor_extrapolate: empty reduced model");
  const long long N = (long long)nw * np;
  hessenberg(c, false);
  DBuf<cplx> Y, scratch;
  DBuf<double> dom;
  DBuf<int> dsing;
  const long long per = eval_scratch_per_cta(m);
  const int ncta = (int)std::min<long long>(nw, (long long)EVAL_CTAS_PER_SM * 152);
  scratch.alloc(per * ncta);
  Y.alloc((long long)m * N);
  dom.alloc(nw); dsing.alloc(1);
  dsing.zero(s);
  GFCC_CUDA(cudaMemcpyAsync(dom.p, omegas_host, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
  EvalArgs ea;
  ea.m = m; ea.np = np; ea.nw = nw;
  ea.H = ms.hH.p; ea.bw = ms.hb.p;
  ea.omegas = dom.p; ea.eta = ms.eta;
  ea.scratch = scratch.p; ea.scratch_per_cta = per;
  ea.Y = Y.p; ea.ldy = N; ea.singular = dsing.p;
  launch_eval_solve(ea, ncta, s);
  for (int j = m - 3; j >= 0; --j) {   // yhat = P y_H, P = H_0 H_1 ... (Hermitian reflectors)
    house_rows_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(Y.p, N, N, j + 1, m - j - 1,
                                                                  ms.hV.p + (long long)j * m, ms.htau.p + j);
    GFCC_LAUNCH_CHECK();
  }
  ZGemmDesc g;   // X0[nu][n] = sum_k S[nu][k] yhat[k][n]
  g.M = (int)c->D; g.N = (int)N; g.K = m;
  g.A = ms.S.p; g.sam = cap; g.sak = 1;
  g.B = Y.p; g.sbk = N; g.sbn = 1;
  g.C = X0; g.scm = N; g.scn = 1;
  g.work = zgemm_work(c);
  zgemm(g, s);
  int hs = 0;
  GFCC_CUDA(cudaMemcpyAsync(&hs, dsing.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  GFCC_CHECK(hs == 0, GFCC_ERR_NONFINITE, "mor_extrapolate: singular reduced system at a new frequency");
  zgemm_work_check(c);
}

}  // namespace gfcc
