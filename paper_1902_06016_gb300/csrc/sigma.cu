// Sigma: Y = M X (+ shift_c X) for a block of complex vectors, M the matrix of Hbar_N on the
// 1h + 2h1p space (Eq. xplin). Vectors use the batch-minor layout X[nu][c] (complex, ld = nb).
//
// Terms (spin orbitals, summation over repeated indices; P(ij) g_ij = g_ij - g_ji):
//   s_i    = -F_mi r_m + F_me r_im^e - 1/2 W_mnie r_mn^e
//   s_ij^a = -W_maij r_m + F_ae r_ij^e - P(ij) F_mi r_mj^a + 1/2 W_mnij r_mn^a
//            + P(ij) W_maei r_mj^e + 1/2 <mn||ef> r_mn^f t_ij^ae
// Mapped onto GEMMs whose N axis is the batch (2 reals per complex column):
//   1h  <- A11 r1 + A12 r2                 (o x o, o x Pv)
//   2h1p <- A21 r1 + Woo r2 + T2p (Vt r2)  (Pv x o, P x P per virtual, three-body as two GEMMs)
//   ring:  CT[(a,i)][(j,c)] = Wr[(a,i)][(m,e)] U[(m,e)][(j,c)],  U = r_mj^e unpacked (antisymmetric),
//          s_ij^a += CT[(a,i)][j] - CT[(a,j)][i]; Wr also carries the off-diagonal F_oo / F_vv terms
//   diagonal: (F_aa - F_ii - F_jj) r_ij^a and -F_ii r_i applied exactly, with the shift.
#include "gfcc_internal.cuh"

#include <algorithm>

namespace gfcc {
namespace {

__device__ __forceinline__ int pair_of(int i, int j) { return j * (j - 1) / 2 + i; }

__device__ __forceinline__ void unpair(int p, int& i, int& j) {
  // FP32 estimate (GB300's FP64 pipe is narrow), corrected to the exact integer below
  int jj = (int)floorf((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (jj * (jj - 1) / 2 > p) --jj;
  while ((jj + 1) * jj / 2 <= p) ++jj;
  j = jj;
  i = p - jj * (jj - 1) / 2;
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// U[((m*v + e)*o + j)*nb + c] = r_mj^e of column c (0 when m == j)
__global__ void unpack_ring_kernel(const cplx* __restrict__ X, cplx* __restrict__ U, int o, int v, int nb) {
  long long total = (long long)o * v * o * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % nb);
    long long r = t / nb;
    int j = (int)(r % o);
    r /= o;
    int e = (int)(r % v);
    int m = (int)(r / v);
    cplx val = make_cuDoubleComplex(0.0, 0.0);
    if (m < j) {
      val = X[((long long)o + (long long)pair_of(m, j) * v + e) * nb + c];
    } else if (m > j) {
      cplx x = X[((long long)o + (long long)pair_of(j, m) * v + e) * nb + c];
      val = make_cuDoubleComplex(-x.x, -x.y);
    }
    U[t] = val;
  }
}

// Y[nu][c] += (diag[nu] + shift[c]) X[nu][c]  (+ ring antisymmetrisation on 2h1p rows)
__global__ void combine_kernel(const cplx* __restrict__ X, cplx* __restrict__ Y, const cplx* __restrict__ CT,
                               const double* __restrict__ diag, const cplx* __restrict__ shift,
                               int o, int v, long long D, int nb) {
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % nb);
    long long nu = t / nb;
    cplx x = X[t];
    double dre = diag[nu], dim = 0.0;
    if (shift) { dre += shift[c].x; dim = shift[c].y; }
    cplx y = Y[t];
    y.x += dre * x.x - dim * x.y;
    y.y += dre * x.y + dim * x.x;
    if (nu >= o && CT) {
      long long r = nu - o;
      int pij = (int)(r / v), a = (int)(r % v);
      int i, j;
      unpair(pij, i, j);
      cplx c1 = CT[(((long long)a * o + i) * o + j) * nb + c];
      cplx c2 = CT[(((long long)a * o + j) * o + i) * nb + c];
      y.x += c1.x - c2.x;
      y.y += c1.y - c2.y;
    }
    Y[t] = y;
  }
}

}  // namespace

void ensure_workspace(gfcc_ctx* c, int nb) {
  if ((size_t)nb <= c->ws.nb_cap) return;
  const long long ov = (long long)c->o * c->v;
  c->ws.ut.alloc(2 * ov * c->o * (long long)nb);
  c->ws.ct.alloc(2 * ov * c->o * (long long)nb);
  c->ws.xe.alloc(2LL * c->v * nb);
  c->ws.nb_cap = nb;
}

// real GEMM whose B and C are complex batch-minor blocks: N' = 2 nb reals per row
static void rgemm_cplx(int M, int K, int nb, double alpha, const double* A, long long lda,
                       const cplx* B, long long ldb_rows, double beta, cplx* C, long long ldc_rows,
                       cudaStream_t s, bool transA = false) {
  GemmDesc g;
  g.M = M; g.N = 2 * nb; g.K = K;
  g.A = A; g.sam = transA ? 1 : lda; g.sak = transA ? lda : 1;
  g.B = reinterpret_cast<const double*>(B); g.sbk = 2 * ldb_rows; g.sbn = 1;
  g.C = reinterpret_cast<double*>(C); g.scm = 2 * ldc_rows; g.scn = 1;
  g.alpha = alpha; g.beta = beta;
  dgemm(g, s);
}

void sigma_batch(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, int ldb, const cplx* shift,
                 int precision, bool transpose, cudaStream_t s) {
  GFCC_CHECK(ldb == nb, GFCC_ERR_ARG, "sigma_batch: internal layout needs ldb == nb");
  if (nb == 0) return;
  const bool lowp = precision == GFCC_PREC_TF32 || precision == GFCC_PREC_BF16;
  // algorithmic flops of the sigma on nb complex columns (ring, oooo, three-body and coupling terms; the
  // method's flops, whatever arithmetic carries them out)
  const double fo = c->o, fv = c->v, fP = c->P;
  const double flops = 2.0 * nb * (2.0 * fo * fv * fo * fv * fo + 2.0 * fP * fP * fv + 4.0 * fP * fv * fv + 4.0 * fo * fP * fv);
  ProfScope prof(lowp ? PROF_SIGMA_LP : PROF_SIGMA_EX, flops, s);
  if (precision == GFCC_PREC_FP64_TC) {
    sigma_emulated(c, X, Y, nb, shift, s, transpose);
    return;
  }
  if (lowp) {
    GFCC_CHECK(c->lp.kind == precision && c->lp.impl, GFCC_ERR_STATE, "sigma: low-precision operands not built");
    sigma_lowprec(c, X, Y, nb, shift, s, transpose);
    return;
  }
  const int o = c->o, v = c->v, P = c->P;
  const long long D = c->D, Pv = (long long)P * v, ov = (long long)o * v;
  Operator& op = c->op;
  ensure_workspace(c, nb);
  if (transpose) build_transpose_operator(c);
  const double* A11 = op.A11.p;
  const double* A12 = transpose ? op.A12T.p : op.A12.p;
  const double* A21 = transpose ? op.A21T.p : op.A21.p;
  const double* Woo = transpose ? op.WooT.p : op.Woo.p;
  const double* Vt = transpose ? op.VtT.p : op.Vt.p;
  const double* T2p = transpose ? op.T2pT.p : op.T2p.p;
  const double* Wr = transpose ? op.WrT.p : op.Wr.p;
  const cplx* X1 = X;
  const cplx* X2 = X + (long long)o * nb;
  cplx* Y1 = Y;
  cplx* Y2 = Y + (long long)o * nb;

  // 1h rows: A11 r1 (+) A12 r2   (transpose: A11^T, and the 1h<-2h1p block of M^T is A21^T)
  rgemm_cplx(o, o, nb, 1.0, A11, o, X1, nb, 0.0, Y1, nb, s, transpose);
  rgemm_cplx(o, (int)Pv, nb, 1.0, A12, transpose ? o : Pv, X2, nb, 1.0, Y1, nb, s, transpose);
  // 2h1p rows: A21 r1
  rgemm_cplx((int)Pv, o, nb, 1.0, A21, transpose ? Pv : o, X1, nb, 0.0, Y2, nb, s, transpose);
  // oooo: Y2[(pij, a)][c] += sum_pmn Woo[pij][pmn] X2[(pmn, a)][c]  (N = v*nb complex)
  {
    GemmDesc g;
    g.M = P; g.N = 2 * v * nb; g.K = P;
    g.A = Woo; g.sam = transpose ? 1 : P; g.sak = transpose ? P : 1;
    g.B = reinterpret_cast<const double*>(X2); g.sbk = 2LL * v * nb; g.sbn = 1;
    g.C = reinterpret_cast<double*>(Y2); g.scm = 2LL * v * nb; g.scn = 1;
    g.alpha = 1.0; g.beta = 1.0;
    dgemm(g, s);
  }
  // three-body: xe = Vt r2 ; Y2 += T2p xe   (transpose: xe = T2p^T r2 ; Y2 += Vt^T xe)
  {
    cplx* xe = reinterpret_cast<cplx*>(c->ws.xe.p);
    if (!transpose) {
      rgemm_cplx(v, (int)Pv, nb, 1.0, Vt, Pv, X2, nb, 0.0, xe, nb, s);
      rgemm_cplx((int)Pv, v, nb, 1.0, T2p, v, xe, nb, 1.0, Y2, nb, s);
    } else {
      rgemm_cplx(v, (int)Pv, nb, 1.0, T2p, v, X2, nb, 0.0, xe, nb, s, true);
      rgemm_cplx((int)Pv, v, nb, 1.0, Vt, Pv, xe, nb, 1.0, Y2, nb, s, true);
    }
  }
  // ring: unpack, GEMM, antisymmetrise (inside combine)
  cplx* U = reinterpret_cast<cplx*>(c->ws.ut.p);
  cplx* CT = reinterpret_cast<cplx*>(c->ws.ct.p);
  unpack_ring_kernel<<<grid_for(ov * o * nb), 256, 0, s>>>(X2 - (long long)o * nb, U, o, v, nb);
  GFCC_LAUNCH_CHECK();
  {
    GemmDesc g;
    g.M = (int)ov; g.N = 2 * o * nb; g.K = (int)ov;
    g.A = Wr; g.sam = ov; g.sak = 1;
    g.B = reinterpret_cast<const double*>(U); g.sbk = 2LL * o * nb; g.sbn = 1;
    g.C = reinterpret_cast<double*>(CT); g.scm = 2LL * o * nb; g.scn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    dgemm(g, s);
  }
  combine_kernel<<<grid_for(D * nb), 256, 0, s>>>(X, Y, CT, op.diag.p, shift, o, v, D, nb);
  GFCC_LAUNCH_CHECK();
  c->stats.sigma_calls++;
  c->stats.sigma_cols += nb;
}

// M^T: 1h-1h A11^T (read transposed), 1h<-2h1p = A21^T, 2h1p<-1h = A12^T, oooo Woo^T,
// three-body (T2p Vt)^T = Vt^T T2p^T. The packed ring block is
//   R[(ij,a),(kl,e)] = d_jl Wr[ai,ke] - d_jk Wr[ai,le] - d_il Wr[aj,ke] + d_ik Wr[aj,le],
// so running the same unpack/GEMM/antisymmetrise with WrT[a,i,m,e] = Wr[e,m,i,a] gives R^T.
void build_transpose_operator(gfcc_ctx* c) {
  Operator& op = c->op;
  if (op.have_T) return;
  const int o = c->o, v = c->v, P = c->P;
  const long long Pv = (long long)P * v, ov = (long long)o * v;
  cudaStream_t s = c->stream;
  // A12T: the 1h <- 2h1p block of M^T is (2h1p <- 1h block)^T = A21^T  [o x Pv] = A21[(Pv) x o]^T
  // stored so that rgemm_cplx(transpose=true) reads A(m,k) = ptr[k*lda + m]:
  //   1h rows use A12T with lda = o  -> A12T must be laid out [Pv][o] = A21 itself
  //   2h1p rows use A21T with lda = Pv -> A21T laid out [o][Pv] = A12 itself
  op.A12T.alloc(Pv * o);
  op.A21T.alloc(o * Pv);
  GFCC_CUDA(cudaMemcpyAsync(op.A12T.p, op.A21.p, sizeof(double) * Pv * o, cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(op.A21T.p, op.A12.p, sizeof(double) * Pv * o, cudaMemcpyDeviceToDevice, s));
  // Woo read transposed in place
  op.WooT.alloc((long long)P * P);
  GFCC_CUDA(cudaMemcpyAsync(op.WooT.p, op.Woo.p, sizeof(double) * P * P, cudaMemcpyDeviceToDevice, s));
  op.VtT.alloc(v * Pv);
  op.T2pT.alloc(Pv * v);
  GFCC_CUDA(cudaMemcpyAsync(op.VtT.p, op.Vt.p, sizeof(double) * v * Pv, cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(op.T2pT.p, op.T2p.p, sizeof(double) * v * Pv, cudaMemcpyDeviceToDevice, s));
  // ring: WrT[a][i][m][e] = Wr[e][m][i][a] reproduces Ring^T through the same unpack/antisymmetrise
  op.WrT.alloc(ov * ov);
  int dims[4] = {v, o, o, v};
  int pm[4] = {3, 2, 1, 0};
  permute(op.Wr.p, dims, 4, pm, op.WrT.p, 1.0, 0.0, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
  op.have_T = true;
}

}  // namespace gfcc
