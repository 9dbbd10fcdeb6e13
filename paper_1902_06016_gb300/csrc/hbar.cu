// One-time construction, on the GPU in FP64, of the H-bar elements that act on the IP
// (1h + 2h1p) space and of the free/left vectors b_p, c_q.
//
// Hbar_N = e^{-T} H e^{T} - E_0 (text after Eq. gfxn1). Spin-orbital elements, with f = diag(eps),
// tau_ij^ab = t_ij^ab + t_i^a t_j^b - t_i^b t_j^a and summation over repeated indices:
//   F_me = t_n^f <mn||ef>
//   F_mi = f_mi + t_n^e <mn||ie> + 1/2 tau_in^ef <mn||ef>
//   F_ae = f_ae + t_m^f <am||ef> - 1/2 tau_mn^af <mn||ef>
//   W_mnij = <mn||ij> + P(ij) t_j^e <mn||ie> + 1/2 tau_ij^ef <mn||ef>
//   W_mnie = <mn||ie> + t_i^f <mn||fe>
//   W_mbej = <mb||ej> + t_j^f <mb||ef> - t_n^b <mn||ej> - (t_jn^fb + t_j^f t_n^b) <mn||ef>
//   W_mbij = <mb||ij> - F_me t_ij^be - t_n^b W_mnij + 1/2 <mb||ef> tau_ij^ef
//            - P(ij) <mn||je> t_in^be + P(ij) t_i^e (<mb||ej> - t_nj^bf <mn||ef>)
// These are then scattered into the GEMM operands of the sigma (see Operator in the internal
// header). b_p and c_q follow from expanding e^{-T} a_p e^{T} and <Phi|(1+Lambda) e^{-T} a_q^+ e^{T}.
#include "gfcc_internal.cuh"
#include "tensor.h"

#include <cmath>
#include <memory>

namespace gfcc {
namespace {

// Decode pair index P -> (i, j), i < j.
__device__ __forceinline__ void unpair(int p, int& i, int& j) {
  // FP32 estimate (GB300's FP64 pipe is narrow), corrected to the exact integer below
  int jj = (int)floorf((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (jj * (jj - 1) / 2 > p) --jj;
  while ((jj + 1) * jj / 2 <= p) ++jj;
  j = jj;
  i = p - jj * (jj - 1) / 2;
}

__global__ void add_diag_kernel(double* F, int n, const double* e, double scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) F[(long long)i * n + i] += scale * e[i];
}

// Wr[(a,i)][(m,e)] = W_maei - d_ae F_mi(off) + 1/2 d_mi F_ae(off); Wmbej stored [m][b][e][j].
__global__ void build_ring_kernel(const double* __restrict__ Wmbej, const double* __restrict__ Fmi,
                                  const double* __restrict__ Fae, double* __restrict__ Wr, int o, int v) {
  long long ov = (long long)o * v;
  long long total = ov * ov;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long row = t / ov, col = t % ov;
    int a = (int)(row / o), i = (int)(row % o);
    int m = (int)(col / v), e = (int)(col % v);
    double w = Wmbej[(((long long)m * v + a) * v + e) * o + i];
    if (a == e && m != i) w -= Fmi[(long long)m * o + i];
    if (m == i && a != e) w += 0.5 * Fae[(long long)a * v + e];
    Wr[t] = w;
  }
}

// Woo[pair(ij)][pair(mn)] = W_mnij
__global__ void build_oooo_kernel(const double* __restrict__ Wmnij, double* __restrict__ Woo, int o) {
  int P = o * (o - 1) / 2;
  long long total = (long long)P * P;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int pij = (int)(t / P), pmn = (int)(t % P);
    int i, j, m, n;
    unpair(pij, i, j);
    unpair(pmn, m, n);
    Woo[t] = Wmnij[(((long long)m * o + n) * o + i) * o + j];
  }
}

// A12[i][(pair(k,l), e)]: +F_le if k == i, -F_ke if l == i, -W_klie  (1h <- 2h1p block)
__global__ void build_a12_kernel(const double* __restrict__ Fme, const double* __restrict__ Wmnie,
                                 double* __restrict__ A12, int o, int v) {
  int P = o * (o - 1) / 2;
  long long cols = (long long)P * v;
  long long total = (long long)o * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / cols);
    long long c = t % cols;
    int pkl = (int)(c / v), e = (int)(c % v);
    int k, l;
    unpair(pkl, k, l);
    double w = -Wmnie[(((long long)k * o + l) * o + i) * v + e];
    if (k == i) w += Fme[(long long)l * v + e];
    if (l == i) w -= Fme[(long long)k * v + e];
    A12[t] = w;
  }
}

// A21[(pair(ij), a)][m] = -W_maij ; Wmbij stored [m][b][i][j]
__global__ void build_a21_kernel(const double* __restrict__ Wmbij, double* __restrict__ A21, int o, int v) {
  int P = o * (o - 1) / 2;
  long long total = (long long)P * v * o;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long row = t / o;
    int m = (int)(t % o);
    int pij = (int)(row / v), a = (int)(row % v);
    int i, j;
    unpair(pij, i, j);
    A21[t] = -Wmbij[(((long long)m * v + a) * o + i) * o + j];
  }
}

// Vt[e][(pair(mn), f)] = <mn||ef>;  T2p[(pair(ij), a)][e] = t_ij^ae
__global__ void build_three_body_kernel(const double* __restrict__ voovv, const double* __restrict__ t2,
                                        double* __restrict__ Vt, double* __restrict__ T2p, int o, int v) {
  int P = o * (o - 1) / 2;
  long long Pv = (long long)P * v;
  long long total = Pv * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // Vt index: e * Pv + (pmn*v + f)
    {
      int e = (int)(t / Pv);
      long long c = t % Pv;
      int pmn = (int)(c / v), f = (int)(c % v);
      int m, n;
      unpair(pmn, m, n);
      Vt[t] = voovv[(((long long)m * o + n) * v + e) * v + f];
    }
    // T2p index: (pij*v + a) * v + e
    {
      long long row = t / v;
      int e = (int)(t % v);
      int pij = (int)(row / v), a = (int)(row % v);
      int i, j;
      unpair(pij, i, j);
      T2p[t] = t2[(((long long)i * o + j) * v + a) * v + e];
    }
  }
}

// Fock-diagonal part and full diagonal of M.
__global__ void build_diag_kernel(const double* __restrict__ Fmi, const double* __restrict__ Fae,
                                  const double* __restrict__ Wmbej, const double* __restrict__ Wmnij,
                                  const double* __restrict__ t2, const double* __restrict__ voovv,
                                  double* __restrict__ dg, double* __restrict__ md, int o, int v) {
  int P = o * (o - 1) / 2;
  long long D = o + (long long)P * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < D;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < o) {
      double d = -Fmi[t * o + t];
      dg[t] = d;
      md[t] = d;
    } else {
      long long r = t - o;
      int pij = (int)(r / v), a = (int)(r % v);
      int i, j;
      unpair(pij, i, j);
      double d = Fae[(long long)a * v + a] - Fmi[(long long)i * o + i] - Fmi[(long long)j * o + j];
      dg[t] = d;
      // ring diagonal W_iaai + W_jaaj, oooo diagonal W_ijij, three-body t_ij^ae <ij||ea>
      double w = Wmbej[(((long long)i * v + a) * v + a) * o + i] + Wmbej[(((long long)j * v + a) * v + a) * o + j]
               + Wmnij[(((long long)i * o + j) * o + i) * o + j];
      double tb = 0.0;
      for (int e = 0; e < v; ++e)
        tb += t2[(((long long)i * o + j) * v + a) * v + e] * voovv[(((long long)i * o + j) * v + e) * v + a];
      md[t] = d + w + tb;
    }
  }
}

// b_p rows [n][D]: b_i = e_i; b_a = (t_k^a ; t_kl^ac)
__global__ void build_b_kernel(const double* __restrict__ t1, const double* __restrict__ t2,
                               double* __restrict__ bv, int o, int v) {
  int n = o + v, P = o * (o - 1) / 2;
  long long D = o + (long long)P * v;
  long long total = (long long)n * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int p = (int)(t / D);
    long long nu = t % D;
    double val = 0.0;
    if (p < o) {
      val = (nu == p) ? 1.0 : 0.0;
    } else {
      int a = p - o;
      if (nu < o) {
        val = t1[nu * v + a];
      } else {
        long long r = nu - o;
        int pkl = (int)(r / v), c = (int)(r % v);
        int k, l;
        unpair(pkl, k, l);
        val = t2[(((long long)k * o + l) * v + a) * v + c];
      }
    }
    bv[t] = val;
  }
}

// c_q rows [n][D]:
//   c_a[k] = l_a^k, c_a[klc] = l_ac^kl
//   c_i[k] = d_ik - t_i^e l_e^k - 1/2 t_in^ef l_ef^kn   (the last sum is precomputed in X2[i][k])
//   c_i[klc] = d_ik l_c^l - d_il l_c^k - t_i^e l_ec^kl
__global__ void build_c_kernel(const double* __restrict__ t1, const double* __restrict__ l1,
                               const double* __restrict__ l2, const double* __restrict__ X2,
                               double* __restrict__ cv, int o, int v) {
  int n = o + v, P = o * (o - 1) / 2;
  long long D = o + (long long)P * v;
  long long total = (long long)n * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int q = (int)(t / D);
    long long nu = t % D;
    double val = 0.0;
    if (q >= o) {
      int a = q - o;
      if (nu < o) {
        val = l1[nu * v + a];
      } else {
        long long r = nu - o;
        int pkl = (int)(r / v), c = (int)(r % v);
        int k, l;
        unpair(pkl, k, l);
        val = l2[(((long long)k * o + l) * v + a) * v + c];
      }
    } else {
      int i = q;
      if (nu < o) {
        int k = (int)nu;
        double s = (i == k) ? 1.0 : 0.0;
        for (int e = 0; e < v; ++e) s -= t1[(long long)i * v + e] * l1[(long long)k * v + e];
        s -= 0.5 * X2[(long long)i * o + k];
        val = s;
      } else {
        long long r = nu - o;
        int pkl = (int)(r / v), c = (int)(r % v);
        int k, l;
        unpair(pkl, k, l);
        double s = 0.0;
        if (i == k) s += l1[(long long)l * v + c];
        if (i == l) s -= l1[(long long)k * v + c];
        for (int e = 0; e < v; ++e)
          s -= t1[(long long)i * v + e] * l2[(((long long)k * o + l) * v + e) * v + c];
        val = s;
      }
    }
    cv[t] = val;
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

__global__ void nonfinite_kernel(const double* x, long long n, int* flag) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[t])) *flag = 1;
}

}  // namespace

HbarCommon::HbarCommon(int o_, int v_)
    : o(o_), v(v_), tau("ijab", {o_, o_, v_, v_}), Fme("me", {o_, v_}), Fmi("mi", {o_, o_}), Fae("ae", {v_, v_}),
      Y("mbej", {o_, v_, v_, o_}), Wmbej("mbej", {o_, v_, v_, o_}) {}

std::unique_ptr<HbarCommon> build_common(const HostInputs& in, int o, int v, cudaStream_t s) {
  const int n = o + v;
  auto h = std::make_unique<HbarCommon>(o, v);
  // ---- upload inputs -------------------------------------------------------------------------
  auto up = [&](std::vector<int> dims, const double* src) {
    std::string lab(dims.size(), 'x');
    for (size_t k = 0; k < dims.size(); ++k) lab[k] = (char)('A' + k);
    auto t = std::make_unique<Tensor>(lab, dims);
    GFCC_CUDA(cudaMemcpyAsync(t->p(), src, t->size() * sizeof(double), kind_to_device(src), s));   // host or device
    return t;
  };
  {
    ProfScope pu(PROF_UPLOAD, 0.0, s);
    h->eps = up({n}, in.eps);
    h->v_oooo = up({o, o, o, o}, in.oooo);
    h->v_ooov = up({o, o, o, v}, in.ooov);
    h->v_oovv = up({o, o, v, v}, in.oovv);
    h->v_ovov = up({o, v, o, v}, in.ovov);
    h->v_ovvv = up({o, v, v, v}, in.ovvv);
    h->t1 = up({o, v}, in.t1);
    h->t2 = up({o, o, v, v}, in.t2);
    h->l1 = up({o, v}, in.l1);
    h->l2 = up({o, o, v, v}, in.l2);
  }
  {  // reject non-finite inputs before any arithmetic
    DBuf<int> flag;
    flag.alloc(1);
    flag.zero(s);
    for (Tensor* t : {h->eps.get(), h->v_oooo.get(), h->v_ooov.get(), h->v_oovv.get(), h->v_ovov.get(),
                      h->v_ovvv.get(), h->t1.get(), h->t2.get(), h->l1.get(), h->l2.get()}) {
      nonfinite_kernel<<<grid_for(t->size()), 256, 0, s>>>(t->p(), t->size(), flag.p);
      GFCC_LAUNCH_CHECK();
    }
    int hf = 0;
    GFCC_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    GFCC_CHECK(hf == 0, GFCC_ERR_NONFINITE, "gfcc_init: non-finite value in the inputs");
  }
  Tensor *t1 = h->t1.get(), *t2 = h->t2.get(), *v_oovv = h->v_oovv.get(), *v_ooov = h->v_ooov.get();
  Tensor *v_ovvv = h->v_ovvv.get(), *v_ovov = h->v_ovov.get();
  Tensor &tau = h->tau, &Fme = h->Fme, &Fmi = h->Fmi, &Fae = h->Fae, &Y = h->Y, &Wmbej = h->Wmbej;

  // tau_ij^ab = t_ij^ab + t_i^a t_j^b - t_i^b t_j^a
  perm(t2->as("ijab"), 1.0, 0.0, tau.as("ijab"), s);
  contract(1.0, t1->as("ia"), t1->as("jb"), 1.0, tau.as("ijab"), s);
  contract(-1.0, t1->as("ib"), t1->as("ja"), 1.0, tau.as("ijab"), s);

  // one-body elements
  contract(1.0, t1->as("nf"), v_oovv->as("mnef"), 0.0, Fme.as("me"), s);
  contract(1.0, t1->as("ne"), v_ooov->as("mnie"), 0.0, Fmi.as("mi"), s);
  contract(0.5, tau.as("inef"), v_oovv->as("mnef"), 1.0, Fmi.as("mi"), s);
  add_diag_kernel<<<(o + 255) / 256, 256, 0, s>>>(Fmi.p(), o, h->eps->p(), 1.0);
  GFCC_LAUNCH_CHECK();
  contract(-1.0, t1->as("mf"), v_ovvv->as("maef"), 0.0, Fae.as("ae"), s);      // <am||ef> = -<ma||ef>
  contract(-0.5, tau.as("mnaf"), v_oovv->as("mnef"), 1.0, Fae.as("ae"), s);
  add_diag_kernel<<<(v + 255) / 256, 256, 0, s>>>(Fae.p(), v, h->eps->p() + o, 1.0);
  GFCC_LAUNCH_CHECK();

  // Y_mbej = t_jn^fb <mn||ef>  (shared by W_mbej, W_mbij and W_abej)
  contract(1.0, t2->as("jnfb"), v_oovv->as("mnef"), 0.0, Y.as("mbej"), s);

  // W_mbej = <mb||ej> + t_j^f <mb||ef> - t_n^b <mn||ej> - Y - t_j^f t_n^b <mn||ef>
  perm(v_ovov->as("mbje"), -1.0, 0.0, Wmbej.as("mbej"), s);                    // <mb||ej> = -<mb||je>
  contract(1.0, t1->as("jf"), v_ovvv->as("mbef"), 1.0, Wmbej.as("mbej"), s);
  contract(1.0, t1->as("nb"), v_ooov->as("mnje"), 1.0, Wmbej.as("mbej"), s);   // <mn||ej> = -<mn||je>
  perm(Y.as("mbej"), -1.0, 1.0, Wmbej.as("mbej"), s);
  {
    Tensor tmp("mnej", {o, o, v, o});
    contract(1.0, t1->as("jf"), v_oovv->as("mnef"), 0.0, tmp.as("mnej"), s);
    contract(-1.0, t1->as("nb"), tmp.as("mnej"), 1.0, Wmbej.as("mbej"), s);
  }
  return h;
}

void build_operator(gfcc_ctx* c, const HostInputs& in) {
  const int o = c->o, v = c->v, P = c->P, n = c->n;
  const long long D = c->D;
  cudaStream_t s = c->stream;
  ProfScope prof(PROF_INIT, 0.0, s);
  std::unique_ptr<HbarCommon> hc = build_common(in, o, v, s);
  Tensor *t1 = hc->t1.get(), *t2 = hc->t2.get(), *l1 = hc->l1.get(), *l2 = hc->l2.get();
  Tensor *v_oooo = hc->v_oooo.get(), *v_ooov = hc->v_ooov.get(), *v_oovv = hc->v_oovv.get();
  Tensor *v_ovov = hc->v_ovov.get(), *v_ovvv = hc->v_ovvv.get();
  Tensor &tau = hc->tau, &Fme = hc->Fme, &Fmi = hc->Fmi, &Fae = hc->Fae, &Y = hc->Y, &Wmbej = hc->Wmbej;

  // W_mnij
  Tensor Wmnij("mnij", {o, o, o, o});
  perm(v_oooo->as("mnij"), 1.0, 0.0, Wmnij.as("mnij"), s);
  contract(1.0, t1->as("je"), v_ooov->as("mnie"), 1.0, Wmnij.as("mnij"), s);
  contract(-1.0, t1->as("ie"), v_ooov->as("mnje"), 1.0, Wmnij.as("mnij"), s);
  contract(0.5, tau.as("ijef"), v_oovv->as("mnef"), 1.0, Wmnij.as("mnij"), s);

  // W_mnie
  Tensor Wmnie("mnie", {o, o, o, v});
  perm(v_ooov->as("mnie"), 1.0, 0.0, Wmnie.as("mnie"), s);
  contract(1.0, t1->as("if"), v_oovv->as("mnfe"), 1.0, Wmnie.as("mnie"), s);

  // W_mbij
  Tensor Wmbij("mbij", {o, v, o, o});
  perm(v_ooov->as("ijmb"), 1.0, 0.0, Wmbij.as("mbij"), s);                      // <mb||ij> = <ij||mb>
  contract(-1.0, Fme.as("me"), t2->as("ijbe"), 1.0, Wmbij.as("mbij"), s);
  contract(-1.0, t1->as("nb"), Wmnij.as("mnij"), 1.0, Wmbij.as("mbij"), s);
  contract(0.5, v_ovvv->as("mbef"), tau.as("ijef"), 1.0, Wmbij.as("mbij"), s);
  contract(-1.0, v_ooov->as("mnje"), t2->as("inbe"), 1.0, Wmbij.as("mbij"), s);
  contract(1.0, v_ooov->as("mnie"), t2->as("jnbe"), 1.0, Wmbij.as("mbij"), s);
  {
    Tensor X("mbej", {o, v, v, o});                                              // <mb||ej> - t_nj^bf <mn||ef>
    perm(v_ovov->as("mbje"), -1.0, 0.0, X.as("mbej"), s);
    perm(Y.as("mbej"), -1.0, 1.0, X.as("mbej"), s);
    contract(1.0, t1->as("ie"), X.as("mbej"), 1.0, Wmbij.as("mbij"), s);
    contract(-1.0, t1->as("je"), X.as("mbei"), 1.0, Wmbij.as("mbij"), s);
  }

  // ---- scatter into the sigma operands -------------------------------------------------------
  Operator& op = c->op;
  const long long ov = (long long)o * v, Pv = (long long)P * v;
  op.Wr.alloc(ov * ov);
  op.Woo.alloc((long long)P * P);
  op.A11.alloc((long long)o * o);
  op.A12.alloc(o * Pv);
  op.A21.alloc(Pv * o);
  op.Vt.alloc(v * Pv);
  op.T2p.alloc(Pv * v);
  op.diag.alloc(D);
  op.mdiag.alloc(D);
  build_ring_kernel<<<grid_for(ov * ov), 256, 0, s>>>(Wmbej.p(), Fmi.p(), Fae.p(), op.Wr.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_oooo_kernel<<<grid_for((long long)P * P), 256, 0, s>>>(Wmnij.p(), op.Woo.p, o);
  GFCC_LAUNCH_CHECK();
  {  // A11[i][m] = -F_mi off the diagonal
    Tensor Ft("im", {o, o});
    perm(Fmi.as("mi"), -1.0, 0.0, Ft.as("im"), s);
    GFCC_CUDA(cudaMemcpyAsync(op.A11.p, Ft.p(), sizeof(double) * o * o, cudaMemcpyDeviceToDevice, s));
    Tensor z("i", {o});
    z.buf.zero(s);
    // zero the diagonal: A11[i][i] += F_ii (= -(-F_ii))
    std::vector<double> hd(o);
    GFCC_CUDA(cudaStreamSynchronize(s));
    std::vector<double> hF((size_t)o * o);
    GFCC_CUDA(cudaMemcpy(hF.data(), op.A11.p, sizeof(double) * o * o, cudaMemcpyDeviceToHost));
    for (int i = 0; i < o; ++i) hF[(size_t)i * o + i] = 0.0;
    GFCC_CUDA(cudaMemcpy(op.A11.p, hF.data(), sizeof(double) * o * o, cudaMemcpyHostToDevice));
  }
  build_a12_kernel<<<grid_for(o * Pv), 256, 0, s>>>(Fme.p(), Wmnie.p(), op.A12.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_a21_kernel<<<grid_for(Pv * o), 256, 0, s>>>(Wmbij.p(), op.A21.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_three_body_kernel<<<grid_for(Pv * v), 256, 0, s>>>(v_oovv->p(), t2->p(), op.Vt.p, op.T2p.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_diag_kernel<<<grid_for(D), 256, 0, s>>>(Fmi.p(), Fae.p(), Wmbej.p(), Wmnij.p(), t2->p(),
                                                v_oovv->p(), op.diag.p, op.mdiag.p, o, v);
  GFCC_LAUNCH_CHECK();

  // ---- free terms and left vectors ------------------------------------------------------------
  c->bvec.alloc((long long)n * D);
  c->cvec.alloc((long long)n * D);
  build_b_kernel<<<grid_for((long long)n * D), 256, 0, s>>>(t1->p(), t2->p(), c->bvec.p, o, v);
  GFCC_LAUNCH_CHECK();
  {
    Tensor X2("ik", {o, o});                                                     // t_in^ef l_ef^kn
    contract(1.0, t2->as("inef"), l2->as("knef"), 0.0, X2.as("ik"), s);
    build_c_kernel<<<grid_for((long long)n * D), 256, 0, s>>>(t1->p(), l1->p(), l2->p(), X2.p(),
                                                              c->cvec.p, o, v);
    GFCC_LAUNCH_CHECK();
  }
  // keep amplitudes for derivative work
  c->t1.alloc(ov);
  c->t2.alloc(ov * ov);
  GFCC_CUDA(cudaMemcpyAsync(c->t1.p, t1->p(), sizeof(double) * ov, cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(c->t2.p, t2->p(), sizeof(double) * ov * ov, cudaMemcpyDeviceToDevice, s));
  auto keep = [&](DBuf<double>& dst, const Tensor& t) {
    dst.alloc(t.size());
    GFCC_CUDA(cudaMemcpyAsync(dst.p, t.p(), sizeof(double) * t.size(), cudaMemcpyDeviceToDevice, s));
  };
  keep(c->k_oovv, *v_oovv);
  keep(c->k_ooov, *v_ooov);
  keep(c->k_ovvv, *v_ovvv);
  keep(c->k_l2, *l2);
  keep(c->k_Fme, Fme);
  GFCC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gfcc
