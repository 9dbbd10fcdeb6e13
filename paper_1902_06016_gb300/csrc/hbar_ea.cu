// One-time construction, on the GPU in FP64, of the electron-attachment (EA, 1p + 2p1h) operator and
// of its free and left vectors.
//
// The retarded Green's function of Eq. gfxn0 has an attachment term <Psi|a_p (w - (H - E_0) + i eta)^{-1}
// a_q^+|Psi> beside the ionisation term the paper works out. In the CC form (Eqs. gfxn1/gfxn2 with the
// field operators exchanged) it is G^EA_pq(w) = c_p^T (w + i eta - M) ^{-1} b_q over the 1p + 2p1h space:
// y = sum_a y^a a_a^+ + sum_{a<b, j} y^{ab}_j a_a^+ a_b^+ a_j, packed [y^a | y^{pair(a,b)}_j at
// v + pair(a,b)*o + j]. With r^{ab}_j antisymmetric in ab (summation over repeated indices):
//   s_a      = F_ae r_e + F_me r^{ae}_m + 1/2 W_amef r^{ef}_m
//   s^{ab}_j = W_abej r_e - F_mj r^{ab}_m + P(ab) F_ae r^{eb}_j + 1/2 W_abef r^{ef}_j
//              + P(ab) W_mbej r^{ae}_m - 1/2 <mn||ef> r^{ef}_n t_mj^ab
//   W_abef = <ab||ef> - P(ab) t_m^b <am||ef> + 1/2 tau_mn^ab <mn||ef>
//   W_amef = <am||ef> - t_n^a <nm||ef>
//   W_abej = <ab||ej> - F_me t_mj^ab + t_j^f W_abef + 1/2 <mn||ej> tau_mn^ab
//            - P(ab) <mb||ef> t_mj^af - P(ab) t_m^a (<mb||ej> - t_nj^bf <mn||ef>)
//   b_q: b_a = unit 1p vector; b_i = (-t_i^e ; -t_in^ef)
//   c_p: c_i = (-l_c^i ; -l_ef^in);  c_a = (d_ac - t_k^a l_c^k - 1/2 t_kl^ad l_cd^kl ;
//        d_ae l_f^n - d_af l_e^n - t_k^a l_ef^kn)
//
// This is the IP operator's block structure with the roles of the index ranges exchanged: the pair
// index runs over virtual pairs, the single index over occupied orbitals; the vvvv block takes the place
// of oooo, the ring block is again (ov) x (ov), the three-body term again factors through a vector over
// the single index. So the operator is scattered into the IP layout (Operator, with the context's o = v
// and v = o) and every sigma, solver and reduced-model kernel runs on it unchanged. The systems become
// those of the IP form: (w' - i eta + M) y = b' with w' = -w and b' = -b (the API negates frequencies
// at the boundary), and G^EA_pq = c_p^T y_q.
#include "gfcc_internal.cuh"
#include "tensor.h"

#include <algorithm>
#include <memory>

namespace gfcc {
namespace {

__device__ __forceinline__ void unpair(long long p, int& i, int& j) {
  // FP32 estimate, corrected to the exact integer below
  int jj = (int)floorf((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while ((long long)jj * (jj - 1) / 2 > p) --jj;
  while ((long long)(jj + 1) * jj / 2 <= p) ++jj;
  j = jj;
  i = (int)(p - (long long)jj * (jj - 1) / 2);
}

__device__ __forceinline__ long long pair_of(int a, int b) { return (long long)b * (b - 1) / 2 + a; }

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// full[a][b][c][d] = <ab||cd> from the packed pairs (a < b, c < d), antisymmetric in ab and in cd
__global__ void unpack_vvvv_kernel(const double* __restrict__ vp, double* __restrict__ full, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long total = (long long)v * v * v * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int d = (int)(t % v);
    long long r = t / v;
    int c = (int)(r % v);
    r /= v;
    int b = (int)(r % v);
    int a = (int)(r / v);
    double x = 0.0;
    if (a != b && c != d) {
      double sg = 1.0;
      int lo1 = a, hi1 = b, lo2 = c, hi2 = d;
      if (a > b) { lo1 = b; hi1 = a; sg = -sg; }
      if (c > d) { lo2 = d; hi2 = c; sg = -sg; }
      x = sg * vp[pair_of(lo1, hi1) * V + pair_of(lo2, hi2)];
    }
    full[t] = x;
  }
}

__global__ void nonfinite_kernel(const double* x, long long n, int* flag) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[t])) *flag = 1;
}

// Ring block in the IP layout, rows (j, a), columns (d, l) (single index first):
//   Wr[(j,a)][(d,l)] = W_ladj + d_jl F_ad (a != d) - 1/2 d_ad F_lj (j != l)
// The Fock terms carry the off-diagonal parts of P(ab) F_ae r^{eb}_j and -F_mj r^{ab}_m through the
// ring's antisymmetrisation, as in the IP operator. Wmbej stored [m][b][e][j].
__global__ void build_ring_ea_kernel(const double* __restrict__ Wmbej, const double* __restrict__ Fae,
                                     const double* __restrict__ Fmi, double* __restrict__ Wr, int o, int v) {
  const long long ov = (long long)o * v;
  const long long total = ov * ov;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long row = t / ov, col = t % ov;
    int j = (int)(row / v), a = (int)(row % v);
    int d = (int)(col / o), l = (int)(col % o);
    double w = Wmbej[(((long long)l * v + a) * v + d) * o + j];
    if (j == l && a != d) w += Fae[(long long)a * v + d];
    if (a == d && j != l) w -= 0.5 * Fmi[(long long)l * o + j];
    Wr[t] = w;
  }
}

// Woo[pair(a,b)][pair(c,d)] = W_abcd   (Wabef stored [a][b][e][f])
__global__ void build_vvvv_kernel(const double* __restrict__ Wabef, double* __restrict__ Woo, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long total = V * V;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int a, b, c, d;
    unpair(t / V, a, b);
    unpair(t % V, c, d);
    Woo[t] = Wabef[(((long long)a * v + b) * v + c) * v + d];
  }
}

// A11[a][e] = F_ae off the diagonal (the diagonal is applied exactly with the shift)
__global__ void build_a11_ea_kernel(const double* __restrict__ Fae, double* __restrict__ A11, int v) {
  long long total = (long long)v * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int a = (int)(t / v), e = (int)(t % v);
    A11[t] = (a == e) ? 0.0 : Fae[t];
  }
}

// A12[a][(pair(c,d), l)] = W_alcd + d_ac F_ld - d_ad F_lc   (1p <- 2p1h; Wamef stored [a][m][e][f])
__global__ void build_a12_ea_kernel(const double* __restrict__ Fme, const double* __restrict__ Wamef,
                                    double* __restrict__ A12, int o, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long cols = V * o;
  const long long total = (long long)v * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int a = (int)(t / cols);
    long long cc = t % cols;
    int l = (int)(cc % o);
    int c, d;
    unpair(cc / o, c, d);
    double w = Wamef[(((long long)a * o + l) * v + c) * v + d];
    if (c == a) w += Fme[(long long)l * v + d];
    if (d == a) w -= Fme[(long long)l * v + c];
    A12[t] = w;
  }
}

// A21[(pair(a,b), j)][c] = W_abcj   (2p1h <- 1p; Wabej stored [a][b][e][j])
__global__ void build_a21_ea_kernel(const double* __restrict__ Wabej, double* __restrict__ A21, int o, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long total = V * o * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % v);
    long long row = t / v;
    int j = (int)(row % o);
    int a, b;
    unpair(row / o, a, b);
    A21[t] = Wabej[(((long long)a * v + b) * v + c) * o + j];
  }
}

// Three-body term as two GEMMs through a vector over the single (occupied) index m:
//   x_m = sum_{n, e<f} <mn||ef> r^{ef}_n,   s^{ab}_j -= t_mj^ab x_m
//   Vt[m][(pair(e,f), n)] = <mn||ef>,  T2p[(pair(a,b), j)][m] = -t_mj^ab
__global__ void build_three_body_ea_kernel(const double* __restrict__ voovv, const double* __restrict__ t2,
                                           double* __restrict__ Vt, double* __restrict__ T2p, int o, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long Vo = V * o;
  const long long total = Vo * o;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    {  // Vt index: m * Vo + (pef * o + n)
      int m = (int)(t / Vo);
      long long cc = t % Vo;
      int n = (int)(cc % o);
      int e, f;
      unpair(cc / o, e, f);
      Vt[t] = voovv[(((long long)m * o + n) * v + e) * v + f];
    }
    {  // T2p index: (pab * o + j) * o + m
      int m = (int)(t % o);
      long long row = t / o;
      int j = (int)(row % o);
      int a, b;
      unpair(row / o, a, b);
      T2p[t] = -t2[(((long long)m * o + j) * v + a) * v + b];
    }
  }
}

// Fock part of the diagonal (applied exactly with the shift) and the full diagonal (preconditioner):
//   1p: F_aa;  2p1h: F_aa + F_bb - F_jj, plus W_jaaj + W_jbbj (ring), W_abab (vvvv), -sum_m <mj||ab> t_mj^ab
__global__ void build_diag_ea_kernel(const double* __restrict__ Fmi, const double* __restrict__ Fae,
                                     const double* __restrict__ Wmbej, const double* __restrict__ Wabef,
                                     const double* __restrict__ t2, const double* __restrict__ voovv,
                                     double* __restrict__ dg, double* __restrict__ md, int o, int v) {
  const long long V = (long long)v * (v - 1) / 2;
  const long long D = v + V * o;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < D;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < v) {
      double d = Fae[t * v + t];
      dg[t] = d;
      md[t] = d;
    } else {
      long long r = t - v;
      int j = (int)(r % o);
      int a, b;
      unpair(r / o, a, b);
      double d = Fae[(long long)a * v + a] + Fae[(long long)b * v + b] - Fmi[(long long)j * o + j];
      dg[t] = d;
      double w = Wmbej[(((long long)j * v + a) * v + a) * o + j] + Wmbej[(((long long)j * v + b) * v + b) * o + j]
               + Wabef[(((long long)a * v + b) * v + a) * v + b];
      double tb = 0.0;
      for (int m = 0; m < o; ++m) {
        long long k = (((long long)m * o + j) * v + a) * v + b;
        tb -= voovv[k] * t2[k];
      }
      md[t] = d + w + tb;
    }
  }
}

// Free terms of the IP form, b' = -b: rows [n][D] by physical orbital q.
__global__ void build_b_ea_kernel(const double* __restrict__ t1, const double* __restrict__ t2,
                                  double* __restrict__ bv, int o, int v) {
  const int n = o + v;
  const long long V = (long long)v * (v - 1) / 2;
  const long long D = v + V * o;
  const long long total = (long long)n * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int q = (int)(t / D);
    long long nu = t % D;
    double val = 0.0;
    if (q >= o) {
      val = (nu == q - o) ? -1.0 : 0.0;
    } else if (nu < v) {
      val = t1[(long long)q * v + nu];
    } else {
      long long r = nu - v;
      int nn = (int)(r % o);
      int e, f;
      unpair(r / o, e, f);
      val = t2[(((long long)q * o + nn) * v + e) * v + f];
    }
    bv[t] = val;
  }
}

// Left vectors c_p, rows [n][D]; X2[a][c] = t_kl^ad l_cd^kl.
__global__ void build_c_ea_kernel(const double* __restrict__ t1, const double* __restrict__ l1,
                                  const double* __restrict__ l2, const double* __restrict__ X2,
                                  double* __restrict__ cv, int o, int v) {
  const int n = o + v;
  const long long V = (long long)v * (v - 1) / 2;
  const long long D = v + V * o;
  const long long total = (long long)n * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int p = (int)(t / D);
    long long nu = t % D;
    double val = 0.0;
    if (p < o) {
      if (nu < v) {
        val = -l1[(long long)p * v + nu];
      } else {
        long long r = nu - v;
        int nn = (int)(r % o);
        int e, f;
        unpair(r / o, e, f);
        val = -l2[(((long long)p * o + nn) * v + e) * v + f];
      }
    } else {
      int a = p - o;
      if (nu < v) {
        int c = (int)nu;
        double s = (a == c) ? 1.0 : 0.0;
        for (int k = 0; k < o; ++k) s -= t1[(long long)k * v + a] * l1[(long long)k * v + c];
        s -= 0.5 * X2[(long long)a * v + c];
        val = s;
      } else {
        long long r = nu - v;
        int nn = (int)(r % o);
        int e, f;
        unpair(r / o, e, f);
        double s = 0.0;
        if (a == e) s += l1[(long long)nn * v + f];
        if (a == f) s -= l1[(long long)nn * v + e];
        for (int k = 0; k < o; ++k)
          s -= t1[(long long)k * v + a] * l2[(((long long)k * o + nn) * v + e) * v + f];
        val = s;
      }
    }
    cv[t] = val;
  }
}

}  // namespace

void build_operator_ea(gfcc_ctx* c, const HostInputs& in) {
  // physical sizes: the context holds the IP-layout sizes (c->o = v, c->v = o)
  const int o = c->v, v = c->o, n = c->n;
  const long long V = (long long)v * (v - 1) / 2;
  const long long D = c->D;
  cudaStream_t s = c->stream;
  GFCC_CHECK(in.vvvv != nullptr, GFCC_ERR_ARG, "gfcc_init_ea: vvvv is null");
  ProfScope prof(PROF_INIT, 0.0, s);
  std::unique_ptr<HbarCommon> hc = build_common(in, o, v, s);
  Tensor *t1 = hc->t1.get(), *t2 = hc->t2.get(), *l1 = hc->l1.get(), *l2 = hc->l2.get();
  Tensor *v_ooov = hc->v_ooov.get(), *v_oovv = hc->v_oovv.get(), *v_ovov = hc->v_ovov.get();
  Tensor *v_ovvv = hc->v_ovvv.get();
  Tensor &tau = hc->tau, &Fme = hc->Fme, &Fmi = hc->Fmi, &Fae = hc->Fae, &Y = hc->Y, &Wmbej = hc->Wmbej;

  // <ab||cd> (packed on input) -> full [a][b][c][d]
  Tensor Wabef("abef", {v, v, v, v});
  {
    DBuf<double> vp;
    vp.alloc(V * V);
    {
      ProfScope pu(PROF_UPLOAD, 0.0, s);
      GFCC_CUDA(cudaMemcpyAsync(vp.p, in.vvvv, sizeof(double) * V * V, kind_to_device(in.vvvv), s));
    }
    DBuf<int> flag;
    flag.alloc(1);
    flag.zero(s);
    nonfinite_kernel<<<grid_for(V * V), 256, 0, s>>>(vp.p, V * V, flag.p);
    GFCC_LAUNCH_CHECK();
    unpack_vvvv_kernel<<<grid_for(Wabef.size()), 256, 0, s>>>(vp.p, Wabef.p(), v);
    GFCC_LAUNCH_CHECK();
    int hf = 0;
    GFCC_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    GFCC_CHECK(hf == 0, GFCC_ERR_NONFINITE, "gfcc_init_ea: non-finite value in vvvv");
  }
  // W_abef = <ab||ef> - t_m^b <am||ef> + t_m^a <bm||ef> + 1/2 tau_mn^ab <mn||ef>   (<am||ef> = -<ma||ef>)
  contract(1.0, t1->as("mb"), v_ovvv->as("maef"), 1.0, Wabef.as("abef"), s);
  contract(-1.0, t1->as("ma"), v_ovvv->as("mbef"), 1.0, Wabef.as("abef"), s);
  contract(0.5, tau.as("mnab"), v_oovv->as("mnef"), 1.0, Wabef.as("abef"), s);

  // W_amef = <am||ef> - t_n^a <nm||ef>
  Tensor Wamef("amef", {v, o, v, v});
  perm(v_ovvv->as("maef"), -1.0, 0.0, Wamef.as("amef"), s);
  contract(-1.0, t1->as("na"), v_oovv->as("nmef"), 1.0, Wamef.as("amef"), s);

  // W_abej
  Tensor Wabej("abej", {v, v, v, o});
  perm(v_ovvv->as("jeab"), -1.0, 0.0, Wabej.as("abej"), s);                   // <ab||ej> = -<je||ab>
  contract(-1.0, Fme.as("me"), t2->as("mjab"), 1.0, Wabej.as("abej"), s);
  contract(1.0, t1->as("jf"), Wabef.as("abef"), 1.0, Wabej.as("abej"), s);
  contract(-0.5, v_ooov->as("mnje"), tau.as("mnab"), 1.0, Wabej.as("abej"), s); // <mn||ej> = -<mn||je>
  {
    Tensor tmp("abej", {v, v, v, o});                                           // <mb||ef> t_mj^af
    contract(1.0, v_ovvv->as("mbef"), t2->as("mjaf"), 0.0, tmp.as("abej"), s);
    perm(tmp.as("abej"), -1.0, 1.0, Wabej.as("abej"), s);
    perm(tmp.as("baej"), 1.0, 1.0, Wabej.as("abej"), s);
    Tensor X("mbej", {o, v, v, o});                                             // <mb||ej> - t_nj^bf <mn||ef>
    perm(v_ovov->as("mbje"), -1.0, 0.0, X.as("mbej"), s);
    perm(Y.as("mbej"), -1.0, 1.0, X.as("mbej"), s);
    contract(1.0, t1->as("ma"), X.as("mbej"), 0.0, tmp.as("abej"), s);
    perm(tmp.as("abej"), -1.0, 1.0, Wabej.as("abej"), s);
    perm(tmp.as("baej"), 1.0, 1.0, Wabej.as("abej"), s);
  }

  // ---- scatter into the sigma operands (IP layout: pair index over virtual pairs) -------------
  Operator& op = c->op;
  const long long ov = (long long)o * v, Vo = V * o;
  op.Wr.alloc(ov * ov);
  op.Woo.alloc(V * V);
  op.A11.alloc((long long)v * v);
  op.A12.alloc(v * Vo);
  op.A21.alloc(Vo * v);
  op.Vt.alloc(o * Vo);
  op.T2p.alloc(Vo * o);
  op.diag.alloc(D);
  op.mdiag.alloc(D);
  build_ring_ea_kernel<<<grid_for(ov * ov), 256, 0, s>>>(Wmbej.p(), Fae.p(), Fmi.p(), op.Wr.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_vvvv_kernel<<<grid_for(V * V), 256, 0, s>>>(Wabef.p(), op.Woo.p, v);
  GFCC_LAUNCH_CHECK();
  build_a11_ea_kernel<<<grid_for((long long)v * v), 256, 0, s>>>(Fae.p(), op.A11.p, v);
  GFCC_LAUNCH_CHECK();
  build_a12_ea_kernel<<<grid_for(v * Vo), 256, 0, s>>>(Fme.p(), Wamef.p(), op.A12.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_a21_ea_kernel<<<grid_for(Vo * v), 256, 0, s>>>(Wabej.p(), op.A21.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_three_body_ea_kernel<<<grid_for(Vo * o), 256, 0, s>>>(v_oovv->p(), t2->p(), op.Vt.p, op.T2p.p, o, v);
  GFCC_LAUNCH_CHECK();
  build_diag_ea_kernel<<<grid_for(D), 256, 0, s>>>(Fmi.p(), Fae.p(), Wmbej.p(), Wabef.p(), t2->p(), v_oovv->p(),
                                                   op.diag.p, op.mdiag.p, o, v);
  GFCC_LAUNCH_CHECK();

  // ---- free terms (IP form, -b_q) and left vectors c_p -------------------------------------
  c->bvec.alloc((long long)n * D);
  c->cvec.alloc((long long)n * D);
  build_b_ea_kernel<<<grid_for((long long)n * D), 256, 0, s>>>(t1->p(), t2->p(), c->bvec.p, o, v);
  GFCC_LAUNCH_CHECK();
  {
    Tensor X2("ac", {v, v});                                                    // t_kl^ad l_cd^kl
    contract(1.0, t2->as("klad"), l2->as("klcd"), 0.0, X2.as("ac"), s);
    build_c_ea_kernel<<<grid_for((long long)n * D), 256, 0, s>>>(t1->p(), l1->p(), l2->p(), X2.p(),
                                                                 c->cvec.p, o, v);
    GFCC_LAUNCH_CHECK();
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gfcc
