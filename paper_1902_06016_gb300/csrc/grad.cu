// Gradient of the Green's function with respect to the doubles amplitudes T2 (adjoint method).
//
// For weights Gbar (the upstream gradient of an autograd backward pass) the function
//   L = Re sum_{w,p,q} conj(Gbar_wpq) G_pq(w),   G_pq(w) = c_q^T A(w)^{-1} b_p  (Eq. gfcclineqn)
// has, with x_wp = A(w)^{-1} b_p and u_wp = A(w)^{-T} sum_q conj(Gbar_wpq) c_q (adjoint solves with the
// transposed sigma), the derivative
//   dL/dt = Re sum_wpq conj(Gbar_wpq) (dc_q/dt)^T x_wp + Re sum_wp u_wp^T (db_p/dt) - Re sum_wp u_wp^T (dM/dt) x_wp.
// The last term is the bilinear form of the sigma equations (the same terms as the forward sigma,
// written with the full antisymmetric 2h1p amplitudes u~ and r):
//   s_i    = -F_ki r_k + F_kc r_ik^c - 1/2 W_klic r_kl^c
//   s_ij^a = -W_kaij r_k + F_ac r_ij^c - P(ij) F_ki r_kj^a + 1/2 W_klij r_kl^a + P(ij) W_kaci r_kj^c
//            - 1/2 (<kl||cd> r_kl^c) t_ij^ad
// so that the gradient of each H-bar element is a contraction of u~ with r over the frequency, orbital
// and index labels; these are propagated back through the H-bar build (the text after Eq. gfxn1
// defines Hbar = e^{-T} H e^{T}; the elements and their T2 dependence are those of the forward build)
// to T2. Forward X and adjoint U are recomputed here, not stored by the forward pass.
#include "gfcc_internal.cuh"
#include "tensor.h"

#include <algorithm>
#include <cmath>

namespace gfcc {

namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

__device__ __forceinline__ int pair_of(int i, int j) { return j * (j - 1) / 2 + i; }   // i < j

// W[nu][s] = sum_q conj(Gbar[s][q]) cvec[qrow[q]][nu], s = w np + p
__global__ void adjoint_rhs_kernel(const double* __restrict__ cvec, long long D, const int* __restrict__ qrow, int nq,
                                   const cplx* __restrict__ Gbar, long long S, cplx* __restrict__ W) {
  const long long total = D * S;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long nu = t / S, sidx = t % S;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double cv = cvec[(long long)qrow[q] * D + nu];
      const cplx g = Gbar[sidx * nq + q];
      re += g.x * cv;
      im -= g.y * cv;
    }
    W[t] = make_cuDoubleComplex(re, im);
  }
}

// Z (batch-minor [D][S] complex) -> real tensors Z1[s][z][i] and Z2[s][z][i][j][a] (full antisymmetric
// in i, j); z = 0 real part, z = 1 imaginary part times sgn (sgn = -1 makes sum_z u_z r_z = Re(u r))
// columns s0 .. s0 + S - 1 of the batch-minor block Z [D][ldS]
__global__ void unpack_kernel(const cplx* __restrict__ Zb, long long ldS, long long s0, long long S, int o, int v,
                              double sgn, double* __restrict__ Z1, double* __restrict__ Z2) {
  const cplx* Z = Zb + s0;
  const long long per = (long long)o + (long long)o * o * v;
  const long long total = S * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long sidx = t / per, e = t % per;
    if (e < o) {
      const cplx x = Z[e * ldS + sidx];
      Z1[(sidx * 2 + 0) * o + e] = x.x;
      Z1[(sidx * 2 + 1) * o + e] = sgn * x.y;
    } else {
      const long long r = e - o;
      const int i = (int)(r / ((long long)o * v)), j = (int)((r / v) % o), a = (int)(r % v);
      double re = 0.0, im = 0.0;
      if (i != j) {
        const int lo = min(i, j), hi = max(i, j);
        const cplx x = Z[((long long)o + (long long)pair_of(lo, hi) * v + a) * ldS + sidx];
        const double f = i < j ? 1.0 : -1.0;
        re = f * x.x;
        im = f * x.y;
      }
      const long long base = (long long)o * o * v;
      Z2[(sidx * 2 + 0) * base + r] = re;
      Z2[(sidx * 2 + 1) * base + r] = sgn * im;
    }
  }
}

// cbar1[i][k] += Re sum_{w,p} conj(Gbar[w p][q]) X[k][w p] for the occupied q = i of the q set
__global__ void cterm_kernel(const cplx* __restrict__ X, long long S, const cplx* __restrict__ Gbar, int nq,
                             const int* __restrict__ qrow, int o, double* __restrict__ cbar1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * o) return;
  const int q = t / o, k = t % o;
  const int i = qrow[q];
  if (i >= o) return;
  double acc = 0.0;
  for (long long sidx = 0; sidx < S; ++sidx) {
    const cplx g = Gbar[sidx * nq + q], x = X[(long long)k * S + sidx];
    acc += g.x * x.x + g.y * x.y;   // Re(conj(g) x)
  }
  atomicAdd(&cbar1[(long long)i * o + k], acc);
}

// b_a[o + pair(k,l) v + c] = t_kl^ac for the virtual p = o + a:  t2bar[k][l][a][c] += Re sum_w u_wp[...]
__global__ void bterm_kernel(const cplx* __restrict__ U, long long S, int nw, int np, const int* __restrict__ prow,
                             int o, int v, double* __restrict__ t2bar) {
  const int P = o * (o - 1) / 2;
  const long long total = (long long)np * P * v;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / ((long long)P * v));
    const long long r = t % ((long long)P * v);
    if (prow[p] < o) continue;
    const int a = prow[p] - o;
    const int pkl = (int)(r / v), cc = (int)(r % v);
    int l = (int)floorf((1.0f + sqrtf(1.0f + 8.0f * (float)pkl)) * 0.5f);
    while (l * (l - 1) / 2 > pkl) --l;
    while ((l + 1) * l / 2 <= pkl) ++l;
    const int k = pkl - l * (l - 1) / 2;
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += U[((long long)o + r) * S + (long long)w * np + p].x;
    atomicAdd(&t2bar[(((long long)k * o + l) * v + a) * v + cc], acc);
  }
}

}  // namespace

void green_adjoint_rhs(gfcc_ctx* c, const std::vector<int>& qorb, const cplx* Gbar_dev, long long S, cplx* W) {
  cudaStream_t s = c->stream;
  const int nq = (int)qorb.size();
  DBuf<int> qrow;
  qrow.alloc(nq);
  GFCC_CUDA(cudaMemcpyAsync(qrow.p, qorb.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
  adjoint_rhs_kernel<<<grid_for((long long)c->D * S), 256, 0, s>>>(c->cvec.p, c->D, qrow.p, nq, Gbar_dev, S, W);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(s));
}

void green_grad_t2_core(gfcc_ctx* c, int nw, const std::vector<int>& porb, const std::vector<int>& qorb,
                        const cplx* Gbar_dev, const cplx* Xp, const cplx* Up, double* t2bar_dev) {
  cudaStream_t s = c->stream;
  const int o = c->o, v = c->v;
  const int np = (int)porb.size(), nq = (int)qorb.size();
  const long long S = (long long)nw * np;
  DBuf<int> qrow, prow;
  qrow.alloc(nq);
  prow.alloc(np);
  GFCC_CUDA(cudaMemcpyAsync(qrow.p, qorb.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(prow.p, porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
  GFCC_CHECK(S < (1LL << 31), GFCC_ERR_ARG, "gradient: too many columns");

  // ---- gradients of the H-bar elements from the sigma bilinear form ------------------------------
  // Every term is a sum over the columns s, so the columns are unpacked and contracted in chunks whose
  // unpacked blocks (and the contractions' operand copies) stay within a few GB.
  Tensor Fmi("ki", {o, o}), Fae("ac", {v, v}), Wmbij("kaij", {o, v, o, o}), Wmnij("klij", {o, o, o, o}),
      Wmbej("kaci", {o, v, v, o}), t2bar("ijab", {o, o, v, v}), tau("ijab", {o, o, v, v});
  t2bar.buf.zero(s);
  tau.buf.zero(s);
  {
    const long long per_col = 2LL * ((long long)o + (long long)o * o * v) * (long long)sizeof(double);
    const long long budget = 3LL << 30;   // bytes of one unpacked block (U2 or R2) per chunk
    const int chunk = (int)std::max<long long>(1, std::min<long long>(S, budget / per_col));
    for (long long s0 = 0; s0 < S; s0 += chunk) {
      const int Si = (int)std::min<long long>(chunk, S - s0);
      const double b0 = s0 == 0 ? 0.0 : 1.0;   // the first chunk sets, the later ones add
      Tensor U1("szi", {Si, 2, o}), U2("szija", {Si, 2, o, o, v});
      Tensor R1("szk", {Si, 2, o}), R2("szkla", {Si, 2, o, o, v});
      const long long nun = (long long)Si * ((long long)o + (long long)o * o * v);
      unpack_kernel<<<grid_for(nun), 256, 0, s>>>(Up, S, s0, Si, o, v, 1.0, U1.p(), U2.p());
      GFCC_LAUNCH_CHECK();
      unpack_kernel<<<grid_for(nun), 256, 0, s>>>(Xp, S, s0, Si, o, v, -1.0, R1.p(), R2.p());
      GFCC_LAUNCH_CHECK();
      // L_M = -Re sum_s u_s^T sigma(x_s); sum over i<j of u sigma = 1/2 sum over all i, j (antisymmetric)
      contract(1.0, U1.as("szi"), R1.as("szk"), b0, Fmi.as("ki"), s);            // -F_ki r_k in s_i
      contract(1.0, U2.as("szija"), R2.as("szkja"), 1.0, Fmi.as("ki"), s);        // -P(ij) F_ki r_kj^a
      contract(-0.5, U2.as("szija"), R2.as("szijc"), b0, Fae.as("ac"), s);       // F_ac r_ij^c
      contract(0.5, U2.as("szija"), R1.as("szk"), b0, Wmbij.as("kaij"), s);      // -W_kaij r_k
      contract(-0.25, U2.as("szija"), R2.as("szkla"), b0, Wmnij.as("klij"), s);  // 1/2 W_klij r_kl^a
      contract(-1.0, U2.as("szija"), R2.as("szkjc"), b0, Wmbej.as("kaci"), s);   // P(ij) W_kaci r_kj^c
      {  // three-body term -1/2 (<kl||cd> r_kl^c) t_ij^ad, explicit in T2
        Tensor Xd("szd", {Si, 2, v});
        const TV voovv{c->k_oovv.p, "klcd", {o, o, v, v}};
        contract(1.0, voovv, R2.as("szklc"), 0.0, Xd.as("szd"), s);
        contract(0.25, U2.as("szija"), Xd.as("szd"), 1.0, t2bar.as("ijad"), s);
      }
      GFCC_CUDA(cudaStreamSynchronize(s));   // the chunk's blocks are released at the end of this scope
    }
  }

  // ---- back through the H-bar build ----------------------------------------------------------------
  const TV t1{c->t1.p, "", {o, v}};
  const TV Fme{c->k_Fme.p, "", {o, v}};
  const TV voovv{c->k_oovv.p, "", {o, o, v, v}};
  const TV vooov{c->k_ooov.p, "", {o, o, o, v}};
  const TV vovvv{c->k_ovvv.p, "", {o, v, v, v}};
  const TV l2{c->k_l2.p, "", {o, o, v, v}};
  auto L = [](const TV& t, const char* lab) { return TV{t.p, lab, t.d}; };
  // Wmbij labels "mbij" below = element [m][b][i][j]
  const TV Wb = Wmbij.as("mbij");
  Tensor Xb("mbej", {o, v, v, o}), Yb("mbej", {o, v, v, o});
  //   + t_i^e X_mbej - t_j^e X_mbei  with X = <mb||ej> - Y_mbej
  contract(1.0, L(t1, "ie"), Wb, 0.0, Xb.as("mbej"), s);
  contract(-1.0, L(t1, "je"), Wb, 1.0, Xb.as("mbei"), s);
  perm(Xb.as("mbej"), -1.0, 0.0, Yb.as("mbej"), s);
  //   + <mn||ie> t_jn^be - <mn||je> t_in^be
  contract(1.0, L(vooov, "mnie"), Wb, 1.0, t2bar.as("jnbe"), s);
  contract(-1.0, L(vooov, "mnje"), Wb, 1.0, t2bar.as("inbe"), s);
  //   + 1/2 <mb||ef> tau_ij^ef
  contract(0.5, L(vovvv, "mbef"), Wb, 1.0, tau.as("ijef"), s);
  //   - t_n^b W_mnij
  contract(-1.0, L(t1, "nb"), Wb, 1.0, Wmnij.as("mnij"), s);
  //   - F_me t_ij^be
  contract(-1.0, L(Fme, "me"), Wb, 1.0, t2bar.as("ijbe"), s);
  // W_mbej = ... - Y_mbej,  Y_mbej = t_jn^fb <mn||ef>
  perm(Wmbej.as("mbej"), -1.0, 1.0, Yb.as("mbej"), s);
  contract(1.0, L(voovv, "mnef"), Yb.as("mbej"), 1.0, t2bar.as("jnfb"), s);
  // W_mnij = ... + 1/2 tau_ij^ef <mn||ef>
  contract(0.5, L(voovv, "mnef"), Wmnij.as("mnij"), 1.0, tau.as("ijef"), s);
  // F_ae = ... - 1/2 tau_mn^af <mn||ef>;  F_mi = ... + 1/2 tau_in^ef <mn||ef>
  contract(-0.5, L(voovv, "mnef"), Fae.as("ae"), 1.0, tau.as("mnaf"), s);
  contract(0.5, L(voovv, "mnef"), Fmi.as("mi"), 1.0, tau.as("inef"), s);
  // tau = t2 + t1 t1 - t1 t1
  perm(tau.as("ijab"), 1.0, 1.0, t2bar.as("ijab"), s);

  // ---- free terms and left vectors -------------------------------------------------------------
  {  // c_i[k] = d_ik - t_i^e l_e^k - 1/2 t_in^ef l_ef^kn for occupied q = i
    Tensor cb("ik", {o, o});
    cb.buf.zero(s);
    cterm_kernel<<<(nq * o + 127) / 128, 128, 0, s>>>(Xp, S, Gbar_dev, nq, qrow.p, o, cb.p());
    GFCC_LAUNCH_CHECK();
    contract(-0.5, cb.as("ik"), L(l2, "knef"), 1.0, t2bar.as("inef"), s);
  }
  bterm_kernel<<<grid_for((long long)np * c->P * v), 256, 0, s>>>(Up, S, nw, np, prow.p, o, v, t2bar.p());
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaMemcpyAsync(t2bar_dev, t2bar.p(), sizeof(double) * t2bar.size(), cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gfcc
