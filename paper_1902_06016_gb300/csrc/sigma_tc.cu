// Low-precision sigma on the tcgen05 tensor cores, for the inner (Krylov) steps of the iterative
// refinement: every GEMM-shaped term of the sigma runs as one tc_gemm launch with bf16 or tf32
// operands and FP32 accumulation; the Fock diagonal, the shift and the small 1h-1h block are applied
// in FP64 in the final combine. The residuals that decide convergence always use the FP64 sigma.
//
//   up:   [Xe ; Y1'] ((v+o) x 2nb) = [Vt ; A12] ((v+o) x Pv) . r2          (split-K over Pv)
//   oooo: C2[(pij,a)][(c,r)]       = Woo (P x P) . r2 arranged [(a,c,r)][pmn]
//   down: C2 += [T2p | A21] (Pv x (v+o)) . [Xe ; r1]
//   ring: CT[(a,i)][(j,c,r)]       = Wr (ov x ov) . U,  U[(j,c,r)][(m,e)] = r_mj^e
#include "gfcc_internal.cuh"
#include "ozaki.cuh"
#include "tc_gemm.cuh"

#include <nvtx3/nvToolsExt.h>

#include <cuda_bf16.h>

#include <algorithm>

namespace gfcc {
namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

__device__ __forceinline__ int pair_of(int i, int j) { return j * (j - 1) / 2 + i; }
__device__ __forceinline__ void unpair(int p, int& i, int& j) {
  // FP32 estimate (GB300's FP64 pipe is narrow), corrected to the exact integer below
  int jj = (int)floorf((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
  while (jj * (jj - 1) / 2 > p) --jj;
  while ((jj + 1) * jj / 2 <= p) ++jj;
  j = jj;
  i = p - jj * (jj - 1) / 2;
}

// real type of a complex vector element: the FP32 Krylov path keeps all its arithmetic in FP32
template <typename VT> struct VReal;
template <> struct VReal<cplx> { using type = double; };
template <> struct VReal<cuFloatComplex> { using type = float; };

// element conversion (round to nearest)
template <TcKind K> struct Elem;
template <> struct Elem<TcKind::BF16> {
  using T = __nv_bfloat16;
  __device__ static T cvt(double x) { return __double2bfloat16(x); }
  __device__ static T cvt(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Elem<TcKind::TF32> {
  using T = float;
  __device__ static T cvt(double x) { return cvt((float)x); }
  __device__ static T cvt(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
};
struct F64Elem {   // FP64 staging for the exact-slice path
  using T = double;
  __device__ static T cvt(double x) { return x; }
};

// dst[r][k] = src[r*ld + k] for k < K, 0 for K <= k < kpad
template <TcKind K>
__global__ void convert_rows_kernel(const double* __restrict__ src, long long ld, long long rows, long long Kc,
                                    typename Elem<K>::T* __restrict__ dst, int kpad) {
  long long total = rows * kpad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t / kpad, k = t % kpad;
    dst[t] = Elem<K>::cvt(k < Kc ? src[r * ld + k] : 0.0);
  }
}
// [T2p | A21]: dst[row][e] = T2p[row][e] (e < v), dst[row][v+m] = A21[row][m] (m < o), rest 0
template <typename E>
__global__ void convert_down_kernel(const double* __restrict__ T2p, const double* __restrict__ A21, long long rows,
                                    int v, int o, typename E::T* __restrict__ dst, int kpad) {
  long long total = rows * kpad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long r = t / kpad;
    int k = (int)(t % kpad);
    double x = 0.0;
    if (k < v) x = T2p[r * v + k];
    else if (k < v + o) x = A21[r * o + (k - v)];
    dst[t] = E::cvt(x);
  }
}

// ---- per-batch operand preparation from the batch-minor block X[nu][c] (complex) ----------------
// Each prepared operand is a transpose of blocks of X into K-major real rows:
//   up:   B[c*2 + r][k]             = r-component of X[o + k][c],                 k < P v
//   oooo: B[(a*nb + c)*2 + r][k]    = r-component of X[o + k v + a][c],           k < P
//   ring: U[(j*nb + c)*2 + r][m v + e] = +-r-component of X[o + pair(m,j) v + e][c] (+ for m < j,
//         - for m > j, 0 for m = j),                                              e < v
// Tiles of 32 k x 32 c go through shared memory, so that X is read along c and the operand written
// along k (both coalesced); the K padding columns are zeroed by zero_pad_kernel.
enum PrepKind { PREP_UP = 0, PREP_OOOO = 1, PREP_RING = 2 };
constexpr int PT = 32;
template <typename E, typename VT, int KIND>
__global__ void __launch_bounds__(256) prep_tiled_kernel(const VT* __restrict__ X, int o, int v, int nb,
                                                         typename E::T* __restrict__ out, int kpad) {
  using R = typename VReal<VT>::type;
  __shared__ VT tile[PT][PT + 1];
  const int g = blockIdx.z;
  const int k0 = blockIdx.x * PT, c0 = blockIdx.y * PT;
  const long long P = (long long)o * (o - 1) / 2;
  long long rowblk = 0, kofs = 0, xbase = o, xstep = 1;
  int klen = 0;
  bool neg = false, zero = false;
  if (KIND == PREP_UP) {
    klen = (int)(P * v);
  } else if (KIND == PREP_OOOO) {
    rowblk = g; klen = (int)P; xbase = o + g; xstep = v;
  } else {
    const int j = g / o, m = g % o;
    rowblk = j; kofs = (long long)m * v; klen = v;
    zero = (m == j);
    neg = m > j;
    const int lo = min(m, j), hi = max(m, j);
    xbase = o + (long long)pair_of(lo, hi) * v;
  }
  if (k0 >= klen) return;
  for (int kk = threadIdx.y; kk < PT; kk += blockDim.y) {
    const int k = k0 + kk, c = c0 + threadIdx.x;
    VT x;
    x.x = R(0); x.y = R(0);
    if (!zero && k < klen && c < nb) x = X[(xbase + (long long)k * xstep) * nb + c];
    tile[kk][threadIdx.x] = x;
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k >= klen) return;
  for (int rr = threadIdx.y; rr < 2 * PT; rr += blockDim.y) {
    const int cc = rr >> 1, r = rr & 1, c = c0 + cc;
    if (c < nb) {
      const VT x = tile[threadIdx.x][cc];
      const R comp = r ? x.y : x.x;
      out[((rowblk * nb + c) * 2 + r) * (long long)kpad + kofs + k] = E::cvt(neg ? -comp : comp);
    }
  }
}
// out[row][k] = 0 for kfrom <= k < kpad
template <typename E>
__global__ void zero_pad_kernel(typename E::T* __restrict__ out, long long rows, int kfrom, int kpad) {
  const int w = kpad - kfrom;
  const long long total = rows * w;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    out[(t / w) * kpad + kfrom + t % w] = E::cvt(0.0);
}
template <typename E, typename VT, int KIND>
void prep_operand(const VT* X, int o, int v, int nb, typename E::T* out, int kpad, cudaStream_t s) {
  const long long P = (long long)o * (o - 1) / 2;
  const long long klen = KIND == PREP_UP ? P * v : (KIND == PREP_OOOO ? P : v);
  const int groups = KIND == PREP_UP ? 1 : (KIND == PREP_OOOO ? v : o * o);
  const long long rows = 2LL * nb * (KIND == PREP_UP ? 1 : (KIND == PREP_OOOO ? v : o));
  const long long kused = KIND == PREP_RING ? (long long)o * v : klen;
  GFCC_CHECK(groups <= 65535 && (klen + PT - 1) / PT < (1LL << 31), GFCC_ERR_ARG, "prep_operand: size");
  dim3 grid((unsigned)((klen + PT - 1) / PT), (unsigned)((nb + PT - 1) / PT), (unsigned)groups);
  prep_tiled_kernel<E, VT, KIND><<<grid, dim3(PT, 8), 0, s>>>(X, o, v, nb, out, kpad);
  GFCC_LAUNCH_CHECK();
  if (kpad > kused) {
    zero_pad_kernel<E><<<grid_for(rows * (kpad - kused)), 256, 0, s>>>(out, rows, (int)kused, kpad);
    GFCC_LAUNCH_CHECK();
  }
}


// ring: U[(j*nb + c)*2 + r][m*v + e] = r_mj^e (component r), K padded
// oooo: B[(a*nb + c)*2 + r][pmn] = X2[(pmn*v + a)][c].r
// up: B[c*2 + r][kk] = X2[kk][c].r  (kk = pmn*v + f)
// sum split-K partials: out[i] = sum_z part[z*stride + i]
__global__ void reduce_splits_kernel(const float* __restrict__ part, int zs, long long stride, long long n,
                                     float* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < zs; ++z) s += part[z * stride + t];
    out[t] = s;
  }
}
// down operand: B[c*2 + r][e] = Xe[e][c*2 + r] (e < v), B[c*2+r][v+m] = X1[m][c].r
template <typename E, typename U, typename VT>
__global__ void prep_down_kernel(const U* __restrict__ up, long long ldu, const VT* __restrict__ X, int o, int v,
                                 int nb, typename E::T* __restrict__ B, int kpad) {
  const long long total = 2LL * nb * kpad;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    using R = typename VReal<VT>::type;
    int n = (int)(t / kpad);
    int k = (int)(t % kpad);
    R val = R(0);
    if (k < v) {
      val = (R)up[(long long)k * ldu + n];
    } else if (k < v + o) {
      const VT x = X[(long long)(k - v) * nb + (n >> 1)];
      val = (n & 1) ? x.y : x.x;
    }
    B[t] = E::cvt(val);
  }
}
// final combine into the FP64 output (FP32 or FP64 GEMM results)
template <typename F, typename VT>
__global__ void combine_lp_kernel(const VT* __restrict__ X, VT* __restrict__ Y, const F* __restrict__ up,
                                  long long ldu, const F* __restrict__ C2, const F* __restrict__ CT,
                                  const double* __restrict__ A11, const double* __restrict__ diag,
                                  const cplx* __restrict__ shift, int o, int v, long long D, int nb) {
  const long long total = D * nb;
  const long long ldct = 2LL * o * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    using R = typename VReal<VT>::type;
    const int c = (int)(t % nb);
    const long long nu = t / nb;
    const VT x = X[t];
    R dre = (R)diag[nu], dim = R(0);
    if (shift) { dre += (R)shift[c].x; dim = (R)shift[c].y; }
    R yr = dre * x.x - dim * x.y;
    R yi = dre * x.y + dim * x.x;
    if (nu < o) {
      const int i = (int)nu;
      yr += (R)up[(long long)(v + i) * ldu + 2 * c];
      yi += (R)up[(long long)(v + i) * ldu + 2 * c + 1];
      for (int m = 0; m < o; ++m) {
        const R a = (R)A11[(long long)i * o + m];
        const VT xm = X[(long long)m * nb + c];
        yr += a * xm.x;
        yi += a * xm.y;
      }
    } else {
      const long long row = nu - o;
      yr += (R)C2[row * 2 * nb + 2 * c];
      yi += (R)C2[row * 2 * nb + 2 * c + 1];
      int pij = (int)(row / v), a = (int)(row % v);
      int i, j;
      unpair(pij, i, j);
      const F* c1 = CT + ((long long)a * o + i) * ldct + ((long long)j * nb + c) * 2;
      const F* c2 = CT + ((long long)a * o + j) * ldct + ((long long)i * nb + c) * 2;
      yr += (R)c1[0] - (R)c2[0];
      yi += (R)c1[1] - (R)c2[1];
    }
    Y[t].x = yr;
    Y[t].y = yi;
  }
}

// dst[nu][k] = src[nu][c0 + k] (k < nk) and back
__global__ void cols_gather_kernel(const cplx* __restrict__ src, int lds, int c0, int nk, cplx* __restrict__ dst,
                                   long long D) {
  const long long total = D * nk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[(t / nk) * lds + c0 + (t % nk)];
}
__global__ void cols_scatter_kernel(const cplx* __restrict__ src, int nk, cplx* __restrict__ dst, int ldd, int c0,
                                    long long D) {
  const long long total = D * nk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    dst[(t / nk) * ldd + c0 + (t % nk)] = src[t];
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// The operator blocks in the roles the sigma GEMMs give them. M^T has the same structure as M with the
// blocks permuted: the ring runs on WrT (as in the FP64 transposed sigma), xe = T2p^T r2 replaces
// xe = Vt r2, the 1h <- 2h1p block is A21^T, the 2h1p <- 1h block A12^T, the three-body output block
// Vt^T, and Woo and A11 are transposed.
struct OpView {
  const double *Wr, *Woo, *Vt, *A12, *T2p, *A21, *A11;
};
static OpView op_view(gfcc_ctx* c, bool transpose) {
  Operator& op = c->op;
  if (!transpose) return {op.Wr.p, op.Woo.p, op.Vt.p, op.A12.p, op.T2p.p, op.A21.p, op.A11.p};
  build_transpose_operator(c);
  if (!op.have_X) {
    const int o = c->o, v = c->v, P = c->P;
    const long long Pv = (long long)P * v;
    cudaStream_t s = c->stream;
    auto tr = [&](const double* src, int rows, int cols, DBuf<double>& dst) {   // dst[cols][rows] = src^T
      dst.alloc((long long)rows * cols);
      int dims[2] = {rows, cols};
      int pm[2] = {1, 0};
      permute(src, dims, 2, pm, dst.p, 1.0, 0.0, s);
    };
    tr(op.Woo.p, P, P, op.WooX);
    tr(op.T2p.p, (int)Pv, v, op.VtX);     // T2p [Pv][v] -> [v][Pv]
    tr(op.A21.p, (int)Pv, o, op.A12X);    // A21 [Pv][o] -> [o][Pv]
    tr(op.Vt.p, v, (int)Pv, op.T2pX);     // Vt [v][Pv]  -> [Pv][v]
    tr(op.A12.p, o, (int)Pv, op.A21X);    // A12 [o][Pv] -> [Pv][o]
    tr(op.A11.p, o, o, op.A11X);
    GFCC_CUDA(cudaStreamSynchronize(s));
    op.have_X = true;
  }
  return {op.WrT.p, op.WooX.p, op.VtX.p, op.A12X.p, op.T2pX.p, op.A21X.p, op.A11X.p};
}

struct LpState {
  TcKind kind;
  int Kr = 0, Kp = 0, Kpv = 0, Kvo = 0;
  DBuf<uint8_t> Wr, Woo, Aup, Adn;            // operands (bf16 or fp32 elements)
  DBuf<uint8_t> Bring, Boo, Bup, Bdn;         // per-batch operands
  DBuf<float> CT, C2, up_part, up;            // outputs
  DBuf<int> err;
  int nb_cap = 0, ksplit = 1;
};

static LpState* lp_state(gfcc_ctx* c, bool transpose = false) {
  return reinterpret_cast<LpState*>(transpose ? c->lp.implT : c->lp.impl);
}

// FP64-accurate sigma from exact bf16 slices (residuals of the iterative refinement)
struct EmuState {
  SlicedRows Wr, Woo, Aup, Adn;
  DBuf<double> stage, CT, C2, up;
  SlicedRows Bring, Boo, Bup, Bdn;
  DBuf<cplx> Xc, Yc;
  OzWork work;
};
static EmuState* emu_state(gfcc_ctx* c, bool transpose = false) {
  return reinterpret_cast<EmuState*>(transpose ? c->lp.emuT : c->lp.emu);
}

void free_low_precision(gfcc_ctx* c) {
  delete lp_state(c);
  delete lp_state(c, true);
  c->lp.impl = nullptr;
  c->lp.implT = nullptr;
  c->lp.kind = 0;
  delete emu_state(c);
  delete emu_state(c, true);
  c->lp.emu = nullptr;
  c->lp.emuT = nullptr;
}

// Free the per-batch buffers of the low-precision and exact-slice states (both actions): they are
// allocated again, at the size needed, by the next sigma. The operands and the error flags stay.
void release_sigma_batch_buffers(gfcc_ctx* c) {
  for (bool tr : {false, true}) {
    if (LpState* st = lp_state(c, tr)) {
      for (DBuf<uint8_t>* b : {&st->Bring, &st->Boo, &st->Bup, &st->Bdn}) b->release();
      for (DBuf<float>* b : {&st->CT, &st->C2, &st->up_part, &st->up}) b->release();
      st->nb_cap = 0;
    }
    if (EmuState* st = emu_state(c, tr)) {
      for (DBuf<double>* b : {&st->stage, &st->CT, &st->C2, &st->up}) b->release();
      for (SlicedRows* r : {&st->Bring, &st->Boo, &st->Bup, &st->Bdn}) {
        r->slices.release();
        r->expo.release();
      }
      st->Xc.release();
      st->Yc.release();
      st->work.islabs.release();
      st->work.acc.release();
    }
  }
}

static void build_emulated(gfcc_ctx* c, bool transpose) {
  if (transpose ? c->lp.emuT : c->lp.emu) return;
  const int o = c->o, v = c->v, P = c->P;
  const long long ov = (long long)o * v, Pv = (long long)P * v;
  cudaStream_t s = c->stream;
  const OpView ov_ = op_view(c, transpose);
  auto* st = new EmuState();
  (transpose ? c->lp.emuT : c->lp.emu) = st;
  oz_slice(ov_.Wr, ov, ov, ov, false, st->Wr, s);
  oz_slice(ov_.Woo, P, P, P, false, st->Woo, s);
  st->Aup.rows = v + o;
  st->Aup.kp = tc_pad_k(TcKind::BF16, Pv);
  st->Aup.reversed = false;
  st->Aup.ns = OZ_SLICES;
  st->Aup.slices.alloc(2LL * (v + o) * OZ_SLICES * st->Aup.kp);
  st->Aup.expo.alloc(v + o);
  oz_slice_into(ov_.Vt, Pv, v, Pv, st->Aup, 0, s);
  oz_slice_into(ov_.A12, Pv, o, Pv, st->Aup, v, s);
  st->stage.alloc(Pv * (v + o));
  convert_down_kernel<F64Elem><<<grid_for(Pv * (v + o)), 256, 0, s>>>(ov_.T2p, ov_.A21, Pv, v, o, st->stage.p, v + o);
  GFCC_LAUNCH_CHECK();
  oz_slice(st->stage.p, v + o, Pv, v + o, false, st->Adn, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
}

void build_emulated(gfcc_ctx* c) { build_emulated(c, false); }

void sigma_emulated(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, const cplx* shift, cudaStream_t s, bool transpose) {
  build_emulated(c, transpose);
  EmuState& st = *emu_state(c, transpose);
  const double* A11 = op_view(c, transpose).A11;
  const int o = c->o, v = c->v, P = c->P;
  const long long ov = (long long)o * v, Pv = (long long)P * v, D = c->D;
  const int chunk = 64;
  for (int c0 = 0; c0 < nb; c0 += chunk) {
    const int nbc = std::min(chunk, nb - c0);
    const long long nring = 2LL * o * nbc, noo = 2LL * v * nbc, nsm = 2LL * nbc;
    st.Xc.alloc(D * chunk);
    st.Yc.alloc(D * chunk);
    st.stage.alloc(std::max({nring * ov, noo * (long long)P, nsm * Pv, nsm * (long long)(v + o), Pv * (v + o)}));
    st.CT.alloc(ov * 2LL * o * chunk);
    st.C2.alloc(Pv * 2LL * chunk);
    st.up.alloc((long long)(v + o) * 2LL * chunk);
    cols_gather_kernel<<<grid_for(D * nbc), 256, 0, s>>>(X, nb, c0, nbc, st.Xc.p, D);
    GFCC_LAUNCH_CHECK();
    // up: [Xe ; Y1'] = [Vt ; A12] r2
    prep_operand<F64Elem, cplx, PREP_UP>(st.Xc.p, o, v, nbc, st.stage.p, (int)Pv, s);
    oz_slice(st.stage.p, Pv, nsm, Pv, true, st.Bup, s);
    oz_gemm(st.Aup, st.Bup, v + o, nsm, st.up.p, nsm, 0.0, st.work, s);
    // oooo into C2
    prep_operand<F64Elem, cplx, PREP_OOOO>(st.Xc.p, o, v, nbc, st.stage.p, P, s);
    oz_slice(st.stage.p, P, noo, P, true, st.Boo, s);
    oz_gemm(st.Woo, st.Boo, P, noo, st.C2.p, noo, 0.0, st.work, s);
    // down: C2 += [T2p | A21] [Xe ; r1]
    prep_down_kernel<F64Elem, double, cplx><<<grid_for(nsm * (v + o)), 256, 0, s>>>(st.up.p, nsm, st.Xc.p, o, v, nbc,
                                                                             st.stage.p, v + o);
    GFCC_LAUNCH_CHECK();
    oz_slice(st.stage.p, v + o, nsm, v + o, true, st.Bdn, s);
    oz_gemm(st.Adn, st.Bdn, Pv, nsm, st.C2.p, nsm, 1.0, st.work, s);
    // ring
    prep_operand<F64Elem, cplx, PREP_RING>(st.Xc.p, o, v, nbc, st.stage.p, (int)ov, s);
    oz_slice(st.stage.p, ov, nring, ov, true, st.Bring, s);
    oz_gemm(st.Wr, st.Bring, ov, nring, st.CT.p, nring, 0.0, st.work, s);
    combine_lp_kernel<double, cplx><<<grid_for(D * nbc), 256, 0, s>>>(st.Xc.p, st.Yc.p, st.up.p, nsm, st.C2.p, st.CT.p,
                                                                A11, c->op.diag.p,
                                                                shift ? shift + c0 : nullptr, o, v, D, nbc);
    GFCC_LAUNCH_CHECK();
    cols_scatter_kernel<<<grid_for(D * nbc), 256, 0, s>>>(st.Yc.p, nbc, Y, nb, c0, D);
    GFCC_LAUNCH_CHECK();
  }
  c->stats.sigma_calls++;
  c->stats.sigma_cols += nb;
}

int emulated_error(gfcc_ctx* c) {
  int any = 0;
  for (bool tr : {false, true}) {
    EmuState* st = emu_state(c, tr);
    if (!st || st->work.err.n == 0) continue;
    int h = 0;
    GFCC_CUDA(cudaMemcpyAsync(&h, st->work.err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
    any |= h;
  }
  return any;
}

template <TcKind K>
static void build_ops(gfcc_ctx* c, LpState& st, const OpView& w) {
  using T = typename Elem<K>::T;
  const int o = c->o, v = c->v, P = c->P;
  const long long ov = (long long)o * v, Pv = (long long)P * v;
  cudaStream_t s = c->stream;
  st.Kr = tc_pad_k(K, ov);
  st.Kp = tc_pad_k(K, P);
  st.Kpv = tc_pad_k(K, Pv);
  st.Kvo = tc_pad_k(K, v + o);
  st.Wr.alloc(sizeof(T) * ov * st.Kr);
  convert_rows_kernel<K><<<grid_for(ov * st.Kr), 256, 0, s>>>(w.Wr, ov, ov, ov, reinterpret_cast<T*>(st.Wr.p), st.Kr);
  GFCC_LAUNCH_CHECK();
  st.Woo.alloc(sizeof(T) * (long long)P * st.Kp);
  convert_rows_kernel<K><<<grid_for((long long)P * st.Kp), 256, 0, s>>>(w.Woo, P, P, P, reinterpret_cast<T*>(st.Woo.p),
                                                                       st.Kp);
  GFCC_LAUNCH_CHECK();
  st.Aup.alloc(sizeof(T) * (long long)(v + o) * st.Kpv);
  convert_rows_kernel<K><<<grid_for((long long)v * st.Kpv), 256, 0, s>>>(w.Vt, Pv, v, Pv,
                                                                        reinterpret_cast<T*>(st.Aup.p), st.Kpv);
  GFCC_LAUNCH_CHECK();
  convert_rows_kernel<K><<<grid_for((long long)o * st.Kpv), 256, 0, s>>>(
      w.A12, Pv, o, Pv, reinterpret_cast<T*>(st.Aup.p) + (long long)v * st.Kpv, st.Kpv);
  GFCC_LAUNCH_CHECK();
  st.Adn.alloc(sizeof(T) * Pv * st.Kvo);
  convert_down_kernel<Elem<K>><<<grid_for(Pv * st.Kvo), 256, 0, s>>>(w.T2p, w.A21, Pv, v, o,
                                                               reinterpret_cast<T*>(st.Adn.p), st.Kvo);
  GFCC_LAUNCH_CHECK();
  st.err.alloc(1);
  st.err.zero(s);
  GFCC_CUDA(cudaStreamSynchronize(s));
}

void build_low_precision(gfcc_ctx* c, int kind) {
  GFCC_CHECK(kind == GFCC_PREC_BF16 || kind == GFCC_PREC_TF32, GFCC_ERR_ARG, "low precision: bf16 or tf32 only");
  if (c->lp.kind == kind && c->lp.impl) return;
  free_low_precision(c);
  auto* st = new LpState();
  c->lp.impl = st;
  st->kind = kind == GFCC_PREC_BF16 ? TcKind::BF16 : TcKind::TF32;
  if (st->kind == TcKind::BF16) build_ops<TcKind::BF16>(c, *st, op_view(c, false));
  else build_ops<TcKind::TF32>(c, *st, op_view(c, false));
  c->lp.kind = kind;
}

// the low-precision operands of M^T, in the kind of the forward ones (built on first use)
static LpState* lp_state_transposed(gfcc_ctx* c) {
  if (!c->lp.implT) {
    LpState* f = lp_state(c);
    GFCC_CHECK(f != nullptr, GFCC_ERR_STATE, "low-precision operator not built");
    auto* st = new LpState();
    c->lp.implT = st;
    st->kind = f->kind;
    if (st->kind == TcKind::BF16) build_ops<TcKind::BF16>(c, *st, op_view(c, true));
    else build_ops<TcKind::TF32>(c, *st, op_view(c, true));
  }
  return lp_state(c, true);
}

int low_precision_error(gfcc_ctx* c) {
  if (emulated_error(c)) return 1;
  for (bool tr : {false, true}) {
    LpState* st = lp_state(c, tr);
    if (!st) continue;
    int h = 0;
    GFCC_CUDA(cudaMemcpyAsync(&h, st->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
    if (h) return 1;
  }
  return 0;
}

template <TcKind K, typename VT>
static void sigma_lp_impl(gfcc_ctx* c, LpState& st, const VT* X, VT* Y, int nb, const cplx* shift, cudaStream_t s,
                          const double* A11) {
  using T = typename Elem<K>::T;
  const int o = c->o, v = c->v, P = c->P;
  const long long ov = (long long)o * v, Pv = (long long)P * v, D = c->D;
  const long long nring = 2LL * o * nb, noo = 2LL * v * nb, nsm = 2LL * nb;
  if (nb > st.nb_cap) {
    st.Bring.alloc(sizeof(T) * nring * st.Kr);
    st.Boo.alloc(sizeof(T) * noo * st.Kp);
    st.Bup.alloc(sizeof(T) * nsm * st.Kpv);
    st.Bdn.alloc(sizeof(T) * nsm * st.Kvo);
    st.CT.alloc(ov * nring);
    st.C2.alloc(Pv * nsm);
    st.up.alloc((long long)(v + o) * nsm);
    st.nb_cap = nb;
  }
  // split-K for the short-and-wide "up" GEMM: about two waves of CTAs
  const int mt = (v + o + 127) / 128;
  const int nk_up = st.Kpv / tc_kblock(K);
  int ksplit = std::max(1, std::min(nk_up, (2 * 152) / std::max(1, mt * (int)((nsm + 255) / 256))));
  const long long part_stride = (long long)(v + o) * nsm;
  st.up_part.alloc(part_stride * ksplit);

  T* Bring = reinterpret_cast<T*>(st.Bring.p);
  T* Boo = reinterpret_cast<T*>(st.Boo.p);
  T* Bup = reinterpret_cast<T*>(st.Bup.p);
  T* Bdn = reinterpret_cast<T*>(st.Bdn.p);
  {
    ProfScope pp(PROF_LP_PREP, 0.0, s);
    prep_operand<Elem<K>, VT, PREP_UP>(X, o, v, nb, Bup, st.Kpv, s);
    prep_operand<Elem<K>, VT, PREP_OOOO>(X, o, v, nb, Boo, st.Kp, s);
    prep_operand<Elem<K>, VT, PREP_RING>(X, o, v, nb, Bring, st.Kr, s);
  }
  // The up, oooo and down products are short or thin (K = Pv split, K = P, K = v + o): each moves more
  // bytes than the tensor pipe needs time for, so they are also timed as one HBM-bound class whose
  // algorithmic bytes are both operands read once and the output written once (read and written for
  // the accumulating down product), at the operand element size es and FP32 outputs.
  const double es = sizeof(T);
  // up (split-K) and its reduction
  {
    ProfScope pb(PROF_LP_SMALL_GEMMS, es * (double)(v + o + nsm) * (double)Pv + 4.0 * (double)(v + o) * nsm, s);
    tc_gemm(K, TcOperand{st.Aup.p, v + o, st.Kpv}, TcOperand{Bup, nsm, st.Kpv}, st.up_part.p, nsm, v + o, nsm, 0,
            ksplit, part_stride, st.err.p, s);
  }
  {
    ProfScope pc(PROF_LP_COMBINE, 0.0, s);
    const int nk_split = (nk_up + ksplit - 1) / ksplit;
    const int zs = (nk_up + nk_split - 1) / nk_split;
    reduce_splits_kernel<<<grid_for(part_stride), 256, 0, s>>>(st.up_part.p, zs, part_stride, part_stride, st.up.p);
    GFCC_LAUNCH_CHECK();
  }
  // oooo into C2 (as [P][(a,c,r)] = [(pij,a)][(c,r)])
  {
    ProfScope pb(PROF_LP_SMALL_GEMMS, es * (double)(P + noo) * (double)P + 4.0 * (double)P * noo, s);
    tc_gemm(K, TcOperand{st.Woo.p, P, st.Kp}, TcOperand{Boo, noo, st.Kp}, st.C2.p, noo, P, noo, 0, 1, 0, st.err.p, s);
  }
  // down: C2 += [T2p | A21] [Xe ; r1]
  {
    ProfScope pp(PROF_LP_PREP, 0.0, s);
    prep_down_kernel<Elem<K>, float, VT><<<grid_for(nsm * st.Kvo), 256, 0, s>>>(st.up.p, nsm, X, o, v, nb, Bdn, st.Kvo);
    GFCC_LAUNCH_CHECK();
  }
  {
    ProfScope pb(PROF_LP_SMALL_GEMMS, es * (double)(Pv + nsm) * (double)(v + o) + 8.0 * (double)Pv * nsm, s);
    tc_gemm(K, TcOperand{st.Adn.p, Pv, st.Kvo}, TcOperand{Bdn, nsm, st.Kvo}, st.C2.p, nsm, Pv, nsm, 1, 1, 0, st.err.p,
            s);
  }
  // ring (its own profiling class and NVTX range, so that its launches can be timed and profiled alone)
  nvtxRangePushA("gfcc_ring_gemm");
  tc_gemm(K, TcOperand{st.Wr.p, ov, st.Kr}, TcOperand{Bring, nring, st.Kr}, st.CT.p, nring, ov, nring, 0, 1, 0,
          st.err.p, s, PROF_TC_RING, ov);
  nvtxRangePop();
  ProfScope pc(PROF_LP_COMBINE, 0.0, s);
  combine_lp_kernel<float, VT><<<grid_for(D * nb), 256, 0, s>>>(X, Y, st.up.p, nsm, st.C2.p, st.CT.p, A11, c->op.diag.p,
                                                     shift, o, v, D, nb);
  GFCC_LAUNCH_CHECK();
}

void sigma_lowprec(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, const cplx* shift, cudaStream_t s, bool transpose) {
  LpState* st = transpose ? lp_state_transposed(c) : lp_state(c);
  GFCC_CHECK(st != nullptr, GFCC_ERR_STATE, "low-precision operator not built");
  const double* A11 = op_view(c, transpose).A11;
  if (st->kind == TcKind::BF16) sigma_lp_impl<TcKind::BF16, cplx>(c, *st, X, Y, nb, shift, s, A11);
  else sigma_lp_impl<TcKind::TF32, cplx>(c, *st, X, Y, nb, shift, s, A11);
  c->stats.sigma_calls++;
  c->stats.sigma_cols += nb;
}

void sigma_lowprec_f32(gfcc_ctx* c, const cuFloatComplex* X, cuFloatComplex* Y, int nb, const cplx* shift,
                       cudaStream_t s, bool transpose) {
  LpState* st = transpose ? lp_state_transposed(c) : lp_state(c);
  GFCC_CHECK(st != nullptr, GFCC_ERR_STATE, "low-precision operator not built");
  const double fo = c->o, fv = c->v, fP = c->P;   // algorithmic flops, as in sigma_batch
  ProfScope prof(PROF_SIGMA_LP,
                 2.0 * nb * (2.0 * fo * fv * fo * fv * fo + 2.0 * fP * fP * fv + 4.0 * fP * fv * fv + 4.0 * fo * fP * fv), s);
  const double* A11 = op_view(c, transpose).A11;
  if (st->kind == TcKind::BF16) sigma_lp_impl<TcKind::BF16, cuFloatComplex>(c, *st, X, Y, nb, shift, s, A11);
  else sigma_lp_impl<TcKind::TF32, cuFloatComplex>(c, *st, X, Y, nb, shift, s, A11);
  c->stats.sigma_calls++;
  c->stats.sigma_cols += nb;
}

// standalone low-precision GEMM check (C = A B^T) for tests of the tensor-core kernel itself
void tc_selftest(int kind, const double* A, const double* B, int M, int N, int K, float* C, cudaStream_t s) {
  const TcKind k = kind == GFCC_PREC_BF16 ? TcKind::BF16 : TcKind::TF32;
  const int kp = tc_pad_k(k, K);
  const size_t es = k == TcKind::BF16 ? 2 : 4;
  DBuf<uint8_t> a, b;
  DBuf<int> err;
  a.alloc(es * (size_t)M * kp);
  b.alloc(es * (size_t)N * kp);
  err.alloc(1);
  err.zero(s);
  if (k == TcKind::BF16) {
    convert_rows_kernel<TcKind::BF16><<<grid_for((long long)M * kp), 256, 0, s>>>(A, K, M, K, reinterpret_cast<__nv_bfloat16*>(a.p), kp);
    GFCC_LAUNCH_CHECK();
    convert_rows_kernel<TcKind::BF16><<<grid_for((long long)N * kp), 256, 0, s>>>(B, K, N, K, reinterpret_cast<__nv_bfloat16*>(b.p), kp);
    GFCC_LAUNCH_CHECK();
  } else {
    convert_rows_kernel<TcKind::TF32><<<grid_for((long long)M * kp), 256, 0, s>>>(A, K, M, K, reinterpret_cast<float*>(a.p), kp);
    GFCC_LAUNCH_CHECK();
    convert_rows_kernel<TcKind::TF32><<<grid_for((long long)N * kp), 256, 0, s>>>(B, K, N, K, reinterpret_cast<float*>(b.p), kp);
    GFCC_LAUNCH_CHECK();
  }
  GFCC_LAUNCH_CHECK();
  tc_gemm(k, TcOperand{a.p, M, kp}, TcOperand{b.p, N, kp}, C, N, M, N, 0, 1, 0, err.p, s);
  int h = 0;
  GFCC_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));
  GFCC_CHECK(h == 0, GFCC_ERR_CUDA, "tensor-core pipeline wait timed out");
}

}  // namespace gfcc
