// Batched restarted GMRES with iterative refinement for the shifted systems of Eq. xplin,
// (w_c - i eta + M) x_c = b_c, one column per (p, w) pair, all columns in lock step.
//
// Each restart cycle is one refinement step: the residual r = b - (shift x + M x) is formed with
// the FP64 sigma, then GMRES(k) on the correction runs with the sigma in the requested
// precision (classical Gram-Schmidt with one re-orthogonalisation, FP64 basis, Givens least
// squares), and x += P V y with the Jacobi right preconditioner P = (shift + diag M)^{-1}.
// Columns whose FP64 residual meets the tolerance are written out and compacted away between
// cycles. The paper used a complex DIIS solver (convergence study after Table 1); any convergent
// solver reaches the same solution of Eq. xplin.
#include "gfcc_internal.cuh"

#include <type_traits>

#include <algorithm>
#include <cmath>

namespace gfcc {
namespace {

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// real component type of a complex vector element
template <typename VT> struct RealOf;
template <> struct RealOf<cplx> { using type = double; };
template <> struct RealOf<cuFloatComplex> { using type = float; };

constexpr int MD_TX = 32, MD_TY = 8, MD_MAXV = 32;
// The kernels below are instantiated for NV = 4, 8, 16, 32 basis vectors (nv <= NV used).
template <typename F>
void with_nv(int nv, F&& f) {
  if (nv <= 4) f(std::integral_constant<int, 4>{});
  else if (nv <= 8) f(std::integral_constant<int, 8>{});
  else if (nv <= 16) f(std::integral_constant<int, 16>{});
  else f(std::integral_constant<int, 32>{});
}

// partial[chunk][i][c] = sum_{nu in chunk} conj(V_i[nu][c]) W[nu][c], i < nv (V_i = V + i*stride);
// per-thread sums in the vector's precision, partials written in FP64.
// Block (MD_TX columns) x (MD_TY): the MD_TY thread rows form IG = NV/8 groups (at least 1); group g
// owns the accumulators of basis vectors [g NPG, (g+1) NPG), NPG = NV / IG, and its threads stride the
// chunk's rows by MD_TY / IG. Fewer accumulators per thread keep the registers, and so the number of
// resident warps, independent of the basis size.
template <int NV> struct MdGroups {
  static constexpr int IG = NV >= 16 ? NV / 8 : 1;
  static constexpr int NPG = NV / IG;
  static constexpr int RPG = MD_TY / IG;   // thread rows per group
};
// sum the per-thread values acc[li] of group g over its RPG thread rows; partial for i = g NPG + li
template <typename VT, int NV, typename R>
__device__ __forceinline__ void md_reduce(const R (&ax)[MdGroups<NV>::NPG], const R (&ay)[MdGroups<NV>::NPG], int nv,
                                          int c, int nb, cplx* __restrict__ partial, cplx (*red)[MD_TX]) {
  using G = MdGroups<NV>;
  const int g = threadIdx.y / G::RPG, yr = threadIdx.y % G::RPG;
#pragma unroll
  for (int li = 0; li < G::NPG; ++li) {
    red[threadIdx.y][threadIdx.x] = make_cuDoubleComplex((double)ax[li], (double)ay[li]);
    __syncthreads();
    const int i = g * G::NPG + li;
    if (yr == 0 && c < nb && i < nv) {
      cplx s = red[threadIdx.y][threadIdx.x];
      for (int k = 1; k < G::RPG; ++k) { s.x += red[threadIdx.y + k][threadIdx.x].x; s.y += red[threadIdx.y + k][threadIdx.x].y; }
      partial[((long long)blockIdx.y * nv + i) * nb + c] = s;
    }
    __syncthreads();
  }
}

template <typename VT, int NV>
__global__ void __launch_bounds__(256, 2) multidot_kernel(const VT* __restrict__ V, long long vstride, int nv,
                                                          const VT* __restrict__ W, long long D, int nb,
                                                          long long rows_per_chunk, cplx* __restrict__ partial) {
  using R = typename RealOf<VT>::type;
  using G = MdGroups<NV>;
  __shared__ cplx red[MD_TY][MD_TX];
  const int c = blockIdx.x * MD_TX + threadIdx.x;
  const int g = threadIdx.y / G::RPG, yr = threadIdx.y % G::RPG;
  const long long r0 = blockIdx.y * rows_per_chunk;
  const long long r1 = min(D, r0 + rows_per_chunk);
  const VT* Vg = V + (long long)g * G::NPG * vstride;
  const int ng = nv - g * G::NPG;   // vectors of this group present (may be <= 0)
  R ax[G::NPG], ay[G::NPG];
#pragma unroll
  for (int i = 0; i < G::NPG; ++i) { ax[i] = R(0); ay[i] = R(0); }
  if (c < nb && ng > 0) {
    for (long long nu = r0 + yr; nu < r1; nu += G::RPG) {
      const VT w = W[nu * nb + c];
#pragma unroll
      for (int i = 0; i < G::NPG; ++i) {
        if (i < ng) {
          const VT vv = Vg[i * vstride + nu * nb + c];
          ax[i] += vv.x * w.x + vv.y * w.y;
          ay[i] += vv.x * w.y - vv.y * w.x;
        }
      }
    }
  }
  md_reduce<VT, NV, R>(ax, ay, nv, c, nb, partial, red);
}

// ---- pipelined Gram-Schmidt sweeps of the FP32 basis ---------------------------------------------
// The three sweeps of a CGS2 Arnoldi step with an FP32 basis (MODE 0: partial sums of conj(V_i) w, the
// layout of multidot_kernel's partials; 1: w -= V h, then partial sums
// of conj(V_i) w; 2: w -= V h, then partial sums of |w|^2), with the loads decoupled from the
// arithmetic: every thread streams its own elements (its NPG basis vectors and w at one row per step)
// through a SW_STAGES-deep ring in shared memory by 8-byte asynchronous copies (cp.async, zero-filled
// outside the batch), so that about three steps of loads are in flight per block without holding
// registers. A block is CW columns wide (32, 16, 8 or 4: narrow batches keep every thread busy) and
// SW_THREADS / CW thread rows high; the thread rows form MdGroups-like groups that each own NPG basis
// vectors (IG groups), and the groups' shares of V h are added through shared memory as above. Each
// thread reads only the ring slots it filled itself.
constexpr int SW_THREADS = 256, SW_STAGES = 4;
template <int NV> struct SwGroups {
  static constexpr int IG = NV >= 16 ? NV / 8 : 1;
  static constexpr int NPG = NV / IG;
};
template <int NV, int CW> constexpr size_t sweep_smem_bytes() {
  return sizeof(float2) * (size_t)SW_STAGES * (SwGroups<NV>::NPG + 1) * SW_THREADS   // load ring
         + sizeof(float2) * 2 * SW_THREADS                                           // shares
         + sizeof(cplx) * SW_THREADS;                                                // reductions
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NV, int MODE, int CW>
__global__ void __launch_bounds__(SW_THREADS, 2) sweep_kernel(const float2* __restrict__ V, long long vstride, int nv,
                                                              float2* __restrict__ W, long long D, int nb,
                                                              long long rows_per_chunk, const cplx* __restrict__ h,
                                                              int hld, cplx* __restrict__ partial) {
  constexpr int TY = SW_THREADS / CW, IG = SwGroups<NV>::IG, NPG = SwGroups<NV>::NPG, RPG = TY / IG;
  constexpr int SLOTS = NPG + 1;
  static_assert(TY % IG == 0, "thread rows per group");
  extern __shared__ __align__(16) unsigned char sw_raw[];
  float2* ring = reinterpret_cast<float2*>(sw_raw);                       // [SW_STAGES][SLOTS][SW_THREADS]
  float2* share = ring + (size_t)SW_STAGES * SLOTS * SW_THREADS;          // [2][TY][CW]
  cplx* red = reinterpret_cast<cplx*>(share + 2 * SW_THREADS);            // [TY][CW]
  const int tid = threadIdx.x, x = tid % CW, y = tid / CW;
  const int g = y / RPG, yr = y % RPG;
  const int c = blockIdx.x * CW + x;
  const int i0 = g * NPG, ng = nv - i0;
  const long long r0 = blockIdx.y * rows_per_chunk;
  const long long r1 = min(D, r0 + rows_per_chunk);
  const long long nsteps = (r1 - r0 + RPG - 1) / RPG;   // the same for every thread (barriers inside)
  const float2* Vg = V + (long long)i0 * vstride;
  auto issue = [&](long long t) {
    float2* st = ring + (size_t)(t % SW_STAGES) * SLOTS * SW_THREADS + tid;
    const long long nu = r0 + t * RPG + yr;
    const bool ok = c < nb && nu < r1;
    const long long off = ok ? nu * nb + c : 0;
    // predicated-off copies zero-fill and read nothing; they are given the valid base address V
#pragma unroll
    for (int li = 0; li < NPG; ++li) {
      const bool on = ok && li < ng;
      cp_async8(st + li * SW_THREADS, on ? Vg + li * vstride + off : V, on);
    }
    cp_async8(st + NPG * SW_THREADS, W + off, ok);
  };
  float2 hv[NPG];
#pragma unroll
  for (int li = 0; li < NPG; ++li) {
    const bool on = MODE != 0 && c < nb && li < ng;
    hv[li] = on ? make_float2((float)h[(long long)c * hld + i0 + li].x, (float)h[(long long)c * hld + i0 + li].y)
                : make_float2(0.f, 0.f);
  }
  float ax[NPG], ay[NPG];
#pragma unroll
  for (int li = 0; li < NPG; ++li) { ax[li] = 0.f; ay[li] = 0.f; }
  float nrm = 0.f;
#pragma unroll
  for (int t = 0; t < SW_STAGES - 1; ++t) {
    if (t < nsteps) issue(t);
    cp_async_commit();
  }
  for (long long t = 0; t < nsteps; ++t) {
    if (t + SW_STAGES - 1 < nsteps) issue(t + SW_STAGES - 1);
    cp_async_commit();
    cp_async_wait<SW_STAGES - 1>();   // this thread's copies of step t have landed
    const float2* st = ring + (size_t)(t % SW_STAGES) * SLOTS * SW_THREADS + tid;
    float2 w = st[NPG * SW_THREADS];
    float2 v[NPG];
#pragma unroll
    for (int li = 0; li < NPG; ++li) v[li] = st[li * SW_THREADS];
    const long long nu = r0 + t * RPG + yr;
    const bool ok = c < nb && nu < r1;
    if constexpr (MODE != 0) {
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int li = 0; li < NPG; ++li) {
        sx += v[li].x * hv[li].x - v[li].y * hv[li].y;
        sy += v[li].x * hv[li].y + v[li].y * hv[li].x;
      }
      if constexpr (IG == 1) {
        w.x -= sx; w.y -= sy;
      } else {
        float2* sh = share + (size_t)(t & 1) * SW_THREADS;
        sh[tid] = make_float2(sx, sy);
        __syncthreads();
#pragma unroll
        for (int gg = 0; gg < IG; ++gg) {
          const float2 o = sh[(gg * RPG + yr) * CW + x];
          w.x -= o.x; w.y -= o.y;
        }
      }
      if (g == 0 && ok) W[nu * nb + c] = w;
    }
    if constexpr (MODE == 0 || MODE == 1) {
#pragma unroll
      for (int li = 0; li < NPG; ++li) {
        ax[li] += v[li].x * w.x + v[li].y * w.y;
        ay[li] += v[li].x * w.y - v[li].y * w.x;
      }
    } else {
      nrm += w.x * w.x + w.y * w.y;
    }
  }
  cp_async_wait<0>();
  if constexpr (MODE == 2) {
    red[tid] = make_cuDoubleComplex(g == 0 ? (double)nrm : 0.0, 0.0);
    __syncthreads();
    if (y == 0 && c < nb) {
      double t2 = 0.0;
      for (int k = 0; k < RPG; ++k) t2 += red[k * CW + x].x;
      partial[(long long)blockIdx.y * nb + c] = make_cuDoubleComplex(t2, 0.0);
    }
  } else {
#pragma unroll
    for (int li = 0; li < NPG; ++li) {
      __syncthreads();
      red[tid] = make_cuDoubleComplex((double)ax[li], (double)ay[li]);
      __syncthreads();
      const int i = i0 + li;
      if (yr == 0 && c < nb && i < nv) {
        cplx sum = red[tid];
        for (int k = 1; k < RPG; ++k) { sum.x += red[tid + k * CW].x; sum.y += red[tid + k * CW].y; }
        partial[((long long)blockIdx.y * nv + i) * nb + c] = sum;
      }
    }
  }
}

// column width of the sweep blocks for a batch of nb columns
int sweep_cw(int nb) { return nb >= 32 ? 32 : nb > 8 ? 16 : nb > 4 ? 8 : 4; }
// rows per chunk of the pipelined sweeps: at most one wave of two resident blocks per SM (a block count
// just above the resident slots would leave a short second wave that takes as long as the first)
long long sweep_rows(long long D, int nb) {
  const int cw = sweep_cw(nb);
  const long long gx = (nb + cw - 1) / cw;
  const long long nchunk = std::max<long long>(1, (152LL * 2) / gx);
  return std::max<long long>(64, (D + nchunk - 1) / nchunk);
}

template <int NV, int MODE, int CW>
void launch_sweep_cw(const float2* V, long long vstride, int nv, float2* W, long long D, int nb, const cplx* h, int hld,
                     cplx* partial, cudaStream_t s) {
  static bool attr[64] = {};   // dynamic shared memory above 48 KB: set once per device
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  GFCC_CHECK(dev >= 0 && dev < 64, GFCC_ERR_ARG, "device ordinal above 63");
  constexpr size_t bytes = sweep_smem_bytes<NV, CW>();
  if (!attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(sweep_kernel<NV, MODE, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    attr[dev] = true;
  }
  const long long rows = sweep_rows(D, nb);
  const dim3 grid((unsigned)((nb + CW - 1) / CW), (unsigned)((D + rows - 1) / rows));
  sweep_kernel<NV, MODE, CW><<<grid, SW_THREADS, bytes, s>>>(V, vstride, nv, W, D, nb, rows, h, hld, partial);
}
template <int MODE>
void launch_sweep(const float2* V, long long vstride, int nv, float2* W, long long D, int nb, const cplx* h, int hld,
                  cplx* partial, cudaStream_t s) {
  with_nv(nv, [&](auto NVc) {
    constexpr int NV = decltype(NVc)::value;
    switch (sweep_cw(nb)) {
      case 32: launch_sweep_cw<NV, MODE, 32>(V, vstride, nv, W, D, nb, h, hld, partial, s); break;
      case 16: launch_sweep_cw<NV, MODE, 16>(V, vstride, nv, W, D, nb, h, hld, partial, s); break;
      case 8: launch_sweep_cw<NV, MODE, 8>(V, vstride, nv, W, D, nb, h, hld, partial, s); break;
      default: launch_sweep_cw<NV, MODE, 4>(V, vstride, nv, W, D, nb, h, hld, partial, s); break;
    }
  });
  GFCC_LAUNCH_CHECK();
}

// rows per chunk of the CGS sweeps: at least 256 chunks and two waves of blocks (two resident blocks
// per SM), with the chunk count trimmed so that the blocks fill their last wave
long long cgs_rows(long long D, int nb) {
  const long long gx = (nb + MD_TX - 1) / MD_TX, slots = 152LL * 2;
  long long nchunk = std::max<long long>(256, 2 * slots / gx);
  nchunk = std::max<long long>(1, (nchunk * gx + slots - 1) / slots * slots / gx);
  return std::max<long long>(64, (D + nchunk - 1) / nchunk);
}

// h[c*hld + hoff + i] (+)= sum_chunk partial[chunk][i][c]
__global__ void reduce_partial_kernel(const cplx* __restrict__ partial, int nchunk, int nv, int nb,
                                      cplx* __restrict__ h, int hld, int hoff, int accumulate) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv * nb) return;
  int i = t / nb, c = t % nb;
  cplx s = make_cuDoubleComplex(0.0, 0.0);
  for (int k = 0; k < nchunk; ++k) {
    cplx p = partial[((long long)k * nv + i) * nb + c];
    s.x += p.x; s.y += p.y;
  }
  cplx* dst = h + (long long)c * hld + hoff + i;
  if (accumulate) { dst->x += s.x; dst->y += s.y; } else { *dst = s; }
}

// W[nu][c] += sign * sum_{i<nv} V_i[nu][c] h[c*hld + hoff + i]
template <typename VT>
__global__ void update_kernel(const VT* __restrict__ V, long long vstride, int nv, VT* __restrict__ W,
                              long long D, int nb, const cplx* __restrict__ h, int hld, int hoff, double sign) {
  using R = typename RealOf<VT>::type;
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % nb);
    const cplx* hc = h + (long long)c * hld + hoff;
    // four independent partial sums keep several loads in flight
    R sx[4] = {R(0), R(0), R(0), R(0)}, sy[4] = {R(0), R(0), R(0), R(0)};
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const VT vv = V[(long long)(i + u) * vstride + t];
        const R hx = (R)hc[i + u].x, hy = (R)hc[i + u].y;
        sx[u] += vv.x * hx - vv.y * hy;
        sy[u] += vv.x * hy + vv.y * hx;
      }
    }
    for (; i < nv; ++i) {
      const VT vv = V[(long long)i * vstride + t];
      const R hx = (R)hc[i].x, hy = (R)hc[i].y;
      sx[0] += vv.x * hx - vv.y * hy;
      sy[0] += vv.x * hy + vv.y * hx;
    }
    W[t].x += (R)sign * ((sx[0] + sx[1]) + (sx[2] + sx[3]));
    W[t].y += (R)sign * ((sy[0] + sy[1]) + (sy[2] + sy[3]));
  }
}

// H[c*hld + i] (+)= hb[c*hbld + i], i < n
__global__ void add_h_kernel(const cplx* __restrict__ hb, int hbld, cplx* __restrict__ H, int hld, int n, int nb,
                             int accumulate) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nb) return;
  int c = t / n, i = t % n;
  cplx v = hb[(long long)c * hbld + i];
  cplx* d = H + (long long)c * hld + i;
  if (accumulate) { d->x += v.x; d->y += v.y; } else { *d = v; }
}

// column 2-norms: partial over chunks then reduce (reuses multidot with V = W)
__global__ void finalize_norm_kernel(const cplx* __restrict__ dots, int nb, double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nb) out[c] = sqrt(fmax(dots[c].x, 0.0));
}

// Z[nu][c] = V[nu][c] / (shift_c + mdiag[nu])
template <typename VT>
__global__ void precond_kernel(const VT* __restrict__ V, VT* __restrict__ Z, const double* __restrict__ md,
                               const cplx* __restrict__ shift, long long D, int nb) {
  using R = typename RealOf<VT>::type;
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % nb);
    long long nu = t / nb;
    const R dr = (R)(shift[c].x + md[nu]), di = (R)shift[c].y;
    const R inv = R(1) / (dr * dr + di * di);
    const VT v = V[t];
    Z[t].x = (v.x * dr + v.y * di) * inv;
    Z[t].y = (v.y * dr - v.x * di) * inv;
  }
}

// V[nu][c] = W[nu][c] * scale[c]  (scale = 1/norm, 0 for broken-down columns), with conversion
template <typename VI, typename VO>
__global__ void scale_cols_kernel(const VI* __restrict__ W, VO* __restrict__ V, const double* __restrict__ nrm,
                                  long long D, int nb) {
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    using R = typename RealOf<VO>::type;
    int c = (int)(t % nb);
    double n = nrm[c];
    const R s = (n > 0.0 && isfinite(n)) ? (R)(1.0 / n) : R(0);
    V[t].x = (R)W[t].x * s;
    V[t].y = (R)W[t].y * s;
  }
}

// R = B - Y
__global__ void residual_kernel(const cplx* __restrict__ B, const cplx* __restrict__ Y, cplx* __restrict__ R,
                                long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    R[t] = make_cuDoubleComplex(B[t].x - Y[t].x, B[t].y - Y[t].y);
}

// Per-column Givens step j on H[c] (column-major (k+1) x k), cs/sn/g; writes the residual
// estimate |g_{j+1}| / bnorm and counts columns still above tol*0.5 that are active in this cycle.
__global__ void givens_kernel(cplx* __restrict__ H, cplx* __restrict__ cs, cplx* __restrict__ sn,
                              cplx* __restrict__ g, const double* __restrict__ hnext,
                              const double* __restrict__ bnorm, int* __restrict__ kc, int* __restrict__ live,
                              int nb, int k, int j, const double* __restrict__ thr, int* __restrict__ n_live) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb) return;
  if (!live[c]) return;
  cplx* Hc = H + (long long)c * (k + 1) * k;
  cplx* col = Hc + (long long)j * (k + 1);
  col[j + 1] = make_cuDoubleComplex(hnext[c], 0.0);
  cplx* csc = cs + (long long)c * k;
  cplx* snc = sn + (long long)c * k;
  cplx* gc = g + (long long)c * (k + 1);
  for (int i = 0; i < j; ++i) {
    cplx a = col[i], b = col[i + 1];
    cplx t = cuCadd(cuCmul(csc[i], a), cuCmul(snc[i], b));
    cplx u = cuCadd(cuCmul(make_cuDoubleComplex(-snc[i].x, snc[i].y), a), cuCmul(cuConj(csc[i]), b));
    col[i] = t;
    col[i + 1] = u;
  }
  cplx a = col[j], b = col[j + 1];
  double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
  cplx cj, sj;
  if (den > 0.0) {
    cj = make_cuDoubleComplex(a.x / den, -a.y / den);
    sj = make_cuDoubleComplex(b.x / den, -b.y / den);
  } else {
    cj = make_cuDoubleComplex(1.0, 0.0);
    sj = make_cuDoubleComplex(0.0, 0.0);
  }
  csc[j] = cj;
  snc[j] = sj;
  col[j] = make_cuDoubleComplex(den, 0.0);
  col[j + 1] = make_cuDoubleComplex(0.0, 0.0);
  cplx gj = gc[j];
  gc[j + 1] = cuCmul(make_cuDoubleComplex(-sj.x, sj.y), gj);
  gc[j] = cuCmul(cj, gj);
  kc[c] = j + 1;
  double est = cuCabs(gc[j + 1]) / bnorm[c];
  if (!(est > thr[c]) || den == 0.0 || !isfinite(est)) {
    live[c] = 0;   // converged (or broken down) within this cycle: stop extending its basis use
  } else {
    atomicAdd(n_live, 1);
  }
}

// y = H[:kc,:kc]^{-1} g (upper triangular), stored in g
__global__ void backsolve_kernel(const cplx* __restrict__ H, cplx* __restrict__ g, const int* __restrict__ kc,
                                 int nb, int k) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb) return;
  const cplx* Hc = H + (long long)c * (k + 1) * k;
  cplx* gc = g + (long long)c * (k + 1);
  int n = kc[c];
  for (int i = n - 1; i >= 0; --i) {
    cplx s = gc[i];
    for (int jj = i + 1; jj < n; ++jj) s = cuCsub(s, cuCmul(Hc[(long long)jj * (k + 1) + i], gc[jj]));
    cplx d = Hc[(long long)i * (k + 1) + i];
    gc[i] = (d.x == 0.0 && d.y == 0.0) ? make_cuDoubleComplex(0.0, 0.0) : cuCdiv(s, d);
  }
  for (int i = n; i <= k; ++i) gc[i] = make_cuDoubleComplex(0.0, 0.0);
}

// X[nu][c] += P_c[nu] * sum_i V_i[nu][c] y_i[c]   (FP64 accumulation)
template <typename VT>
__global__ void correct_kernel(const VT* __restrict__ V, long long vstride, int nv, const cplx* __restrict__ y,
                               int yld, cplx* __restrict__ X, const double* __restrict__ md,
                               const cplx* __restrict__ shift, long long D, int nb) {
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    // the correction is formed in the basis precision; only its addition to x is FP64
    using R = typename RealOf<VT>::type;
    int c = (int)(t % nb);
    long long nu = t / nb;
    R sr = R(0), si = R(0);
    const cplx* yc = y + (long long)c * yld;
    for (int i = 0; i < nv; ++i) {
      const cplx yi = yc[i];
      if (yi.x != 0.0 || yi.y != 0.0) {
        const VT vv = V[i * vstride + t];
        const R yr = (R)yi.x, yim = (R)yi.y;
        sr += vv.x * yr - vv.y * yim;
        si += vv.x * yim + vv.y * yr;
      }
    }
    const R dr = (R)(shift[c].x + md[nu]), di = (R)shift[c].y;
    const R inv = R(1) / (dr * dr + di * di);
    X[t].x += (double)((sr * dr + si * di) * inv);
    X[t].y += (double)((si * dr - sr * di) * inv);
  }
}

// dst[nu][k] = src[nu][cols[k]]  (column gather between batch-minor blocks)
__global__ void gather_cols_kernel(const cplx* __restrict__ src, int lds, const int* __restrict__ cols, int nk,
                                   cplx* __restrict__ dst, int ldd, long long D) {
  long long total = D * nk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int k = (int)(t % nk);
    long long nu = t / nk;
    dst[nu * ldd + k] = src[nu * lds + cols[k]];
  }
}
// dst[nu][cols[k]] = src[nu][k]
__global__ void scatter_cols_kernel(const cplx* __restrict__ src, int lds, const int* __restrict__ cols, int nk,
                                    cplx* __restrict__ dst, int ldd, long long D) {
  long long total = D * nk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int k = (int)(t % nk);
    long long nu = t / nk;
    dst[nu * ldd + cols[k]] = src[nu * lds + k];
  }
}

__global__ void nonfinite_cplx_kernel(const cplx* x, long long n, int* flag) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[t].x) || !isfinite(x[t].y)) *flag = 1;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// column norms of a batch-minor block: out[c] = ||W_c||  (device array)
template <typename VT>
static void col_norms(const VT* W, long long D, int nb, double* out, DBuf<cplx>& partial, DBuf<cplx>& tmp,
                      cudaStream_t s) {
  const long long rows = std::max<long long>(256, (D + 511) / 512);
  const int nchunk = (int)((D + rows - 1) / rows);
  partial.alloc((long long)nchunk * nb);
  tmp.alloc(nb);
  dim3 grid((nb + MD_TX - 1) / MD_TX, nchunk);
  multidot_kernel<VT, 4><<<grid, dim3(MD_TX, MD_TY), 0, s>>>(W, 0, 1, W, D, nb, rows, partial.p);
  GFCC_LAUNCH_CHECK();
  reduce_partial_kernel<<<(nb + 255) / 256, 256, 0, s>>>(partial.p, nchunk, 1, nb, tmp.p, 1, 0, 0);
  GFCC_LAUNCH_CHECK();
  finalize_norm_kernel<<<(nb + 255) / 256, 256, 0, s>>>(tmp.p, nb, out);
  GFCC_LAUNCH_CHECK();
}

// h[c][hoff + i] (+)= V_i^H W_c for i < nv, with chunked partial sums
template <typename VT>
static void multidot(const VT* V, long long vstride, int nv, const VT* W, long long D, int nb, cplx* h, int hld,
                     int hoff, bool accumulate, DBuf<cplx>& partial, cudaStream_t s) {
  for (int i0 = 0; i0 < nv; i0 += MD_MAXV) {
    int n = std::min(MD_MAXV, nv - i0);
    const long long rows = cgs_rows(D, nb);
    const int nchunk = (int)((D + rows - 1) / rows);
    partial.alloc((long long)nchunk * n * nb);
    dim3 grid((nb + MD_TX - 1) / MD_TX, nchunk);
    with_nv(n, [&](auto NVc) {
      multidot_kernel<VT, decltype(NVc)::value><<<grid, dim3(MD_TX, MD_TY), 0, s>>>(V + i0 * vstride, vstride, n, W, D,
                                                                                  nb, rows, partial.p);
    });
    GFCC_LAUNCH_CHECK();
    reduce_partial_kernel<<<(n * nb + 255) / 256, 256, 0, s>>>(partial.p, nchunk, n, nb, h, hld, hoff + i0,
                                                               accumulate ? 1 : 0);
    GFCC_LAUNCH_CHECK();
  }
}

// inner action W = (shift + M) Z in the basis precision
static void inner_sigma(gfcc_ctx* c, const cplx* Z, cplx* W, int nb, const cplx* sh, int prec, bool tr, cudaStream_t s) {
  sigma_batch(c, Z, W, nb, nb, sh, prec, tr, s);
}
static void inner_sigma(gfcc_ctx* c, const cuFloatComplex* Z, cuFloatComplex* W, int nb, const cplx* sh, int prec,
                        bool tr, cudaStream_t s) {
  (void)prec;
  sigma_lowprec_f32(c, Z, W, nb, sh, s, tr);
}

// Restarted GMRES with iterative refinement; VT is the precision of the Krylov basis (FP64 for the
// plain FP64 path, FP32 when the inner sigma runs on the tensor cores: the residual of every cycle is
// recomputed with the FP64-accurate sigma and the solution is accumulated in FP64, so the basis
// precision only bounds the progress of one cycle, not the final accuracy).
template <typename VT>
static void gmres_impl(gfcc_ctx* c, const cplx* Bin, cplx* Xout, cplx* Rout, const cplx* shifts_dev, int nb0,
                       SolveStatus& st, bool transpose, const cplx* X0) {
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int k = std::max(1, std::min(c->opts.restart, 256));
  const double tol = c->opts.tol;
  const int inner_prec = c->opts.precision;
  int resid_prec = c->opts.residual_precision;
  if (resid_prec < 0) resid_prec = inner_prec == GFCC_PREC_FP64 ? GFCC_PREC_FP64 : GFCC_PREC_FP64_TC;
  // a cycle with a low-precision inner operator cannot gain more than about its rounding level: stop
  // it once the inner estimate has dropped by this factor
  const double inner_rtol = (inner_prec == GFCC_PREC_FP64 || inner_prec == GFCC_PREC_FP64_TC) ? 0.0 : 1e-4;
  st.relres.assign(nb0, 0.0);
  st.iters.assign(nb0, 0);
  st.converged.assign(nb0, 0);
  if (nb0 == 0) return;

  std::vector<cplx> hshift(nb0);
  GFCC_CUDA(cudaMemcpyAsync(hshift.data(), shifts_dev, sizeof(cplx) * nb0, cudaMemcpyDeviceToHost, s));

  DBuf<cplx> Bw, Xw, Rw, Yw, Ztmp, H, cs, sn, g, partial, tmpc, shw, hb;
  DBuf<VT> V, Zw, Ww;
  DBuf<double> nrm, bnorm, thr;
  DBuf<int> kc, live, nlive, cols, flag;
  Bw.alloc(D * nb0); Xw.alloc(D * nb0); Rw.alloc(D * nb0); Yw.alloc(D * nb0); Ztmp.alloc(D * nb0);
  Zw.alloc(D * nb0); Ww.alloc(D * nb0);
  V.alloc((long long)(k + 1) * D * nb0);
  V.zero(s);
  H.alloc((long long)nb0 * (k + 1) * k);
  cs.alloc((long long)nb0 * k); sn.alloc((long long)nb0 * k); g.alloc((long long)nb0 * (k + 1));
  hb.alloc((long long)nb0 * (k + 1));
  tmpc.alloc(nb0);
  nrm.alloc(nb0); bnorm.alloc(nb0); thr.alloc(nb0); kc.alloc(nb0); live.alloc(nb0); nlive.alloc(1); cols.alloc(nb0);
  shw.alloc(nb0);
  flag.alloc(1);
  {  // chunk partial sums of the Gram-Schmidt sweeps and norms, at their largest (no regrowth per step)
    const long long rows_cn = std::max<long long>(256, (D + 511) / 512);
    long long md = 0;   // the chunk count of the sweeps depends on the batch width
    for (int b = 1; b <= nb0; ++b) {
      md = std::max(md, (D + cgs_rows(D, b) - 1) / cgs_rows(D, b) * b);
      md = std::max(md, (D + sweep_rows(D, b) - 1) / sweep_rows(D, b) * b);
    }
    partial.alloc(std::max(md * (k + 1), (D + rows_cn - 1) / rows_cn * nb0));
  }
  GFCC_CUDA(cudaMemcpyAsync(Bw.p, Bin, sizeof(cplx) * D * nb0, cudaMemcpyDeviceToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(shw.p, shifts_dev, sizeof(cplx) * nb0, cudaMemcpyDeviceToDevice, s));
  if (X0) GFCC_CUDA(cudaMemcpyAsync(Xw.p, X0, sizeof(cplx) * D * nb0, cudaMemcpyDeviceToDevice, s));
  else Xw.zero(s);
  {  // non-finite right-hand sides or shifts
    flag.zero(s);
    nonfinite_cplx_kernel<<<grid_for(D * nb0), 256, 0, s>>>(Bw.p, D * nb0, flag.p);
    GFCC_LAUNCH_CHECK();
    nonfinite_cplx_kernel<<<1, 256, 0, s>>>(shw.p, nb0, flag.p);
    GFCC_LAUNCH_CHECK();
    int hf = 0;
    GFCC_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    GFCC_CHECK(hf == 0, GFCC_ERR_NONFINITE, "solve: non-finite right-hand side or frequency");
  }
  col_norms<cplx>(Bw.p, D, nb0, bnorm.p, partial, tmpc, s);
  std::vector<double> hbn(nb0);
  GFCC_CUDA(cudaMemcpyAsync(hbn.data(), bnorm.p, sizeof(double) * nb0, cudaMemcpyDeviceToHost, s));
  GFCC_CUDA(cudaStreamSynchronize(s));

  std::vector<int> map(nb0);   // working column -> original column
  for (int i = 0; i < nb0; ++i) map[i] = i;
  int nb = nb0;
  std::vector<double> hres(nb0);
  const int max_cycles = std::max(1, c->opts.max_restarts);

  for (int cycle = 0; cycle <= max_cycles && nb > 0; ++cycle) {
    // FP64-accurate residual R = B - (shift X + M X)
    sigma_batch(c, Xw.p, Yw.p, nb, nb, shw.p, resid_prec, transpose, s);
    residual_kernel<<<grid_for(D * nb), 256, 0, s>>>(Bw.p, Yw.p, Rw.p, D * nb);
    GFCC_LAUNCH_CHECK();
    col_norms<cplx>(Rw.p, D, nb, nrm.p, partial, tmpc, s);
    GFCC_CUDA(cudaMemcpyAsync(hres.data(), nrm.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    c->stats.restarts++;
    if (c->opts.verbose) {
      double mx = 0.0;
      for (int w = 0; w < nb; ++w) mx = std::max(mx, hbn[map[w]] > 0.0 ? hres[w] / hbn[map[w]] : 0.0);
      fprintf(stderr, "gfcc gmres: cycle %d, %d columns, max relative residual %.3e\n", cycle, nb, mx);
    }
    if ((inner_prec != GFCC_PREC_FP64 || resid_prec != GFCC_PREC_FP64) && low_precision_error(c))
      throw Error{GFCC_ERR_CUDA, "solve: a tensor-core pipeline wait timed out"};

    // classify columns
    std::vector<int> done, keep;
    for (int w = 0; w < nb; ++w) {
      int orig = map[w];
      double bn = hbn[orig];
      double rel = bn > 0.0 ? hres[w] / bn : 0.0;
      GFCC_CHECK(std::isfinite(rel), GFCC_ERR_NONFINITE, "solve: non-finite residual (singular shift?)");
      st.relres[orig] = rel;
      if (rel <= tol || cycle == max_cycles) {
        done.push_back(w);
        st.converged[orig] = rel <= tol ? 1 : 0;
      } else {
        keep.push_back(w);
      }
    }
    if (!done.empty()) {  // write finished columns out
      std::vector<int> hd(done.size()), ho(done.size());
      for (size_t q = 0; q < done.size(); ++q) { hd[q] = done[q]; ho[q] = map[done[q]]; }
      DBuf<int> dsrc, ddst;
      dsrc.alloc(hd.size()); ddst.alloc(ho.size());
      GFCC_CUDA(cudaMemcpyAsync(dsrc.p, hd.data(), sizeof(int) * hd.size(), cudaMemcpyHostToDevice, s));
      GFCC_CUDA(cudaMemcpyAsync(ddst.p, ho.data(), sizeof(int) * ho.size(), cudaMemcpyHostToDevice, s));
      gather_cols_kernel<<<grid_for(D * hd.size()), 256, 0, s>>>(Xw.p, nb, dsrc.p, (int)hd.size(), Ztmp.p,
                                                                  (int)hd.size(), D);
      GFCC_LAUNCH_CHECK();
      scatter_cols_kernel<<<grid_for(D * hd.size()), 256, 0, s>>>(Ztmp.p, (int)hd.size(), ddst.p, (int)hd.size(),
                                                                   Xout, nb0, D);
      GFCC_LAUNCH_CHECK();
      if (Rout) {
        gather_cols_kernel<<<grid_for(D * hd.size()), 256, 0, s>>>(Rw.p, nb, dsrc.p, (int)hd.size(), Ztmp.p,
                                                                    (int)hd.size(), D);
        GFCC_LAUNCH_CHECK();
        scatter_cols_kernel<<<grid_for(D * hd.size()), 256, 0, s>>>(Ztmp.p, (int)hd.size(), ddst.p,
                                                                     (int)hd.size(), Rout, nb0, D);
        GFCC_LAUNCH_CHECK();
      }
      GFCC_CUDA(cudaStreamSynchronize(s));
    }
    if (keep.empty()) { nb = 0; break; }
    if ((int)keep.size() < nb) {  // compact B, X, R, shifts
      int nk = (int)keep.size();
      GFCC_CUDA(cudaMemcpyAsync(cols.p, keep.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, s));
      for (DBuf<cplx>* b : {&Bw, &Xw, &Rw}) {
        gather_cols_kernel<<<grid_for(D * nk), 256, 0, s>>>(b->p, nb, cols.p, nk, Ztmp.p, nk, D);
        GFCC_LAUNCH_CHECK();
        GFCC_CUDA(cudaMemcpyAsync(b->p, Ztmp.p, sizeof(cplx) * D * nk, cudaMemcpyDeviceToDevice, s));
      }
      std::vector<cplx> nsh(nk);
      std::vector<int> nmap(nk);
      for (int q = 0; q < nk; ++q) { nsh[q] = hshift[map[keep[q]]]; nmap[q] = map[keep[q]]; }
      GFCC_CUDA(cudaMemcpyAsync(shw.p, nsh.data(), sizeof(cplx) * nk, cudaMemcpyHostToDevice, s));
      std::vector<double> nres(nk);
      for (int q = 0; q < nk; ++q) nres[q] = hres[keep[q]];
      GFCC_CUDA(cudaMemcpyAsync(nrm.p, nres.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, s));
      hres = nres;
      map = nmap;
      nb = nk;
      GFCC_CUDA(cudaStreamSynchronize(s));
    }
    {  // ||b|| of the working set and the per-column stopping level of this cycle
      std::vector<double> wb(nb), th(nb);
      for (int q = 0; q < nb; ++q) {
        wb[q] = hbn[map[q]];
        th[q] = std::max(0.5 * tol, inner_rtol * hres[q] / wb[q]);
      }
      GFCC_CUDA(cudaMemcpyAsync(bnorm.p, wb.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
      GFCC_CUDA(cudaMemcpyAsync(thr.p, th.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    }
    // GMRES(k) on the correction: V0 = R / ||R||, g = (||R||, 0, ...)
    scale_cols_kernel<cplx, VT><<<grid_for(D * nb), 256, 0, s>>>(Rw.p, V.p, nrm.p, D, nb);
    GFCC_LAUNCH_CHECK();
    {
      std::vector<cplx> g0((size_t)nb * (k + 1), make_cuDoubleComplex(0.0, 0.0));
      for (int q = 0; q < nb; ++q) g0[(size_t)q * (k + 1)] = make_cuDoubleComplex(hres[q], 0.0);
      GFCC_CUDA(cudaMemcpyAsync(g.p, g0.data(), sizeof(cplx) * g0.size(), cudaMemcpyHostToDevice, s));
      std::vector<int> ones(nb, 1);
      GFCC_CUDA(cudaMemcpyAsync(live.p, ones.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
      GFCC_CUDA(cudaMemsetAsync(kc.p, 0, sizeof(int) * nb, s));
      GFCC_CUDA(cudaMemsetAsync(H.p, 0, sizeof(cplx) * (size_t)nb * (k + 1) * k, s));
    }
    const long long vstride = D * nb;
    for (int j = 0; j < k; ++j) {
      VT* Vj = V.p + j * vstride;
      VT* Vn = V.p + (j + 1) * vstride;
      {
        ProfScope pk(PROF_KRYLOV, 0.0, s);
        precond_kernel<VT><<<grid_for(D * nb), 256, 0, s>>>(Vj, Zw.p, c->op.mdiag.p, shw.p, D, nb);
        GFCC_LAUNCH_CHECK();
      }
      inner_sigma(c, Zw.p, Ww.p, nb, shw.p, inner_prec, transpose, s);
      ProfScope pk2(PROF_KRYLOV, 0.0, s);
      // CGS with one re-orthogonalisation: h1 = V^H w, w -= V h1, h2 = V^H w, w -= V h2; H[:, j] = h1 + h2.
      // With an FP32 basis of at most MD_MAXV vectors this takes three sweeps: h1; the first update with
      // h2 fused; the second update with ||w||^2 fused.
      const int nv = j + 1;
      bool fused = false;
      if constexpr (sizeof(VT) == sizeof(cuFloatComplex)) {
        if (nv <= MD_MAXV) {
          fused = true;
          // algorithmic HBM bytes of the three sweeps: V read three times, w read three times and
          // written twice
          ProfScope pcgs(PROF_KRYLOV_CGS, (3.0 * nv + 5.0) * (double)D * nb * sizeof(VT), s);
          const long long rows = sweep_rows(D, nb);
          const int nchunk = (int)((D + rows - 1) / rows);
          const double vbytes = (double)D * nb * sizeof(VT);   // one basis vector of the batch
          const int small = nb < MD_TX ? 1 : 0;
          const float2* Vf = reinterpret_cast<const float2*>(V.p);
          float2* Wf = reinterpret_cast<float2*>(Ww.p);
          {
            ProfScope pk(small ? PROF_CGS_SMALL_NB : PROF_CGS_MULTIDOT, (nv + 1.0) * vbytes, s);
            launch_sweep<0>(Vf, vstride, nv, Wf, D, nb, nullptr, 0, partial.p, s);
          }
          reduce_partial_kernel<<<(nv * nb + 255) / 256, 256, 0, s>>>(partial.p, nchunk, nv, nb, hb.p, k + 1, 0, 0);
          GFCC_LAUNCH_CHECK();
          add_h_kernel<<<(nb * nv + 255) / 256, 256, 0, s>>>(hb.p, k + 1, H.p + (long long)j * (k + 1), (k + 1) * k, nv,
                                                             nb, 0);
          GFCC_LAUNCH_CHECK();
          {
            ProfScope pk(small ? PROF_CGS_SMALL_NB : PROF_CGS_UPDATE_DOT, (nv + 2.0) * vbytes, s);
            launch_sweep<1>(Vf, vstride, nv, Wf, D, nb, hb.p, k + 1, partial.p, s);
          }
          reduce_partial_kernel<<<(nv * nb + 255) / 256, 256, 0, s>>>(partial.p, nchunk, nv, nb, hb.p, k + 1, 0, 0);
          GFCC_LAUNCH_CHECK();
          add_h_kernel<<<(nb * nv + 255) / 256, 256, 0, s>>>(hb.p, k + 1, H.p + (long long)j * (k + 1), (k + 1) * k, nv,
                                                             nb, 1);
          GFCC_LAUNCH_CHECK();
          {
            ProfScope pk(small ? PROF_CGS_SMALL_NB : PROF_CGS_UPDATE_NORM, (nv + 2.0) * vbytes, s);
            launch_sweep<2>(Vf, vstride, nv, Wf, D, nb, hb.p, k + 1, partial.p, s);
          }
          reduce_partial_kernel<<<(nb + 255) / 256, 256, 0, s>>>(partial.p, nchunk, 1, nb, tmpc.p, 1, 0, 0);
          GFCC_LAUNCH_CHECK();
          finalize_norm_kernel<<<(nb + 255) / 256, 256, 0, s>>>(tmpc.p, nb, nrm.p);
          GFCC_LAUNCH_CHECK();
        }
      }
      if (!fused) {
        for (int pass = 0; pass < 2; ++pass) {
          multidot<VT>(V.p, vstride, nv, Ww.p, D, nb, hb.p, k + 1, 0, false, partial, s);
          update_kernel<VT><<<grid_for(D * nb), 256, 0, s>>>(V.p, vstride, nv, Ww.p, D, nb, hb.p, k + 1, 0, -1.0);
          GFCC_LAUNCH_CHECK();
          add_h_kernel<<<(nb * nv + 255) / 256, 256, 0, s>>>(hb.p, k + 1, H.p + (long long)j * (k + 1), (k + 1) * k,
                                                             nv, nb, pass == 0 ? 0 : 1);
          GFCC_LAUNCH_CHECK();
        }
        col_norms<VT>(Ww.p, D, nb, nrm.p, partial, tmpc, s);
      }
      scale_cols_kernel<VT, VT><<<grid_for(D * nb), 256, 0, s>>>(Ww.p, Vn, nrm.p, D, nb);
      GFCC_LAUNCH_CHECK();
      GFCC_CUDA(cudaMemsetAsync(nlive.p, 0, sizeof(int), s));
      givens_kernel<<<(nb + 127) / 128, 128, 0, s>>>(H.p, cs.p, sn.p, g.p, nrm.p, bnorm.p, kc.p, live.p, nb, k, j,
                                                     thr.p, nlive.p);
      GFCC_LAUNCH_CHECK();
      int hl = 0;
      GFCC_CUDA(cudaMemcpyAsync(&hl, nlive.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      GFCC_CUDA(cudaStreamSynchronize(s));
      c->stats.gmres_iters++;
      for (int q = 0; q < nb; ++q) st.iters[map[q]]++;
      if (hl == 0) break;
    }
    backsolve_kernel<<<(nb + 127) / 128, 128, 0, s>>>(H.p, g.p, kc.p, nb, k);
    GFCC_LAUNCH_CHECK();
    // X += P V y (only the first kc basis vectors carry weight; later y entries are zero)
    correct_kernel<VT><<<grid_for(D * nb), 256, 0, s>>>(V.p, vstride, k, g.p, k + 1, Xw.p, c->op.mdiag.p, shw.p, D, nb);
    GFCC_LAUNCH_CHECK();
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
}

void gmres_batched(gfcc_ctx* c, const cplx* Bin, cplx* Xout, cplx* Rout, const cplx* shifts_dev, int nb0,
                   SolveStatus& st, bool transpose, const cplx* X0) {
  const bool f32 = c->opts.precision == GFCC_PREC_TF32 || c->opts.precision == GFCC_PREC_BF16;
  if (f32) gmres_impl<cuFloatComplex>(c, Bin, Xout, Rout, shifts_dev, nb0, st, transpose, X0);
  else gmres_impl<cplx>(c, Bin, Xout, Rout, shifts_dev, nb0, st, transpose, X0);
}

// ------------------------------------------------------------------------------------------------
namespace {
__global__ void gather_rows_kernel(const double* __restrict__ src, int ld_src, const int* __restrict__ rows,
                                   int nrows, long long D, cplx* __restrict__ dst, int ldb) {
  long long total = D * nrows;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int kq = (int)(t % nrows);
    long long nu = t / nrows;
    dst[nu * ldb + kq] = make_cuDoubleComplex(src[(long long)rows[kq] * ld_src + nu], 0.0);
  }
}
__global__ void cols_to_batch_kernel(const cplx* __restrict__ src, int lds, int ncols, long long D,
                                     cplx* __restrict__ dst, int ldb) {
  long long total = D * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int cc = (int)(t % ncols);
    long long nu = t / ncols;
    dst[nu * ldb + cc] = src[(long long)cc * lds + nu];
  }
}
__global__ void batch_to_cols_kernel(const cplx* __restrict__ src, int ldb, int ncols, long long D,
                                     cplx* __restrict__ dst, int ldd) {
  long long total = D * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long nu = t % D;
    int cc = (int)(t / D);
    dst[(long long)cc * ldd + nu] = src[nu * ldb + cc];
  }
}
}  // namespace

void gather_rows_real_to_cplx(const double* src, int ld_src, const int* rows, int nrows, int D, cplx* dst,
                              int ldb, cudaStream_t s) {
  if (nrows == 0) return;
  gather_rows_kernel<<<grid_for((long long)D * nrows), 256, 0, s>>>(src, ld_src, rows, nrows, D, dst, ldb);
  GFCC_LAUNCH_CHECK();
}
void pack_cols_to_batch(const cplx* src, int ld_src, int ncols, int D, cplx* dst, int ldb, cudaStream_t s) {
  if (ncols == 0) return;
  cols_to_batch_kernel<<<grid_for((long long)D * ncols), 256, 0, s>>>(src, ld_src, ncols, D, dst, ldb);
  GFCC_LAUNCH_CHECK();
}
void batch_to_cols(const cplx* src, int ldb, int ncols, int D, cplx* dst, int ld_dst, cudaStream_t s) {
  if (ncols == 0) return;
  batch_to_cols_kernel<<<grid_for((long long)D * ncols), 256, 0, s>>>(src, ldb, ncols, D, dst, ld_dst);
  GFCC_LAUNCH_CHECK();
}

// G[c][q] = sum_nu c_q[nu] X[nu][c]  as a complex GEMM with a real-valued left operand: do it as a
// real GEMM on the interleaved columns: G'[q][2c+r] = sum_nu cvec[q][nu] X'[nu][2c+r]
// G[c][q] = sum_nu c_q[nu] X[nu][c]: each block reduces a chunk of rows for every (q, c) pair
// (threads over pairs, X rows read coalesced, c_q[nu] broadcast), then the chunks are summed.
namespace {
__global__ void green_partial_kernel(const double* __restrict__ cq, long long D, int nq, const cplx* __restrict__ X,
                                     int ldb, int ncols, long long rows, cplx* __restrict__ part) {
  const long long r0 = blockIdx.x * rows, r1 = min(D, r0 + rows);
  const int npair = nq * ncols;
  for (int t = threadIdx.x; t < npair; t += blockDim.x) {
    const int q = t / ncols, c = t % ncols;
    const double* cr = cq + (long long)q * D;
    double sr = 0.0, si = 0.0;
    for (long long nu = r0; nu < r1; ++nu) {
      const double w = cr[nu];
      const cplx x = X[nu * ldb + c];
      sr = fma(w, x.x, sr);
      si = fma(w, x.y, si);
    }
    part[(long long)blockIdx.x * npair + t] = make_cuDoubleComplex(sr, si);
  }
}
__global__ void green_reduce_kernel(const cplx* __restrict__ part, int nchunk, int nq, int ncols, cplx* __restrict__ G) {
  const int npair = nq * ncols;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair) return;
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < nchunk; ++k) {
    sr += part[(long long)k * npair + t].x;
    si += part[(long long)k * npair + t].y;
  }
  const int q = t / ncols, c = t % ncols;
  G[(long long)c * nq + q] = make_cuDoubleComplex(sr, si);
}
}  // namespace

void green_from_batch(const double* cvec, int D, const int* qrows_host, int nq, const cplx* X, int ldb,
                      int ncols, cplx* G, cudaStream_t s) {
  if (nq == 0 || ncols == 0) return;
  DBuf<double> Cq;
  DBuf<cplx> part;
  Cq.alloc((long long)nq * D);
  for (int q = 0; q < nq; ++q)
    GFCC_CUDA(cudaMemcpyAsync(Cq.p + (long long)q * D, cvec + (long long)qrows_host[q] * D, sizeof(double) * D,
                              cudaMemcpyDeviceToDevice, s));
  const long long rows = std::max<long long>(64, (D + 2 * 152 * 4 - 1) / (2 * 152 * 4));
  const int nchunk = (int)((D + rows - 1) / rows);
  part.alloc((long long)nchunk * nq * ncols);
  green_partial_kernel<<<nchunk, 256, 0, s>>>(Cq.p, D, nq, X, ldb, ncols, rows, part.p);
  GFCC_LAUNCH_CHECK();
  green_reduce_kernel<<<(nq * ncols + 255) / 256, 256, 0, s>>>(part.p, nchunk, nq, ncols, G);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gfcc
