// C ABI of libgfcc (declared in include/gfcc.h): argument checks, host/device marshalling, batching
// and the host side of the adaptive MOR refinement loop. All arithmetic runs in the kernels of the
// other translation units.
#include "gfcc_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <fstream>
#include <new>

using gfcc::cplx;
using gfcc::DBuf;

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void copy_out(void* dst, const void* src_dev, size_t n, cudaStream_t s) {
  gfcc::ProfScope prof(gfcc::PROF_DOWNLOAD, 0.0, s);
  GFCC_CUDA(cudaMemcpyAsync(dst, src_dev, n, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

int choose_batch(gfcc_ctx* c, long long ncols) {
  if (c->opts.max_batch > 0) return (int)std::min<long long>(ncols, c->opts.max_batch);
  size_t freeb = gfcc::device_free_bytes();
  if (freeb == 0) freeb = 8ull << 30;
  const long long D = c->D, ov = (long long)c->o * c->v;
  const long long per_col = (long long)sizeof(cplx) * (D * (c->opts.restart + 10)) + 16LL * ov * c->o * 2 + 4096;
  long long nb = (long long)(0.5 * (double)freeb) / per_col;
  nb = std::max<long long>(1, std::min<long long>({nb, ncols, 1024}));
  return (int)nb;
}

__global__ void spectral_kernel(const cplx* G, int nw, int np, int nq, const int* qidx, double* A) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double s = 0.0;
  for (int p = 0; p < np; ++p)
    if (qidx[p] >= 0) s += G[((long long)w * np + p) * nq + qidx[p]].y;
  A[w] = -s / 3.14159265358979323846;
}

// Gbar[w][p][q] = -(i/pi) Abar[w] where q = qidx[p] >= 0, 0 elsewhere (adjoint of spectral_kernel)
__global__ void spectral_adjoint_kernel(const double* Abar, int nw, int np, int nq, const int* qidx, cplx* Gbar) {
  const long long total = (long long)nw * np * nq;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t / ((long long)np * nq)), p = (int)((t / nq) % np), q = (int)(t % nq);
    Gbar[t] = make_cuDoubleComplex(0.0, qidx[p] == q ? -Abar[w] / 3.14159265358979323846 : 0.0);
  }
}

// MX = B - shift X - R   (all batch-minor [D][nb])
__global__ void mx_kernel(const cplx* B, const cplx* X, const cplx* R, const cplx* shift, cplx* MX, long long D, int nb) {
  long long total = D * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t % nb);
    cplx sx = cuCmul(shift[c], X[t]);
    MX[t] = make_cuDoubleComplex(B[t].x - sx.x - R[t].x, B[t].y - sx.y - R[t].y);
  }
}

__global__ void rownorm2_kernel(const double* rows, long long D, const int* idx, int n, double* out) {
  __shared__ double red[256];
  int r = blockIdx.x;
  const double* x = rows + (long long)idx[r] * D;
  double s = 0.0;
  for (long long t = threadIdx.x; t < D; t += blockDim.x) s += x[t] * x[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = red[0];
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

// part[chunk][w][p][q] = sum_{nu in chunk} Y[nu][w*nq + q] X[nu][w*np + p]  (bilinear, no conjugation)
__global__ void bilinear_partial_kernel(const cplx* __restrict__ X, const cplx* __restrict__ Y, long long D, int nw,
                                        int np, int nq, long long rows, cplx* __restrict__ part) {
  const long long r0 = blockIdx.x * rows, r1 = min(D, r0 + rows);
  const int ntrip = nw * np * nq;
  const int ldx = nw * np, ldy = nw * nq;
  for (int t = threadIdx.x; t < ntrip; t += blockDim.x) {
    const int w = t / (np * nq), p = (t / nq) % np, q = t % nq;
    double sr = 0.0, si = 0.0;
    for (long long nu = r0; nu < r1; ++nu) {
      const cplx x = X[nu * ldx + w * np + p], y = Y[nu * ldy + w * nq + q];
      sr += x.x * y.x - x.y * y.y;
      si += x.x * y.y + x.y * y.x;
    }
    part[(long long)blockIdx.x * ntrip + t] = make_cuDoubleComplex(sr, si);
  }
}
// dw = -sum_chunk part, de = i * sum_chunk part
__global__ void bilinear_reduce_kernel(const cplx* __restrict__ part, int nchunk, int ntrip, cplx* __restrict__ dw,
                                       cplx* __restrict__ de) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntrip) return;
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < nchunk; ++k) { sr += part[(long long)k * ntrip + t].x; si += part[(long long)k * ntrip + t].y; }
  if (dw) dw[t] = make_cuDoubleComplex(-sr, -si);
  if (de) de[t] = make_cuDoubleComplex(-si, sr);
}

std::vector<int> q_positions(const std::vector<int>& porb, const std::vector<int>& qorb) {
  std::vector<int> qi(porb.size(), -1);
  for (size_t p = 0; p < porb.size(); ++p)
    for (size_t q = 0; q < qorb.size(); ++q)
      if (qorb[q] == porb[p]) { qi[p] = (int)q; break; }
  return qi;
}

// Solve the columns (wcol[k] - i eta + M) x_k = b_{pcol[k]}; writes X (batch-minor, [D][ncols]) and R
// into caller-provided device buffers when non-null, and G [ncols][nq] when Gdev is non-null.
void solve_pairs(gfcc_ctx* c, const std::vector<double>& wcol, const std::vector<int>& pcol, double eta,
                 const std::vector<int>& qorb, cplx* Gdev, cplx* Xall, cplx* Rall, gfcc_stats* st_out,
                 const cplx* X0all = nullptr) {
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int nq = (int)qorb.size();
  const long long ncols = (long long)wcol.size();
  const int nbmax = choose_batch(c, ncols);
  c->stats = gfcc::Stats{};
  DBuf<cplx> B, X, R, sh, X0;
  DBuf<int> rows;
  B.alloc(D * nbmax); X.alloc(D * nbmax); R.alloc(D * nbmax); sh.alloc(nbmax); rows.alloc(nbmax);
  double maxres = 0.0;
  int notconv = 0;
  for (long long c0 = 0; c0 < ncols; c0 += nbmax) {
    const int nb = (int)std::min<long long>(nbmax, ncols - c0);
    std::vector<int> hr(nb);
    std::vector<cplx> hs(nb);
    for (int k = 0; k < nb; ++k) {
      const long long col = c0 + k;
      hr[k] = pcol[col];
      hs[k] = make_cuDoubleComplex(wcol[col], -eta);
    }
    GFCC_CUDA(cudaMemcpyAsync(rows.p, hr.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    GFCC_CUDA(cudaMemcpyAsync(sh.p, hs.data(), sizeof(cplx) * nb, cudaMemcpyHostToDevice, s));
    gfcc::gather_rows_real_to_cplx(c->bvec.p, (int)D, rows.p, nb, (int)D, B.p, nb, s);
    if (X0all) {   // initial guesses of this batch (columns c0 .. c0+nb of [D][ncols])
      X0.alloc(D * nbmax);
      GFCC_CUDA(cudaMemcpy2DAsync(X0.p, sizeof(cplx) * nb, X0all + c0, sizeof(cplx) * ncols, sizeof(cplx) * nb, D,
                                  cudaMemcpyDeviceToDevice, s));
    }
    gfcc::SolveStatus st;
    gfcc::gmres_batched(c, B.p, X.p, R.p, sh.p, nb, st, false, X0all ? X0.p : nullptr);
    for (int k = 0; k < nb; ++k) {
      maxres = std::max(maxres, st.relres[k]);
      if (!st.converged[k]) ++notconv;
    }
    if (Gdev) gfcc::green_from_batch(c->cvec.p, (int)D, qorb.data(), nq, X.p, nb, nb, Gdev + c0 * nq, s);
    if (Xall) {  // copy columns into the big batch-minor block [D][ncols]
      GFCC_CUDA(cudaMemcpy2DAsync(Xall + c0, sizeof(cplx) * ncols, X.p, sizeof(cplx) * nb, sizeof(cplx) * nb, D,
                                  cudaMemcpyDeviceToDevice, s));
    }
    if (Rall) {
      GFCC_CUDA(cudaMemcpy2DAsync(Rall + c0, sizeof(cplx) * ncols, R.p, sizeof(cplx) * nb, sizeof(cplx) * nb, D,
                                  cudaMemcpyDeviceToDevice, s));
    }
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
  c->stats.max_rel_res = maxres;
  c->stats.not_converged = notconv;
  if (st_out) {
    st_out->sigma_calls = c->stats.sigma_calls;
    st_out->sigma_cols = c->stats.sigma_cols;
    st_out->gmres_iters = c->stats.gmres_iters;
    st_out->restarts = c->stats.restarts;
    st_out->max_rel_res = maxres;
    st_out->not_converged = notconv;
  }
}

// Solve all (w, p) columns, column w * np + p (see solve_pairs).
void solve_columns(gfcc_ctx* c, const std::vector<double>& ws, double eta, const std::vector<int>& porb,
                   const std::vector<int>& qorb, cplx* Gdev, cplx* Xall, cplx* Rall, gfcc_stats* st_out,
                   const cplx* X0all = nullptr) {
  const size_t np = porb.size();
  std::vector<double> wcol(ws.size() * np);
  std::vector<int> pcol(ws.size() * np);
  for (size_t k = 0; k < wcol.size(); ++k) {
    wcol[k] = ws[k / np];
    pcol[k] = porb[k % np];
  }
  solve_pairs(c, wcol, pcol, eta, qorb, Gdev, Xall, Rall, st_out, X0all);
}

// Adjoint solves (w - i eta + M)^T y = c_q for every (w, q): columns (w, q) of Yall [D][nw*nq].
void solve_adjoint_columns(gfcc_ctx* c, const std::vector<double>& ws, double eta, const std::vector<int>& qorb,
                           cplx* Yall) {
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int nq = (int)qorb.size();
  const long long ncols = (long long)ws.size() * nq;
  const int nbmax = choose_batch(c, ncols);
  DBuf<cplx> B, Y, sh;
  DBuf<int> rows;
  B.alloc(D * nbmax); Y.alloc(D * nbmax); sh.alloc(nbmax); rows.alloc(nbmax);
  for (long long c0 = 0; c0 < ncols; c0 += nbmax) {
    const int nb = (int)std::min<long long>(nbmax, ncols - c0);
    std::vector<int> hr(nb);
    std::vector<cplx> hs(nb);
    for (int k = 0; k < nb; ++k) {
      const long long col = c0 + k;
      hr[k] = qorb[col % nq];
      hs[k] = make_cuDoubleComplex(ws[col / nq], -eta);
    }
    GFCC_CUDA(cudaMemcpyAsync(rows.p, hr.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    GFCC_CUDA(cudaMemcpyAsync(sh.p, hs.data(), sizeof(cplx) * nb, cudaMemcpyHostToDevice, s));
    gfcc::gather_rows_real_to_cplx(c->cvec.p, (int)D, rows.p, nb, (int)D, B.p, nb, s);
    gfcc::SolveStatus st;
    gfcc::gmres_batched(c, B.p, Y.p, nullptr, sh.p, nb, st, true);
    for (int k = 0; k < nb; ++k)
      GFCC_CHECK(st.converged[k], GFCC_ERR_NOT_CONVERGED, "adjoint solve did not converge");
    GFCC_CUDA(cudaMemcpy2DAsync(Yall + c0, sizeof(cplx) * ncols, Y.p, sizeof(cplx) * nb, sizeof(cplx) * nb, D,
                                cudaMemcpyDeviceToDevice, s));
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
}

// Solves A(w) U = W (transpose: A(w)^T U = W) for general right sides: W, U batch-minor [D][nw np],
// column w np + p at frequency ws[w].
void solve_rhs(gfcc_ctx* c, const std::vector<double>& ws, double eta, int np, const cplx* Wall, cplx* Uall,
               bool transpose) {
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const long long ncols = (long long)ws.size() * np;
  const int nbmax = choose_batch(c, ncols);
  DBuf<cplx> B, Y, sh;
  B.alloc(D * nbmax); Y.alloc(D * nbmax); sh.alloc(nbmax);
  for (long long c0 = 0; c0 < ncols; c0 += nbmax) {
    const int nb = (int)std::min<long long>(nbmax, ncols - c0);
    std::vector<cplx> hs(nb);
    for (int k = 0; k < nb; ++k) hs[k] = make_cuDoubleComplex(ws[(c0 + k) / np], -eta);
    GFCC_CUDA(cudaMemcpyAsync(sh.p, hs.data(), sizeof(cplx) * nb, cudaMemcpyHostToDevice, s));
    GFCC_CUDA(cudaMemcpy2DAsync(B.p, sizeof(cplx) * nb, Wall + c0, sizeof(cplx) * ncols, sizeof(cplx) * nb, D,
                                cudaMemcpyDeviceToDevice, s));
    gfcc::SolveStatus st;
    gfcc::gmres_batched(c, B.p, Y.p, nullptr, sh.p, nb, st, transpose);
    for (int k = 0; k < nb; ++k)
      GFCC_CHECK(st.converged[k], GFCC_ERR_NOT_CONVERGED, transpose ? "adjoint solve did not converge"
                                                                     : "derivative solve did not converge");
    GFCC_CUDA(cudaMemcpy2DAsync(Uall + c0, sizeof(cplx) * ncols, Y.p, sizeof(cplx) * nb, sizeof(cplx) * nb, D,
                                cudaMemcpyDeviceToDevice, s));
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
}

// Solve at frequencies ws for the model's p set and append the solutions to the subspace.
void mor_add_chunk(gfcc_ctx* c, const std::vector<double>& ws);
void mor_add_frequencies(gfcc_ctx* c, const std::vector<double>& ws) {
  // bounded memory: the solutions, residuals, images, right-hand sides, initial guesses and derivative
  // solves of a chunk of frequencies (6 vectors per column), and the growth of S, Z and the residual
  // basis they cause (4 columns per column, doubled while a buffer is regrown), take at most about a
  // quarter of the free device memory; the chunks keep the frequency order, so the columns reach the
  // subspace in the same order as in one piece
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) { cudaGetLastError(); totalb = 0; }
  freeb = gfcc::device_free_bytes();
  if (freeb == 0) freeb = 16ull << 30;
  if (freeb < totalb / 3) {   // scratch of earlier calls (e.g. adjoint solves) holds much of the device
    gfcc::release_scratch(c);
    freeb = gfcc::device_free_bytes();
    if (freeb == 0) freeb = 16ull << 30;
  }
  const long long per_w = (long long)c->D * (long long)c->mor.porb.size() * (long long)sizeof(cplx) * 14;
  const size_t per_chunk = (size_t)std::max<long long>(1, (long long)(0.25 * (double)freeb) / std::max(per_w, 1LL));
  for (size_t i0 = 0; i0 < ws.size(); i0 += per_chunk) {
    const std::vector<double> part(ws.begin() + i0, ws.begin() + std::min(ws.size(), i0 + per_chunk));
    mor_add_chunk(c, part);
  }
}
void mor_add_chunk(gfcc_ctx* c, const std::vector<double>& ws) {
  gfcc::MorState& ms = c->mor;
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int np = (int)ms.porb.size();
  const long long ncols = (long long)ws.size() * np;
  DBuf<cplx> X, R, MX, B, sh;
  DBuf<int> rows;
  X.alloc(D * ncols); R.alloc(D * ncols); MX.alloc(D * ncols); B.alloc(D * ncols); sh.alloc(ncols);
  rows.alloc(ncols);
  DBuf<cplx> X0;
  if (ms.m > 0 && c->opts.mor_guess) {   // initial guesses x0_p(w) = S yhat_p(w) from the current model
    X0.alloc(D * ncols);
    gfcc::mor_extrapolate(c, ws.data(), (int)ws.size(), X0.p);
  }
  solve_columns(c, ws, ms.eta, ms.porb, ms.qorb, nullptr, X.p, R.p, nullptr, X0.p);
  ms.solve_iters += c->stats.gmres_iters;
  ms.solve_cols += ncols;
  std::vector<int> hr(ncols);
  std::vector<cplx> hs(ncols);
  for (long long k = 0; k < ncols; ++k) {
    hr[k] = ms.porb[k % np];
    hs[k] = make_cuDoubleComplex(ws[k / np], -ms.eta);
  }
  GFCC_CUDA(cudaMemcpyAsync(rows.p, hr.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(sh.p, hs.data(), sizeof(cplx) * ncols, cudaMemcpyHostToDevice, s));
  gfcc::gather_rows_real_to_cplx(c->bvec.p, (int)D, rows.p, (int)ncols, (int)D, B.p, (int)ncols, s);
  mx_kernel<<<grid_for(D * ncols), 256, 0, s>>>(B.p, X.p, R.p, sh.p, MX.p, D, (int)ncols);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(s));
  if (c->opts.deriv_indicator) {   // exact dG/dw = -c_q^T A^{-1} x_p at the new samples
    DBuf<cplx> Zd, dG;
    const int nq = (int)ms.qorb.size();
    Zd.alloc(D * ncols);
    dG.alloc(ncols * nq);
    solve_rhs(c, ws, ms.eta, np, X.p, Zd.p, false);
    gfcc::green_from_batch(c->cvec.p, (int)D, ms.qorb.data(), nq, Zd.p, (int)ncols, (int)ncols, dG.p, s);
    std::vector<cplx> h((size_t)ncols * nq);
    GFCC_CUDA(cudaMemcpyAsync(h.data(), dG.p, sizeof(cplx) * h.size(), cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    for (size_t k = 0; k < ws.size(); ++k) {
      std::vector<cplx> d(h.begin() + (long long)k * np * nq, h.begin() + (long long)(k + 1) * np * nq);
      for (cplx& z : d) z = make_cuDoubleComplex(-z.x, -z.y);
      ms.dG_exact.push_back({ws[k], std::move(d)});
    }
  }
  gfcc::mor_append(c, X.p, MX.p, (int)ncols);
  for (double w : ws) ms.sampled.push_back(w);
  std::sort(ms.sampled.begin(), ms.sampled.end());
}

// ---- block Krylov subspace (multi-shift reuse) ------------------------------------------------
// Extend the subspace of a kind-1 model by up to nblocks Krylov blocks: the next block is M applied to
// the newest orthonormal block (its columns of Z = M S), or B for the first one; each block's images
// M X come from the FP64-accurate sigma. The space K_k(M, B) is the same for every shift w - i eta, so the
// Galerkin model over it gives the block FOM solution of Eq. xplin at every frequency at once.
void krylov_extend(gfcc_ctx* c, int nblocks, int m_max) {
  gfcc::MorState& ms = c->mor;
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const int np = (int)ms.porb.size();
  int prec = c->opts.residual_precision;
  if (prec < 0) prec = c->opts.precision == GFCC_PREC_FP64 ? GFCC_PREC_FP64 : GFCC_PREC_FP64_TC;
  DBuf<cplx> X, MX;
  for (int j = 0; j < nblocks; ++j) {
    const int nc = ms.kblocks == 0 ? np : ms.knext;
    if (nc == 0 || ms.m + nc > m_max) break;
    X.alloc(D * nc);
    MX.alloc(D * nc);
    if (ms.kblocks == 0) {
      DBuf<int> rows;
      rows.alloc(np);
      GFCC_CUDA(cudaMemcpyAsync(rows.p, ms.porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
      gfcc::gather_rows_real_to_cplx(c->bvec.p, (int)D, rows.p, np, (int)D, X.p, np, s);
      GFCC_CUDA(cudaStreamSynchronize(s));
    } else {
      GFCC_CUDA(cudaMemcpy2DAsync(X.p, sizeof(cplx) * nc, ms.Z.p + (ms.m - nc), sizeof(cplx) * ms.m_cap,
                                  sizeof(cplx) * nc, D, cudaMemcpyDeviceToDevice, s));
    }
    gfcc::sigma_batch(c, X.p, MX.p, nc, nc, nullptr, prec, false, s);
    const int m0 = ms.m;
    gfcc::mor_append(c, X.p, MX.p, nc);
    ms.knext = ms.m - m0;
    ++ms.kblocks;
    if (ms.knext == 0) break;   // the Krylov space is invariant: nothing new to add
  }
  if (prec != GFCC_PREC_FP64) {
    GFCC_CHECK(gfcc::emulated_error(c) == 0, GFCC_ERR_CUDA, "exact-slice sigma: tensor-core pipeline wait timed out");
  }
}

// ---- per-orbital (SISO) reduced models -------------------------------------------------------
// Model k of c->siso is an ordinary reduced model with the single orbital p = q = porb_k; the routines of
// mor.cu act on c->mor, so a model is swapped into c->mor for the duration of each call on it.
struct ModelSwap {
  gfcc_ctx* c;
  gfcc::MorState* m;
  ModelSwap(gfcc_ctx* c_, gfcc::MorState* m_) : c(c_), m(m_) { std::swap(c->mor, *m); }
  ~ModelSwap() { std::swap(c->mor, *m); }
  ModelSwap(const ModelSwap&) = delete;
  ModelSwap& operator=(const ModelSwap&) = delete;
};

// Solve every (model k, w) pair of add (sorted by model, then frequency) in one batched solve and append
// each model's solutions to its own subspace.
void siso_add_chunk(gfcc_ctx* c, const std::vector<std::pair<int, double>>& add, double eta);
void siso_add_frequencies(gfcc_ctx* c, const std::vector<std::pair<int, double>>& add, double eta) {
  // bounded memory: at most kSisoChunk columns (their solutions, residuals and images) at a time
  constexpr size_t kSisoChunk = 256;
  for (size_t i0 = 0; i0 < add.size(); i0 += kSisoChunk) {
    const std::vector<std::pair<int, double>> part(add.begin() + i0, add.begin() + std::min(add.size(), i0 + kSisoChunk));
    siso_add_chunk(c, part, eta);
  }
}
void siso_add_chunk(gfcc_ctx* c, const std::vector<std::pair<int, double>>& add, double eta) {
  cudaStream_t s = c->stream;
  const long long D = c->D;
  const long long ncols = (long long)add.size();
  if (ncols == 0) return;
  std::vector<double> wcol(ncols);
  std::vector<int> pcol(ncols);
  std::vector<long long> first(c->siso.size() + 1, 0);   // columns [first[k], first[k+1]) belong to model k
  for (long long j = 0; j < ncols; ++j) {
    wcol[j] = add[j].second;
    pcol[j] = c->siso[add[j].first].porb[0];
    ++first[add[j].first + 1];
  }
  for (size_t k = 0; k < c->siso.size(); ++k) first[k + 1] += first[k];
  DBuf<cplx> X, R, MX, B, sh, X0, Xk, MXk;
  DBuf<int> rows;
  X.alloc(D * ncols); R.alloc(D * ncols); MX.alloc(D * ncols); B.alloc(D * ncols); sh.alloc(ncols);
  rows.alloc(ncols);
  bool guess = false;   // initial guesses from the models that already have a subspace (none at the seeds)
  for (size_t k = 0; k < c->siso.size(); ++k) guess = guess || (first[k + 1] > first[k] && c->siso[k].m > 0);
  guess = guess && c->opts.mor_guess;
  if (guess) {   // each model's prediction x0_p(w) = S yhat_p(w) at its new frequencies, zero for empty models
    X0.alloc(D * ncols);
    X0.zero(s);
    for (size_t k = 0; k < c->siso.size(); ++k) {
      const long long nk = first[k + 1] - first[k];
      if (nk == 0 || c->siso[k].m == 0) continue;
      DBuf<cplx> tmp;
      tmp.alloc(D * nk);
      {
        ModelSwap sw(c, &c->siso[k]);
        gfcc::mor_extrapolate(c, wcol.data() + first[k], (int)nk, tmp.p);
      }
      GFCC_CUDA(cudaMemcpy2DAsync(X0.p + first[k], sizeof(cplx) * ncols, tmp.p, sizeof(cplx) * nk, sizeof(cplx) * nk, D,
                                  cudaMemcpyDeviceToDevice, s));
      GFCC_CUDA(cudaStreamSynchronize(s));
    }
  }
  solve_pairs(c, wcol, pcol, eta, {}, nullptr, X.p, R.p, nullptr, guess ? X0.p : nullptr);
  c->siso_iters += c->stats.gmres_iters;
  c->siso_cols += ncols;
  std::vector<cplx> hs(ncols);
  for (long long j = 0; j < ncols; ++j) hs[j] = make_cuDoubleComplex(wcol[j], -eta);
  GFCC_CUDA(cudaMemcpyAsync(rows.p, pcol.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice, s));
  GFCC_CUDA(cudaMemcpyAsync(sh.p, hs.data(), sizeof(cplx) * ncols, cudaMemcpyHostToDevice, s));
  gfcc::gather_rows_real_to_cplx(c->bvec.p, (int)D, rows.p, (int)ncols, (int)D, B.p, (int)ncols, s);
  mx_kernel<<<grid_for(D * ncols), 256, 0, s>>>(B.p, X.p, R.p, sh.p, MX.p, D, (int)ncols);
  GFCC_LAUNCH_CHECK();
  for (size_t k = 0; k < c->siso.size(); ++k) {
    const long long nk = first[k + 1] - first[k];
    if (nk == 0) continue;
    Xk.alloc(D * nk);
    MXk.alloc(D * nk);
    GFCC_CUDA(cudaMemcpy2DAsync(Xk.p, sizeof(cplx) * nk, X.p + first[k], sizeof(cplx) * ncols, sizeof(cplx) * nk, D,
                                cudaMemcpyDeviceToDevice, s));
    GFCC_CUDA(cudaMemcpy2DAsync(MXk.p, sizeof(cplx) * nk, MX.p + first[k], sizeof(cplx) * ncols, sizeof(cplx) * nk, D,
                                cudaMemcpyDeviceToDevice, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    ModelSwap sw(c, &c->siso[k]);
    gfcc::mor_append(c, Xk.p, MXk.p, (int)nk);
    for (long long j = first[k]; j < first[k + 1]; ++j) c->mor.sampled.push_back(wcol[j]);
    std::sort(c->mor.sampled.begin(), c->mor.sampled.end());
  }
}

// interval error estimates of the current model c->mor on the grid (residual indicator, as in
// gfcc_mor_refine): e[k] = largest relative residual estimate at grid points strictly inside
// (sampled[k], sampled[k+1])
std::vector<double> interval_errors(gfcc_ctx* c, const std::vector<double>& grid, DBuf<double>& dres) {
  const int ngrid = (int)grid.size();
  std::vector<double> res(ngrid);
  gfcc::mor_eval(c, grid.data(), ngrid, nullptr, nullptr, dres.p);
  GFCC_CUDA(cudaMemcpyAsync(res.data(), dres.p, sizeof(double) * ngrid, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  const std::vector<double>& smp = c->mor.sampled;
  std::vector<double> e(smp.size() > 0 ? smp.size() - 1 : 0, 0.0);
  for (size_t k = 0; k + 1 < smp.size(); ++k)
    for (int g = 0; g < ngrid; ++g)
      if (grid[g] > smp[k] && grid[g] < smp[k + 1]) e[k] = std::max(e[k], res[g]);
  return e;
}

// midpoints of the intervals whose estimate is above tol, largest estimate first (ties: lower frequency),
// at most max_new of them, returned in increasing order
std::vector<double> choose_midpoints(const std::vector<double>& smp, const std::vector<double>& e, double tol,
                                     int max_new) {
  std::vector<std::pair<double, double>> cand;   // (-error, midpoint)
  for (size_t k = 0; k < e.size(); ++k)
    if (e[k] > tol) cand.push_back({-e[k], 0.5 * (smp[k] + smp[k + 1])});
  std::sort(cand.begin(), cand.end());
  std::vector<double> nw;
  for (int k = 0; k < (int)cand.size() && k < max_new; ++k) nw.push_back(cand[k].second);
  std::sort(nw.begin(), nw.end());
  return nw;
}

// elementwise out[i] = max(out[i], x[i])
__global__ void max_into_kernel(const double* __restrict__ x, double* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fmax(out[i], x[i]);
}

}  // namespace

#define API_BEGIN                                                  \
  gfcc::StreamScope api_stream_scope_(c ? c->stream : nullptr);   \
  try {
#define API_END(ctx)                                                   \
  }                                                                    \
  catch (gfcc::Error & e) {                                            \
    if (ctx) (ctx)->last_error = e.msg;                                \
    return e.code;                                                     \
  }                                                                    \
  catch (std::bad_alloc&) {                                            \
    if (ctx) (ctx)->last_error = "host allocation failed";             \
    return GFCC_ERR_OOM;                                               \
  }                                                                    \
  catch (std::exception & e) {                                         \
    if (ctx) (ctx)->last_error = e.what();                             \
    return GFCC_ERR_ARG;                                               \
  }                                                                    \
  return GFCC_OK;

extern "C" {

int gfcc_default_opts(gfcc_opts* o) {
  if (!o) return GFCC_ERR_ARG;
  o->tol = 1e-8;
  o->restart = 30;
  o->max_restarts = 200;
  o->precision = GFCC_PREC_FP64;
  o->max_batch = 0;
  o->drop_tol = 1e-10;
  o->verbose = 0;
  o->residual_precision = -1;
  o->deriv_indicator = 0;
  o->mor_guess = 1;
  return GFCC_OK;
}

static int check_opts(const gfcc_opts* o, std::string& why) {
  if (!(o->tol > 0.0 && o->tol < 1.0)) { why = "opts.tol must be in (0, 1)"; return GFCC_ERR_ARG; }
  if (o->restart < 1 || o->restart > 256) { why = "opts.restart must be in [1, 256]"; return GFCC_ERR_ARG; }
  if (o->max_restarts < 1) { why = "opts.max_restarts must be >= 1"; return GFCC_ERR_ARG; }
  if (o->precision < GFCC_PREC_FP64 || o->precision > GFCC_PREC_FP64_TC) { why = "opts.precision unknown"; return GFCC_ERR_ARG; }
  if (o->max_batch < 0) { why = "opts.max_batch must be >= 0"; return GFCC_ERR_ARG; }
  if (!(o->drop_tol > 0.0 && o->drop_tol < 1.0)) { why = "opts.drop_tol must be in (0, 1)"; return GFCC_ERR_ARG; }
  if (o->deriv_indicator != 0 && o->deriv_indicator != 1) { why = "opts.deriv_indicator must be 0 or 1"; return GFCC_ERR_ARG; }
  if (o->mor_guess != 0 && o->mor_guess != 1) { why = "opts.mor_guess must be 0 or 1"; return GFCC_ERR_ARG; }
  if (o->residual_precision != -1 && o->residual_precision != GFCC_PREC_FP64 && o->residual_precision != GFCC_PREC_FP64_TC) {
    why = "opts.residual_precision must be -1, GFCC_PREC_FP64 or GFCC_PREC_FP64_TC";
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

static int init_context(gfcc_t* out, int sector, int o, int v, const double* eps, const gfcc_vblocks* vb,
                        const double* vvvv, const double* t1, const double* t2, const double* l1, const double* l2,
                        const gfcc_opts* opts, void* stream) {
  if (!out) return GFCC_ERR_ARG;
  *out = nullptr;
  if (!eps || !vb || !t1 || !t2 || !l1 || !l2 || !vb->oooo || !vb->ooov || !vb->oovv || !vb->ovov || !vb->ovvv)
    return GFCC_ERR_ARG;
  if (sector == 0 ? (o < 2 || v < 1) : (o < 1 || v < 2 || !vvvv)) return GFCC_ERR_ARG;
  // block sizes of the operator: the EA space has the IP layout with the index ranges exchanged
  const int po = sector == 0 ? o : v, pv = sector == 0 ? v : o;
  const long long P = (long long)po * (po - 1) / 2;
  const long long D = po + P * pv;
  if (D >= (1LL << 31) || (long long)o * v * o * v >= (1LL << 40) || P * P >= (1LL << 40)) return GFCC_ERR_ARG;
  gfcc_ctx* c = new (std::nothrow) gfcc_ctx();
  if (!c) return GFCC_ERR_OOM;
  c->o = po; c->v = pv; c->n = o + v; c->P = (int)P; c->D = (int)D;
  c->sector = sector;
  c->stream = (cudaStream_t)stream;
  if (opts) c->opts = *opts; else gfcc_default_opts(&c->opts);
  std::string why;
  int rc = check_opts(&c->opts, why);
  if (rc != GFCC_OK) { delete c; return rc; }
  int status = GFCC_OK;
  gfcc::StreamScope stream_scope(c->stream);
  try {
    GFCC_CUDA(cudaGetDevice(&c->device));
    gfcc::HostInputs in{eps, vb->oooo, vb->ooov, vb->oovv, vb->ovov, vb->ovvv, t1, t2, l1, l2};
    in.vvvv = vvvv;
    if (sector == 0) gfcc::build_operator(c, in);
    else gfcc::build_operator_ea(c, in);
    if (c->opts.precision == GFCC_PREC_TF32 || c->opts.precision == GFCC_PREC_BF16)
      gfcc::build_low_precision(c, c->opts.precision);
  } catch (gfcc::Error& e) {
    status = e.code;
    fprintf(stderr, "gfcc_init: %s\n", e.msg.c_str());
  } catch (std::bad_alloc&) {
    status = GFCC_ERR_OOM;
  }
  if (status != GFCC_OK) { delete c; return status; }
  *out = c;
  return GFCC_OK;
}

int gfcc_init(gfcc_t* out, int o, int v, const double* eps, const gfcc_vblocks* vb, const double* t1,
              const double* t2, const double* l1, const double* l2, const gfcc_opts* opts, void* stream) {
  return init_context(out, 0, o, v, eps, vb, nullptr, t1, t2, l1, l2, opts, stream);
}

int gfcc_init_ea(gfcc_t* out, int o, int v, const double* eps, const gfcc_vblocks* vb, const double* vvvv,
                 const double* t1, const double* t2, const double* l1, const double* l2, const gfcc_opts* opts,
                 void* stream) {
  return init_context(out, 1, o, v, eps, vb, vvvv, t1, t2, l1, l2, opts, stream);
}

int gfcc_sector(gfcc_t c, int* sector) {
  if (!c || !sector) return GFCC_ERR_ARG;
  *sector = c->sector;
  return GFCC_OK;
}

int gfcc_dim(gfcc_t c, int* D) {
  if (!c || !D) return GFCC_ERR_ARG;
  *D = c->D;
  return GFCC_OK;
}

int gfcc_set_opts(gfcc_t c, const gfcc_opts* opts) {
  if (!c || !opts) return GFCC_ERR_ARG;
  std::string why;
  int rc = check_opts(opts, why);
  if (rc != GFCC_OK) { c->last_error = why; return rc; }
  API_BEGIN
  c->opts = *opts;
  if ((opts->precision == GFCC_PREC_TF32 || opts->precision == GFCC_PREC_BF16) && c->lp.kind != opts->precision)
    gfcc::build_low_precision(c, opts->precision);
  API_END(c)
}

int gfcc_sigma(gfcc_t c, const double* X, double* Y, int nvec, int ld, int precision, int transpose) {
  if (!c) return GFCC_ERR_ARG;
  if (nvec < 0 || (nvec > 0 && (!X || !Y || ld < c->D)) || precision < 0 || precision > GFCC_PREC_FP64_TC) {
    c->last_error = "gfcc_sigma: bad arguments";
    return GFCC_ERR_ARG;
  }
  API_BEGIN
  if (nvec == 0) return GFCC_OK;
  cudaStream_t s = c->stream;
  const long long D = c->D;
  if ((precision == GFCC_PREC_TF32 || precision == GFCC_PREC_BF16) && c->lp.kind != precision)
    gfcc::build_low_precision(c, precision);
  const int nbmax = std::max(1, std::min(nvec, c->opts.max_batch > 0 ? c->opts.max_batch : 256));
  DBuf<cplx> stage, Xb, Yb;
  stage.alloc((long long)nbmax * ld);
  Xb.alloc(D * nbmax);
  Yb.alloc(D * nbmax);
  const cplx* Xc = reinterpret_cast<const cplx*>(X);
  cplx* Yc = reinterpret_cast<cplx*>(Y);
  const bool xdev = is_device_ptr(X), ydev = is_device_ptr(Y);
  for (int c0 = 0; c0 < nvec; c0 += nbmax) {
    const int nb = std::min(nbmax, nvec - c0);
    const cplx* src = Xc + (long long)c0 * ld;
    if (!xdev) {
      GFCC_CUDA(cudaMemcpyAsync(stage.p, src, sizeof(cplx) * nb * ld, cudaMemcpyHostToDevice, s));
      src = stage.p;
    }
    gfcc::pack_cols_to_batch(src, ld, nb, (int)D, Xb.p, nb, s);
    gfcc::sigma_batch(c, Xb.p, Yb.p, nb, nb, nullptr, precision, transpose != 0, s);
    if (ydev) {
      gfcc::batch_to_cols(Yb.p, nb, nb, (int)D, Yc + (long long)c0 * ld, ld, s);
    } else {
      gfcc::batch_to_cols(Yb.p, nb, nb, (int)D, stage.p, ld, s);
      GFCC_CUDA(cudaMemcpyAsync(Yc + (long long)c0 * ld, stage.p, sizeof(cplx) * nb * ld, cudaMemcpyDeviceToHost, s));
    }
    GFCC_CUDA(cudaStreamSynchronize(s));
  }
  API_END(c)
}

int gfcc_vectors(gfcc_t c, const int* orbitals, int norb, int transpose, double* out, int ld) {
  if (!c) return GFCC_ERR_ARG;
  if (norb < 0 || (norb > 0 && (!orbitals || !out || ld < c->D))) { c->last_error = "gfcc_vectors: bad arguments"; return GFCC_ERR_ARG; }
  for (int k = 0; k < norb; ++k)
    if (orbitals[k] < 0 || orbitals[k] >= c->n) { c->last_error = "gfcc_vectors: orbital out of range"; return GFCC_ERR_ARG; }
  API_BEGIN
  const double* src = transpose ? c->cvec.p : c->bvec.p;
  DBuf<double> neg;
  if (c->sector == 1 && !transpose) neg.alloc(c->D);   // EA free terms are held as -b_q (the IP form)
  for (int k = 0; k < norb; ++k) {
    const double* row = src + (long long)orbitals[k] * c->D;
    if (neg.p) {
      gfcc::axpby(c->D, -1.0, row, 0.0, neg.p, c->stream);
      row = neg.p;
    }
    copy_out(out + (long long)k * ld, row, sizeof(double) * c->D, c->stream);
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
  }
  API_END(c)
}

static int check_orbitals(gfcc_t c, const int* orb, int n, const char* what) {
  if (n <= 0 || !orb) { c->last_error = std::string(what) + ": empty orbital set"; return GFCC_ERR_ARG; }
  for (int k = 0; k < n; ++k)
    if (orb[k] < 0 || orb[k] >= c->n) { c->last_error = std::string(what) + ": orbital out of range"; return GFCC_ERR_ARG; }
  return GFCC_OK;
}

// Frequencies as the solver sees them: the EA systems (w + i eta - M) y = b are solved in the IP form
// (w' - i eta + M) y = -b at w' = -w.
static std::vector<double> solver_freqs(gfcc_t c, const double* w, int n) {
  std::vector<double> ws(w, w + n);
  if (c->sector == 1)
    for (double& x : ws) x = -x;
  return ws;
}
static double user_freq(gfcc_t c, double w) { return c->sector == 1 ? -w : w; }

int gfcc_solve_full(gfcc_t c, const double* omegas, int nw, double eta, const int* orbitals, int np,
                    const int* qorb, int nq, double* G, double* A, double* X, int ldx, gfcc_stats* stats) {
  if (!c) return GFCC_ERR_ARG;
  if (nw < 0 || (nw > 0 && !omegas) || !std::isfinite(eta) || eta < 0.0) { c->last_error = "gfcc_solve_full: bad frequencies or eta"; return GFCC_ERR_ARG; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_solve_full");
  if (rc) return rc;
  if (qorb) { rc = check_orbitals(c, qorb, nq, "gfcc_solve_full(q)"); if (rc) return rc; }
  if (X && ldx < c->D) { c->last_error = "gfcc_solve_full: ldx < D"; return GFCC_ERR_ARG; }
  for (int k = 0; k < nw; ++k)
    if (!std::isfinite(omegas[k])) { c->last_error = "gfcc_solve_full: non-finite frequency"; return GFCC_ERR_NONFINITE; }
  API_BEGIN
  if (nw == 0) return GFCC_OK;
  cudaStream_t s = c->stream;
  const long long D = c->D;
  std::vector<int> porb(orbitals, orbitals + np);
  std::vector<int> qv = qorb ? std::vector<int>(qorb, qorb + nq) : porb;
  nq = (int)qv.size();
  std::vector<double> ws = solver_freqs(c, omegas, nw);
  const long long ncols = (long long)nw * np;
  DBuf<cplx> Gd, Xd;
  DBuf<double> Ad;
  DBuf<int> dq;
  const bool needG = G || A;
  if (needG) Gd.alloc(ncols * nq);
  if (X) Xd.alloc(D * ncols);
  gfcc_stats st{};
  solve_columns(c, ws, eta, porb, qv, needG ? Gd.p : nullptr, X ? Xd.p : nullptr, nullptr, &st);
  if (A) {
    std::vector<int> qi = q_positions(porb, qv);
    dq.alloc(np);
    Ad.alloc(nw);
    GFCC_CUDA(cudaMemcpyAsync(dq.p, qi.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    spectral_kernel<<<(nw + 127) / 128, 128, 0, s>>>(Gd.p, nw, np, nq, dq.p, Ad.p);
    GFCC_LAUNCH_CHECK();
    copy_out(A, Ad.p, sizeof(double) * nw, s);
  }
  if (G) copy_out(G, Gd.p, sizeof(cplx) * ncols * nq, s);
  if (X) {
    if (is_device_ptr(X)) {
      gfcc::batch_to_cols(Xd.p, (int)ncols, (int)ncols, (int)D, reinterpret_cast<cplx*>(X), ldx, s);
    } else {
      DBuf<cplx> stage;
      stage.alloc(ncols * ldx);
      gfcc::batch_to_cols(Xd.p, (int)ncols, (int)ncols, (int)D, stage.p, ldx, s);
      GFCC_CUDA(cudaMemcpyAsync(X, stage.p, sizeof(cplx) * ncols * ldx, cudaMemcpyDeviceToHost, s));
      GFCC_CUDA(cudaStreamSynchronize(s));
    }
  }
  GFCC_CUDA(cudaStreamSynchronize(s));
  if (stats) *stats = st;
  if (st.not_converged > 0) {
    c->last_error = "gfcc_solve_full: " + std::to_string(st.not_converged) + " column(s) not converged";
    return GFCC_ERR_NOT_CONVERGED;
  }
  API_END(c)
}

int gfcc_green_derivatives(gfcc_t c, const double* omegas, int nw, double eta, const int* orbitals, int np,
                           const int* qorb, int nq, double* G, double* dG_domega, double* dG_deta) {
  if (!c) return GFCC_ERR_ARG;
  if (nw <= 0 || !omegas || !std::isfinite(eta) || eta < 0.0) { c->last_error = "gfcc_green_derivatives: bad frequencies or eta"; return GFCC_ERR_ARG; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_green_derivatives");
  if (rc) return rc;
  if (qorb) { rc = check_orbitals(c, qorb, nq, "gfcc_green_derivatives(q)"); if (rc) return rc; }
  for (int k = 0; k < nw; ++k)
    if (!std::isfinite(omegas[k])) { c->last_error = "gfcc_green_derivatives: non-finite frequency"; return GFCC_ERR_NONFINITE; }
  API_BEGIN
  cudaStream_t s = c->stream;
  const long long D = c->D;
  std::vector<int> porb(orbitals, orbitals + np);
  std::vector<int> qv = qorb ? std::vector<int>(qorb, qorb + nq) : porb;
  nq = (int)qv.size();
  std::vector<double> ws = solver_freqs(c, omegas, nw);
  const long long nx = (long long)nw * np, ny = (long long)nw * nq;
  DBuf<cplx> X, Y, Gd, dwd, ded, part;
  X.alloc(D * nx);
  Y.alloc(D * ny);
  if (G) Gd.alloc(nx * nq);
  gfcc_stats st{};
  solve_columns(c, ws, eta, porb, qv, G ? Gd.p : nullptr, X.p, nullptr, &st);
  GFCC_CHECK(st.not_converged == 0, GFCC_ERR_NOT_CONVERGED, "gfcc_green_derivatives: forward solve did not converge");
  solve_adjoint_columns(c, ws, eta, qv, Y.p);
  const int ntrip = (int)(nx * nq);
  const long long rows = std::max<long long>(64, (D + 2 * 152 - 1) / (2 * 152));
  const int nchunk = (int)((D + rows - 1) / rows);
  part.alloc((long long)nchunk * ntrip);
  dwd.alloc(ntrip);
  ded.alloc(ntrip);
  bilinear_partial_kernel<<<nchunk, 256, 0, s>>>(X.p, Y.p, D, nw, np, nq, rows, part.p);
  GFCC_LAUNCH_CHECK();
  bilinear_reduce_kernel<<<(ntrip + 255) / 256, 256, 0, s>>>(part.p, nchunk, ntrip, dwd.p, ded.p);
  GFCC_LAUNCH_CHECK();
  if (c->sector == 1)   // EA: the solver's frequency is -w, so dG/dw changes sign (eta enters both forms alike)
    gfcc::axpby(2LL * ntrip, -1.0, reinterpret_cast<const double*>(dwd.p), 0.0, reinterpret_cast<double*>(dwd.p), s);
  if (G) copy_out(G, Gd.p, sizeof(cplx) * ntrip, s);
  if (dG_domega) copy_out(dG_domega, dwd.p, sizeof(cplx) * ntrip, s);
  if (dG_deta) copy_out(dG_deta, ded.p, sizeof(cplx) * ntrip, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
  API_END(c)
}

int gfcc_green_grad_t2(gfcc_t c, const double* omegas, int nw, double eta, const int* orbitals, int np,
                       const int* qorb, int nq, const double* Gbar, double* G, double* grad_t2) {
  if (!c) return GFCC_ERR_ARG;
  if (nw <= 0 || !omegas || !std::isfinite(eta) || eta < 0.0 || !Gbar || !grad_t2) {
    c->last_error = "gfcc_green_grad_t2: bad frequencies, eta or null pointers";
    return GFCC_ERR_ARG;
  }
  if (c->sector != 0) { c->last_error = "gfcc_green_grad_t2: available for the IP space only"; return GFCC_ERR_STATE; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_green_grad_t2");
  if (rc) return rc;
  if (qorb) { rc = check_orbitals(c, qorb, nq, "gfcc_green_grad_t2(q)"); if (rc) return rc; }
  for (int k = 0; k < nw; ++k)
    if (!std::isfinite(omegas[k])) { c->last_error = "gfcc_green_grad_t2: non-finite frequency"; return GFCC_ERR_NONFINITE; }
  API_BEGIN
  cudaStream_t s = c->stream;
  const long long D = c->D;
  std::vector<int> porb(orbitals, orbitals + np);
  std::vector<int> qv = qorb ? std::vector<int>(qorb, qorb + nq) : porb;
  nq = (int)qv.size();
  std::vector<double> ws = solver_freqs(c, omegas, nw);
  const long long S = (long long)nw * np;
  DBuf<cplx> X, W, U, Gb, Gd;
  DBuf<double> t2b;
  X.alloc(D * S); W.alloc(D * S); U.alloc(D * S);
  Gb.alloc(S * nq);
  GFCC_CUDA(cudaMemcpyAsync(Gb.p, Gbar, sizeof(cplx) * S * nq, gfcc::kind_to_device(Gbar), s));
  if (G) Gd.alloc(S * nq);
  gfcc_stats st{};
  solve_columns(c, ws, eta, porb, qv, G ? Gd.p : nullptr, X.p, nullptr, &st);
  GFCC_CHECK(st.not_converged == 0, GFCC_ERR_NOT_CONVERGED, "gfcc_green_grad_t2: forward solve did not converge");
  gfcc::green_adjoint_rhs(c, qv, Gb.p, S, W.p);
  solve_rhs(c, ws, eta, np, W.p, U.p, true);
  const long long n2 = (long long)c->o * c->o * c->v * c->v;
  t2b.alloc(n2);
  gfcc::green_grad_t2_core(c, nw, porb, qv, Gb.p, X.p, U.p, t2b.p);
  copy_out(grad_t2, t2b.p, sizeof(double) * n2, s);
  if (G) copy_out(G, Gd.p, sizeof(cplx) * S * nq, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
  API_END(c)
}

int gfcc_mor_build(gfcc_t c, const double* seeds, int ns, double eta, const int* orbitals, int np,
                   const int* qorb, int nq) {
  if (!c) return GFCC_ERR_ARG;
  if (ns <= 0 || !seeds || !std::isfinite(eta) || eta <= 0.0) { c->last_error = "gfcc_mor_build: bad seeds or eta"; return GFCC_ERR_ARG; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_mor_build");
  if (rc) return rc;
  if (qorb) { rc = check_orbitals(c, qorb, nq, "gfcc_mor_build(q)"); if (rc) return rc; }
  for (int k = 0; k < ns; ++k)
    if (!std::isfinite(seeds[k])) { c->last_error = "gfcc_mor_build: non-finite seed"; return GFCC_ERR_NONFINITE; }
  API_BEGIN
  c->siso.clear();
  gfcc::MorState& ms = c->mor;
  ms.reset();
  ms.eta = eta;
  ms.porb.assign(orbitals, orbitals + np);
  ms.qorb = qorb ? std::vector<int>(qorb, qorb + nq) : ms.porb;
  {  // ||b_p||^2
    DBuf<int> idx;
    DBuf<double> out;
    idx.alloc(np); out.alloc(np);
    GFCC_CUDA(cudaMemcpyAsync(idx.p, ms.porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, c->stream));
    rownorm2_kernel<<<np, 256, 0, c->stream>>>(c->bvec.p, c->D, idx.p, np, out.p);
    GFCC_LAUNCH_CHECK();
    ms.bnorm.resize(np);
    GFCC_CUDA(cudaMemcpyAsync(ms.bnorm.data(), out.p, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
    for (double& x : ms.bnorm) x = std::sqrt(x);
    for (double x : ms.bnorm) GFCC_CHECK(x > 0.0, GFCC_ERR_ARG, "gfcc_mor_build: zero right-hand side");
  }
  gfcc::mor_init_basis(c);
  std::vector<double> ws = solver_freqs(c, seeds, ns);
  std::sort(ws.begin(), ws.end());
  ws.erase(std::unique(ws.begin(), ws.end()), ws.end());
  mor_add_frequencies(c, ws);
  GFCC_CHECK(ms.m > 0, GFCC_ERR_RANK, "gfcc_mor_build: every seed solution was dropped");
  ms.built = true;
  API_END(c)
}

int gfcc_mor_refine(gfcc_t c, double wmin, double wmax, int ngrid, double tol, int m_max, int* m_out,
                    double* max_err) {
  if (!c) return GFCC_ERR_ARG;
  if (!c->mor.built && c->siso.empty()) { c->last_error = "gfcc_mor_refine: call gfcc_mor_build first"; return GFCC_ERR_STATE; }
  if (!(wmax > wmin) || ngrid < 2 || !(tol > 0.0) || m_max < 1 || !std::isfinite(wmin) || !std::isfinite(wmax)) {
    c->last_error = "gfcc_mor_refine: bad arguments";
    return GFCC_ERR_ARG;
  }
  if (!c->siso.empty() && c->opts.deriv_indicator) {
    c->last_error = "gfcc_mor_refine: the derivative indicator is not available for per-orbital models";
    return GFCC_ERR_ARG;
  }
  API_BEGIN
  if (c->sector == 1) {   // EA: the window in the solver's frequency w' = -w
    const double lo = -wmax, hi = -wmin;
    wmin = lo;
    wmax = hi;
  }
  std::vector<double> grid(ngrid);
  for (int k = 0; k < ngrid; ++k) grid[k] = wmin + (wmax - wmin) * (double)k / (double)(ngrid - 1);
  DBuf<double> dres;
  dres.alloc(ngrid);
  bool converged = false;
  double emax = 0.0;
  if (!c->siso.empty()) {   // per-orbital models: each refines its own frequencies, all solved together
    const double eta = c->siso[0].eta;
    for (int round = 0; round < 10000; ++round) {
      emax = 0.0;
      std::vector<std::pair<int, double>> add;
      for (size_t k = 0; k < c->siso.size(); ++k) {
        ModelSwap sw(c, &c->siso[k]);
        gfcc::MorState& ms = c->mor;
        std::vector<double> e = interval_errors(c, grid, dres);
        double ek = 0.0;
        for (double x : e) ek = std::max(ek, x);
        ms.history.push_back({ms.m, ek});
        ms.last_max_err = ek;
        emax = std::max(emax, ek);
        if (ek <= tol) continue;
        for (double w : choose_midpoints(ms.sampled, e, tol, m_max - ms.m)) add.push_back({(int)k, w});
      }
      if (emax <= tol) { converged = true; break; }
      if (add.empty()) break;
      siso_add_frequencies(c, add, eta);
    }
    int m = 0;
    for (const gfcc::MorState& ms : c->siso) m += ms.m;
    if (m_out) *m_out = m;
    if (max_err) *max_err = emax;
    if (!converged) {
      c->last_error = "gfcc_mor_refine: model order bound reached before the tolerance";
      return GFCC_ERR_NOT_CONVERGED;
    }
    return GFCC_OK;
  }
  gfcc::MorState& ms = c->mor;
  const int np = (int)ms.porb.size();
  if (ms.kind == 1) {   // Krylov subspace: grow it until the residual estimate meets tol on the whole grid
    GFCC_CHECK(!c->opts.deriv_indicator, GFCC_ERR_ARG,
               "gfcc_mor_refine: the derivative indicator needs sampled frequencies (not a Krylov model)");
    std::vector<double> res(ngrid);
    for (int round = 0; round < 100000; ++round) {
      gfcc::mor_eval(c, grid.data(), ngrid, nullptr, nullptr, dres.p);
      GFCC_CUDA(cudaMemcpyAsync(res.data(), dres.p, sizeof(double) * ngrid, cudaMemcpyDeviceToHost, c->stream));
      GFCC_CUDA(cudaStreamSynchronize(c->stream));
      emax = 0.0;
      for (double x : res) emax = std::max(emax, x);
      ms.history.push_back({ms.m, emax});
      ms.last_max_err = emax;
      if (emax <= tol) { converged = true; break; }
      const int m0 = ms.m;
      krylov_extend(c, std::max(1, ms.kblocks / 4), m_max);   // about 25 % more blocks per round
      if (ms.m == m0) break;                                   // order bound reached or space exhausted
    }
    if (m_out) *m_out = ms.m;
    if (max_err) *max_err = emax;
    if (!converged) {
      c->last_error = "gfcc_mor_refine: model order bound reached before the tolerance";
      return GFCC_ERR_NOT_CONVERGED;
    }
    return GFCC_OK;
  }
  for (int round = 0; round < 10000; ++round) {
    std::vector<double> e = interval_errors(c, grid, dres);
    const std::vector<double>& smp = ms.sampled;
    if (c->opts.deriv_indicator && smp.size() > 1) {   // derivative mismatch at the sampled ends
      const int nq = (int)ms.qorb.size();
      const int ns = (int)smp.size();
      DBuf<cplx> dGh;
      dGh.alloc((long long)ns * np * nq);
      gfcc::mor_eval(c, smp.data(), ns, nullptr, nullptr, nullptr, dGh.p);
      std::vector<cplx> h((size_t)ns * np * nq);
      GFCC_CUDA(cudaMemcpyAsync(h.data(), dGh.p, sizeof(cplx) * h.size(), cudaMemcpyDeviceToHost, c->stream));
      GFCC_CUDA(cudaStreamSynchronize(c->stream));
      std::vector<double> d(ns, 0.0);
      for (int k = 0; k < ns; ++k) {
        const std::vector<cplx>* ex = nullptr;
        for (auto& pr : ms.dG_exact)
          if (pr.first == smp[k]) { ex = &pr.second; break; }
        if (!ex) continue;
        double num = 0.0, den = 0.0;
        for (int t = 0; t < np * nq; ++t) {
          const cplx a = h[(size_t)k * np * nq + t], b = (*ex)[t];
          num = std::max(num, std::hypot(a.x - b.x, a.y - b.y));
          den = std::max(den, std::hypot(b.x, b.y));
        }
        d[k] = den > 0.0 ? num / den : 0.0;
      }
      for (size_t k = 0; k < e.size(); ++k) e[k] = std::max(e[k], std::max(d[k], d[k + 1]));
    }
    emax = 0.0;
    for (double x : e) emax = std::max(emax, x);
    ms.history.push_back({ms.m, emax});
    ms.last_max_err = emax;
    if (emax <= tol) { converged = true; break; }
    std::vector<double> nw = choose_midpoints(smp, e, tol, (m_max - ms.m) / np);
    if (nw.empty()) break;
    mor_add_frequencies(c, nw);
  }
  if (m_out) *m_out = ms.m;
  if (max_err) *max_err = emax;
  if (!converged) {
    c->last_error = "gfcc_mor_refine: model order bound reached before the tolerance";
    return GFCC_ERR_NOT_CONVERGED;
  }
  API_END(c)
}

int gfcc_mor_eval(gfcc_t c, const double* omegas, int nw, double* G, double* A, double* maxres) {
  if (!c) return GFCC_ERR_ARG;
  if (!c->mor.built && c->siso.empty()) { c->last_error = "gfcc_mor_eval: no reduced model"; return GFCC_ERR_STATE; }
  if (nw < 0 || (nw > 0 && !omegas)) { c->last_error = "gfcc_mor_eval: bad frequencies"; return GFCC_ERR_ARG; }
  for (int k = 0; k < nw; ++k)
    if (!std::isfinite(omegas[k])) { c->last_error = "gfcc_mor_eval: non-finite frequency"; return GFCC_ERR_NONFINITE; }
  API_BEGIN
  if (nw == 0) return GFCC_OK;
  cudaStream_t s = c->stream;
  const std::vector<double> wsol = solver_freqs(c, omegas, nw);
  omegas = wsol.data();
  if (!c->siso.empty()) {   // per-orbital models: G_pp on the diagonal of [nw][np][np], zero elsewhere
    const int np = (int)c->siso.size();
    DBuf<cplx> Gd, Gk;
    DBuf<double> Ad, Rd, Rk;
    DBuf<int> dq;
    Gd.alloc((long long)nw * np * np);
    Gk.alloc(nw);
    Gd.zero(s);
    if (maxres) {
      Rd.alloc(nw);
      Rk.alloc(nw);
      Rd.zero(s);
    }
    for (int k = 0; k < np; ++k) {
      ModelSwap sw(c, &c->siso[k]);
      gfcc::mor_eval(c, omegas, nw, Gk.p, nullptr, maxres ? Rk.p : nullptr);
      GFCC_CUDA(cudaMemcpy2DAsync(Gd.p + (long long)k * (np + 1), sizeof(cplx) * np * np, Gk.p, sizeof(cplx),
                                  sizeof(cplx), nw, cudaMemcpyDeviceToDevice, s));
      if (maxres) {
        max_into_kernel<<<(nw + 255) / 256, 256, 0, s>>>(Rk.p, Rd.p, nw);
        GFCC_LAUNCH_CHECK();
      }
      GFCC_CUDA(cudaStreamSynchronize(s));
    }
    if (A) {
      std::vector<int> qi(np);
      for (int k = 0; k < np; ++k) qi[k] = k;
      dq.alloc(np);
      Ad.alloc(nw);
      GFCC_CUDA(cudaMemcpyAsync(dq.p, qi.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
      spectral_kernel<<<(nw + 127) / 128, 128, 0, s>>>(Gd.p, nw, np, np, dq.p, Ad.p);
      GFCC_LAUNCH_CHECK();
      copy_out(A, Ad.p, sizeof(double) * nw, s);
    }
    if (G) copy_out(G, Gd.p, sizeof(cplx) * nw * np * np, s);
    if (maxres) copy_out(maxres, Rd.p, sizeof(double) * nw, s);
    GFCC_CUDA(cudaStreamSynchronize(s));
    return GFCC_OK;
  }
  gfcc::MorState& ms = c->mor;
  const int np = (int)ms.porb.size(), nq = (int)ms.qorb.size();
  DBuf<cplx> Gd;
  DBuf<double> Ad, Rd;
  if (G) Gd.alloc((long long)nw * np * nq);
  if (A) Ad.alloc(nw);
  if (maxres) Rd.alloc(nw);
  gfcc::mor_eval(c, omegas, nw, G ? Gd.p : nullptr, A ? Ad.p : nullptr, maxres ? Rd.p : nullptr);
  if (G) copy_out(G, Gd.p, sizeof(cplx) * nw * np * nq, s);
  if (A) copy_out(A, Ad.p, sizeof(double) * nw, s);
  if (maxres) copy_out(maxres, Rd.p, sizeof(double) * nw, s);
  GFCC_CUDA(cudaStreamSynchronize(s));
  API_END(c)
}

int gfcc_mor_info(gfcc_t c, double* w, int cap, int* ns, int* m, int* np, int* nq) {
  if (!c) return GFCC_ERR_ARG;
  if (!c->siso.empty()) {   // union of the per-orbital models' frequencies, total order
    std::vector<double> all;
    int mt = 0;
    for (const gfcc::MorState& ms : c->siso) {
      all.insert(all.end(), ms.sampled.begin(), ms.sampled.end());
      mt += ms.m;
    }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    if (ns) *ns = (int)all.size();
    if (m) *m = mt;
    if (np) *np = (int)c->siso.size();
    if (nq) *nq = (int)c->siso.size();
    if (c->sector == 1) {
      for (double& x : all) x = -x;
      std::sort(all.begin(), all.end());
    }
    if (w)
      for (int k = 0; k < cap && k < (int)all.size(); ++k) w[k] = all[k];
    return GFCC_OK;
  }
  const gfcc::MorState& ms = c->mor;
  if (ns) *ns = (int)ms.sampled.size();
  if (m) *m = ms.m;
  if (np) *np = (int)ms.porb.size();
  if (nq) *nq = (int)ms.qorb.size();
  if (w)
    for (int k = 0; k < cap && k < (int)ms.sampled.size(); ++k) w[k] = user_freq(c, ms.sampled[k]);
  return GFCC_OK;
}

int gfcc_mor_model_info(gfcc_t c, int k, int* orbital, double* w, int cap, int* ns, int* m) {
  if (!c) return GFCC_ERR_ARG;
  const int nmod = c->siso.empty() ? (c->mor.built ? 1 : 0) : (int)c->siso.size();
  if (k < 0 || k >= nmod) { c->last_error = "gfcc_mor_model_info: no such model"; return GFCC_ERR_ARG; }
  const gfcc::MorState& ms = c->siso.empty() ? c->mor : c->siso[k];
  if (orbital) *orbital = c->siso.empty() ? -1 : ms.porb[0];
  if (ns) *ns = (int)ms.sampled.size();
  if (m) *m = ms.m;
  if (w)
    for (int j = 0; j < cap && j < (int)ms.sampled.size(); ++j) w[j] = user_freq(c, ms.sampled[j]);
  return GFCC_OK;
}

int gfcc_mor_stats(gfcc_t c, long long* arnoldi_steps, long long* columns) {
  if (!c) return GFCC_ERR_ARG;
  const bool siso = !c->siso.empty();
  if (arnoldi_steps) *arnoldi_steps = siso ? c->siso_iters : c->mor.solve_iters;
  if (columns) *columns = siso ? c->siso_cols : c->mor.solve_cols;
  return GFCC_OK;
}

int gfcc_mor_build_siso(gfcc_t c, const double* seeds, int ns, double eta, const int* orbitals, int np) {
  if (!c) return GFCC_ERR_ARG;
  if (ns <= 0 || !seeds || !std::isfinite(eta) || eta <= 0.0) { c->last_error = "gfcc_mor_build_siso: bad seeds or eta"; return GFCC_ERR_ARG; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_mor_build_siso");
  if (rc) return rc;
  for (int k = 0; k < ns; ++k)
    if (!std::isfinite(seeds[k])) { c->last_error = "gfcc_mor_build_siso: non-finite seed"; return GFCC_ERR_NONFINITE; }
  for (int a = 0; a < np; ++a)
    for (int b = a + 1; b < np; ++b)
      if (orbitals[a] == orbitals[b]) { c->last_error = "gfcc_mor_build_siso: repeated orbital"; return GFCC_ERR_ARG; }
  API_BEGIN
  c->mor.reset();
  c->siso.clear();
  c->siso.resize(np);
  c->siso_iters = 0;
  c->siso_cols = 0;
  std::vector<int> idx(orbitals, orbitals + np);
  std::vector<double> bn(np);
  {  // ||b_p||^2
    DBuf<int> di;
    DBuf<double> out;
    di.alloc(np); out.alloc(np);
    GFCC_CUDA(cudaMemcpyAsync(di.p, idx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, c->stream));
    rownorm2_kernel<<<np, 256, 0, c->stream>>>(c->bvec.p, c->D, di.p, np, out.p);
    GFCC_LAUNCH_CHECK();
    GFCC_CUDA(cudaMemcpyAsync(bn.data(), out.p, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
  }
  for (int k = 0; k < np; ++k) {
    GFCC_CHECK(bn[k] > 0.0, GFCC_ERR_ARG, "gfcc_mor_build_siso: zero right-hand side");
    ModelSwap sw(c, &c->siso[k]);
    gfcc::MorState& ms = c->mor;
    ms.eta = eta;
    ms.porb = {orbitals[k]};
    ms.qorb = {orbitals[k]};
    ms.bnorm = {std::sqrt(bn[k])};
    gfcc::mor_init_basis(c);
  }
  std::vector<double> ws = solver_freqs(c, seeds, ns);
  std::sort(ws.begin(), ws.end());
  ws.erase(std::unique(ws.begin(), ws.end()), ws.end());
  std::vector<std::pair<int, double>> add;
  for (int k = 0; k < np; ++k)
    for (double w : ws) add.push_back({k, w});
  siso_add_frequencies(c, add, eta);
  for (gfcc::MorState& ms : c->siso) {
    GFCC_CHECK(ms.m > 0, GFCC_ERR_RANK, "gfcc_mor_build_siso: every seed solution of an orbital was dropped");
    ms.built = true;
  }
  API_END(c)
}

int gfcc_mor_build_krylov(gfcc_t c, int nblocks, double eta, const int* orbitals, int np, const int* qorb, int nq) {
  if (!c) return GFCC_ERR_ARG;
  if (nblocks < 1 || !std::isfinite(eta) || eta <= 0.0) { c->last_error = "gfcc_mor_build_krylov: bad block count or eta"; return GFCC_ERR_ARG; }
  int rc = check_orbitals(c, orbitals, np, "gfcc_mor_build_krylov");
  if (rc) return rc;
  if (qorb) { rc = check_orbitals(c, qorb, nq, "gfcc_mor_build_krylov(q)"); if (rc) return rc; }
  API_BEGIN
  c->siso.clear();
  gfcc::MorState& ms = c->mor;
  ms.reset();
  ms.kind = 1;
  ms.eta = eta;
  ms.porb.assign(orbitals, orbitals + np);
  ms.qorb = qorb ? std::vector<int>(qorb, qorb + nq) : ms.porb;
  {  // ||b_p||^2
    DBuf<int> idx;
    DBuf<double> out;
    idx.alloc(np); out.alloc(np);
    GFCC_CUDA(cudaMemcpyAsync(idx.p, ms.porb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, c->stream));
    rownorm2_kernel<<<np, 256, 0, c->stream>>>(c->bvec.p, c->D, idx.p, np, out.p);
    GFCC_LAUNCH_CHECK();
    ms.bnorm.resize(np);
    GFCC_CUDA(cudaMemcpyAsync(ms.bnorm.data(), out.p, sizeof(double) * np, cudaMemcpyDeviceToHost, c->stream));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
    for (double& x : ms.bnorm) x = std::sqrt(x);
    for (double x : ms.bnorm) GFCC_CHECK(x > 0.0, GFCC_ERR_ARG, "gfcc_mor_build_krylov: zero right-hand side");
  }
  gfcc::mor_init_basis(c);
  krylov_extend(c, nblocks, 2147483647);   // no order bound here: dependent columns are dropped anyway
  GFCC_CHECK(ms.m > 0, GFCC_ERR_RANK, "gfcc_mor_build_krylov: empty subspace");
  ms.built = true;
  API_END(c)
}

int gfcc_mor_save(gfcc_t c, const char* path) {
  if (!c || !path) return GFCC_ERR_ARG;
  if (!c->siso.empty()) { c->last_error = "gfcc_mor_save: per-orbital model sets are not saved"; return GFCC_ERR_STATE; }
  if (c->mor.kind != 0) { c->last_error = "gfcc_mor_save: Krylov models are not saved"; return GFCC_ERR_STATE; }
  if (!c->mor.built) { c->last_error = "gfcc_mor_save: no reduced model"; return GFCC_ERR_STATE; }
  API_BEGIN
  const gfcc::MorState& ms = c->mor;
  const long long D = c->D;
  const int m = ms.m, cap = ms.m_cap, np = (int)ms.porb.size(), nq = (int)ms.qorb.size();
  const int qn = ms.qn, qcap = ms.q_cap;
  std::ofstream f(path, std::ios::binary);
  GFCC_CHECK(f.good(), GFCC_ERR_ARG, std::string("gfcc_mor_save: cannot open ") + path);
  // the EA space has its own tag: its block sizes can equal those of an IP space with o and v exchanged
  const char magic[8] = {'G', 'F', 'C', 'C', 'M', 'O', 'R', c->sector == 1 ? 'E' : '2'};
  f.write(magic, 8);
  int hdr[7] = {c->o, c->v, (int)D, m, np, nq, qn};
  f.write(reinterpret_cast<const char*>(hdr), sizeof(hdr));
  f.write(reinterpret_cast<const char*>(&ms.eta), sizeof(double));
  int ns = (int)ms.sampled.size();
  f.write(reinterpret_cast<const char*>(&ns), sizeof(int));
  f.write(reinterpret_cast<const char*>(ms.sampled.data()), sizeof(double) * ns);
  f.write(reinterpret_cast<const char*>(ms.porb.data()), sizeof(int) * np);
  f.write(reinterpret_cast<const char*>(ms.qorb.data()), sizeof(int) * nq);
  f.write(reinterpret_cast<const char*>(ms.bnorm.data()), sizeof(double) * np);
  std::vector<cplx> h;
  auto dump2d = [&](const cplx* dev, long long rows, int width, int ld) {   // rows x width out of ld
    h.resize((size_t)rows * width);
    GFCC_CUDA(cudaMemcpy2D(h.data(), sizeof(cplx) * width, dev, sizeof(cplx) * ld, sizeof(cplx) * width, rows,
                           cudaMemcpyDeviceToHost));
    f.write(reinterpret_cast<const char*>(h.data()), sizeof(cplx) * h.size());
  };
  dump2d(ms.S.p, D, m, cap);
  dump2d(ms.Z.p, D, m, cap);
  dump2d(ms.Hh.p, m, m, cap);      // col-major: m columns of m entries
  dump2d(ms.bh.p, np, m, cap);
  dump2d(ms.ch.p, m, nq, nq);
  dump2d(ms.Q.p, D, qn, qcap);
  dump2d(ms.RS.p, m, qn, qcap);
  dump2d(ms.RZ.p, m, qn, qcap);
  dump2d(ms.RB.p, np, qn, qcap);
  GFCC_CHECK(f.good(), GFCC_ERR_ARG, "gfcc_mor_save: write failed");
  API_END(c)
}

int gfcc_mor_load(gfcc_t c, const char* path) {
  if (!c || !path) return GFCC_ERR_ARG;
  API_BEGIN
  std::ifstream f(path, std::ios::binary);
  GFCC_CHECK(f.good(), GFCC_ERR_ARG, std::string("gfcc_mor_load: cannot open ") + path);
  char magic[8];
  f.read(magic, 8);
  GFCC_CHECK(f.good() && std::memcmp(magic, c->sector == 1 ? "GFCCMORE" : "GFCCMOR2", 8) == 0, GFCC_ERR_ARG,
             "gfcc_mor_load: not a model file of this space (IP or EA)");
  int hdr[7];
  f.read(reinterpret_cast<char*>(hdr), sizeof(hdr));
  GFCC_CHECK(f.good() && hdr[0] == c->o && hdr[1] == c->v && hdr[2] == c->D, GFCC_ERR_ARG,
             "gfcc_mor_load: size mismatch");
  const int m = hdr[3], np = hdr[4], nq = hdr[5], qn = hdr[6];
  GFCC_CHECK(m > 0 && np > 0 && nq > 0 && qn >= m && np <= c->n && nq <= c->n && m <= c->D, GFCC_ERR_ARG,
             "gfcc_mor_load: corrupt header");
  c->siso.clear();
  gfcc::MorState& ms = c->mor;
  ms.reset();
  f.read(reinterpret_cast<char*>(&ms.eta), sizeof(double));
  int ns = 0;
  f.read(reinterpret_cast<char*>(&ns), sizeof(int));
  GFCC_CHECK(f.good() && ns > 0 && ns < (1 << 24), GFCC_ERR_ARG, "gfcc_mor_load: corrupt header");
  ms.sampled.resize(ns);
  ms.porb.resize(np);
  ms.qorb.resize(nq);
  ms.bnorm.resize(np);
  f.read(reinterpret_cast<char*>(ms.sampled.data()), sizeof(double) * ns);
  f.read(reinterpret_cast<char*>(ms.porb.data()), sizeof(int) * np);
  f.read(reinterpret_cast<char*>(ms.qorb.data()), sizeof(int) * nq);
  f.read(reinterpret_cast<char*>(ms.bnorm.data()), sizeof(double) * np);
  GFCC_CHECK(f.good(), GFCC_ERR_ARG, "gfcc_mor_load: truncated file");
  const long long D = c->D;
  const int cap = std::max(m, 64), qcap = std::max(qn, 128);
  ms.m_cap = cap;
  ms.q_cap = qcap;
  ms.S.alloc(D * cap); ms.Z.alloc(D * cap);
  ms.Hh.alloc((long long)cap * cap);
  ms.bh.alloc((long long)cap * np);
  ms.ch.alloc((long long)nq * cap);
  ms.Q.alloc(D * qcap);
  ms.RS.alloc((long long)qcap * cap); ms.RZ.alloc((long long)qcap * cap);
  ms.RB.alloc((long long)qcap * np);
  for (DBuf<cplx>* b : {&ms.S, &ms.Z, &ms.Hh, &ms.bh, &ms.ch, &ms.Q, &ms.RS, &ms.RZ, &ms.RB}) b->zero(c->stream);
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<cplx> h;
  auto load2d = [&](cplx* dev, long long rows, int width, int ld) {
    h.resize((size_t)rows * width);
    f.read(reinterpret_cast<char*>(h.data()), sizeof(cplx) * h.size());
    GFCC_CHECK(f.good(), GFCC_ERR_ARG, "gfcc_mor_load: truncated file");
    GFCC_CUDA(cudaMemcpy2D(dev, sizeof(cplx) * ld, h.data(), sizeof(cplx) * width, sizeof(cplx) * width, rows,
                           cudaMemcpyHostToDevice));
  };
  load2d(ms.S.p, D, m, cap);
  load2d(ms.Z.p, D, m, cap);
  load2d(ms.Hh.p, m, m, cap);
  load2d(ms.bh.p, np, m, cap);
  load2d(ms.ch.p, m, nq, nq);
  load2d(ms.Q.p, D, qn, qcap);
  load2d(ms.RS.p, m, qn, qcap);
  load2d(ms.RZ.p, m, qn, qcap);
  load2d(ms.RB.p, np, qn, qcap);
  ms.m = m;
  ms.qn = qn;
  ms.built = true;
  ++ms.version;
  API_END(c)
}

int gfcc_tc_gemm(int precision, const double* A, const double* B, int M, int N, int K, float* C) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (precision != GFCC_PREC_BF16 && precision != GFCC_PREC_TF32))
    return GFCC_ERR_ARG;
  try {
    DBuf<double> a, b;
    DBuf<float> cdev;
    a.alloc((size_t)M * K);
    b.alloc((size_t)N * K);
    cdev.alloc((size_t)M * N);
    GFCC_CUDA(cudaMemcpy(a.p, A, sizeof(double) * M * K, cudaMemcpyHostToDevice));
    GFCC_CUDA(cudaMemcpy(b.p, B, sizeof(double) * N * K, cudaMemcpyHostToDevice));
    gfcc::tc_selftest(precision, a.p, b.p, M, N, K, cdev.p, nullptr);
    GFCC_CUDA(cudaMemcpy(C, cdev.p, sizeof(float) * M * N, cudaMemcpyDeviceToHost));
  } catch (gfcc::Error& e) {
    fprintf(stderr, "gfcc_tc_gemm: %s\n", e.msg.c_str());
    return e.code;
  }
  return GFCC_OK;
}

int gfcc_spectral(const double* G, int nw, const int* orbitals, int np, const int* qorb, int nq, double* A,
                  int adjoint, void* stream) {
  if (nw < 0 || np < 1 || !orbitals || (qorb && nq < 1) || !G || !A) return GFCC_ERR_ARG;
  if (nw == 0) return GFCC_OK;
  gfcc::StreamScope stream_scope(reinterpret_cast<cudaStream_t>(stream));
  try {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int> porb(orbitals, orbitals + np);
    std::vector<int> qv = qorb ? std::vector<int>(qorb, qorb + nq) : porb;
    nq = (int)qv.size();
    std::vector<int> qi = q_positions(porb, qv);
    const long long ng = (long long)nw * np * nq;
    DBuf<int> dq;
    DBuf<cplx> Gd;
    DBuf<double> Ad;
    dq.alloc(np);
    Gd.alloc(ng);
    Ad.alloc(nw);
    GFCC_CUDA(cudaMemcpyAsync(dq.p, qi.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    if (!adjoint) {
      GFCC_CUDA(cudaMemcpyAsync(Gd.p, G, sizeof(cplx) * ng, cudaMemcpyDefault, s));
      spectral_kernel<<<(nw + 127) / 128, 128, 0, s>>>(Gd.p, nw, np, nq, dq.p, Ad.p);
      GFCC_LAUNCH_CHECK();
      GFCC_CUDA(cudaMemcpyAsync(A, Ad.p, sizeof(double) * nw, cudaMemcpyDefault, s));
    } else {
      GFCC_CUDA(cudaMemcpyAsync(Ad.p, A, sizeof(double) * nw, cudaMemcpyDefault, s));
      spectral_adjoint_kernel<<<grid_for(ng), 256, 0, s>>>(Ad.p, nw, np, nq, dq.p, Gd.p);
      GFCC_LAUNCH_CHECK();
      GFCC_CUDA(cudaMemcpyAsync(const_cast<double*>(G), Gd.p, sizeof(cplx) * ng, cudaMemcpyDefault, s));
    }
    GFCC_CUDA(cudaStreamSynchronize(s));
  } catch (gfcc::Error& e) {
    fprintf(stderr, "gfcc_spectral: %s\n", e.msg.c_str());
    return e.code;
  }
  return GFCC_OK;
}

const char* gfcc_last_error(gfcc_t c) { return c ? c->last_error.c_str() : "null context"; }

void gfcc_free(gfcc_t c) {
  if (!c) return;
  gfcc::StreamScope stream_scope(c->stream);   // the context's buffers return to the pool in its stream's order
  delete c;
}

}  // extern "C"

gfcc_ctx::~gfcc_ctx() {
  gfcc::free_low_precision(this);
  gfcc::zgemm_work_free(this);
}

extern "C" {

}  // extern "C"
