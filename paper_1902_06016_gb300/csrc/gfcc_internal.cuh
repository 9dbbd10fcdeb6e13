// Internal declarations shared by the translation units of libgfcc (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuComplex.h>
#include <cstdint>
#include <cstdio>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/gfcc.h"

namespace gfcc {

// ---------------------------------------------------------------------------------------------
// error handling: every internal failure becomes a status code plus a message on the context
// ---------------------------------------------------------------------------------------------
struct Error {
  int code;
  std::string msg;
};

#define GFCC_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::gfcc::Error{GFCC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define GFCC_CHECK(cond, code, msg)                                                        \
  do {                                                                                     \
    if (!(cond)) throw ::gfcc::Error{(code), (msg)};                                       \
  } while (0)

// every kernel launch is followed by this check; it also counts the launches of the library
#define GFCC_LAUNCH_CHECK()                     \
  do {                                          \
    ::gfcc::count_launch();                     \
    GFCC_CUDA(cudaGetLastError());              \
  } while (0)

// launch counting and optional per-kernel-class timing (profile.cu)
void count_launch();
enum ProfClass {
  PROF_TC_GEMM = 0,      // tcgen05 GEMM, tf32/bf16-rounded operands
  PROF_F64_GEMM = 1,     // FP64 SIMT GEMM
  PROF_TC_SLICE = 2,     // tcgen05 GEMM on exact bf16 slices
  PROF_SIGMA_LP = 3,     // whole low-precision sigma (operand prep, GEMMs, combine)
  PROF_SIGMA_EX = 4,     // whole FP64-accurate sigma (exact slices or FP64 SIMT)
  PROF_KRYLOV = 5,       // Arnoldi: preconditioner, Gram-Schmidt, norms, Givens, corrections
  PROF_MOR_ORTHO = 6,    // subspace orthonormalisation and projections
  PROF_MOR_EVAL = 7,     // Hessenberg reduction and per-frequency reduced solves
  PROF_INIT = 8,         // H-bar build, b and c vectors
  PROF_MOR_PANEL = 9,    // column-by-column Gram-Schmidt inside the panels of a new block
  PROF_MOR_BASIS = 10,   // extension of the orthonormal residual basis Q
  PROF_TC_RING = 11,     // the ring-term GEMM of the low-precision sigma (tf32/bf16 tcgen05)
  PROF_OZ_ZGEMM = 12,    // whole FP64-accurate complex GEMMs on exact slices (operand gathers to scatter)
  PROF_OZ_SLICE = 13,    // splitting FP64 rows into exact bf16 slices (every use)
  PROF_KRYLOV_CGS = 14,  // the three fused Gram-Schmidt sweeps of an FP32-basis Arnoldi step (bytes)
  PROF_CGS_MULTIDOT = 15,     // first sweep alone (batches of >= 32 columns; bytes)
  PROF_CGS_UPDATE_DOT = 16,   // second sweep alone (batches of >= 32 columns; bytes)
  PROF_CGS_UPDATE_NORM = 17,  // third sweep alone (batches of >= 32 columns; bytes)
  PROF_CGS_SMALL_NB = 18,     // the three sweeps of batches of fewer than 32 columns (bytes)
  PROF_EVAL_HESS = 19,        // Householder reduction of Hhat to Hessenberg form (evaluation, guesses)
  PROF_EVAL_SOLVE = 20,       // per-frequency shifted Hessenberg solves
  PROF_ORTHO_GRAM = 21,       // block Gram-Schmidt coefficient products (basis^H block)
  PROF_ORTHO_UPDATE = 22,     // block Gram-Schmidt updates (block -= basis coefficients)
  PROF_ORTHO_CHOLQR = 23,     // Cholesky QR of the panels
  PROF_OZ_ACCUM = 24,         // accumulation of the exact-slice diagonals and the output pass (every use)
  PROF_LP_PREP = 25,          // operand preparation of the low-precision sigma (K-major operands)
  PROF_LP_COMBINE = 26,       // the combine pass of the low-precision sigma (up reduction, final sum)
  PROF_UPLOAD = 27,           // copies of the caller's inputs to the device in gfcc_init
  PROF_DOWNLOAD = 28,         // copies of results into the caller's output buffers
  PROF_ALLOC = 29,            // device allocations of the library's buffers (host time of each allocation)
  PROF_FREE = 30,             // device frees of the library's buffers (host time of each free)
  PROF_LP_SMALL_GEMMS = 31,   // the up, oooo and down GEMMs of the low-precision sigma (algorithmic bytes)
  PROF_NCLASS = 32
};
struct ProfScope {   // records CUDA events around one launch on stream s when profiling is on
  int cls;
  double flops;
  cudaStream_t s;
  void* rec = nullptr;
  ProfScope(int cls, double flops, cudaStream_t s);
  ~ProfScope();
};

// ---------------------------------------------------------------------------------------------
// device buffers owned by the context
// ---------------------------------------------------------------------------------------------
// host-side accounting of device allocations and frees while profiling is on (classes 29, 30)
bool alloc_profiling();
void note_alloc(int cls, double ms);

// Device memory (memory.cu): a stream-ordered pool per device that keeps its reserve. Allocations
// and frees are ordered on the stream of the innermost StreamScope of the calling thread (each
// entry point opens one with its context's stream); device_free_bytes() is the device's free memory
// plus the pool's unused reserve.
cudaStream_t current_alloc_stream();
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s);
  ~StreamScope();
  StreamScope(const StreamScope&) = delete;
  StreamScope& operator=(const StreamScope&) = delete;
};
cudaError_t pool_alloc(void** p, size_t bytes);
void pool_free(void* p);
size_t device_free_bytes();

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; n = o.n;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) {
      if (alloc_profiling()) {
        const auto t0 = std::chrono::steady_clock::now();
        pool_free(p);
        note_alloc(PROF_FREE, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
      } else {
        pool_free(p);
      }
    }
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e;
    void* q = nullptr;
    if (alloc_profiling()) {
      const auto t0 = std::chrono::steady_clock::now();
      e = pool_alloc(&q, count * sizeof(T));
      note_alloc(PROF_ALLOC, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    } else {
      e = pool_alloc(&q, count * sizeof(T));
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      throw Error{GFCC_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed"};
    }
    p = static_cast<T*>(q);
    n = count;
  }
  void zero(cudaStream_t s) {
    if (p && n) GFCC_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
};

using cplx = cuDoubleComplex;

// ---------------------------------------------------------------------------------------------
// The similarity-transformed Hamiltonian on the 1h+2h1p space, laid out for the sigma GEMMs.
// Index conventions: o occupied, v virtual, P = o(o-1)/2 pairs i<j, pair(i,j) = j(j-1)/2 + i,
// packed vector index: 1h i -> i, 2h1p (i<j,a) -> o + pair(i,j)*v + a.
// ---------------------------------------------------------------------------------------------
struct Operator {
  DBuf<double> Wr;     // [(a,i)][(m,e)]  ov x ov : W_maei - d_ae F_mi(off) + 1/2 d_mi F_ae(off)
  DBuf<double> Woo;    // [pair(ij)][pair(mn)]  P x P : W_mnij
  DBuf<double> A11;    // [i][m]  o x o : -F_mi (off-diagonal)
  DBuf<double> A12;    // [i][(pair(mn),e)]  o x Pv : 1h <- 2h1p block
  DBuf<double> A21;    // [(pair(ij),a)][m]  Pv x o : 2h1p <- 1h block (-W_maij)
  DBuf<double> Vt;     // [e][(pair(mn),f)]  v x Pv : <mn||ef>   (three-body, first half)
  DBuf<double> T2p;    // [(pair(ij),a)][e]  Pv x v : t_ij^ae     (three-body, second half)
  DBuf<double> diag;   // [D] Fock-diagonal part: -F_ii (1h), F_aa - F_ii - F_jj (2h1p)
  DBuf<double> mdiag;  // [D] full diagonal of M (Jacobi preconditioner)
  // transposed-action copies are built lazily (adjoint systems)
  bool have_T = false;
  DBuf<double> WrT, WooT, A12T, A21T, VtT, T2pT;
  // explicitly transposed blocks for the tensor-core operands of M^T (built lazily): the roles of the
  // forward blocks in M^T, stored in the forward layouts: WooX = Woo^T [P][P], VtX = T2p^T [v][Pv],
  // A12X = A21^T [o][Pv], T2pX = Vt^T [Pv][v], A21X = A12^T [Pv][o], A11X = A11^T [o][o]
  bool have_X = false;
  DBuf<double> WooX, VtX, A12X, T2pX, A21X, A11X;
};

// low-precision (tensor-core) copies of the sigma operands; the state lives in sigma_tc.cu
struct LowPrecision {
  int kind = 0;          // GFCC_PREC_* of the built operands (0: none)
  void* impl = nullptr;
  void* emu = nullptr;   // exact-slice (FP64-accurate) operands
  void* implT = nullptr; // the same for the transposed action M^T (adjoint systems), built on first use
  void* emuT = nullptr;
};

struct Workspace {
  DBuf<double> ut;      // unpacked 2h1p  [(m,e)][(j,c)] complex -> 2*ov*o*nb doubles
  DBuf<double> ct;      // ring product   [(a,i)][(j,c)] complex
  DBuf<double> xe;      // three-body X_e [e][c] complex
  size_t nb_cap = 0;
};

struct MorState {
  bool built = false;
  int kind = 0;                    // subspace: 0 solutions at sampled frequencies, 1 block Krylov space of M on B
  int kblocks = 0;                 // (kind 1) Krylov blocks in the subspace
  int knext = 0;                   // (kind 1) columns of the newest block, whose M-images start the next one
  double eta = 0.0;
  std::vector<int> porb, qorb;     // orbital sets
  std::vector<double> sampled;     // sampled frequencies (sorted)
  int m = 0, m_cap = 0;            // model order and capacity
  DBuf<cplx> S, Z;                 // [D][m_cap] batch-minor: column i of S at S[nu*m_cap + i]; Z = M S
  DBuf<cplx> Hh;                   // [m_cap x m_cap] col-major  Hhat = S^H Z
  DBuf<cplx> bh;                   // [m_cap x np]    col-major  S^H B
  DBuf<cplx> ch;                   // [nq x m_cap]    col-major  C S  (ld nq)
  // orthonormal basis Q of span[B, S, Z] and the coefficients of B, S, Z in it, for residual norms
  // ||(w - i eta) S y + Z y - b_p|| = ||(w - i eta) RS y + RZ y - RB e_p|| without cancellation
  int qn = 0, q_cap = 0;
  DBuf<cplx> Q;                    // [D][q_cap] batch-minor
  DBuf<cplx> RS, RZ;               // [q_cap x m_cap] col-major (ld q_cap)
  DBuf<cplx> RB;                   // [q_cap x np]    col-major (ld q_cap)
  std::vector<double> bnorm;       // ||b_p||
  // exact dG/dw [np x nq] at the sampled frequencies (only with opts.deriv_indicator)
  std::vector<std::pair<double, std::vector<cplx>>> dG_exact;
  std::vector<std::pair<int, double>> history;
  long long solve_iters = 0, solve_cols = 0;   // Arnoldi steps (summed over batches) and columns solved
  // Hessenberg form of the current model (mor.cu: hessenberg()), valid while hess_version == version:
  // H = P^H Hhat P, P^H bhat, chat P, RS P, RZ P, RB, and the reflectors (column j of hV, tau in htau)
  long long version = 0, hess_version = -1;
  bool hess_res = false;
  int hess_qn = 0;
  DBuf<cplx> hH, hb, hc, hA1, hA2, hRB, hV;
  DBuf<double> htau;
  double last_max_err = -1.0;
  void reset() {
    built = false;
    kind = 0;
    kblocks = 0;
    knext = 0;
    eta = 0.0;
    porb.clear(); qorb.clear(); sampled.clear(); bnorm.clear(); history.clear(); dG_exact.clear();
    solve_iters = 0; solve_cols = 0;
    ++version;
    hess_version = -1;
    for (DBuf<cplx>* b : {&hH, &hb, &hc, &hA1, &hA2, &hRB, &hV}) b->release();
    htau.release();
    m = 0; m_cap = 0; qn = 0; q_cap = 0;
    for (DBuf<cplx>* b : {&S, &Z, &Hh, &bh, &ch, &Q, &RS, &RZ, &RB}) b->release();
    last_max_err = -1.0;
  }
};

struct Stats {
  long long sigma_calls = 0, sigma_cols = 0, gmres_iters = 0, restarts = 0;
  double max_rel_res = 0.0;
  int not_converged = 0;
};

}  // namespace gfcc

struct gfcc_ctx {
  // o, v, P, D: the block sizes of the operator. IP space: o occupied, v virtual, P = o(o-1)/2 pairs.
  // EA space (sector 1): the same layout with the roles exchanged, o = the virtual count (the pair
  // index), v = the occupied count, P = v(v-1)/2 virtual pairs. n = o + v either way.
  int o = 0, v = 0, n = 0, P = 0, D = 0;
  int sector = 0;   // 0: ionisation (IP), 1: electron attachment (EA)
  cudaStream_t stream = nullptr;
  int device = 0;
  gfcc_opts opts{};
  std::string last_error;
  gfcc::Operator op;
  gfcc::LowPrecision lp;
  gfcc::Workspace ws;
  gfcc::MorState mor;                 // the reduced model (MIMO, Eq. model), or the model being worked on
  std::vector<gfcc::MorState> siso;   // per-orbital (SISO) reduced models of G_pp (gfcc_mor_build_siso)
  long long siso_iters = 0, siso_cols = 0;   // Arnoldi steps and columns of the SISO models' solves
  gfcc::Stats stats;
  gfcc::DBuf<double> bvec;   // [n][D]  b_p rows
  gfcc::DBuf<double> cvec;   // [n][D]  c_q rows
  gfcc::DBuf<double> t1, t2; // kept for derivative work
  // kept for the T2 gradient: <mn||ef>, <mn||ie>, <ma||ef>, lambda2, F_me (row-major as the inputs)
  gfcc::DBuf<double> k_oovv, k_ooov, k_ovvv, k_l2, k_Fme;
  void* zwork = nullptr;     // grow-only workspace of the exact-slice complex GEMMs (ozaki.cu)
  ~gfcc_ctx();
};

namespace gfcc {

// ---- gemm.cu -----------------------------------------------------------------------------------
// C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n), with element strides and batch strides
// (blockIdx.z). Real FP64 SIMT kernel; complex data whose re/im pairs lie along N is handled by
// passing N' = 2N with unit n-stride.
struct GemmDesc {
  int M = 0, N = 0, K = 0, batch = 1;
  const double* A = nullptr; long long sam = 0, sak = 0, bsa = 0;
  const double* B = nullptr; long long sbk = 0, sbn = 0, bsb = 0;
  double* C = nullptr; long long scm = 0, scn = 0, bsc = 0;
  double alpha = 1.0, beta = 0.0;
};
void dgemm(const GemmDesc& g, cudaStream_t s);

// complex FP64 GEMM, op(A) may be conjugated; strides in complex elements
struct ZGemmDesc {
  int M = 0, N = 0, K = 0, batch = 1;
  const cplx* A = nullptr; long long sam = 0, sak = 0, bsa = 0; bool conjA = false;
  const cplx* B = nullptr; long long sbk = 0, sbn = 0, bsb = 0; bool conjB = false;
  cplx* C = nullptr; long long scm = 0, scn = 0, bsc = 0;
  cplx alpha = {1.0, 0.0}, beta = {0.0, 0.0};
  void* work = nullptr;   // optional grow-only workspace (zgemm_work(ctx)) for the exact-slice path
  // optional cache of the exact slices of A (zgemm_slice_cache(ctx, i)): sliced on the first call after
  // zgemm_slice_cache_reset and reused by later calls until the next reset (A's data must not change)
  void* a_cache = nullptr;
};
void zgemm(const ZGemmDesc& g, cudaStream_t s);
// the context's workspace for exact-slice complex GEMMs (created on first use, freed with the context)
void* zgemm_work(gfcc_ctx* c);
void zgemm_work_free(gfcc_ctx* c);
// throws GFCC_ERR_CUDA if a tensor-core wait of a GEMM that used the context's workspace timed out
void zgemm_work_check(gfcc_ctx* c);
// slice cache i (0 or 1) of the context's workspace, and its invalidation
void* zgemm_slice_cache(gfcc_ctx* c, int i);
void zgemm_slice_cache_reset(void* cache);

// ---- grad.cu: T2 gradient of L = Re sum conj(Gbar) G ------------------------------------------
// W[nu][w np + p] = sum_q conj(Gbar[w][p][q]) c_q[nu]   (right sides of the adjoint solves)
void green_adjoint_rhs(gfcc_ctx* c, const std::vector<int>& qorb, const cplx* Gbar_dev, long long S, cplx* W);
// from the forward solutions X and adjoint solutions U ([D][nw np] batch-minor): t2bar[o][o][v][v]
void green_grad_t2_core(gfcc_ctx* c, int nw, const std::vector<int>& porb, const std::vector<int>& qorb,
                        const cplx* Gbar_dev, const cplx* X, const cplx* U, double* t2bar_dev);

// row-major contiguous helpers
void dgemm_rm(int M, int N, int K, double alpha, const double* A, int lda, bool transA,
              const double* B, int ldb, bool transB, double beta, double* C, int ldc, cudaStream_t s);

// ---- tensor.cu ---------------------------------------------------------------------------------
// dst = alpha * permute(src) + beta * dst for up to 6-D tensors (row-major);
// dst index order is src axes perm[0], perm[1], ...
void permute(const double* src, const int* dims, int nd, const int* perm, double* dst,
             double alpha, double beta, cudaStream_t s);
void axpby(long long n, double alpha, const double* x, double beta, double* y, cudaStream_t s);

// ---- hbar.cu -----------------------------------------------------------------------------------
// Copy kind for a copy from src (host or device memory) into device memory. An explicit kind: on this
// GPU's driver, cudaMemcpyDefault from page-locked host memory into freshly allocated device memory ran
// at 25-37 GB/s, the explicit host-to-device kind at 208 GB/s.
inline cudaMemcpyKind kind_to_device(const void* src) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, src) != cudaSuccess) {
    cudaGetLastError();
    return cudaMemcpyHostToDevice;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? cudaMemcpyDeviceToDevice
                                                                              : cudaMemcpyHostToDevice;
}

struct HostInputs {
  const double *eps, *oooo, *ooov, *oovv, *ovov, *ovvv, *t1, *t2, *l1, *l2;
  const double* vvvv = nullptr;   // packed [pair(a,b)][pair(c,d)] <ab||cd> (EA space only)
};
void build_operator(gfcc_ctx* c, const HostInputs& in);
// hbar_ea.cu: the EA (1p + 2p1h) operator in the block layout of the IP one (see gfcc_init_ea)
void build_operator_ea(gfcc_ctx* c, const HostInputs& in);

// ---- sigma.cu ----------------------------------------------------------------------------------
// Y = M X (+ shift*X per column) on a batch in batch-minor layout X[nu][c] (complex), c < nb,
// leading dimension ldb (complex elements per row). shift may be null.
void sigma_batch(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, int ldb, const cplx* shift,
                 int precision, bool transpose, cudaStream_t s);
void ensure_workspace(gfcc_ctx* c, int nb);
void build_transpose_operator(gfcc_ctx* c);

// ---- sigma_tc.cu (tcgen05 low-precision sigma for the inner solves) ---------------------------
void build_low_precision(gfcc_ctx* c, int kind);
void free_low_precision(gfcc_ctx* c);
// free the per-batch buffers of the tensor-core sigma states (reallocated on demand)
void release_sigma_batch_buffers(gfcc_ctx* c);
// free every grow-only scratch buffer of the context (sigma batch buffers, the FP64 sigma workspace, the
// exact-slice complex GEMM workspace) after checking the workspace's error flag; used when device memory
// runs short for the reduced model's own buffers
void release_scratch(gfcc_ctx* c);
void sigma_lowprec(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, const cplx* shift, cudaStream_t s,
                   bool transpose = false);
// the same with FP32 complex vectors (the FP32 Krylov basis of the mixed-precision solver)
void sigma_lowprec_f32(gfcc_ctx* c, const cuFloatComplex* X, cuFloatComplex* Y, int nb, const cplx* shift,
                       cudaStream_t s, bool transpose = false);
int low_precision_error(gfcc_ctx* c);   // 1 if a tensor-core pipeline wait timed out
int emulated_error(gfcc_ctx* c);
void build_emulated(gfcc_ctx* c);
void sigma_emulated(gfcc_ctx* c, const cplx* X, cplx* Y, int nb, const cplx* shift, cudaStream_t s,
                    bool transpose = false);
void tc_selftest(int kind, const double* A, const double* B, int M, int N, int K, float* C, cudaStream_t s);

// ---- krylov.cu ---------------------------------------------------------------------------------
struct SolveStatus {
  std::vector<double> relres;   // per column
  std::vector<int> iters;       // per column
  std::vector<int> converged;   // per column
};
// Solve (shift_c + M) x_c = b_c for nb columns (batch-minor layout, ld = nb), starting from X0 (same
// layout) when it is non-null, else from zero.
void gmres_batched(gfcc_ctx* c, const cplx* B, cplx* X, cplx* R, const cplx* shifts, int nb,
                   SolveStatus& st, bool transpose, const cplx* X0 = nullptr);

// ---- kernels shared between units ------------------------------------------------------------
void gather_rows_real_to_cplx(const double* src, int ld_src, const int* rows, int nrows, int D,
                              cplx* dst, int ldb, cudaStream_t s);   // dst[nu][k] = src[rows[k]][nu]
void pack_cols_to_batch(const cplx* src, int ld_src, int ncols, int D, cplx* dst, int ldb,
                        cudaStream_t s);   // dst[nu][c] = src[c][nu]
void batch_to_cols(const cplx* src, int ldb, int ncols, int D, cplx* dst, int ld_dst,
                   cudaStream_t s);        // dst[c][nu] = src[nu][c]
void green_from_batch(const double* cvec, int D, const int* qrows, int nq, const cplx* X, int ldb,
                      int ncols, cplx* G, cudaStream_t s);   // G[c][q] = sum_nu c_q[nu] X[nu][c]

// mor.cu
void mor_init_basis(gfcc_ctx* c);   // Q <- orth(B), after porb/qorb/eta are set
void mor_append(gfcc_ctx* c, const cplx* X, const cplx* MX, int ncols);
// x0_p(w) = S yhat_p(w) from the current reduced model, X0 [D][nw np] (device)
void mor_extrapolate(gfcc_ctx* c, const double* omegas, int nw, cplx* X0);
// Ghat, A and residual estimates at the frequencies omegas (host); dG_dev (optional): dGhat/dw
void mor_eval(gfcc_ctx* c, const double* omegas, int nw, cplx* G_dev, double* A_dev,
              double* maxres_dev, cplx* dG_dev = nullptr);

}  // namespace gfcc
