/*
 * gfcc.h - C ABI of libgfcc: IP Green's-function coupled cluster (GFCCSD) linear systems and their
 * model-order reduction on one GB300 GPU.
 *
 * Method (Peng, Van Beeumen, Williams-Young, Kowalski, Yang, "Approximate Green's function coupled
 * cluster method employing effective dimension reduction", arXiv 1902.06016):
 *   Eq. xp      X_p(w) = sum_i x^i a_i + sum_{i<j,a} x^{ij}_a a_a^+ a_j a_i   (1h + 2h1p space)
 *   Eq. xplin   (w + Hbar_N - i eta) X_p(w)|Phi> = abar_p |Phi>
 *   Eq. gfxn2   G_pq(w) = <Phi|(1 + Lambda) abar_q^+ X_p(w)|Phi> = c_q^T X_p(w)
 *   Eq. gfcclineqn / model   MIMO system, Galerkin reduced model Hhat = S^H Hbar S, bhat = S^H b,
 *                            chat^T = c^T S over an orthonormal subspace S of solved X_p(w_k)
 *   MOR text after Eq. model: adaptive refinement by midpoints of adjacent sampled frequencies.
 *   A(w) = -(1/pi) sum_p Im G_pp(w)   (spectral function, returned exactly as written).
 *
 * Conventions (all entry points):
 *   - Status: 0 = success, negative = error (GFCC_ERR_*); gfcc_last_error() gives the message.
 *   - Indices: o occupied and v virtual spin-orbitals, n = o + v, occupied first. P = o(o-1)/2.
 *     Vector dimension D = o + P*v. Packed vector index: i for x^i; o + pair(i,j)*v + a for
 *     x^{ij}_a with i < j and pair(i,j) = j(j-1)/2 + i.
 *   - Complex numbers are interleaved (re, im) doubles. A block of nvec vectors is column-major:
 *     vector c starts at element c*ld (complex units), ld >= D.
 *   - Pointer arguments marked "host or device" may point to host memory or to device memory on
 *     the context's GPU; the kind is detected with cudaPointerGetAttributes. Host buffers are
 *     copied synchronously; device buffers are used in place on the context's stream.
 *   - All inputs are copied (the caller keeps ownership); all outputs are caller-allocated.
 *   - Calls on one context are not thread-safe; distinct contexts are independent.
 */
#ifndef GFCC_H
#define GFCC_H

#ifdef __cplusplus
extern "C" {
#endif

#define GFCC_OK 0
#define GFCC_ERR_ARG (-1)            /* invalid argument (sizes, null pointers, ranges) */
#define GFCC_ERR_NOT_CONVERGED (-2)  /* iteration cap reached before the tolerance */
#define GFCC_ERR_RANK (-3)           /* subspace became rank deficient / empty */
#define GFCC_ERR_NONFINITE (-4)      /* NaN or Inf in inputs or iterates */
#define GFCC_ERR_OOM (-5)            /* device allocation failed */
#define GFCC_ERR_CUDA (-6)           /* CUDA runtime error */
#define GFCC_ERR_STATE (-7)          /* call out of order (e.g. mor_eval before mor_build) */

/* arithmetic of the H-bar sigma contractions */
#define GFCC_PREC_FP64 0        /* FP64 everywhere */
#define GFCC_PREC_TF32 1        /* every sigma GEMM on tcgen05 kind::tf32, FP32 accumulate; FP64 diagonal */
#define GFCC_PREC_BF16 2        /* every sigma GEMM on tcgen05 kind::f16 with bf16 operands, FP32 accumulate */
#define GFCC_PREC_FP64_TC 3     /* FP64-accurate: exact integer bf16 slices of the FP64 operands on tcgen05,
                                   exact FP32 partial sums recombined in FP64 (Ozaki scheme) */

typedef struct gfcc_ctx* gfcc_t;

/* Antisymmetrised two-electron integral blocks <pq||rs>, real, row-major, occupied index range
 * first: oooo[i][j][k][l], ooov[i][j][k][a], oovv[i][j][a][b], ovov[i][a][j][b], ovvv[i][a][b][c].
 * Host or device pointers. (No vvvv block is needed by the IP space.) */
typedef struct {
  const double* oooo;
  const double* ooov;
  const double* oovv;
  const double* ovov;
  const double* ovvv;
} gfcc_vblocks;

typedef struct {
  double tol;          /* relative residual ||b - A x|| / ||b|| at which a column is converged (1e-8) */
  int restart;         /* Krylov dimension per restart cycle (GMRES(k)); default 30 */
  int max_restarts;    /* cycle cap per column; default 200 */
  int precision;       /* GFCC_PREC_* of the inner (Krylov) sigma; residuals are always FP64. With
                          TF32/BF16 the Krylov basis is FP32, with FP64/FP64_TC it is FP64. */
  int max_batch;       /* max columns (p, w) per batched solve; 0 = choose from memory */
  double drop_tol;     /* subspace rank-truncation threshold (relative), default 1e-10 */
  int verbose;         /* 0 silent, 1 per-call summary on stderr */
  int residual_precision; /* sigma of the refinement residuals: GFCC_PREC_FP64 (FP64 CUDA cores) or
                             GFCC_PREC_FP64_TC; -1 (default) = FP64_TC when precision is a tensor-core
                             kind, FP64 otherwise */
  int deriv_indicator;  /* 1: the refinement also compares dG/dw of the reduced model with the exact
                           dG/dw = -c^T A^{-1} x at every sampled frequency (one more solve per column
                           at each new sample); default 0 */
  int mor_guess;        /* 1 (default): solves at frequencies added by gfcc_mor_refine start from the
                           current reduced model's prediction x0_p(w) = S yhat_p(w); 0: from zero.
                           The solutions agree to the solver tolerance either way. */
} gfcc_opts;

typedef struct {
  long long sigma_calls;   /* batched sigma launches */
  long long sigma_cols;    /* complex columns processed by sigma */
  long long gmres_iters;   /* Arnoldi steps summed over batches */
  long long restarts;      /* restart (iterative-refinement) cycles summed over batches */
  double max_rel_res;      /* largest final relative residual over the columns of the call */
  int not_converged;       /* columns that hit the cycle cap */
} gfcc_stats;

/* Fill *opts with the defaults listed above. */
int gfcc_default_opts(gfcc_opts* opts);

/* Create a context on the current CUDA device: copy the ground-state inputs and build the H-bar
 * elements of the IP space on the GPU (Hbar_N = e^{-T} H e^{T} - E_0, text after Eq. gfxn1),
 * the free terms b_p (Eq. xplin) and the left vectors c_q (Eq. gfxn2) for all n orbitals.
 *   eps[n]      orbital energies (the reference Fock matrix is diag(eps)).
 *   vb          integral blocks.
 *   t1[o][v], t2[o][o][v][v] (t_ij^ab, antisymmetric), l1[o][v] (lambda^i_a), l2[o][o][v][v]
 *               (lambda^ij_ab).
 *   All arrays: host or device (copied to the device with the copy kind of their memory).
 *   opts        may be NULL (defaults).  stream: cudaStream_t or NULL for the legacy stream.
 * Errors: GFCC_ERR_ARG (o < 2, v < 1, null pointers), GFCC_ERR_NONFINITE, GFCC_ERR_OOM, GFCC_ERR_CUDA. */
int gfcc_init(gfcc_t* ctx, int o, int v, const double* eps, const gfcc_vblocks* vb,
              const double* t1, const double* t2, const double* l1, const double* l2,
              const gfcc_opts* opts, void* stream);

/* Create a context for the electron-attachment (EA) half of the Green's function instead: the second
 * term <Psi| a_p (w - (H - E_0) + i eta)^{-1} a_q^+ |Psi> of the retarded Green's function of Eq. gfxn0,
 * which the paper names beside the IP term (IP/EA-EOM-CC, Introduction) but does not write out. In the
 * CC form (Eqs. gfxn1/gfxn2 with the field operators exchanged):
 *   G^EA_pq(w) = <Phi|(1 + Lambda) abar_p (w - Hbar_N + i eta)^{-1} abar_q^+ |Phi> = c_p^T y_q(w),
 *   (w + i eta - M_EA) y_q(w) = b_q,  b_q = e^{-T} a_q^+ e^{T}|Phi>,  c_p = <Phi|(1+Lambda) e^{-T} a_p e^{T}
 * over the 1p + 2p1h space y = sum_a y^a a_a^+ + sum_{a<b,j} y^{ab}_j a_a^+ a_b^+ a_j.
 *   Arguments as gfcc_init (o >= 1, v >= 2), plus
 *   vvvv[V][V]  the virtual block <ab||cd> in packed pair form, V = v(v-1)/2, row pair(a,b) and column
 *               pair(c,d) = d(d-1)/2 + c for a < b, c < d (virtual indices from 0). Host or device; copied.
 * The space has dimension D = v + V*o; packed vector index a for y^a, v + pair(a,b)*o + j for y^{ab}_j.
 * Every other entry point then works on the EA systems, with these conventions:
 *   - frequencies (omegas, seeds, [wmin, wmax], the sampled frequencies reported by gfcc_mor_info and
 *     gfcc_mor_model_info) are the physical w of the formula above; internally the systems are solved in
 *     the IP form (w' - i eta + M_EA) y = -b_q at w' = -w, so refinement ties go to the higher w, and
 *     saved models carry their own tag (a model of one space does not load into the other);
 *   - the orbital set named "p set" / orbitals is the set of free terms b_q (the solved columns) and the
 *     "q set" / qorb the set of left vectors c_p: G[(w*np + k)*nq + l] = G^EA_{qorb[l], orbitals[k]}(w);
 *   - gfcc_vectors returns b_q (transpose = 0) and c_p (transpose = 1); gfcc_sigma applies M_EA;
 *   - A(w) = -(1/pi) sum_p Im G_pp(w) as for the IP space (positive peaks, since the attachment
 *     broadening is + i eta);
 *   - gfcc_green_derivatives returns dG^EA/dw and dG^EA/deta; gfcc_green_grad_t2 returns GFCC_ERR_STATE.
 * Errors: as gfcc_init; GFCC_ERR_ARG also for a null vvvv. */
int gfcc_init_ea(gfcc_t* ctx, int o, int v, const double* eps, const gfcc_vblocks* vb, const double* vvvv,
                 const double* t1, const double* t2, const double* l1, const double* l2, const gfcc_opts* opts,
                 void* stream);

/* The space of a context: *sector = 0 (IP, gfcc_init) or 1 (EA, gfcc_init_ea). */
int gfcc_sector(gfcc_t ctx, int* sector);

/* Dimension D of the context's space (1h+2h1p, or 1p+2p1h for an EA context). */
int gfcc_dim(gfcc_t ctx, int* D);

/* Replace the options (tolerance, restart length, precision, ...) of an existing context. */
int gfcc_set_opts(gfcc_t ctx, const gfcc_opts* opts);

/* Y = M X (transpose = 0) or Y = M^T X (transpose = 1) for nvec complex vectors, where M is the
 * matrix of Hbar_N on the 1h+2h1p space (Eq. xplin). X, Y: host or device, column-major with
 * leading dimension ld (complex units). precision: GFCC_PREC_*. */
int gfcc_sigma(gfcc_t ctx, const double* X, double* Y, int nvec, int ld, int precision,
               int transpose);

/* b_p (transpose = 0) or c_q (transpose = 1) rows for the given orbitals: out[k*ld + nu], real,
 * host or device. Eqs. xplin and gfxn2. */
int gfcc_vectors(gfcc_t ctx, const int* orbitals, int norb, int transpose, double* out, int ld);

/* Full-dimension solves of Eq. xplin for every (w, p): (w - i eta + M) X_p(w) = b_p, by batched
 * restarted GMRES with iterative refinement (FP64 residuals, inner sigma in opts.precision).
 *   omegas[nw] (host), orbitals[np] (host, p set), qorb[nq] (host, q set; NULL = same as p set).
 *   G  (optional, host or device): G[(w*np + p)*nq + q] complex = c_q^T X_p(w).
 *   A  (optional, host or device): A[w] = -(1/pi) sum_{p in set, p also in q set} Im G_pp(w).
 *   X  (optional, host or device): X[(w*np + p)*ldx ...] complex solutions, ldx >= D.
 *   stats (optional, host).
 * Returns GFCC_ERR_NOT_CONVERGED (outputs still written) if a column hit the cycle cap. */
int gfcc_solve_full(gfcc_t ctx, const double* omegas, int nw, double eta, const int* orbitals,
                    int np, const int* qorb, int nq, double* G, double* A, double* X, int ldx,
                    gfcc_stats* stats);

/* Spectral function A(w) = -(1/pi) sum_p Im G_pp(w) (the definition after Eq. gfxn0, returned as
 * written) from G [nw][np][nq] complex laid out as in gfcc_solve_full: the sum runs over the orbitals p
 * of the p set that also appear in the q set (qorb NULL: the same set, nq ignored).
 *   adjoint = 0: reads G, writes A[nw].
 *   adjoint = 1: the adjoint map (the vector-Jacobian product of a backward pass): reads A as the
 *                upstream gradient Abar[nw] and writes G[w][p][q] = -(i/pi) Abar[w] where q is the
 *                position of p in the q set, 0 elsewhere.
 * G and A: host or device (copied with cudaMemcpyDefault); stream: cudaStream_t or NULL. The call
 * returns when the result has been written. No context is needed.
 * Errors: GFCC_ERR_ARG (null pointers, empty orbital sets), GFCC_ERR_OOM, GFCC_ERR_CUDA. */
int gfcc_spectral(const double* G, int nw, const int* orbitals, int np, const int* qorb, int nq, double* A,
                  int adjoint, void* stream);

/* Derivatives of G_pq(w) (Eq. gfcclineqn) with respect to the frequency and the broadening. With
 * A(w) = w - i eta + M, x_p = A^{-1} b_p (forward solves, as gfcc_solve_full) and the adjoint solutions
 * y_q = A^{-T} c_q (transposed sigma), G_pq = c_q^T x_p, dG_pq/dw = -y_q^T x_p and dG_pq/deta = i y_q^T x_p.
 * Outputs (each optional, host or device, complex, layout [(w*np + p)*nq + q] as in gfcc_solve_full).
 * The adjoint solves use the transposed sigma in the context's precision (with a TF32/BF16 context, GMRES-IR
 * with the low-precision M^T inside and exact-slice FP64-accurate residuals, like the forward solves).
 * GFCC_ERR_NOT_CONVERGED if a solve hit the cap. */
int gfcc_green_derivatives(gfcc_t ctx, const double* omegas, int nw, double eta, const int* orbitals, int np,
                           const int* qorb, int nq, double* G, double* dG_domega, double* dG_deta);

/* Gradient of L = Re sum_{w,p,q} conj(Gbar[w][p][q]) G_pq(w) with respect to the doubles amplitudes
 * t2[i][j][a][b] (the vector-Jacobian product of an autograd backward pass; G_pq(w) = c_q^T A(w)^{-1} b_p
 * as in Eq. gfcclineqn, with M, b_p and c_q built from T by the H-bar expressions of the text after
 * Eq. gfxn1 and Eqs. xplin, gfxn2). Adjoint method: forward solves x, adjoint solves
 * u = A^{-T} sum_q conj(Gbar) c_q with the transposed sigma, the sigma bilinear form in u and x, then back
 * through the H-bar build; the forward solutions are recomputed here. Lambda and T1 are held fixed.
 *   omegas[nw], orbitals[np], qorb[nq] (NULL = p set) as in gfcc_solve_full.
 *   Gbar (host or device): complex [nw][np][nq] weights.
 *   G (optional, host or device): the forward G, layout as in gfcc_solve_full.
 *   grad_t2 (host or device): [o][o][v][v] real, dL/dt2 with every array element treated as independent
 *   (for antisymmetric amplitudes the derivative along t_ij^ab, i<j, a<b, is
 *   g[i][j][a][b] - g[j][i][a][b] - g[i][j][b][a] + g[j][i][b][a]).
 * Errors: GFCC_ERR_ARG, GFCC_ERR_NOT_CONVERGED (a forward or adjoint solve hit the cap), GFCC_ERR_CUDA. */
int gfcc_green_grad_t2(gfcc_t ctx, const double* omegas, int nw, double eta, const int* orbitals, int np,
                       const int* qorb, int nq, const double* Gbar, double* G, double* grad_t2);

/* Start a reduced model (Eq. model): solve Eq. xplin at the seed frequencies for every p in
 * orbitals (host), orthonormalise the solutions into S (columns whose norm after two
 * Gram-Schmidt passes falls below opts.drop_tol of their norm before are dropped), and project:
 * Hhat = S^H M S, bhat = S^H b, chat = c^T S. qorb/nq as in gfcc_solve_full. */
int gfcc_mor_build(gfcc_t ctx, const double* seeds, int ns, double eta, const int* orbitals,
                   int np, const int* qorb, int nq);

/* Per-orbital (single-input single-output) reduced models of the diagonal elements G_pp, the variant
 * the paper's conclusion proposes (separate models for the diagonal elements): for each orbital p of
 * orbitals (host, np distinct entries) a model as in gfcc_mor_build with the single orbital p as both
 * p and q set, its subspace spanned by X_p(w_k) alone. All models start from the same seeds; their
 * seed solutions run as one batched solve. gfcc_mor_refine then refines every model on its own
 * frequencies (all models' new solutions again in one batched solve per round; m_max bounds each
 * model's order; the derivative indicator is not available), gfcc_mor_eval writes Ghat_pp on the
 * diagonal of G [nw][np][np] (zeros elsewhere), A from those diagonals and maxres as the max over the
 * models; gfcc_mor_info reports the union of the sampled frequencies and the total order, and
 * gfcc_mor_model_info each model. gfcc_mor_build replaces such a set by one MIMO model; sets are not
 * saved by gfcc_mor_save (GFCC_ERR_STATE).
 * Errors: GFCC_ERR_ARG (bad seeds, eta, orbitals), GFCC_ERR_RANK (all seed solutions of an orbital
 * dropped), GFCC_ERR_NOT_CONVERGED, GFCC_ERR_CUDA. */
int gfcc_mor_build_siso(gfcc_t ctx, const double* seeds, int ns, double eta, const int* orbitals, int np);

/* Reduced model on a block Krylov subspace instead of solutions at sampled frequencies (multi-shift
 * reuse; not in the paper, next to its Eq. model): S = orth[B, M B, ..., M^(k-1) B] for B = [b_p], k =
 * nblocks, each block orthonormalised against the previous ones as in gfcc_mor_build (columns that fall
 * below opts.drop_tol are dropped, and the next block starts from M applied to the kept ones), with
 * M X from the FP64-accurate sigma (opts.residual_precision). The Krylov space of M is that of every
 * shifted matrix w - i eta + M, so the Galerkin model Hhat = S^H M S, bhat, chat gives the block FOM
 * solution of Eq. xplin at every frequency from one subspace. gfcc_mor_refine on such a model adds
 * max(1, floor(k/4)) blocks per round until the largest residual estimate over all its grid points is
 * <= tol (m_max bounds the order; no derivative indicator); gfcc_mor_eval, gfcc_mor_info (no sampled
 * frequencies) and gfcc_mor_model_info work as for gfcc_mor_build; gfcc_mor_save returns
 * GFCC_ERR_STATE. orbitals / qorb as in gfcc_mor_build.
 * Errors: GFCC_ERR_ARG, GFCC_ERR_RANK (empty subspace), GFCC_ERR_CUDA. */
int gfcc_mor_build_krylov(gfcc_t ctx, int nblocks, double eta, const int* orbitals, int np, const int* qorb, int nq);

/* Model k of the current set (a per-orbital set: k < np; a MIMO model: k = 0): its orbital (-1 for a
 * MIMO model), up to cap sampled frequencies (host), their count and the model order. Any output
 * pointer may be NULL. GFCC_ERR_ARG if there is no model k. */
int gfcc_mor_model_info(gfcc_t ctx, int k, int* orbital, double* w, int cap, int* ns, int* m);

/* Adaptive refinement (MOR text after Eq. model): on a uniform grid of ngrid points over
 * [wmin, wmax], estimate for each interval between adjacent sampled frequencies the largest relative
 * residual ||(w - i eta + M) S yhat_p - b_p|| / ||b_p|| (grid points strictly inside, all p); add
 * the midpoints of intervals above tol (largest first, ties to the lower frequency) while the
 * model order stays <= m_max; re-solve, re-project and repeat until every estimate is <= tol.
 * With opts.deriv_indicator the estimate of an interval is the larger of the residual estimate and
 * d_k, d_{k+1} at its ends, d_k = max_pq |dGhat/dw - dG/dw| / max_pq |dG/dw| at the sampled w_k
 * (exact derivatives from the extra solves made when w_k was added; samples added before the option
 * was set, or restored by gfcc_mor_load, count d_k = 0).
 * m_out (host, optional) receives the final order; max_err (host, optional) the last estimate.
 * Returns GFCC_ERR_NOT_CONVERGED if m_max stopped the refinement first. */
int gfcc_mor_refine(gfcc_t ctx, double wmin, double wmax, int ngrid, double tol, int m_max,
                    int* m_out, double* max_err);

/* Evaluate the reduced model at nw frequencies (host array): Ghat (optional, host or device,
 * layout as in gfcc_solve_full) and A (optional, host or device). maxres (optional, host or
 * device): per-frequency max over p of the relative residual estimate. */
int gfcc_mor_eval(gfcc_t ctx, const double* omegas, int nw, double* G, double* A, double* maxres);

/* Sampled frequencies of the current model: writes up to cap values to w (host) and the count to
 * *ns; *m receives the model order, *np and *nq the sizes of the p and q orbital sets. Any output
 * pointer may be NULL. */
int gfcc_mor_info(gfcc_t ctx, double* w, int cap, int* ns, int* m, int* np, int* nq);

/* Work of the full-dimension solves made by gfcc_mor_build and gfcc_mor_refine since the last build:
 * Arnoldi steps summed over the solver's batches and columns solved (either pointer may be NULL). */
int gfcc_mor_stats(gfcc_t ctx, long long* arnoldi_steps, long long* columns);

/* Save / load the reduced model (sampled frequencies, S, Z = M S and the projected matrices) so that
 * refinement resumes without re-solving. The file is a flat binary written by this library. */
int gfcc_mor_save(gfcc_t ctx, const char* path);
int gfcc_mor_load(gfcc_t ctx, const char* path);

/* Diagnostic entry point of the tensor-core GEMM used by the low-precision sigma:
 * C[M][N] = A[M][K] . B[N][K]^T with A, B rounded to bf16 (GFCC_PREC_BF16) or tf32 (GFCC_PREC_TF32)
 * and FP32 accumulation. Host pointers, row-major; runs on the current device. The paper has no
 * counterpart: it exists to test the kernel in isolation. */
int gfcc_tc_gemm(int precision, const double* A, const double* B, int M, int N, int K, float* C);

/* Allocation-free variant of gfcc_tc_gemm, for callers that cannot allocate device memory at the
 * point of the call (a framework that owns all device memory, a path where the device-wide
 * synchronisation of cudaMalloc/cudaFree is not acceptable, code that must not hit out-of-memory
 * after start-up). The paper has no counterpart. A, B, C are device pointers on the current device
 * (row-major A[M][K], B[N][K], C[M][N]); C must be 16-byte aligned (GFCC_ERR_ARG otherwise, before any
 * device work); stream is a cudaStream_t or NULL. The call is synchronous: it waits on the stream and
 * returns after the product is complete. The rounded operand copies and the error flag live in a fixed 32 MiB __device__
 * array inside the library, reserved on every GPU that loads it until the process exits: the call
 * allocates nothing, and rejects with GFCC_ERR_ARG any size whose two rounded operands (K padded
 * to 64 bf16 or 32 tf32 elements, each copy rounded up to 256 bytes) plus 256 bytes do not fit.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture. The address is kept for the life of the CUDA context: do not
 * call this entry point on a device after resetting it (cudaDeviceReset). All calls share the array: calls whose work overlaps on a
 * GPU (different streams or threads) race and must be serialised by the caller. */
int gfcc_tc_gemm_noalloc(int precision, const double* A, const double* B, int M, int N, int K, float* C,
                         void* stream);

/* Autotuner of the tensor-core GEMM (the paper has no counterpart): on the first launch of each shape
 * bucket (precision, exact-slice or not, M tiles, ceil(log2(N tiles)), K per split, splits) whose output
 * is overwritten, every distinct M-tile group size of the L2 budgets 16, 40, 64, 96 and 128 MB is timed
 * twice with CUDA events on the launching stream and the fastest is kept for the rest of the process
 * (the group size orders the work units without changing their arithmetic; no tuning under stream
 * capture; environment variable GFCC_AUTOTUNE=0 keeps the 40 MB default). Entry i (in tuning order):
 * the bucket, the chosen and the default group size, and their best times in milliseconds. Any output
 * pointer may be NULL. GFCC_ERR_ARG when there is no entry i. */
int gfcc_autotune_info(int i, int* kind, int* exact, int* tiles_m, int* tiles_n_log2, int* gm, int* gm_default,
                       double* ms_best, double* ms_default);

/* Device memory. The library's buffers come from a stream-ordered memory pool of its own on each
 * device (cudaMallocFromPoolAsync / cudaFreeAsync on the context's stream), which keeps the memory it
 * has reserved when buffers are freed: frees do not wait for the device, and a context created after
 * another one was freed reuses its memory. A context should therefore be freed (gfcc_free) before the
 * stream it was created with is destroyed. This call waits for every device the library has used and
 * returns the pools' unused reserve to the device, for callers that need that memory elsewhere.
 * GFCC_ERR_CUDA if a device reports an error. The paper has no counterpart. */
int gfcc_release_cached_memory(void);

/* Number of CUDA kernels launched by this library since it was loaded (all contexts). */
long long gfcc_launch_count(void);

/* Turn per-launch CUDA-event timing of the GEMM kernel classes and of the pipeline phases on
 * (enable = 1) or off, clearing earlier records. Kernel classes: 0 tcgen05 GEMM with tf32/bf16-
 * rounded operands (inner solves); 1 FP64 SIMT GEMM; 2 tcgen05 GEMM on exact bf16 slices
 * (FP64-accurate products). Phases (whole regions, nested ones counted in both): 3 low-precision
 * sigma; 4 FP64-accurate sigma; 5 Arnoldi orthogonalisation and updates; 6 MOR orthonormalisation
 * and projections; 7 reduced-model evaluation; 8 H-bar build; 9 column-by-column Gram-Schmidt
 * inside new blocks; 10 extension of the residual basis; 11 the ring-term GEMM of the low-precision
 * sigma (counted here instead of class 0); 12 whole FP64-accurate complex GEMMs on exact slices;
 * 13 splitting of FP64 rows into exact slices; 14 the fused Gram-Schmidt sweeps of FP32-basis Arnoldi
 * steps; 15, 16, 17 the first, second and third of those sweeps alone for batches of at least 32
 * columns; 18 the three sweeps of batches of fewer than 32 columns (classes 14-18 count algorithmic
 * HBM bytes in the "flops" field, as do classes 13 and 24; classes 3 and 4 count the sigma's algorithmic
 * flops, whatever arithmetic carries them out); 19 Householder reductions of Hhat to Hessenberg form; 20 the
 * per-frequency shifted Hessenberg solves; 21, 22 the coefficient products and updates of the block
 * Gram-Schmidt passes; 23 the Cholesky QR of the panels; 24 the accumulation and output passes of the
 * exact-slice products; 25 the operand preparation and 26 the combine pass of the low-precision sigma;
 * 27 the copies of the caller's inputs to the device in gfcc_init; 28 the copies of results into the
 * caller's output buffers (device to host for host buffers); 29 and 30 the library's device
 * allocations and frees: their count and the host milliseconds spent inside cudaMalloc and cudaFree
 * (host clock, not events; cudaFree also waits for the device); 31 the up, oooo and down GEMMs of the
 * low-precision sigma again (also in class 0), with their algorithmic HBM bytes in the "flops" field
 * (operands read once, outputs written once, the accumulated down output read and written).
 * Events are recorded on the stream each region is launched on. */
int gfcc_profile(int enable);

/* Sum over the recorded launches of class cls: number of launches, device milliseconds (CUDA
 * events, waits for completion) and algorithmic flops (2 M N K per launch, K padded). */
int gfcc_profile_read(int cls, long long* launches, double* ms, double* flops);

/* Message of the last error on this context ("" if none). Valid until the next call. */
const char* gfcc_last_error(gfcc_t ctx);

/* Release all device memory of the context. NULL is allowed. */
void gfcc_free(gfcc_t ctx);

#ifdef __cplusplus
}
#endif
#endif /* GFCC_H */
