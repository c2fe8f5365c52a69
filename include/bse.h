/*
 * bse.h -- C ABI of the GB300 (sm_103a) DMPT/TDA Bethe-Salpeter hot path.
 *
 * The library applies the Tamm-Dancoff Liouville operator (D + K1e - K1d) of
 * Eq. (evp) (Yu, Jin, Galli, Govoni, "GPU-Accelerated Solution of the
 * Bethe-Salpeter Equation for Large and Heterogeneous Systems", Section 2) to
 * blocks of trial vectors, builds the screened integrals tau_vw of Eqs. (tau),
 * (tau_from_tau_u) with the low-rank chi_bar of Eq. (pdep), and finds the lowest
 * vertical excitation energies with a block Davidson solver (Section 3).
 *
 * Conventions used by every call
 * ------------------------------
 *  - Gamma point, cubic cell of edge L (bohr), FFT grid N^3, real-space index
 *    r = x + N*(y + N*z) (x fastest). Hartree atomic units.
 *  - Plane-wave sphere S given by Miller indices miller[n_half][3]: row 0 is
 *    (0,0,0), rows k >= 1 hold one representative of each {+G_k, -G_k}. Every
 *    |component| must be <= (N-1)/4 so that all products are alias-free.
 *  - Gamma-packed real vectors of length n_pw = 2*n_half:
 *      p[0] = c(0), p[1] = 0 (pad; inputs must hold 0, outputs always hold 0),
 *      p[2k] = sqrt(2) Re c(G_k), p[2k+1] = sqrt(2) Im c(G_k),
 *    where f(r) = Omega^{-1/2} sum_{G in S} c(G) e^{iG.r}. Dot products of packed
 *    vectors equal L2 inner products of the functions.
 *  - A block of trial vectors is [n_vec][n_occ][n_pw] row-major: the N_occ
 *    auxiliary orbitals a_{s,v} of each A_s (Eq. evp, Delta rho_s = sum_v |a_sv><psi_v|).
 *  - v(G) = 4 pi/|G|^2 for G != 0, v(0) = 0, and the head term Xi of Eq. (pdep) is 0.
 *
 * Ownership: the caller owns every pointer it passes; input arrays are read during
 * the call only. The context owns its device buffers (tau, plans, workspaces); it
 * obtains every one of them from the allocator given to bse_create (or, without one,
 * from cudaMallocAsync on the context stream) and returns them before bse_destroy
 * returns. All device work is ordered on the stream given to bse_create; calls return
 * after that work has completed.
 *
 * Errors: every call returns a bse_status. On error no output is valid (except
 * BSE_ERR_NOT_CONVERGED, see bse_davidson) and bse_last_error() describes it. The
 * library never traps or aborts; device waits are bounded.
 */
#ifndef BSE_H_
#define BSE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSE_OK = 0,
  BSE_ERR_INVALID_ARG = -1,   /* bad size, pointer, or layout */
  BSE_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  BSE_ERR_OOM = -3,           /* device allocation failed */
  BSE_ERR_NUMERIC = -4,       /* non-finite input or breakdown (e.g. Cholesky) */
  BSE_ERR_NOT_CONVERGED = -5, /* Davidson hit max_it; outputs hold the last Ritz values */
  BSE_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
  BSE_ERR_STATE = -7          /* call order violated (e.g. apply before build_tau) */
} bse_status;

typedef enum {
  BSE_PREC_FP64 = 0,   /* plain method: every step in FP64 */
  BSE_PREC_MIXED = 1   /* FP32 FFTs / pair products / tau streaming, BF16x3 tensor-core
                          projections with FP32 accumulation, FP64 Davidson algebra */
} bse_precision;

typedef struct bse_ctx bse_ctx;   /* opaque, library-owned */

/* One Gamma-point system (all host pointers, FP64 unless noted). */
typedef struct {
  int n_grid;              /* N: FFT grid N^3; N in {16, 32, 48, 64, 72, 96} */
  double L;                /* cubic cell edge (bohr) */
  int n_half;              /* rows of miller */
  const int32_t* miller;   /* [n_half][3] (x, y, z) integer components of G_k */
  int n_occ;               /* N_occ occupied orbitals */
  const double* psi;       /* [n_occ][2*n_half] packed, orthonormal (Section 2, Eq. wannier) */
  const double* eps;       /* [n_occ] occupied energies eps_v (Ha), Eq. (d) */
  const double* v_loc;     /* [N^3] local potential samples (Ha), H_KS of Eq. (ham) */
  double scissor;          /* Delta (Ha): H_QP = H_KS + Delta on the conduction space, Eq. (ham) */
  int n_pdep;              /* N_PDEP (may be 0: unscreened) */
  const double* pdep;      /* [n_pdep][2*n_half] packed, orthonormal, entries 0,1 zero (Eq. pdep) */
  const double* lambda;    /* [n_pdep] PDEP eigenvalues, each in (-1, 0) (Eq. pdep) */
  double overlap_thr;      /* > 0: keep tau_vw iff O_vw >= overlap_thr (Eq. overlap) */
  int64_t keep_pairs;      /* used when overlap_thr <= 0: number of v <= w pairs to keep */
  int spin;                /* 0 singlet (K1e factor 2, Eq. k1e), 1 triplet (factor 0) */
  /* Explicit quasi-particle energies (Eq. ham). n_qp = 0: the scissor form above. n_qp > n_occ:
   * H_QP = H_KS + sum_{n <= N_QP} |psi_n>(eps^QP_n - eps_n - Delta)<psi_n| + Delta, with
   * Delta the mean of eps^QP_n - eps_n over n = N_mid..N_QP, N_mid = (N_occ + N_QP) / 2
   * (1-based, integer division); eps^QP_v replaces eps_v in D and `eps`, `scissor` are
   * ignored. */
  int n_qp;
  const double* qp_psi;    /* [n_qp - n_occ][2*n_half] packed KS states n_occ+1..N_QP (orthonormal,
                              orthogonal to psi); the occupied terms of the sum vanish under P_c */
  const double* qp_eps_ks; /* [n_qp] KS energies eps_n of states 1..N_QP (Ha) */
  const double* qp_eps;    /* [n_qp] QP energies eps^QP_n of states 1..N_QP (Ha) */
  /* Spin-polarised systems with spin-conserving excitations (Section 2: the paper's code
   * supports them; Eqs. evp-k1d are written for one channel). n_up = 0: closed shell. n_up > 0:
   * orbitals [0, n_up) of psi/eps are spin up and [n_up, n_occ) spin down, each its own
   * spin-orbital; each channel has its own projector P_c (occupied orbitals of that channel),
   * K1e couples both channels through the Hartree potential of the total density change with
   * factor 1 (`spin` is ignored), and tau_vw (K1d) is kept only within a channel. Both
   * channels share v_loc and the PDEP basis. */
  int n_up;
} bse_system;

/* Caller-supplied device allocator (e.g. the PyTorch caching allocator). alloc returns
 * `bytes` of device memory on the current device, aligned to at least 256 bytes, or NULL
 * when it cannot (the call then fails with BSE_ERR_OOM); free returns a block obtained from
 * alloc. Both are called from the thread that makes the library call (for bse_solve_batch,
 * from one worker thread per context, possibly at the same time) and in the order of the
 * context stream: a freed block may still be read by work already queued on that stream,
 * so the allocator may hand it out again only to work ordered after it on that stream, as a
 * stream-ordered or caching allocator bound to that stream does. `user` is passed through. */
typedef void* (*bse_alloc_fn)(size_t bytes, void* user);
typedef void (*bse_free_fn)(void* ptr, void* user);

/* Create a context: validates the system, uploads it, computes psi_v(r).
 * alloc_fn, free_fn: the device allocator for every buffer the context owns; both NULL
 * selects cudaMallocAsync / cudaFreeAsync on the context stream; exactly one NULL is
 * BSE_ERR_INVALID_ARG. user: passed to both. stream: a cudaStream_t (NULL = legacy
 * default stream). Device = current device. On failure *out may hold a context that
 * only carries the error text (bse_last_error); release it with bse_destroy. */
int bse_create(const bse_system* sys, int precision, bse_alloc_fn alloc_fn, bse_free_fn free_fn,
               void* user, void* stream, bse_ctx** out);

/* Overlaps O_vw (Eq. overlap, grid quadrature of FP64 densities, accumulated in float-float
 * arithmetic to about 1e-14 relative, in both precision modes), the pair rule, and the screened
 * integrals tau_vw = W[psi_v psi_w] for every kept pair v <= w (Eqs. tau,
 * tau_from_tau_u, pdep). Pair rule: keep iff O_vw >= thr; with keep_pairs the
 * threshold is the midpoint of the gap between the k-th and (k+1)-th largest
 * off-diagonal overlaps (k = keep_pairs - n_occ), moved to the nearest gap of at
 * least 1e-9 of its midpoint, checked at k+1, k-1, k+2, k-2, ...; diagonal pairs
 * are always kept. Outputs (nullable): number of kept v <= w pairs, threshold. */
int bse_build_tau(bse_ctx* ctx, int64_t* n_pairs_out, double* thr_out);

/* Kept pairs in row-major (v, w), v <= w order; host arrays of length n_pairs. */
int bse_get_pairs(const bse_ctx* ctx, int32_t* v_out, int32_t* w_out);

/* Overlap matrix O (host [n_occ][n_occ], FP64), available after bse_build_tau. */
int bse_get_overlaps(const bse_ctx* ctx, double* o_out);

/* R = P_c (D + K1e - K1d) A for a block of n_vec trial vectors (Eqs. evp, d, k1e, k1d).
 * a_in, a_out: DEVICE pointers [n_vec][n_occ][n_pw], double for BSE_PREC_FP64 and
 * float for BSE_PREC_MIXED. a_in must lie in the conduction space (P_c a = a) with
 * zero pad entries; a_out must not alias a_in. Requires bse_build_tau first. */
int bse_apply_liouville(bse_ctx* ctx, int n_vec, const void* a_in, void* a_out);

/* The same operator as bse_apply_liouville, for callers that cannot allocate device
 * memory at call time: processes whose device memory is handed out by an external pool
 * with a fixed budget, or latency-critical paths where an allocation (which may
 * synchronise the device) is not allowed. The paper has no counterpart; this is a
 * library addition.
 *
 * The r-space workspaces of the call live in one fixed 32 MiB array compiled into the
 * library (every GPU that loads the library holds it until the process exits). No
 * cudaMalloc, cudaFree or allocating library routine is called; the context must
 * still have been created and bse_build_tau run. Limit: 2 * ceil(n_vec*n_occ/2) +
 * ceil(n_vec/2) complex grids of N^3 points plus n_vec*n_occ*max(n_occ, n_qp - n_occ)
 * projector coefficients (each part rounded up to 256 bytes) must fit in 32 MiB; larger requests
 * return BSE_ERR_INVALID_ARG with the byte count in bse_last_error(). The projector
 * runs on the SIMT GEMM in both precisions.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * once for that device. All calls share
 * the one array and it keeps the previous call's contents (the call clears what it
 * reads before writing): calls that overlap on the GPU, on any stream or from any
 * thread, race on it and must be serialised by the caller. Arguments and result as in
 * bse_apply_liouville. */
int bse_apply_liouville_static(bse_ctx* ctx, int n_vec, const void* a_in, void* a_out);

typedef struct {
  int n_eig;        /* number of lowest excitations wanted */
  int block;        /* trial vectors added per iteration (also the initial count) */
  int max_sub;      /* maximum subspace size; restart keeps 2*n_eig Ritz vectors */
  int max_it;       /* iteration limit */
  double res_tol;   /* converged when every ||L x - theta x||_2 <= res_tol (Ha) */
  int precond;      /* 0 diagonal: t = P_c r / max(1/2|G|^2 + V(0) + Delta - eps_v - theta, 0.1 Ha);
                       1 learned (bse_precond_load); the diagonal step replaces it when no
                       network is loaded, on a non-finite output, and for good once the largest
                       residual gains less than 1% over eight iterations */
} bse_davidson_opts;

typedef struct {
  int iterations;
  int n_apply;          /* trial vectors passed through the operator */
  double ms_total;      /* wall time of the call (CUDA events on the context stream) */
  double ms_apply;      /* of which operator applications */
  double res_max;       /* largest residual norm at exit */
  int precond_fallbacks;/* learned corrections replaced by the diagonal ones */
} bse_davidson_stats;

/* Lowest n_eig eigenpairs of the Liouville operator (Eq. evp) by block Davidson.
 * omega_out: host [n_eig] (Ha), ascending. vec_out (nullable): DEVICE
 * [n_eig][n_occ][n_pw] in the context precision. stats (nullable).
 * On BSE_ERR_NOT_CONVERGED omega_out, vec_out and stats hold the last Ritz pairs. */
int bse_davidson(bse_ctx* ctx, const bse_davidson_opts* opts, double* omega_out,
                 void* vec_out, bse_davidson_stats* stats);

/* Wannier localisation of the occupied orbitals (Section 2, Eqs. wannier and spread): the
 * orthogonal U that jointly diagonalises, approximately, the six matrices
 * A^(n)_vw = <psi_v|M^(n)|psi_w>, M = cos(2 pi x/L), sin(2 pi x/L), cos(2 pi y/L), ... (JADE),
 * i.e. minimises sigma^2(U) = sum_n [Tr(U^T B^(n) U) - sum_v ((U^T A^(n) U)_vv)^2]. U starts
 * from the eigenvectors of A^(1) (sweeps on A^(1) alone), then sweeps of Givens rotations on
 * all six run until every rotation has |sin| <= tol or max_sweeps is reached. The context
 * then works in the localised frame: its orbitals become psi~_v = sum_w U_wv psi_w, so that
 * the overlap rule (Eq. overlap) and tau act on localised orbitals, and the occupied energies
 * of D (Eq. d) become the matrix E = U^T diag(eps) U (D a_v = P_c H a_v - sum_w E_vw a_w);
 * excitation energies are unchanged, eigenvectors come out in the localised frame (rotate
 * back with U). Must run before bse_build_tau; closed-shell systems only. Outputs
 * (nullable): U_out host [n_occ][n_occ] (column v = coefficients of psi~_v), spread_out
 * host [2] = sigma^2 before and after. */
int bse_localize(bse_ctx* ctx, int max_sweeps, double tol, double* U_out, double* spread_out);

/* Lanczos chains for the optical absorption spectrum (Section 4: the spectrum of bulk Si is
 * computed with a Lanczos recursion of N_Lanczos applications of the Liouville operator per
 * polarisation direction, instead of an iterative diagonalisation). For each direction
 * dirs[p] (0 = x, 1 = y, 2 = z), p < n_pol <= 3, the chain starts from the dipole block
 * d_v = P_c(-d psi_v / d r_i), v = 1..N_occ (the commutator [H, r_i] of the local
 * Hamiltonian acting on the occupied orbitals; velocity form), and runs
 *   w = L q_k - beta_k q_{k-1}, alpha_k = <q_k|w>, w -= alpha_k q_k, w <- P_c w,
 *   beta_{k+1} = |w|, q_{k+1} = w / beta_{k+1}
 * for n_steps applications of the operator, the directions together as one block on the
 * device. Outputs (host, FP64): alpha_out, beta_out [n_pol][n_steps] (beta[p][0] = 0;
 * beta[p][k] couples steps k-1 and k; after a breakdown, beta = 0, the chain continues with
 * zeros), norm2_out [n_pol] = |d|^2. The vectors are in the context precision; the
 * coefficients are accumulated in FP64. Requires bse_build_tau first. */
int bse_lanczos(bse_ctx* ctx, int n_pol, const int* dirs, int n_steps, double* alpha_out, double* beta_out,
                double* norm2_out);

/* Spectral function of one chain on the GPU: g(omega + i eta) = <d|(omega + i eta - L)^{-1}|d>
 * = norm2 / (z - alpha_0 - beta_1^2 / (z - alpha_1 - beta_2^2 / ...)) for n_omega
 * frequencies (Ha), eta > 0 the broadening; the absorption line shape is -Im g / pi.
 * alpha, beta: one chain's n_steps coefficients as returned by bse_lanczos; all arrays are
 * host FP64; g_re, g_im: host [n_omega]. Uses the context's stream and allocator only. */
int bse_lanczos_spectrum(bse_ctx* ctx, int n_steps, const double* alpha, const double* beta, double norm2,
                         int n_omega, const double* omega, double eta, double* g_re, double* g_im);

/* Batched solves (library addition; the paper distributes one system over many GPUs,
 * Section 3): for each of n independent contexts -- typically many small systems of
 * uneven grid and orbital counts -- builds tau if needed and runs bse_davidson with the
 * same options. A pool of host threads (BSE_BATCH_WORKERS, default 16) takes the systems in
 * order, one thread per system at a time; a system that runs out of device memory is solved
 * again, alone, after the others. Contexts created on distinct CUDA streams run their
 * kernels concurrently on the device; contexts sharing a stream serialise. omega_out: host [n][opts->n_eig]; stats (nullable): host [n];
 * status_out (nullable): host [n] per-system status. Returns BSE_OK or the first
 * failing status. */
int bse_solve_batch(bse_ctx* const* ctxs, int n, const bse_davidson_opts* opts, double* omega_out,
                    bse_davidson_stats* stats, int* status_out);

/* ---- Learned Davidson preconditioner (library addition; the paper's Davidson of
 * Section 3 has no learned component). A per-element MLP 5 -> 64 -> 64 -> 1 rescales the
 * diagonal step: features f = (1/2|G|^2, eps_v, theta, d - theta, r_e sqrt(dim)/||r||),
 * x = (f - mu)/sigma, h1 = act(relu(W1 x + b1)), h2 = act(relu(W2 h1 + b2)),
 * o = w3.h2 + b3, t = P_c(exp(clip(o,-8,8)) r / max(d - theta, 0.1 Ha)), with
 * d = 1/2|G|^2 + V(0) + Delta - eps_v and act = bfloat16 rounding (FP32 weights, BF16
 * activations). A zero last layer is the diagonal preconditioner. Parameters: float
 * [BSE_PRECOND_NPARAM] = W1[64x5] b1[64] W2[64x64] b2[64] w3[64] b3 mu[5] sigma[5].
 * Loss over samples (theta, r, t*): the scale-free misfit mean(1 - <y,t*>^2/(|y|^2 |t*|^2)),
 * y = P_c(g r) -- Davidson keeps only a correction's direction. ---- */
#define BSE_PRECOND_NPARAM 4619

/* Runs the plain solver twice on an FP64 context: once to ref_eig (<= 32) eigenpairs
 * (res_tol 1e-8), once with opts (diagonal preconditioner), capturing up to max_samples
 * (residual, Ritz value, Ritz vector) triples of the corrections it computes. Targets
 * are the exact Jacobi-Davidson corrections t* = y/(u.y) - u, y = (L - theta)^{-1} u (the
 * solution of (I - uu^T)(L - theta)(I - uu^T) t = -r with t.u = 0): the component of y in
 * the span of the reference eigenvectors x_j is sum_j x_j (x_j.u)/(lambda_j - theta), the
 * rest is solved by conjugate gradients on the complement of that span (relative residual
 * 1e-12, where L - theta is positive definite as long as theta lies below the eigenvalues
 * not in the reference set). Replaces the context's samples; *n_out (nullable) receives
 * their number. */
int bse_precond_collect(bse_ctx* ctx, const bse_davidson_opts* opts, int ref_eig, int max_samples,
                        int* n_out);

/* Copies up to n of the context's samples to host arrays (each nullable): u_out, r_out,
 * t_out [n][n_occ][n_pw] (Ritz vectors -- only for samples from bse_precond_collect --,
 * residuals, targets), theta_out [n]; *n_out (nullable) = samples held. */
int bse_precond_get_samples(bse_ctx* ctx, int n, double* u_out, double* r_out, double* t_out, double* theta_out,
                            int* n_out);

/* Replaces the context's samples with caller data: host [n][n_occ][n_pw] residuals r and
 * targets t, host [n] Ritz values theta (FP64). */
int bse_precond_set_samples(bse_ctx* ctx, int n, const double* r, const double* t, const double* theta);

/* Loss and gradient (host double [BSE_PRECOND_NPARAM]; mu, sigma entries 0) of the
 * parameters over the context's samples; act_bf16 selects bfloat16 activations. */
int bse_precond_grad(bse_ctx* ctx, const float* params, int act_bf16, double* loss_out, double* grad_out);

/* Adam training on the GPU over the samples of n_ctx contexts (one step per context per
 * epoch), starting from init; mu and sigma are set from the samples' feature moments.
 * params_out: host float [BSE_PRECOND_NPARAM]; loss_hist (nullable): host [epochs]. */
int bse_precond_train(bse_ctx* const* ctxs, int n_ctx, const float* init, int epochs, double lr,
                      int act_bf16, float* params_out, double* loss_hist);

/* Installs (or with NULL removes) the network used by bse_davidson when opts.precond = 1. */
int bse_precond_load(bse_ctx* ctx, const float* params);

/* Per-region profile (library addition; the paper reports module wall times only,
 * Fig. 3). When enabled, each instrumented region of the hot path is bracketed by
 * CUDA events recorded on the context stream, so a region's time is the device time
 * of the kernels it launches. bytes / flops are the region's ALGORITHMIC traffic and
 * work (each operand read once, each result written once), not measured counters. */
typedef struct {
  char name[32];
  int64_t calls;   /* times the region ran */
  double ms;       /* summed device time */
  double bytes;    /* summed algorithmic bytes */
  double flops;    /* summed algorithmic floating-point operations */
} bse_prof_entry;

/* mode 1: enable, 0: disable, -1: clear accumulated entries. */
int bse_profile(bse_ctx* ctx, int mode);

/* Copies up to cap entries to out (nullable), sets *n_out (nullable) to the number of
 * regions and *launches (nullable) to the kernel launches this library has issued in
 * this process. ctx may be NULL to read the launch count alone. */
int bse_profile_read(bse_ctx* ctx, bse_prof_entry* out, int cap, int* n_out, int64_t* launches);

/* Human-readable description of the last error on this context (never NULL). */
const char* bse_last_error(const bse_ctx* ctx);

/* Library build string (compile flags, arch). */
const char* bse_version(void);

void bse_destroy(bse_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* BSE_H_ */
