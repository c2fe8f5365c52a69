// Internal launcher declarations (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include "common.cuh"

namespace bse {

// ---- fft.cu ----
bool fft_supported(int N);
void twiddle_table(int N, std::vector<double2>& out);
template <typename T>
cudaError_t fft3d(cplx<T>* data, long n_batch, int N, int sign, const cplx<T>* table, cudaStream_t st);
template <typename T, typename TI>
cudaError_t sphere_unpack(const TI* P, long n_fields, int n_pw, int n_half, const int* gpos,
                          const int* gneg, cplx<T>* grids, long n3, bool zero_first,
                          bool accumulate, cudaStream_t st);
// g2h: 1/2|G|^2 per packed coordinate; esh: Delta - eps_v per orbital (both may be null
// when add_in is)
template <typename T, typename TO>
cudaError_t sphere_pack(const cplx<T>* grids, long n_fields, int n_pw, int n_half, const int* gpos,
                        const int* gneg, long n3, double scale, TO* out, const TO* add_in,
                        const T* g2h, const T* esh, int n_occ, cudaStream_t st);
template <typename T>
cudaError_t grid_coulomb(cplx<T>* grids, long n_grids, int N, double L, double omega, int mode,
                         double scale, cudaStream_t st);

// column-ordered plane-wave sphere for the pruned sphere <-> grid transforms (device
// arrays; see fft.cu): NS points (+G and -G), NC (x, y) columns, NX distinct x values
struct SphereMap {
  int NS = 0, NC = 0, NX = 0;
  const int *fpos = nullptr, *fneg = nullptr;   // [n_half] sphere position of +G_k, -G_k
  const int *zs = nullptr, *jcol = nullptr;     // [NS] z index, column of each point
  const int *cstart = nullptr;                  // [NC + 1] first point of each column
  const int *cy = nullptr, *cxi = nullptr;      // [NC] y index, x slot of each column
  const int *xs = nullptr, *xcol = nullptr;     // [NX] x index of each slot, [NX + 1] first column
};
struct SphereMapHost {
  int NS = 0, NC = 0, NX = 0;
  std::vector<int> fpos, fneg, zs, jcol, cstart, cy, cxi, xs, xcol;
};
void build_sphere_map(int N, int n_half, const int* miller, SphereMapHost& h);
size_t sphere_scratch_per_grid(int N, const SphereMap& m);
template <typename T>
cudaError_t sphere_to_grid(const T* P, long n_fields, int n_pw, int n_half, int N, const SphereMap& m,
                           const cplx<T>* table, cplx<T>* scratch, cplx<T>* grids, cudaStream_t st);
template <typename T>
cudaError_t grid_to_sphere(cplx<T>* grids, long n_fields, int n_pw, int n_half, int N, const SphereMap& m,
                           const cplx<T>* table, cplx<T>* scratch, double scale, T* out, const T* add_in,
                           const T* g2h, const T* esh, int n_occ, cudaStream_t st);

// ---- gemm.cu ----
// C = alpha A A^T, A n x K row-major: upper-triangle tiles, then mirrored
// symmetric Gram A A^T of FP64 data given as FP32 hi / lo splits, in float-float arithmetic
// (about 1e-14 relative)
cudaError_t gram_ff(int n, long K, const float* Ahi, const float* Alo, long lda, double* C, long ldc,
                    cudaStream_t st);
template <typename T, typename TC>
cudaError_t gemm(bool at, bool bt, int M, int N, int K, double alpha, const T* A, long lda,
                 const T* B, long ldb, double beta, TC* C, long ldc, int splitk, cudaStream_t st);

// ---- ops.cu ----
template <typename T>
cudaError_t pair_product(int nb, const int* pv, const int* pw, const T* upsi, long n3, double scale,
                         cplx<T>* grids, cudaStream_t st);
template <typename T>
cudaError_t scatter_tau4(int nb, const cplx<T>* grids, long n3, long p0, const int2* slot, long n_ent, T* tau4,
                         cudaStream_t st);
template <typename T>
cudaError_t deinterleave_pairs(int nb, const cplx<T>* grids, long n3, long p0, long n_pairs, T* tau,
                               cudaStream_t st);
cudaError_t square_fields_split(int n, const double* u, long n3, float* rho_hi, float* rho_lo, cudaStream_t st);
// clears C[row][w] (rows x n_occ) where orbital row % n_occ and w lie in different spin channels
template <typename T>
cudaError_t mask_cross_channel(int rows, int n_occ, int n_up, T* C, cudaStream_t st);
cudaError_t normalize_overlap(int n, double* gram, double* diag, cudaStream_t st);
template <typename T>
cudaError_t hartree_density(int n_vec, int n_occ, long n3, const T* a, const T* upsi, T* h,
                            cudaStream_t st);
template <typename T>
cudaError_t k1d_combine(int n_vec, int n_occ, long n3, const T* a, const T* tau, long n_pairs, const int* nbr_ptr,
                        const int* nbr_w, const int* nbr_p, const T* vloc, const T* vh,
                        const T* upsi, double spin_factor, T* out, cudaStream_t st);
// ---- tc_gemm.cu (tcgen05 BF16x3) ----
size_t tc_map_bytes();
bool tc_make_map(void* map_out, const void* ptr, long rows, long cols, long ld);
// wait_limit: polls of each pipeline wait before a CTA gives up, raises *err and drains
// (negative: the default)
cudaError_t tc_gemm_bf16x3(const void* mAh, const void* mAl, const void* mBh, const void* mBl, int M, int N,
                           int K, double alpha, double beta, float* out, long ldo, int splits, int* err,
                           cudaStream_t st, long long wait_limit = -1);
cudaError_t bf16_split(const float* X, long rows, int cols, long ld_in, void* hi, void* lo, long ld_out,
                       cudaStream_t st);
cudaError_t bf16_split64(const double* X, long rows, int cols, long ld_in, void* hi, void* lo, long ld_out,
                         bool transpose, cudaStream_t st);

// ---- precond.cu (learned preconditioner) ----
// parameter layout: W1[H x F] b1[H] W2[H x H] b2[H] w3[H] b3 mu[F] sigma[F]
namespace mlpl {
constexpr int H = 64, F = 5, W1 = 0, B1 = W1 + H * F, W2 = B1 + H, B2 = W2 + H * H, W3 = B2 + H,
              B3 = W3 + H, MU = B3 + 1, SG = MU + F, N = SG + F;
}
template <typename T>
cudaError_t precond_learned(int k, int n_occ, int n_pw, const float* params, const T* R,
                            const double* theta, const double* rnorm2, const int* which,
                            const double* g2p, const double* eps, double v0, double shift, T* out,
                            int* bad, cudaStream_t st);
cudaError_t mlp_train_forward(const float* params, long rows, int n_occ, int n_pw, const double* r,
                              const double* theta, const double* rnorm2, const double* g2p,
                              const double* eps, double v0, double shift, int bf, float* X, float* H1,
                              float* H2, float* O, double* G, double* Y, cudaStream_t st);
cudaError_t mlp_loss(long rows, long dim, const double* py, const double* tstar, const double* tn2,
                     const double* ab, const double* r, double inv_n, double* dg, double* loss,
                     cudaStream_t st);
cudaError_t mlp_train_backward(const float* params, long rows, const float* H1, const float* H2,
                               const float* O, const double* G, const double* dg, float* DO,
                               float* DZ1, float* DZ2, cudaStream_t st);
cudaError_t adam_step(int n_train, float* p, const double* g, float* m, float* v, float lr, int step,
                      cudaStream_t st);
cudaError_t feature_moments(long rows, int n_occ, int n_pw, const double* r, const double* theta,
                            const double* rnorm2, const double* g2p, const double* eps, double v0,
                            double shift, double* mom, cudaStream_t st);
cudaError_t jd_targets(int ns, long dim, const double* Y, const double* U, const double* uy, double* T,
                       cudaStream_t st);
cudaError_t shift_scale(int ns, int nr, double* C, const double* lam, const double* th, cudaStream_t st);
cudaError_t row_dots(int ns, long dim, const double* A, const double* B, double* out, cudaStream_t st);

// ---- lanczos.cu (absorption spectrum) ----
// d_v = -d psi_v / d r_i, packed (gdir: G_i per packed coordinate); P_c is applied by the caller
template <typename T>
cudaError_t dipole_rhs(int n_occ, int n_pw, const double* psi, const double* gdir, T* out, cudaStream_t st);
// W[p] -= coef[p * ldc] X[p] for chains p < n_chain; rec (nullable) receives the coefficients
template <typename T>
cudaError_t lanczos_axpy(int n_chain, long dim, T* W, const T* X, const double* coef, long ldc, double* rec,
                         long ld_rec, cudaStream_t st);
// Q[p] = W[p] / sqrt(n2[p]) (0 when n2 = 0); beta[p * ld_beta] = sqrt(n2[p])
template <typename T>
cudaError_t lanczos_normalize(int n_chain, long dim, const T* W, const double* n2, T* Q, double* beta, long ld_beta,
                              cudaStream_t st);
cudaError_t continued_fraction(int m, const double* alpha, const double* beta, double norm2, int n_omega,
                               const double* omega, double eta, double* gre, double* gim, cudaStream_t st);

// ---- jade.cu (Wannier localisation) ----
// W[w][r] = M_op(r) u[w][r] (squared: M_op(r)^2 u[w][r]); op = 2 axis + (0 cos, 1 sin)
cudaError_t jade_weight(int n, long n3, int N, int op, const double* u, double* W, bool squared, cudaStream_t st);
// one round of disjoint Givens rotations: angles from matrices 0..K_use-1, applied to all K
// matrices A [K][n][n] and to U [n][n]; smax collects the largest |sin| (float bits)
cudaError_t jade_round(int K_use, int K, int n, double* A, double* U, const int2* pairs, int np, double2* cs,
                       unsigned* smax, cudaStream_t st);
cudaError_t set_identity(int n, double* U, cudaStream_t st);
void jade_schedule(int n, std::vector<int2>& pairs, int& rounds, int& per_round);

// ---- k1d_sym.cu (tau stored once per pair) ----
// Row-block lists of the symmetric-layout K1d kernel (device arrays). Row block b = orbitals
// 4b..4b+3. Upper entries: for each b, every neighbour w >= 4b of any of b's rows, in
// increasing w; entry e stores tau_{4b+i, w}, i = 0..3, in the entry-major tau (tau4_off).
// Transposed tiles: for each b, every earlier block J < b with a pair to b; tile k names J's
// entries (J, 4b+i) (-1 where absent) and the rows j of J that pair with b.
struct K1dLists {
  long n_ent = 0;                 // upper entries
  int n_blocks = 0;               // ceil(n_occ / 4)
  const int* bptr = nullptr;      // [n_blocks + 1] upper entries of block b: bptr[b] .. bptr[b+1]
  const int* bw = nullptr;        // [n_ent] neighbour w of each entry
  const int* tptr = nullptr;      // [n_blocks + 1] transposed tiles of block b
  const int* tinfo = nullptr;     // [n_tiles] (J << 4) | (mask of J's rows j that pair with b)
  const int4* tent = nullptr;     // [n_tiles] entries (J, 4b+i), i = 0..3, -1 where absent
};
int k1d_sym_num_variants();
int k1d_sym_padded_vectors(int n_vec, int variant);
template <typename T>
int k1d_sym_default_variant(int n_occ, int n_vec);
template <typename T>
bool k1d_sym_fits(int n_occ, int variant);
template <typename T>
cudaError_t k1d_sym_tiled(int n_vec, int n_occ, long n3, const T* a, const T* tau4, const K1dLists& L,
                          const T* vloc, const T* vh, const T* upsi, double sf, T* out, int variant,
                          cudaStream_t st, long n_pts = -1);

// ---- k1d.cu ----
// tile variants of the K1d kernel, numbered 1 .. k1d_num_variants(); 0 = default for the width
int k1d_num_variants();
int k1d_padded_vectors(int n_vec, int variant);
template <typename T>
int k1d_default_variant(int n_occ, int n_vec);
template <typename T>
bool k1d_fits(int n_occ, int variant);
template <typename T>
cudaError_t k1d_tiled(int n_vec, int n_occ, long n3, const T* a, const T* tau4, long n_ent, const int* bptr,
                      const int* bw, int n_blocks, const T* vloc, const T* vh,
                      const T* upsi, double sf, T* out, int variant, cudaStream_t st, long n_pts = -1);
template <typename T>
cudaError_t scale_columns(int rows, int cols, T* C, long ldc, const double* f, cudaStream_t st);
template <typename TI, typename TO>
cudaError_t convert(long n, const TI* in, TO* out, cudaStream_t st);
template <typename T>
cudaError_t pair_grid_to_rows(int n, const T* grids, long n3, T* rows, cudaStream_t st);
template <typename T>
cudaError_t residuals(int k, long dim, const T* X, const T* LX, const double* theta, T* R,
                      double* norms2, cudaStream_t st);
template <typename T>
cudaError_t row_norms2(int k, long dim, const T* X, double* norms2, cudaStream_t st);
template <typename T>
cudaError_t precond_diag(int k, int n_occ, int n_pw, const T* R, const double* theta,
                         const int* which, const T* g2h, const double* eps, double v0,
                         double shift, T* out, cudaStream_t st);
template <typename T>
cudaError_t zero_pad_column(int rows, int n_pw, T* X, cudaStream_t st);
template <typename T>
cudaError_t scale_rows(int k, long dim, T* X, const double* s, cudaStream_t st);
template <typename T>
cudaError_t set_unit(T* x, long dim, long idx, cudaStream_t st);
cudaError_t symmetrize(int m, double* A, long lda, cudaStream_t st);
cudaError_t mirror_new(double* A, long lda, int m0, int m1, cudaStream_t st);
cudaError_t eigh_lowest(int m, int k, const double* A, long lda, double* work, double* V, double* w,
                        int* info, bool single, cudaStream_t st);
cudaError_t cholesky_inverse(int b, const double* S, long lds, double* Linv, int* info,
                             cudaStream_t st);
bool finite_check_host(const double* x, long n);

}  // namespace bse
