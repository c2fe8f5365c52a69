// Kernels of the Lanczos absorption-spectrum driver (Section 4: the spectrum of bulk Si comes
// from a Lanczos recursion of N_Lanczos applications of the Liouville operator per
// polarisation direction). The operator itself is the hot path of bse_apply_liouville; these
// kernels build the dipole start block, carry the three-term recursion on the device (so a
// chain of any length runs without host round trips) and evaluate the continued fraction.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace bse {

namespace {

// d_v = -d psi_v / d r_i in packed form: c'(G) = -i G_i c(G), i.e. p'[2k] = G_i p[2k+1],
// p'[2k+1] = -G_i p[2k] (G = 0 and the pad stay 0). gdir: G_i per packed coordinate.
template <typename T>
__global__ void dipole_rhs_kernel(int n_occ, int n_pw, const double* __restrict__ psi,
                                  const double* __restrict__ gdir, T* __restrict__ out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long half = (long)n_occ * (n_pw / 2);
  if (idx >= half) return;
  const long v = idx / (n_pw / 2), k = idx - v * (n_pw / 2);
  const double* p = psi + v * n_pw + 2 * k;
  T* o = out + v * n_pw + 2 * k;
  const double g = (k == 0) ? 0.0 : gdir[2 * k];
  o[0] = (T)(g * p[1]);
  o[1] = (T)(-g * p[0]);
}

// W[p] -= coef[p * ldc] * X[p] for each chain p; with alpha_out, also records the
// coefficient at alpha_out[p * ld_out]
template <typename T>
__global__ void lanczos_axpy_kernel(long dim, T* __restrict__ W, const T* __restrict__ X,
                                    const double* __restrict__ coef, long ldc, double* __restrict__ rec,
                                    long ld_rec) {
  const int p = blockIdx.y;
  const double a = coef[(long)p * ldc];
  if (rec && blockIdx.x == 0 && threadIdx.x == 0) rec[(long)p * ld_rec] = a;
  const T at = (T)a;
  T* w = W + (long)p * dim;
  const T* x = X + (long)p * dim;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (long)gridDim.x * blockDim.x)
    w[i] -= at * x[i];
}

// Q[p] = W[p] / sqrt(n2[p]) (zero after a breakdown, n2 = 0); records beta = sqrt(n2)
template <typename T>
__global__ void lanczos_normalize_kernel(long dim, const T* __restrict__ W, const double* __restrict__ n2,
                                         T* __restrict__ Q, double* __restrict__ beta, long ld_beta) {
  const int p = blockIdx.y;
  const double b = sqrt(fmax(n2[p], 0.0));
  if (blockIdx.x == 0 && threadIdx.x == 0) beta[(long)p * ld_beta] = b;
  const T s = (b > 0.0) ? (T)(1.0 / b) : (T)0;
  const T* w = W + (long)p * dim;
  T* q = Q + (long)p * dim;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (long)gridDim.x * blockDim.x)
    q[i] = s * w[i];
}

// g(omega + i eta) = norm2 / (z - alpha_0 - beta_1^2 / (z - alpha_1 - ...)), bottom up; one
// thread per frequency
__global__ void continued_fraction_kernel(int m, const double* __restrict__ alpha, const double* __restrict__ beta,
                                          double norm2, int n_omega, const double* __restrict__ omega, double eta,
                                          double* __restrict__ gre, double* __restrict__ gim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_omega) return;
  const double zr = omega[i], zi = eta;
  double fr = 0.0, fi = 0.0;   // f_{k+1}
  for (int k = m - 1; k >= 0; --k) {
    const double b2 = (k + 1 < m) ? beta[k + 1] * beta[k + 1] : 0.0;
    const double dr = zr - alpha[k] - b2 * fr, di = zi - b2 * fi;   // z - alpha_k - b2 f
    const double den = dr * dr + di * di;
    fr = dr / den;
    fi = -di / den;
  }
  gre[i] = norm2 * fr;
  gim[i] = norm2 * fi;
}

inline unsigned blocks_for(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

template <typename T>
cudaError_t dipole_rhs(int n_occ, int n_pw, const double* psi, const double* gdir, T* out, cudaStream_t st) {
  const long half = (long)n_occ * (n_pw / 2);
  if (half <= 0) return cudaSuccess;
  dipole_rhs_kernel<T><<<blocks_for(half), 256, 0, st>>>(n_occ, n_pw, psi, gdir, out);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t lanczos_axpy(int n_chain, long dim, T* W, const T* X, const double* coef, long ldc, double* rec,
                         long ld_rec, cudaStream_t st) {
  if (n_chain <= 0 || dim <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long>(1184, (dim + 255) / 256), (unsigned)n_chain);
  lanczos_axpy_kernel<T><<<grid, 256, 0, st>>>(dim, W, X, coef, ldc, rec, ld_rec);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t lanczos_normalize(int n_chain, long dim, const T* W, const double* n2, T* Q, double* beta, long ld_beta,
                              cudaStream_t st) {
  if (n_chain <= 0 || dim <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long>(1184, (dim + 255) / 256), (unsigned)n_chain);
  lanczos_normalize_kernel<T><<<grid, 256, 0, st>>>(dim, W, n2, Q, beta, ld_beta);
  note_launch();
  return cudaGetLastError();
}

cudaError_t continued_fraction(int m, const double* alpha, const double* beta, double norm2, int n_omega,
                               const double* omega, double eta, double* gre, double* gim, cudaStream_t st) {
  if (n_omega <= 0) return cudaSuccess;
  continued_fraction_kernel<<<blocks_for(n_omega), 256, 0, st>>>(m, alpha, beta, norm2, n_omega, omega, eta, gre,
                                                                  gim);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t dipole_rhs<float>(int, int, const double*, const double*, float*, cudaStream_t);
template cudaError_t dipole_rhs<double>(int, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t lanczos_axpy<float>(int, long, float*, const float*, const double*, long, double*, long,
                                         cudaStream_t);
template cudaError_t lanczos_axpy<double>(int, long, double*, const double*, const double*, long, double*, long,
                                          cudaStream_t);
template cudaError_t lanczos_normalize<float>(int, long, const float*, const double*, float*, double*, long,
                                              cudaStream_t);
template cudaError_t lanczos_normalize<double>(int, long, const double*, const double*, double*, double*, long,
                                               cudaStream_t);

}  // namespace bse
