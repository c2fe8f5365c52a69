// Pointwise, streaming and small dense kernels of the Liouville operator and the
// Davidson solver.
#include "common.cuh"
#include "kernels.h"
#include <atomic>
#include <cmath>

namespace bse {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static inline unsigned nblk(long total, int t = 256) { return (unsigned)((total + t - 1) / t); }

// ---------------------------------------------------------------------------------
// tau build: pair densities psi_v psi_w (Eq. tau), two pairs per complex grid
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void pair_product_kernel(int nb, const int* __restrict__ pv, const int* __restrict__ pw,
                                    const T* __restrict__ upsi, long n3, T scale,
                                    cplx<T>* __restrict__ grids) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long c = blockIdx.y;
  if (r >= n3) return;
  const long idx = c * n3 + r;
  const int p0 = (int)(2 * c), p1 = p0 + 1;
  cplx<T> F;
  F.x = upsi[pair_off<T>(pv[p0], r, n3)] * upsi[pair_off<T>(pw[p0], r, n3)] * scale;
  F.y = p1 < nb ? upsi[pair_off<T>(pv[p1], r, n3)] * upsi[pair_off<T>(pw[p1], r, n3)] * scale : (T)0;
  grids[idx] = F;
}

template <typename T>
cudaError_t pair_product(int nb, const int* pv, const int* pw, const T* upsi, long n3, double scale,
                         cplx<T>* grids, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  dim3 grid(nblk(n3), (nb + 1) / 2);
  pair_product_kernel<T><<<grid, 256, 0, st>>>(nb, pv, pw, upsi, n3, (T)scale, grids); note_launch();
  return cudaGetLastError();
}

// pairs p0 .. p0+nb-1 (two per complex grid) into the point-tiled tau array
template <typename T>
__global__ void deinterleave_kernel(int nb, const cplx<T>* __restrict__ grids, long n3, long p0,
                                    long n_pairs, T* __restrict__ tau) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long c = blockIdx.y;
  if (r >= n3) return;
  const cplx<T> F = grids[c * n3 + r];
  tau[tau_off(p0 + 2 * c, r, n_pairs)] = F.x;
  if (2 * c + 1 < nb) tau[tau_off(p0 + 2 * c + 1, r, n_pairs)] = F.y;
}

template <typename T>
cudaError_t deinterleave_pairs(int nb, const cplx<T>* grids, long n3, long p0, long n_pairs, T* tau,
                               cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  if (n3 % TAU_TB) return cudaErrorInvalidValue;
  dim3 grid(nblk(n3), (nb + 1) / 2);
  deinterleave_kernel<T><<<grid, 256, 0, st>>>(nb, grids, n3, p0, n_pairs, tau); note_launch();
  return cudaGetLastError();
}

// pair values of the batch into the entry-major tau: pair p = (v, w) goes to slot v % 4 of
// entry (block of v, w) and, for v != w, to slot w % 4 of entry (block of w, v);
// slot[p] = (4 e1 + i1, 4 e2 + i2 or -1)
template <typename T>
__global__ void scatter_tau4_kernel(int nb, const cplx<T>* __restrict__ grids, long n3, long p0,
                                    const int2* __restrict__ slot, long n_ent, T* __restrict__ tau4) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long c = blockIdx.y;
  if (r >= n3) return;
  const cplx<T> F = grids[c * n3 + r];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (2 * c + q >= nb) break;
    const T val = q ? F.y : F.x;
    const int2 s = slot[p0 + 2 * c + q];
    tau4[tau4_off(s.x >> 2, r, n_ent) + (s.x & 3)] = val;
    if (s.y >= 0) tau4[tau4_off(s.y >> 2, r, n_ent) + (s.y & 3)] = val;
  }
}

template <typename T>
cudaError_t scatter_tau4(int nb, const cplx<T>* grids, long n3, long p0, const int2* slot, long n_ent, T* tau4,
                         cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  if (n3 % TAU_TB) return cudaErrorInvalidValue;
  dim3 grid(nblk(n3), (nb + 1) / 2);
  scatter_tau4_kernel<T><<<grid, 256, 0, st>>>(nb, grids, n3, p0, slot, n_ent, tau4); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// overlap (Eq. overlap): |psi_v|^2 on the grid, Gram by GEMM, then normalisation
// ---------------------------------------------------------------------------------
// |psi_v(r)|^2 in FP64, stored as the FP32 split hi = fp32(x), lo = fp32(x - hi)
__global__ void square_fields_split_kernel(int n, const double* __restrict__ u, long n3,
                                           float* __restrict__ hi, float* __restrict__ lo) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n3) return;
  const long v = idx / n3, r = idx - v * n3;
  const double x = u[pair_off<double>(v, r, n3)];
  const double rho = x * x;
  const float h = (float)rho;
  hi[idx] = h;
  lo[idx] = (float)(rho - (double)h);
}
cudaError_t square_fields_split(int n, const double* u, long n3, float* rho_hi, float* rho_lo, cudaStream_t st) {
  const long tot = (long)n * n3;
  if (!tot) return cudaSuccess;
  square_fields_split_kernel<<<nblk(tot), 256, 0, st>>>(n, u, n3, rho_hi, rho_lo); note_launch();
  return cudaGetLastError();
}

__global__ void overlap_diag_kernel(int n, const double* g, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = g[(long)i * n + i];
}
__global__ void normalize_overlap_kernel(int n, double* g, const double* d) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (long)i * n);
  g[idx] = (i == j) ? 1.0 : g[idx] / sqrt(d[i] * d[j]);
}
// O_vw = Gram_vw / sqrt(Gram_vv Gram_ww); the diagonal becomes exactly 1
cudaError_t normalize_overlap(int n, double* gram, double* diag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  overlap_diag_kernel<<<nblk(n), 256, 0, st>>>(n, gram, diag); note_launch();
  normalize_overlap_kernel<<<nblk((long)n * n), 256, 0, st>>>(n, gram, diag); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Hartree pair density of Eq. (k1e): h_s(r) = sum_w u_psi_w(r) u_a_sw(r)
// ---------------------------------------------------------------------------------
template <typename T, int SV>
__global__ void hartree_density_kernel(int n_vec, int n_occ, long n3, const T* __restrict__ a,
                                       const T* __restrict__ upsi, T* __restrict__ h) {
  // SV vectors per thread, so each psi_w(r) is read once per SV vectors
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s0 = blockIdx.y * SV;
  if (r >= n3) return;
  const int ns = min(SV, n_vec - s0);
  T acc[SV];
#pragma unroll
  for (int q = 0; q < SV; ++q) acc[q] = 0;
  for (int w = 0; w < n_occ; ++w) {
    const T u = upsi[pair_off<T>(w, r, n3)];
#pragma unroll
    for (int q = 0; q < SV; ++q)
      if (q < ns) acc[q] += u * a[pair_off<T>((long)(s0 + q) * n_occ + w, r, n3)];
  }
#pragma unroll
  for (int q = 0; q < SV; ++q)
    if (q < ns) h[pair_off<T>(s0 + q, r, n3)] = acc[q];
}
template <typename T>
cudaError_t hartree_density(int n_vec, int n_occ, long n3, const T* a, const T* upsi, T* h,
                            cudaStream_t st) {
  if (!n_vec) return cudaSuccess;
  constexpr int SV = 8;
  dim3 grid(nblk(n3), (n_vec + SV - 1) / SV);
  hartree_density_kernel<T, SV><<<grid, 256, 0, st>>>(n_vec, n_occ, n3, a, upsi, h); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// screened direct term (Eq. k1d) fused with the real-space part of D (Eq. d) and
// K1e (Eq. k1e):
//   u_R,sv(r) = V_loc(r) u_a,sv(r) + s V_H,s(r) u_psi,v(r) - sum_{w in nbr(v)} tau_vw(r) u_a,sw(r)
// ---------------------------------------------------------------------------------
template <typename T, int SCH>
__global__ void __launch_bounds__(256) k1d_combine_kernel(
    int n_vec, int n_occ, long n3, const T* __restrict__ a, const T* __restrict__ tau, long n_pairs,
    const int* __restrict__ nbr_ptr, const int* __restrict__ nbr_w, const int* __restrict__ nbr_p,
    const T* __restrict__ vloc, const T* __restrict__ vh, const T* __restrict__ upsi, T sf,
    T* __restrict__ out) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n3) return;
  const int v = blockIdx.y;
  const int s0 = blockIdx.z * SCH;
  T acc[SCH];
#pragma unroll
  for (int j = 0; j < SCH; ++j) acc[j] = 0;
  const int e0 = nbr_ptr[v], e1 = nbr_ptr[v + 1];
  for (int e = e0; e < e1; ++e) {
    const int w = nbr_w[e];
    const T t = tau[tau_off(nbr_p[e], r, n_pairs)];
#pragma unroll
    for (int j = 0; j < SCH; ++j) {
      const int s = s0 + j;
      if (s < n_vec) acc[j] += t * a[pair_off<T>((long)s * n_occ + w, r, n3)];
    }
  }
  const T vl = vloc[r];
  const T up = upsi[pair_off<T>(v, r, n3)];
#pragma unroll
  for (int j = 0; j < SCH; ++j) {
    const int s = s0 + j;
    if (s >= n_vec) break;
    const long f = (long)s * n_occ + v;
    out[pair_off<T>(f, r, n3)] = vl * a[pair_off<T>(f, r, n3)] + sf * vh[pair_off<T>(s, r, n3)] * up - acc[j];
  }
}

template <typename T>
cudaError_t k1d_combine(int n_vec, int n_occ, long n3, const T* a, const T* tau, long n_pairs, const int* nbr_ptr,
                        const int* nbr_w, const int* nbr_p, const T* vloc, const T* vh,
                        const T* upsi, double spin_factor, T* out, cudaStream_t st) {
  constexpr int SCH = 8;
  if (!n_vec) return cudaSuccess;
  dim3 grid(nblk(n3), n_occ, (n_vec + SCH - 1) / SCH);
  k1d_combine_kernel<T, SCH><<<grid, 256, 0, st>>>(n_vec, n_occ, n3, a, tau, n_pairs, nbr_ptr, nbr_w, nbr_p,
                                                   vloc, vh, upsi, (T)spin_factor, out); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void scale_columns_kernel(int rows, int cols, T* C, long ldc, const double* f) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)rows * cols) return;
  const long i = idx / cols, j = idx - i * cols;
  C[i * ldc + j] = (T)((double)C[i * ldc + j] * f[j]);
}
template <typename T>
cudaError_t scale_columns(int rows, int cols, T* C, long ldc, const double* f, cudaStream_t st) {
  const long tot = (long)rows * cols;
  if (!tot) return cudaSuccess;
  scale_columns_kernel<T><<<nblk(tot), 256, 0, st>>>(rows, cols, C, ldc, f); note_launch();
  return cudaGetLastError();
}

template <typename TI, typename TO>
__global__ void convert_kernel(long n, const TI* in, TO* out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (TO)in[i];
}
template <typename TI, typename TO>
cudaError_t convert(long n, const TI* in, TO* out, cudaStream_t st) {
  if (!n) return cudaSuccess;
  convert_kernel<TI, TO><<<nblk(n), 256, 0, st>>>(n, in, out); note_launch();
  return cudaGetLastError();
}

// real fields of a pair-layout buffer -> rows [n][n3]
template <typename T>
__global__ void pair_grid_to_rows_kernel(int n, const T* g, long n3, T* rows) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n3) return;
  const long f = idx / n3, r = idx - f * n3;
  rows[idx] = g[pair_off<T>(f, r, n3)];
}
template <typename T>
cudaError_t pair_grid_to_rows(int n, const T* grids, long n3, T* rows, cudaStream_t st) {
  const long tot = (long)n * n3;
  if (!tot) return cudaSuccess;
  pair_grid_to_rows_kernel<T><<<nblk(tot), 256, 0, st>>>(n, grids, n3, rows); note_launch();
  return cudaGetLastError();
}

// block reduction of doubles
__device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();   // previous users of sh are done
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[lane] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-thread sum of squares with the accuracy of double precision. For single precision
// the square is split exactly into p + e (e = fma(x, x, -p)) and p is added with an
// error-free two-sum whose rounding error joins e in a compensation term, so the work stays
// in FP32 instructions (FP64 runs at a small fraction of the FP32 rate on this part). The
// rounding-mode intrinsics keep the compiler from contracting the sums into FMAs.
template <typename T>
struct SqSum {
  double s = 0.0;
  __device__ __forceinline__ void add(T x) { s = fma((double)x, (double)x, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct SqSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    c = __fadd_rn(c, __fadd_rn(err, e));
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// R_i = LX_i - theta_i X_i (data precision) and ||R_i||^2 to double accuracy
template <typename T>
__global__ void residual_kernel(long dim, const T* X, const T* LX, const double* theta, T* R,
                                double* norms2) {
  __shared__ double sh[32];
  const int i = blockIdx.y;
  const T th = (T)theta[i];
  SqSum<T> acc;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < dim; e += (long)gridDim.x * blockDim.x) {
    const T r = fma(-th, X[i * dim + e], LX[i * dim + e]);
    R[i * dim + e] = r;
    acc.add(r);
  }
  const double tot = block_sum(acc.get(), sh);
  if (threadIdx.x == 0) atomicAdd(norms2 + i, tot);
}
template <typename T>
cudaError_t residuals(int k, long dim, const T* X, const T* LX, const double* theta, T* R,
                      double* norms2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(norms2, 0, sizeof(double) * k, st);
  if (e != cudaSuccess) return e;
  long nb = (dim + 255) / 256;
  if (nb > 592) nb = 592;
  dim3 grid((unsigned)nb, k);
  residual_kernel<T><<<grid, 256, 0, st>>>(dim, X, LX, theta, R, norms2); note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void row_norms2_kernel(long dim, const T* X, double* norms2) {
  __shared__ double sh[32];
  const int i = blockIdx.y;
  SqSum<T> acc;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < dim; e += (long)gridDim.x * blockDim.x)
    acc.add(X[i * dim + e]);
  const double tot = block_sum(acc.get(), sh);
  if (threadIdx.x == 0) atomicAdd(norms2 + i, tot);
}
template <typename T>
cudaError_t row_norms2(int k, long dim, const T* X, double* norms2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(norms2, 0, sizeof(double) * k, st);
  if (e != cudaSuccess || !k) return e;
  long nb = (dim + 255) / 256;
  if (nb > 592) nb = 592;
  dim3 grid((unsigned)nb, k);
  row_norms2_kernel<T><<<grid, 256, 0, st>>>(dim, X, norms2); note_launch();
  return cudaGetLastError();
}

// diagonal preconditioner t = r / max(d - theta, 0.1 Ha), d = 1/2|G|^2 + V(0) + Delta - eps_v.
// The positive floor keeps the preconditioner positive definite: where d < theta the
// diagonal carries no information about L - theta. The pad coordinate is set to 0.
template <typename T>
__global__ void precond_diag_kernel(int n_occ, int n_pw, const T* R, const double* theta,
                                    const int* which, const T* g2h, const double* eps,
                                    double v0, double shift, T* out) {
  // one CTA per (orbital row v, corrected vector t): d - theta = 1/2|G|^2 + (V(0) + Delta -
  // eps_v - theta), the bracket one value per row
  const long dim = (long)n_occ * n_pw;
  const int v = blockIdx.x, t = blockIdx.y;
  const int i = which[t];
  const T cs = (T)(v0 + shift - eps[v] - theta[i]);
  const T* r = R + (long)i * dim + (long)v * n_pw;
  T* o = out + (long)t * dim + (long)v * n_pw;
  for (int j = threadIdx.x; j < n_pw; j += blockDim.x) {
    T den = g2h[j] + cs;
    if (den < (T)0.1) den = (T)0.1;
    T val;
    if constexpr (sizeof(T) == 4) val = __fdividef(r[j], den);   // a preconditioner: fast division
    else val = r[j] / den;
    o[j] = (j == 1) ? (T)0 : val;
  }
}
template <typename T>
cudaError_t precond_diag(int k, int n_occ, int n_pw, const T* R, const double* theta,
                         const int* which, const T* g2h, const double* eps, double v0,
                         double shift, T* out, cudaStream_t st) {
  if (!k) return cudaSuccess;
  dim3 grid(n_occ, k);
  precond_diag_kernel<T><<<grid, 256, 0, st>>>(n_occ, n_pw, R, theta, which, g2h, eps, v0, shift, out); note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void zero_pad_kernel(int rows, int n_pw, T* X) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) X[i * n_pw + 1] = (T)0;
}
template <typename T>
cudaError_t zero_pad_column(int rows, int n_pw, T* X, cudaStream_t st) {
  if (!rows) return cudaSuccess;
  zero_pad_kernel<T><<<nblk(rows), 256, 0, st>>>(rows, n_pw, X); note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void scale_rows_kernel(long dim, T* X, const double* s) {
  const int i = blockIdx.y;
  const T f = (T)s[i];
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < dim; e += (long)gridDim.x * blockDim.x)
    X[i * dim + e] *= f;
}
template <typename T>
cudaError_t scale_rows(int k, long dim, T* X, const double* s, cudaStream_t st) {
  if (!k) return cudaSuccess;
  long nb = (dim + 255) / 256;
  if (nb > 1184) nb = 1184;
  dim3 grid((unsigned)nb, k);
  scale_rows_kernel<T><<<grid, 256, 0, st>>>(dim, X, s); note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void set_unit_kernel(T* x, long idx) { x[idx] = (T)1; }
template <typename T>
cudaError_t set_unit(T* x, long dim, long idx, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(x, 0, sizeof(T) * dim, st);
  if (e != cudaSuccess) return e;
  set_unit_kernel<T><<<1, 1, 0, st>>>(x, idx); note_launch();
  return cudaGetLastError();
}

__global__ void symmetrize_kernel(int m, double* A, long lda) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)m * m) return;
  const int i = (int)(idx / m), j = (int)(idx - (long)i * m);
  if (j <= i) return;
  const double v = 0.5 * (A[(long)i * lda + j] + A[(long)j * lda + i]);
  A[(long)i * lda + j] = v;
  A[(long)j * lda + i] = v;
}
// after columns [m0, m1) of the upper block were computed: copy them to the rows,
// averaging inside the new diagonal block
__global__ void mirror_new_kernel(double* A, long lda, int m0, int m1) {
  const int nn = m1 - m0;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)m1 * nn) return;
  const int i = (int)(idx / nn), j = m0 + (int)(idx - (long)i * nn);
  if (i < m0) {
    A[(long)j * lda + i] = A[(long)i * lda + j];
  } else if (i < j) {
    const double v = 0.5 * (A[(long)i * lda + j] + A[(long)j * lda + i]);
    A[(long)i * lda + j] = v;
    A[(long)j * lda + i] = v;
  }
}
cudaError_t mirror_new(double* A, long lda, int m0, int m1, cudaStream_t st) {
  const long tot = (long)m1 * (m1 - m0);
  if (tot <= 0) return cudaSuccess;
  mirror_new_kernel<<<nblk(tot), 256, 0, st>>>(A, lda, m0, m1); note_launch();
  return cudaGetLastError();
}

cudaError_t symmetrize(int m, double* A, long lda, cudaStream_t st) {
  const long tot = (long)m * m;
  if (!tot) return cudaSuccess;
  symmetrize_kernel<<<nblk(tot), 256, 0, st>>>(m, A, lda); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Cholesky S = L L^T (b x b, FP64) and Linv = L^{-1} (lower), one CTA.
// info[0] = 0 on success, j+1 if the j-th pivot is not positive and finite.
// ---------------------------------------------------------------------------------
constexpr int CHOL_MAX = 128;
__global__ void __launch_bounds__(256) cholesky_kernel(int b, const double* __restrict__ S, long lds,
                                                      double* __restrict__ Linv, int* info) {
  extern __shared__ __align__(16) double csm[];
  const int ld = b + 1;
  double* A = csm;
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long e = tid; e < (long)b * b; e += nt) {
    const int i = (int)(e / b), j = (int)(e - (long)i * b);
    A[i * ld + j] = S[(long)i * lds + j];
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const double d = A[j * ld + j];
      if (!(d > 0.0) || !isfinite(d)) { if (!bad) bad = j + 1; A[j * ld + j] = 1.0; }
      else A[j * ld + j] = sqrt(d);
    }
    __syncthreads();
    const double djj = A[j * ld + j];
    for (int i = j + 1 + tid; i < b; i += nt) A[i * ld + j] /= djj;
    __syncthreads();
    for (long e = tid; e < (long)(b - j - 1) * (b - j - 1); e += nt) {
      const int i = j + 1 + (int)(e / (b - j - 1)), k = j + 1 + (int)(e % (b - j - 1));
      if (k <= i) A[i * ld + k] -= A[i * ld + j] * A[k * ld + j];
    }
    __syncthreads();
  }
  // Linv column c by forward substitution
  for (int c = tid; c < b; c += nt) {
    for (int i = 0; i < b; ++i) {
      double x;
      if (i < c) x = 0.0;
      else {
        double sacc = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) sacc -= A[i * ld + k] * Linv[(long)k * b + c];
        x = sacc / A[i * ld + i];
      }
      Linv[(long)i * b + c] = x;
    }
  }
  if (tid == 0) info[0] = bad;
}

cudaError_t cholesky_inverse(int b, const double* S, long lds, double* Linv, int* info,
                             cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  if (b > CHOL_MAX) return cudaErrorInvalidValue;
  const size_t smem = (size_t)b * (b + 1) * sizeof(double);
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)CHOL_MAX * (CHOL_MAX + 1) * 8));
  });
  if (e0 != cudaSuccess) return e0;
  cholesky_kernel<<<1, 256, smem, st>>>(b, S, lds, Linv, info); note_launch();
  return cudaGetLastError();
}

bool finite_check_host(const double* x, long n) {
  for (long i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

// ---------------------------------------------------------------------------------
// P_c of a spin-polarised system (one projector per channel): the coefficients <psi_w|x_row>
// of a row whose orbital (row % n_occ) lies in the other channel than w are cleared
template <typename T>
__global__ void mask_cross_channel_kernel(int rows, int n_occ, int n_up, T* C) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)rows * n_occ) return;
  const int w = (int)(idx % n_occ);
  const int v = (int)((idx / n_occ) % n_occ);
  if ((v >= n_up) != (w >= n_up)) C[idx] = (T)0;
}
template <typename T>
cudaError_t mask_cross_channel(int rows, int n_occ, int n_up, T* C, cudaStream_t st) {
  const long tot = (long)rows * n_occ;
  if (tot <= 0) return cudaSuccess;
  mask_cross_channel_kernel<T><<<nblk(tot), 256, 0, st>>>(rows, n_occ, n_up, C); note_launch();
  return cudaGetLastError();
}
template cudaError_t mask_cross_channel<float>(int, int, int, float*, cudaStream_t);
template cudaError_t mask_cross_channel<double>(int, int, int, double*, cudaStream_t);

// explicit instantiations
// ---------------------------------------------------------------------------------
#define INST_T(T)                                                                                  \
  template cudaError_t pair_product<T>(int, const int*, const int*, const T*, long, double,        \
                                       cplx<T>*, cudaStream_t);                                    \
  template cudaError_t deinterleave_pairs<T>(int, const cplx<T>*, long, long, long, T*, cudaStream_t);       \
  template cudaError_t scatter_tau4<T>(int, const cplx<T>*, long, long, const int2*, long, T*, cudaStream_t); \
  template cudaError_t hartree_density<T>(int, int, long, const T*, const T*, T*, cudaStream_t);   \
  template cudaError_t k1d_combine<T>(int, int, long, const T*, const T*, long, const int*, const int*,   \
                                      const int*, const T*, const T*, const T*, double, T*,        \
                                      cudaStream_t);                                               \
  template cudaError_t scale_columns<T>(int, int, T*, long, const double*, cudaStream_t);          \
  template cudaError_t pair_grid_to_rows<T>(int, const T*, long, T*, cudaStream_t);                \
  template cudaError_t residuals<T>(int, long, const T*, const T*, const double*, T*, double*,     \
                                    cudaStream_t);                                                 \
  template cudaError_t row_norms2<T>(int, long, const T*, double*, cudaStream_t);                  \
  template cudaError_t precond_diag<T>(int, int, int, const T*, const double*, const int*,         \
                                       const T*, const double*, double, double, T*,                \
                                       cudaStream_t);                                              \
  template cudaError_t zero_pad_column<T>(int, int, T*, cudaStream_t);                             \
  template cudaError_t scale_rows<T>(int, long, T*, const double*, cudaStream_t);                  \
  template cudaError_t set_unit<T>(T*, long, long, cudaStream_t);
INST_T(float)
INST_T(double)
template cudaError_t convert<double, float>(long, const double*, float*, cudaStream_t);
template cudaError_t convert<float, double>(long, const float*, double*, cudaStream_t);
template cudaError_t convert<double, double>(long, const double*, double*, cudaStream_t);
template cudaError_t convert<float, float>(long, const float*, float*, cudaStream_t);

}  // namespace bse
