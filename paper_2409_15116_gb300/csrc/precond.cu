// Learned Davidson preconditioner (a library addition: the paper's Davidson of Section 3
// uses no learned component): a per-element MLP 5 -> 64 -> 64 -> 1 that rescales the
// diagonal step,
//
//   x = (f - mu)/sigma,  f = (1/2|G|^2, eps_v, theta, d - theta, r_e sqrt(dim)/||r||),
//   h1 = act(relu(W1 x + b1)),  h2 = act(relu(W2 h1 + b2)),  o = w3 . h2 + b3,
//   g = exp(clip(o, -8, 8)) / max(d - theta, 0.1),   t = g r  (then P_c by the caller),
//
// with d = 1/2|G|^2 + V(0) + Delta - eps_v and act = bfloat16 rounding (FP32 weights,
// BF16 activations) or the identity. A zero last layer is exactly the diagonal
// preconditioner. Training kernels compute the activations, the loss gradient in g and
// the per-row back-propagation; the weight gradients are reductions over rows done as
// GEMMs. Parameter layout (float): W1[64x5] b1[64] W2[64x64] b2[64] w3[64] b3 mu[5] sigma[5].
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include "common.cuh"
#include "kernels.h"

namespace bse {

constexpr int MH = 64, MF = 5;
constexpr int P_W1 = 0, P_B1 = P_W1 + MH * MF, P_W2 = P_B1 + MH, P_B2 = P_W2 + MH * MH,
              P_W3 = P_B2 + MH, P_B3 = P_W3 + MH, P_MU = P_B3 + 1, P_SG = P_MU + MF,
              P_N = P_SG + MF;
static_assert(P_N == 4619, "parameter count");

__device__ __forceinline__ float act_round(float x, int bf) {
  return bf ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// features of element (v, j) of a residual with Ritz value th and norm rn (dim = n_occ*n_pw)
__device__ __forceinline__ void mlp_features(const float* P, double g2, double epsv, double v0,
                                             double shift, double th, double re, double rn,
                                             double dim, float* x, double* den) {
  const double d = 0.5 * g2 + v0 + shift - epsv;
  const double f[MF] = {0.5 * g2, epsv, th, d - th, rn > 0 ? re * sqrt(dim) / rn : 0.0};
#pragma unroll
  for (int k = 0; k < MF; ++k) x[k] = (float)((f[k] - (double)P[P_MU + k]) / (double)P[P_SG + k]);
  *den = fmax(d - th, 0.1);
}

// forward pass of one element; returns o (pre-clip); h1, h2 optional outputs
__device__ __forceinline__ float mlp_forward_row(const float* P, const float* x, int bf, float* h1,
                                                 float* h2) {
  float a1[MH];
#pragma unroll 8
  for (int k = 0; k < MH; ++k) {
    float z = P[P_B1 + k];
#pragma unroll
    for (int i = 0; i < MF; ++i) z = fmaf(P[P_W1 + k * MF + i], x[i], z);
    a1[k] = act_round(fmaxf(z, 0.f), bf);
    if (h1) h1[k] = a1[k];
  }
  float o = P[P_B3];
  for (int k = 0; k < MH; ++k) {
    float z = P[P_B2 + k];
#pragma unroll 8
    for (int j = 0; j < MH; ++j) z = fmaf(P[P_W2 + k * MH + j], a1[j], z);
    const float a2 = act_round(fmaxf(z, 0.f), bf);
    if (h2) h2[k] = a2;
    o = fmaf(P[P_W3 + k], a2, o);
  }
  return o;
}

// ---------------------------------------------------------------------------------
// inference inside Davidson: out[t] = g * R[which[t]]  (pad coordinate 0)
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) precond_learned_kernel(
    const float* __restrict__ params, int n_occ, int n_pw, const T* __restrict__ R,
    const double* __restrict__ theta, const double* __restrict__ rnorm2, const int* __restrict__ which,
    const double* __restrict__ g2p, const double* __restrict__ eps, double v0, double shift, T* out,
    int* bad) {
  __shared__ float P[P_N];
  for (int i = threadIdx.x; i < P_N; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const long dim = (long)n_occ * n_pw;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y, t = blockIdx.z;
  if (j >= n_pw) return;
  const int i = which[t];
  const long e = (long)v * n_pw + j;
  const double re = (double)R[(long)i * dim + e];
  float x[MF];
  double den;
  mlp_features(P, g2p[j], eps[v], v0, shift, theta[i], re, sqrt(rnorm2[i]), (double)dim, x, &den);
  const float o = mlp_forward_row(P, x, 1, nullptr, nullptr);
  const double g = exp((double)fminf(fmaxf(o, -8.f), 8.f)) / den;
  const double val = g * re;
  if (!isfinite(val)) atomicExch(bad, 1);
  out[t * dim + e] = (j == 1) ? (T)0 : (T)val;
}

template <typename T>
cudaError_t precond_learned(int k, int n_occ, int n_pw, const float* params, const T* R,
                            const double* theta, const double* rnorm2, const int* which,
                            const double* g2p, const double* eps, double v0, double shift, T* out,
                            int* bad, cudaStream_t st) {
  if (!k) return cudaSuccess;
  dim3 grid((n_pw + 255) / 256, n_occ, k);
  precond_learned_kernel<T><<<grid, 256, 0, st>>>(params, n_occ, n_pw, R, theta, rnorm2, which, g2p,
                                                  eps, v0, shift, out, bad);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t precond_learned<float>(int, int, int, const float*, const float*, const double*, const double*, const int*, const double*, const double*, double, double, float*, int*, cudaStream_t);
template cudaError_t precond_learned<double>(int, int, int, const float*, const double*, const double*, const double*, const int*, const double*, const double*, double, double, double*, int*, cudaStream_t);

// ---------------------------------------------------------------------------------
// training: rows are (sample s, orbital v, packed index j), s over ns samples
// ---------------------------------------------------------------------------------
// forward: X [rows x 5], H1 [rows x 64], H2 [rows x 64], O [rows], Y = g * r [rows] (double)
__global__ void __launch_bounds__(128) mlp_train_forward_kernel(
    const float* __restrict__ params, long rows, int n_occ, int n_pw, const double* __restrict__ r,
    const double* __restrict__ theta, const double* __restrict__ rnorm2, const double* __restrict__ g2p,
    const double* __restrict__ eps, double v0, double shift, int bf, float* __restrict__ X,
    float* __restrict__ H1, float* __restrict__ H2, float* __restrict__ O, double* __restrict__ G,
    double* __restrict__ Y) {
  __shared__ float P[P_N];
  for (int i = threadIdx.x; i < P_N; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const long dim = (long)n_occ * n_pw;
  const long s = row / dim;
  const int e = (int)(row - s * dim);
  const int v = e / n_pw, j = e - v * n_pw;
  const double re = r[row];
  float x[MF];
  double den;
  mlp_features(P, g2p[j], eps[v], v0, shift, theta[s], re, sqrt(rnorm2[s]), (double)dim, x, &den);
#pragma unroll
  for (int k = 0; k < MF; ++k) X[row * MF + k] = x[k];
  const float o = mlp_forward_row(P, x, bf, H1 + row * MH, H2 + row * MH);
  O[row] = o;
  const double g = (j == 1) ? 0.0 : exp((double)fminf(fmaxf(o, -8.f), 8.f)) / den;
  G[row] = g;
  Y[row] = g * re;
}

// scale-free misfit: with y = P_c(g r), a = <y,t*>, b = |y|^2, c = |t*|^2 per sample,
// loss_s = 1 - a^2/(b c) and dg = r (2 a^2/(b^2 c) y - 2 a/(b c) t*), both times inv_n
__global__ void mlp_loss_kernel(long rows, long dim, const double* __restrict__ py,
                                const double* __restrict__ tstar, const double* __restrict__ tn2,
                                const double* __restrict__ ab, const double* __restrict__ r,
                                double inv_n, double* __restrict__ dg, double* __restrict__ loss) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const long s = row / dim;
  const double a = ab[2 * s], b = ab[2 * s + 1], c = tn2[s];
  dg[row] = r[row] * (2.0 * a * a / (b * b * c) * py[row] - 2.0 * a / (b * c) * tstar[row]) * inv_n;
  if (row - s * dim == 0) atomicAdd(loss, (1.0 - a * a / (b * c)) * inv_n);
}

// backward per row: DO [rows], DZ1 [rows x 64], DZ2 [rows x 64]
__global__ void __launch_bounds__(128) mlp_train_backward_kernel(
    const float* __restrict__ params, long rows, const float* __restrict__ H1,
    const float* __restrict__ H2, const float* __restrict__ O, const double* __restrict__ G,
    const double* __restrict__ dg, float* __restrict__ DO, float* __restrict__ DZ1,
    float* __restrict__ DZ2) {
  __shared__ float P[P_N];
  for (int i = threadIdx.x; i < P_N; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const float o = O[row];
  const float dov = (o > -8.f && o < 8.f) ? (float)(dg[row] * G[row]) : 0.f;
  DO[row] = dov;
  float dz2[MH];
#pragma unroll 8
  for (int k = 0; k < MH; ++k) {
    dz2[k] = (H2[row * MH + k] > 0.f) ? dov * P[P_W3 + k] : 0.f;
    DZ2[row * MH + k] = dz2[k];
  }
  for (int jj = 0; jj < MH; ++jj) {
    float a = 0.f;
#pragma unroll 8
    for (int k = 0; k < MH; ++k) a = fmaf(P[P_W2 + k * MH + jj], dz2[k], a);
    DZ1[row * MH + jj] = (H1[row * MH + jj] > 0.f) ? a : 0.f;
  }
}

// Adam on float parameters with double gradients; indices >= n_train are left untouched
__global__ void adam_kernel(int n_train, float* p, const double* g, float* m, float* v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_train) return;
  const float gi = (float)g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi; v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// sums of the features and their squares (for mu, sigma)
__global__ void feature_moments_kernel(long rows, const float* __restrict__ Xraw_unused, int n_occ,
                                       int n_pw, const double* __restrict__ r,
                                       const double* __restrict__ theta, const double* __restrict__ rnorm2,
                                       const double* __restrict__ g2p, const double* __restrict__ eps,
                                       double v0, double shift, double* __restrict__ mom) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double f[MF] = {0, 0, 0, 0, 0};
  if (row < rows) {
    const long dim = (long)n_occ * n_pw;
    const long s = row / dim;
    const int e = (int)(row - s * dim);
    const int v = e / n_pw, j = e - v * n_pw;
    const double d = 0.5 * g2p[j] + v0 + shift - eps[v];
    const double rn = sqrt(rnorm2[s]);
    f[0] = 0.5 * g2p[j]; f[1] = eps[v]; f[2] = theta[s]; f[3] = d - theta[s];
    f[4] = rn > 0 ? r[row] * sqrt((double)dim) / rn : 0.0;
  }
  for (int k = 0; k < MF; ++k) {
    double a = f[k], b = f[k] * f[k];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(mom + k, a); atomicAdd(mom + MF + k, b); }
  }
}

// t* = y / (u . y) - u  per sample row block (y = shifted-inverse image of the Ritz vector u)
__global__ void jd_target_kernel(long dim, const double* __restrict__ Y, const double* __restrict__ U,
                                 const double* __restrict__ uy, double* __restrict__ T) {
  const int s = blockIdx.y;
  const double a = uy[s];
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < dim; e += (long)gridDim.x * blockDim.x)
    T[s * dim + e] = Y[s * dim + e] / a - U[s * dim + e];
}
// C[s][j] /= (lambda_j - theta_s), guarded away from zero
__global__ void shift_scale_kernel(int ns, int nr, double* C, const double* lam, const double* th) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * nr) return;
  const int s = idx / nr, j = idx - s * nr;
  double den = lam[j] - th[s];
  if (fabs(den) < 1e-10) den = den >= 0 ? 1e-10 : -1e-10;
  C[idx] /= den;
}
__global__ void row_dots_kernel(long dim, const double* A, const double* B, double* out) {
  __shared__ double red[32];
  const int s = blockIdx.y;
  double acc = 0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < dim; e += (long)gridDim.x * blockDim.x)
    acc += A[s * dim + e] * B[s * dim + e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(out + s, t);
  }
}

// ---- launchers ----
static inline unsigned nb(long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t mlp_train_forward(const float* params, long rows, int n_occ, int n_pw, const double* r,
                              const double* theta, const double* rnorm2, const double* g2p,
                              const double* eps, double v0, double shift, int bf, float* X, float* H1,
                              float* H2, float* O, double* G, double* Y, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  mlp_train_forward_kernel<<<nb(rows, 128), 128, 0, st>>>(params, rows, n_occ, n_pw, r, theta, rnorm2,
                                                          g2p, eps, v0, shift, bf, X, H1, H2, O, G, Y);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_loss(long rows, long dim, const double* py, const double* tstar, const double* tn2,
                     const double* ab, const double* r, double inv_n, double* dg, double* loss,
                     cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  mlp_loss_kernel<<<nb(rows, 256), 256, 0, st>>>(rows, dim, py, tstar, tn2, ab, r, inv_n, dg, loss);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_train_backward(const float* params, long rows, const float* H1, const float* H2,
                               const float* O, const double* G, const double* dg, float* DO,
                               float* DZ1, float* DZ2, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  mlp_train_backward_kernel<<<nb(rows, 128), 128, 0, st>>>(params, rows, H1, H2, O, G, dg, DO, DZ1, DZ2);
  note_launch();
  return cudaGetLastError();
}
cudaError_t adam_step(int n_train, float* p, const double* g, float* m, float* v, float lr, int step,
                      cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<nb(n_train, 256), 256, 0, st>>>(n_train, p, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
  note_launch();
  return cudaGetLastError();
}
cudaError_t feature_moments(long rows, int n_occ, int n_pw, const double* r, const double* theta,
                            const double* rnorm2, const double* g2p, const double* eps, double v0,
                            double shift, double* mom, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  feature_moments_kernel<<<nb(rows, 256), 256, 0, st>>>(rows, nullptr, n_occ, n_pw, r, theta, rnorm2,
                                                        g2p, eps, v0, shift, mom);
  note_launch();
  return cudaGetLastError();
}
cudaError_t jd_targets(int ns, long dim, const double* Y, const double* U, const double* uy, double* T,
                       cudaStream_t st) {
  if (ns <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<long>(nb(dim, 256), 1184), ns);
  jd_target_kernel<<<grid, 256, 0, st>>>(dim, Y, U, uy, T);
  note_launch();
  return cudaGetLastError();
}
cudaError_t shift_scale(int ns, int nr, double* C, const double* lam, const double* th, cudaStream_t st) {
  if (ns * nr <= 0) return cudaSuccess;
  shift_scale_kernel<<<nb((long)ns * nr, 256), 256, 0, st>>>(ns, nr, C, lam, th);
  note_launch();
  return cudaGetLastError();
}
cudaError_t row_dots(int ns, long dim, const double* A, const double* B, double* out, cudaStream_t st) {
  if (ns <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * ns, st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)std::min<long>(nb(dim, 256), 1184), ns);
  row_dots_kernel<<<grid, 256, 0, st>>>(dim, A, B, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bse
