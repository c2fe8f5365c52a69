// Symmetric eigensolver for the Davidson Rayleigh-Ritz matrix (m <= 160), one CTA,
// returning the k lowest eigenpairs. Input and outputs are double; the arithmetic runs
// in double (plain path) or in single precision (mixed path, whose matrix entries carry
// single-precision vector data: FP64 runs at a small fraction of the FP32 rate here,
// and the Sturm bisection is a long chain of dependent divisions).
//
//  1. Householder tridiagonalisation T = Q^T A Q in shared memory (reflector vectors kept
//     in the strictly lower part of A).
//  2. Each of the k lowest eigenvalues of T by bisection on the Sturm count of the
//     LDL^T recurrence (one thread per eigenvalue).
//  3. Eigenvectors of T by inverse iteration (tridiagonal elimination with partial
//     pivoting), re-orthogonalised against earlier members of the same cluster.
//  4. Back-transformation v = Q z with the stored reflectors.
#include "common.cuh"
#include "kernels.h"

namespace bse {

constexpr int EIGH_MAX = 160;
constexpr int EIGH_KMAX = 64;

template <typename R> struct EighTol;
template <> struct EighTol<double> { static constexpr double eps = 2.2e-16, tiny = 1e-300, pivtiny = 1e-290; };
template <> struct EighTol<float> { static constexpr float eps = 1.2e-7f, tiny = 1e-37f, pivtiny = 1e-35f; };

template <typename R>
__device__ __forceinline__ R blk_sum(R v, R* sh) {
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  R t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

// Sturm count: number of eigenvalues of T (diag d, off-diagonal e) strictly below x
template <typename R>
__device__ int sturm_count(int m, const R* d, const R* e2, R x, R pivmin) {
  int cnt = 0;
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Z (eigenvectors of T, vector j at Z + j * zld) and S (elimination factors, 3 m per
// vector at S + j * sld) live in shared memory after the matrix when they fit, else in the
// global work buffer; the odd strides keep one-thread-per-vector loops free of bank
// conflicts.
template <typename R>
__global__ void __launch_bounds__(512) eigh_lowest_kernel(int m, int k, const double* __restrict__ Ain,
                                                         long lda, R* __restrict__ Zg,
                                                         R* __restrict__ Sg, int in_smem,
                                                         double* __restrict__ V,
                                                         double* __restrict__ w, int* info) {
  using Tol = EighTol<R>;
  extern __shared__ __align__(16) unsigned char eigh_smem[];
  const int ld = m + 1;
  R* A = reinterpret_cast<R*>(eigh_smem);   // m x (m+1)
  R* d = A + (long)m * ld;      // m
  R* e = d + m;                 // m
  R* e2 = e + m;                // m
  R* p = e2 + m;                // m
  R* lam = p + m;               // EIGH_KMAX
  const int zld = m | 1, sld = (3 * m) | 1;
  R* Z = in_smem ? lam + EIGH_KMAX : Zg;
  R* S = in_smem ? Z + (long)k * zld : Sg;
  __shared__ R red[32];
  __shared__ R dots[EIGH_KMAX];
  __shared__ R s_alpha, s_scale;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long x = tid; x < (long)m * m; x += nt) {
    const int i = (int)(x / m), j = (int)(x - (long)i * m);
    A[i * ld + j] = (R)Ain[(long)i * lda + j];
  }
  __syncthreads();
  // ---- 1. tridiagonalisation ----
  for (int c = 0; c + 2 < m; ++c) {
    const int n = m - c - 1;                      // length of the column below the diagonal
    R s2 = 0;
    for (int i = tid; i < n; i += nt) { const R x = A[(c + 1 + i) * ld + c]; s2 += x * x; }
    s2 = blk_sum(s2, red);
    if (tid == 0) {
      const R x0 = A[(c + 1) * ld + c];
      const R nrm = sqrt(s2);
      const R alpha = (x0 >= 0) ? -nrm : nrm;
      d[c] = A[c * ld + c];
      e[c] = (nrm == (R)0) ? (R)0 : alpha;
      // v = x - alpha e1, |v|^2 = s2 - 2 alpha x0 + alpha^2
      const R vn2 = s2 - (R)2 * alpha * x0 + alpha * alpha;
      s_alpha = alpha;
      s_scale = (nrm == (R)0 || vn2 <= (R)0) ? (R)0 : (R)1 / sqrt(vn2);
    }
    __syncthreads();
    const R sc = s_scale;
    // u = v / |v| stored in place of the column (zero reflector if sc == 0)
    for (int i = tid; i < n; i += nt) {
      const R x = A[(c + 1 + i) * ld + c];
      A[(c + 1 + i) * ld + c] = (i == 0 ? x - s_alpha : x) * sc;
    }
    __syncthreads();
    if (sc == (R)0) continue;
    // p = B u over the trailing block B = A[c+1:, c+1:] (symmetric, both halves valid):
    // one warp per row, lanes along the row, shuffle reduction
    {
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int i = wid; i < n; i += nw) {
        const R* row = A + (c + 1 + i) * ld + (c + 1);
        R acc = 0;
        for (int j = lane; j < n; j += 32) acc += row[j] * A[(c + 1 + j) * ld + c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) p[i] = acc;
      }
    }
    R kk = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) kk += A[(c + 1 + i) * ld + c] * p[i];
    kk = blk_sum(kk, red);
    // q = p - K u (kept in p), B -= 2 (u q^T + q u^T)
    for (int i = tid; i < n; i += nt) p[i] -= kk * A[(c + 1 + i) * ld + c];
    __syncthreads();
    {
      // rank-2 update, one warp per row (no per-element index division)
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int i = wid; i < n; i += nw) {
        const R ui = A[(c + 1 + i) * ld + c], pi = p[i];
        R* row = A + (c + 1 + i) * ld + (c + 1);
        for (int j = lane; j < n; j += 32) row[j] -= (R)2 * (ui * p[j] + pi * A[(c + 1 + j) * ld + c]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      d[m - 2] = A[(m - 2) * ld + (m - 2)];
      e[m - 2] = A[(m - 1) * ld + (m - 2)];
    }
    d[m - 1] = A[(m - 1) * ld + (m - 1)];
    e[m - 1] = (R)0;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) e2[i] = e[i] * e[i];
  __syncthreads();
  // ---- 2. bisection for the k lowest eigenvalues ----
  R gl = (R)1e30, gu = (R)-1e30, tnorm = 0;
  for (int i = 0; i < m; ++i) {
    const R r = (i > 0 ? fabs(e[i - 1]) : (R)0) + (i + 1 < m ? fabs(e[i]) : (R)0);
    gl = fmin(gl, d[i] - r);
    gu = fmax(gu, d[i] + r);
  }
  tnorm = fmax(fabs(gl), fabs(gu));
  const R pivmin = Tol::pivtiny + Tol::tiny * tnorm * tnorm;
  if constexpr (sizeof(R) == 4) {
    // multisection: warp w brackets eigenvalues j = w, w + nw, ...; its 32 lanes evaluate the
    // Sturm count at 32 interior points of the current bracket, which shrinks 33-fold a step
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int j = wid; j < k; j += nw) {
      R lo = gl - 50 * Tol::eps * tnorm - Tol::tiny, hi = gu + 50 * Tol::eps * tnorm + Tol::tiny;
      for (int it = 0; it < 64; ++it) {
        if (!(hi - lo > Tol::eps * fmax(fabs(lo), fabs(hi)) + Tol::tiny)) break;
        const R x = lo + (hi - lo) * (R)(lane + 1) / (R)33;
        const int cnt = sturm_count(m, d, e2, x, pivmin);
        const int q = __popc(__ballot_sync(0xffffffffu, cnt <= j));
        const R nlo = (q == 0) ? lo : lo + (hi - lo) * (R)q / (R)33;
        const R nhi = (q == 32) ? hi : lo + (hi - lo) * (R)(q + 1) / (R)33;
        if (!(nlo > lo || nhi < hi)) break;        // no progress at this precision
        lo = nlo; hi = nhi;
      }
      if (lane == 0) lam[j] = (R)0.5 * (lo + hi);
    }
  } else {
    // bisection, one thread per eigenvalue (FP64 runs at a small fraction of the FP32 rate,
    // so every Sturm evaluation counts)
    for (int j = tid; j < k; j += nt) {
      R lo = gl - 50 * Tol::eps * tnorm - Tol::tiny, hi = gu + 50 * Tol::eps * tnorm + Tol::tiny;
      for (int it = 0; it < 200 && hi - lo > Tol::eps * fmax(fabs(lo), fabs(hi)) + Tol::tiny; ++it) {
        const R mid = (R)0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(m, d, e2, mid, pivmin) > j) hi = mid; else lo = mid;
      }
      lam[j] = (R)0.5 * (lo + hi);
    }
  }
  __syncthreads();
  // ---- 3. inverse iteration, one thread per eigenvector (Z column-major, m x k) ----
  const R ortol = (R)1e-3 * tnorm;
  for (int j = tid; j < k; j += nt) {
    R* z = Z + (long)j * zld;
    // perturb the shift slightly inside clusters so the factorisation stays regular
    R mu = lam[j];
    for (int i = 0; i < j; ++i)
      if (fabs(lam[i] - mu) < 50 * Tol::eps * tnorm) mu = lam[i] + 50 * Tol::eps * tnorm * (j - i);
    for (int i = 0; i < m; ++i) z[i] = (R)1 / sqrt((R)m) * ((R)1 + (R)0.001 * ((i * 7 + j * 13) % 11));
    for (int pass = 0; pass < 3; ++pass) {
      // solve (T - mu I) y = z by elimination with partial pivoting; the upper factor has
      // up to two super-diagonals (u0 diag, u1, u2); y overwrites z
      R* u0 = S + (long)j * sld;
      R* u1 = u0 + m;
      R* u2 = u1 + m;
      R a0 = d[0] - mu, b0 = (m > 1) ? e[0] : (R)0, c0 = (R)0;
      R rhs = z[0];
      for (int i = 0; i + 1 < m; ++i) {
        const R sub = e[i];
        const R a1 = d[i + 1] - mu, b1 = (i + 2 < m) ? e[i + 1] : (R)0;
        R r1 = z[i + 1];
        if (fabs(sub) > fabs(a0)) {          // swap rows i and i+1
          const R f = a0 / sub;
          u0[i] = sub; u1[i] = a1; u2[i] = b1;
          z[i] = r1;
          const R na0 = b0 - f * a1, nb0 = c0 - f * b1;
          r1 = rhs - f * r1;
          a0 = na0; b0 = nb0; c0 = (R)0; rhs = r1;
        } else {
          if (a0 == (R)0) a0 = pivmin;
          const R f = sub / a0;
          u0[i] = a0; u1[i] = b0; u2[i] = c0;
          z[i] = rhs;
          a0 = a1 - f * b0; b0 = b1 - f * c0; c0 = (R)0; rhs = r1 - f * rhs;
        }
      }
      if (a0 == (R)0) a0 = pivmin;
      u0[m - 1] = a0;
      z[m - 1] = rhs;
      // back substitution
      for (int i = m - 1; i >= 0; --i) {
        R s = z[i];
        if (i + 1 < m) s -= u1[i] * z[i + 1];
        if (i + 2 < m) s -= u2[i] * z[i + 2];
        z[i] = s / u0[i];
      }
      R nn = 0;
      for (int i = 0; i < m; ++i) nn += z[i] * z[i];
      nn = (R)1 / sqrt(nn);
      for (int i = 0; i < m; ++i) z[i] *= nn;
    }
  }
  __syncthreads();
  // re-orthogonalise inside clusters (eigenvalues within ortol), in eigenvalue order: the
  // projections on all earlier members at once (one warp per member), twice
  {
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int j = 1; j < k; ++j) {
      bool any = false;
      for (int i = 0; i < j; ++i) any |= fabs(lam[j] - lam[i]) <= ortol;
      if (any) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int i = wid; i < j; i += nw) {
            R dt = 0;
            if (fabs(lam[j] - lam[i]) <= ortol)
              for (int r = lane; r < m; r += 32) dt += Z[(long)i * zld + r] * Z[(long)j * zld + r];
            for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
            if (lane == 0) dots[i] = dt;
          }
          __syncthreads();
          for (int r = tid; r < m; r += nt) {
            R acc = 0;
            for (int i = 0; i < j; ++i) acc += dots[i] * Z[(long)i * zld + r];
            Z[(long)j * zld + r] -= acc;
          }
          __syncthreads();
        }
      }
      R nn = 0;
      for (int r = tid; r < m; r += nt) nn += Z[(long)j * zld + r] * Z[(long)j * zld + r];
      nn = blk_sum(nn, red);
      const R inv = (R)1 / sqrt(nn);
      for (int r = tid; r < m; r += nt) Z[(long)j * zld + r] *= inv;
      __syncthreads();
    }
  }
  // ---- 4. back-transformation: v = H_0 H_1 ... H_{m-3} z, applied to all k vectors ----
  for (int c = m - 3; c >= 0; --c) {
    const int n = m - c - 1;
    // one warp per vector: dot = u . z[c+1:], z[c+1:] -= 2 dot u
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int j = wid; j < k; j += nw) {
      R* z = Z + (long)j * zld;
      R dot = 0;
      for (int i = lane; i < n; i += 32) dot += A[(c + 1 + i) * ld + c] * z[c + 1 + i];
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      for (int i = lane; i < n; i += 32) z[c + 1 + i] -= (R)2 * dot * A[(c + 1 + i) * ld + c];
    }
    __syncthreads();
  }
  // outputs: V row-major m x k (component r of eigenvector j at V[r*k + j]), w[0..k)
  for (long x = tid; x < (long)m * k; x += nt) {
    const int r = (int)(x / k), j = (int)(x - (long)r * k);
    V[x] = (double)Z[(long)j * zld + r];
  }
  for (int j = tid; j < k; j += nt) w[j] = (double)lam[j];
  if (tid == 0) info[0] = 0;
}

// k lowest eigenpairs of the symmetric m x m matrix A (lda): eigenvalues ascending in w[0..k),
// eigenvectors as the columns of V (row-major m x k). work: at least 4*m*k + 2*k doubles.
// single: single-precision Householder, bisection and inverse iteration, then the
// eigenvalues refined in double as Rayleigh quotients of the computed vectors against A
// (double input and outputs; the values come out accurate to double precision).
template <typename R>
static cudaError_t launch_eigh(int m, int k, const double* A, long lda, double* work, double* V, double* w,
                               int* info, cudaStream_t st) {
  constexpr size_t SMEM_MAX = 220 * 1024;
  const size_t base = ((size_t)m * (m + 1) + 4 * (size_t)m + EIGH_KMAX) * sizeof(R);
  const size_t extra = ((size_t)k * (m | 1) + (size_t)k * ((3 * m) | 1)) * sizeof(R);
  const bool in_smem = base + extra <= SMEM_MAX;
  const size_t smem = in_smem ? base + extra : base;
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(eigh_lowest_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_MAX);
  });
  if (e0 != cudaSuccess) return e0;
  R* Z = reinterpret_cast<R*>(work);       // k vectors of stride m | 1
  R* scratch = Z + (size_t)k * (m | 1);    // k x ((3 m) | 1)
  eigh_lowest_kernel<R><<<1, 512, smem, st>>>(m, k, A, lda, Z, scratch, in_smem ? 1 : 0, V, w, info);
  note_launch();
  return cudaGetLastError();
}

// theta_j = v_j^T A v_j / v_j^T v_j in double for the columns of V (row-major m x k): one
// CTA per eigenpair. With single-precision eigenvectors (error ~1e-6) the refined values
// are accurate to second order, i.e. to double precision.
__global__ void rayleigh_refine_kernel(int m, int k, const double* __restrict__ A, long lda,
                                       const double* __restrict__ V, double* __restrict__ w) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  double num = 0, den = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double vi = V[(long)i * k + j];
    double av = 0;
    for (int l = 0; l < m; ++l) av += A[(long)i * lda + l] * V[(long)l * k + j];
    num += vi * av;
    den += vi * vi;
  }
  num = blk_sum(num, red);
  den = blk_sum(den, red);
  if (threadIdx.x == 0) w[j] = num / den;
}

cudaError_t eigh_lowest(int m, int k, const double* A, long lda, double* work, double* V, double* w,
                        int* info, bool single, cudaStream_t st) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  if (m > EIGH_MAX || k > EIGH_KMAX || k > m) return cudaErrorInvalidValue;
  if (!single) return launch_eigh<double>(m, k, A, lda, work, V, w, info, st);
  cudaError_t e = launch_eigh<float>(m, k, A, lda, work, V, w, info, st);
  if (e != cudaSuccess) return e;
  rayleigh_refine_kernel<<<k, 128, 0, st>>>(m, k, A, lda, V, w);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bse
