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

template <typename R>
__global__ void __launch_bounds__(512) eigh_lowest_kernel(int m, int k, const double* __restrict__ Ain,
                                                         long lda, R* __restrict__ Z,
                                                         R* __restrict__ S, double* __restrict__ V,
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
  __shared__ R red[32];
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
      e[c] = (nrm == 0.0) ? 0.0 : alpha;
      // v = x - alpha e1, |v|^2 = s2 - 2 alpha x0 + alpha^2
      const R vn2 = s2 - 2.0 * alpha * x0 + alpha * alpha;
      s_alpha = alpha;
      s_scale = (nrm == 0.0 || vn2 <= 0.0) ? 0.0 : 1.0 / sqrt(vn2);
    }
    __syncthreads();
    const R sc = s_scale;
    // u = v / |v| stored in place of the column (zero reflector if sc == 0)
    for (int i = tid; i < n; i += nt) {
      const R x = A[(c + 1 + i) * ld + c];
      A[(c + 1 + i) * ld + c] = (i == 0 ? x - s_alpha : x) * sc;
    }
    __syncthreads();
    if (sc == 0.0) continue;
    // p = B u over the trailing block B = A[c+1:, c+1:] (symmetric, both halves valid)
    for (int i = tid; i < n; i += nt) {
      R acc = 0;
      const R* row = A + (c + 1 + i) * ld + (c + 1);
      for (int j = 0; j < n; ++j) acc += row[j] * A[(c + 1 + j) * ld + c];
      p[i] = acc;
    }
    R kk = 0;
    __syncthreads();
    for (int i = tid; i < n; i += nt) kk += A[(c + 1 + i) * ld + c] * p[i];
    kk = blk_sum(kk, red);
    // q = p - K u (kept in p), B -= 2 (u q^T + q u^T)
    for (int i = tid; i < n; i += nt) p[i] -= kk * A[(c + 1 + i) * ld + c];
    __syncthreads();
    for (int x = tid; x < n * n; x += nt) {
      const int i = x / n, j = x - i * n;
      const R ui = A[(c + 1 + i) * ld + c], uj = A[(c + 1 + j) * ld + c];
      A[(c + 1 + i) * ld + (c + 1 + j)] -= 2.0 * (ui * p[j] + p[i] * uj);
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      d[m - 2] = A[(m - 2) * ld + (m - 2)];
      e[m - 2] = A[(m - 1) * ld + (m - 2)];
    }
    d[m - 1] = A[(m - 1) * ld + (m - 1)];
    e[m - 1] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) e2[i] = e[i] * e[i];
  __syncthreads();
  // ---- 2. bisection for the k lowest eigenvalues ----
  R gl = (R)1e30, gu = (R)-1e30, tnorm = 0;
  for (int i = 0; i < m; ++i) {
    const R r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
    gl = fmin(gl, d[i] - r);
    gu = fmax(gu, d[i] + r);
  }
  tnorm = fmax(fabs(gl), fabs(gu));
  const R pivmin = Tol::pivtiny + Tol::tiny * tnorm * tnorm;
  for (int j = tid; j < k; j += nt) {
    R lo = gl - 50 * Tol::eps * tnorm - Tol::tiny, hi = gu + 50 * Tol::eps * tnorm + Tol::tiny;
    for (int it = 0; it < 200 && hi - lo > Tol::eps * fmax(fabs(lo), fabs(hi)) + Tol::tiny; ++it) {
      const R mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(m, d, e2, mid, pivmin) > j) hi = mid; else lo = mid;
    }
    lam[j] = 0.5 * (lo + hi);
  }
  __syncthreads();
  // ---- 3. inverse iteration, one thread per eigenvector (Z column-major, m x k) ----
  const R ortol = (R)1e-3 * tnorm;
  for (int j = tid; j < k; j += nt) {
    R* z = Z + (long)j * m;
    // perturb the shift slightly inside clusters so the factorisation stays regular
    R mu = lam[j];
    for (int i = 0; i < j; ++i)
      if (fabs(lam[i] - mu) < 50 * Tol::eps * tnorm) mu = lam[i] + 50 * Tol::eps * tnorm * (j - i);
    for (int i = 0; i < m; ++i) z[i] = (R)1 / sqrt((R)m) * ((R)1 + (R)0.001 * ((i * 7 + j * 13) % 11));
    for (int pass = 0; pass < 3; ++pass) {
      // solve (T - mu I) y = z by elimination with partial pivoting; the upper factor has
      // up to two super-diagonals (u0 diag, u1, u2); y overwrites z
      R* u0 = S + (long)j * 3 * m;
      R* u1 = u0 + m;
      R* u2 = u1 + m;
      R a0 = d[0] - mu, b0 = (m > 1) ? e[0] : 0.0, c0 = 0.0;
      R rhs = z[0];
      for (int i = 0; i + 1 < m; ++i) {
        const R sub = e[i];
        const R a1 = d[i + 1] - mu, b1 = (i + 2 < m) ? e[i + 1] : 0.0;
        R r1 = z[i + 1];
        if (fabs(sub) > fabs(a0)) {          // swap rows i and i+1
          const R f = a0 / sub;
          u0[i] = sub; u1[i] = a1; u2[i] = b1;
          z[i] = r1;
          const R na0 = b0 - f * a1, nb0 = c0 - f * b1;
          r1 = rhs - f * r1;
          a0 = na0; b0 = nb0; c0 = 0.0; rhs = r1;
        } else {
          if (a0 == 0.0) a0 = pivmin;
          const R f = sub / a0;
          u0[i] = a0; u1[i] = b0; u2[i] = c0;
          z[i] = rhs;
          a0 = a1 - f * b0; b0 = b1 - f * c0; c0 = 0.0; rhs = r1 - f * rhs;
        }
      }
      if (a0 == 0.0) a0 = pivmin;
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
  // re-orthogonalise inside clusters (modified Gram-Schmidt in eigenvalue order)
  for (int j = 1; j < k; ++j) {
    for (int i = 0; i < j; ++i) {
      if (fabs(lam[j] - lam[i]) > ortol) continue;
      R dot = 0;
      for (int r = tid; r < m; r += nt) dot += Z[(long)i * m + r] * Z[(long)j * m + r];
      dot = blk_sum(dot, red);
      for (int r = tid; r < m; r += nt) Z[(long)j * m + r] -= dot * Z[(long)i * m + r];
      __syncthreads();
    }
    R nn = 0;
    for (int r = tid; r < m; r += nt) nn += Z[(long)j * m + r] * Z[(long)j * m + r];
    nn = blk_sum(nn, red);
    const R inv = (R)1 / sqrt(nn);
    for (int r = tid; r < m; r += nt) Z[(long)j * m + r] *= inv;
    __syncthreads();
  }
  // ---- 4. back-transformation: v = H_0 H_1 ... H_{m-3} z, applied to all k vectors ----
  for (int c = m - 3; c >= 0; --c) {
    const int n = m - c - 1;
    // one warp per vector: dot = u . z[c+1:], z[c+1:] -= 2 dot u
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int j = wid; j < k; j += nw) {
      R* z = Z + (long)j * m;
      R dot = 0;
      for (int i = lane; i < n; i += 32) dot += A[(c + 1 + i) * ld + c] * z[c + 1 + i];
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      for (int i = lane; i < n; i += 32) z[c + 1 + i] -= 2.0 * dot * A[(c + 1 + i) * ld + c];
    }
    __syncthreads();
  }
  // outputs: V row-major m x k (component r of eigenvector j at V[r*k + j]), w[0..k)
  for (long x = tid; x < (long)m * k; x += nt) {
    const int r = (int)(x / k), j = (int)(x - (long)r * k);
    V[x] = (double)Z[(long)j * m + r];
  }
  for (int j = tid; j < k; j += nt) w[j] = (double)lam[j];
  if (tid == 0) info[0] = 0;
}

// k lowest eigenpairs of the symmetric m x m matrix A (lda): eigenvalues ascending in w[0..k),
// eigenvectors as the columns of V (row-major m x k). work: at least 4*m*k doubles.
// single: single-precision arithmetic (double input and outputs).
template <typename R>
static cudaError_t launch_eigh(int m, int k, const double* A, long lda, double* work, double* V, double* w,
                               int* info, cudaStream_t st) {
  const size_t smem = ((size_t)m * (m + 1) + 4 * (size_t)m + EIGH_KMAX) * sizeof(R);
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    const size_t mx = ((size_t)EIGH_MAX * (EIGH_MAX + 1) + 4 * EIGH_MAX + EIGH_KMAX) * sizeof(R);
    return cudaFuncSetAttribute(eigh_lowest_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
  });
  if (e0 != cudaSuccess) return e0;
  R* Z = reinterpret_cast<R*>(work);       // m x k, column-major
  R* scratch = Z + (size_t)m * k;          // 3 m per vector
  eigh_lowest_kernel<R><<<1, 512, smem, st>>>(m, k, A, lda, Z, scratch, V, w, info);
  note_launch();
  return cudaGetLastError();
}

cudaError_t eigh_lowest(int m, int k, const double* A, long lda, double* work, double* V, double* w,
                        int* info, bool single, cudaStream_t st) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  if (m > EIGH_MAX || k > EIGH_KMAX || k > m) return cudaErrorInvalidValue;
  return single ? launch_eigh<float>(m, k, A, lda, work, V, w, info, st)
                : launch_eigh<double>(m, k, A, lda, work, V, w, info, st);
}

}  // namespace bse
