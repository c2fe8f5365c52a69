// Wannier localisation of the occupied orbitals by joint approximate diagonalisation (JADE),
// Section 2 (Eqs. wannier, spread): the six matrices A^(n)_vw = <psi_v|M^(n)|psi_w> of
// M = cos(2 pi x/L), sin(2 pi x/L), ... (and the diagonals of B^(n) = <psi|M^2|psi> for the
// spread) are grid quadratures of the FP64 orbitals; U is built by sweeps of Givens rotations.
// A sweep visits every pair (p, q) once, in rounds of disjoint pairs (a round-robin
// tournament), so the rotations of one round commute: one kernel computes all their angles
// from the current matrices, one rotates the affected rows of all six matrices, one the
// columns and U's columns. Each round is O(K n^2) work (the paper's code collects the
// rotations of a round into one matrix-matrix product instead).
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace bse {

namespace {

// W[w][r] = M_op(r) u[w][r] for the grid point r = x + N (y + N z);
// op = 2 axis + (0 cos, 1 sin), axis 0 x, 1 y, 2 z
__global__ void jade_weight_kernel(int n, long n3, int N, int op, const double* __restrict__ u,
                                   double* __restrict__ W, int squared) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n3) return;
  const long r = idx % n3;
  const int axis = op >> 1;
  const long c = (axis == 0) ? (r % N) : (axis == 1) ? ((r / N) % N) : (r / ((long)N * N));
  double s, co;
  sincospi(2.0 * (double)c / (double)N, &s, &co);
  double m = (op & 1) ? s : co;
  if (squared) m *= m;
  W[idx] = m * u[idx];
}

// angles of the round's pairs from matrices 0 .. K_use-1; cs[k] = (cos, sin); smax receives
// the largest |sin| (as the bits of a non-negative float, which order like integers)
__global__ void jade_angles_kernel(int K_use, int n, const double* __restrict__ A, const int2* __restrict__ pairs,
                                   int np, double2* __restrict__ cs, unsigned* __restrict__ smax) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const int p = pairs[k].x, q = pairs[k].y;
  double c = 1.0, s = 0.0;
  if (p < n && q < n) {
    double g11 = 0, g22 = 0, g12 = 0;
    for (int m = 0; m < K_use; ++m) {
      const double* Am = A + (size_t)m * n * n;
      const double h0 = Am[(size_t)p * n + p] - Am[(size_t)q * n + q];
      const double h1 = Am[(size_t)p * n + q] + Am[(size_t)q * n + p];
      g11 += h0 * h0; g22 += h1 * h1; g12 += h0 * h1;
    }
    const double th = 0.25 * atan2(2.0 * g12, g11 - g22);
    sincos(th, &s, &c);
  }
  cs[k] = make_double2(c, s);
  atomicMax(smax, __float_as_uint((float)fabs(s)));
}

// rows p, q of matrix blockIdx.y: A <- R^T A
__global__ void jade_rows_kernel(int n, double* __restrict__ A, const int2* __restrict__ pairs,
                                 const double2* __restrict__ cs) {
  const int k = blockIdx.x;
  const int p = pairs[k].x, q = pairs[k].y;
  if (p >= n || q >= n) return;
  const double c = cs[k].x, s = cs[k].y;
  double* Am = A + (size_t)blockIdx.y * n * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double ap = Am[(size_t)p * n + j], aq = Am[(size_t)q * n + j];
    Am[(size_t)p * n + j] = c * ap + s * aq;
    Am[(size_t)q * n + j] = -s * ap + c * aq;
  }
}

// columns p, q of matrix blockIdx.y (the last index is U): X <- X R
__global__ void jade_cols_kernel(int n, int K, double* __restrict__ A, double* __restrict__ U,
                                 const int2* __restrict__ pairs, const double2* __restrict__ cs) {
  const int k = blockIdx.x;
  const int p = pairs[k].x, q = pairs[k].y;
  if (p >= n || q >= n) return;
  const double c = cs[k].x, s = cs[k].y;
  double* X = (blockIdx.y < (unsigned)K) ? A + (size_t)blockIdx.y * n * n : U;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double xp = X[(size_t)i * n + p], xq = X[(size_t)i * n + q];
    X[(size_t)i * n + p] = c * xp + s * xq;
    X[(size_t)i * n + q] = -s * xp + c * xq;
  }
}

__global__ void set_identity_kernel(int n, double* U) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  U[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

inline unsigned nb(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t jade_weight(int n, long n3, int N, int op, const double* u, double* W, bool squared, cudaStream_t st) {
  jade_weight_kernel<<<nb((long)n * n3), 256, 0, st>>>(n, n3, N, op, u, W, squared ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t jade_round(int K_use, int K, int n, double* A, double* U, const int2* pairs, int np, double2* cs,
                       unsigned* smax, cudaStream_t st) {
  jade_angles_kernel<<<nb(np), 256, 0, st>>>(K_use, n, A, pairs, np, cs, smax);
  note_launch();
  jade_rows_kernel<<<dim3((unsigned)np, (unsigned)K), 128, 0, st>>>(n, A, pairs, cs);
  note_launch();
  jade_cols_kernel<<<dim3((unsigned)np, (unsigned)(K + 1)), 128, 0, st>>>(n, K, A, U, pairs, cs);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(int n, double* U, cudaStream_t st) {
  set_identity_kernel<<<nb((long)n * n), 256, 0, st>>>(n, U);
  note_launch();
  return cudaGetLastError();
}

// round-robin tournament of n players (padded to even m): m-1 rounds of m/2 disjoint pairs,
// every pair once; pairs with the padding index n are idle
void jade_schedule(int n, std::vector<int2>& pairs, int& rounds, int& per_round) {
  const int m = n + (n & 1);
  rounds = m - 1;
  per_round = m / 2;
  pairs.clear();
  for (int r = 0; r < m - 1; ++r) {
    auto put = [&](int a, int b) { pairs.push_back(make_int2(std::min(a, b), std::max(a, b))); };
    put(r, m - 1);
    for (int i = 1; i < m / 2; ++i) put((r + i) % (m - 1), (r - i + (m - 1)) % (m - 1));
  }
}

}  // namespace bse
