// Tiled SIMT GEMM, C = alpha * op(A) op(B) + beta * C, with optional split-K.
//
// Used for the conduction projector P_c = 1 - sum_v |psi_v><psi_v| (Section 2), the
// PDEP projection of Eq. (pdep), the overlap Gram of Eq. (overlap) and the Davidson
// subspace algebra. op(A) is A (row-major M x K) or A^T (A stored K x M); op(B) is B
// (row-major K x N) or B^T (B stored N x K). With DFLUSH the products accumulate in
// the input precision over 256-term runs and the runs are summed in double: FP32
// products with FP64 accumulation for the Davidson Gram and Rayleigh-Ritz matrices.
#include "common.cuh"
#include "kernels.h"

namespace bse {

template <typename T, typename TC, bool AT, bool BT, int TM, int TN, bool DFLUSH>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, double alpha,
                                                  const T* __restrict__ A, long lda,
                                                  const T* __restrict__ B, long ldb, double beta,
                                                  TC* __restrict__ C, long ldc, int k_chunk,
                                                  int atomic) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long i0 = (long)blockIdx.y * BM, j0 = (long)blockIdx.x * BN;
  const long kbeg = (long)blockIdx.z * k_chunk;
  const long kend = (kbeg + k_chunk < K) ? kbeg + k_chunk : K;
  T acc[TM][TN];
  double dacc[DFLUSH ? TM : 1][DFLUSH ? TN : 1];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) acc[m][n] = (T)0;
  if constexpr (DFLUSH) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TN; ++n) dacc[m][n] = 0.0;
  }
  int tiles = 0;
  for (long kt = kbeg; kt < kend; kt += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int ii, kk;
      if (!AT) { ii = e / BK; kk = e - ii * BK; } else { kk = e / BM; ii = e - kk * BM; }
      const long gi = i0 + ii, gk = kt + kk;
      T v = (T)0;
      if (gi < M && gk < kend) v = AT ? A[gk * lda + gi] : A[gi * lda + gk];
      As[kk][ii] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int jj, kk;
      if (BT) { jj = e / BK; kk = e - jj * BK; } else { kk = e / BN; jj = e - kk * BN; }
      const long gj = j0 + jj, gk = kt + kk;
      T v = (T)0;
      if (gj < N && gk < kend) v = BT ? B[gj * ldb + gk] : B[gk * ldb + gj];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int m = 0; m < TM; ++m) a[m] = As[kk][ty + 16 * m];
#pragma unroll
      for (int n = 0; n < TN; ++n) b[n] = Bs[kk][tx + 16 * n];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) acc[m][n] = fma(a[m], b[n], acc[m][n]);
    }
    __syncthreads();
    if constexpr (DFLUSH) {
      if (++tiles == 16) {
        tiles = 0;
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int n = 0; n < TN; ++n) { dacc[m][n] += (double)acc[m][n]; acc[m][n] = (T)0; }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const long i = i0 + ty + 16 * m;
    if (i >= M) continue;
#pragma unroll
    for (int n = 0; n < TN; ++n) {
      const long j = j0 + tx + 16 * n;
      if (j >= N) continue;
      double v = (double)acc[m][n];
      if constexpr (DFLUSH) v += dacc[m][n];
      v *= alpha;
      TC* c = C + i * ldc + j;
      if (atomic) {
        atomicAdd(c, (TC)v);
      } else {
        if (beta != 0.0) v += beta * (double)(*c);
        *c = (TC)v;
      }
    }
  }
}

template <typename TC>
__global__ void scale_matrix_kernel(int M, int N, TC* C, long ldc, double beta) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * N) return;
  const long i = idx / N, j = idx - i * N;
  C[i * ldc + j] = beta == 0.0 ? (TC)0 : (TC)(beta * (double)C[i * ldc + j]);
}

template <typename T, typename TC, bool AT, bool BT, int TM, int TN, bool DFLUSH>
static cudaError_t launch(int M, int N, int K, double alpha, const T* A, long lda, const T* B,
                          long ldb, double beta, TC* C, long ldc, int splitk, cudaStream_t st) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  const long gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splitk <= 0) {
    const long tiles = gx * gy;
    const long want = 2 * 152;
    long s = tiles >= want ? 1 : (want + tiles - 1) / tiles;
    const long kmax = (K + 255) / 256;   // at least 256 terms per split
    if (s > kmax) s = kmax;
    if (s < 1) s = 1;
    splitk = (int)s;
  }
  int k_chunk = (int)((K + splitk - 1) / splitk);
  k_chunk = (k_chunk + 15) / 16 * 16;
  if (k_chunk <= 0) k_chunk = 16;
  splitk = (int)((K + k_chunk - 1) / k_chunk);
  if (splitk < 1) splitk = 1;
  int atomic = 0;
  if (splitk > 1) {
    const long tot = (long)M * N;
    scale_matrix_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, C, ldc, beta); note_launch();
    atomic = 1;
  }
  if (K == 0) {
    if (splitk <= 1) {
      const long tot = (long)M * N;
      scale_matrix_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, C, ldc, beta); note_launch();
    }
    return cudaGetLastError();
  }
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)splitk);
  gemm_kernel<T, TC, AT, BT, TM, TN, DFLUSH><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb,
                                                                  beta, C, ldc, k_chunk, atomic); note_launch();
  return cudaGetLastError();
}

template <typename T, typename TC, int TM, int TN>
static cudaError_t dispatch_t(bool at, bool bt, int M, int N, int K, double alpha, const T* A,
                              long lda, const T* B, long ldb, double beta, TC* C, long ldc,
                              int splitk, cudaStream_t st) {
  constexpr bool DF = sizeof(T) < sizeof(TC);
  if (!at && bt) return launch<T, TC, false, true, TM, TN, DF>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  if (!at && !bt) return launch<T, TC, false, false, TM, TN, DF>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  if (at && !bt) return launch<T, TC, true, false, TM, TN, DF>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  return launch<T, TC, true, true, TM, TN, DF>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
}

// Tile shape follows the operands: a side of at most 16 gets a 16-wide tile, so the
// tall-skinny products of the Davidson algebra (16-32 rows against millions of
// columns) do not pad a 64-wide tile.
template <typename T, typename TC>
cudaError_t gemm(bool at, bool bt, int M, int N, int K, double alpha, const T* A, long lda,
                 const T* B, long ldb, double beta, TC* C, long ldc, int splitk, cudaStream_t st) {
  const bool sm = M <= 16, sn = N <= 16;
  if (sm && !sn) return dispatch_t<T, TC, 1, 4>(at, bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  if (sn && !sm) return dispatch_t<T, TC, 4, 1>(at, bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  if (sm && sn) return dispatch_t<T, TC, 1, 1>(at, bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  if (M <= 32 || N <= 32) return dispatch_t<T, TC, 2, 2>(at, bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
  return dispatch_t<T, TC, 4, 4>(at, bt, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk, st);
}

template cudaError_t gemm<double, double>(bool, bool, int, int, int, double, const double*, long, const double*, long, double, double*, long, int, cudaStream_t);
template cudaError_t gemm<float, float>(bool, bool, int, int, int, double, const float*, long, const float*, long, double, float*, long, int, cudaStream_t);
template cudaError_t gemm<float, double>(bool, bool, int, int, int, double, const float*, long, const float*, long, double, double*, long, int, cudaStream_t);

}  // namespace bse
