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

template <typename T, typename TC, bool AT, bool BT, int TM, int TN, bool DFLUSH, bool TRI = false>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, double alpha,
                                                  const T* __restrict__ A, long lda,
                                                  const T* __restrict__ B, long ldb, double beta,
                                                  TC* __restrict__ C, long ldc, int k_chunk,
                                                  int atomic) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  long ti = blockIdx.y, tj = blockIdx.x;
  if constexpr (TRI) {
    // blockIdx.x enumerates the tiles (ti <= tj) of the upper triangle, row by row
    const int nt = (N + BN - 1) / BN;
    long r = blockIdx.x;
    ti = 0;
    while (r >= nt - ti) { r -= nt - ti; ++ti; }
    tj = ti + r;
  }
  const long i0 = ti * BM, j0 = tj * BN;
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

// ---------------------------------------------------------------------------------
// Tall-skinny products of the Davidson algebra in single precision.
//
// ts_tn:  C (M x N, double) = alpha A B^T + beta C with A M x K, B N x K, N <= 32 and K
//         in the millions (Gram, Rayleigh-Ritz and CGS coefficient matrices). A CTA takes
//         a 2048-long stretch of K and a 64-row tile of A, streamed through a four-stage
//         cp.async ring in 32-wide chunks; each warp computes the whole 64 x 32 tile on
//         its own 4-wide slice of every chunk (lane: 8 x 8 outputs as packed FP32 pairs),
//         so every accumulator sums 256 products in FP32; the eight warp partials are
//         added in double and accumulated into C with double-precision atomics.
// ts_nn:  C (M x N) = alpha op(A) B + beta C with op(A) M x K small (K <= 256) and N in the
//         millions (CGS update, Cholesky-QR, Ritz vectors, restart). op(A) sits in shared
//         memory; a thread owns four adjacent columns and a band of up to 16 rows,
//         streaming B straight from global memory in 16-byte loads.
// ---------------------------------------------------------------------------------
namespace {

constexpr int TS_KS = 2048;    // K per CTA (ts_tn)
constexpr int TS_KC = 32;      // K per staged chunk
constexpr int TS_STAGES = 4;

// staged chunk row: 32 floats in eight 16-byte groups, group g stored at g ^ (row >> SWS) % 8,
// so that lanes reading the same group of different rows hit distinct banks
template <int SWS>
__device__ __forceinline__ int ts_off(int row, int g) { return row * TS_KC + ((g ^ ((row >> SWS) & 7)) << 2); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;   // 0: fill the 16 bytes with zeros, read nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}

// BM rows of A per CTA (64 or 32); SYM: B is A (a Gram matrix, M = N <= 32), staged once
template <int BM, bool SYM>
__global__ void __launch_bounds__(256, 2) ts_gemm_tn_kernel(int M, int N, long K, double alpha,
                                                           const float* __restrict__ A, long lda,
                                                           const float* __restrict__ B, long ldb,
                                                           double* __restrict__ C, long ldc) {
  static_assert(BM == 64 || (BM == 32), "row tile");
  static_assert(!SYM || BM == 32, "Gram tile");
  constexpr int RI = BM / 8;                         // rows of A per lane
  constexpr int SWS = (BM == 64) ? 3 : 2;
  constexpr int ROWS = SYM ? BM : BM + 32;           // staged rows per chunk
  constexpr int STAGE = ROWS * TS_KC;                // floats per stage
  constexpr int PIECES = ROWS * 8 / 256;             // 16-byte copies per thread per chunk
  extern __shared__ __align__(16) float ts_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long i0 = (long)blockIdx.y * BM;
  const long kbeg = (long)blockIdx.x * TS_KS;
  const long kend = min(K, kbeg + TS_KS);
  const int nch = (int)((kend - kbeg + TS_KC - 1) / TS_KC);
  auto issue = [&](int ch) {
    float* st = ts_smem + (ch % TS_STAGES) * STAGE;
#pragma unroll
    for (int q = 0; q < PIECES; ++q) {
      const int e = tid + 256 * q;
      const int row = e >> 3, g = e & 7;
      const long k = kbeg + (long)ch * TS_KC + 4 * g;
      const float* src;
      bool ok;
      if (row < BM) {
        const long i = i0 + row;
        ok = (i < M) && (k < kend);
        src = ok ? A + i * lda + k : A;
      } else {
        const int j = row - BM;
        ok = (j < N) && (k < kend);
        src = ok ? B + (long)j * ldb + k : B;
      }
      cp_async16(st + ts_off<SWS>(row, g), src, ok);
    }
  };
#pragma unroll
  for (int s0 = 0; s0 < TS_STAGES - 1; ++s0) {
    if (s0 < nch) issue(s0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  const int ib = lane >> 2, jb = lane & 3;
  float2 acc[RI][4];
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int ch = 0; ch < nch; ++ch) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(TS_STAGES - 2) : "memory");
    __syncthreads();
    if (ch + TS_STAGES - 1 < nch) issue(ch + TS_STAGES - 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const float* as = ts_smem + (ch % TS_STAGES) * STAGE;
    const float* bs = SYM ? as : as + BM * TS_KC;
    // this warp's four k values: group `warp` of every row
    float2 bp[4][4];    // [k][j pair]
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) {
      const float4 u = *reinterpret_cast<const float4*>(bs + ts_off<SWS>(8 * jb + 2 * jp, warp));
      const float4 v = *reinterpret_cast<const float4*>(bs + ts_off<SWS>(8 * jb + 2 * jp + 1, warp));
      bp[0][jp] = make_float2(u.x, v.x);
      bp[1][jp] = make_float2(u.y, v.y);
      bp[2][jp] = make_float2(u.z, v.z);
      bp[3][jp] = make_float2(u.w, v.w);
    }
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const float4 a = *reinterpret_cast<const float4*>(as + ts_off<SWS>(RI * ib + i, warp));
      const float ak[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float2 ai = make_float2(ak[kk], ak[kk]);
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) acc[i][jp] = __ffma2_rn(ai, bp[kk][jp], acc[i][jp]);
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // eight warp partials -> double sums -> atomics
  float* red = ts_smem;                              // [8][BM][32]
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp)
      *reinterpret_cast<float2*>(red + ((size_t)warp * BM + RI * ib + i) * 32 + 8 * jb + 2 * jp) = acc[i][jp];
  __syncthreads();
  for (int o = tid; o < BM * 32; o += 256) {
    const int i = o >> 5, j = o & 31;
    if (i0 + i >= M || j >= N) continue;
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += (double)red[w * BM * 32 + o];
    atomicAdd(C + (i0 + i) * ldc + j, alpha * sum);
  }
}

template <int MT, bool AT>
__global__ void __launch_bounds__(256) ts_gemm_nn_kernel(int M, long N, int K, double alpha,
                                                        const float* __restrict__ A, long lda,
                                                        const float* __restrict__ B, long ldb,
                                                        double beta, float* __restrict__ C, long ldc) {
  extern __shared__ __align__(16) float ts_smem[];
  float* S = ts_smem;                                // [K][MT]: op(A)[i0 + i][k]
  const int i0 = blockIdx.x * MT;                    // row band (fastest: bands share B in L2)
  for (int e = threadIdx.x; e < K * MT; e += 256) {
    const int k = e / MT, i = e - k * MT;
    const int gi = i0 + i;
    S[e] = (gi < M) ? (AT ? A[(long)k * lda + gi] : A[(long)gi * lda + k]) : 0.f;
  }
  __syncthreads();
  const long d = 4 * ((long)blockIdx.y * 256 + threadIdx.x);
  if (d >= N) return;
  float2 acc[MT][2];
#pragma unroll
  for (int i = 0; i < MT; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  const float* bp = B + d;
  int k = 0;
  for (; k + 4 <= K; k += 4) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(bp + (long)(k + u) * ldb);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float* sk = S + (k + u) * MT;
      const float2 v0 = make_float2(v[u].x, v[u].y), v1 = make_float2(v[u].z, v[u].w);
#pragma unroll
      for (int i = 0; i < MT; i += 4) {
        const float4 s4 = *reinterpret_cast<const float4*>(sk + i);
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 sq = make_float2(sv[q], sv[q]);
          acc[i + q][0] = __ffma2_rn(sq, v0, acc[i + q][0]);
          acc[i + q][1] = __ffma2_rn(sq, v1, acc[i + q][1]);
        }
      }
    }
  }
  for (; k < K; ++k) {
    const float4 v = *reinterpret_cast<const float4*>(bp + (long)k * ldb);
    const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
    const float* sk = S + k * MT;
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const float2 sq = make_float2(sk[i], sk[i]);
      acc[i][0] = __ffma2_rn(sq, v0, acc[i][0]);
      acc[i][1] = __ffma2_rn(sq, v1, acc[i][1]);
    }
  }
  const float al = (float)alpha, be = (float)beta;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    if (i0 + i >= M) break;
    float4* cp = reinterpret_cast<float4*>(C + (long)(i0 + i) * ldc + d);
    float4 r = make_float4(al * acc[i][0].x, al * acc[i][0].y, al * acc[i][1].x, al * acc[i][1].y);
    if (be != 0.f) {
      const float4 c0 = *cp;
      r.x += be * c0.x; r.y += be * c0.y; r.z += be * c0.z; r.w += be * c0.w;
    }
    *cp = r;
  }
}

bool aligned(const void* p, size_t b) { return ((uintptr_t)p % b) == 0; }

template <int BM, bool SYM>
cudaError_t ts_tn_launch(int M, int N, long K, double alpha, const float* A, long lda, const float* B,
                         long ldb, double* C, long ldc, cudaStream_t st) {
  // the reduction area (8 x BM x 32 floats) and the staging ring, whichever is larger
  constexpr size_t red = 8 * (size_t)BM * 32 * sizeof(float);
  constexpr size_t ring = (size_t)TS_STAGES * (SYM ? BM : BM + 32) * TS_KC * sizeof(float);
  constexpr size_t smem = red > ring ? red : ring;
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(ts_gemm_tn_kernel<BM, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e0 != cudaSuccess) return e0;
  dim3 grid((unsigned)((K + TS_KS - 1) / TS_KS), (unsigned)((M + BM - 1) / BM));
  ts_gemm_tn_kernel<BM, SYM><<<grid, 256, smem, st>>>(M, N, K, alpha, A, lda, B, ldb, C, ldc); note_launch();
  return cudaGetLastError();
}

// C = alpha A B^T + beta C, A M x K, B N x K (both row-major), N <= 32
cudaError_t ts_gemm_tn(int M, int N, long K, double alpha, const float* A, long lda, const float* B,
                       long ldb, double beta, double* C, long ldc, cudaStream_t st) {
  const long tot = (long)M * N;
  scale_matrix_kernel<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, C, ldc, beta); note_launch();
  if (K == 0) return cudaGetLastError();
  if (M <= 32 && A == B && lda == ldb && M == N)
    return ts_tn_launch<32, true>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  if (M <= 32) return ts_tn_launch<32, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  return ts_tn_launch<64, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
}

template <int MT>
cudaError_t ts_nn_launch(bool at, int M, long N, int K, double alpha, const float* A, long lda,
                         const float* B, long ldb, double beta, float* C, long ldc, cudaStream_t st) {
  const size_t smem = (size_t)K * MT * sizeof(float);
  dim3 grid((unsigned)((M + MT - 1) / MT), (unsigned)((N / 4 + 255) / 256));
  if (at) ts_gemm_nn_kernel<MT, true><<<grid, 256, smem, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else ts_gemm_nn_kernel<MT, false><<<grid, 256, smem, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  note_launch();
  return cudaGetLastError();
}

// C = alpha op(A) B + beta C, op(A) M x K (A stored K x M when at), B K x N row-major
cudaError_t ts_gemm_nn(bool at, int M, long N, int K, double alpha, const float* A, long lda,
                       const float* B, long ldb, double beta, float* C, long ldc, cudaStream_t st) {
  if (M <= 4) return ts_nn_launch<4>(at, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  if (M <= 8) return ts_nn_launch<8>(at, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
  return ts_nn_launch<16>(at, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

}  // namespace

// ---------------------------------------------------------------------------------
// Symmetric Gram C = alpha A A^T (A n x K row-major, C n x n): only the tiles on and
// above the diagonal are computed (split over K with atomics), then mirrored.
// ---------------------------------------------------------------------------------
namespace {
template <typename TC>
__global__ void mirror_upper_kernel(int n, TC* C, long ldc) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (long)i * n);
  if (i > j) C[i * ldc + j] = C[(long)j * ldc + i];
}
}  // namespace

template <typename T, typename TC>
cudaError_t gram_sym(int n, int K, double alpha, const T* A, long lda, TC* C, long ldc, cudaStream_t st) {
  constexpr int TM = 4, BM = 64;
  if (n <= 0) return cudaSuccess;
  constexpr bool DF = sizeof(T) < sizeof(TC);
  const long nt = (n + BM - 1) / BM;
  const long tiles = nt * (nt + 1) / 2;
  long s = tiles >= 304 ? 1 : (304 + tiles - 1) / tiles;
  const long kmax = (K + 255) / 256;
  if (s > kmax) s = kmax;
  if (s < 1) s = 1;
  int k_chunk = (int)((K + s - 1) / s);
  k_chunk = (k_chunk + 15) / 16 * 16;
  if (k_chunk <= 0) k_chunk = 16;
  const int splitk = (int)((K + k_chunk - 1) / k_chunk);
  const long tot = (long)n * n;
  scale_matrix_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, n, C, ldc, 0.0); note_launch();
  if (K > 0) {
    dim3 grid((unsigned)tiles, 1, (unsigned)(splitk < 1 ? 1 : splitk));
    gemm_kernel<T, TC, false, true, TM, TM, DF, true><<<grid, 256, 0, st>>>(n, n, K, alpha, A, lda, A, lda, 0.0, C,
                                                                           ldc, k_chunk, 1); note_launch();
  }
  mirror_upper_kernel<TC><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, C, ldc); note_launch();
  return cudaGetLastError();
}
template cudaError_t gram_sym<double, double>(int, int, double, const double*, long, double*, long, cudaStream_t);

// Tile shape follows the operands: a side of at most 16 gets a 16-wide tile, so the
// tall-skinny products of the Davidson algebra (16-32 rows against millions of
// columns) do not pad a 64-wide tile.
template <typename T, typename TC>
cudaError_t gemm(bool at, bool bt, int M, int N, int K, double alpha, const T* A, long lda,
                 const T* B, long ldb, double beta, TC* C, long ldc, int splitk, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4 && sizeof(TC) == 8) {
    if (!at && bt && N <= 32 && K >= 4096 && K % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 &&
        aligned(A, 16) && aligned(B, 16))
      return ts_gemm_tn(M, N, K, alpha, (const float*)A, lda, (const float*)B, ldb, beta, (double*)C, ldc, st);
  }
  if constexpr (sizeof(T) == 4 && sizeof(TC) == 4) {
    if (!bt && M <= 64 && K <= 256 && N >= 1024 && N / 1024 < 65535 && N % 4 == 0 && ldb % 4 == 0 && ldc % 4 == 0 &&
        aligned(B, 16) && aligned(C, 16))
      return ts_gemm_nn(at, M, N, K, alpha, (const float*)A, lda, (const float*)B, ldb, beta, (float*)C, ldc, st);
  }
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
