// Tiled SIMT GEMM, C = alpha * op(A) op(B) + beta * C, with optional split-K, plus the
// tall-skinny products of the Davidson algebra and the float-float overlap Gram (below).
//
// The tiled GEMM serves the conduction projector P_c = 1 - sum_v |psi_v><psi_v| (Section
// 2) and the PDEP projection of Eq. (pdep) in the FP64 path, and the Davidson subspace
// algebra where the tall-skinny kernels do not apply. op(A) is A (row-major M x K) or A^T (A stored K x M); op(B) is B
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

// ---------------------------------------------------------------------------------
// Tall-skinny products of the Davidson algebra in single precision.
//
// ts_tn:  C (M x N, double) = alpha A B^T + beta C with A M x K, B N x K, N <= 32 and K
//         in the millions (Gram, Rayleigh-Ritz and CGS coefficient matrices). A CTA takes
//         a stretch of K (2048 by default) and a BM-row tile of A, streamed through a
//         three-stage cp.async ring. Its eight warps are RG row groups x KG k groups: a warp
//         owns an (8 LR) x (4 LC) block of C over its share of every staged chunk (KW
//         consecutive k), a lane an LR x LC block. The packed FP32x2 accumulators pair
//         consecutive k (even k in .x, odd k in .y), so both operands of every packed FMA
//         are adjacent words of one 16-byte shared-memory load and no register moves are
//         needed. The k-group partials are added in shared memory and accumulated into C
//         with double-precision atomics.
// ts_nn:  C (M x N) = alpha op(A) B + beta C with op(A) M x K small (K <= 256) and N in the
//         millions (CGS update, Cholesky-QR, Ritz vectors, restart). op(A) sits in shared
//         memory; a thread owns four adjacent columns and a band of up to 16 rows, and
//         streams its 16-byte pieces of B through a private cp.async ring twelve rows deep.
// ---------------------------------------------------------------------------------
namespace {

constexpr int TN_KS = 2048;    // K per CTA (ts_tn)
constexpr int TN_STAGES = 3;

// staged row of G 16-byte groups, group g stored at g ^ (row % 8): eight consecutive rows
// read at the same group hit eight distinct bank quads
template <int G>
__device__ __forceinline__ int tn_off(int row, int g) { return row * (4 * G) + ((g ^ (row & 7)) << 2); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;   // 0: fill the 16 bytes with zeros, read nothing
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}

// tile shape of one instantiation
template <int LR, int LC, int RG, bool SYM>
struct TnShape {
  static constexpr int WR = 8 * LR, BN = 4 * LC, BM = RG * WR, KG = 8 / RG;
  // k per warp per chunk: 16, or 8 where a 16-wide share would make the ring too large for
  // two CTAs per SM
  static constexpr int ROWS = SYM ? BM : BM + BN;
  static constexpr int KW = (ROWS * 16 * KG * 4 * TN_STAGES <= 110 * 1024) ? 16 : 8;
  static constexpr int KC = KW * KG;                 // k per chunk
  static constexpr int G = KC / 4;                   // 16-byte groups per staged row
  static constexpr int STAGE = ROWS * KC;            // floats per stage
  static constexpr int PIECES = ROWS * G;            // 16-byte copies per chunk
  static constexpr size_t RING = (size_t)TN_STAGES * STAGE * sizeof(float);
  static constexpr size_t RED = (size_t)KG * BM * BN * sizeof(float);
  static constexpr size_t SMEM = RING > RED ? RING : RED;
  static_assert(RG * KG == 8 && PIECES % 256 == 0 && G >= 8, "tile shape");
  static_assert(!SYM || BM == BN, "Gram tile");
};

// acc += (a.x b.x, a.y b.y) + (a.z b.z, a.w b.w): four consecutive k in two packed FMAs
__device__ __forceinline__ void tn_mac(float2& acc, const float4& a, const float4& b) {
  acc = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), acc);
  acc = __ffma2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w), acc);
}

template <int LR, int LC, int RG, bool SYM>
__global__ void __launch_bounds__(256, 2) ts_tn_kernel(int M, int N, long K, long ks, double alpha,
                                                      const float* __restrict__ A, long lda,
                                                      const float* __restrict__ B, long ldb,
                                                      double* __restrict__ C, long ldc) {
  using S = TnShape<LR, LC, RG, SYM>;
  extern __shared__ __align__(16) float ts_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = warp / S::KG, kg = warp % S::KG;
  const int ib = lane >> 2, jb = lane & 3;
  const long i0 = (long)blockIdx.x * S::BM;
  const long kbeg = (long)blockIdx.y * ks;
  const long kend = min(K, kbeg + ks);
  const int nch = (int)((kend - kbeg + S::KC - 1) / S::KC);
  // staging: thread tid copies group pg of rows prow + RPP q (q = 0 .. PIECES / 256 - 1);
  // whether a round q holds rows of A or of B is known at compile time
  constexpr int RPP = 256 / S::G;
  static_assert(RPP % 8 == 0 && (SYM || S::BM % RPP == 0), "staging rounds");
  const int prow = tid / S::G, pg = tid % S::G;
  const int dst0 = prow * (4 * S::G) + ((pg ^ (prow & 7)) << 2);
  const float* srcA = A + (i0 + prow) * lda + 4 * pg;
  const float* srcB = B + 4 * pg;
  const long rowsA = (long)M - i0 - prow;            // round q of A is valid while q RPP < rowsA
  auto issue = [&](int ch) {
    float* st = ts_smem + (ch % TN_STAGES) * S::STAGE + dst0;
    const long kc = (long)ch * S::KC;
    const bool kok = kbeg + kc + 4 * pg < kend;
#pragma unroll
    for (int q = 0; q < S::PIECES / 256; ++q) {
      if (SYM || q * RPP < S::BM) {
        const bool ok = kok && (q * RPP < rowsA);
        cp_async16(st + q * RPP * 4 * S::G, ok ? srcA + (long)q * RPP * lda + kbeg + kc : A, ok);
      } else {
        const int j = prow + q * RPP - S::BM;
        const bool ok = kok && (j < N);
        cp_async16(st + q * RPP * 4 * S::G, ok ? srcB + (long)j * ldb + kbeg + kc : B, ok);
      }
    }
  };
#pragma unroll
  for (int s0 = 0; s0 < TN_STAGES - 1; ++s0) {
    if (s0 < nch) issue(s0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  // operand loads: offsets of this lane's first A row and first two B rows, per k step;
  // further rows are 8 apart and keep the same swizzle, so they are immediate offsets
  constexpr int NQ = S::KW / 4;
  int offa[NQ], offb[2][NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int g = kg * NQ + q;
    offa[q] = (rg * S::WR + ib) * (4 * S::G) + ((g ^ ib) << 2);
    offb[0][q] = jb * (4 * S::G) + ((g ^ jb) << 2);
    offb[1][q] = (4 + jb) * (4 * S::G) + ((g ^ (4 + jb)) << 2);
  }
  constexpr int ROW8 = 8 * 4 * S::G;                 // floats between rows r and r + 8
  float2 acc[LR][LC];
#pragma unroll
  for (int r = 0; r < LR; ++r)
#pragma unroll
    for (int c = 0; c < LC; ++c) acc[r][c] = make_float2(0.f, 0.f);
  for (int ch = 0; ch < nch; ++ch) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(TN_STAGES - 2) : "memory");
    __syncthreads();
    if (ch + TN_STAGES - 1 < nch) issue(ch + TN_STAGES - 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const float* as = ts_smem + (ch % TN_STAGES) * S::STAGE;
    const float* bs = SYM ? as : as + S::BM * S::KC;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float* aq = as + offa[q];
      // the narrower operand stays in registers for the step, the other streams through
      if constexpr (LR <= LC) {
        float4 a[LR];
#pragma unroll
        for (int r = 0; r < LR; ++r) a[r] = *reinterpret_cast<const float4*>(aq + r * ROW8);
#pragma unroll
        for (int c = 0; c < LC; ++c) {
          const float4 b = *reinterpret_cast<const float4*>(bs + offb[c & 1][q] + (c >> 1) * ROW8);
#pragma unroll
          for (int r = 0; r < LR; ++r) tn_mac(acc[r][c], a[r], b);
        }
      } else {
        float4 b[LC];
#pragma unroll
        for (int c = 0; c < LC; ++c) b[c] = *reinterpret_cast<const float4*>(bs + offb[c & 1][q] + (c >> 1) * ROW8);
#pragma unroll
        for (int r = 0; r < LR; ++r) {
          const float4 a = *reinterpret_cast<const float4*>(aq + r * ROW8);
#pragma unroll
          for (int c = 0; c < LC; ++c) tn_mac(acc[r][c], a, b[c]);
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // k-group partials -> shared memory -> one double atomic per output
  float* red = ts_smem;                              // [KG][BM][BN]
#pragma unroll
  for (int r = 0; r < LR; ++r)
#pragma unroll
    for (int c = 0; c < LC; ++c)
      red[((size_t)kg * S::BM + rg * S::WR + r * 8 + ib) * S::BN + c * 4 + jb] = acc[r][c].x + acc[r][c].y;
  __syncthreads();
  for (int o = tid; o < S::BM * S::BN; o += 256) {
    const int i = o / S::BN, j = o % S::BN;
    if (i0 + i >= M || j >= N) continue;
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < S::KG; ++w) sum += red[w * S::BM * S::BN + o];
    atomicAdd(C + (i0 + i) * ldc + j, alpha * (double)sum);
  }
}

constexpr int NN_PD = 12;      // B rows in flight per thread (ts_nn)

template <int MT, bool AT>
__global__ void __launch_bounds__(256) ts_gemm_nn_kernel(int M, long N, int K, double alpha,
                                                        const float* __restrict__ A, long lda,
                                                        const float* __restrict__ B, long ldb,
                                                        double beta, float* __restrict__ C, long ldc) {
  extern __shared__ __align__(16) float ts_smem[];
  float* S = ts_smem;                                // [K][MT]: op(A)[i0 + i][k]
  // per-thread ring of NN_PD rows of B (16 bytes each), filled by cp.async: the loads in
  // flight take no registers, so each thread keeps NN_PD of them outstanding
  float4* ring = reinterpret_cast<float4*>(ts_smem + ((K * MT + 3) / 4) * 4);   // [NN_PD][256]
  const int i0 = blockIdx.x * MT;                    // row band (fastest: bands share B in L2)
  for (int e = threadIdx.x; e < K * MT; e += 256) {
    const int k = e / MT, i = e - k * MT;
    const int gi = i0 + i;
    S[e] = (gi < M) ? (AT ? A[(long)k * lda + gi] : A[(long)gi * lda + k]) : 0.f;
  }
  const long d = 4 * ((long)blockIdx.y * 256 + threadIdx.x);
  const bool act = d < N;
  const float* bp = B + (act ? d : 0);
  auto fetch = [&](int k) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(ring + (k % NN_PD) * 256 + threadIdx.x);
    const int nb = (act && k < K) ? 16 : 0;        // 0: zero-fill, read nothing
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
                 ::"r"(sa), "l"(bp + (long)(k < K ? k : 0) * ldb), "r"(nb) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
#pragma unroll
  for (int k = 0; k < NN_PD - 1; ++k) fetch(k);
  __syncthreads();
  float2 acc[MT][2];
#pragma unroll
  for (int i = 0; i < MT; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  for (int k = 0; k < K; ++k) {
    fetch(k + NN_PD - 1);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NN_PD - 1) : "memory");
    const float4 v = ring[(k % NN_PD) * 256 + threadIdx.x];
    const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
    const float* sk = S + k * MT;
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
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (!act) return;
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

template <int LR, int LC, int RG, bool SYM>
cudaError_t ts_tn_launch(int M, int N, long K, double alpha, const float* A, long lda, const float* B,
                         long ldb, double* C, long ldc, cudaStream_t st, long ks = TN_KS) {
  using S = TnShape<LR, LC, RG, SYM>;
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(ts_tn_kernel<LR, LC, RG, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)S::SMEM);
  });
  if (e0 != cudaSuccess) return e0;
  while ((K + ks - 1) / ks > 65535) ks *= 2;
  dim3 grid((unsigned)((M + S::BM - 1) / S::BM), (unsigned)((K + ks - 1) / ks));
  ts_tn_kernel<LR, LC, RG, SYM><<<grid, 256, S::SMEM, st>>>(M, N, K, ks, alpha, A, lda, B, ldb, C, ldc);
  note_launch();
  return cudaGetLastError();
}

// C = alpha A B^T + beta C, A M x K, B N x K (both row-major), N <= 32. The row tile is the
// one of 32, 64 or 128 rows that pads M least (ties: the larger tile); the column tile is
// 16 or 32 wide.
cudaError_t ts_gemm_tn(int M, int N, long K, double alpha, const float* A, long lda, const float* B,
                       long ldb, double beta, double* C, long ldc, cudaStream_t st) {
  const long tot = (long)M * N;
  scale_matrix_kernel<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, C, ldc, beta); note_launch();
  if (K == 0) return cudaGetLastError();
  if (A == B && lda == ldb && M == N && M <= 32) {
    if (M <= 16) return ts_tn_launch<2, 4, 1, true>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
    return ts_tn_launch<4, 8, 1, true>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  }
  int bm = 128;
  for (int cand : {64, 32}) {
    const long pc = (M + cand - 1) / cand * (long)cand, pb = (M + bm - 1) / bm * (long)bm;
    if (pc < pb) bm = cand;
  }
  if (N <= 16) {
    if (M <= 16) return ts_tn_launch<2, 4, 1, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
    if (bm == 32) return ts_tn_launch<4, 4, 1, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
    if (bm == 64) return ts_tn_launch<8, 4, 1, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
    return ts_tn_launch<8, 4, 2, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  }
  if (bm == 32) return ts_tn_launch<4, 8, 1, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  if (bm == 64) return ts_tn_launch<4, 8, 2, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
  return ts_tn_launch<4, 8, 4, false>(M, N, K, alpha, A, lda, B, ldb, C, ldc, st);
}

template <int MT>
cudaError_t ts_nn_launch(bool at, int M, long N, int K, double alpha, const float* A, long lda,
                         const float* B, long ldb, double beta, float* C, long ldc, cudaStream_t st) {
  // op(A) for K <= 256 rows plus the B ring: at most 16 KB + 48 KB
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    const int mx = (int)((256 * MT + 3) / 4 * 16 + (size_t)NN_PD * 256 * 16);
    cudaError_t e = cudaFuncSetAttribute(ts_gemm_nn_kernel<MT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ts_gemm_nn_kernel<MT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  });
  if (e0 != cudaSuccess) return e0;
  const size_t smem = ((size_t)K * MT + 3) / 4 * 16 + (size_t)NN_PD * 256 * 16;
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
// C[i][j] = C[j][i] for i > j: completes a symmetric result of which only the entries on
// and above the diagonal were computed
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


// ---------------------------------------------------------------------------------
// Symmetric Gram of FP64 data in float-float arithmetic: C = A A^T (A n x K, FP64, given as
// the split hi = fp32(x), lo = fp32(x - hi) in two FP32 arrays). Per output the exact product
// hi_a hi_b (p + e, e = fma(hi_a, hi_b, -p)) is added to an FP32 sum by an error-free
// two-sum, and the rounding error, e and the cross terms hi_a lo_b + lo_a hi_b collect in
// an FP32 compensation term (lo_a lo_b, 2^-48 relative, is dropped). A CTA owns a 64 x 64
// tile on or above the diagonal and a 2048-long stretch of K; its partial sums join C in
// double precision. The result agrees with an FP64 GEMM to about 1e-14 relative while
// using only FP32 instructions (FP64 runs at a small fraction of the FP32 rate here).
// ---------------------------------------------------------------------------------
namespace {
constexpr int FF_T = 64, FF_KC = 32, FF_KS = 2048, FF_LD = FF_T + 4;

__global__ void __launch_bounds__(256) gram_ff_kernel(int n, long K, const float* __restrict__ Ahi,
                                                      const float* __restrict__ Alo, long lda,
                                                      double* __restrict__ C, long ldc) {
  __shared__ __align__(16) float sh[4][FF_KC][FF_LD];   // A hi, A lo, B hi, B lo: [k][row]
  // upper-triangle tile (bi <= bj) of this CTA
  int bi = 0, rem = blockIdx.x;
  const int nt = (n + FF_T - 1) / FF_T;
  while (rem >= nt - bi) { rem -= nt - bi; ++bi; }
  const int bj = bi + rem;
  const int i0 = bi * FF_T, j0 = bj * FF_T;
  const long kbeg = (long)blockIdx.y * FF_KS, kend = min(K, kbeg + FF_KS);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float s[4][4], c[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = 0.f;
  for (long k0 = kbeg; k0 < kend; k0 += FF_KC) {
    __syncthreads();
    // stage: 64 rows x 32 k of each operand, split into hi / lo, transposed to [k][row]
#pragma unroll
    for (int q = 0; q < (2 * FF_T * FF_KC) / 256; ++q) {
      const int e = tid + 256 * q;
      const int op = e / (FF_T * FF_KC), rr = (e / FF_KC) % FF_T, kk = e % FF_KC;
      const int row = (op ? j0 : i0) + rr;
      const long k = k0 + kk;
      const bool ok = row < n && k < kend;
      sh[2 * op][kk][rr] = ok ? Ahi[(long)row * lda + k] : 0.f;
      sh[2 * op + 1][kk][rr] = ok ? Alo[(long)row * lda + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < FF_KC; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&sh[0][kk][4 * ty]);
      const float4 al = *reinterpret_cast<const float4*>(&sh[1][kk][4 * ty]);
      const float4 bh = *reinterpret_cast<const float4*>(&sh[2][kk][4 * tx]);
      const float4 bl = *reinterpret_cast<const float4*>(&sh[3][kk][4 * tx]);
      const float ahv[4] = {ah.x, ah.y, ah.z, ah.w}, alv[4] = {al.x, al.y, al.z, al.w};
      const float bhv[4] = {bh.x, bh.y, bh.z, bh.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = __fmul_rn(ahv[i], bhv[j]);
          const float pe = __fmaf_rn(ahv[i], bhv[j], -p);
          const float t = __fadd_rn(s[i][j], p);
          const float bp = __fsub_rn(t, s[i][j]);
          const float err = __fadd_rn(__fsub_rn(s[i][j], __fsub_rn(t, bp)), __fsub_rn(p, bp));
          s[i][j] = t;
          c[i][j] = __fmaf_rn(ahv[i], blv[j], __fmaf_rn(alv[i], bhv[j], __fadd_rn(c[i][j], __fadd_rn(err, pe))));
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = i0 + 4 * ty + i, col = j0 + 4 * tx + j;
      if (row < n && col < n) atomicAdd(C + (long)row * ldc + col, (double)s[i][j] + (double)c[i][j]);
    }
}
}  // namespace

cudaError_t gram_ff(int n, long K, const float* Ahi, const float* Alo, long lda, double* C, long ldc,
                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long tot = (long)n * n;
  scale_matrix_kernel<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, n, C, ldc, 0.0); note_launch();
  if (K > 0) {
    const long nt = (n + FF_T - 1) / FF_T;
    dim3 grid((unsigned)(nt * (nt + 1) / 2), (unsigned)((K + FF_KS - 1) / FF_KS));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    gram_ff_kernel<<<grid, 256, 0, st>>>(n, K, Ahi, Alo, lda, C, ldc); note_launch();
  }
  mirror_upper_kernel<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, C, ldc); note_launch();
  return cudaGetLastError();
}

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
