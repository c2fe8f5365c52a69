// BF16x3 tensor-core GEMM for sm_103a (tcgen05 + TMA): out = alpha * A B^T + beta * out.
//
// Used in the mixed-precision path for the conduction projector P_c (Section 2) and the
// PDEP projection of Eq. (pdep). Each FP32 operand x is split as hi = bf16(x),
// lo = bf16(x - hi), and the product is accumulated in FP32 as hi*hi + hi*lo + lo*hi
// (the three-term bfloat16 scheme of Henry, Tang and Heinecke, ARITH 2019), which keeps
// each product to about 1e-5 relative while running on the 5th-generation tensor cores.
//
// A [M x K] and B [N x K] are bf16, K-major (row-major with K contiguous), with leading
// dimensions padded to multiples of 8. A CTA computes a 128 x 128 tile: one thread
// issues TMA loads (128-byte swizzled 64-wide K slices of A_hi, A_lo, B_hi, B_lo) into a
// 3-stage ring guarded by mbarriers, one thread issues tcgen05.mma (kind::f16,
// accumulator in TMEM), and four warps read the accumulator back with tcgen05.ld for
// the epilogue. Optional split-K adds partial tiles with atomics. Every wait is bounded:
// on timeout the CTA raises an error flag, drains and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include "common.cuh"
#include "kernels.h"

namespace bse {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 3;
constexpr int TC_TILE = TC_BM * TC_BK * 2;          // 16 KB per operand tile (BM == BN)
constexpr int TC_STAGE_BYTES = 4 * TC_TILE;         // A_hi, A_lo, B_hi, B_lo
constexpr int TC_EPI_LD = 17;                        // floats per row of a warp's epilogue chunk
constexpr int TC_EPI_BYTES = 4 * 32 * TC_EPI_LD * 4; // four warps x 32 rows x 16 (+1) floats
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 256 + TC_EPI_BYTES;
constexpr long long TC_WAIT_LIMIT = 1ll << 26;      // try_wait polls before giving up (default)
constexpr long long TC_DRAIN_LIMIT = 1ll << 26;     // polls per wait while draining after a give-up

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar) : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

struct TcArgs {
  int M, N, K;
  int kt_per_split;
  float alpha, beta;
  float* out;
  long ldo;
  int atomic;
  int* err;
  long long wait_limit;   // polls of each pipeline wait before the CTA gives up
};

__global__ void __launch_bounds__(128, 1) tc_gemm_bf16x3_kernel(
    const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
    const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, TcArgs g) {
  extern __shared__ __align__(16) uint8_t tc_raw[];
  uint8_t* base = tc_raw + ((1024 - (su32(tc_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + TC_STAGES * TC_STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accb = empty + TC_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accb + 1);
  float* epi = reinterpret_cast<float*>(base + TC_STAGES * TC_STAGE_BYTES + 256);   // [4][32][17]
  __shared__ int s_abort, s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;
  const int kt_all = (g.K + TC_BK - 1) / TC_BK;
  const int kt0 = blockIdx.z * g.kt_per_split;
  const int kt1 = min(kt0 + g.kt_per_split, kt_all);
  const int nk = kt1 - kt0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) { mbar_init(su32(full + s), 1); mbar_init(su32(empty + s), 1); }
    mbar_init(su32(accb), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(TC_BN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);
  if (nk > 0) {
    if (warp == 0 && lane == 0) {
      // TMA producer
      for (int it = 0; it < nk; ++it) {
        const int s = it % TC_STAGES;
        if (it >= TC_STAGES && !mbar_wait(su32(empty + s), ((it / TC_STAGES) - 1) & 1, g.wait_limit)) {
          s_abort = 1; break;
        }
        if (*(volatile int*)&s_abort) break;
        const uint32_t fb = su32(full + s);
        mbar_expect_tx(fb, TC_STAGE_BYTES);
        const uint32_t st = su32(base + s * TC_STAGE_BYTES);
        const int x = (kt0 + it) * TC_BK;
        tma_load_2d(st, &tAh, x, m0, fb);
        tma_load_2d(st + TC_TILE, &tAl, x, m0, fb);
        tma_load_2d(st + 2 * TC_TILE, &tBh, x, n0, fb);
        tma_load_2d(st + 3 * TC_TILE, &tBl, x, n0, fb);
        s_issued = it + 1;
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      for (int it = 0; it < nk; ++it) {
        const int s = it % TC_STAGES;
        if (!mbar_wait(su32(full + s), (it / TC_STAGES) & 1, g.wait_limit)) { s_abort = 1; break; }
        s_consumed = it + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = su32(base + s * TC_STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          const uint32_t off = kk * 32;   // 16 bf16 along K inside the 128-byte swizzle row
          const uint64_t ah = sw128_desc(st + off), al = sw128_desc(st + TC_TILE + off);
          const uint64_t bh = sw128_desc(st + 2 * TC_TILE + off), bl = sw128_desc(st + 3 * TC_TILE + off);
          umma_bf16(tmem, ah, bh, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          umma_bf16(tmem, ah, bl, idesc, 1u);
          umma_bf16(tmem, al, bh, idesc, 1u);
        }
        umma_commit(su32(empty + s));
      }
      umma_commit(su32(accb));
    }
    // epilogue: all four warps
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait(su32(accb), 0, g.wait_limit) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) s_abort = 1;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    float* ew = epi + warp * 32 * TC_EPI_LD;
    // lane (r4, q): rows r4 + 8 i of this warp's 32, columns 4 q .. 4 q + 3 of the chunk
    const int q = lane & 3, r4 = lane >> 2;
    const bool vec = (g.ldo % 4) == 0 && (((uintptr_t)g.out) % 16) == 0;
    if (ok) {
#pragma unroll 1
      for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // transpose through shared memory: the accumulator comes one row per lane, the
        // global accesses go as 16-byte pieces of eight rows per instruction
#pragma unroll
        for (int j = 0; j < 16; ++j) ew[lane * TC_EPI_LD + j] = g.alpha * __uint_as_float(v[j]);
        __syncwarp();
        const int col = n0 + c0 + 4 * q;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rl = r4 + 8 * i;
          const int row = m0 + warp * 32 + rl;
          if (row >= g.M) continue;
          const float* e = ew + rl * TC_EPI_LD + 4 * q;
          float4 val = make_float4(e[0], e[1], e[2], e[3]);
          float* o = g.out + (long)row * g.ldo + col;
          if (vec && col + 3 < g.N) {
            float4* o4 = reinterpret_cast<float4*>(o);
            if (g.atomic) {
              atomicAdd(o4, val);
            } else {
              if (g.beta != 0.f) {
                const float4 old = *o4;
                val.x += g.beta * old.x; val.y += g.beta * old.y; val.z += g.beta * old.z; val.w += g.beta * old.w;
              }
              *o4 = val;
            }
          } else {
            const float vv[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (col + j >= g.N) break;
              if (g.atomic) atomicAdd(o + j, vv[j]);
              else o[j] = (g.beta == 0.f) ? vv[j] : vv[j] + g.beta * o[j];
            }
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    // drain before the shared memory and TMEM are released: the TMA loads issued but never
    // consumed, then the MMAs issued (the accumulator barrier is committed after the last
    // one, on the abort path too); each wait again bounded
    for (int it = s_consumed; it < s_issued; ++it)
      mbar_wait(su32(full + it % TC_STAGES), (it / TC_STAGES) & 1, TC_DRAIN_LIMIT);
    if (nk > 0) mbar_wait(su32(accb), 0, TC_DRAIN_LIMIT);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
  }
}

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool get_encoder() {
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

// 2-D bf16 tensor map over [rows x cols] with row stride ld (elements), box 64 x 128, 128B swizzle
bool tc_make_map(void* map_out, const void* ptr, long rows, long cols, long ld) {
  if (!get_encoder()) return false;
  if ((ld * 2) % 16 || ((uintptr_t)ptr) % 16) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t tc_gemm_bf16x3(const void* mAh, const void* mAl, const void* mBh, const void* mBl, int M, int N,
                           int K, double alpha, double beta, float* out, long ldo, int splits, int* err,
                           cudaStream_t st, long long wait_limit) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(tc_gemm_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  });
  if (e0 != cudaSuccess) return e0;
  const int kt_all = (K + TC_BK - 1) / TC_BK;
  if (splits < 1) splits = 1;
  if (splits > kt_all) splits = kt_all > 0 ? kt_all : 1;
  const int kper = (kt_all + splits - 1) / splits;
  splits = kt_all > 0 ? (kt_all + kper - 1) / kper : 1;
  TcArgs a;
  a.M = M; a.N = N; a.K = K; a.kt_per_split = kper; a.alpha = (float)alpha; a.beta = (float)beta;
  // beta = 1 (an update out += alpha A B^T) also goes through reductions: each element
  // receives one FP32 add, the same value as a read-modify-write, without the epilogue
  // waiting on loads of the old output
  a.out = out; a.ldo = ldo; a.atomic = (splits > 1 || beta == 1.0) ? 1 : 0; a.err = err;
  a.wait_limit = wait_limit < 0 ? TC_WAIT_LIMIT : wait_limit;
  if (splits > 1 && beta != 1.0) {
    // partial tiles are added atomically: pre-scale the output (beta = 0 clears it)
    cudaError_t e = (beta == 0.0) ? cudaSuccess : cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    if (ldo == N) e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)M * N, st);
    else e = cudaMemset2DAsync(out, sizeof(float) * ldo, 0, sizeof(float) * N, M, st);
    if (e != cudaSuccess) return e;
  }
  CUtensorMap Ah, Al, Bh, Bl;
  memcpy(&Ah, mAh, sizeof(CUtensorMap)); memcpy(&Al, mAl, sizeof(CUtensorMap));
  memcpy(&Bh, mBh, sizeof(CUtensorMap)); memcpy(&Bl, mBl, sizeof(CUtensorMap));
  dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, splits);
  tc_gemm_bf16x3_kernel<<<grid, 128, TC_SMEM, st>>>(Ah, Al, Bh, Bl, a);
  note_launch();
  return cudaGetLastError();
}

// x -> (hi, lo) bf16 with hi = RN(x), lo = RN(x - hi); columns [cols, ld_out) are zero.
// One CTA per row; a thread converts two adjacent columns and stores them as bf16 pairs
// (ld_out is a multiple of 8, so every output row starts 16-byte aligned).
__global__ void bf16_split_kernel(const float* __restrict__ X, long rows, int cols, long ld_in,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_out) {
  for (long i = blockIdx.x; i < rows; i += gridDim.x) {
    const float* x = X + i * ld_in;
    __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(hi + i * ld_out);
    __nv_bfloat162* l2 = reinterpret_cast<__nv_bfloat162*>(lo + i * ld_out);
    for (long j = 2 * threadIdx.x; j < ld_out; j += 2 * blockDim.x) {
      const float x0 = j < cols ? x[j] : 0.f, x1 = j + 1 < cols ? x[j + 1] : 0.f;
      const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      const float2 hf = __bfloat1622float2(h);
      h2[j >> 1] = h;
      l2[j >> 1] = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    }
  }
}
// same from an FP64 source
__global__ void bf16_split64_kernel(const double* __restrict__ X, long rows, int cols, long ld_in,
                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ld_out) return;
  for (long i = blockIdx.y; i < rows; i += gridDim.y) {
    const float x = j < cols ? (float)X[i * ld_in + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i * ld_out + j] = h;
    lo[i * ld_out + j] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
// transposed split: out[j][i] from X[i][j] (for B operands that must be K-major)
__global__ void bf16_split64_t_kernel(const double* __restrict__ X, long rows, int cols, long ld_in,
                                      __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_out) {
  // out has cols rows and ld_out >= rows columns
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // source row -> output column
  if (i >= ld_out) return;
  for (long j = blockIdx.y; j < cols; j += gridDim.y) {
    const float x = i < rows ? (float)X[i * ld_in + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[j * ld_out + i] = h;
    lo[j * ld_out + i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

cudaError_t bf16_split(const float* X, long rows, int cols, long ld_in, void* hi, void* lo, long ld_out,
                       cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (ld_out % 8 || ((uintptr_t)hi) % 16 || ((uintptr_t)lo) % 16) return cudaErrorInvalidValue;
  const unsigned nb = (unsigned)(rows < 2147483647L ? rows : 2147483647L);
  bf16_split_kernel<<<nb, 256, 0, st>>>(X, rows, cols, ld_in, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ld_out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t bf16_split64(const double* X, long rows, int cols, long ld_in, void* hi, void* lo, long ld_out,
                         bool transpose, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (!transpose) {
    dim3 grid((unsigned)((ld_out + 255) / 256), (unsigned)(rows < 65535 ? rows : 65535));
    bf16_split64_kernel<<<grid, 256, 0, st>>>(X, rows, cols, ld_in, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ld_out);
  } else {
    dim3 grid((unsigned)((ld_out + 255) / 256), (unsigned)(cols < 65535 ? cols : 65535));
    bf16_split64_t_kernel<<<grid, 256, 0, st>>>(X, rows, cols, ld_in, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, ld_out);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace bse
