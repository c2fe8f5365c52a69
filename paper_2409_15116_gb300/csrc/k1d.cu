// Screened direct term K1d of Eq. (k1d), fused with the real-space parts of D (Eq. d)
// and K1e (Eq. k1e):
//
//   u_R,sv(r) = V_loc(r) u_a,sv(r) + s V_H,s(r) u_psi,v(r) - sum_{w in nbr(v)} tau_vw(r) u_a,sw(r)
//
// At each grid point the sum is a sparse (N_occ x N_occ) times dense (N_occ x n_vec)
// product whose sparse factor tau(r) changes from point to point. A CTA owns a tile of
// TR consecutive points and a chunk of SC trial vectors: it stages a(r) for every orbital
// of the chunk in shared memory (read from HBM once, 128-byte rows), then streams tau
// through rows grouped four at a time (one localisation site): each tau value is
// loaded once per tile and reused for the SC vectors, each staged a value feeds the
// four rows of a block. tau_vw(r) for pairs outside the overlap list is simply absent
// (Eq. overlap); blocks list the union of their rows' neighbours with -1 for the
// missing entries.
#include "common.cuh"
#include "kernels.h"

namespace bse {

template <typename T, int TR, int SC>
__global__ void __launch_bounds__(256, 3) k1d_tile_kernel(
    int n_vec, int n_occ, long n3, const T* __restrict__ a, const T* __restrict__ tau,
    const int* __restrict__ bptr, const int* __restrict__ bw, const int4* __restrict__ bp,
    int n_blocks, const T* __restrict__ vloc, const T* __restrict__ vh,
    const T* __restrict__ upsi, T sf, T* __restrict__ out) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char k1d_smem[];
  T* A = reinterpret_cast<T*>(k1d_smem);            // [n_occ][SC][TR]
  T* VH = A + (size_t)n_occ * SC * TR;               // [SC][TR]
  const int n_sc = (n_vec + SC - 1) / SC;
  const int sc = blockIdx.x % n_sc;
  const long tile = blockIdx.x / n_sc;
  const long r0 = tile * TR;
  const int s0 = sc * SC;
  const int ns = min(SC, n_vec - s0);
  const int tid = threadIdx.x;
  // stage a(f, r0 .. r0+TR) for the fields f of this vector chunk
  const long f_lo = (long)s0 * n_occ, f_hi = (long)(s0 + ns) * n_occ;
  const long c_lo = f_lo >> 1, c_hi = (f_hi + 1) >> 1;
  const C* ac = reinterpret_cast<const C*>(a);
  if ((n_occ & 1) == 0) {
    // even N_occ: complex grid c holds orbitals (2k, 2k+1) of one vector; a warp moves
    // two 128-byte rows (16 complex values each) per iteration, no per-element division
    const int half = n_occ >> 1;
    const int rows = ns * half;
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int sub = lane / TR, t = lane % TR;        // TR divides 32
    constexpr int RPW = 32 / TR;                     // rows per warp pass
    for (int row = wid * RPW + sub; row < rows; row += nw * RPW) {
      const int sl = row / half, k = row - sl * half;
      const C z = ac[(c_lo + row) * n3 + r0 + t];
      A[((2 * k) * SC + sl) * TR + t] = z.x;
      A[((2 * k + 1) * SC + sl) * TR + t] = z.y;
    }
  } else {
    for (long e = tid; e < (c_hi - c_lo) * TR; e += blockDim.x) {
      const long c = c_lo + e / TR;
      const int t = (int)(e % TR);
      const C z = ac[c * n3 + r0 + t];
      const long f0 = 2 * c, f1 = f0 + 1;
      if (f0 >= f_lo) {
        const long q = f0 - f_lo;
        A[((q % n_occ) * SC + q / n_occ) * TR + t] = z.x;
      }
      if (f1 < f_hi) {
        const long q = f1 - f_lo;
        A[((q % n_occ) * SC + q / n_occ) * TR + t] = z.y;
      }
    }
  }
  for (int e = tid; e < SC * TR; e += blockDim.x) {
    const int s = e / TR, t = e % TR;
    VH[e] = (s < ns) ? vh[pair_off<T>(s0 + s, r0 + t, n3)] : (T)0;
  }
  __syncthreads();
  const int t = tid % TR, g = tid / TR, G = blockDim.x / TR;
  const long r = r0 + t;
  const T vl = vloc[r];
  for (int rb = g; rb < n_blocks; rb += G) {
    T acc[4][SC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int s = 0; s < SC; ++s) acc[i][s] = (T)0;
    const int e0 = bptr[rb], e1 = bptr[rb + 1];
    // two-deep software pipeline on the tau loads (entries e+1 and e+2 in flight)
    T tq[2][4];
    int wq[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const int e = e0 + d;
      wq[d] = 0;
      tq[d][0] = tq[d][1] = tq[d][2] = tq[d][3] = (T)0;
      if (e < e1) {
        const int4 p = bp[e];
        wq[d] = bw[e];
        tq[d][0] = p.x >= 0 ? tau[(long)p.x * n3 + r] : (T)0;
        tq[d][1] = p.y >= 0 ? tau[(long)p.y * n3 + r] : (T)0;
        tq[d][2] = p.z >= 0 ? tau[(long)p.z * n3 + r] : (T)0;
        tq[d][3] = p.w >= 0 ? tau[(long)p.w * n3 + r] : (T)0;
      }
    }
    for (int e = e0; e < e1; ++e) {
      const int w = wq[0];
      const T t0 = tq[0][0], t1 = tq[0][1], t2 = tq[0][2], t3 = tq[0][3];
      wq[0] = wq[1];
#pragma unroll
      for (int i = 0; i < 4; ++i) tq[0][i] = tq[1][i];
      if (e + 2 < e1) {
        const int4 p = bp[e + 2];
        wq[1] = bw[e + 2];
        tq[1][0] = p.x >= 0 ? tau[(long)p.x * n3 + r] : (T)0;
        tq[1][1] = p.y >= 0 ? tau[(long)p.y * n3 + r] : (T)0;
        tq[1][2] = p.z >= 0 ? tau[(long)p.z * n3 + r] : (T)0;
        tq[1][3] = p.w >= 0 ? tau[(long)p.w * n3 + r] : (T)0;
      }
      const T* Aw = A + (size_t)w * SC * TR + t;
#pragma unroll
      for (int s = 0; s < SC; ++s) {
        const T av = Aw[s * TR];
        acc[0][s] = fma(t0, av, acc[0][s]);
        acc[1][s] = fma(t1, av, acc[1][s]);
        acc[2][s] = fma(t2, av, acc[2][s]);
        acc[3][s] = fma(t3, av, acc[3][s]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int v = 4 * rb + i;
      if (v >= n_occ) break;
      const T up = upsi[pair_off<T>(v, r, n3)];
      const T* Av = A + (size_t)v * SC * TR + t;
#pragma unroll
      for (int s = 0; s < SC; ++s) {
        if (s >= ns) break;
        const long f = (long)(s0 + s) * n_occ + v;
        out[pair_off<T>(f, r, n3)] = vl * Av[s * TR] + sf * VH[s * TR + t] * up - acc[i][s];
      }
    }
  }
}

template <typename T, int TR, int SC>
static cudaError_t launch_k1d(int n_vec, int n_occ, long n3, const T* a, const T* tau,
                              const int* bptr, const int* bw, const int4* bp, int n_blocks,
                              const T* vloc, const T* vh, const T* upsi, double sf, T* out,
                              cudaStream_t st) {
  const size_t smem = ((size_t)n_occ * SC * TR + SC * TR) * sizeof(T);
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(k1d_tile_kernel<T, TR, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e0 != cudaSuccess) return e0;
  const long tiles = n3 / TR;
  const long blocks = tiles * ((n_vec + SC - 1) / SC);
  k1d_tile_kernel<T, TR, SC><<<(unsigned)blocks, 256, smem, st>>>(
      n_vec, n_occ, n3, a, tau, bptr, bw, bp, n_blocks, vloc, vh, upsi, (T)sf, out);
  note_launch();
  return cudaGetLastError();
}

// shared-memory budget of the a(r) stage; SC (vectors per CTA) is the largest power of
// two with n_occ * SC * TR * sizeof(T) within it. A budget near 72 KB lets three CTAs
// (24 warps) share an SM, which the tau loads need for latency hiding.
#ifndef BSE_K1D_SMEM_KB
#define BSE_K1D_SMEM_KB 72
#endif
constexpr size_t K1D_SMEM_BUDGET = (size_t)BSE_K1D_SMEM_KB * 1024;

#ifndef BSE_K1D_TR
#define BSE_K1D_TR 16
#endif

template <typename T>
int k1d_vectors_per_cta(int n_occ) {
  constexpr int TR = BSE_K1D_TR;
  for (int sc = 8; sc >= 1; sc >>= 1)
    if ((size_t)n_occ * sc * TR * sizeof(T) + sc * TR * sizeof(T) <= K1D_SMEM_BUDGET) return sc;
  return 0;
}

// whether SC vectors per CTA fit the 200 KB opt-in shared memory
template <typename T>
bool k1d_fits(int n_occ, int sc) {
  constexpr int TR = BSE_K1D_TR;
  return (size_t)n_occ * sc * TR * sizeof(T) + sc * TR * sizeof(T) <= 200 * 1024;
}

// sc: vectors per CTA (8, 4, 2 or 1; 0 picks the largest within the default budget)
template <typename T>
cudaError_t k1d_tiled(int n_vec, int n_occ, long n3, const T* a, const T* tau, const int* bptr,
                      const int* bw, const int4* bp, int n_blocks, const T* vloc, const T* vh,
                      const T* upsi, double sf, T* out, int sc, cudaStream_t st) {
  constexpr int TR = BSE_K1D_TR;
  if (n_vec <= 0) return cudaSuccess;
  if (n3 % TR) return cudaErrorInvalidValue;
  if (sc == 0) sc = k1d_vectors_per_cta<T>(n_occ);
  if (!k1d_fits<T>(n_occ, sc)) return cudaErrorInvalidValue;
  switch (sc) {
    case 8: return launch_k1d<T, TR, 8>(n_vec, n_occ, n3, a, tau, bptr, bw, bp, n_blocks, vloc, vh, upsi, sf, out, st);
    case 4: return launch_k1d<T, TR, 4>(n_vec, n_occ, n3, a, tau, bptr, bw, bp, n_blocks, vloc, vh, upsi, sf, out, st);
    case 2: return launch_k1d<T, TR, 2>(n_vec, n_occ, n3, a, tau, bptr, bw, bp, n_blocks, vloc, vh, upsi, sf, out, st);
    case 1: return launch_k1d<T, TR, 1>(n_vec, n_occ, n3, a, tau, bptr, bw, bp, n_blocks, vloc, vh, upsi, sf, out, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t k1d_tiled<float>(int, int, long, const float*, const float*, const int*, const int*, const int4*, int, const float*, const float*, const float*, double, float*, int, cudaStream_t);
template cudaError_t k1d_tiled<double>(int, int, long, const double*, const double*, const int*, const int*, const int4*, int, const double*, const double*, const double*, double, double*, int, cudaStream_t);
template bool k1d_fits<float>(int, int);
template bool k1d_fits<double>(int, int);
template int k1d_vectors_per_cta<float>(int);
template int k1d_vectors_per_cta<double>(int);

}  // namespace bse
