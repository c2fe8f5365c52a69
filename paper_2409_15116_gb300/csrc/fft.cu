// Batched 3D FFTs on N^3 grids (N in {16,32,48,64,72,96}) and plane-wave sphere
// scatter / gather for Gamma-packed real fields.
//
// The transforms move the auxiliary orbitals a_sv, the pair densities of Eq. (k1e),
// the densities psi_v psi_w of Eq. (tau) and the outputs of Eq. (evp) between the
// plane-wave sphere and the real-space grid (the paper uses cuFFT, Section 3; these
// kernels are written for sm_103a instead). Each 3D transform is three passes of
// 1D transforms along x, y, z; a CTA moves TX lines of one axis into shared memory
// (coalesced rows), runs a self-sorting (Stockham) mixed-radix transform with
// radix-2/3/4/8 butterflies, and writes the lines back. Unnormalised:
//   sign = -1:  F(n) = sum_m f(m) exp(-2 pi i n m / N)
//   sign = +1:  f(m) = sum_n F(n) exp(+2 pi i n m / N)
// Two real fields travel in one complex grid (real part = even field, imaginary
// part = odd field); they separate again through Hermitian symmetry at the sphere.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <vector>

namespace bse {

// ---------------------------------------------------------------------------------
// radix plans (product of radices = N)
// ---------------------------------------------------------------------------------
template <int N> struct Plan;
template <> struct Plan<16> { static constexpr int n = 2, r0 = 4, r1 = 4, r2 = 1, TX = 16; };
template <> struct Plan<32> { static constexpr int n = 2, r0 = 8, r1 = 4, r2 = 1, TX = 16; };
template <> struct Plan<48> { static constexpr int n = 3, r0 = 4, r1 = 4, r2 = 3, TX = 16; };
template <> struct Plan<64> { static constexpr int n = 2, r0 = 8, r1 = 8, r2 = 1, TX = 16; };
template <> struct Plan<72> { static constexpr int n = 3, r0 = 8, r1 = 3, r2 = 3, TX = 24; };
template <> struct Plan<96> { static constexpr int n = 3, r0 = 8, r1 = 4, r2 = 3, TX = 16; };

// R-point DFT in registers, direction exp(sign * 2 pi i q r / R)
template <typename C, int R> struct Dft;
template <typename C> struct Dft<C, 2> {
  static __device__ __forceinline__ void run(C* v, int) {
    C a = v[0], b = v[1]; v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};
template <typename C> struct Dft<C, 3> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using T = decltype(v[0].x);
    const T h = (T)0.86602540378443864676;   // sqrt(3)/2
    C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m; m.x = v[0].x - (T)0.5 * s.x; m.y = v[0].y - (T)0.5 * s.y;
    C t = cmul_si(d, sign); t.x *= h; t.y *= h;
    v[0] = cadd(v[0], s); v[1] = cadd(m, t); v[2] = csub(m, t);
  }
};
template <typename C> struct Dft<C, 4> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    C a2 = cadd(v[1], v[3]), a3 = cmul_si(csub(v[1], v[3]), sign);
    v[0] = cadd(a0, a2); v[2] = csub(a0, a2); v[1] = cadd(a1, a3); v[3] = csub(a1, a3);
  }
};
template <typename C> struct Dft<C, 8> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using T = decltype(v[0].x);
    const T r2 = (T)0.70710678118654752440;   // 1/sqrt(2)
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    Dft<C, 4>::run(e, sign); Dft<C, 4>::run(o, sign);
    // twiddles w8^q = exp(sign 2 pi i q / 8)
    C w1 = cmk<C>(r2, sign * r2), w3 = cmk<C>(-r2, sign * r2);
    C t0 = o[0], t1 = cmul(o[1], w1), t2 = cmul_si(o[2], sign), t3 = cmul(o[3], w3);
    v[0] = cadd(e[0], t0); v[4] = csub(e[0], t0);
    v[1] = cadd(e[1], t1); v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2); v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3); v[7] = csub(e[3], t3);
  }
};

// Shared-memory position of element k of line i: one pad slot per 16 complex values
// and an odd line stride, so strided butterfly writes and the transposed line loads of
// the y / z passes fall into distinct banks.
template <int N> struct Pad {
  static constexpr int raw = N + N / 16;
  static constexpr int LS = raw | 1;
};
template <int N>
__device__ __forceinline__ int sidx(int i, int k) { return i * Pad<N>::LS + k + (k >> 4); }

// one Stockham stage of radix R over TX lines of length N (src -> dst, both smem)
template <typename C, int N, int R, int TX>
__device__ __forceinline__ void stage(const C* src, C* dst, const C* tw, int Ns, int sign) {
  constexpr int NB = N / R;
  const int step = N / (Ns * R);
  for (int e = threadIdx.x; e < TX * NB; e += blockDim.x) {
    const int i = e / NB, j = e - i * NB;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[sidx<N>(i, j + r * NB)];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * k * step) % N]);
    Dft<C, R>::run(v, sign);
    const int o = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[sidx<N>(i, o + r * Ns)] = v[r];
  }
}

// all stages of the TX lines held in buf0 (buf1 is scratch); returns the buffer holding
// the result. Ends with a barrier.
template <typename C, int N>
__device__ __forceinline__ const C* line_fft(C* buf0, C* buf1, const C* tw, int sign) {
  constexpr int TX = Plan<N>::TX;
  C* src = buf0; C* dst = buf1;
  int Ns = 1;
  stage<C, N, Plan<N>::r0, TX>(src, dst, tw, Ns, sign);
  __syncthreads();
  { C* t = src; src = dst; dst = t; } Ns *= Plan<N>::r0;
  if constexpr (Plan<N>::n > 1) {
    stage<C, N, Plan<N>::r1, TX>(src, dst, tw, Ns, sign);
    __syncthreads();
    { C* t = src; src = dst; dst = t; } Ns *= Plan<N>::r1;
  }
  if constexpr (Plan<N>::n > 2) {
    stage<C, N, Plan<N>::r2, TX>(src, dst, tw, Ns, sign);
    __syncthreads();
    { C* t = src; src = dst; dst = t; }
  }
  return src;
}

template <typename T, int N>
__global__ void __launch_bounds__(256) fft_axis_kernel(cplx<T>* __restrict__ data, int axis,
                                                      int sign, const cplx<T>* __restrict__ table) {
  using C = cplx<T>;
  constexpr int TX = Plan<N>::TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + TX * Pad<N>::LS;
  C* tw = buf1 + TX * Pad<N>::LS;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    C t = table[i];
    if (sign > 0) t.y = -t.y;
    tw[i] = t;
  }
  const long n3 = (long)N * N * N;
  long base, sk, si;
  if (axis == 0) {
    base = (long)blockIdx.x * TX * N; sk = 1; si = N;
  } else {
    constexpr int nxt = N / TX;
    long t = blockIdx.x;
    const int xt = (int)(t % nxt); t /= nxt;
    const int o = (int)(t % N);
    const long b = t / N;
    if (axis == 1) { base = b * n3 + (long)o * N * N + xt * TX; sk = N; }
    else { base = b * n3 + (long)o * N + xt * TX; sk = (long)N * N; }
    si = 1;
  }
  for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
    int i, k;
    if (axis == 0) { i = e / N; k = e - i * N; } else { k = e / TX; i = e - k * TX; }
    buf0[sidx<N>(i, k)] = data[base + i * si + k * sk];
  }
  __syncthreads();
  const C* src = line_fft<C, N>(buf0, buf1, tw, sign);
  for (int e = threadIdx.x; e < TX * N; e += blockDim.x) {
    int i, k;
    if (axis == 0) { i = e / N; k = e - i * N; } else { k = e / TX; i = e - k * TX; }
    data[base + i * si + k * sk] = src[sidx<N>(i, k)];
  }
}

template <typename T, int N>
static cudaError_t launch_fft3d(cplx<T>* data, long n_batch, int sign, const cplx<T>* table,
                                cudaStream_t st) {
  constexpr int TX = Plan<N>::TX;
  const size_t smem = (size_t)(2 * TX * Pad<N>::LS + N) * sizeof(cplx<T>);
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  cudaError_t e0 = once_status(once, once_st, [&] {
    return cudaFuncSetAttribute(fft_axis_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e0 != cudaSuccess) return e0;
  const long blocks = n_batch * (long)N * N / TX;
  if (blocks <= 0) return cudaSuccess;
  for (int axis = 0; axis < 3; ++axis) {
    fft_axis_kernel<T, N><<<(unsigned)blocks, 256, smem, st>>>(data, axis, sign, table); note_launch();
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft3d(cplx<T>* data, long n_batch, int N, int sign, const cplx<T>* table,
                  cudaStream_t st) {
  switch (N) {
    case 16: return launch_fft3d<T, 16>(data, n_batch, sign, table, st);
    case 32: return launch_fft3d<T, 32>(data, n_batch, sign, table, st);
    case 48: return launch_fft3d<T, 48>(data, n_batch, sign, table, st);
    case 64: return launch_fft3d<T, 64>(data, n_batch, sign, table, st);
    case 72: return launch_fft3d<T, 72>(data, n_batch, sign, table, st);
    case 96: return launch_fft3d<T, 96>(data, n_batch, sign, table, st);
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t fft3d<float>(float2*, long, int, int, const float2*, cudaStream_t);
template cudaError_t fft3d<double>(double2*, long, int, int, const double2*, cudaStream_t);

// ---------------------------------------------------------------------------------
// Pruned transforms between the plane-wave sphere and the grid.
//
// A field on the sphere occupies few grid lines: its (x, y) columns form a disc and its
// x values a band of at most N/2. The sphere -> grid transform therefore runs z lines
// only for the sphere's columns, y lines only for x in the band, and x lines for the
// whole grid; the grid -> sphere transform runs the same lines in the opposite order,
// keeping only what the next pass reads. Per complex grid g the compact stages are
//   S [NS]          the full sphere (+G and -G), ordered by column, then z
//   I1[N][NC]       z-transformed columns             (z, column)
//   I2[N][N][NX]    y-transformed band                (z, y, x slot)
// and each transformed line is exactly the zero-padded full-grid line's transform. Where a
// z plane (two copies) fits in shared memory, the y and x passes run fused, one CTA per
// plane, and I2 is never written.
// ---------------------------------------------------------------------------------

template <typename C, int N>
__device__ __forceinline__ void load_twiddles(C* tw, const C* table, int sign) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    C t = table[i];
    if (sign > 0) t.y = -t.y;
    tw[i] = t;
  }
}

template <typename C, int N>
__device__ __forceinline__ void zero_lines(C* buf) {
  for (int e = threadIdx.x; e < Plan<N>::TX * Pad<N>::LS; e += blockDim.x) buf[e] = cmk<C>(0, 0);
}

// z lines of the sphere's columns. inverse: S -> I1; forward: I1 -> S
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) sph_z_kernel(cplx<T>* __restrict__ S, cplx<T>* __restrict__ I1,
                                                   SphereMap m, int sign, const cplx<T>* __restrict__ table) {
  using C = cplx<T>;
  constexpr int TL = Plan<N>::TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + TL * Pad<N>::LS;
  C* tw = buf1 + TL * Pad<N>::LS;
  load_twiddles<C, N>(tw, table, sign);
  const int nt = (m.NC + TL - 1) / TL;
  const long g = blockIdx.x / nt;
  const int c0 = (int)(blockIdx.x % nt) * TL;
  const int nl = min(TL, m.NC - c0);
  const int j0 = m.cstart[c0], j1 = m.cstart[c0 + nl];
  C* Sg = S + g * m.NS;
  C* I1g = I1 + g * (long)N * m.NC;
  if (INV) {
    zero_lines<C, N>(buf0);
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) buf0[sidx<N>(m.jcol[j] - c0, m.zs[j])] = Sg[j];
  } else {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e % TL, z = e / TL;
      buf0[sidx<N>(l, z)] = (l < nl) ? I1g[(long)z * m.NC + c0 + l] : cmk<C>(0, 0);
    }
  }
  __syncthreads();
  const C* src = line_fft<C, N>(buf0, buf1, tw, sign);
  if (INV) {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e % TL, z = e / TL;
      if (l < nl) I1g[(long)z * m.NC + c0 + l] = src[sidx<N>(l, z)];
    }
  } else {
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) Sg[j] = src[sidx<N>(m.jcol[j] - c0, m.zs[j])];
  }
}

// y lines of the band. inverse: I1 -> I2; forward: I2 -> I1
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) sph_y_kernel(cplx<T>* __restrict__ I1, cplx<T>* __restrict__ I2,
                                                   SphereMap m, int sign, const cplx<T>* __restrict__ table) {
  using C = cplx<T>;
  constexpr int TL = Plan<N>::TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + TL * Pad<N>::LS;
  C* tw = buf1 + TL * Pad<N>::LS;
  load_twiddles<C, N>(tw, table, sign);
  const int nt = (m.NX + TL - 1) / TL;
  const long gz = blockIdx.x / nt;                   // g * N + z
  const int x0 = (int)(blockIdx.x % nt) * TL;
  const int nl = min(TL, m.NX - x0);
  const int ca = m.xcol[x0], cb = m.xcol[x0 + nl];
  C* I1r = I1 + gz * m.NC;                           // I1[g][z][.]
  C* I2r = I2 + gz * (long)N * m.NX;                 // I2[g][z][.][.]
  if (INV) {
    zero_lines<C, N>(buf0);
    __syncthreads();
    for (int c = ca + threadIdx.x; c < cb; c += blockDim.x) buf0[sidx<N>(m.cxi[c] - x0, m.cy[c])] = I1r[c];
  } else {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e % TL, y = e / TL;
      buf0[sidx<N>(l, y)] = (l < nl) ? I2r[(long)y * m.NX + x0 + l] : cmk<C>(0, 0);
    }
  }
  __syncthreads();
  const C* src = line_fft<C, N>(buf0, buf1, tw, sign);
  if (INV) {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e % TL, y = e / TL;
      if (l < nl) I2r[(long)y * m.NX + x0 + l] = src[sidx<N>(l, y)];
    }
  } else {
    for (int c = ca + threadIdx.x; c < cb; c += blockDim.x) I1r[c] = src[sidx<N>(m.cxi[c] - x0, m.cy[c])];
  }
}

// x lines of the whole grid. inverse: I2 -> grid; forward: grid -> I2
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(256) sph_x_kernel(cplx<T>* __restrict__ I2, cplx<T>* __restrict__ grid,
                                                   SphereMap m, int sign, const cplx<T>* __restrict__ table) {
  using C = cplx<T>;
  constexpr int TL = Plan<N>::TX;
  static_assert(N % TL == 0, "line tile");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + TL * Pad<N>::LS;
  C* tw = buf1 + TL * Pad<N>::LS;
  load_twiddles<C, N>(tw, table, sign);
  constexpr int nt = N / TL;
  const long gz = blockIdx.x / nt;
  const int y0 = (int)(blockIdx.x % nt) * TL;
  C* I2r = I2 + (gz * N + y0) * m.NX;                // I2[g][z][y0 + l][xi]
  C* Gr = grid + (gz * N + y0) * N;                  // grid[g][z][y0 + l][x]
  if (INV) {
    zero_lines<C, N>(buf0);
    __syncthreads();
    for (int e = threadIdx.x; e < TL * m.NX; e += blockDim.x) {
      const int l = e / m.NX, xi = e - l * m.NX;
      buf0[sidx<N>(l, m.xs[xi])] = I2r[e];
    }
  } else {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e / N, x = e - l * N;
      buf0[sidx<N>(l, x)] = Gr[e];
    }
  }
  __syncthreads();
  const C* src = line_fft<C, N>(buf0, buf1, tw, sign);
  if (INV) {
    for (int e = threadIdx.x; e < TL * N; e += blockDim.x) {
      const int l = e / N, x = e - l * N;
      Gr[e] = src[sidx<N>(l, x)];
    }
  } else {
    for (int e = threadIdx.x; e < TL * m.NX; e += blockDim.x) {
      const int l = e / m.NX, xi = e - l * m.NX;
      I2r[e] = src[sidx<N>(l, m.xs[xi])];
    }
  }
}

// ---- fused y + x passes: one CTA per (grid, z plane) ----
// Two-stage radix plans (N = R0 * R1), so a plane needs one out-of-place row stage in
// shared memory. Composite radices 6, 9 and 12 run as two small DFTs in registers with
// twiddles taken from the N-point table.
template <int N> struct Plan2;
template <> struct Plan2<16> { static constexpr int r0 = 4, r1 = 4; };
template <> struct Plan2<32> { static constexpr int r0 = 8, r1 = 4; };
template <> struct Plan2<48> { static constexpr int r0 = 8, r1 = 6; };
template <> struct Plan2<64> { static constexpr int r0 = 8, r1 = 8; };
template <> struct Plan2<72> { static constexpr int r0 = 8, r1 = 9; };
template <> struct Plan2<96> { static constexpr int r0 = 8, r1 = 12; };

// X[k1 + A k2] = sum_n v[n] w^(n k), w = exp(sign 2 pi i / (A B)), n = B n1 + n2; tw[m] is
// exp(sign 2 pi i m / N) and A B divides N
template <typename C, int A, int B, int N>
__device__ __forceinline__ void dft_composite(C* v, int sign, const C* tw) {
  constexpr int R = A * B;
  C y[R];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
    C t[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) t[n1] = v[B * n1 + n2];
    Dft<C, A>::run(t, sign);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = (n2 * k1 == 0) ? t[k1] : cmul(t[k1], tw[(n2 * k1 * (N / R)) % N]);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
    Dft<C, B>::run(t, sign);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
  }
}

template <typename C, int R, int N>
__device__ __forceinline__ void dft_any(C* v, int sign, const C* tw) {
  if constexpr (R == 6) dft_composite<C, 2, 3, N>(v, sign, tw);
  else if constexpr (R == 9) dft_composite<C, 3, 3, N>(v, sign, tw);
  else if constexpr (R == 12) dft_composite<C, 4, 3, N>(v, sign, tw);
  else Dft<C, R>::run(v, sign);
}

// Plane-kernel line addressing: element q of line l at l * PLS + q + q / 32, with an odd
// line stride PLS. Stages between shared buffers run with consecutive lanes on consecutive
// lines (LF: lines fast), so every such access steps by PLS or by one element and stays
// free of bank conflicts; only a stage that reads or writes global memory runs with
// consecutive lanes along the line, for coalescing. (A bank-conflict count of the stages'
// access patterns over candidate paddings picked this layout.)
template <int N> struct PPad { static constexpr int LS = (N + (N >> 5) + 1) | 1; };
template <int N>
__device__ __forceinline__ int lidx(int l, int q) { return l * PPad<N>::LS + q + (q >> 5); }

// One Stockham stage of radix R over n_lines lines of length N, Ns = product of the
// earlier radices. Load / store go through functors ld(line, q) and st(line, q, value).
template <typename C, int N, int R, bool LF, typename LD, typename ST>
__device__ __forceinline__ void pstage(int Ns, int sign, int n_lines, const C* tw, LD ld, ST st) {
  constexpr int NB = N / R;
  const int step = N / (Ns * R);
  for (int e = threadIdx.x; e < n_lines * NB; e += blockDim.x) {
    int i, j;
    if (LF) { j = e / n_lines; i = e - j * n_lines; } else { i = e / NB; j = e - i * NB; }
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(i, j + r * NB);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[(r * k * step) % N]);
    dft_any<C, R, N>(v, sign, tw);
    const int o = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(i, o + r * Ns, v[r]);
  }
}

// rows of the buffer shared by column buffer B and the row block of the x passes: the x lines of
// a plane run in XH passes of N / XH rows each
template <int N, int XH>
constexpr int plane_rows() { return (N / XH > N / 2 + 1) ? N / XH : N / 2 + 1; }

template <typename T, int N, int XH = 1>
constexpr size_t plane_smem_base() {
  // column buffer A [NX <= N/2 + 1 slots] + (column buffer B | row block P) + twiddles + slots
  constexpr int NXM = N / 2 + 1;
  return (size_t)(NXM * PPad<N>::LS + plane_rows<N, XH>() * PPad<N>::LS + N) * sizeof(cplx<T>) +
         (size_t)N * sizeof(int);
}
// plus, for the inverse, the prefetched columns of the next plane (NC values)
template <typename T, int N, int XH = 1>
size_t plane_smem(bool inverse, int NC) {
  return plane_smem_base<T, N, XH>() + (inverse ? (size_t)NC * sizeof(cplx<T>) + 16 : 0);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_groups() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// inverse: I1[g][z][.] (z-transformed columns) -> grid plane (g, z); forward: the reverse.
// Column buffers hold the band's x slots as lines over y; the row plane holds lines over x.
// Persistent: a CTA takes planes gz = blockIdx.x, blockIdx.x + gridDim.x, ... of the n_planes
// (g, z) planes. Twiddles and x slots are set up once per CTA; in the inverse the next
// plane's columns are copied (cp.async, 16 bytes per copy where aligned) into a prefetch
// buffer while the current plane is transformed.
// threads of a plane CTA: 512 on the 96^3 grid (a 96-point line stage has 768 to 1,152
// butterflies; two such CTAs per SM measured fastest), 256 elsewhere
template <int N> constexpr int plane_threads() { return N >= 96 ? 512 : 256; }

// x passes per plane: two on the 96^3 grid in single precision, where the half-height row block
// leaves room for two CTAs per SM (forward 15.6 -> 13.0 ms, inverse 14.4 -> 12.9 ms per 6-vector
// launch of the large workload); one elsewhere (two measured within 2% on the 72^3 grid)
template <typename T, int N> constexpr int plane_xh() { return (N >= 96 && sizeof(T) == 4) ? 2 : 1; }

template <typename T, int N, bool INV, int XH = 1>
__global__ void __launch_bounds__(plane_threads<N>())
    sph_plane_kernel(cplx<T>* __restrict__ I1, cplx<T>* __restrict__ grid, SphereMap m, int sign,
                     const cplx<T>* __restrict__ table, long n_planes) {
  using C = cplx<T>;
  constexpr int R0 = Plan2<N>::r0, R1 = Plan2<N>::r1;
  constexpr int NXM = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* colA = reinterpret_cast<C*>(smem_raw);          // [NXM][LS]
  C* colB = colA + NXM * PPad<N>::LS;                // [NXM][LS], shares space with P
  C* P = colB;                                       // [N / XH][LS]
  C* tw = P + plane_rows<N, XH>() * PPad<N>::LS;
  int* slot = reinterpret_cast<int*>(tw + N);        // slot of x in the band, -1 outside
  C* pre = reinterpret_cast<C*>(smem_raw + ((plane_smem_base<T, N, XH>() + 15) & ~(size_t)15));  // [NC], inverse
  constexpr int NY = N / XH;                         // rows of one x pass
  load_twiddles<C, N>(tw, table, sign);
  for (int x = threadIdx.x; x < N; x += blockDim.x) slot[x] = -1;
  __syncthreads();
  for (int l = threadIdx.x; l < m.NX; l += blockDim.x) slot[m.xs[l]] = l;
  const int nx = m.NX;
  // the columns of plane gz into the prefetch buffer (16-byte copies when the row is aligned)
  auto prefetch = [&](long gz) {
    const C* src = I1 + gz * m.NC;
    if (sizeof(C) == 8 && (m.NC & 1) == 0) {
      for (int c = 2 * threadIdx.x; c < m.NC; c += 2 * blockDim.x) cp_async16(pre + c, src + c);
    } else if (sizeof(C) == 16) {
      for (int c = threadIdx.x; c < m.NC; c += blockDim.x) cp_async16(pre + c, src + c);
    } else {
      for (int c = threadIdx.x; c < m.NC; c += blockDim.x) cp_async8(pre + c, src + c);
    }
    cp_async_commit_all();
  };
  long gz = blockIdx.x;
  if (INV && gz < n_planes) prefetch(gz);
  for (; gz < n_planes; gz += gridDim.x) {
    C* I1r = I1 + gz * m.NC;
    C* Gp = grid + gz * (long)N * N;
    if (INV) {
      for (int e = threadIdx.x; e < nx * PPad<N>::LS; e += blockDim.x) colA[e] = cmk<C>(0, 0);
      cp_async_wait_all_groups();
      __syncthreads();
      for (int c = threadIdx.x; c < m.NC; c += blockDim.x) colA[lidx<N>(m.cxi[c], m.cy[c])] = pre[c];
      __syncthreads();
      if (gz + gridDim.x < n_planes) prefetch(gz + gridDim.x);
      // y lines of the band: A -> B -> A
      pstage<C, N, R0, true>(1, sign, nx, tw, [&](int l, int q) { return colA[lidx<N>(l, q)]; },
                             [&](int l, int q, C v) { colB[lidx<N>(l, q)] = v; });
      __syncthreads();
      pstage<C, N, R1, true>(R0, sign, nx, tw, [&](int l, int q) { return colB[lidx<N>(l, q)]; },
                             [&](int l, int q, C v) { colA[lidx<N>(l, q)] = v; });
      __syncthreads();
      // x lines, NY rows per pass: the first stage reads the band from the column buffer (zero
      // outside it), the second writes the rows to global memory
#pragma unroll 1
      for (int h = 0; h < XH; ++h) {
        const int y0 = h * NY;
        pstage<C, N, R0, true>(1, sign, NY, tw,
                               [&](int y, int x) { const int s = slot[x]; return s >= 0 ? colA[lidx<N>(s, y0 + y)] : cmk<C>(0, 0); },
                               [&](int y, int x, C v) { P[lidx<N>(y, x)] = v; });
        __syncthreads();
        pstage<C, N, R1, false>(R0, sign, NY, tw, [&](int y, int x) { return P[lidx<N>(y, x)]; },
                                [&](int y, int x, C v) { Gp[(y0 + y) * N + x] = v; });
        if (h + 1 < XH) __syncthreads();             // the next pass overwrites P
      }
    } else {
      __syncthreads();                                // the previous plane's gather is done with colA
      // x lines, NY rows per pass: the first stage reads the rows from global memory, the
      // second keeps the band
#pragma unroll 1
      for (int h = 0; h < XH; ++h) {
        const int y0 = h * NY;
        pstage<C, N, R0, false>(1, sign, NY, tw, [&](int y, int x) { return Gp[(y0 + y) * N + x]; },
                                [&](int y, int x, C v) { P[lidx<N>(y, x)] = v; });
        __syncthreads();
        pstage<C, N, R1, true>(R0, sign, NY, tw, [&](int y, int x) { return P[lidx<N>(y, x)]; },
                               [&](int y, int x, C v) { const int s = slot[x]; if (s >= 0) colA[lidx<N>(s, y0 + y)] = v; });
        __syncthreads();
      }
      // y lines of the band: A -> B -> A
      pstage<C, N, R0, true>(1, sign, nx, tw, [&](int l, int q) { return colA[lidx<N>(l, q)]; },
                             [&](int l, int q, C v) { colB[lidx<N>(l, q)] = v; });
      __syncthreads();
      pstage<C, N, R1, true>(R0, sign, nx, tw, [&](int l, int q) { return colB[lidx<N>(l, q)]; },
                             [&](int l, int q, C v) { colA[lidx<N>(l, q)] = v; });
      __syncthreads();
      for (int c = threadIdx.x; c < m.NC; c += blockDim.x) I1r[c] = colA[lidx<N>(m.cxi[c], m.cy[c])];
    }
  }
}

template <typename T, int N>
static cudaError_t launch_pruned(bool inverse, cplx<T>* S, cplx<T>* I1, cplx<T>* I2, cplx<T>* grid,
                                 long n_grids, const SphereMap& m, const cplx<T>* table, cudaStream_t st) {
  constexpr int TL = Plan<N>::TX;
  const size_t smem = (size_t)(2 * TL * Pad<N>::LS + N) * sizeof(cplx<T>);
  constexpr int XH = plane_xh<T, N>();
  constexpr int PNT = plane_threads<N>();
  const size_t psmem = plane_smem<T, N, XH>(inverse, m.NC);
  constexpr bool use_plane = plane_smem_base<T, N, XH>() <= 200 * 1024;
  static std::once_flag once;
  static cudaError_t once_st = cudaSuccess;
  static int n_sm = 0;
  cudaError_t e0 = once_status(once, once_st, [&] {
    cudaError_t e = cudaSuccess;
    const void* ks[6] = {(const void*)sph_z_kernel<T, N, true>, (const void*)sph_z_kernel<T, N, false>,
                         (const void*)sph_y_kernel<T, N, true>, (const void*)sph_y_kernel<T, N, false>,
                         (const void*)sph_x_kernel<T, N, true>, (const void*)sph_x_kernel<T, N, false>};
    for (const void* k : ks)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if constexpr (use_plane) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sph_plane_kernel<T, N, true, XH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sph_plane_kernel<T, N, false, XH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    }
    if (e == cudaSuccess) {
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    return e;
  });
  if (e0 != cudaSuccess) return e0;
  // persistent plane kernels: as many CTAs as fit on the device at this shared-memory size
  long plane_grid = 0;
  if constexpr (use_plane) {
    if (psmem > 220 * 1024) return cudaErrorInvalidValue;
    int occ = 0;
    static std::mutex mu;
    static std::map<std::pair<bool, size_t>, int> occ_of;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = occ_of.find(std::make_pair(inverse, psmem));
      if (it == occ_of.end()) {
        cudaError_t e = inverse ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sph_plane_kernel<T, N, true, XH>, PNT, psmem)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sph_plane_kernel<T, N, false, XH>, PNT, psmem);
        if (e != cudaSuccess) return e;
        occ_of[std::make_pair(inverse, psmem)] = occ;
      } else {
        occ = it->second;
      }
    }
    if (occ < 1) return cudaErrorInvalidValue;
    plane_grid = std::min<long>(n_grids * N, (long)occ * n_sm);
  }
  if (n_grids <= 0) return cudaSuccess;
  const long bz = n_grids * ((m.NC + TL - 1) / TL);
  const long by = n_grids * N * ((m.NX + TL - 1) / TL);
  const long bx = n_grids * N * (N / TL);
  const long bp = n_grids * N;
  if (inverse) {
    sph_z_kernel<T, N, true><<<(unsigned)bz, 256, smem, st>>>(S, I1, m, +1, table); note_launch();
    if constexpr (use_plane) {
      sph_plane_kernel<T, N, true, XH><<<(unsigned)plane_grid, PNT, psmem, st>>>(I1, grid, m, +1, table, bp);
      note_launch();
    } else {
      sph_y_kernel<T, N, true><<<(unsigned)by, 256, smem, st>>>(I1, I2, m, +1, table); note_launch();
      sph_x_kernel<T, N, true><<<(unsigned)bx, 256, smem, st>>>(I2, grid, m, +1, table); note_launch();
    }
  } else {
    if constexpr (use_plane) {
      sph_plane_kernel<T, N, false, XH><<<(unsigned)plane_grid, PNT, psmem, st>>>(I1, grid, m, -1, table, bp);
      note_launch();
    } else {
      sph_x_kernel<T, N, false><<<(unsigned)bx, 256, smem, st>>>(I2, grid, m, -1, table); note_launch();
      sph_y_kernel<T, N, false><<<(unsigned)by, 256, smem, st>>>(I1, I2, m, -1, table); note_launch();
    }
    sph_z_kernel<T, N, false><<<(unsigned)bz, 256, smem, st>>>(S, I1, m, -1, table); note_launch();
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pruned(bool inverse, cplx<T>* S, cplx<T>* I1, cplx<T>* I2, cplx<T>* grid, long n_grids,
                          int N, const SphereMap& m, const cplx<T>* table, cudaStream_t st) {
  switch (N) {
    case 16: return launch_pruned<T, 16>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    case 32: return launch_pruned<T, 32>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    case 48: return launch_pruned<T, 48>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    case 64: return launch_pruned<T, 64>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    case 72: return launch_pruned<T, 72>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    case 96: return launch_pruned<T, 96>(inverse, S, I1, I2, grid, n_grids, m, table, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t sphere_scratch_per_grid(int N, const SphereMap& m) {
  return (size_t)m.NS + (size_t)N * m.NC + (size_t)N * N * m.NX;
}

// packed fields (two per complex grid) -> real-space grids, unnormalised sign +1 transform.
// scratch: n_grids * sphere_scratch_per_grid complex values, disjoint from grids.
template <typename T>
cudaError_t sphere_to_grid(const T* P, long n_fields, int n_pw, int n_half, int N, const SphereMap& m,
                           const cplx<T>* table, cplx<T>* scratch, cplx<T>* grids, cudaStream_t st) {
  const long ng = (n_fields + 1) / 2;
  if (ng == 0) return cudaSuccess;
  cplx<T>* S = scratch;
  cplx<T>* I1 = S + ng * m.NS;
  cplx<T>* I2 = I1 + ng * (long)N * m.NC;
  cudaError_t e = sphere_unpack<T, T>(P, n_fields, n_pw, n_half, m.fpos, m.fneg, S, m.NS, false, false, st);
  if (e != cudaSuccess) return e;
  return pruned<T>(true, S, I1, I2, grids, ng, N, m, table, st);
}

// real-space grids (read only) -> packed fields: scale * sphere values plus the optional
// diagonal term of sphere_pack; sign -1 transform.
template <typename T>
cudaError_t grid_to_sphere(cplx<T>* grids, long n_fields, int n_pw, int n_half, int N, const SphereMap& m,
                           const cplx<T>* table, cplx<T>* scratch, double scale, T* out, const T* add_in,
                           const T* g2h, const T* esh, int n_occ, cudaStream_t st) {
  const long ng = (n_fields + 1) / 2;
  if (ng == 0) return cudaSuccess;
  cplx<T>* S = scratch;
  cplx<T>* I1 = S + ng * m.NS;
  cplx<T>* I2 = I1 + ng * (long)N * m.NC;
  cudaError_t e = pruned<T>(false, S, I1, I2, grids, ng, N, m, table, st);
  if (e != cudaSuccess) return e;
  return sphere_pack<T, T>(S, n_fields, n_pw, n_half, m.fpos, m.fneg, m.NS, scale, out, add_in, g2h, esh,
                           n_occ, st);
}

template cudaError_t sphere_to_grid<float>(const float*, long, int, int, int, const SphereMap&, const float2*, float2*, float2*, cudaStream_t);
template cudaError_t sphere_to_grid<double>(const double*, long, int, int, int, const SphereMap&, const double2*, double2*, double2*, cudaStream_t);
template cudaError_t grid_to_sphere<float>(float2*, long, int, int, int, const SphereMap&, const float2*, float2*, double, float*, const float*, const float*, const float*, int, cudaStream_t);
template cudaError_t grid_to_sphere<double>(double2*, long, int, int, int, const SphereMap&, const double2*, double2*, double, double*, const double*, const double*, const double*, int, cudaStream_t);

// Column-ordered sphere from Miller indices (host): +G_k and -G_k (k > 0) sorted by
// (x slot, y, z) with x slots the sorted distinct x grid indices.
void build_sphere_map(int N, int n_half, const int* miller, SphereMapHost& h) {
  auto wrap = [N](int v) { return ((v % N) + N) % N; };
  struct Pt { int x, y, z, k, neg; };
  std::vector<Pt> pts;
  pts.reserve(2 * (size_t)n_half);
  for (int k = 0; k < n_half; ++k) {
    const int* q = miller + 3 * k;
    pts.push_back({wrap(q[0]), wrap(q[1]), wrap(q[2]), k, 0});
    if (k > 0) pts.push_back({wrap(-q[0]), wrap(-q[1]), wrap(-q[2]), k, 1});
  }
  std::sort(pts.begin(), pts.end(), [](const Pt& a, const Pt& b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
  h.NS = (int)pts.size();
  h.fpos.assign(n_half, -1);
  h.fneg.assign(n_half, -1);
  h.zs.resize(h.NS);
  h.jcol.resize(h.NS);
  h.cstart.clear(); h.cy.clear(); h.cxi.clear(); h.xs.clear(); h.xcol.clear();
  for (int j = 0; j < h.NS; ++j) {
    const Pt& p = pts[j];
    const bool new_x = (j == 0) || p.x != pts[j - 1].x;
    const bool new_c = new_x || p.y != pts[j - 1].y;
    if (new_x) { h.xs.push_back(p.x); h.xcol.push_back((int)h.cy.size()); }
    if (new_c) { h.cstart.push_back(j); h.cy.push_back(p.y); h.cxi.push_back((int)h.xs.size() - 1); }
    h.zs[j] = p.z;
    h.jcol[j] = (int)h.cy.size() - 1;
    (p.neg ? h.fneg : h.fpos)[p.k] = j;
  }
  h.NC = (int)h.cy.size();
  h.NX = (int)h.xs.size();
  h.cstart.push_back(h.NS);
  h.xcol.push_back(h.NC);
  if (h.fneg[0] < 0) h.fneg[0] = h.fpos[0];
}

bool fft_supported(int N) {
  return N == 16 || N == 32 || N == 48 || N == 64 || N == 72 || N == 96;
}

// exp(-2 pi i m / N), m = 0..N-1, computed on the host in double precision
void twiddle_table(int N, std::vector<double2>& out) {
  out.resize(N);
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < N; ++m) {
    const double a = two_pi * (double)m / (double)N;
    out[m].x = std::cos(a);
    out[m].y = -std::sin(a);
  }
}

// ---------------------------------------------------------------------------------
// sphere scatter / gather
// ---------------------------------------------------------------------------------

// grids[c] (pre-zeroed) <- F = A + iB with A, B the packed fields 2c, 2c+1 (B = 0 if absent)
template <typename T, typename TI>
__global__ void sphere_unpack_kernel(const TI* __restrict__ P, long n_fields, int n_pw, int n_half,
                                     const int* __restrict__ gpos, const int* __restrict__ gneg,
                                     cplx<T>* __restrict__ grids, long n3, int accumulate) {
  using C = cplx<T>;
  const long n_c = (n_fields + 1) / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_half) return;
  for (long c = blockIdx.y; c < n_c; c += gridDim.y) {
  const long fa = 2 * c, fb = 2 * c + 1;
  const bool hb = fb < n_fields;
  const T a0 = (T)P[fa * n_pw + 2 * k], a1 = (T)P[fa * n_pw + 2 * k + 1];
  const T b0 = hb ? (T)P[fb * n_pw + 2 * k] : (T)0, b1 = hb ? (T)P[fb * n_pw + 2 * k + 1] : (T)0;
  C* g = grids + c * n3;
  if (k == 0) {
    C F; F.x = a0; F.y = b0;
    if (accumulate) F = cadd(g[gpos[0]], F);
    g[gpos[0]] = F;
    continue;
  }
  const T s = (T)0.70710678118654752440;
  // cA = (a0 + i a1)/sqrt2, cB = (b0 + i b1)/sqrt2
  const T ax = a0 * s, ay = a1 * s, bx = b0 * s, by = b1 * s;
  C Fp, Fm;
  Fp.x = ax - by; Fp.y = ay + bx;       // cA + i cB
  Fm.x = ax + by; Fm.y = -ay + bx;      // conj(cA) + i conj(cB)
  if (accumulate) { Fp = cadd(g[gpos[k]], Fp); Fm = cadd(g[gneg[k]], Fm); }
  g[gpos[k]] = Fp;
  g[gneg[k]] = Fm;
  }
}

// packed fields 2c, 2c+1 <- scale * grids[c] on the sphere (Hermitian separation), plus
// the optional diagonal term (g2h[j] + esh[f % n_occ]) * add_in[f] with g2h = 1/2|G|^2 per
// packed coordinate and esh_v = Delta - eps_v (Eq. d).
template <typename T, typename TO>
__global__ void sphere_pack_kernel(const cplx<T>* __restrict__ grids, long n_fields, int n_pw,
                                   int n_half, const int* __restrict__ gpos,
                                   const int* __restrict__ gneg, long n3, double scale,
                                   TO* __restrict__ out, const TO* __restrict__ add_in,
                                   const T* __restrict__ g2h, const T* __restrict__ esh, int n_occ) {
  using C = cplx<T>;
  const long n_c = (n_fields + 1) / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_half) return;
  for (long c = blockIdx.y; c < n_c; c += gridDim.y) {
  const C* g = grids + c * n3;
  const T sc = (T)scale;
  C Fp = g[gpos[k]];
  Fp.x *= sc; Fp.y *= sc;
  T a0, a1, b0, b1;
  if (k == 0) {
    a0 = Fp.x; a1 = 0; b0 = Fp.y; b1 = 0;
  } else {
    C Fm = g[gneg[k]];
    Fm.x *= sc; Fm.y *= sc;
    const T r2 = (T)1.41421356237309504880;
    // cA = (Fp + conj Fm)/2, cB = (Fp - conj Fm)/(2i)
    a0 = (T)0.5 * (Fp.x + Fm.x) * r2;
    a1 = (T)0.5 * (Fp.y - Fm.y) * r2;
    b0 = (T)0.5 * (Fp.y + Fm.y) * r2;
    b1 = (T)(-0.5) * (Fp.x - Fm.x) * r2;
  }
  const long fa = 2 * c, fb = 2 * c + 1;
  const int j0 = 2 * k, j1 = 2 * k + 1;
  if (add_in) {
    const T ea = esh[fa % n_occ];
    a0 += (g2h[j0] + ea) * (T)add_in[fa * n_pw + j0];
    if (k) a1 += (g2h[j1] + ea) * (T)add_in[fa * n_pw + j1];
  }
  out[fa * n_pw + j0] = (TO)a0;
  out[fa * n_pw + j1] = (TO)a1;
  if (fb < n_fields) {
    if (add_in) {
      const T eb = esh[fb % n_occ];
      b0 += (g2h[j0] + eb) * (T)add_in[fb * n_pw + j0];
      if (k) b1 += (g2h[j1] + eb) * (T)add_in[fb * n_pw + j1];
    }
    out[fb * n_pw + j0] = (TO)b0;
    out[fb * n_pw + j1] = (TO)b1;
  }
  }
}

template <typename T, typename TI>
cudaError_t sphere_unpack(const TI* P, long n_fields, int n_pw, int n_half, const int* gpos,
                          const int* gneg, cplx<T>* grids, long n3, bool zero_first,
                          bool accumulate, cudaStream_t st) {
  const long n_c = (n_fields + 1) / 2;
  if (n_c == 0) return cudaSuccess;
  if (zero_first) {
    cudaError_t e = cudaMemsetAsync(grids, 0, (size_t)n_c * n3 * sizeof(cplx<T>), st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((n_half + 255) / 256), (unsigned)(n_c < 65535 ? n_c : 65535));
  sphere_unpack_kernel<T, TI><<<grid, 256, 0, st>>>(
      P, n_fields, n_pw, n_half, gpos, gneg, grids, n3, accumulate ? 1 : 0); note_launch();
  return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t sphere_pack(const cplx<T>* grids, long n_fields, int n_pw, int n_half, const int* gpos,
                        const int* gneg, long n3, double scale, TO* out, const TO* add_in,
                        const T* g2h, const T* esh, int n_occ, cudaStream_t st) {
  const long n_c = (n_fields + 1) / 2;
  if (n_c == 0) return cudaSuccess;
  dim3 grid((unsigned)((n_half + 255) / 256), (unsigned)(n_c < 65535 ? n_c : 65535));
  sphere_pack_kernel<T, TO><<<grid, 256, 0, st>>>(
      grids, n_fields, n_pw, n_half, gpos, gneg, n3, scale, out, add_in, g2h, esh, n_occ); note_launch();
  return cudaGetLastError();
}

template cudaError_t sphere_unpack<double, double>(const double*, long, int, int, const int*, const int*, double2*, long, bool, bool, cudaStream_t);
template cudaError_t sphere_unpack<float, float>(const float*, long, int, int, const int*, const int*, float2*, long, bool, bool, cudaStream_t);
template cudaError_t sphere_unpack<float, double>(const double*, long, int, int, const int*, const int*, float2*, long, bool, bool, cudaStream_t);
template cudaError_t sphere_pack<double, double>(const double2*, long, int, int, const int*, const int*, long, double, double*, const double*, const double*, const double*, int, cudaStream_t);
template cudaError_t sphere_pack<float, float>(const float2*, long, int, int, const int*, const int*, long, double, float*, const float*, const float*, const float*, int, cudaStream_t);

// ---------------------------------------------------------------------------------
// multiply complex grids by a real, even function of |G| (keeps field pairs separable)
//   mode 0: v(G)/Omega = 4 pi / (|G|^2 Omega), 0 at G = 0          (Hartree, Eq. k1e)
//   mode 1: v(G)^{1/2} = sqrt(4 pi) / |G|, 0 at G = 0               (Eq. tau_from_tau_u)
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void grid_coulomb_kernel(cplx<T>* __restrict__ grids, long n_grids, int N, double L,
                                    double omega, int mode, double scale) {
  const int n3 = N * N * N;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n3) return;
  // the factor depends on the point only: computed once, then applied to a stride of grids
  const int x = r % N, y = (r / N) % N, z = r / (N * N);
  const int nx = x < N / 2 ? x : x - N, ny = y < N / 2 ? y : y - N, nz = z < N / 2 ? z : z - N;
  const double g = 6.283185307179586476925286766559 / L;
  const double g2 = g * g * (double)(nx * nx + ny * ny + nz * nz);
  double f = 0.0;
  if (g2 > 0) f = (mode == 0) ? 12.566370614359172953850573533118 / (g2 * omega)
                              : 3.5449077018110320545963349666823 / sqrt(g2);
  const T ft = (T)(f * scale);
  for (long b = blockIdx.y; b < n_grids; b += gridDim.y) {
    cplx<T> v = grids[b * n3 + r];
    v.x *= ft; v.y *= ft;
    grids[b * n3 + r] = v;
  }
}

template <typename T>
cudaError_t grid_coulomb(cplx<T>* grids, long n_grids, int N, double L, double omega, int mode,
                         double scale, cudaStream_t st) {
  if (n_grids == 0) return cudaSuccess;
  const long n3 = (long)N * N * N;
  dim3 grid((unsigned)((n3 + 255) / 256), (unsigned)(n_grids < 8 ? n_grids : 8));
  grid_coulomb_kernel<T><<<grid, 256, 0, st>>>(grids, n_grids, N, L, omega, mode, scale); note_launch();
  return cudaGetLastError();
}
template cudaError_t grid_coulomb<float>(float2*, long, int, double, double, int, double, cudaStream_t);
template cudaError_t grid_coulomb<double>(double2*, long, int, double, double, int, double, cudaStream_t);

}  // namespace bse
