// Screened direct term K1d of Eq. (k1d), fused with the real-space parts of D (Eq. d)
// and K1e (Eq. k1e):
//
//   u_R,sv(r) = V_loc(r) u_a,sv(r) + s V_H,s(r) u_psi,v(r) - sum_{w in nbr(v)} tau_vw(r) u_a,sw(r)
//
// At each grid point the sum is a sparse (N_occ x N_occ) times dense (N_occ x n_vec)
// product whose sparse factor tau(r) changes from point to point, so no operand is shared
// across points and the work is SIMT multiply-adds fed from memory. A CTA owns a tile of
// TR consecutive points and a chunk of SC trial vectors:
//
//  * a(r) for every orbital of the chunk is copied into shared memory with cp.async
//    (no registers held, all copies in flight at once), laid out [w][t][s] so that a lane
//    reads the SC values it needs for orbital w as one or two 16-byte loads;
//  * groups of TR lanes (one lane per point; TR = 8, 16 or 32) walk row blocks of four orbitals (one
//    localisation site); each block lists the union of its rows' neighbours w (Eq. overlap);
//  * tau is stored entry-major: the four rows' values of one block entry at one point are
//    adjacent, so a lane fetches them with one 16-byte load (zeros stand in for rows
//    without that neighbour) and only the neighbour index w is broadcast in the group;
//  * tau values go straight from global memory to registers through a ring of PD entries,
//    so PD entries of loads are in flight per lane while the oldest one is consumed; tau is
//    point-tiled, so the tau a CTA reads is one contiguous stretch of memory (the ring
//    variants keep the entries in flight in shared memory instead, by cp.async, which frees
//    the registers: k1d_ring_kernel);
//  * each tau value feeds SC multiply-adds and each staged a value four, accumulated in
//    packed FP32x2 FMAs for single precision.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace bse {

namespace {

constexpr int K1D_PD = 8;                       // tau prefetch depth (entries per lane)
constexpr size_t K1D_SMEM_MAX = 220 * 1024;     // opt-in dynamic shared memory used at most

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// SC consecutive values from shared memory in 16-, 8- or 4-byte loads
template <typename T, int SC>
__device__ __forceinline__ void lds_vec(T (&v)[SC], const T* p) {
  constexpr int B = SC * (int)sizeof(T);
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int k = 0; k < B / 16; ++k) reinterpret_cast<uint4*>(v)[k] = reinterpret_cast<const uint4*>(p)[k];
  } else if constexpr (B == 8) {
    *reinterpret_cast<uint2*>(v) = *reinterpret_cast<const uint2*>(p);
  } else {
    v[0] = p[0];
  }
}

// Staged a(r) layout [w][s / CH][t][CH] with CH = 16 bytes of values: the CH values of one
// (orbital, point) chunk are one 16-byte load, and the eight lanes of a quarter-warp (eight
// consecutive points) read 128 contiguous bytes, free of bank conflicts.
template <typename T, int SC>
struct ALayout {
  static constexpr int CH = (SC * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : SC;
  static constexpr int NCH = SC / CH;
  // offset of chunk 0 of (w, t) given TR points per tile; chunk c is at + c * TR * CH
  template <int TR>
  __device__ __forceinline__ static size_t base(int w, int t) { return ((size_t)w * NCH * TR + t) * CH; }
};

// SC values of one (orbital, point) of the staged layout
template <typename T, int SC, int TR>
__device__ __forceinline__ void lds_a(T (&v)[SC], const T* A, int w, int t) {
  using L = ALayout<T, SC>;
  const T* p = A + L::template base<TR>(w, t);
#pragma unroll
  for (int c = 0; c < L::NCH; ++c) {
    T tmp[L::CH];
    lds_vec<T, L::CH>(tmp, p + (size_t)c * TR * L::CH);
#pragma unroll
    for (int q = 0; q < L::CH; ++q) v[c * L::CH + q] = tmp[q];
  }
}

// accumulators of one lane: four rows x SC vectors
template <typename T, int SC, bool PACKED = (sizeof(T) == 4 && SC % 2 == 0)>
struct RowAcc {
  T acc[4][SC];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int s = 0; s < SC; ++s) acc[i][s] = (T)0;
  }
  __device__ __forceinline__ void mac(const T (&tv)[4], const T (&av)[SC]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int s = 0; s < SC; ++s) acc[i][s] = fma(tv[i], av[s], acc[i][s]);
  }
  __device__ __forceinline__ T get(int i, int s) const { return acc[i][s]; }
};

template <int SC>
struct RowAcc<float, SC, true> {
  float2 acc[4][SC / 2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < SC / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void mac(const float (&tv)[4], const float (&av)[SC]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 ti = make_float2(tv[i], tv[i]);
#pragma unroll
      for (int j = 0; j < SC / 2; ++j)
        acc[i][j] = __ffma2_rn(ti, make_float2(av[2 * j], av[2 * j + 1]), acc[i][j]);
    }
  }
  __device__ __forceinline__ float get(int i, int s) const { return (s & 1) ? acc[i][s >> 1].y : acc[i][s >> 1].x; }
};

// group-wide broadcast of lane j's value (lanes of a group = TR consecutive lanes)
template <int TR>
__device__ __forceinline__ int gshfl(unsigned mask, int v, int j) { return __shfl_sync(mask, v, j, TR); }

// the four rows' tau of one entry at one point (16 bytes per 16-byte load)
template <typename T>
__device__ __forceinline__ void ld_tau4(T (&tv)[4], const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    tv[0] = q.x; tv[1] = q.y; tv[2] = q.z; tv[3] = q.w;
  } else {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    tv[0] = q0.x; tv[1] = q0.y; tv[2] = q1.x; tv[3] = q1.y;
  }
}

// CTAs per SM the register budget is sized for by default: two of 256 threads, one of 512,
// and one for the wide vector chunks (SC >= 12), whose accumulators want more than 128
// registers. Variant 14 holds 12-vector chunks to two CTAs per SM (two 96 KB a(r) stages fit):
// twice the tau loads in flight per SM, 8.1 against 10.4 ms for 12 vectors on the 72^3 x 256
// workload, where the kernel is bound by the loads in flight rather than by instructions
template <int SC, int NT>
constexpr int k1d_min_blocks() { return SC >= 12 ? 1 : 512 / NT; }

// L2 prefetch of a byte range (16-byte aligned start, size a multiple of 16): no registers
// or shared memory are held while the data moves
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// PF: the first CTA of each 32-point tau tile (first vector chunk) asks L2 for a group's
// next row block of tau (the whole tile's stretch of it) while the group works on the
// current one, and for the first block while a(r) is staged; the other CTAs of the tile and
// the other vector chunks then find it in L2
template <typename T, int TR, int SC, int NT, int MINB, bool PF = false>
__global__ void __launch_bounds__(NT, MINB) k1d_tile_kernel(
    int n_vec, int n_occ, long n3, const T* __restrict__ a, const T* __restrict__ tau4, long n_ent,
    const int* __restrict__ bptr, const int* __restrict__ bw, int n_blocks, const T* __restrict__ vloc,
    const T* __restrict__ vh, const T* __restrict__ upsi, T sf, T* __restrict__ out) {
  // ring depth (divides TR); half as deep in double precision, whose values take two registers
  constexpr int PD0 = (sizeof(T) == 8) ? K1D_PD / 2 : K1D_PD;
  constexpr int PD = (PD0 < TR) ? PD0 : TR;
  extern __shared__ __align__(16) unsigned char k1d_smem[];
  T* A = reinterpret_cast<T*>(k1d_smem);            // [n_occ][SC / CH][TR][CH]
  T* VH = A + (size_t)n_occ * TR * SC;               // [TR][SC]
  const int n_sc = (n_vec + SC - 1) / SC;
  const int chunk = blockIdx.x % n_sc;
  const long r0 = (long)(blockIdx.x / n_sc) * TR;
  const int s0 = chunk * SC;
  const int ns = min(SC, n_vec - s0);
  const int tid = threadIdx.x;
  const int t = tid % TR, g = tid / TR;
  constexpr int G = NT / TR;
  const long r = r0 + t;
  const bool leader = PF && t == 0 && chunk == 0 && (r0 % TAU_TB) == 0;
  const T* tau_tile = tau4 + tau4_off(0, r0 - r0 % TAU_TB, n_ent);
  auto prefetch_block = [&](int b) {
    const int f0 = __ldg(bptr + b), f1 = __ldg(bptr + b + 1);
    prefetch_l2(tau_tile + (size_t)f0 * 4 * TAU_TB, (unsigned)(f1 - f0) * 4u * TAU_TB * (unsigned)sizeof(T));
  };
  if (leader && g < n_blocks) prefetch_block(g);
  // stage a(field (s0+s, w), r0+t) in layout order, so the lanes of a warp fill
  // consecutive shared-memory words
  {
    using L = ALayout<T, SC>;
    const int n_items = n_occ * TR * SC;
    for (int it = tid; it < n_items; it += NT) {
      const int q = it % L::CH, tt = (it / L::CH) % TR, c = (it / (L::CH * TR)) % L::NCH;
      const int w = it / (SC * TR);
      const int s = c * L::CH + q;
      if (s < ns)
        cp_async<sizeof(T)>(A + it, a + pair_off<T>((long)(s0 + s) * n_occ + w, r0 + tt, n3));
    }
  }
  if (g < SC) VH[t * SC + g] = (g < ns) ? vh[pair_off<T>(s0 + g, r, n3)] : (T)0;
  cp_async_wait_all();
  __syncthreads();
  const T vl = vloc[r];
  const T* tau_r = tau4 + tau4_off(0, r, n_ent);     // entry e at tau_r[e * 4 TAU_TB]
  const unsigned gmask = (TR == 32) ? 0xffffffffu : (((1u << TR) - 1u) << ((tid & 31) & ~(TR - 1)));
  for (int rb = g; rb < n_blocks; rb += G) {
    if (leader && rb + G < n_blocks) prefetch_block(rb + G);
    RowAcc<T, SC> acc;
    acc.zero();
    const int e0 = bptr[rb], e1 = bptr[rb + 1];
    // neighbour indices in batches of TR: lane t of the group holds entry base + t. Three
    // batches are live (current, next, the one after), so an index load has more than a
    // batch of work to arrive before it is needed.
    auto ld_w = [&](int base) { const int e = base + t; return (e < e1) ? bw[e] : 0; };
    int wA = ld_w(e0), wB = ld_w(e0 + TR), wC;
    // ring of PD entries in flight: slot d holds tau (four rows) and the neighbour w
    T tq[PD][4];
    int wq[PD];
    auto issue = [&](int e, T (&tv)[4]) {
      if (e < e1) {
        ld_tau4<T>(tv, tau_r + (size_t)e * (4 * TAU_TB));
      } else {
        tv[0] = tv[1] = tv[2] = tv[3] = (T)0;
      }
    };
#pragma unroll
    for (int d = 0; d < PD; ++d) {
      wq[d] = gshfl<TR>(gmask, wA, d);
      issue(e0 + d, tq[d]);
    }
    for (int base = e0; base < e1; base += TR) {
      wC = ld_w(base + 2 * TR);
#pragma unroll
      for (int d = 0; d < TR; ++d) {
        if (base + d >= e1) break;
        const int sl = d % PD;
        T av[SC];
        lds_a<T, SC, TR>(av, A, wq[sl], t);
        acc.mac(tq[sl], av);
        // refill the slot with entry base + d + PD (index from batch A or B)
        const int j = d + PD;
        wq[sl] = (j < TR) ? gshfl<TR>(gmask, wA, j) : gshfl<TR>(gmask, wB, j - TR);
        issue(base + j, tq[sl]);
      }
      wA = wB;
      wB = wC;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int v = 4 * rb + i;
      if (v >= n_occ) break;
      const T up = sf * upsi[pair_off<T>(v, r, n3)];
      T av[SC], hv[SC];
      lds_a<T, SC, TR>(av, A, v, t);
      lds_vec<T, SC>(hv, VH + t * SC);
#pragma unroll
      for (int s = 0; s < SC; ++s) {
        if (s >= ns) break;
        const long f = (long)(s0 + s) * n_occ + v;
        out[pair_off<T>(f, r, n3)] = vl * av[s] + hv[s] * up - acc.get(i, s);
      }
    }
  }
}

// The same product with tau streamed through a shared-memory ring (RING variants): each
// group keeps D entries of tau in flight as 16-byte cp.async copies (no registers held), one
// copy per lane per entry, and reads each entry back with one 16-byte shared load when it
// is consumed. A lane refills the slot of entry e + D right after consuming entry e; one
// commit group per entry keeps the per-thread wait (cp.async.wait_group D-1) exact. The
// neighbour index of an entry is broadcast in the group when the entry is consumed.
template <int D>
__device__ __forceinline__ void cp_async_wait_ring() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 1) : "memory");
}
__device__ __forceinline__ void cp_async_commit_one() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int TR, int SC, int NT, int D>
__global__ void __launch_bounds__(NT, 2) k1d_ring_kernel(
    int n_vec, int n_occ, long n3, const float* __restrict__ a, const float* __restrict__ tau4, long n_ent,
    const int* __restrict__ bptr, const int* __restrict__ bw, int n_blocks, const float* __restrict__ vloc,
    const float* __restrict__ vh, const float* __restrict__ upsi, float sf, float* __restrict__ out) {
  using T = float;
  extern __shared__ __align__(16) unsigned char k1d_ring_smem[];
  constexpr int G = NT / TR;
  T* A = reinterpret_cast<T*>(k1d_ring_smem);        // [n_occ][SC / CH][TR][CH]
  T* VH = A + (size_t)n_occ * TR * SC;                // [TR][SC]
  float4* RING = reinterpret_cast<float4*>(VH + TR * SC + 4 - (TR * SC) % 4);  // [G][D][TR]
  const int n_sc = (n_vec + SC - 1) / SC;
  const int chunk = blockIdx.x % n_sc;
  const long r0 = (long)(blockIdx.x / n_sc) * TR;
  const int s0 = chunk * SC;
  const int ns = min(SC, n_vec - s0);
  const int tid = threadIdx.x;
  const int t = tid % TR, g = tid / TR;
  const long r = r0 + t;
  {
    using L = ALayout<T, SC>;
    const int n_items = n_occ * TR * SC;
    for (int it = tid; it < n_items; it += NT) {
      const int q = it % L::CH, tt = (it / L::CH) % TR, c = (it / (L::CH * TR)) % L::NCH;
      const int w = it / (SC * TR);
      const int s = c * L::CH + q;
      if (s < ns) cp_async<4>(A + it, a + pair_off<T>((long)(s0 + s) * n_occ + w, r0 + tt, n3));
    }
  }
  cp_async_commit_one();
  if (g < SC) VH[t * SC + g] = (g < ns) ? vh[pair_off<T>(s0 + g, r, n3)] : (T)0;
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const T vl = vloc[r];
  const T* tau_r = tau4 + tau4_off(0, r, n_ent);
  float4* ring = RING + (size_t)g * D * TR + t;       // slot k at ring[k * TR]
  const unsigned gmask = (TR == 32) ? 0xffffffffu : (((1u << TR) - 1u) << ((tid & 31) & ~(TR - 1)));
  for (int rb = g; rb < n_blocks; rb += G) {
    RowAcc<T, SC> acc;
    acc.zero();
    const int e0 = bptr[rb], e1 = bptr[rb + 1];
    auto ld_w = [&](int base) { const int e = base + t; return (e < e1) ? bw[e] : 0; };
    int wA = ld_w(e0), wB = ld_w(e0 + TR);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (e0 + k < e1) cp_async16_cg(ring + k * TR, tau_r + (size_t)(e0 + k) * (4 * TAU_TB));
      cp_async_commit_one();
    }
    int slot = 0;
    for (int base = e0; base < e1; base += TR) {
      const int wC = ld_w(base + 2 * TR);
#pragma unroll
      for (int d = 0; d < TR; ++d) {
        const int e = base + d;
        if (e >= e1) break;
        const int w = gshfl<TR>(gmask, wA, d);
        cp_async_wait_ring<D>();
        const float4 q = ring[slot * TR];
        const T tv[4] = {q.x, q.y, q.z, q.w};
        T av[SC];
        lds_a<T, SC, TR>(av, A, w, t);
        acc.mac(tv, av);
        // the slot is free once this lane has read it (each lane reads only its own copy)
        if (e + D < e1) cp_async16_cg(ring + slot * TR, tau_r + (size_t)(e + D) * (4 * TAU_TB));
        cp_async_commit_one();
        slot = (slot + 1 == D) ? 0 : slot + 1;
      }
      wA = wB;
      wB = wC;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int v = 4 * rb + i;
      if (v >= n_occ) break;
      const T up = sf * upsi[pair_off<T>(v, r, n3)];
      T av[SC], hv[SC];
      lds_a<T, SC, TR>(av, A, v, t);
      lds_vec<T, SC>(hv, VH + t * SC);
#pragma unroll
      for (int s = 0; s < SC; ++s) {
        if (s >= ns) break;
        const long f = (long)(s0 + s) * n_occ + v;
        out[pair_off<T>(f, r, n3)] = vl * av[s] + hv[s] * up - acc.get(i, s);
      }
    }
  }
}

template <typename T, int TR, int SC, int NT, int D>
cudaError_t launch_ring(int n_vec, int n_occ, long n3, const T* a, const T* tau4, long n_ent, const int* bptr,
                        const int* bw, int n_blocks, const T* vloc, const T* vh, const T* upsi, double sf, T* out,
                        long n_pts, cudaStream_t st) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorInvalidValue;
  } else {
    const size_t smem = ((size_t)n_occ * TR * SC + (size_t)TR * SC + 4) * sizeof(T) +
                        (size_t)(NT / TR) * D * TR * sizeof(float4);
    static std::once_flag once;
    static cudaError_t once_st = cudaSuccess;
    cudaError_t e0 = once_status(once, once_st, [&] {
      return cudaFuncSetAttribute(k1d_ring_kernel<TR, SC, NT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)K1D_SMEM_MAX);
    });
    if (e0 != cudaSuccess) return e0;
    if (smem > K1D_SMEM_MAX) return cudaErrorInvalidValue;
    const long blocks = (n_pts / TR) * ((n_vec + SC - 1) / SC);
    k1d_ring_kernel<TR, SC, NT, D><<<(unsigned)blocks, NT, smem, st>>>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw,
                                                                        n_blocks, vloc, vh, upsi, (float)sf, out);
    note_launch();
    return cudaGetLastError();
  }
}

// tile variants: (points per CTA, vectors per CTA, threads per CTA)
struct Variant { int tr, sc, nt; };
constexpr Variant kVariants[] = {{0, 0, 0},     {16, 8, 512}, {8, 8, 256},  {16, 4, 256},
                                 {8, 4, 256},   {16, 2, 256}, {16, 1, 256}, {16, 8, 256},
                                 {8, 8, 512},   {32, 4, 512}, {32, 8, 512}, {32, 2, 256},
                                 {8, 12, 256},  {8, 16, 256}, {8, 12, 256}, {8, 12, 256},
                                 {8, 8, 256},   {8, 4, 256},
                                 // shared-memory tau rings (single precision): 18 .. 20
                                 {8, 8, 256},   {8, 4, 256},  {8, 12, 256}};
// ring depth of the shared-memory ring variants (0: register ring); each is the depth that
// measured fastest for its chunk width with two CTAs per SM (deeper rings take shared memory
// that L1 needs: 8 vectors, depth 12 ran 5-10% slower than depth 8)
constexpr int ring_depth(int v) { return v == 18 ? 8 : v == 19 ? 16 : v == 20 ? 4 : 0; }
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0])) - 1;

template <typename T>
size_t variant_smem(int n_occ, int v) {
  const Variant q = kVariants[v];
  return ((size_t)n_occ * q.tr * q.sc + (size_t)q.tr * q.sc + 4) * sizeof(T) +
         (size_t)(q.nt / q.tr) * ring_depth(v) * q.tr * 16;
}

template <typename T, int TR, int SC, int NT, int MINB = k1d_min_blocks<SC, NT>(), bool PF = false>
cudaError_t launch_k1d(int n_vec, int n_occ, long n3, const T* a, const T* tau4, long n_ent, const int* bptr,
                       const int* bw, int n_blocks, const T* vloc, const T* vh,
                       const T* upsi, double sf, T* out, long n_pts, cudaStream_t st) {
  static_assert(NT % TR == 0 && 32 % TR == 0 && NT / TR >= SC, "tile shape");
  if constexpr (sizeof(T) == 8 && SC >= 8) {
    return cudaErrorInvalidValue;   // 4 x SC double accumulators per lane do not fit the register budget
  } else {
    const size_t smem = ((size_t)n_occ * TR * SC + (size_t)TR * SC) * sizeof(T);
    static std::once_flag once;
    static cudaError_t once_st = cudaSuccess;
    cudaError_t e0 = once_status(once, once_st, [&] {
      return cudaFuncSetAttribute(k1d_tile_kernel<T, TR, SC, NT, MINB, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)K1D_SMEM_MAX);
    });
    if (e0 != cudaSuccess) return e0;
    const long blocks = (n_pts / TR) * ((n_vec + SC - 1) / SC);
    k1d_tile_kernel<T, TR, SC, NT, MINB, PF><<<(unsigned)blocks, NT, smem, st>>>(
        n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi, (T)sf, out);
    note_launch();
    return cudaGetLastError();
  }
}

}  // namespace

int k1d_num_variants() { return kNumVariants; }

// whether variant v (1 .. k1d_num_variants()) fits the opt-in shared memory
template <typename T>
bool k1d_fits(int n_occ, int v) {
  if (v < 1 || v > kNumVariants) return false;
  if (sizeof(T) == 8 && kVariants[v].sc >= 8) return false;
  if (sizeof(T) == 8 && ring_depth(v) > 0) return false;
  return variant_smem<T>(n_occ, v) <= K1D_SMEM_MAX;
}

// vectors a launch of variant v computes for n_vec trial vectors (chunks of SC, the last
// one padded)
int k1d_padded_vectors(int n_vec, int v) {
  if (v < 1 || v > kNumVariants) return 1 << 30;
  const int sc = kVariants[v].sc;
  return (n_vec + sc - 1) / sc * sc;
}

// default variant without tuning: among the variants that fit, the least padded vectors,
// then an a(r) stage that leaves room for two CTAs per SM, then the first in the list; 0 when
// none fits
template <typename T>
int k1d_default_variant(int n_occ, int n_vec) {
  int best = 0;
  long best_key = 0;
  for (int v = 1; v <= kNumVariants; ++v) {
    if (!k1d_fits<T>(n_occ, v)) continue;
    const long key = (long)k1d_padded_vectors(std::max(1, n_vec), v) * 4 +
                     (variant_smem<T>(n_occ, v) <= K1D_SMEM_MAX / 2 ? 0 : 2);
    if (!best || key < best_key) { best = v; best_key = key; }
  }
  return best;
}

template <typename T>
cudaError_t k1d_tiled(int n_vec, int n_occ, long n3, const T* a, const T* tau4, long n_ent, const int* bptr,
                      const int* bw, int n_blocks, const T* vloc, const T* vh,
                      const T* upsi, double sf, T* out, int variant, cudaStream_t st, long n_pts) {
  if (n_vec <= 0) return cudaSuccess;
  if (n_pts < 0) n_pts = n3;
  if (n_pts > n3 || n_pts % TAU_TB) return cudaErrorInvalidValue;
  if (variant == 0) variant = k1d_default_variant<T>(n_occ, n_vec);
  if (!k1d_fits<T>(n_occ, variant)) return cudaErrorInvalidValue;
  if (n3 % TAU_TB || TAU_TB % kVariants[variant].tr) return cudaErrorInvalidValue;
#define BSE_K1D_CASE(V, TR, SC, NT)                                                                  \
  case V:                                                                                            \
    return launch_k1d<T, TR, SC, NT>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi, sf, \
                                 out, n_pts, st);
  switch (variant) {
    BSE_K1D_CASE(1, 16, 8, 512)
    BSE_K1D_CASE(2, 8, 8, 256)
    BSE_K1D_CASE(3, 16, 4, 256)
    BSE_K1D_CASE(4, 8, 4, 256)
    BSE_K1D_CASE(5, 16, 2, 256)
    BSE_K1D_CASE(6, 16, 1, 256)
    BSE_K1D_CASE(7, 16, 8, 256)
    BSE_K1D_CASE(8, 8, 8, 512)
    BSE_K1D_CASE(9, 32, 4, 512)
    BSE_K1D_CASE(10, 32, 8, 512)
    BSE_K1D_CASE(11, 32, 2, 256)
    BSE_K1D_CASE(12, 8, 12, 256)
    BSE_K1D_CASE(13, 8, 16, 256)
    case 14:   // 12-vector chunks held to the register budget of two CTAs per SM
      return launch_k1d<T, 8, 12, 256, 2>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi, sf,
                                          out, n_pts, st);
    // the same tile shapes with the L2 prefetch of the next row block
    case 15:
      return launch_k1d<T, 8, 12, 256, 2, true>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi,
                                                sf, out, n_pts, st);
    case 16:
      return launch_k1d<T, 8, 8, 256, 2, true>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi,
                                               sf, out, n_pts, st);
    case 17:
      return launch_k1d<T, 8, 4, 256, 2, true>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi,
                                               sf, out, n_pts, st);
#define BSE_K1D_RING(V, TR, SC, NT, D)                                                                 \
  case V:                                                                                              \
    return launch_ring<T, TR, SC, NT, D>(n_vec, n_occ, n3, a, tau4, n_ent, bptr, bw, n_blocks, vloc, vh, upsi, sf, \
                                         out, n_pts, st);
    BSE_K1D_RING(18, 8, 8, 256, 8)
    BSE_K1D_RING(19, 8, 4, 256, 16)
    BSE_K1D_RING(20, 8, 12, 256, 4)
#undef BSE_K1D_RING
    default: return cudaErrorInvalidValue;
  }
#undef BSE_K1D_CASE
}

template cudaError_t k1d_tiled<float>(int, int, long, const float*, const float*, long, const int*, const int*, int, const float*, const float*, const float*, double, float*, int, cudaStream_t, long);
template cudaError_t k1d_tiled<double>(int, int, long, const double*, const double*, long, const int*, const int*, int, const double*, const double*, const double*, double, double*, int, cudaStream_t, long);
template bool k1d_fits<float>(int, int);
template bool k1d_fits<double>(int, int);
template int k1d_default_variant<float>(int, int);
template int k1d_default_variant<double>(int, int);

}  // namespace bse
