// Screened direct term K1d of Eq. (k1d) for tau stored once per pair (the memory-saving
// layout), fused with the real-space parts of D (Eq. d) and K1e (Eq. k1e):
//
//   u_R,sv(r) = V_loc(r) u_a,sv(r) + s V_H,s(r) u_psi,v(r) - sum_{w in nbr(v)} tau_vw(r) u_a,sw(r)
//
// tau is symmetric (tau_vw = tau_wv, Eq. tau). Row block b (orbitals 4b..4b+3) keeps "upper"
// entries, one per neighbour w >= 4b of any of its rows, with the four rows' tau_{4b+i, w}(r)
// side by side (zero where a row lacks the neighbour); the rows' neighbours in earlier blocks
// J < b come from J's entries (J, 4b+i), i = 0..3, read as a 4x4 tile and used transposed
// (each of J's rows w = 4J+j gives the coefficients tau_{4J+j, 4b+i}). Every pair is stored
// once (twice inside a site's own 4x4 block): about half of the ordered entry-major layout of
// k1d.cu, which is faster where it fits (the transposed reading costs issue slots) -- this
// layout serves the systems whose ordered layout would not fit the device.
//
// The CTA structure follows k1d.cu: a tile of TR points x SC vectors, a(r) staged in shared
// memory by cp.async, groups of TR lanes walking row blocks with four-row register
// accumulators, upper entries through a register ring of PD 16-byte loads, transposed tiles
// through a ring of TD tiles; the first CTA of each 32-point tile asks L2 to prefetch each of
// its groups' next row block (bulk prefetch, no registers or shared memory held). Variants with
// RD > 0 or RT > 0 keep the upper entries or the tiles in flight in shared-memory rings filled by
// cp.async instead, which frees registers but passes every tau value through shared memory
// twice; for 1,024 orbitals (2-vector chunks) the all-register form is the fastest.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace bse {

namespace {

constexpr int K1D_PD = 8;                       // tau prefetch depth (entries per lane)
constexpr size_t K1D_SMEM_MAX = 227 * 1024;     // opt-in dynamic shared memory used at most (the limit)

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


// L2 prefetch of a byte range (16-byte aligned start, size a multiple of 16): no registers
// or shared memory are held while the data moves
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// the four rows' tau of entry e at the lane's point, zeros for e < 0
template <typename T>
__device__ __forceinline__ void ld_tau4_or_zero(T (&tv)[4], const T* tau_r, int e) {
  if (e >= 0) ld_tau4<T>(tv, tau_r + (size_t)e * (4 * TAU_TB));
  else tv[0] = tv[1] = tv[2] = tv[3] = (T)0;
}

// the four entries of transposed tile k (rows of block b, each holding J's four rows)
template <typename T>
__device__ __forceinline__ void ld_tile(T (&tv)[4][4], int& inf, const T* tau_r, const int4* __restrict__ tent,
                                        const int* __restrict__ tinfo, int k, int k1) {
  if (k < k1) {
    const int4 q = __ldg(tent + k);
    inf = __ldg(tinfo + k);
    ld_tau4_or_zero<T>(tv[0], tau_r, q.x);
    ld_tau4_or_zero<T>(tv[1], tau_r, q.y);
    ld_tau4_or_zero<T>(tv[2], tau_r, q.z);
    ld_tau4_or_zero<T>(tv[3], tau_r, q.w);
  } else {
    inf = 0;
  }
}

// asks L2 for row block rb's tau at the CTA's point tile: its upper entries (one contiguous
// stretch) and the entries of each transposed tile (one short stretch each)
template <typename T>
__device__ __forceinline__ void prefetch_block(const T* tau_tile, const K1dLists& L, int rb) {
  constexpr unsigned EB = 4u * TAU_TB * sizeof(T);
  const int e0 = __ldg(L.bptr + rb), e1 = __ldg(L.bptr + rb + 1);
  prefetch_l2(tau_tile + (size_t)e0 * 4 * TAU_TB, (unsigned)(e1 - e0) * EB);
  const int k0 = __ldg(L.tptr + rb), k1 = __ldg(L.tptr + rb + 1);
  for (int k = k0; k < k1; ++k) {
    const int4 q = __ldg(L.tent + k);
    int lo = 0x7fffffff, hi = -1;
    if (q.x >= 0) { lo = min(lo, q.x); hi = max(hi, q.x); }
    if (q.y >= 0) { lo = min(lo, q.y); hi = max(hi, q.y); }
    if (q.z >= 0) { lo = min(lo, q.z); hi = max(hi, q.z); }
    if (q.w >= 0) { lo = min(lo, q.w); hi = max(hi, q.w); }
    if (hi >= 0) prefetch_l2(tau_tile + (size_t)lo * 4 * TAU_TB, (unsigned)(hi - lo + 1) * EB);
  }
}

// CTAs per SM the register budget is sized for: two of 256 threads, one of 512, and one for
// the wide vector chunks (SC >= 12), whose a(r) stage leaves room for one CTA anyway
template <int SC, int NT>
constexpr int k1d_min_blocks() { return SC >= 12 ? 1 : 512 / NT; }

__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_one() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// RD, RT > 0 (single precision): the upper entries (RD of them) and the transposed tiles (RT
// of them) in flight in per-group shared-memory rings filled by cp.async (16 bytes per lane
// per entry, one commit group per entry or tile, so cp.async.wait_group RD-1 or RT-1 before a
// slot is read is exact) instead of registers; absent entries of a tile are zeroed in its slot
template <typename T, int TR, int SC, int NT, int RD = 0, int RT = 0, int MINB = k1d_min_blocks<SC, NT>()>
__global__ void __launch_bounds__(NT, MINB) k1d_sym_kernel(
    int n_vec, int n_occ, long n3, const T* __restrict__ a, const T* __restrict__ tau4, K1dLists L,
    const T* __restrict__ vloc, const T* __restrict__ vh, const T* __restrict__ upsi, T sf,
    T* __restrict__ out) {
  // ring depth (divides TR); half as deep in double precision, whose values take two
  // registers, and for 8-vector chunks, whose 32 accumulators share the 128-register budget
  constexpr int PD0 = (sizeof(T) == 8 || SC == 8) ? K1D_PD / 2 : K1D_PD;
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
  const int n_blocks = L.n_blocks;
  const long n_ent = L.n_ent;
  // tau of the CTA's 32-point tile (entry e at tau_tile[e * 4 TAU_TB]) and at the lane's point
  const T* tau_tile = tau4 + tau4_off(0, r0 - r0 % TAU_TB, n_ent);
  const T* tau_r = tau4 + tau4_off(0, r, n_ent);
  // the first row block of every group is on its way to L2 while a(r) is staged
  const bool pf = (chunk == 0) && (r0 % TAU_TB == 0);
  if (pf && t == 0 && g < n_blocks) prefetch_block<T>(tau_tile, L, g);
  // stage a(field (s0+s, w), r0+t) in layout order, so the lanes of a warp fill
  // consecutive shared-memory words
  {
    using AL = ALayout<T, SC>;
    const int n_items = n_occ * TR * SC;
    for (int it = tid; it < n_items; it += NT) {
      const int q = it % AL::CH, tt = (it / AL::CH) % TR, c = (it / (AL::CH * TR)) % AL::NCH;
      const int w = it / (SC * TR);
      const int s = c * AL::CH + q;
      if (s < ns)
        cp_async<sizeof(T)>(A + it, a + pair_off<T>((long)(s0 + s) * n_occ + w, r0 + tt, n3));
    }
  }
  if (g < SC) VH[t * SC + g] = (g < ns) ? vh[pair_off<T>(s0 + g, r, n3)] : (T)0;
  cp_async_wait_all();
  __syncthreads();
  const T vl = vloc[r];
  const unsigned gmask = (TR == 32) ? 0xffffffffu : (((1u << TR) - 1u) << ((tid & 31) & ~(TR - 1)));
  // shared-memory rings: upper entries [G][RD][TR], tiles [G][RT][4][TR] (16 bytes each)
  float4* ringU = reinterpret_cast<float4*>(VH + TR * SC + 4 - (TR * SC) % 4) + (size_t)g * RD * TR + t;
  float4* ringT = reinterpret_cast<float4*>(VH + TR * SC + 4 - (TR * SC) % 4) + (size_t)G * RD * TR +
                  (size_t)g * RT * 4 * TR + t;
  for (int rb = g; rb < n_blocks; rb += G) {
    if (pf && t == 0 && rb + G < n_blocks) prefetch_block<T>(tau_tile, L, rb + G);
    RowAcc<T, SC> acc;
    acc.zero();
    if constexpr (RD > 0 && sizeof(T) == 4) {
      const int e0 = __ldg(L.bptr + rb), e1 = __ldg(L.bptr + rb + 1);
      auto ld_w = [&](int base) { const int e = base + t; return (e < e1) ? __ldg(L.bw + e) : 0; };
      int wA = ld_w(e0), wB = ld_w(e0 + TR);
#pragma unroll
      for (int k = 0; k < RD; ++k) {
        if (e0 + k < e1) cp_async16_cg(ringU + k * TR, tau_r + (size_t)(e0 + k) * (4 * TAU_TB));
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
          cp_async_wait_n<RD - 1>();
          const float4 q = ringU[slot * TR];
          const T tv[4] = {q.x, q.y, q.z, q.w};
          T av[SC];
          lds_a<T, SC, TR>(av, A, w, t);
          acc.mac(tv, av);
          if (e + RD < e1) cp_async16_cg(ringU + slot * TR, tau_r + (size_t)(e + RD) * (4 * TAU_TB));
          cp_async_commit_one();
          slot = (slot + 1 == RD) ? 0 : slot + 1;
        }
        wA = wB;
        wB = wC;
      }
    } else
    // ---- upper entries (w >= 4 rb): tau_{4rb+i, w} from one 16-byte load ----
    {
      const int e0 = __ldg(L.bptr + rb), e1 = __ldg(L.bptr + rb + 1);
      // neighbour indices in batches of TR: lane t of the group holds entry base + t. Three
      // batches are live (current, next, the one after), so an index load has more than a
      // batch of work to arrive before it is needed.
      auto ld_w = [&](int base) { const int e = base + t; return (e < e1) ? __ldg(L.bw + e) : 0; };
      int wA = ld_w(e0), wB = ld_w(e0 + TR), wC;
      // ring of PD entries in flight: slot d holds tau (four rows) and the neighbour w
      T tq[PD][4];
      int wq[PD];
#pragma unroll
      for (int d = 0; d < PD; ++d) {
        wq[d] = gshfl<TR>(gmask, wA, d);
        ld_tau4_or_zero<T>(tq[d], tau_r, (e0 + d < e1) ? e0 + d : -1);
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
          ld_tau4_or_zero<T>(tq[sl], tau_r, (base + j < e1) ? base + j : -1);
        }
        wA = wB;
        wB = wC;
      }
    }
    if constexpr (RT > 0 && sizeof(T) == 4) {
      const int k0 = __ldg(L.tptr + rb), k1 = __ldg(L.tptr + rb + 1);
      int tinf[RT];
      auto issue_tile = [&](int k, int h) {
        if (k < k1) {
          const int4 q = __ldg(L.tent + k);
          tinf[h] = __ldg(L.tinfo + k);
          const int qi[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float4* dst = ringT + (h * 4 + i) * TR;
            if (qi[i] >= 0) cp_async16_cg(dst, tau_r + (size_t)qi[i] * (4 * TAU_TB));
            else *dst = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        } else {
          tinf[h] = 0;
        }
        cp_async_commit_one();
      };
#pragma unroll
      for (int h = 0; h < RT; ++h) issue_tile(k0 + h, h);
      for (int k = k0; k < k1; k += RT) {
#pragma unroll
        for (int h = 0; h < RT; ++h) {
          if (k + h >= k1) break;
          cp_async_wait_n<RT - 1>();
          float tt[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float4 q = ringT[(h * 4 + i) * TR];
            tt[i][0] = q.x; tt[i][1] = q.y; tt[i][2] = q.z; tt[i][3] = q.w;
          }
          const int J = tinf[h] >> 4, jm = tinf[h] & 15;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (!((jm >> j) & 1)) continue;
            T av[SC];
            lds_a<T, SC, TR>(av, A, 4 * J + j, t);
            const T cv[4] = {tt[0][j], tt[1][j], tt[2][j], tt[3][j]};
            acc.mac(cv, av);
          }
          issue_tile(k + h + RT, h);
        }
      }
    } else
    // ---- transposed tiles of earlier blocks J < rb: tau_{4J+j, 4rb+i} from J's entries
    // (J, 4rb+i); each of J's rows j that has a pair with rb is one step ----
    {
      // TD tiles in flight (one in double precision, whose values take two registers)
      constexpr int TD = (sizeof(T) == 8) ? 1 : 2;
      const int k0 = __ldg(L.tptr + rb), k1 = __ldg(L.tptr + rb + 1);
      T tt[TD][4][4];
      int tinf[TD];
#pragma unroll
      for (int h = 0; h < TD; ++h) ld_tile<T>(tt[h], tinf[h], tau_r, L.tent, L.tinfo, k0 + h, k1);
      for (int k = k0; k < k1; k += TD) {
#pragma unroll
        for (int h = 0; h < TD; ++h) {
          if (k + h >= k1) break;
          const int J = tinf[h] >> 4, jm = tinf[h] & 15;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (!((jm >> j) & 1)) continue;
            T av[SC];
            lds_a<T, SC, TR>(av, A, 4 * J + j, t);
            const T cv[4] = {tt[h][0][j], tt[h][1][j], tt[h][2][j], tt[h][3][j]};
            acc.mac(cv, av);
          }
          ld_tile<T>(tt[h], tinf[h], tau_r, L.tent, L.tinfo, k + h + TD, k1);
        }
      }
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

// tile variants: (points per CTA, vectors per CTA, threads per CTA)
struct Variant { int tr, sc, nt, rd, rt; };
constexpr Variant kVariants[] = {{0, 0, 0, 0, 0},    {8, 4, 256, 0, 0},  {8, 8, 256, 0, 0},  {8, 12, 256, 0, 0},
                                 {8, 16, 256, 0, 0}, {16, 4, 256, 0, 0}, {16, 8, 256, 0, 0}, {16, 8, 512, 0, 0},
                                 {8, 8, 512, 0, 0},  {16, 2, 256, 0, 0}, {16, 1, 256, 0, 0}, {32, 4, 512, 0, 0},
                                 {32, 2, 256, 0, 0},
                                 // shared-memory rings (single precision): upper depth, tiles in flight
                                 {8, 4, 256, 12, 3}, {8, 4, 256, 8, 4},  {8, 2, 256, 8, 1},  {8, 8, 256, 8, 2},
                                 {8, 4, 256, 16, 2}, {8, 2, 256, 4, 2},  {16, 2, 256, 8, 1},
                                 // 2-vector chunks of 8 points: both in registers, then one of the two
                                 // streams (upper entries, tiles) in a shared-memory ring
                                 {8, 2, 256, 0, 0},  {8, 2, 256, 8, 0},  {8, 2, 256, 0, 2}};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0])) - 1;

template <typename T>
size_t variant_smem(int n_occ, int v) {
  const Variant q = kVariants[v];
  return ((size_t)n_occ * q.tr * q.sc + (size_t)q.tr * q.sc + 4) * sizeof(T) +
         (size_t)(q.nt / q.tr) * (q.rd + 4 * q.rt) * q.tr * 16;
}

template <typename T, int TR, int SC, int NT, int RD = 0, int RT = 0>
cudaError_t launch_k1d(int n_vec, int n_occ, long n3, const T* a, const T* tau4, const K1dLists& L,
                       const T* vloc, const T* vh, const T* upsi, double sf, T* out, long n_pts, cudaStream_t st) {
  static_assert(NT % TR == 0 && 32 % TR == 0 && NT / TR >= SC, "tile shape");
  if constexpr (sizeof(T) == 8 && (SC >= 8 || RD > 0 || RT > 0)) {
    return cudaErrorInvalidValue;   // double accumulators do not fit; the rings are single precision
  } else {
    const size_t smem = ((size_t)n_occ * TR * SC + (size_t)TR * SC + 4) * sizeof(T) +
                        (size_t)(NT / TR) * (RD + 4 * RT) * TR * 16;
    static std::once_flag once;
    static cudaError_t once_st = cudaSuccess;
    cudaError_t e0 = once_status(once, once_st, [&] {
      return cudaFuncSetAttribute(k1d_sym_kernel<T, TR, SC, NT, RD, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)K1D_SMEM_MAX);
    });
    if (e0 != cudaSuccess) return e0;
    const long blocks = (n_pts / TR) * ((n_vec + SC - 1) / SC);
    k1d_sym_kernel<T, TR, SC, NT, RD, RT><<<(unsigned)blocks, NT, smem, st>>>(n_vec, n_occ, n3, a, tau4, L, vloc, vh,
                                                                      upsi, (T)sf, out);
    note_launch();
    return cudaGetLastError();
  }
}

}  // namespace

int k1d_sym_num_variants() { return kNumVariants; }

// whether variant v (1 .. k1d_sym_num_variants()) fits the opt-in shared memory
template <typename T>
bool k1d_sym_fits(int n_occ, int v) {
  if (v < 1 || v > kNumVariants) return false;
  if (sizeof(T) == 8 && (kVariants[v].sc >= 8 || kVariants[v].rd > 0 || kVariants[v].rt > 0)) return false;
  return variant_smem<T>(n_occ, v) <= K1D_SMEM_MAX;
}

// vectors a launch of variant v computes for n_vec trial vectors (chunks of SC, the last
// one padded)
int k1d_sym_padded_vectors(int n_vec, int v) {
  if (v < 1 || v > kNumVariants) return 1 << 30;
  const int sc = kVariants[v].sc;
  return (n_vec + sc - 1) / sc * sc;
}

// default variant without tuning: among the variants that fit, the least padded vectors;
// then a(r) stages that leave room for two CTAs per SM; then the first in the list.
// 0 when none fits
template <typename T>
int k1d_sym_default_variant(int n_occ, int n_vec) {
  int best = 0;
  long best_key = 0;
  for (int v = 1; v <= kNumVariants; ++v) {
    if (!k1d_sym_fits<T>(n_occ, v)) continue;
    const long key = (long)k1d_sym_padded_vectors(std::max(1, n_vec), v) * 4 +
                     (variant_smem<T>(n_occ, v) <= K1D_SMEM_MAX / 2 ? 0 : 2);
    if (!best || key < best_key) { best = v; best_key = key; }
  }
  return best;
}

template <typename T>
cudaError_t k1d_sym_tiled(int n_vec, int n_occ, long n3, const T* a, const T* tau4, const K1dLists& L, const T* vloc,
                      const T* vh, const T* upsi, double sf, T* out, int variant, cudaStream_t st, long n_pts) {
  if (n_vec <= 0) return cudaSuccess;
  if (n_pts < 0) n_pts = n3;
  if (n_pts > n3 || n_pts % TAU_TB) return cudaErrorInvalidValue;
  if (variant == 0) variant = k1d_sym_default_variant<T>(n_occ, n_vec);
  if (!k1d_sym_fits<T>(n_occ, variant)) return cudaErrorInvalidValue;
  if (n3 % TAU_TB || TAU_TB % kVariants[variant].tr) return cudaErrorInvalidValue;
  if (L.n_blocks != (n_occ + 3) / 4) return cudaErrorInvalidValue;
#define BSE_K1D_CASE(V, TR, SC, NT)                                                                  \
  case V:                                                                                            \
    return launch_k1d<T, TR, SC, NT>(n_vec, n_occ, n3, a, tau4, L, vloc, vh, upsi, sf, out, n_pts, st);
  switch (variant) {
    BSE_K1D_CASE(1, 8, 4, 256)
    BSE_K1D_CASE(2, 8, 8, 256)
    BSE_K1D_CASE(3, 8, 12, 256)
    BSE_K1D_CASE(4, 8, 16, 256)
    BSE_K1D_CASE(5, 16, 4, 256)
    BSE_K1D_CASE(6, 16, 8, 256)
    BSE_K1D_CASE(7, 16, 8, 512)
    BSE_K1D_CASE(8, 8, 8, 512)
    BSE_K1D_CASE(9, 16, 2, 256)
    BSE_K1D_CASE(10, 16, 1, 256)
    BSE_K1D_CASE(11, 32, 4, 512)
    BSE_K1D_CASE(12, 32, 2, 256)
#define BSE_K1D_RING(V, TR, SC, NT, RD, RT) \
  case V: return launch_k1d<T, TR, SC, NT, RD, RT>(n_vec, n_occ, n3, a, tau4, L, vloc, vh, upsi, sf, out, n_pts, st);
    BSE_K1D_RING(13, 8, 4, 256, 12, 3)
    BSE_K1D_RING(14, 8, 4, 256, 8, 4)
    BSE_K1D_RING(15, 8, 2, 256, 8, 1)
    BSE_K1D_RING(16, 8, 8, 256, 8, 2)
    BSE_K1D_RING(17, 8, 4, 256, 16, 2)
    BSE_K1D_RING(18, 8, 2, 256, 4, 2)
    BSE_K1D_RING(19, 16, 2, 256, 8, 1)
#undef BSE_K1D_RING
    BSE_K1D_CASE(20, 8, 2, 256)
#define BSE_K1D_RING(V, TR, SC, NT, RD, RT) \
  case V: return launch_k1d<T, TR, SC, NT, RD, RT>(n_vec, n_occ, n3, a, tau4, L, vloc, vh, upsi, sf, out, n_pts, st);
    BSE_K1D_RING(21, 8, 2, 256, 8, 0)
    BSE_K1D_RING(22, 8, 2, 256, 0, 2)
#undef BSE_K1D_RING
    default: return cudaErrorInvalidValue;
  }
#undef BSE_K1D_CASE
}

template cudaError_t k1d_sym_tiled<float>(int, int, long, const float*, const float*, const K1dLists&, const float*,
                                      const float*, const float*, double, float*, int, cudaStream_t, long);
template cudaError_t k1d_sym_tiled<double>(int, int, long, const double*, const double*, const K1dLists&, const double*,
                                       const double*, const double*, double, double*, int, cudaStream_t, long);
template bool k1d_sym_fits<float>(int, int);
template bool k1d_sym_fits<double>(int, int);
template int k1d_sym_default_variant<float>(int, int);
template int k1d_sym_default_variant<double>(int, int);

}  // namespace bse
