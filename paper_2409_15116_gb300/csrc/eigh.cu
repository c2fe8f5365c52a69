// FP64 symmetric eigensolver for the Davidson Rayleigh-Ritz matrix (m <= 160), one CTA.
//
// One-sided (Hestenes) Jacobi on G = A + s I, with the shift s taken from Gershgorin's
// lower bound so that G is positive definite: plane rotations orthogonalise the columns
// of G in place, V accumulates them, and at convergence the columns of V are the
// eigenvectors of A. Each warp owns disjoint column pairs of a round-robin round (its
// three dot products are warp-shuffle reductions), so a round needs a single CTA-wide
// barrier. Eigenvalues are recomputed as v_i^T (A + s I) v_i - s, i.e. v_i . g_i - s.
#include "common.cuh"
#include "kernels.h"

namespace bse {

constexpr int EIGH_MAX = 160;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(512) hestenes_kernel(int m, const double* __restrict__ A, long lda,
                                                      double* __restrict__ Vc, double* __restrict__ Vout,
                                                      double* __restrict__ w, int* info) {
  extern __shared__ __align__(16) double G[];   // column-major, G[j*m + i] = G(i, j)
  __shared__ double red[32];
  __shared__ double shift_s;
  __shared__ int rot_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  // Gershgorin lower bound of the spectrum
  double lo = 1e300;
  for (int i = tid; i < m; i += blockDim.x) {
    double off = 0;
    for (int j = 0; j < m; ++j)
      if (j != i) off += fabs(A[(long)i * lda + j]);
    lo = fmin(lo, A[(long)i * lda + i] - off);
  }
  for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if (lane == 0) red[warp] = lo;
  __syncthreads();
  if (tid == 0) {
    double l = red[0];
    for (int i = 1; i < nwarps; ++i) l = fmin(l, red[i]);
    shift_s = (l < 0 ? -l : 0.0) + 0.25 * (fabs(l) + 1e-3);
  }
  __syncthreads();
  const double s0 = shift_s;
  for (long e = tid; e < (long)m * m; e += blockDim.x) {
    const int j = (int)(e / m), i = (int)(e - (long)j * m);
    G[e] = A[(long)i * lda + j] + (i == j ? s0 : 0.0);
    Vc[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int mp = (m + 1) & ~1, half = mp / 2;
  int sweep = 0;
  for (; sweep < 40 && m > 1; ++sweep) {
    if (tid == 0) rot_count = 0;
    __syncthreads();
    for (int rnd = 0; rnd < mp - 1; ++rnd) {
      for (int t = warp; t < half; t += nwarps) {
        int p = (t == 0) ? 0 : ((t - 1 + rnd) % (mp - 1)) + 1;
        int q = ((mp - 2 - t + rnd) % (mp - 1)) + 1;
        if (p > q) { const int x = p; p = q; q = x; }
        if (q >= m) continue;
        double* gp = G + (long)p * m;
        double* gq = G + (long)q * m;
        double a = 0, b = 0, g = 0;
        for (int i = lane; i < m; i += 32) {
          const double x = gp[i], y = gq[i];
          a += x * x; b += y * y; g += x * y;
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        double* vp = Vc + (long)p * m;
        double* vq = Vc + (long)q * m;
        for (int i = lane; i < m; i += 32) {
          const double x = gp[i], y = gq[i];
          gp[i] = c * x - s * y; gq[i] = s * x + c * y;
          const double u = vp[i], z = vq[i];
          vp[i] = c * u - s * z; vq[i] = s * u + c * z;
        }
        if (lane == 0) atomicAdd(&rot_count, 1);
      }
      __syncthreads();
    }
    if (rot_count == 0) break;
    __syncthreads();
  }
  // eigenvalues: theta_i = v_i . g_i - s (g_i = (A + sI) v_i)
  __shared__ double th[EIGH_MAX];
  for (int i = warp; i < m; i += nwarps) {
    double d = 0;
    for (int k = lane; k < m; k += 32) d += Vc[(long)i * m + k] * G[(long)i * m + k];
    d = warp_sum(d);
    if (lane == 0) th[i] = d - s0;
  }
  __syncthreads();
  for (long e = tid; e < (long)m * m; e += blockDim.x) {
    const int i = (int)(e / m), k = (int)(e - (long)i * m);   // column i, row k
    const double di = th[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (th[j] < di) || (th[j] == di && j < i);
    Vout[(long)k * m + rank] = Vc[e];
    if (k == 0) w[rank] = di;
  }
  if (tid == 0) info[0] = (sweep >= 40) ? -1 : sweep;
}

cudaError_t jacobi_eigh(int m, const double* A, long lda, double* work, double* V, double* w,
                        int* info, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if (m > EIGH_MAX) return cudaErrorInvalidValue;
  const size_t smem = (size_t)m * m * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(hestenes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)EIGH_MAX * EIGH_MAX * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  hestenes_kernel<<<1, 512, smem, st>>>(m, A, lda, work, V, w, info);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bse
