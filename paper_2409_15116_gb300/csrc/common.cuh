// Shared device helpers for the BSE hot-path kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <mutex>

// Runs a one-time set-up call (e.g. a kernel attribute) once per process, thread-safe;
// every caller gets the status of that one call.
template <typename F>
inline cudaError_t once_status(std::once_flag& flag, cudaError_t& status, F&& fn) {
  std::call_once(flag, [&] { status = fn(); });
  return status;
}

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmk(double x, double y) {
  C c; c.x = x; c.y = y; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by sign * i  (sign = +1 or -1)
template <typename C> __device__ __forceinline__ C cmul_si(C a, int sign) {
  C r; if (sign > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r;
}

// Real fields are stored two per complex grid ("pair layout"): field f lives in
// component f%2 of complex grid f/2, i.e. at real offset (f/2)*2*n3 + 2*r + f%2.
template <typename T>
__device__ __forceinline__ size_t pair_off(long f, long r, long n3) {
  return (size_t)(f >> 1) * 2 * (size_t)n3 + 2 * (size_t)r + (size_t)(f & 1);
}

// tau_p(r) for n_pairs pairs is stored point-tiled: tiles of TAU_TB consecutive grid
// points, each holding all pairs' values at those points, [n3/TAU_TB][n_pairs][TAU_TB].
// A CTA that works on a few points reads one contiguous stretch of tau, and a warp that
// covers 32 points reads whole 128-byte lines.
constexpr int TAU_TB = 32;
__host__ __device__ __forceinline__ size_t tau_off(long p, long r, long n_pairs) {
  return ((size_t)(r / TAU_TB) * (size_t)n_pairs + (size_t)p) * TAU_TB + (size_t)(r % TAU_TB);
}

// Entry-major tau of the tiled K1d kernel. The row-block lists hold, for every block of
// four orbital rows, the union of the rows' neighbours w (one "entry" each); entry e keeps
// the four rows' tau_{v_i w}(r) side by side, point-tiled like tau:
// [n3/TAU_TB][n_ent][TAU_TB][4], zero where a row does not have that neighbour. A lane
// reads an entry's four values at its point as one 16-byte load (two for FP64), and the
// lanes of eight consecutive points read 128 contiguous bytes.
__host__ __device__ __forceinline__ size_t tau4_off(long e, long r, long n_ent) {
  return (((size_t)(r / TAU_TB) * (size_t)n_ent + (size_t)e) * TAU_TB + (size_t)(r % TAU_TB)) * 4;
}

namespace bse {
// count of kernel launches issued by this library (host side, all contexts)
void note_launch();
long long launch_count();
}  // namespace bse

__device__ __forceinline__ int iceil_div(int a, int b) { return (a + b - 1) / b; }
