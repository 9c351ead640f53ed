// Device helpers shared by the kernels: complex arithmetic on float2/double2,
// precision traits, and the lattice index functions (site = x + Lx * t).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mgk {

// Number of kernel launches made by this library (all threads), for reporting.
void count_launch();
unsigned long long launch_count();

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename R> using cplx_t = typename cplx_of<R>::type;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }
// i * a
template <typename C> __device__ __forceinline__ C ci(C a) { return {-a.y, a.x}; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
  return {a.x * s, a.y * s};
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// One hop of the Wilson stencil in direction x (sigma_1) or t (sigma_2):
//   (1 - s sigma_1) phi = (phi0 - s phi1) (1, -s)^T
//   (1 - s sigma_2) phi = (phi0 + i s phi1) (1, -i s)^T
// accumulated as a += u * projection (both components).
template <typename R>
__device__ __forceinline__ void hop_x(cplx_t<R>& a0, cplx_t<R>& a1, cplx_t<R> u, cplx_t<R> f0,
                                      cplx_t<R> f1, R s) {
  // h = u * (f0 - s f1); a0 += h; a1 += -s h
  cplx_t<R> p = mk(f0.x - s * f1.x, f0.y - s * f1.y);
  cplx_t<R> h = cmul(u, p);
  a0 = cadd(a0, h);
  a1 = mk(a1.x - s * h.x, a1.y - s * h.y);
}

template <typename R>
__device__ __forceinline__ void hop_t(cplx_t<R>& a0, cplx_t<R>& a1, cplx_t<R> u, cplx_t<R> f0,
                                      cplx_t<R> f1, R s) {
  // h = u * (f0 + i s f1); a0 += h; a1 += -i s h
  cplx_t<R> p = mk(f0.x - s * f1.y, f0.y + s * f1.x);
  cplx_t<R> h = cmul(u, p);
  a0 = cadd(a0, h);
  a1 = mk(a1.x + s * h.y, a1.y - s * h.x);   // -i s h = s (h.y, -h.x)
}

__device__ __forceinline__ float2 bf2_to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }

// Fixed-order block reduction of (a, b) pairs held one per thread.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? sh[2 * l] : 0.0;
    b = l < nw ? sh[2 * l + 1] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

// Single-pass deterministic reduction.  Every block writes its partial sum;
// the last block to finish (found with an atomic ticket) adds the partials in
// a fixed order and resets the ticket.  ws = [64 tickets (as doubles)][partials].
// rhs selects the output and ticket; blk in [0, G) is this block's slot.
// Returns true in the block that wrote the sum (all its threads).
__device__ __forceinline__ bool finish_reduction_g(double re, double im, double* ws, double* out,
                                                   double* sh, int rhs, int blk, int G) {
  unsigned* tickets = (unsigned*)ws;
  double* partials = ws + 64;
  __shared__ bool last;
  block_sum2(re, im, sh);
  if (threadIdx.x == 0) {
    partials[2 * ((long long)rhs * G + blk)] = re;
    partials[2 * ((long long)rhs * G + blk) + 1] = im;
    __threadfence();
    last = atomicAdd(&tickets[rhs], 1u) == (unsigned)(G - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  re = 0.0;
  im = 0.0;
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    re += __ldcg(&partials[2 * ((long long)rhs * G + i)]);
    im += __ldcg(&partials[2 * ((long long)rhs * G + i) + 1]);
  }
  __syncthreads();
  block_sum2(re, im, sh);
  if (threadIdx.x == 0) {
    out[2 * rhs] = re;
    out[2 * rhs + 1] = im;
    tickets[rhs] = 0u;
  }
  return true;
}

__device__ __forceinline__ bool finish_reduction(double re, double im, double* ws, double* out,
                                                 double* sh) {
  return finish_reduction_g(re, im, ws, out, sh, blockIdx.y, blockIdx.x, gridDim.x);
}

// Block map of the geometric blocking S_j: coarse site and in-block offset.
__host__ __device__ __forceinline__ int coarse_site(int x, int t, int Lx, int bx, int bt) {
  return (t / bt) * (Lx / bx) + x / bx;
}
__host__ __device__ __forceinline__ int block_offset(int x, int t, int bx, int bt) {
  return (t % bt) * bx + x % bx;
}

}  // namespace mgk
