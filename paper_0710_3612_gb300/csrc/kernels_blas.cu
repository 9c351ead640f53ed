// Vector kernels of the Krylov solvers: deterministic reductions (fixed block
// count and fixed summation tree, so repeated solves give identical bits),
// CG updates on per-RHS device scalars, precision conversions.
#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace mgk {

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

static constexpr int RT = 256;   // threads per reduction block

int reduce_blocks(long long count) {
  long long g = (count + RT - 1) / RT;           // one entry per thread until 608 blocks

  if (g < 1) g = 1;
  if (g > 608) g = 608;           // 4 x 152 SMs
  return (int)g;
}

template <typename R, bool NORM>
__global__ void __launch_bounds__(RT) k_dot(const cplx_t<R>* __restrict__ a,
                                            const cplx_t<R>* __restrict__ b, long long count,
                                            double* ws, double* out) {
  __shared__ double sh[2 * RT / 32];
  const int rhs = blockIdx.y;
  const cplx_t<R>* pa = a + (long long)rhs * count;
  const cplx_t<R>* pb = NORM ? pa : b + (long long)rhs * count;
  double re = 0.0, im = 0.0;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    cplx_t<R> u = pa[i];
    if (NORM) {
      re = fma((double)u.x, (double)u.x, re);
      re = fma((double)u.y, (double)u.y, re);
    } else {
      cplx_t<R> v = pb[i];
      re = fma((double)u.x, (double)v.x, re);
      re = fma((double)u.y, (double)v.y, re);
      im = fma((double)u.x, (double)v.y, im);
      im = fma(-(double)u.y, (double)v.x, im);
    }
  }
  finish_reduction(re, im, ws, out, sh);
}

template <typename R>
cudaError_t dot(const void* a, const void* b, long long count, int nrhs, double* partials,
                double* out, cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  int g = reduce_blocks(count);
  k_dot<R, false><<<dim3(g, nrhs), RT, 0, s>>>((const cplx_t<R>*)a, (const cplx_t<R>*)b, count,
                                               partials, out);
  count_launch();
  return cudaGetLastError();
}

template <typename R>
cudaError_t norm2(const void* a, long long count, int nrhs, double* partials, double* out,
                  cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  int g = reduce_blocks(count);
  k_dot<R, true><<<dim3(g, nrhs), RT, 0, s>>>((const cplx_t<R>*)a, nullptr, count, partials, out);
  count_launch();
  return cudaGetLastError();
}

static inline dim3 grid1(long long count, int nrhs) {
  long long g = (count + RT - 1) / RT;
  return dim3((unsigned)g, nrhs);
}

template <typename R>
__global__ void k_axpby(R a, const cplx_t<R>* __restrict__ x, R b, cplx_t<R>* __restrict__ y,
                        long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  i += (long long)blockIdx.y * count;
  cplx_t<R> u = x[i], v = y[i];
  y[i] = mk(a * u.x + b * v.x, a * u.y + b * v.y);
}

template <typename R>
cudaError_t axpby(double a, const void* x, double b, void* y, long long count, int nrhs,
                  cudaStream_t s) {
  k_axpby<R><<<grid1(count, nrhs), RT, 0, s>>>((R)a, (const cplx_t<R>*)x, (R)b, (cplx_t<R>*)y,
                                                count); count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_scale_inv_sqrt(const cplx_t<R>* __restrict__ x, cplx_t<R>* __restrict__ y,
                                 const double* nrm, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double n2 = nrm[2 * blockIdx.y];
  const R sc = n2 > 0.0 ? (R)(1.0 / sqrt(n2)) : (R)0;
  i += (long long)blockIdx.y * count;
  cplx_t<R> u = x[i];
  y[i] = mk(u.x * sc, u.y * sc);
}

template <typename R>
cudaError_t scale_inv_sqrt(const void* x, void* y, const double* nrm, long long count, int nrhs,
                           cudaStream_t s) {
  k_scale_inv_sqrt<R><<<grid1(count, nrhs), RT, 0, s>>>((const cplx_t<R>*)x, (cplx_t<R>*)y, nrm,
                                                         count); count_launch();
  return cudaGetLastError();
}

__device__ void cg_control_step(const double* rr, const double* pq, const double* stop, int* ctrl,
                                cudaGraphConditionalHandle cond);

template <typename R>
__global__ void __launch_bounds__(RT) k_cg_xr(cplx_t<R>* __restrict__ x, cplx_t<R>* __restrict__ r,
                                              const cplx_t<R>* __restrict__ p,
                                              const cplx_t<R>* __restrict__ q, const double* rz,
                                              const double* pq, const int* frozen,
                                              long long count, double* ws, double* rr,
                                              float2* __restrict__ r32, CgControl cc) {
  __shared__ double sh[2 * RT / 32];
  const int rhs = blockIdx.y;
  const bool skip = frozen && frozen[rhs];
  const double d = pq[2 * rhs];
  const R alpha = (d != 0.0 && !skip) ? (R)(rz[2 * rhs] / d) : (R)0;
  double acc = 0.0;
  const long long base = (long long)rhs * count;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const long long k = base + i;
    cplx_t<R> rv = r[k];
    if (!skip) {
      const cplx_t<R> xv = x[k], pv = p[k], qv = q[k];
      x[k] = mk(fma(alpha, pv.x, xv.x), fma(alpha, pv.y, xv.y));
      rv = mk(fma(-alpha, qv.x, rv.x), fma(-alpha, qv.y, rv.y));
      r[k] = rv;
    }
    if (r32) r32[k] = make_float2((float)rv.x, (float)rv.y);
    acc = fma((double)rv.x, (double)rv.x, acc);
    acc = fma((double)rv.y, (double)rv.y, acc);
  }
  const bool done = finish_reduction(acc, 0.0, ws, rr, sh);
  // loop control in the block that completes the last right-hand side's sum
  if (cc.ctrl && done && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(cc.tick, 1u) == gridDim.y - 1) {
      __threadfence();
      *cc.tick = 0u;
      cg_control_step(rr, pq, cc.stop, cc.ctrl, cc.cond);
    }
  }
}

template <typename R>
cudaError_t cg_xr(void* x, void* r, const void* p, const void* q, const double* rz,
                  const double* pq, const int* frozen, long long count, int nrhs, double* ws,
                  double* rr, cudaStream_t s, void* r32, const CgControl* cc) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  int g = reduce_blocks(count);
  k_cg_xr<R><<<dim3(g, nrhs), RT, 0, s>>>((cplx_t<R>*)x, (cplx_t<R>*)r, (const cplx_t<R>*)p,
                                          (const cplx_t<R>*)q, rz, pq, frozen, count, ws, rr,
                                          (float2*)r32, cc ? *cc : CgControl{});
  count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_cg_p(cplx_t<R>* __restrict__ p, const cplx_t<R>* __restrict__ z,
                       const double* rz_new, const double* rz_old, const int* frozen,
                       long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= count || (frozen && frozen[rhs])) return;
  const double d = rz_old[2 * rhs];
  const R beta = d != 0.0 ? (R)(rz_new[2 * rhs] / d) : (R)0;
  i += (long long)rhs * count;
  cplx_t<R> pv = p[i], zv = z[i];
  p[i] = mk(fma(beta, pv.x, zv.x), fma(beta, pv.y, zv.y));
}

template <typename R>
cudaError_t cg_p(void* p, const void* z, const double* rz_new, const double* rz_old,
                 const int* frozen, long long count, int nrhs, cudaStream_t s) {
  k_cg_p<R><<<grid1(count, nrhs), RT, 0, s>>>((cplx_t<R>*)p, (const cplx_t<R>*)z, rz_new, rz_old,
                                               frozen, count); count_launch();
  return cudaGetLastError();
}

// Device-side loop control of the graph-resident CG for nrhs right-hand
// sides.  ctrl = {iterations, status, limit, nrhs}; frozen[rhs] (ctrl + 4) is
// set when a right-hand side converges (rr <= stop) or breaks down, and
// it_done[rhs] (ctrl + 4 + nrhs) records its iteration count.  status: 0
// running, 1 all converged, 2 a breakdown, 3 limit reached.  Sets the WHILE
// condition of the enclosing graph node.
__device__ void cg_control_step(const double* rr, const double* pq, const double* stop, int* ctrl,
                                cudaGraphConditionalHandle cond) {
  const int it = ctrl[0] + 1;
  const int nrhs = ctrl[3];
  int* frozen = ctrl + 4;
  int* it_done = ctrl + 4 + nrhs;
  ctrl[0] = it;
  int running = 0, broken = 0;
  for (int k = 0; k < nrhs; ++k) {
    if (frozen[k]) continue;
    const double r = __ldcg(rr + 2 * k), d = __ldcg(pq + 2 * k);
    if (!(d > 0.0) || !(r == r)) {
      frozen[k] = 2;
      it_done[k] = it;
      broken = 1;
    } else if (r <= stop[2 * k]) {
      frozen[k] = 1;
      it_done[k] = it;
    } else {
      ++running;
    }
  }
  int status = running ? 0 : 1;
  if (broken) status = 2;
  else if (running && it >= ctrl[2]) status = 3;
  if (status == 3)
    for (int k = 0; k < nrhs; ++k)
      if (!frozen[k]) it_done[k] = it;
  ctrl[1] = status;
  cudaGraphSetConditional(cond, status == 0 ? 1u : 0u);
}

__global__ void k_cg_control(const double* rr, const double* pq, const double* stop, int* ctrl,
                             cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cg_control_step(rr, pq, stop, ctrl, cond);
}

cudaError_t cg_control(const double* rr, const double* pq, const double* stop, int* ctrl,
                       cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_cg_control<<<1, 32, 0, s>>>(rr, pq, stop, ctrl, cond);
  count_launch();
  return cudaGetLastError();
}

// Initialises ctrl and stop[rhs] = tol2 * bn[rhs]; right-hand sides with
// b = 0 start frozen (x = 0 is exact).
__global__ void k_set_control(int* ctrl, int maxiter, int nrhs, const double* bn, double tol2,
                              double* stop) {
  if (threadIdx.x != 0) return;
  ctrl[0] = 0;
  ctrl[1] = 0;
  ctrl[2] = maxiter;
  ctrl[3] = nrhs;
  for (int k = 0; k < nrhs; ++k) {
    stop[2 * k] = tol2 * bn[2 * k];
    stop[2 * k + 1] = 0.0;
    ctrl[4 + k] = bn[2 * k] == 0.0 ? 1 : 0;
    ctrl[4 + nrhs + k] = 0;
  }
}

cudaError_t set_control(int* ctrl, int maxiter, int nrhs, const double* bn, double tol2,
                        double* stop, cudaStream_t s) {
  k_set_control<<<1, 32, 0, s>>>(ctrl, maxiter, nrhs, bn, tol2, stop);
  count_launch();
  return cudaGetLastError();
}

// Flexible CG with the FP32 preconditioned residual z32, per right-hand side:
// zr[rhs] = {Re<z32, q>, Re<r, z32>} in one deterministic pass.
__global__ void __launch_bounds__(RT) k_dot2_zq_rz(const float2* __restrict__ z,
                                                   const double2* __restrict__ q,
                                                   const double2* __restrict__ r, long long count,
                                                   double* ws, double* zr) {
  __shared__ double sh[2 * RT / 32];
  const long long base = (long long)blockIdx.y * count;
  double a = 0.0, b = 0.0;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const float2 zv = z[base + i];
    const double2 qv = q[base + i], rv = r[base + i];
    a = fma((double)zv.x, qv.x, a);
    a = fma((double)zv.y, qv.y, a);
    b = fma(rv.x, (double)zv.x, b);
    b = fma(rv.y, (double)zv.y, b);
  }
  finish_reduction(a, b, ws, zr, sh);
}

cudaError_t dot2_zq_rz(const void* z32, const void* q, const void* r, long long count, int nrhs,
                       double* ws, double* zr, cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  k_dot2_zq_rz<<<dim3(reduce_blocks(count), nrhs), RT, 0, s>>>(
      (const float2*)z32, (const double2*)q, (const double2*)r, count, ws, zr);
  count_launch();
  return cudaGetLastError();
}

// beta = -zr[0] / Re(pq); p = z32 + beta p; rz <- {zr[1], 0}; per rhs, frozen
// right-hand sides untouched.
__global__ void k_cg_p_pr(double2* __restrict__ p, const float2* __restrict__ z, const double* zr,
                          const double* pq, double* rz, const int* frozen, long long count) {
  const int rhs = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (frozen && frozen[rhs]) return;
  if (i == 0) {
    rz[2 * rhs] = zr[2 * rhs + 1];
    rz[2 * rhs + 1] = 0.0;
  }
  if (i >= count) return;
  const double d = pq[2 * rhs];
  const double beta = d != 0.0 ? -zr[2 * rhs] / d : 0.0;
  const long long k = (long long)rhs * count + i;
  const double2 pv = p[k];
  const float2 zv = z[k];
  p[k] = make_double2(fma(beta, pv.x, (double)zv.x), fma(beta, pv.y, (double)zv.y));
}

cudaError_t cg_p_pr(void* p, const void* z32, const double* zr, const double* pq, double* rz,
                    const int* frozen, long long count, int nrhs, cudaStream_t s) {
  k_cg_p_pr<<<grid1(count, nrhs), RT, 0, s>>>((double2*)p, (const float2*)z32, zr, pq, rz, frozen,
                                               count);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reliable-update flexible CG (FP32 iteration, FP64 solution and true
// residual).  Per-thread partial sums are kept in FP32 (a thread covers a few
// entries) and the blocks are combined in FP64 by the deterministic
// single-pass reduction, so no FP64 arithmetic runs per entry.
// ---------------------------------------------------------------------------

// ab[rhs] = <a, b> of FP32 vectors.
__global__ void __launch_bounds__(RT) k_rdot(const float2* __restrict__ a,
                                             const float2* __restrict__ b, long long count,
                                             double* ws, double* out) {
  __shared__ double sh[2 * RT / 32];
  const long long base = (long long)blockIdx.y * count;
  float re = 0.f, im = 0.f;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const float2 u = a[base + i], v = b[base + i];
    re = fmaf(u.x, v.x, fmaf(u.y, v.y, re));
    im = fmaf(u.x, v.y, fmaf(-u.y, v.x, im));
  }
  finish_reduction((double)re, (double)im, ws, out, sh);
}

cudaError_t rdot(const void* a, const void* b, long long count, int nrhs, double* ws, double* out,
                 cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  k_rdot<<<dim3(reduce_blocks(count), nrhs), RT, 0, s>>>((const float2*)a, (const float2*)b,
                                                         count, ws, out);
  count_launch();
  return cudaGetLastError();
}

// alpha = rz / pq; x += alpha p; r -= alpha q; rr = |r|^2 (FP32 vectors, alpha
// rounded to FP32 once per right-hand side); frozen right-hand sides keep x
// and r and report their |r|^2.
__global__ void __launch_bounds__(RT) k_rcg_xr(float2* __restrict__ x, float2* __restrict__ r,
                                               const float2* __restrict__ p,
                                               const float2* __restrict__ q, const double* rz,
                                               const double* pq, const int* frozen,
                                               long long count, double* ws, double* rr) {
  __shared__ double sh[2 * RT / 32];
  const int rhs = blockIdx.y;
  const bool skip = frozen && frozen[rhs];
  const double d = pq[2 * rhs];
  const float alpha = (d != 0.0 && !skip) ? (float)(rz[2 * rhs] / d) : 0.f;
  float acc = 0.f;
  const long long base = (long long)rhs * count;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const long long k = base + i;
    float2 rv = r[k];
    if (!skip) {
      const float2 xv = x[k], pv = p[k], qv = q[k];
      x[k] = make_float2(fmaf(alpha, pv.x, xv.x), fmaf(alpha, pv.y, xv.y));
      rv = make_float2(fmaf(-alpha, qv.x, rv.x), fmaf(-alpha, qv.y, rv.y));
      r[k] = rv;
    }
    acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc));
  }
  finish_reduction((double)acc, 0.0, ws, rr, sh);
}

cudaError_t rcg_xr(void* x32, void* r32, const void* p32, const void* q32, const double* rz,
                   const double* pq, const int* frozen, long long count, int nrhs, double* ws,
                   double* rr, cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  k_rcg_xr<<<dim3(reduce_blocks(count), nrhs), RT, 0, s>>>(
      (float2*)x32, (float2*)r32, (const float2*)p32, (const float2*)q32, rz, pq, frozen, count,
      ws, rr);
  count_launch();
  return cudaGetLastError();
}

// zr[rhs] = {Re<z, q>, Re<r, z>} of FP32 vectors.
__global__ void __launch_bounds__(RT) k_rdot2_zq_rz(const float2* __restrict__ z,
                                                    const float2* __restrict__ q,
                                                    const float2* __restrict__ r, long long count,
                                                    double* ws, double* zr) {
  __shared__ double sh[2 * RT / 32];
  const long long base = (long long)blockIdx.y * count;
  float a = 0.f, b = 0.f;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const float2 zv = z[base + i], qv = q[base + i], rv = r[base + i];
    a = fmaf(zv.x, qv.x, fmaf(zv.y, qv.y, a));
    b = fmaf(rv.x, zv.x, fmaf(rv.y, zv.y, b));
  }
  finish_reduction((double)a, (double)b, ws, zr, sh);
}

cudaError_t rdot2_zq_rz(const void* z32, const void* q32, const void* r32, long long count,
                        int nrhs, double* ws, double* zr, cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  k_rdot2_zq_rz<<<dim3(reduce_blocks(count), nrhs), RT, 0, s>>>(
      (const float2*)z32, (const float2*)q32, (const float2*)r32, count, ws, zr);
  count_launch();
  return cudaGetLastError();
}

// beta = -zr[0] / Re(pq); p = z + beta p (FP32); rz <- {zr[1], 0}.
__global__ void k_rcg_p(float2* __restrict__ p, const float2* __restrict__ z, const double* zr,
                        const double* pq, double* rz, const int* frozen, long long count) {
  const int rhs = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (frozen && frozen[rhs]) return;
  if (i == 0) {
    rz[2 * rhs] = zr[2 * rhs + 1];
    rz[2 * rhs + 1] = 0.0;
  }
  if (i >= count) return;
  const double d = pq[2 * rhs];
  const float beta = d != 0.0 ? (float)(-zr[2 * rhs] / d) : 0.f;
  const long long k = (long long)rhs * count + i;
  const float2 pv = p[k], zv = z[k];
  p[k] = make_float2(fmaf(beta, pv.x, zv.x), fmaf(beta, pv.y, zv.y));
}

cudaError_t rcg_p(void* p32, const void* z32, const double* zr, const double* pq, double* rz,
                  const int* frozen, long long count, int nrhs, cudaStream_t s) {
  k_rcg_p<<<grid1(count, nrhs), RT, 0, s>>>((float2*)p32, (const float2*)z32, zr, pq, rz, frozen,
                                             count);
  count_launch();
  return cudaGetLastError();
}

// Reliable-update test, one thread: for every running right-hand side,
// rmax = max(rmax, rr); an update is due when some rr < delta^2 rmax.  Sets
// *due (and the IF condition of the enclosing graph node when cond_set).
__global__ void k_ru_check(const double* rr, double* rmax, const int* ctrl, double delta2,
                           int* due, int* count, cudaGraphConditionalHandle cond, int cond_set) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nrhs = ctrl[3];
  const int* frozen = ctrl + 4;
  int any = 0;
  for (int k = 0; k < nrhs; ++k) {
    if (frozen[k]) continue;
    const double r = rr[2 * k];
    if (r > rmax[2 * k]) rmax[2 * k] = r;
    if (r < delta2 * rmax[2 * k]) any = 1;
  }
  *due = any;
  if (any) *count += 1;
  if (cond_set) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

cudaError_t ru_check(const double* rr, double* rmax, const int* ctrl, double delta2, int* due,
                     int* count, cudaGraphConditionalHandle cond, bool cond_set, cudaStream_t s) {
  k_ru_check<<<1, 32, 0, s>>>(rr, rmax, ctrl, delta2, due, count, cond, cond_set ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

// x64 += x32, x32 = 0 (the FP32 increment folded into the FP64 solution).
__global__ void k_ru_fold(double2* __restrict__ x, float2* __restrict__ x32, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float2 v = x32[i];
  const double2 xv = x[i];
  x[i] = make_double2(xv.x + (double)v.x, xv.y + (double)v.y);
  x32[i] = make_float2(0.f, 0.f);
}

cudaError_t ru_fold(void* x64, void* x32, long long count, cudaStream_t s) {
  k_ru_fold<<<grid1(count, 1), RT, 0, s>>>((double2*)x64, (float2*)x32, count);
  count_launch();
  return cudaGetLastError();
}

// r32 = (float) r64 and rr = rmax = |r64|^2 (FP64) per right-hand side.
__global__ void __launch_bounds__(RT) k_ru_residual(const double2* __restrict__ r,
                                                    float2* __restrict__ r32, long long count,
                                                    double* ws, double* rr) {
  __shared__ double sh[2 * RT / 32];
  const long long base = (long long)blockIdx.y * count;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < count;
       i += (long long)gridDim.x * RT) {
    const double2 v = r[base + i];
    r32[base + i] = make_float2((float)v.x, (float)v.y);
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  finish_reduction(acc, 0.0, ws, rr, sh);
}

__global__ void k_copy_slots(const double* src, double* dst, int n2) {
  const int i = threadIdx.x;
  if (i < n2) dst[i] = src[i];
}

cudaError_t ru_residual(const void* r64, void* r32, long long count, int nrhs, double* ws,
                        double* rr, double* rmax, cudaStream_t s) {
  if (nrhs > 64) return cudaErrorInvalidValue;
  k_ru_residual<<<dim3(reduce_blocks(count), nrhs), RT, 0, s>>>((const double2*)r64, (float2*)r32,
                                                                count, ws, rr);
  count_launch();
  if (rmax) {
    k_copy_slots<<<1, 128, 0, s>>>(rr, rmax, 2 * nrhs);
    count_launch();
  }
  return cudaGetLastError();
}

__global__ void k_f64_to_f32_scaled(const double2* __restrict__ in, float2* __restrict__ out,
                                    const double* nrm, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double n2 = nrm[2 * blockIdx.y];
  const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  i += (long long)blockIdx.y * count;
  double2 v = in[i];
  out[i] = make_float2((float)(v.x * sc), (float)(v.y * sc));
}

cudaError_t f64_to_f32_scaled(const void* in, void* out, const double* nrm, long long count,
                              int nrhs, cudaStream_t s) {
  k_f64_to_f32_scaled<<<grid1(count, nrhs), RT, 0, s>>>((const double2*)in, (float2*)out, nrm,
                                                         count); count_launch();
  return cudaGetLastError();
}

__global__ void k_f32_acc_scaled(const float2* __restrict__ in, double2* __restrict__ x,
                                 const double* nrm, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double sc = nrm ? sqrt(nrm[2 * blockIdx.y]) : 1.0;
  i += (long long)blockIdx.y * count;
  float2 v = in[i];
  double2 xv = x[i];
  x[i] = make_double2(fma((double)v.x, sc, xv.x), fma((double)v.y, sc, xv.y));
}

cudaError_t f32_accumulate_scaled(const void* in, void* x, const double* nrm, long long count,
                                  int nrhs, cudaStream_t s) {
  k_f32_acc_scaled<<<grid1(count, nrhs), RT, 0, s>>>((const float2*)in, (double2*)x, nrm, count); count_launch();
  return cudaGetLastError();
}

__global__ void k_cvt_64_32(const double2* __restrict__ in, float2* __restrict__ out,
                            long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_cvt_32_64(const float2* __restrict__ in, double2* __restrict__ out,
                            long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = make_double2(in[i].x, in[i].y);
}
cudaError_t convert_f64_f32(const void* in, void* out, long long count, cudaStream_t s) {
  k_cvt_64_32<<<grid1(count, 1), RT, 0, s>>>((const double2*)in, (float2*)out, count); count_launch();
  return cudaGetLastError();
}
cudaError_t convert_f32_f64(const void* in, void* out, long long count, cudaStream_t s) {
  k_cvt_32_64<<<grid1(count, 1), RT, 0, s>>>((const float2*)in, (double2*)out, count); count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_lincomb(cplx_t<R>* out, R a, const cplx_t<R>* u, R b, const cplx_t<R>* v, R c,
                          const cplx_t<R>* w, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  i += (long long)blockIdx.y * count;
  cplx_t<R> uu = u[i], vv = v[i];
  R re = a * uu.x + b * vv.x, im = a * uu.y + b * vv.y;
  if (w) {
    cplx_t<R> ww = w[i];
    re += c * ww.x;
    im += c * ww.y;
  }
  out[i] = mk(re, im);
}

template <typename R>
cudaError_t lincomb(void* out, double a, const void* u, double b, const void* v, double c,
                    const void* w, long long count, int nrhs, cudaStream_t s) {
  k_lincomb<R><<<grid1(count, nrhs), RT, 0, s>>>((cplx_t<R>*)out, (R)a, (const cplx_t<R>*)u, (R)b,
                                                  (const cplx_t<R>*)v, (R)c,
                                                  (const cplx_t<R>*)w, count); count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_sub_from(const cplx_t<R>* __restrict__ b, cplx_t<R>* __restrict__ r,
                           long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) r[i] = csub(b[i], r[i]);
}
template <typename R>
cudaError_t sub_from(const void* b, void* r, long long count, cudaStream_t s) {
  k_sub_from<R><<<grid1(count, 1), RT, 0, s>>>((const cplx_t<R>*)b, (cplx_t<R>*)r, count); count_launch();
  return cudaGetLastError();
}

#define INST(R)                                                                              \
  template cudaError_t dot<R>(const void*, const void*, long long, int, double*, double*,    \
                              cudaStream_t);                                                 \
  template cudaError_t norm2<R>(const void*, long long, int, double*, double*, cudaStream_t); \
  template cudaError_t axpby<R>(double, const void*, double, void*, long long, int,          \
                                cudaStream_t);                                               \
  template cudaError_t scale_inv_sqrt<R>(const void*, void*, const double*, long long, int,  \
                                         cudaStream_t);                                      \
  template cudaError_t cg_xr<R>(void*, void*, const void*, const void*, const double*,       \
                                const double*, const int*, long long, int, double*, double*, \
                                cudaStream_t, void*, const CgControl*);                      \
  template cudaError_t cg_p<R>(void*, const void*, const double*, const double*, const int*, \
                               long long, int, cudaStream_t);                                \
  template cudaError_t sub_from<R>(const void*, void*, long long, cudaStream_t);             \
  template cudaError_t lincomb<R>(void*, double, const void*, double, const void*, double,   \
                                  const void*, long long, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace mgk
