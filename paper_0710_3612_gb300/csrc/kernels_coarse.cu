// Coarse-grid kernels of the V-cycle and the adaptive setup:
//  * coarse_apply     -- 9-point block stencil of the Galerkin operator (Eq. Galerkin)
//  * restrict/prolong -- P^dagger and P built from block vectors (Sec. 2, Eq. P1)
//  * block Gram-Schmidt of the chirality halves of the relaxed vectors (Sec. 3)
//  * Galerkin build: level 1 from W = D P on blocks plus a one-site halo,
//    levels >= 2 from the block formula P(i)^dagger A_l[i, e] P(i + e)
//  * coarsest level: dense FP32 Gauss-Jordan inverse and GEMV (the FP64
//    refinement around them lives in the host orchestration)
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mgk {

// ---------------------------------------------------------------------------
// Coarse stencil apply: y(j)[r] = sum_d sum_c A[j][d][r][c] x(j + d)[c]
// ---------------------------------------------------------------------------
template <typename W> struct wload;
template <> struct wload<double2> {
  static __device__ __forceinline__ double2 get(const double2* p) { return *p; }
};
template <> struct wload<float2> {
  static __device__ __forceinline__ float2 get(const float2* p) { return *p; }
};
template <> struct wload<__nv_bfloat162> {
  static __device__ __forceinline__ float2 get(const __nv_bfloat162* p) { return bf2_to_f2(*p); }
};

// One CTA per (coarse site, rhs), 9 n threads: thread (d, r) forms the partial
// row product A[j][d][r][:] . x(j + d); the 9 partials of a row are summed in
// a fixed order (deterministic).  The 9 neighbour vectors are staged in shared
// memory; each thread streams one contiguous block row with vector loads.
template <typename R> struct row_dot;
template <> struct row_dot<double> {
  template <typename WT>
  static __device__ __forceinline__ double2 run(const WT* row, const double2* x, int n) {
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < n; ++c) cfma(acc, row[c], x[c]);
    return acc;
  }
};
template <> struct row_dot<float> {
  static __device__ __forceinline__ float2 run(const float2* row, const float2* x, int n) {
    float2 acc = make_float2(0.f, 0.f);
    const float4* r4 = (const float4*)row;
    for (int c = 0; c < n / 2; ++c) {
      const float4 w = r4[c];
      cfma(acc, make_float2(w.x, w.y), x[2 * c]);
      cfma(acc, make_float2(w.z, w.w), x[2 * c + 1]);
    }
    return acc;
  }
  static __device__ __forceinline__ float2 run(const __nv_bfloat162* row, const float2* x, int n) {
    float2 acc = make_float2(0.f, 0.f);
    const uint2* r2 = (const uint2*)row;
    for (int c = 0; c < n / 2; ++c) {
      const uint2 w = r2[c];
      cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.x), x[2 * c]);
      cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.y), x[2 * c + 1]);
    }
    return acc;
  }
};

template <typename R, typename WT>
__global__ void __launch_bounds__(576, 2) k_coarse_apply(const cplx_t<R>* __restrict__ in,
                                                      cplx_t<R>* out,
                                                      const WT* __restrict__ A, int Lx, int Lt,
                                                      int n, Epilogue ep) {
  extern __shared__ unsigned char smraw[];
  cplx_t<R>* xs = (cplx_t<R>*)smraw;            // [9][n] neighbour vectors
  cplx_t<R>* part = xs + 9 * n;                 // [9][n] partial row products
  const int V = Lx * Lt;
  const int j = blockIdx.x;
  const int x = j % Lx, t = j / Lx;
  const cplx_t<R>* vin = in + (long long)blockIdx.y * V * n;
  // BF16 rows of up to 24 entries are loaded into registers before the
  // neighbour vectors are staged, so the two global reads overlap
  constexpr bool kBf16 = std::is_same<WT, __nv_bfloat162>::value;
  constexpr int PRE = 6;                         // 16-byte chunks (4 entries each)
  const bool pre = kBf16 && n <= 4 * PRE && n % 4 == 0;
  uint4 rv[PRE];
  if constexpr (kBf16) {
    if (pre && threadIdx.x < 9 * n) {
      const int d = threadIdx.x / n, r = threadIdx.x % n;
      const uint4* row4 = (const uint4*)(A + (((long long)j * 9 + d) * n + r) * n);
#pragma unroll
      for (int k = 0; k < PRE; ++k)
        if (k < n / 4) rv[k] = __ldg(row4 + k);
    }
  }
  // epilogue operands are read up front as well (off the critical path)
  cplx_t<R> eu = mk((R)0, (R)0), ew = mk((R)0, (R)0);
  if (threadIdx.x < n) {
    const long long o = ((long long)blockIdx.y * V + j) * n + threadIdx.x;
    if (ep.U) eu = ((const cplx_t<R>*)ep.U)[o];
    if (ep.W) ew = ((const cplx_t<R>*)ep.W)[o];
  }
  for (int q = threadIdx.x; q < 9 * n; q += blockDim.x) {
    const int d = q / n, c = q % n;
    int xn = x + d % 3 - 1, tn = t + d / 3 - 1;
    xn = xn < 0 ? xn + Lx : (xn >= Lx ? xn - Lx : xn);
    tn = tn < 0 ? tn + Lt : (tn >= Lt ? tn - Lt : tn);
    xs[q] = vin[(long long)(xn + Lx * tn) * n + c];
  }
  __syncthreads();
  const int q = threadIdx.x;
  if (q < 9 * n) {
    const int d = q / n, r = q % n;
    bool done = false;
    if constexpr (kBf16 && sizeof(R) == 4) {
      if (pre) {
        const float2* xv = xs + d * n;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < PRE; ++k) {
          if (k < n / 4) {
            const uint4 w = rv[k];
            cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.x), xv[4 * k]);
            cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.y), xv[4 * k + 1]);
            cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.z), xv[4 * k + 2]);
            cfma(acc, bf2_to_f2(*(const __nv_bfloat162*)&w.w), xv[4 * k + 3]);
          }
        }
        part[q] = acc;
        done = true;
      }
    }
    if (!done) {
      const WT* row = A + (((long long)j * 9 + d) * n + r) * n;
      part[q] = row_dot<R>::run(row, xs + d * n, n);
    }
  }
  __syncthreads();
  if (q < n) {
    cplx_t<R> acc = part[q];
#pragma unroll
    for (int d = 1; d < 9; ++d) acc = cadd(acc, part[d * n + q]);
    const long long o = ((long long)blockIdx.y * V + j) * n + q;
    acc = mk((R)ep.ca * acc.x, (R)ep.ca * acc.y);
    if (ep.U) acc = mk(acc.x + (R)ep.cu * eu.x, acc.y + (R)ep.cu * eu.y);
    if (ep.W) acc = mk(acc.x + (R)ep.cw * ew.x, acc.y + (R)ep.cw * ew.y);
    out[o] = acc;
  }
}

// Multi-RHS coarse apply on tensor cores (BF16 operands, FP32 accumulation).
// One CTA per coarse site j.  The complex contraction Y = sum_d A_j,d X_{j+d}
// (n x 9n times 9n x nrhs) is realified with K ordered as (re, im) pairs, so
// that one 32-bit register of an A fragment is one complex block entry --
// (re, -im) for the rows of Re Y and (im, re) for the rows of Im Y -- and one
// register of a B fragment is one complex entry of X.  mma.sync m16n8k16:
// M = 16 complex rows (Re and Im tiles), N = 8 right-hand sides, K = 8
// complex columns per step.  X is staged in shared memory as a pair of bf16
// splits, X = Xhi + Xlo (Xlo = bf16(X - Xhi)), each [9n][16 + 8] per chunk of
// 16 right-hand sides (padding keeps the fragment loads conflict-free); two
// MMAs per product carry X to about 16 significant bits, so only the stored
// BF16 blocks round.
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *(uint32_t*)&v; }

// CTA = (coarse site j, chunk of 16 right-hand sides), two warps, one 8-wide
// n-tile each; the A fragments of a K step are loaded once per warp.
static constexpr int MMA_RC = 16;            // right-hand sides per CTA

__global__ void __launch_bounds__(64) k_coarse_apply_mma(const float2* __restrict__ in, float2* out,
                                                         const __nv_bfloat162* __restrict__ A,
                                                         int Lx, int Lt, int n, int nrhs,
                                                         Epilogue ep) {
  extern __shared__ __nv_bfloat162 Xs[];
  constexpr int RS = MMA_RC + 8;             // padded row: conflict-free fragment loads
  const int V = Lx * Lt;
  const int j = blockIdx.x, rhs0 = blockIdx.y * MMA_RC;
  const int x = j % Lx, t = j / Lx;
  const int tid = threadIdx.x;
  __nv_bfloat162* Xl = Xs + 9 * n * RS;
  // stage X(j + d) for the 9 displacements, this chunk of right-hand sides
  // (dof fastest: one 8 n-byte segment per (d, rhs)), as hi + lo bf16 parts
  for (int q = tid; q < 9 * n * MMA_RC; q += blockDim.x) {
    const int sdof = q % n, rr = (q / n) % MMA_RC, d = q / (n * MMA_RC), c = d * n + sdof;
    int xn = x + d % 3 - 1, tn = t + d / 3 - 1;
    xn = xn < 0 ? xn + Lx : (xn >= Lx ? xn - Lx : xn);
    tn = tn < 0 ? tn + Lt : (tn >= Lt ? tn - Lt : tn);
    float2 v = make_float2(0.f, 0.f);
    if (rhs0 + rr < nrhs) v = in[((long long)(rhs0 + rr) * V + xn + Lx * tn) * n + sdof];
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(hi);
    Xs[c * RS + rr] = hi;
    Xl[c * RS + rr] = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tg = lane & 3;
  const int nt = warp;                        // 8 right-hand sides per warp
  const __nv_bfloat162 zero = __floats2bfloat162_rn(0.f, 0.f);
  for (int r0 = 0; r0 < n; r0 += 16) {
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    const int ra = r0 + g, rb = r0 + g + 8;
#pragma unroll 2
    for (int c0 = 0; c0 < 9 * n; c0 += 8) {
      const int d = c0 / n, s0 = c0 % n;
      const __nv_bfloat162* Ab = A + (((long long)j * 9 + d) * n) * n;
      __nv_bfloat162 e[4];
      e[0] = ra < n ? Ab[ra * n + s0 + tg] : zero;
      e[1] = rb < n ? Ab[rb * n + s0 + tg] : zero;
      e[2] = ra < n ? Ab[ra * n + s0 + tg + 4] : zero;
      e[3] = rb < n ? Ab[rb * n + s0 + tg + 4] : zero;
      uint32_t aRe[4], aIm[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        aRe[u] = bf2_bits(__halves2bfloat162(e[u].x, __hneg(e[u].y)));   // (re, -im)
        aIm[u] = bf2_bits(__halves2bfloat162(e[u].y, e[u].x));           // (im, re)
      }
      const int i0 = (c0 + tg) * RS + nt * 8 + g, i1 = (c0 + tg + 4) * RS + nt * 8 + g;
      const uint32_t b0 = bf2_bits(Xs[i0]), b1 = bf2_bits(Xs[i1]);
      const uint32_t l0 = bf2_bits(Xl[i0]), l1 = bf2_bits(Xl[i1]);
      mma_bf16_16816(re, aRe, b0, b1);
      mma_bf16_16816(im, aIm, b0, b1);
      mma_bf16_16816(re, aRe, l0, l1);
      mma_bf16_16816(im, aIm, l0, l1);
    }
    // c[0], c[1]: row g, rhs 2tg, 2tg+1; c[2], c[3]: row g + 8
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + g + (u >= 2 ? 8 : 0);
      const int rhs = rhs0 + nt * 8 + 2 * tg + (u & 1);
      if (r >= n || rhs >= nrhs) continue;
      const long long o = ((long long)rhs * V + j) * n + r;
      float2 y = make_float2((float)ep.ca * re[u], (float)ep.ca * im[u]);
      if (ep.U) {
        const float2 w = ((const float2*)ep.U)[o];
        y = make_float2(y.x + (float)ep.cu * w.x, y.y + (float)ep.cu * w.y);
      }
      if (ep.W) {
        const float2 w = ((const float2*)ep.W)[o];
        y = make_float2(y.x + (float)ep.cw * w.x, y.y + (float)ep.cw * w.y);
      }
      out[o] = y;
    }
  }
}

bool coarse_apply_tensor(int weights, int n, int nrhs) {
  return weights == W_BF16 && nrhs >= 8 && n % 8 == 0 && n <= 32 && nrhs <= 64;
}

static std::atomic<int> g_coarse_tensor_kernel{0};

void set_coarse_tensor_kernel(int kind) { g_coarse_tensor_kernel.store(kind); }

cudaError_t coarse_apply(const void* in, void* out, const void* A, int weights, int Lx, int Lt,
                         int n, int nrhs, const Epilogue& ep, cudaStream_t s) {
  if (n % 2 || 9 * n > 576) return cudaErrorInvalidValue;
  if (coarse_apply_tensor(weights, n, nrhs) && g_coarse_tensor_kernel.load() == 0 &&
      coarse_apply_tcgen05_ok(n, nrhs))
    return coarse_apply_tcgen05(in, out, A, Lx, Lt, n, nrhs, ep, s);
  if (coarse_apply_tensor(weights, n, nrhs)) {
    const size_t smem = (size_t)2 * 9 * n * (MMA_RC + 8) * sizeof(__nv_bfloat162);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_coarse_apply_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           64 * 1024);
      attr = true;
    }
    dim3 grid(Lx * Lt, (nrhs + MMA_RC - 1) / MMA_RC);
    k_coarse_apply_mma<<<grid, 64, smem, s>>>((const float2*)in, (float2*)out,
                                              (const __nv_bfloat162*)A, Lx, Lt, n, nrhs, ep);
    count_launch();
    return cudaGetLastError();
  }
  dim3 grid(Lx * Lt, nrhs);
  const int threads = (9 * n + 31) / 32 * 32;
  if (weights == W_F64)
    k_coarse_apply<double, double2><<<grid, threads, 18 * n * sizeof(double2), s>>>(
        (const double2*)in, (double2*)out, (const double2*)A, Lx, Lt, n, ep);
  else if (weights == W_F32)
    k_coarse_apply<float, float2><<<grid, threads, 18 * n * sizeof(float2), s>>>(
        (const float2*)in, (float2*)out, (const float2*)A, Lx, Lt, n, ep);
  else
    k_coarse_apply<float, __nv_bfloat162><<<grid, threads, 18 * n * sizeof(float2), s>>>(
        (const float2*)in, (float2*)out, (const __nv_bfloat162*)A, Lx, Lt, n, ep);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_coarse_convert(const double2* __restrict__ a, void* out, int weights,
                                 long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 v = a[i];
  if (weights == W_F32)
    ((float2*)out)[i] = make_float2((float)v.x, (float)v.y);
  else
    ((__nv_bfloat162*)out)[i] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

cudaError_t coarse_convert(const void* A64, void* out, int weights, long long count,
                           cudaStream_t s) {
  k_coarse_convert<<<(unsigned)((count + 255) / 256), 256, 0, s>>>((const double2*)A64, out,
                                                                   weights, count); count_launch();
  return cudaGetLastError();
}

// out = a X + b Y + c I on 9-point block stencils [site][d][r][s] (I: the
// identity blocks of the d = 4 displacement); out may alias X or Y.
__global__ void k_coarse_lincomb(double a, const double2* X, double b, const double2* Y, double c,
                                 double2* out, long long count, int n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int q = (int)(i % ((long long)9 * n * n));
  const int d = q / (n * n), r = (q / n) % n, sc = q % n;
  const double2 x = X[i], y = Y[i];
  double re = a * x.x + b * y.x, im = a * x.y + b * y.y;
  if (d == 4 && r == sc) re += c;
  out[i] = make_double2(re, im);
}

cudaError_t coarse_lincomb(double a, const void* X, double b, const void* Y, double c, void* out,
                           long long sites, int n, cudaStream_t s) {
  const long long count = sites * 9 * n * n;
  k_coarse_lincomb<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(
      a, (const double2*)X, b, (const double2*)Y, c, (double2*)out, count, n);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Column probing of a coarse operator whose couplings reach one block (the
// Galerkin product of the smoothed prolongator, Sec. 3).  Sites are coloured
// by (x mod Kx, t mod Kt) with Kx, Kt >= 3 dividing the extents, so that two
// sites of one colour are never within one block of the same site.
// ---------------------------------------------------------------------------
__global__ void k_probe_vectors(double2* __restrict__ out, int Lxc, int Ltc, int nc, int Kx, int Kt,
                                int cx, int ct) {
  const long long Vc = (long long)Lxc * Ltc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nc * Vc * nc) return;
  const int r = (int)(idx % nc), s = (int)(idx / (Vc * nc));
  const int j = (int)((idx / nc) % Vc), jx = j % Lxc, jt = j / Lxc;
  const bool on = r == s && jx % Kx == cx && jt % Kt == ct;
  out[idx] = make_double2(on ? 1.0 : 0.0, 0.0);
}

__global__ void k_probe_scatter(const double2* __restrict__ y, double2* __restrict__ Ac, int Lxc,
                                int Ltc, int nc, int Kx, int Kt, int cx, int ct) {
  const long long Vc = (long long)Lxc * Ltc;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Vc * 9 * nc * nc) return;
  const int sc = (int)(idx % nc), r = (int)((idx / nc) % nc), d = (int)((idx / ((long long)nc * nc)) % 9);
  const int j = (int)(idx / (9LL * nc * nc)), jx = j % Lxc, jt = j / Lxc;
  const int xn = (jx + d % 3 - 1 + Lxc) % Lxc, tn = (jt + d / 3 - 1 + Ltc) % Ltc;
  if (xn % Kx == cx && tn % Kt == ct) Ac[idx] = y[((long long)sc * Vc + j) * nc + r];
}

cudaError_t probe_vectors(void* out, int Lxc, int Ltc, int nc, int Kx, int Kt, int cx, int ct,
                          cudaStream_t s) {
  const long long n = (long long)nc * Lxc * Ltc * nc;
  k_probe_vectors<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double2*)out, Lxc, Ltc, nc, Kx, Kt,
                                                            cx, ct);
  count_launch();
  return cudaGetLastError();
}

cudaError_t probe_scatter(const void* y, void* Ac, int Lxc, int Ltc, int nc, int Kx, int Kt, int cx,
                          int ct, cudaStream_t s) {
  const long long n = (long long)Lxc * Ltc * 9 * nc * nc;
  k_probe_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)y, (double2*)Ac, Lxc,
                                                            Ltc, nc, Kx, Kt, cx, ct);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Restriction and prolongation.  Vst[i][c][k][a]: component c*h + a of vector
// k at fine site i, orthonormal per (block, chirality).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_site(int j, int o, int Lxc, int Lx, int bx, int bt) {
  const int jx = j % Lxc, jt = j / Lxc;
  return (jx * bx + o % bx) + Lx * (jt * bt + o / bx);
}

// One warp per output (j, c, k): the lanes stride over the bx*bt*h entries of
// the block-chirality vector, the warp sums the products in a fixed
// butterfly order.
template <typename R>
__global__ void __launch_bounds__(256) k_restrict(const cplx_t<R>* __restrict__ fine,
                                                  cplx_t<R>* __restrict__ coarse,
                                                  const cplx_t<R>* __restrict__ Vst, int Lx,
                                                  int Lt, int bx, int bt, int h, int Nv) {
  const int Lxc = Lx / bx, Vc = Lxc * (Lt / bt), nc = 2 * Nv, nf = 2 * h;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= Vc * nc) return;
  const int j = w / nc, s = w % nc, c = s / Nv, k = s % Nv;
  const cplx_t<R>* f = fine + (long long)blockIdx.y * Lx * Lt * nf;
  const int m = bx * bt * h;
  double re = 0.0, im = 0.0;
  for (int e = lane; e < m; e += 32) {
    const int o = e / h, a = e % h;
    const int i = block_site(j, o, Lxc, Lx, bx, bt);
    const cplx_t<R> v = Vst[(((long long)i * 2 + c) * Nv + k) * h + a];
    const cplx_t<R> r = f[(long long)i * nf + c * h + a];
    re += (double)v.x * r.x + (double)v.y * r.y;
    im += (double)v.x * r.y - (double)v.y * r.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) coarse[(long long)blockIdx.y * Vc * nc + w] = mk((R)re, (R)im);
}

// One CTA per coarse site j stages the block's vectors and the block's slice
// of every right-hand side in shared memory, so the vectors are read once per
// site for all right-hand sides and every output is a short in-CTA sum.
// (The warp-per-output kernels serve blocks too large for shared memory.)
// Transfer kernels with one CTA per coarse site j.  The block's null-vector
// rows and the inputs of all right-hand sides are staged in shared memory;
// each output is then summed by a group of G consecutive lanes (G a power of
// two, chosen so that the outputs x G fill the CTA), which split the terms and
// combine them with a fixed shuffle tree.
template <typename C>
__device__ __forceinline__ C group_sum(C v, int G) {
  for (int off = G >> 1; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Restriction: coarse(j, c Nv + k) = sum over the T = b2 h entries t = (o, a)
// of chirality c in block j of conj(v_k(t)) r(t).  Shared layouts keep t
// fastest: sv[(c Nv + k) T + t], sr[(rhs 2 + c) T + t].
template <typename R>
__global__ void __launch_bounds__(256) k_restrict_multi(const cplx_t<R>* __restrict__ fine,
                                                        cplx_t<R>* __restrict__ coarse,
                                                        const cplx_t<R>* __restrict__ Vst, int Lx,
                                                        int Lt, int bx, int bt, int h, int Nv,
                                                        int nrhs, int G) {
  using C = cplx_t<R>;
  extern __shared__ unsigned char smraw[];
  const int b2 = bx * bt, nf = 2 * h, nc = 2 * Nv, T = b2 * h, Lxc = Lx / bx, Vc = Lxc * (Lt / bt);
  const int TP = T | 1;                                 // odd row stride: conflict-free row reads
  C* sv = (C*)smraw;
  C* sr = sv + 2 * Nv * TP;
  const int j = blockIdx.x, V = Lx * Lt;
  for (int q = threadIdx.x; q < b2 * 2 * Nv * h; q += blockDim.x) {
    const int o = q / (2 * Nv * h), rest = q % (2 * Nv * h);
    const int ck = rest / h, a = rest % h;                // ck = c Nv + k
    sv[ck * TP + o * h + a] = Vst[(long long)block_site(j, o, Lxc, Lx, bx, bt) * 2 * Nv * h + rest];
  }
  for (int q = threadIdx.x; q < nrhs * b2 * nf; q += blockDim.x) {
    const int comp = q % nf, o = (q / nf) % b2, rhs = q / (nf * b2);
    const int c = comp / h, a = comp % h;
    sr[(rhs * 2 + c) * TP + o * h + a] =
        fine[((long long)rhs * V + block_site(j, o, Lxc, Lx, bx, bt)) * nf + comp];
  }
  __syncthreads();
  const int g = threadIdx.x % G, per = blockDim.x / G, nout = nrhs * nc;
  for (int q0 = 0; q0 < nout; q0 += per) {
    const int q = q0 + threadIdx.x / G;
    C acc = mk((R)0, (R)0);
    if (q < nout) {
      const int sidx = q % nc, rhs = q / nc, c = sidx / Nv;
      const C* v = sv + sidx * TP;
      const C* r = sr + (rhs * 2 + c) * TP;
      for (int t = g; t < T; t += G) cfmac(acc, v[t], r[t]);
    }
    acc = group_sum(acc, G);
    if (q < nout && g == 0) coarse[((long long)(q / nc) * Vc + j) * nc + q % nc] = acc;
  }
}

// Prolongation: fine(i, c, a) (+)= sum over k of v_k(i, c, a) e(j, c Nv + k);
// G lanes split the Nv terms of one output.
template <typename R>
__global__ void __launch_bounds__(256) k_prolong_multi(const cplx_t<R>* __restrict__ coarse,
                                                       cplx_t<R>* __restrict__ fine,
                                                       const cplx_t<R>* __restrict__ Vst, int Lx,
                                                       int Lt, int bx, int bt, int h, int Nv,
                                                       int nrhs, bool accumulate, int G) {
  using C = cplx_t<R>;
  extern __shared__ unsigned char smraw[];
  const int b2 = bx * bt, nf = 2 * h, nc = 2 * Nv, Lxc = Lx / bx, Vc = Lxc * (Lt / bt);
  const int RS = (Nv * h) | 1;                       // odd row stride: conflict-free row reads
  C* sv = (C*)smraw;                                 // [b2][2] rows of [Nv][h], stride RS
  C* se = sv + b2 * 2 * RS;                          // [nrhs][nc]
  const int j = blockIdx.x, V = Lx * Lt;
  for (int q = threadIdx.x; q < b2 * 2 * Nv * h; q += blockDim.x) {
    const int o = q / (2 * Nv * h), rest = q % (2 * Nv * h);
    sv[(o * 2 + rest / (Nv * h)) * RS + rest % (Nv * h)] =
        Vst[(long long)block_site(j, o, Lxc, Lx, bx, bt) * 2 * Nv * h + rest];
  }
  for (int q = threadIdx.x; q < nrhs * nc; q += blockDim.x)
    se[q] = coarse[((long long)(q / nc) * Vc + j) * nc + q % nc];
  __syncthreads();
  const int g = threadIdx.x % G, per = blockDim.x / G, nout = nrhs * b2 * nf;
  for (int q0 = 0; q0 < nout; q0 += per) {
    const int q = q0 + threadIdx.x / G;
    C acc = mk((R)0, (R)0);
    int o = 0, comp = 0, rhs = 0;
    if (q < nout) {
      comp = q % nf;
      o = (q / nf) % b2;
      rhs = q / (nf * b2);
      const int c = comp / h, a = comp % h;
      for (int k = g; k < Nv; k += G)
        cfma(acc, sv[(o * 2 + c) * RS + k * h + a], se[rhs * nc + c * Nv + k]);
    }
    acc = group_sum(acc, G);
    if (q < nout && g == 0) {
      const long long gi = ((long long)rhs * V + block_site(j, o, Lxc, Lx, bx, bt)) * nf + comp;
      fine[gi] = accumulate ? cadd(fine[gi], acc) : acc;
    }
  }
}

// Lanes per output: the largest power of two <= min(terms, 16) whose product
// with the output count still fits in one 256-thread CTA (at least 1).
static int transfer_group(int outputs, int terms) {
  int G = 16;
  while (G > 1 && (G > terms || (long long)outputs * G > 256)) G >>= 1;
  return G;
}

static size_t transfer_multi_smem(int bx, int bt, int h, int Nv, int nrhs, size_t csz, bool restr) {
  const size_t b2 = (size_t)bx * bt;
  const size_t vrows = restr ? (size_t)2 * Nv * ((b2 * h) | 1) : b2 * 2 * (((size_t)Nv * h) | 1);
  return csz * (vrows + (restr ? (size_t)nrhs * 2 * ((b2 * h) | 1) : (size_t)nrhs * 2 * Nv));
}

template <typename R>
cudaError_t restrict_op(const void* fine, void* coarse, const void* Vst, int Lx, int Lt, int bx,
                        int bt, int h, int Nv, int nrhs, cudaStream_t s) {
  const size_t sm = transfer_multi_smem(bx, bt, h, Nv, nrhs, sizeof(cplx_t<R>), true);
  if (sm <= 96 * 1024) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_restrict_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr = true;
    }
    k_restrict_multi<R><<<(Lx / bx) * (Lt / bt), 256, sm, s>>>(
        (const cplx_t<R>*)fine, (cplx_t<R>*)coarse, (const cplx_t<R>*)Vst, Lx, Lt, bx, bt, h, Nv,
        nrhs, transfer_group(nrhs * 2 * Nv, bx * bt * h));
    count_launch();
    return cudaGetLastError();
  }
  const int warps = (Lx / bx) * (Lt / bt) * 2 * Nv;
  k_restrict<R><<<dim3((warps + 7) / 8, nrhs), 256, 0, s>>>(
      (const cplx_t<R>*)fine, (cplx_t<R>*)coarse, (const cplx_t<R>*)Vst, Lx, Lt, bx, bt, h, Nv);
  count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_prolong(const cplx_t<R>* __restrict__ coarse, cplx_t<R>* __restrict__ fine,
                          const cplx_t<R>* __restrict__ Vst, int Lx, int Lt, int bx, int bt, int h,
                          int Nv, bool accumulate) {
  const int V = Lx * Lt, nf = 2 * h, nc = 2 * Nv;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V * nf) return;
  const int i = idx / nf, comp = idx % nf, c = comp / h, a = comp % h;
  const int x = i % Lx, t = i / Lx;
  const int j = coarse_site(x, t, Lx, bx, bt);
  const cplx_t<R>* e = coarse + (long long)blockIdx.y * (V / (bx * bt)) * nc + (long long)j * nc +
                       c * Nv;
  const cplx_t<R>* v = Vst + ((long long)i * 2 + c) * Nv * h + a;
  cplx_t<R> acc = mk((R)0, (R)0);
  for (int k = 0; k < Nv; ++k) cfma(acc, v[(long long)k * h], e[k]);
  const long long o = (long long)blockIdx.y * V * nf + idx;
  fine[o] = accumulate ? cadd(fine[o], acc) : acc;
}

template <typename R>
cudaError_t prolong_op(const void* coarse, void* fine, const void* Vst, int Lx, int Lt, int bx,
                       int bt, int h, int Nv, int nrhs, bool accumulate, cudaStream_t s) {
  const size_t sm = transfer_multi_smem(bx, bt, h, Nv, nrhs, sizeof(cplx_t<R>), false);
  if (sm <= 96 * 1024) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_prolong_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr = true;
    }
    k_prolong_multi<R><<<(Lx / bx) * (Lt / bt), 256, sm, s>>>(
        (const cplx_t<R>*)coarse, (cplx_t<R>*)fine, (const cplx_t<R>*)Vst, Lx, Lt, bx, bt, h, Nv,
        nrhs, accumulate, transfer_group(nrhs * bx * bt * 2 * h, Nv));
    count_launch();
    return cudaGetLastError();
  }
  const int tot = Lx * Lt * 2 * h;
  k_prolong<R><<<dim3((tot + 255) / 256, nrhs), 256, 0, s>>>(
      (const cplx_t<R>*)coarse, (cplx_t<R>*)fine, (const cplx_t<R>*)Vst, Lx, Lt, bx, bt, h, Nv,
      accumulate); count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Chirality-split block modified Gram-Schmidt, one warp per (block, chirality).
// The m = bx*bt*h entries of a block vector are spread over the 32 lanes
// (entry e = lane + 32 q); orthonormalised vectors are kept in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

static constexpr int GS_MAXQ = 8;   // up to 256 entries per block vector

__global__ void __launch_bounds__(32) k_block_gs(const double2* __restrict__ E,
                                                 double2* __restrict__ Vst, int Lx, int Lt,
                                                 int bx, int bt, int h, int Nv, double tol,
                                                 int* flag) {
  extern __shared__ double2 Q[];   // [Nv][m]
  const int V = Lx * Lt, nf = 2 * h, Lxc = Lx / bx;
  const int j = blockIdx.x >> 1, c = blockIdx.x & 1, lane = threadIdx.x;
  const int m = bx * bt * h, nq = (m + 31) / 32;
  for (int k = 0; k < Nv; ++k) {
    double2 u[GS_MAXQ];
    double n0 = 0.0;
#pragma unroll
    for (int q = 0; q < GS_MAXQ; ++q) {
      u[q] = make_double2(0.0, 0.0);
      const int e = lane + 32 * q;
      if (q < nq && e < m) {
        const int o = e / h, a = e % h;
        const int i = block_site(j, o, Lxc, Lx, bx, bt);
        u[q] = E[((long long)k * V + i) * nf + c * h + a];
        n0 += u[q].x * u[q].x + u[q].y * u[q].y;
      }
    }
    n0 = warp_sum(n0);
    for (int pass = 0; pass < 2; ++pass) {
      for (int kk = 0; kk < k; ++kk) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int q = 0; q < GS_MAXQ; ++q) {
          const int e = lane + 32 * q;
          if (q < nq && e < m) {
            double2 w = Q[kk * m + e];
            re += w.x * u[q].x + w.y * u[q].y;
            im += w.x * u[q].y - w.y * u[q].x;
          }
        }
        re = warp_sum(re);
        im = warp_sum(im);
#pragma unroll
        for (int q = 0; q < GS_MAXQ; ++q) {
          const int e = lane + 32 * q;
          if (q < nq && e < m) {
            double2 w = Q[kk * m + e];
            u[q].x -= re * w.x - im * w.y;
            u[q].y -= re * w.y + im * w.x;
          }
        }
      }
    }
    double n1 = 0.0;
#pragma unroll
    for (int q = 0; q < GS_MAXQ; ++q)
      if (q < nq) n1 += u[q].x * u[q].x + u[q].y * u[q].y;
    n1 = warp_sum(n1);
    if (!(n1 > tol * tol * n0)) {
      if (lane == 0) atomicExch(flag, 1);
      n1 = n1 > 0.0 ? n1 : 1.0;
    }
    const double inv = 1.0 / sqrt(n1);
#pragma unroll
    for (int q = 0; q < GS_MAXQ; ++q) {
      const int e = lane + 32 * q;
      if (q < nq && e < m) {
        double2 w = make_double2(u[q].x * inv, u[q].y * inv);
        Q[k * m + e] = w;
        const int o = e / h, a = e % h;
        const int i = block_site(j, o, Lxc, Lx, bx, bt);
        Vst[(((long long)i * 2 + c) * Nv + k) * h + a] = w;
      }
    }
    __syncwarp();
  }
}

cudaError_t block_gram_schmidt(const void* E, void* Vst, int Lx, int Lt, int bx, int bt, int h,
                               int Nv, double breakdown_tol, int* flag, cudaStream_t s) {
  const int m = bx * bt * h;
  if (m > 32 * GS_MAXQ) return cudaErrorInvalidValue;
  const int Vc = (Lx / bx) * (Lt / bt);
  const size_t smem = (size_t)Nv * m * sizeof(double2);
  k_block_gs<<<2 * Vc, 32, smem, s>>>((const double2*)E, (double2*)Vst, Lx, Lt, bx, bt, h, Nv,
                                     breakdown_tol, flag); count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Level-1 Galerkin.  W_{j,s} = D P e_{j,s} on the extended block
// [-1, bx] x [-1, bt] (local coordinates of block j); then
// A_c[j][d][r][s] = sum_x W_{j,r}(x)^dagger W_{j+d,s}(x) over the overlap of
// the two extended blocks, taken in unwrapped coordinates so that the two
// couplings of a coarse extent of 2 stay in separate displacement slots.
// ---------------------------------------------------------------------------
__global__ void k_galerkin_W(const double2* __restrict__ U, double diag,
                             const double2* __restrict__ Vst, double2* __restrict__ Wbuf, int Lx,
                             int Lt, int bx, int bt, int Nv) {
  const int Lxc = Lx / bx, Vc = Lxc * (Lt / bt), nc = 2 * Nv;
  const int ex_w = bx + 2, E = (bx + 2) * (bt + 2);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Vc * nc * E) return;
  const int e = (int)(idx % E);
  const int s = (int)((idx / E) % nc);
  const int j = (int)(idx / ((long long)E * nc));
  const int c = s / Nv, k = s % Nv;
  const int lx = e % ex_w - 1, lt = e / ex_w - 1;          // local coords in [-1, b]
  const int jx = j % Lxc, jt = j / Lxc;
  const int V = Lx * Lt;
  auto gsite = [&](int ax, int at) {                         // local -> global (wrapped)
    int gx = jx * bx + ax, gt = jt * bt + at;
    gx = (gx % Lx + Lx) % Lx;
    gt = (gt % Lt + Lt) % Lt;
    return gx + Lx * gt;
  };
  auto inblock = [&](int ax, int at) { return ax >= 0 && ax < bx && at >= 0 && at < bt; };
  // P e_{j,s} at a local site: only spin c is non-zero (h = 1 on level 1).
  auto pval = [&](int ax, int at, double2& f0, double2& f1) {
    const double2 v = Vst[((long long)gsite(ax, at) * 2 + c) * Nv + k];
    f0 = c == 0 ? v : make_double2(0.0, 0.0);
    f1 = c == 1 ? v : make_double2(0.0, 0.0);
  };
  const int site = gsite(lx, lt);
  double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
  double2 f0, f1;
  if (inblock(lx + 1, lt)) { pval(lx + 1, lt, f0, f1); hop_x<double>(a0, a1, U[site], f0, f1, 1.0); }
  if (inblock(lx - 1, lt)) {
    pval(lx - 1, lt, f0, f1);
    hop_x<double>(a0, a1, cconj(U[gsite(lx - 1, lt)]), f0, f1, -1.0);
  }
  if (inblock(lx, lt + 1)) { pval(lx, lt + 1, f0, f1); hop_t<double>(a0, a1, U[V + site], f0, f1, 1.0); }
  if (inblock(lx, lt - 1)) {
    pval(lx, lt - 1, f0, f1);
    hop_t<double>(a0, a1, cconj(U[V + gsite(lx, lt - 1)]), f0, f1, -1.0);
  }
  double2 w0 = make_double2(-0.5 * a0.x, -0.5 * a0.y), w1 = make_double2(-0.5 * a1.x, -0.5 * a1.y);
  if (inblock(lx, lt)) {
    pval(lx, lt, f0, f1);
    w0.x += diag * f0.x; w0.y += diag * f0.y;
    w1.x += diag * f1.x; w1.y += diag * f1.y;
  }
  Wbuf[2 * idx] = w0;
  Wbuf[2 * idx + 1] = w1;
}

__global__ void k_galerkin_WW(const double2* __restrict__ Wbuf, double2* __restrict__ Ac, int Lx,
                              int Lt, int bx, int bt, int Nv) {
  const int Lxc = Lx / bx, Ltc = Lt / bt, Vc = Lxc * Ltc, nc = 2 * Nv;
  const int ex_w = bx + 2, E = (bx + 2) * (bt + 2);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Vc * 9 * nc * nc) return;
  const int sc = (int)(idx % nc);
  const int r = (int)((idx / nc) % nc);
  const int d = (int)((idx / (nc * nc)) % 9);
  const int j = (int)(idx / (9LL * nc * nc));
  const int dx = d % 3 - 1, dt = d / 3 - 1;
  const int jx = j % Lxc, jt = j / Lxc;
  const int j2 = ((jx + dx + Lxc) % Lxc) + Lxc * ((jt + dt + Ltc) % Ltc);
  const int x0 = max(-1, dx * bx - 1), x1 = min(bx, dx * bx + bx);
  const int t0 = max(-1, dt * bt - 1), t1 = min(bt, dt * bt + bt);
  const double2* Wa = Wbuf + ((long long)j * nc + r) * E * 2;
  const double2* Wb = Wbuf + ((long long)j2 * nc + sc) * E * 2;
  double2 acc = make_double2(0.0, 0.0);
  for (int lt = t0; lt <= t1; ++lt)
    for (int lx = x0; lx <= x1; ++lx) {
      const int e1 = (lt + 1) * ex_w + (lx + 1);
      const int e2 = (lt - dt * bt + 1) * ex_w + (lx - dx * bx + 1);
      cfmac(acc, Wa[2 * e1], Wb[2 * e2]);
      cfmac(acc, Wa[2 * e1 + 1], Wb[2 * e2 + 1]);
    }
  Ac[(((long long)j * 9 + d) * nc + r) * nc + sc] = acc;
}

cudaError_t galerkin_fine(const void* U64, double diag, const void* Vst, void* Wbuf, void* Ac,
                          int Lx, int Lt, int bx, int bt, int Nv, cudaStream_t s) {
  const long long Vc = (long long)(Lx / bx) * (Lt / bt), nc = 2 * Nv;
  const long long nW = Vc * nc * (bx + 2) * (bt + 2);
  k_galerkin_W<<<(unsigned)((nW + 255) / 256), 256, 0, s>>>(
      (const double2*)U64, diag, (const double2*)Vst, (double2*)Wbuf, Lx, Lt, bx, bt, Nv); count_launch();
  const long long nA = Vc * 9 * nc * nc;
  k_galerkin_WW<<<(unsigned)((nA + 255) / 256), 256, 0, s>>>((const double2*)Wbuf,
                                                              (double2*)Ac, Lx, Lt, bx, bt, Nv); count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Level >= 2 Galerkin, one CTA per coarse site j; the CTA accumulates the 9
// blocks of A_{l+1}[j] in shared memory.  For each fine site i of S_j and
// each fine displacement e: T = A_l[i][e] P(i+e) (nf x nc), then
// A_{l+1}[j][disp(i,e)] += P(i)^dagger T, disp = floor((o_i + e) / b).
// ---------------------------------------------------------------------------
__global__ void k_galerkin_coarse(const double2* __restrict__ Af, const double2* __restrict__ Vst,
                                  double2* __restrict__ Ac, int Lx, int Lt, int bx, int bt,
                                  int nf, int Nv) {
  extern __shared__ double2 sm[];
  const int nc = 2 * Nv, h = nf / 2, Lxc = Lx / bx;
  double2* acc = sm;                  // [9][nc][nc]
  double2* T = sm + 9 * nc * nc;      // [nf][nc]
  const int j = blockIdx.x;
  const int jx = j % Lxc, jt = j / Lxc;
  for (int q = threadIdx.x; q < 9 * nc * nc; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int o = 0; o < bx * bt; ++o) {
    const int ox = o % bx, ot = o / bx;
    const int x = jx * bx + ox, t = jt * bt + ot;
    const int i = x + Lx * t;
    for (int e = 0; e < 9; ++e) {
      const int ex = e % 3 - 1, et = e / 3 - 1;
      const int x2 = (x + ex + Lx) % Lx, t2 = (t + et + Lt) % Lt;
      const int i2 = x2 + Lx * t2;
      const int ddx = (ox + ex < 0) ? -1 : ((ox + ex >= bx) ? 1 : 0);
      const int ddt = (ot + et < 0) ? -1 : ((ot + et >= bt) ? 1 : 0);
      const int d = (ddx + 1) + 3 * (ddt + 1);
      const double2* Ablk = Af + ((long long)i * 9 + e) * nf * nf;
      // T[a][s] = sum_b A[a][c_s h + b] V_{k_s}(i2)[c_s h + b]
      for (int q = threadIdx.x; q < nf * nc; q += blockDim.x) {
        const int a = q / nc, s = q % nc, cs = s / Nv, ks = s % Nv;
        const double2* v = Vst + (((long long)i2 * 2 + cs) * Nv + ks) * h;
        const double2* arow = Ablk + (long long)a * nf + cs * h;
        double2 tv = make_double2(0.0, 0.0);
        for (int b = 0; b < h; ++b) cfma(tv, arow[b], v[b]);
        T[q] = tv;
      }
      __syncthreads();
      // acc[d][r][s] += sum_a conj(V_{k_r}(i)[c_r h + a]) T[c_r h + a][s]
      for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        const int r = q / nc, s = q % nc, cr = r / Nv, kr = r % Nv;
        const double2* v = Vst + (((long long)i * 2 + cr) * Nv + kr) * h;
        double2 g = acc[d * nc * nc + q];
        for (int a = 0; a < h; ++a) cfmac(g, v[a], T[(cr * h + a) * nc + s]);
        acc[d * nc * nc + q] = g;
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < 9 * nc * nc; q += blockDim.x)
    Ac[(long long)j * 9 * nc * nc + q] = acc[q];
}

cudaError_t galerkin_coarse(const void* Af, const void* Vst, void* Ac, int Lx, int Lt, int bx,
                            int bt, int nf, int Nv, cudaStream_t s) {
  const int nc = 2 * Nv, Vc = (Lx / bx) * (Lt / bt);
  const size_t smem = (size_t)(9 * nc * nc + nf * nc) * sizeof(double2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_galerkin_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set = true;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  k_galerkin_coarse<<<Vc, 256, smem, s>>>((const double2*)Af, (const double2*)Vst, (double2*)Ac,
                                          Lx, Lt, bx, bt, nf, Nv); count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coarsest level: dense matrix, FP32 Gauss-Jordan inverse, GEMV.
// ---------------------------------------------------------------------------
__global__ void k_coarse_to_dense(const double2* __restrict__ A, float2* __restrict__ M, int Lx,
                                  int Lt, int n, long long ld) {
  const int V = Lx * Lt;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)V * n * n) return;
  const int c = (int)(idx % n), r = (int)((idx / n) % n), j = (int)(idx / ((long long)n * n));
  const int x = j % Lx, t = j / Lx;
  for (int d = 0; d < 9; ++d) {       // aliased displacements land on the same entry: add
    const int xn = (x + d % 3 - 1 + Lx) % Lx, tn = (t + d / 3 - 1 + Lt) % Lt;
    const int jn = xn + Lx * tn;
    const double2 v = A[(((long long)j * 9 + d) * n + r) * n + c];
    float2* dst = M + ((long long)j * n + r) * ld + (long long)jn * n + c;
    dst->x += (float)v.x;
    dst->y += (float)v.y;
  }
}

__global__ void k_pad_identity(float2* __restrict__ M, long long N, long long ld) {
  const long long i = N + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) M[i * ld + i] = make_float2(1.f, 0.f);
}

cudaError_t coarse_to_dense_f32(const void* A, void* dense, int Lx, int Lt, int n, long long ld,
                                cudaStream_t s) {
  const long long N = (long long)Lx * Lt * n;
  if (ld < N) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(dense, 0, (size_t)(ld * ld * sizeof(float2)), s);
  if (e != cudaSuccess) return e;
  const long long tot = (long long)Lx * Lt * n * n;
  k_coarse_to_dense<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const double2*)A,
                                                                  (float2*)dense, Lx, Lt, n, ld); count_launch();
  if (ld > N) {
    k_pad_identity<<<(unsigned)((ld - N + 255) / 256), 256, 0, s>>>((float2*)dense, N, ld);
    count_launch();
  }
  return cudaGetLastError();
}

// Sweep (Gauss-Jordan) inversion.  Sweeping pivot block k of M with
// P = M_kk^{-1}:  M_ij -= M_ik P M_kj (i, j != k);  M_kj <- P M_kj;
// M_ik <- -M_ik P;  M_kk <- P.  After all pivots M holds its inverse.
//
// The matrix is Hermitian and, after sweeping the blocks K = {0..k-1}, so is
// its swept form up to sign: S_ij = S_ji^H when i, j are both swept or both
// unswept, S_ij = -S_ji^H otherwise.  Only the lower 64 x 64 tiles are kept
// current (diagonal tiles in full): the panels of column k and row k are
// rebuilt from them and the rank-64 update touches lower tiles only (half
// the flops).  Pivot blocks are the 64 x 64 diagonal tiles; every pivot block
// is Hermitian positive definite (a Schur complement of a positive definite
// matrix), so the sweep needs no pivoting.  Per pivot block two kernels: the
// panels, then the update, whose first CTA also inverts the next pivot block.
static constexpr int GJB = 64;
static constexpr int GJS = GJB + 1;              // shared row stride (float2)

// In-place inversion of the Hermitian positive definite 64 x 64 block
// a[][GJS] in shared memory by 256 threads: the same sweep, blocked in four
// 16 x 16 sub-pivots K.  Each sub-pivot is swept element by element (one
// entry per thread, 16 steps), then the rest of the block is updated with
// rank-16 products: a_ij -= a_iK P a_Kj, a_Kj <- P a_Kj, a_iK <- -a_iK P for
// i, j outside K.  tmp holds 2 x 16 x 48 complex (the row and column panels).
__device__ void sweep_block64(float2* a, float2* tmp) {
  const int tid = threadIdx.x;
  float2* TR = tmp;                                    // [16][48]  P a_Kj
  float2* TC = tmp + 16 * 48;                          // [48][16]  a_iK P
  for (int K = 0; K < 4; ++K) {
    const int k0 = 16 * K;
    {                                                  // sweep the 16 x 16 sub-pivot
      const int r = k0 + (tid >> 4), c = k0 + (tid & 15);
      for (int p = k0; p < k0 + 16; ++p) {
        const float2 piv = a[p * GJS + p];
        const float den = piv.x * piv.x + piv.y * piv.y;
        const float2 inv = make_float2(piv.x / den, -piv.y / den);
        const float2 arp = a[r * GJS + p], apc = a[p * GJS + c], arc = a[r * GJS + c];
        float2 v;
        if (r == p && c == p) v = inv;
        else if (r == p) v = cmul(inv, apc);
        else if (c == p) v = make_float2(-(arp.x * inv.x - arp.y * inv.y),
                                         -(arp.x * inv.y + arp.y * inv.x));
        else v = csub(arc, cmul(cmul(arp, inv), apc));
        __syncthreads();
        a[r * GJS + c] = v;
        __syncthreads();
      }
    }
    // panels: TR[q][x] = sum_s P[q][s] a[k0+s][col(x)], TC[x][q] = sum_s a[row(x)][k0+s] P[s][q]
    for (int o = tid; o < 2 * 16 * 48; o += 256) {
      const int e = o % (16 * 48);
      float2 acc = make_float2(0.f, 0.f);
      if (o < 16 * 48) {
        const int q = e / 48, x = e % 48, col = x < k0 ? x : x + 16;
        for (int s2 = 0; s2 < 16; ++s2)
          cfma(acc, a[(k0 + q) * GJS + k0 + s2], a[(k0 + s2) * GJS + col]);
        TR[e] = acc;
      } else {
        const int x = e / 16, q = e % 16, row = x < k0 ? x : x + 16;
        for (int s2 = 0; s2 < 16; ++s2)
          cfma(acc, a[row * GJS + k0 + s2], a[(k0 + s2) * GJS + k0 + q]);
        TC[e] = acc;
      }
    }
    __syncthreads();
    // rank-16 update of the 48 x 48 entries outside row and column block K
    float2 nv[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      const int e = tid + 256 * u, xi = e / 48, xj = e % 48;
      const int row = xi < k0 ? xi : xi + 16, col = xj < k0 ? xj : xj + 16;
      float2 acc = a[row * GJS + col];
      for (int s2 = 0; s2 < 16; ++s2) {
        const float2 c = a[row * GJS + k0 + s2], rv = TR[s2 * 48 + xj];
        acc.x -= c.x * rv.x - c.y * rv.y;
        acc.y -= c.x * rv.y + c.y * rv.x;
      }
      nv[u] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      const int e = tid + 256 * u, xi = e / 48, xj = e % 48;
      const int row = xi < k0 ? xi : xi + 16, col = xj < k0 ? xj : xj + 16;
      a[row * GJS + col] = nv[u];
    }
    for (int o = tid; o < 16 * 48; o += 256) {         // panel write-back
      const int q = o / 48, x = o % 48, col = x < k0 ? x : x + 16;
      a[(k0 + q) * GJS + col] = TR[o];
      const int x2 = o / 16, q2 = o % 16, row = x2 < k0 ? x2 : x2 + 16;
      const float2 w = TC[o];
      a[row * GJS + k0 + q2] = make_float2(-w.x, -w.y);
    }
    __syncthreads();
  }
}

// Inverts the first pivot block: P = M_00^{-1}.
__global__ void __launch_bounds__(256) k_gj_pivot0(const float2* __restrict__ M, int N,
                                                   float2* __restrict__ P) {
  extern __shared__ float2 gsm[];
  for (int q = threadIdx.x; q < GJB * GJB; q += 256)
    gsm[(q / GJB) * GJS + q % GJB] = M[(long long)(q / GJB) * N + q % GJB];
  __syncthreads();
  sweep_block64(gsm, gsm + GJB * GJS);
  for (int q = threadIdx.x; q < GJB * GJB; q += 256) P[q] = gsm[(q / GJB) * GJS + q % GJB];
}

// Panels of pivot block k for blocks b != k, each output block split over 4
// CTAs of 16 rows (blockIdx.y): Cold_b = M_bk and Cn_b = M_bk P (column
// panel, blockIdx.x < nb), R_b = P M_kb (row panel).  M_bk and M_kb come from
// the stored lower tiles by the sign rule.
__global__ void __launch_bounds__(256) k_gj_panel(const float2* __restrict__ M, int N, int k,
                                                  const float2* __restrict__ P,
                                                  float2* __restrict__ Cold,
                                                  float2* __restrict__ Cn,
                                                  float2* __restrict__ Rp) {
  extern __shared__ float2 gsm[];
  float2* sP = gsm;
  float2* sX = gsm + GJB * GJS;
  const int nb = N / GJB;
  const int b = blockIdx.x % nb, col_panel = blockIdx.x < nb, r0 = 16 * blockIdx.y;
  if (b == k) return;
  // stored tile read row by row; a transposed source is read along its rows
  // (r fastest) so that the global loads stay coalesced
  const bool transposed = col_panel ? (b < k) : (b > k);
#pragma unroll
  for (int q = threadIdx.x; q < GJB * GJB; q += 256) {
    sP[(q / GJB) * GJS + q % GJB] = P[q];
    const int r = transposed ? q % GJB : q / GJB, c = transposed ? q / GJB : q % GJB;
    float2 x;
    if (col_panel) {
      // M_bk: stored for b > k; for b < k it is -(M_kb)^H (swept row, unswept column)
      if (!transposed) {
        x = M[(long long)(b * GJB + r) * N + k * GJB + c];
      } else {
        const float2 v = M[(long long)(k * GJB + c) * N + b * GJB + r];
        x = make_float2(-v.x, v.y);
      }
    } else {
      // M_kb: stored for b < k; for b > k it is (M_bk)^H (both unswept)
      if (!transposed) {
        x = M[(long long)(k * GJB + r) * N + b * GJB + c];
      } else {
        const float2 v = M[(long long)(b * GJB + c) * N + k * GJB + r];
        x = make_float2(v.x, -v.y);
      }
    }
    sX[r * GJS + c] = x;
  }
  __syncthreads();
  const int r = r0 + (threadIdx.x >> 4), c0 = threadIdx.x & 15;
  float2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
  if (col_panel) {
    for (int q = 0; q < GJB; ++q) {
      const float2 xv = sX[r * GJS + q];
#pragma unroll
      for (int u = 0; u < 4; ++u) cfma(acc[u], xv, sP[q * GJS + c0 + 16 * u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + 16 * u;
      Cold[(long long)(b * GJB + r) * GJB + c] = sX[r * GJS + c];
      Cn[(long long)(b * GJB + r) * GJB + c] = acc[u];
    }
  } else {
    for (int q = 0; q < GJB; ++q) {
      const float2 pv = sP[r * GJS + q];
#pragma unroll
      for (int u = 0; u < 4; ++u) cfma(acc[u], pv, sX[q * GJS + c0 + 16 * u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Rp[(long long)r * N + b * GJB + c0 + 16 * u] = acc[u];
  }
}

// Lower tiles (I, J) for pivot block k: M_IJ -= Cold_I R_J for I, J != k, and
// the sweep's write-back: M_kJ = R_J (J < k), M_Ik = -Cn_I (I > k), M_kk = P.
// CTA 0 takes tile (k+1, k+1) and, after updating it, inverts it into Pnext
// (the next pivot block), overlapping that sweep with the other tiles.
//
// The complex product runs on the tensor cores as a real GEMM: with complex
// entries interleaved (re, im), Out (64 x 128) = C (64 x 128) B (128 x 128),
// where B realifies R: B[2k][2j] = Re R_kj, B[2k][2j+1] = Im R_kj,
// B[2k+1][2j] = -Im R_kj, B[2k+1][2j+1] = Re R_kj.  mma.sync m16n8k8 TF32 with
// each operand split x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and three
// products hi hi + hi lo + lo hi, FP32 accumulation: about FP32 accuracy.
// 8 warps in a 2 x 4 grid, 32 x 32 real outputs each; lane (g, t) = (lane/4,
// lane%4) holds complex outputs (row g or g + 8, column t) of each 16 x 4
// complex sub-tile, so the epilogue works on whole complex numbers.
static constexpr int GJC = 66;                   // sC row stride (float2), conflict-free A loads
static constexpr int GJR = 68;                   // sR row stride (float2), conflict-free B loads

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_gj_update(float2* __restrict__ M, int N, int k,
                                                   const float2* __restrict__ P,
                                                   float2* __restrict__ Pnext,
                                                   const float2* __restrict__ Cold,
                                                   const float2* __restrict__ Cn,
                                                   const float2* __restrict__ Rp) {
  extern __shared__ float2 gsm[];
  const int nt = N / GJB;
  // tile index: CTA 0 -> (k+1, k+1) if it exists; the rest in order, skipping it
  const long long kp = (k + 1 < nt) ? (long long)(k + 1) * (k + 2) / 2 + (k + 1) : -1;
  long long t = blockIdx.x;
  if (kp >= 0) t = (t == 0) ? kp : (t <= kp ? t - 1 : t);
  int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
  while ((long long)I * (I + 1) / 2 > t) --I;
  const int J = (int)(t - (long long)I * (I + 1) / 2);
  const int tid = threadIdx.x;
  float2* tile = M + (long long)I * GJB * N + J * GJB;
  if (I == k || J == k) {                              // pivot row / column / block
    for (int q = tid; q < GJB * GJB; q += 256) {
      const int r = q / GJB, c = q % GJB;
      float2 v;
      if (I == k && J == k) {
        v = P[q];
      } else if (I == k) {
        v = Rp[(long long)r * N + J * GJB + c];
      } else {
        const float2 w = Cn[(long long)(I * GJB + r) * GJB + c];
        v = make_float2(-w.x, -w.y);
      }
      tile[(long long)r * N + c] = v;
    }
    return;
  }
  float2* sC = gsm;                                    // Cold_I [64][GJC]
  float2* sR = gsm + GJB * GJC;                        // R_J    [64][GJR]
  {                                                    // two complex per 16-byte load,
    float4 vc[8], vr[8];                               // all 16 loads in flight first
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = tid + 256 * u, r = q / (GJB / 2), c = 2 * (q % (GJB / 2));
      vc[u] = *(const float4*)&Cold[(long long)(I * GJB + r) * GJB + c];
      vr[u] = *(const float4*)&Rp[(long long)r * N + J * GJB + c];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = tid + 256 * u, r = q / (GJB / 2), c = 2 * (q % (GJB / 2));
      *(float4*)&sC[r * GJC + c] = vc[u];
      *(float4*)&sR[r * GJR + c] = vr[u];
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;             // rows 32 wm.., complex cols 16 wn..
  const float* sCf = (const float*)sC;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][n][e] = 0.f;
#pragma unroll 2
  for (int kk = 0; kk < 2 * GJB / 8; ++kk) {           // 16 real k-steps of 8
    uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int row = 32 * wm + 16 * mt + g;
      const float* r0 = sCf + row * 2 * GJC + 8 * kk;
      const float* r8 = r0 + 8 * 2 * GJC;
      split_tf32(r0[tq], ah[mt][0], al[mt][0]);
      split_tf32(r8[tq], ah[mt][1], al[mt][1]);
      split_tf32(r0[tq + 4], ah[mt][2], al[mt][2]);
      split_tf32(r8[tq + 4], ah[mt][3], al[mt][3]);
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      // B[8kk + tq][8n' + g] and B[8kk + tq + 4][8n' + g], n' = 4 wn + n
      const int j = 16 * wn + 4 * n + (g >> 1), d = g & 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kr = 8 * kk + tq + 4 * h;            // real row of B
        const float2 v = sR[(kr >> 1) * GJR + j];
        const float x = (kr & 1) ? (d ? v.x : -v.y) : (d ? v.y : v.x);
        split_tf32(x, bh[n][h], bl[n][h]);
      }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        mma_tf32(acc[mt][n], al[mt], bh[n]);
        mma_tf32(acc[mt][n], ah[mt], bl[n]);
        mma_tf32(acc[mt][n], ah[mt], bh[n]);
      }
  }
  const bool next_pivot = (long long)t == kp;
  if (next_pivot) __syncthreads();                     // sC is reused for the new tile
  float2 old[2][4][2];                                 // all tile loads before the stores
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        old[mt][n][h] = tile[(long long)(32 * wm + 16 * mt + g + 8 * h) * N + 16 * wn + 4 * n + tq];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 32 * wm + 16 * mt + g + 8 * h, c = 16 * wn + 4 * n + tq;
        const float2 o = old[mt][n][h];
        const float2 nv = make_float2(o.x - acc[mt][n][2 * h], o.y - acc[mt][n][2 * h + 1]);
        tile[(long long)r * N + c] = nv;
        if (next_pivot) sC[r * GJS + c] = nv;
      }
  if (next_pivot) {
    __syncthreads();
    sweep_block64(sC, sR);
    for (int q = tid; q < GJB * GJB; q += 256) Pnext[q] = sC[(q / GJB) * GJS + q % GJB];
  }
}

// ---- tcgen05 variant of the update ---------------------------------------
// The same update, M_IJ -= Cold_I R_J, on the 5th-generation tensor cores:
// one CTA per "tall tile" of two 64-row blocks (2p, 2p+1) and one 64-column
// block J, an M = 128, N = 128 (realified), K = 8 tcgen05.mma of kind::tf32
// per step with the FP32 accumulator in tensor memory (row r of the tile in
// TMEM lane r).  The 64 complex pivot columns (K = 128 real) are staged in four
// quarters of 16; each stage writes A = Cold rows (complex entries interleaved
// (re, im) along K) and B = R_J realified (B[n][k], n = 2j + d, k = 2q + c:
// Re R for c = d, Im R for (c, d) = (0, 1), -Im R for (c, d) = (1, 0)) into
// shared memory in the K-major no-swizzle core-matrix layout (8 rows x 16 B
// per core matrix), as TF32 hi/lo splits; three MMAs per step (lo hi, hi lo,
// hi hi).  One elected thread issues the MMAs and commits them to an
// mbarrier; every thread waits on it (bounded: a wait that runs out sets
// *err and the CTA gives up) before reusing shared memory or reading the
// accumulator with tcgen05.ld.  Warps w and w + 4 read TMEM lanes 32 (w % 4)
// .. + 31, columns split in halves.
static constexpr int TC_K = 32;                  // real K per stage (16 complex pivot columns)
static constexpr int TC_OPF = 128 * TC_K;        // floats per operand split (16 KB)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// float offset of element (row, k) of a [128][TC_K] operand, core matrices
// (row / 8, k / 4) of 32 floats, K fastest
__device__ __forceinline__ int tc_off(int row, int k) {
  return ((row >> 3) * (TC_K / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor: start address and offsets in 16-byte
// units; leading-dimension offset = next core matrix along K (128 B), stride
// offset = next 8-row group (TC_K / 4 core matrices), version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((TC_K / 4 * 128u) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 128, M = 128
constexpr uint32_t TC_IDESC =
    (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(dtmem), "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(m);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
    __nanosleep(64);
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// number of tall tiles of row pair p: column blocks 0 .. min(2p + 1, nt - 1)
__device__ __forceinline__ int tc_tiles_of_pair(int p, int nt) { return min(2 * p + 2, nt); }

__global__ void __launch_bounds__(256, 2) k_gj_update_tc(float2* __restrict__ M, int N, int k,
                                                         const float2* __restrict__ P,
                                                         float2* __restrict__ Pnext,
                                                         const float2* __restrict__ Cold,
                                                         const float2* __restrict__ Cn,
                                                         const float2* __restrict__ Rp,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char tc_dyn[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  const int nt = N / GJB, npairs = (nt + 1) / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tall tile of this CTA; CTA 0 takes the one holding block (k+1, k+1)
  long long target = -1;
  if (k + 1 < nt) {
    long long cum = 0;
    for (int q = 0; q < (k + 1) / 2; ++q) cum += tc_tiles_of_pair(q, nt);
    target = cum + (k + 1);
  }
  long long t = blockIdx.x;
  if (target >= 0) t = (t == 0) ? target : (t <= target ? t - 1 : t);
  int p = 0;
  for (; p < npairs; ++p) {
    const int c = tc_tiles_of_pair(p, nt);
    if (t < c) break;
    t -= c;
  }
  const int J = (int)t;
  // role of each 64-row half: 0 skip, 1 update, 2 copy R_J (pivot row),
  // 3 copy P (pivot block), 4 copy -Cn_I (pivot column)
  int role[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int I = 2 * p + h;
    if (I >= nt || J > I) role[h] = 0;
    else if (I == k && J == k) role[h] = 3;
    else if (I == k) role[h] = 2;
    else if (J == k) role[h] = 4;
    else role[h] = 1;
  }
  // copies (no MMA involved)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (role[h] < 2) continue;
    const int I = 2 * p + h;
    float2* tile = M + (long long)I * GJB * N + J * GJB;
    for (int q = tid; q < GJB * GJB; q += 256) {
      const int r = q / GJB, c = q % GJB;
      float2 v;
      if (role[h] == 3) v = P[q];
      else if (role[h] == 2) v = Rp[(long long)r * N + J * GJB + c];
      else {
        const float2 w = Cn[(long long)(I * GJB + r) * GJB + c];
        v = make_float2(-w.x, -w.y);
      }
      tile[(long long)r * N + c] = v;
    }
  }
  if (role[0] != 1 && role[1] != 1) return;             // CTA-uniform
  // operands from a 1024-byte aligned base (the allocation has 1 KB of slack)
  unsigned char* tc_raw = tc_dyn + ((1024u - (smem_u32(tc_dyn) & 1023u)) & 1023u);
  float* Ahi = (float*)tc_raw;
  float* Alo = Ahi + TC_OPF;
  float* Bhi = Alo + TC_OPF;
  float* Blo = Bhi + TC_OPF;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n"
                 :: "r"(smem_u32(&tmem_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_sh;
  bool ok = true;
  constexpr int KC = TC_K / 2;                           // complex pivot columns per stage
  constexpr int PER = 128 * KC / 256;                    // operand slots per thread and stage
  // A: 128 rows x KC complex pivot columns of Cold (rows of a missing second
  // block, when nt is odd, are zero).  Thread e writes float2 slot e % 16 of
  // core matrix e / 16 (consecutive threads, consecutive slots: no bank
  // conflicts); slot w holds row w / 2, complex column w % 2 of it.
  // B: R_J realified, rows q of the pivot block; slot w of core matrix cm
  // (8 n x 4 k) holds n = 2 j + d with j = 4 (cm / 8) + w / 4, d = (w / 2) % 2,
  // k = 2 q .. 2 q + 1 with q = 2 (cm % 8) + w % 2: (Re, -Im) for d = 0,
  // (Im, Re) for d = 1.  The next stage's entries are loaded into registers
  // while the tensor cores work on the current one.
  float2 va[PER], vb[PER];
  auto load_stage = [&](int kh) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + 256 * i, cm = e >> 4, w = e & 15;
      const int row = 8 * (cm / (TC_K / 4)) + (w >> 1), c = 2 * (cm % (TC_K / 4)) + (w & 1);
      const int I = 2 * p + (row >> 6);
      va[i] = I < nt ? Cold[((long long)I * GJB + (row & 63)) * GJB + KC * kh + c]
                     : make_float2(0.f, 0.f);
      const int j = 4 * (cm / (TC_K / 4)) + (w >> 2);
      const int ql = 2 * (cm % (TC_K / 4)) + (w & 1);
      vb[i] = Rp[(long long)(KC * kh + ql) * N + J * GJB + j];
    }
  };
  auto store_stage = [&]() {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + 256 * i, w = e & 15;
      const int o = (e >> 4) * 32 + 2 * w;                 // == tc_off of the slot
      uint32_t h0, l0, h1, l1;
      split_tf32(va[i].x, h0, l0);
      split_tf32(va[i].y, h1, l1);
      *(float2*)(Ahi + o) = make_float2(__uint_as_float(h0), __uint_as_float(h1));
      *(float2*)(Alo + o) = make_float2(__uint_as_float(l0), __uint_as_float(l1));
      const int d = (w >> 1) & 1;
      const float b0 = d ? vb[i].y : vb[i].x, b1 = d ? vb[i].x : -vb[i].y;
      split_tf32(b0, h0, l0);
      split_tf32(b1, h1, l1);
      *(float2*)(Bhi + o) = make_float2(__uint_as_float(h0), __uint_as_float(h1));
      *(float2*)(Blo + o) = make_float2(__uint_as_float(l0), __uint_as_float(l1));
    }
  };
  load_stage(0);
  for (int kh = 0; kh < GJB / KC && ok; ++kh) {
    store_stage();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll 1
      for (int kk = 0; kk < TC_K / 8; ++kk) {
        const uint32_t off = kk * 2 * 128;          // two core matrices along K per step
        tc_mma(tmem, tc_desc(al + off), tc_desc(bh + off), (kh | kk) ? 1u : 0u);
        tc_mma(tmem, tc_desc(ah + off), tc_desc(bl + off), 1u);
        tc_mma(tmem, tc_desc(ah + off), tc_desc(bh + off), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                   :: "r"(smem_u32(&mbar)) : "memory");
    }
    if (kh + 1 < GJB / KC) load_stage(kh + 1);          // overlaps the MMAs of stage kh
    ok = mbar_wait(&mbar, (uint32_t)(kh & 1), err);
    ok = __syncthreads_and(ok);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // epilogue: row r = 32 (warp % 4) + lane of the tall tile, columns split by warp / 4
  const int quarter = warp & 3, chalf = warp >> 2;
  const int r = 32 * quarter + lane, h = r >> 6, rr = r & 63, I = 2 * p + h;
  const bool next_pivot = (I == k + 1 && J == k + 1);
  float2* sw = (float2*)tc_raw;            // the new pivot block [64][GJS] + sweep scratch
  if (ok) {
    float v[32];
#pragma unroll 1
    for (int c2 = 0; c2 < 2; ++c2) {
      const int col0 = 64 * chalf + 32 * c2;             // real column of the chunk
      tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)col0, v);
      if (role[h] == 1) {
        float2* rowp = M + ((long long)I * GJB + rr) * N + J * GJB + col0 / 2;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float2 o = rowp[i];
          const float2 nv = make_float2(o.x - v[2 * i], o.y - v[2 * i + 1]);
          rowp[i] = nv;
          if (next_pivot) sw[rr * GJS + col0 / 2 + i] = nv;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" :: "r"(tmem));
  if (ok && (role[0] == 1 && 2 * p == k + 1 && J == k + 1 || role[1] == 1 && 2 * p + 1 == k + 1 && J == k + 1)) {
    sweep_block64(sw, sw + GJB * GJS);
    for (int q = tid; q < GJB * GJB; q += 256) Pnext[q] = sw[(q / GJB) * GJS + q % GJB];
  }
}

// Work layout: P[2][64 x 64] (pivot inverse, double-buffered by pivot parity),
// Cold [N][64], Cn [N][64], Rp [64][N].
static void gj_work_split(void* work, int N, float2** Pb, float2** Cold, float2** Cn, float2** Rp) {
  Pb[0] = (float2*)work;
  Pb[1] = Pb[0] + GJB * GJB;
  *Cold = Pb[1] + GJB * GJB;
  *Cn = *Cold + (long long)N * GJB;
  *Rp = *Cn + (long long)N * GJB;
}

cudaError_t gauss_jordan_begin(void* M, int N, void* work, cudaStream_t s) {
  if (N % GJB != 0) return cudaErrorInvalidValue;
  float2 *Pb[2], *Cold, *Cn, *Rp;
  gj_work_split(work, N, Pb, &Cold, &Cn, &Rp);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * GJB * GJS * sizeof(float2)));
    cudaFuncSetAttribute(k_gj_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(GJB * (GJC + GJR) * sizeof(float2)));
    attr = true;
  }
  k_gj_pivot0<<<1, 256, (GJB * GJS + 2 * 16 * 48) * sizeof(float2), s>>>((const float2*)M, N, Pb[0]);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gauss_jordan_panel(void* M, int N, int k, void* work, cudaStream_t s) {
  float2 *Pb[2], *Cold, *Cn, *Rp;
  gj_work_split(work, N, Pb, &Cold, &Cn, &Rp);
  const int nb = N / GJB;
  k_gj_panel<<<dim3(2 * nb, GJB / 16), 256, 2 * GJB * GJS * sizeof(float2), s>>>(
      (const float2*)M, N, k, Pb[k & 1], Cold, Cn, Rp);
  count_launch();
  return cudaGetLastError();
}

// Tall tiles of a pivot step: sum over row pairs p of min(2p + 2, nt).
static int tc_tile_count(int nt) {
  int c = 0;
  for (int p = 0; p < (nt + 1) / 2; ++p) c += std::min(2 * p + 2, nt);
  return c;
}

cudaError_t gauss_jordan_update_tc(void* M, int N, int k, void* work, cudaStream_t s) {
  float2 *Pb[2], *Cold, *Cn, *Rp;
  gj_work_split(work, N, Pb, &Cold, &Cn, &Rp);
  const int nb = N / GJB;
  const size_t sm = 4 * TC_OPF * sizeof(float) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gj_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  k_gj_update_tc<<<tc_tile_count(nb), 256, sm, s>>>((float2*)M, N, k, Pb[k & 1], Pb[(k + 1) & 1],
                                                    Cold, Cn, Rp, (int*)(Rp + (long long)GJB * N));
  count_launch();
  return cudaGetLastError();
}

cudaError_t gauss_jordan_update(void* M, int N, int k, void* work, cudaStream_t s) {
  float2 *Pb[2], *Cold, *Cn, *Rp;
  gj_work_split(work, N, Pb, &Cold, &Cn, &Rp);
  const int nb = N / GJB;
  k_gj_update<<<nb * (nb + 1) / 2, 256, GJB * (GJC + GJR) * sizeof(float2), s>>>(
      (float2*)M, N, k, Pb[k & 1], Pb[(k + 1) & 1], Cold, Cn, Rp);
  count_launch();
  return cudaGetLastError();
}

// y = B x: one warp per row, FP32 products and accumulation, result widened.
// B has leading dimension ld (even, >= N); xtmp holds ld complex64, zero beyond N.
__global__ void k_x_to_f32(const double2* __restrict__ x, float2* __restrict__ xf, int N, int ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) xf[i] = i < N ? make_float2((float)x[i].x, (float)x[i].y) : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_gemv(const float2* __restrict__ B,
                                              const float2* __restrict__ xf,
                                              double2* __restrict__ y, int N, int ld,
                                              bool accumulate) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N) return;
  const float4* b4 = (const float4*)(B + (long long)row * ld);
  const float4* x4 = (const float4*)xf;
  float2 acc = make_float2(0.f, 0.f);
  for (int q = lane; q < ld / 2; q += 32) {
    const float4 bv = b4[q], xv = x4[q];
    cfma(acc, make_float2(bv.x, bv.y), make_float2(xv.x, xv.y));
    cfma(acc, make_float2(bv.z, bv.w), make_float2(xv.z, xv.w));
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    double2 v = make_double2(acc.x, acc.y);
    if (accumulate) { v.x += y[row].x; v.y += y[row].y; }
    y[row] = v;
  }
}

cudaError_t dense_gemv_f32(const void* B, const void* x, void* y, int N, int ld, void* xtmp,
                           bool accumulate, cudaStream_t s) {
  if (ld % 2 || ld < N) return cudaErrorInvalidValue;
  k_x_to_f32<<<(ld + 255) / 256, 256, 0, s>>>((const double2*)x, (float2*)xtmp, N, ld); count_launch();
  k_gemv<<<(N + 7) / 8, 256, 0, s>>>((const float2*)B, (const float2*)xtmp, (double2*)y, N, ld,
                                     accumulate); count_launch();
  return cudaGetLastError();
}

// Hermitian inverse in packed lower-triangular 64 x 64 tiles.  Tile (I, J),
// I >= J, is stored at k = I (I + 1) / 2 + J, row-major.  y = B x reads every
// stored tile once: tile (I, J) contributes B_IJ x_J to rows of block I and,
// off the diagonal, B_IJ^H x_I to rows of block J; partial products go to a
// buffer and a second kernel sums them per row in a fixed order.
static constexpr int HT = 64;


__global__ void k_pack_hermitian(const float2* __restrict__ M, float2* __restrict__ P, int ld) {
  const int k = blockIdx.x;
  int I = (int)((sqrtf(8.f * k + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= k) ++I;
  while (I * (I + 1) / 2 > k) --I;
  const int J = k - I * (I + 1) / 2;
  for (int q = threadIdx.x; q < HT * HT; q += blockDim.x) {
    const int r = q / HT, c = q % HT;
    float2 v;
    if (I != J || r >= c) {
      v = M[(long long)(I * HT + r) * ld + J * HT + c];
    } else {     // upper half of a diagonal tile: Hermitian image of the lower half
      const float2 w = M[(long long)(J * HT + c) * ld + I * HT + r];
      v = make_float2(w.x, -w.y);
    }
    P[(long long)k * HT * HT + q] = v;
  }
}

cudaError_t pack_hermitian(const void* M, void* P, int ld, cudaStream_t s) {
  if (ld % HT) return cudaErrorInvalidValue;
  const int nt = ld / HT;
  k_pack_hermitian<<<nt * (nt + 1) / 2, 256, 0, s>>>((const float2*)M, (float2*)P, ld);
  count_launch();
  return cudaGetLastError();
}

// One work item of k_hgemv_mma: rows 16 mt0 .. 16 (mt0 + MT) - 1 of the tile
// product (pass 0: T X_J, pass 1: T^H X_I) for right-hand sides 16 ng .. 16 ng + 15.
template <int MT>
__device__ __forceinline__ void hgemv_mma_item(const float2* sT, const float2* sXJ,
                                               const float2* sXI, int pass, int mt0, int ng,
                                               int k, int ntiles, int nrhs,
                                               float2* __restrict__ part) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  const float2* sX = pass ? sXI : sXJ;
  const float* sTf = (const float*)sT;
  float acc[MT][4][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][n][e] = 0.f;
#pragma unroll 2
  for (int kk = 0; kk < 2 * HT / 8; ++kk) {
    uint32_t ah[MT][4], al[MT][4], bh[4][2], bl[4][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int m = 16 * (mt0 + mt) + g;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int mm = m + 8 * (f & 1), kr = 8 * kk + tq + 4 * (f >> 1);
        float a;
        if (pass == 0) {
          a = sTf[mm * 2 * GJC + kr];                      // T[m][kr/2], (re, im) along K
        } else {
          const float2 t = sT[(kr >> 1) * GJC + mm];       // conj(T[kr/2][m])
          a = (kr & 1) ? -t.y : t.x;
        }
        split_tf32(a, ah[mt][f], al[mt][f]);
      }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int j = 16 * ng + 4 * n + (g >> 1), d = g & 1;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int kr = 8 * kk + tq + 4 * hh;
        const float2 v = sX[(kr >> 1) * GJR + j];
        const float x = (kr & 1) ? (d ? v.x : -v.y) : (d ? v.y : v.x);
        split_tf32(x, bh[n][hh], bl[n][hh]);
      }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        mma_tf32(acc[mt][n], al[mt], bh[n]);
        mma_tf32(acc[mt][n], ah[mt], bl[n]);
        mma_tf32(acc[mt][n], ah[mt], bh[n]);
      }
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int m = 16 * (mt0 + mt) + g + 8 * hh, r = 16 * ng + 4 * n + tq;
        if (r < nrhs)
          part[(long long)r * ntiles * 2 * HT + (2LL * k + pass) * HT + m] =
              make_float2(acc[mt][n][2 * hh], acc[mt][n][2 * hh + 1]);
      }
}

// Tensor-core variant for 16..64 right-hand sides: per stored tile T (64 x 64
// complex) the row products T X_J and, off the diagonal, the column products
// T^H X_I, as realified GEMMs on mma.sync m16n8k8 TF32 with three products per
// FP32-accurate product (the layout and fragment mapping of k_gj_update: A =
// T rows, or T^H built from T's columns with the imaginary part negated; B =
// X realified, rows k of the tile, columns = right-hand sides).  X comes as an
// FP32 copy xs [nrhs][ld] (zero beyond N); right-hand sides are padded to a
// multiple of 16 with zeros (warps whose 16 columns are all padding skip the
// products).  Partial sums go to the buffer layout of k_hgemv_tiles.
__global__ void __launch_bounds__(256) k_hgemv_mma(const float2* __restrict__ P,
                                                   const float2* __restrict__ xs, int ld,
                                                   int ntiles, int nrhs,
                                                   float2* __restrict__ part) {
  extern __shared__ float2 hsm[];
  float2* sT = hsm;                                      // [64][GJC]
  float2* sXJ = sT + HT * GJC;                           // [64 k][GJR]: X_J[k][rhs]
  float2* sXI = sXJ + HT * GJR;
  const int k = blockIdx.x, tid = threadIdx.x;
  int I = (int)((sqrtf(8.f * k + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= k) ++I;
  while (I * (I + 1) / 2 > k) --I;
  const int J = k - I * (I + 1) / 2;
  {
    const float4* src = (const float4*)(P + (long long)k * HT * HT);
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = src[tid + 256 * u];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = 2 * (tid + 256 * u), r = e / HT, c = e % HT;
      *(float4*)&sT[r * GJC + c] = v[u];
    }
  }
  for (int e = tid; e < HT * HT; e += 256) {             // rhs r = e / 64, row kk = e % 64
    const int r = e / HT, kk = e % HT;
    float2 xj = make_float2(0.f, 0.f), xi = make_float2(0.f, 0.f);
    if (r < nrhs) {
      xj = xs[(long long)r * ld + J * HT + kk];
      xi = xs[(long long)r * ld + I * HT + kk];
    }
    sXJ[kk * GJR + r] = xj;
    sXI[kk * GJR + r] = xi;
  }
  __syncthreads();
  // Work items (product, MT 16-row tiles, 16 right-hand sides) are spread
  // over the 8 warps: one row tile per item up to 32 right-hand sides (so
  // that 16 right-hand sides still occupy every warp), two beyond (the A
  // fragments are then shared by two row tiles).
  const int warp = tid >> 5;
  const int NG = (nrhs + 15) / 16, npass = I == J ? 1 : 2;
  if (NG <= 2) {
    for (int item = warp; item < npass * 4 * NG; item += 8)
      hgemv_mma_item<1>(sT, sXJ, sXI, item / (4 * NG), (item / NG) % 4, item % NG, k, ntiles, nrhs,
                        part);
  } else {
    for (int item = warp; item < npass * 2 * NG; item += 8)
      hgemv_mma_item<2>(sT, sXJ, sXI, item / (2 * NG), 2 * ((item / NG) % 2), item % NG, k, ntiles,
                        nrhs, part);
  }
}

__global__ void k_x32_pad(const double2* __restrict__ x, float2* __restrict__ xs, int N, int ld,
                          int nrhs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)ld * nrhs) return;
  const int r = (int)(i / ld), c = (int)(i % ld);
  const double2 v = c < N ? x[(long long)r * N + c] : make_double2(0.0, 0.0);
  xs[i] = make_float2((float)v.x, (float)v.y);
}

__global__ void __launch_bounds__(256) k_hgemv_tiles(const float2* __restrict__ P,
                                                     const double2* __restrict__ x, int N,
                                                     int nrhs, float2* __restrict__ part) {
  __shared__ float2 T[HT][HT + 1];
  __shared__ float2 xi[HT], xj[HT];
  __shared__ float2 red[4][HT];
  const int k = blockIdx.x;
  const long long ntiles = gridDim.x;
  int I = (int)((sqrtf(8.f * k + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= k) ++I;
  while (I * (I + 1) / 2 > k) --I;
  const int J = k - I * (I + 1) / 2;
  const float4* src = (const float4*)(P + (long long)k * HT * HT);
  float4 buf[HT * HT / 2 / 256];                 // all 8 loads in flight before the stores
#pragma unroll
  for (int u = 0; u < HT * HT / 2 / 256; ++u) buf[u] = src[threadIdx.x + 256 * u];
#pragma unroll
  for (int u = 0; u < HT * HT / 2 / 256; ++u) {
    const int e = 2 * (threadIdx.x + 256 * u), r = e / HT, c = e % HT;
    T[r][c] = make_float2(buf[u].x, buf[u].y);
    T[r][c + 1] = make_float2(buf[u].z, buf[u].w);
  }
  const int r = threadIdx.x % HT, g = threadIdx.x / HT;
  for (int rhs = 0; rhs < nrhs; ++rhs) {
    const double2* xr = x + (long long)rhs * N;
    float2* pr = part + (long long)rhs * ntiles * 2 * HT;
    __syncthreads();                             // T loaded / previous rhs done with xi, xj, red
    if (threadIdx.x < HT) {
      const int gi = I * HT + threadIdx.x, gj = J * HT + threadIdx.x;
      xi[threadIdx.x] = gi < N ? make_float2((float)xr[gi].x, (float)xr[gi].y) : make_float2(0.f, 0.f);
      xj[threadIdx.x] = gj < N ? make_float2((float)xr[gj].x, (float)xr[gj].y) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // u = T x_J: row r = t % 64, quarter g = t / 64 of the columns
    float2 u = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int c = g * 16; c < g * 16 + 16; ++c) cfma(u, T[r][c], xj[c]);
    red[g][r] = u;
    __syncthreads();
    if (threadIdx.x < HT) {
      float2 a = red[0][threadIdx.x];
      a = cadd(a, red[1][threadIdx.x]);
      a = cadd(a, red[2][threadIdx.x]);
      a = cadd(a, red[3][threadIdx.x]);
      pr[(2LL * k) * HT + threadIdx.x] = a;
    }
    if (I == J) continue;
    __syncthreads();
    // v = T^H x_I: column c = t % 64, quarter g of the rows
    float2 v = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int rr = g * 16; rr < g * 16 + 16; ++rr) cfmac(v, T[rr][r], xi[rr]);
    red[g][r] = v;
    __syncthreads();
    if (threadIdx.x < HT) {
      float2 a = red[0][threadIdx.x];
      a = cadd(a, red[1][threadIdx.x]);
      a = cadd(a, red[2][threadIdx.x]);
      a = cadd(a, red[3][threadIdx.x]);
      pr[(2LL * k + 1) * HT + threadIdx.x] = a;
    }
  }
}

// Variant for up to four right-hand sides: two warps per stored tile, each
// streaming two chunks of 16 rows straight from global memory, lane l holding
// columns 2l and 2l + 1 of every row (one 16-byte load per row).  The row
// products B_IJ x_J are summed across the warp by a transposing butterfly
// (after it, lanes 2r and 2r + 1 hold row r of the chunk); the column
// products B_IJ^H x_I stay in registers and the two warps' sums are added
// through shared memory.  The partial sums use the buffer layout of
// k_hgemv_tiles.
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ float2 ld_x32(const double2* p) {
  const double2 v = *p;
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float2 ld_x32(const float2* p) { return *p; }

template <int NR, typename XT = double2>
__global__ void __launch_bounds__(64) k_hgemv_warp(const float2* __restrict__ P,
                                                   const XT* __restrict__ x, int N,
                                                   int ntiles, int nrhs,
                                                   float2* __restrict__ part,
                                                   double2* __restrict__ x64) {
  __shared__ float4 colsum[NR][32];                      // column partials of warp 1
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x;                              // one tile, rows split by warp
  int I = (int)((sqrtf(8.f * k + 1.f) - 1.f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= k) ++I;
  while (I * (I + 1) / 2 > k) --I;
  const int J = k - I * (I + 1) / 2;
  const float4* src = (const float4*)(P + (long long)k * HT * HT) + lane;
  for (int q0 = 0; q0 < nrhs; q0 += NR) {
    float2 xj0[NR], xj1[NR], xi0[NR], xi1[NR], ac0[NR], ac1[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      xj0[q] = xj1[q] = xi0[q] = xi1[q] = ac0[q] = ac1[q] = make_float2(0.f, 0.f);
      if (q0 + q < nrhs) {
        const XT* xr = x + (long long)(q0 + q) * N;
        const int cj = J * HT + 2 * lane, ri = I * HT + lane;
        if (cj < N) xj0[q] = ld_x32(xr + cj);
        if (cj + 1 < N) xj1[q] = ld_x32(xr + cj + 1);
        if (ri < N) xi0[q] = ld_x32(xr + ri);
        if (ri + 32 < N) xi1[q] = ld_x32(xr + ri + 32);
        if (x64 && I == J && w == 0) {         // the FP64 copy of x, once per row block
          double2* xo = x64 + (long long)(q0 + q) * N;
          if (ri < N) xo[ri] = make_double2(xi0[q].x, xi0[q].y);
          if (ri + 32 < N) xo[ri + 32] = make_double2(xi1[q].x, xi1[q].y);
        }
      }
    }
#pragma unroll(NR == 1 ? 2 : 1)
    for (int cc = 0; cc < 2; ++cc) {
      const int ch = 2 * w + cc;                         // rows 16 ch .. 16 ch + 15
      float4 t[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) t[i] = __ldg(src + (ch * 16 + i) * (HT / 2));
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        float2 p[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float2 a = make_float2(t[i].x, t[i].y), b = make_float2(t[i].z, t[i].w);
          p[i] = make_float2(0.f, 0.f);
          cfma(p[i], a, xj0[q]);
          cfma(p[i], b, xj1[q]);
          const float2 xr = shfl2(w == 0 ? xi0[q] : xi1[q], (ch * 16 + i) & 31);
          cfmac(ac0[q], a, xr);
          cfmac(ac1[q], b, xr);
        }
        float2 v8[8], v4[4], v2[2];
        bool hi = lane & 16;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          v8[i] = cadd(hi ? p[i + 8] : p[i], shfl_xor2(hi ? p[i] : p[i + 8], 16));
        hi = lane & 8;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          v4[i] = cadd(hi ? v8[i + 4] : v8[i], shfl_xor2(hi ? v8[i] : v8[i + 4], 8));
        hi = lane & 4;
#pragma unroll
        for (int i = 0; i < 2; ++i)
          v2[i] = cadd(hi ? v4[i + 2] : v4[i], shfl_xor2(hi ? v4[i] : v4[i + 2], 4));
        hi = lane & 2;
        float2 v = cadd(hi ? v2[1] : v2[0], shfl_xor2(hi ? v2[0] : v2[1], 2));
        v = cadd(v, shfl_xor2(v, 1));
        if (!(lane & 1) && q0 + q < nrhs)
          part[(long long)(q0 + q) * ntiles * 2 * HT + 2LL * k * HT + ch * 16 + (lane >> 1)] = v;
      }
    }
    if (I != J) {                                        // column partials: warp 0 + warp 1
      if (w == 1) {
#pragma unroll
        for (int q = 0; q < NR; ++q) colsum[q][lane] = make_float4(ac0[q].x, ac0[q].y, ac1[q].x, ac1[q].y);
      }
      __syncthreads();
      if (w == 0) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const float4 o = colsum[q][lane];
          if (q0 + q < nrhs)
            *(float4*)(part + (long long)(q0 + q) * ntiles * 2 * HT + (2LL * k + 1) * HT + 2 * lane) =
                make_float4(ac0[q].x + o.x, ac0[q].y + o.y, ac1[q].x + o.z, ac1[q].y + o.w);
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per 64-row block: 4 groups of 64 threads each sum a quarter of the
// 64-wide tile row in order; the quarters are added in a fixed order.
__global__ void __launch_bounds__(256) k_hgemv_reduce(const float2* __restrict__ part,
                                                      double2* __restrict__ y, int N, int nt,
                                                      bool accumulate,
                                                      float2* __restrict__ y32) {
  __shared__ float2 red[4][HT];
  const int I = blockIdx.x, rr = threadIdx.x % HT, g = threadIdx.x / HT;
  part += (long long)blockIdx.y * (nt * (nt + 1) / 2) * 2 * HT;
  y += (long long)blockIdx.y * N;
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int J = g; J < nt; J += 4) {
    const long long o = J <= I ? (2LL * (I * (I + 1) / 2 + J)) * HT + rr
                               : (2LL * (J * (J + 1) / 2 + I) + 1) * HT + rr;
    acc = cadd(acc, part[o]);
  }
  red[g][rr] = acc;
  __syncthreads();
  const int row = I * HT + threadIdx.x;
  if (threadIdx.x < HT && row < N) {
    float2 a = red[0][threadIdx.x];
    a = cadd(a, red[1][threadIdx.x]);
    a = cadd(a, red[2][threadIdx.x]);
    a = cadd(a, red[3][threadIdx.x]);
    double2 v = make_double2(a.x, a.y);
    if (accumulate) { v.x += y[row].x; v.y += y[row].y; }
    y[row] = v;
    if (y32) y32[(long long)blockIdx.y * N + row] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t hermitian_gemv_tiles(const void* P, const void* x, int N, int ld, int nrhs,
                                 void* part, cudaStream_t s, void* xscratch) {
  if (ld % HT || ld < N) return cudaErrorInvalidValue;
  const int nt = ld / HT, ntiles = nt * (nt + 1) / 2;
  if (nrhs >= 16 && nrhs <= 64 && xscratch) {   // tensor cores
    const long long n = (long long)ld * nrhs;
    k_x32_pad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2*)x, (float2*)xscratch, N,
                                                        ld, nrhs);
    count_launch();
    const size_t sm = (size_t)HT * (GJC + 2 * GJR) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_hgemv_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    k_hgemv_mma<<<ntiles, 256, sm, s>>>((const float2*)P, (const float2*)xscratch, ld, ntiles,
                                        nrhs, (float2*)part);
    count_launch();
    return cudaGetLastError();
  }
  if (nrhs <= 4) {                               // streamed from global, one warp per tile
    const dim3 grid(ntiles);
    if (nrhs == 1)
      k_hgemv_warp<1><<<grid, 64, 0, s>>>((const float2*)P, (const double2*)x, N, ntiles, nrhs,
                                           (float2*)part, nullptr);
    else if (nrhs == 2)
      k_hgemv_warp<2><<<grid, 64, 0, s>>>((const float2*)P, (const double2*)x, N, ntiles, nrhs,
                                           (float2*)part, nullptr);
    else
      k_hgemv_warp<4><<<grid, 64, 0, s>>>((const float2*)P, (const double2*)x, N, ntiles, nrhs,
                                           (float2*)part, nullptr);
  } else {
    k_hgemv_tiles<<<ntiles, 256, 0, s>>>((const float2*)P, (const double2*)x, N, nrhs,
                                         (float2*)part);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t hermitian_gemv_reduce(const void* part, void* y, int N, int ld, int nrhs,
                                  bool accumulate, cudaStream_t s, void* y32) {
  if (ld % HT || ld < N) return cudaErrorInvalidValue;
  const int nt = ld / HT;
  k_hgemv_reduce<<<dim3(nt, nrhs), 256, 0, s>>>((const float2*)part, (double2*)y, N, nt,
                                                accumulate, (float2*)y32);
  count_launch();
  return cudaGetLastError();
}

bool hermitian_gemv_f32in_ok(int nrhs) { return nrhs >= 1 && nrhs <= 4; }

cudaError_t hermitian_gemv_tiles_f32in(const void* P, const void* x32, int N, int ld, int nrhs,
                                       void* part, void* x64, cudaStream_t s) {
  if (ld % HT || ld < N || !hermitian_gemv_f32in_ok(nrhs)) return cudaErrorInvalidValue;
  const int nt = ld / HT, ntiles = nt * (nt + 1) / 2;
  const dim3 grid(ntiles);
  if (nrhs == 1)
    k_hgemv_warp<1, float2><<<grid, 64, 0, s>>>((const float2*)P, (const float2*)x32, N, ntiles,
                                                 nrhs, (float2*)part, (double2*)x64);
  else if (nrhs == 2)
    k_hgemv_warp<2, float2><<<grid, 64, 0, s>>>((const float2*)P, (const float2*)x32, N, ntiles,
                                                 nrhs, (float2*)part, (double2*)x64);
  else
    k_hgemv_warp<4, float2><<<grid, 64, 0, s>>>((const float2*)P, (const float2*)x32, N, ntiles,
                                                 nrhs, (float2*)part, (double2*)x64);
  count_launch();
  return cudaGetLastError();
}

cudaError_t hermitian_gemv_f32(const void* P, const void* x, void* y, int N, int ld, int nrhs,
                               void* part, bool accumulate, cudaStream_t s) {
  cudaError_t e = hermitian_gemv_tiles(P, x, N, ld, nrhs, part, s, nullptr);
  if (e != cudaSuccess) return e;
  return hermitian_gemv_reduce(part, y, N, ld, nrhs, accumulate, s);
}

__global__ void k_block_map(int Lx, int Lt, int bx, int bt, int32_t* coarse, int32_t* offset) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Lx * Lt) return;
  const int x = i % Lx, t = i / Lx;
  coarse[i] = coarse_site(x, t, Lx, bx, bt);
  offset[i] = block_offset(x, t, bx, bt);
}

cudaError_t block_map(int Lx, int Lt, int bx, int bt, int32_t* coarse, int32_t* offset,
                      cudaStream_t s) {
  k_block_map<<<(Lx * Lt + 255) / 256, 256, 0, s>>>(Lx, Lt, bx, bt, coarse, offset); count_launch();
  return cudaGetLastError();
}

#define INST(R)                                                                                \
  template cudaError_t restrict_op<R>(const void*, void*, const void*, int, int, int, int, int, \
                                      int, int, cudaStream_t);                                 \
  template cudaError_t prolong_op<R>(const void*, void*, const void*, int, int, int, int, int,  \
                                     int, int, bool, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace mgk
