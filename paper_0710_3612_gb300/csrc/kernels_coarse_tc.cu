// Multi-right-hand-side coarse stencil apply on the 5th-generation tensor
// cores (tcgen05, accumulator in tensor memory): Y(j) = sum_d A(j, d) X(j + d)
// for up to 64 right-hand sides, the Galerkin operator of Eq. Galerkin applied
// on a coarse level of the V-cycle (Sec. 2).
//
// Formulation (right-hand sides on the MMA M axis).  Per coarse site j the
// complex product is made real with the real and imaginary parts of X side
// by side along K and of Y side by side along N:
//   D[(r, s)][(p, i)] = sum_{d, q, c} X_s[r][(d, q, c)] B[(p, i)][(d, q, c)],
// r = right-hand side, s = 0 / 1 the BF16 high / low part of X (X = hi + lo,
// lo = bf16(X - hi), about 16 significant bits), q = Re / Im of X, c = column
// of the block, p = Re / Im of Y, i = row of the block, and
//   B[(Re, i)][(d, Re, c)] =  Re A(j,d)[i][c],  B[(Re, i)][(d, Im, c)] = -Im A(j,d)[i][c],
//   B[(Im, i)][(d, Re, c)] =  Im A(j,d)[i][c],  B[(Im, i)][(d, Im, c)] =  Re A(j,d)[i][c].
// Y[r][i] = D[(r, 0)][(., i)] + D[(r, 1)][(., i)].  MMA shape M = 128 (64
// right-hand sides x 2 parts; rows of missing right-hand sides stay zero),
// N = 2n, K = 16 per instruction (kind::f16, BF16 operands, FP32
// accumulation); the blocks are the stored BF16 copy of the operator, so only
// they round.
//
// Pipeline.  A CTA owns the sites j = blockIdx.x + k gridDim.x (k = 0, 1, ...)
// and walks them in chunks of one stencil row dt (3 displacements, K = 6n per
// chunk).  All threads stage a chunk into one of 3 shared-memory stages (X
// converted to the hi/lo rows, A expanded to B, both in the K-major no-swizzle
// core-matrix layout: 8 rows x 16 bytes per core matrix); one thread issues
// the chunk's MMAs and commits them to the stage's mbarrier, which frees the
// stage for chunk + 3.  Two accumulators in tensor memory alternate between
// sites: after the last chunk of site k is issued the CTA reads site k - 1's
// accumulator (tcgen05.ld) and writes its outputs, so staging, MMAs and the
// epilogue overlap.  The global loads of the next chunk go to registers while
// the tensor cores work.  Every wait is bounded: one that runs out sets the
// error flag read by coarse_tc_take_error, and the CTA frees its tensor memory
// and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mgk {

namespace {

__device__ int g_coarse_tc_err;

template <int NDOF>
struct CoarseTC {
  static constexpr int n = NDOF;
  static constexpr int KC = 6 * n;                       // K of one chunk (one stencil row)
  static constexpr int KSTEPS = KC / 16;
  static constexpr int NC = 2 * n;                       // MMA N
  static constexpr int M = 128;                          // MMA M
  static constexpr int A_ELEMS = M * KC;                 // bf16 elements of the X operand
  static constexpr int B_ELEMS = NC * KC;                // bf16 elements of the block operand
  static constexpr int STAGE_BYTES = 2 * (A_ELEMS + B_ELEMS);
  static constexpr int S = 3;                            // stages
  static constexpr int TCOLS = 2 * NC <= 64 ? 64 : 128;  // tensor-memory columns (2 accumulators)
  static constexpr int THREADS = 256;
  static constexpr int XI = 64 * 3 * (n / 2) / THREADS;  // X float4 items per thread and chunk
  static constexpr int AI = (3 * n * (n / 2) + THREADS - 1) / THREADS;   // block uint2 items
  static constexpr int SMEM = S * STAGE_BYTES + 128;     // + alignment slack
  static_assert(n % 8 == 0 && KC % 16 == 0 && NC % 16 == 0 && NC <= 256, "shape");
  static_assert(64 * 3 * (n / 2) % THREADS == 0, "X items");
  static constexpr uint32_t IDESC = tc::idesc_bf16(M, NC);
};

// Element offset of (row, k) in a K-major operand with KC columns: core
// matrix (row / 8, k / 8) of 64 elements, 8 elements (16 bytes) per row.
template <int KC>
__device__ __forceinline__ int op_off(int row, int k) {
  return ((row >> 3) * (KC / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ int wrap(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

template <int NDOF>
__global__ void __launch_bounds__(256, NDOF == 16 ? 2 : 1)
    k_coarse_apply_tc(const float2* __restrict__ in, float2* out,
                      const __nv_bfloat162* __restrict__ A, int Lx, int Lt, int nrhs, Epilogue ep) {
  using C = CoarseTC<NDOF>;
  constexpr int n = C::n, KC = C::KC, S = C::S;
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ __align__(8) uint64_t mbar[S];
  __shared__ __align__(8) uint64_t accbar[2];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int V = Lx * Lt;
  const int ns = (V - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int U = 3 * ns;
  __nv_bfloat16* base =
      (__nv_bfloat16*)(dyn + ((128u - (tc::saddr(dyn) & 127u)) & 127u));
  // rows of missing right-hand sides are never written: clear every stage once
  {
    uint4* z = (uint4*)base;
    for (int q = tid; q < S * C::STAGE_BYTES / 16; q += C::THREADS) z[q] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) tc::tmem_alloc(&tmem_sh, C::TCOLS);
  if (tid == 0) {
    for (int q = 0; q < S; ++q) tc::mbar_init(&mbar[q], 1);
    tc::mbar_init(&accbar[0], 1);
    tc::mbar_init(&accbar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;

  float4 xr[C::XI];
  uint2 ar[C::AI];
  // chunk u: site k = u / 3 of this CTA, stencil row dt = u % 3 - 1
  auto load = [&](int u) {
    const int k = u / 3, c = u % 3;
    const int j = (int)blockIdx.x + k * (int)gridDim.x;
    const int x = j % Lx, t = j / Lx, tn = wrap(t + c - 1, Lt);
#pragma unroll
    for (int i = 0; i < C::XI; ++i) {
      const int e = tid + C::THREADS * i, g = e >> 5;
      const int cp = (g % (n / 8)) * 4 + (e & 3), q = g / (n / 8);
      const int dl = q % 3, r = (q / 3) * 8 + ((e >> 2) & 7);
      const int xn = wrap(x + dl - 1, Lx);
      xr[i] = r < nrhs ? __ldg((const float4*)(in + ((long long)r * V + xn + Lx * tn) * n + 2 * cp))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < C::AI; ++i) {
      const int e = tid + C::THREADS * i, g = e >> 5;
      if (e < 3 * n * (n / 2)) {
        const int cp = (g % (n / 8)) * 4 + (e & 3), q = g / (n / 8);
        const int row = (q % (n / 8)) * 8 + ((e >> 2) & 7), dl = q / (n / 8);
        const int d = dl + 3 * c;
        ar[i] = __ldg((const uint2*)(A + (((long long)j * 9 + d) * n + row) * n + 2 * cp));
      }
    }
  };
  auto store = [&](int st) {
    __nv_bfloat16* Aop = base + (size_t)st * (C::A_ELEMS + C::B_ELEMS);
    __nv_bfloat16* Bop = Aop + C::A_ELEMS;
#pragma unroll
    for (int i = 0; i < C::XI; ++i) {
      const int e = tid + C::THREADS * i, g = e >> 5;
      const int cp = (g % (n / 8)) * 4 + (e & 3), q = g / (n / 8);
      const int dl = q % 3, r = (q / 3) * 8 + ((e >> 2) & 7);
      if (r >= nrhs) continue;
      const float4 v = xr[i];                      // (re, im) of columns 2 cp, 2 cp + 1
      const __nv_bfloat162 hre = __floats2bfloat162_rn(v.x, v.z);
      const __nv_bfloat162 him = __floats2bfloat162_rn(v.y, v.w);
      const float2 fre = __bfloat1622float2(hre), fim = __bfloat1622float2(him);
      const __nv_bfloat162 lre = __floats2bfloat162_rn(v.x - fre.x, v.z - fre.y);
      const __nv_bfloat162 lim = __floats2bfloat162_rn(v.y - fim.x, v.w - fim.y);
      const int kre = dl * 2 * n + 2 * cp, kim = kre + n;
      *(__nv_bfloat162*)(Aop + op_off<KC>(2 * r, kre)) = hre;
      *(__nv_bfloat162*)(Aop + op_off<KC>(2 * r, kim)) = him;
      *(__nv_bfloat162*)(Aop + op_off<KC>(2 * r + 1, kre)) = lre;
      *(__nv_bfloat162*)(Aop + op_off<KC>(2 * r + 1, kim)) = lim;
    }
#pragma unroll
    for (int i = 0; i < C::AI; ++i) {
      const int e = tid + C::THREADS * i, g = e >> 5;
      if (e < 3 * n * (n / 2)) {
        const int cp = (g % (n / 8)) * 4 + (e & 3), q = g / (n / 8);
        const int row = (q % (n / 8)) * 8 + ((e >> 2) & 7), dl = q / (n / 8);
        const __nv_bfloat162 c0 = *(const __nv_bfloat162*)&ar[i].x;   // (re, im) of column 2 cp
        const __nv_bfloat162 c1 = *(const __nv_bfloat162*)&ar[i].y;   // column 2 cp + 1
        const __nv_bfloat162 are = __halves2bfloat162(c0.x, c1.x);
        const __nv_bfloat162 aim = __halves2bfloat162(c0.y, c1.y);
        const int kre = dl * 2 * n + 2 * cp, kim = kre + n;
        *(__nv_bfloat162*)(Bop + op_off<KC>(row, kre)) = are;
        *(__nv_bfloat162*)(Bop + op_off<KC>(row, kim)) = __hneg2(aim);
        *(__nv_bfloat162*)(Bop + op_off<KC>(n + row, kre)) = aim;
        *(__nv_bfloat162*)(Bop + op_off<KC>(n + row, kim)) = are;
      }
    }
  };
  // outputs of site k from accumulator k % 2
  auto epilogue = [&](int k) -> bool {
    const int buf = k & 1;
    bool good = tc::mbar_wait(&accbar[buf], (uint32_t)((k >> 1) & 1), &g_coarse_tc_err);
    good = __syncthreads_and(good);
    if (!good) return false;
    tc::fence_after_sync();
    constexpr int H = n / 2;                       // block rows of this warp's half
    const int qd = warp & 3, hh = warp >> 2;
    const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * C::NC + hh * H);
    float vre[H], vim[H];
    tc::tmem_ld8(tb, vre);
    tc::tmem_ld8(tb + n, vim);
    if constexpr (H == 12) {
      tc::tmem_ld4(tb + 8, vre + 8);
      tc::tmem_ld4(tb + n + 8, vim + 8);
    }
    tc::tmem_wait_ld();
    tc::fence_before_sync();
#pragma unroll
    for (int i = 0; i < H; ++i) {
      vre[i] += __shfl_xor_sync(0xffffffffu, vre[i], 1);   // hi + lo rows
      vim[i] += __shfl_xor_sync(0xffffffffu, vim[i], 1);
    }
    const int r = 16 * qd + (lane >> 1);
    const int j = (int)blockIdx.x + k * (int)gridDim.x;
    if ((lane & 1) == 0 && r < nrhs) {
      const long long o = ((long long)r * V + j) * n + hh * H;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        float2 y = make_float2((float)ep.ca * vre[i], (float)ep.ca * vim[i]);
        if (ep.U) {
          const float2 w = ((const float2*)ep.U)[o + i];
          y = make_float2(y.x + (float)ep.cu * w.x, y.y + (float)ep.cu * w.y);
        }
        if (ep.W) {
          const float2 w = ((const float2*)ep.W)[o + i];
          y = make_float2(y.x + (float)ep.cw * w.x, y.y + (float)ep.cw * w.y);
        }
        out[o + i] = y;
      }
    }
    return true;
  };

  bool ok = true;
  if (U > 0) load(0);
  for (int u = 0; u < U; ++u) {
    const int st = u % S, k = u / 3, c = u % 3;
    if (u >= S) ok = tc::mbar_wait(&mbar[st], (uint32_t)((u / S - 1) & 1), &g_coarse_tc_err);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    store(st);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::saddr(base + (size_t)st * (C::A_ELEMS + C::B_ELEMS));
      const uint32_t b0 = a0 + 2 * C::A_ELEMS;
      const uint32_t d = tmem + (uint32_t)((k & 1) * C::NC);
#pragma unroll
      for (int kk = 0; kk < C::KSTEPS; ++kk) {
        const uint64_t da = tc::desc(a0 + 256 * kk, 128, (KC / 8) * 128);
        const uint64_t db = tc::desc(b0 + 256 * kk, 128, (KC / 8) * 128);
        tc::mma_bf16(d, da, db, C::IDESC, (c | kk) ? 1u : 0u);
      }
      tc::commit(&mbar[st]);
      if (c == 2) tc::commit(&accbar[k & 1]);
    }
    if (u + 1 < U) load(u + 1);
    if (c == 2 && k >= 1) {
      ok = epilogue(k - 1);
      if (!ok) break;
    }
  }
  if (ok && U > 0) ok = epilogue(ns - 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
}

template <int NDOF>
cudaError_t launch_tc(const void* in, void* out, const void* A, int Lx, int Lt, int nrhs,
                      const Epilogue& ep, cudaStream_t s) {
  using C = CoarseTC<NDOF>;
  static int grid_max = 0;
  if (!grid_max) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_apply_tc<NDOF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_apply_tc<NDOF>, C::THREADS,
                                                  C::SMEM);
    // at most 512 / TCOLS CTAs of this kernel share an SM's tensor memory
    per = per < 1 ? 1 : (per > 512 / C::TCOLS ? 512 / C::TCOLS : per);
    grid_max = sms * per;
  }
  const int V = Lx * Lt;
  const int grid = V < grid_max ? V : grid_max;
  k_coarse_apply_tc<NDOF><<<grid, C::THREADS, C::SMEM, s>>>(
      (const float2*)in, (float2*)out, (const __nv_bfloat162*)A, Lx, Lt, nrhs, ep);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool coarse_apply_tcgen05_ok(int n, int nrhs) {
  return (n == 16 || n == 24) && nrhs >= 1 && nrhs <= 64;
}

cudaError_t coarse_apply_tcgen05(const void* in, void* out, const void* A, int Lx, int Lt, int n,
                                 int nrhs, const Epilogue& ep, cudaStream_t s) {
  if (!coarse_apply_tcgen05_ok(n, nrhs) || Lx < 1 || Lt < 1) return cudaErrorInvalidValue;
  return n == 16 ? launch_tc<16>(in, out, A, Lx, Lt, nrhs, ep, s)
                 : launch_tc<24>(in, out, A, Lx, Lt, nrhs, ep, s);
}

cudaError_t coarse_tc_take_error(int* flag) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_coarse_tc_err, sizeof(int));
  if (e != cudaSuccess) return e;
  if (v) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_coarse_tc_err, &zero, sizeof(int));
  }
  *flag = v;
  return e;
}

}  // namespace mgk
