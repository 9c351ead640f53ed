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
// Sliding window.  A CTA walks strips of consecutive sites along x (one
// row t, up to SL sites).  The X operand is staged per coarse site as a
// block of 128 rows x 2n (the hi / lo rows of 64 right-hand sides, Re and Im
// halves along K), K-major without swizzle (8 rows x 16 bytes per core
// matrix).  A ring of NCOL columns x 3 rows of blocks holds the neighbourhood
// of the current site; stepping to the next site converts one new column (3
// blocks) into the slot of the oldest column, and the site's blocks of A into
// B (2n x 18n).  The raw data of each step (the new column of X in FP32 and
// the site's BF16 blocks) is fetched R steps ahead by the tensor memory
// accelerator into a ring of raw slots: three 2D tensor loads of X (one per
// row of the column: nrhs rows of n complex, with the 128-byte swizzle when a
// row is 128 bytes, so that the conversion reads are free of bank conflicts)
// and one bulk copy of the blocks, all completing on the slot's mbarrier.
//
// Roles, synchronised through mbarriers only: warps 0-7 convert and write
// outputs, warp 8 issues the MMAs, warp 9 issues the loads.  The loader fills
// raw slot q % R with load q once the converting threads have released the
// slot's previous load (empty[q % R]); the load completes rawbar[q % R].
// When a site's operands are in place the 256 converting threads arrive on
// full[g % 2]; warp 8 waits there, issues the site's 9 displacements x 2n / 16
// K-steps into accumulator g % 2 of tensor memory (each K-step reading its
// neighbour's staged block through its own descriptor) and commits them to
// done[g % 2].  The converting threads wait on done before they overwrite a
// ring slot or B buffer the MMAs may still read, and before they read an
// accumulator (tcgen05.ld) to write the outputs.  Every wait is bounded: one
// that runs out sets the flag read by coarse_tc_take_error, and the CTA
// frees its tensor memory and returns.
#include <cuda.h>
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
  static constexpr int KB = 2 * n;                       // K of one staged block (Re, Im)
  static constexpr int KA = 18 * n;                      // K of a site: 9 blocks
  static constexpr int BSTEPS = KB / 16;                 // K-steps per block
  static constexpr int NC = 2 * n;                       // MMA N
  static constexpr int M = 128;                          // MMA M
  static constexpr int XBLK = M * KB;                    // bf16 elements of a staged block
  static constexpr int BELEM = NC * KA;                  // bf16 elements of a site's B
  static constexpr int NCOL = n <= 16 ? 4 : 3;           // ring columns
  static constexpr int NB = n <= 16 ? 2 : 1;             // B buffers
  static constexpr int FIXED = 2 * (3 * NCOL * XBLK + NB * BELEM);   // operand bytes
  static constexpr int TCOLS = 2 * NC <= 64 ? 64 : 128;  // tensor-memory columns (2 accumulators)
  static constexpr int PRODUCERS = 256;                  // warps 0-7
  static constexpr int THREADS = PRODUCERS + 64;         // + the MMA warp and the load warp
  static constexpr int C8 = n / 8;                       // 8-column groups of a block row
  static constexpr int P = n / 2;                        // 16-byte chunks per raw X row
  static constexpr bool SWZ = n == 16;                   // raw X rows of 128 bytes, swizzled
  static constexpr int ACH = 9 * n * n / 4;              // 16-byte chunks of a site's blocks
  static constexpr int XITEMS = 64 * 3 * C8;             // conversion items of a column
  static constexpr int XI = (XITEMS + PRODUCERS - 1) / PRODUCERS;
  static constexpr int BITEMS = 9 * n * C8;              // expansion items of a site's blocks
  static constexpr int BI = (BITEMS + PRODUCERS - 1) / PRODUCERS;
  static_assert(n % 8 == 0 && KB % 16 == 0 && NC % 16 == 0 && NC <= 256, "shape");
  static_assert(ACH % 8 == 0 && FIXED % (SWZ ? 1024 : 128) == 0, "chunks, alignment");
  static constexpr uint32_t IDESC = tc::idesc_bf16(M, NC);
  // raw bytes of one step for nr rows of right-hand sides (nr a multiple of 8)
  // (a multiple of 1024 when the X rows are swizzled: each load's boxes start on
  // a 1024-byte boundary)
  static __host__ __device__ constexpr int raw_bytes(int nr) { return 3 * nr * P * 16 + ACH * 16; }
};

// Byte offset of (row, k) (k a multiple of 8) in a K-major operand with K
// columns: core matrix (row / 8, k / 8) of 128 bytes, 16 bytes per row.
template <int K>
__host__ __device__ __forceinline__ int op_byte(int row, int k) {
  return ((row >> 3) * (K / 8) + (k >> 3)) * 128 + (row & 7) * 16;
}


__device__ __forceinline__ int wrap(int a, int L) {
  a %= L;
  return a < 0 ? a + L : a;
}

__device__ __forceinline__ uint32_t bf2u(__nv_bfloat162 v) { return *(uint32_t*)&v; }

// 2D tensor load of one box into shared memory, completing on mbar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];\n"
      :: "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(tc::saddr(mbar)) : "memory");
}
// contiguous bulk copy (bytes a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
      :: "r"(dst), "l"(src), "r"(bytes), "r"(tc::saddr(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               :: "r"(tc::saddr(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n"
               :: "r"(tc::saddr(m)) : "memory");
}

template <int NDOF>
__global__ void __launch_bounds__(320, 1)
    k_coarse_apply_tc(const __grid_constant__ CUtensorMap xmap, float2* out,
                      const __nv_bfloat162* __restrict__ A, int Lx, int Lt, int nrhs, int SL,
                      int R, Epilogue ep) {
  using C = CoarseTC<NDOF>;
  constexpr int n = C::n, KB = C::KB, KA = C::KA, C8 = C::C8, P = C::P, NCOL = C::NCOL;
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ __align__(8) uint64_t full[2], done[2], rawbar[4], empty[4];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int V = Lx * Lt;
  const int NR = (nrhs + 7) & ~7;                        // raw rows per column row
  const int spr = (Lx + SL - 1) / SL;                    // strips per row
  const int NS = spr * Lt;
  unsigned char* xs = dyn + ((1024u - (tc::saddr(dyn) & 1023u)) & 1023u);
  unsigned char* bs = xs + 2 * 3 * NCOL * C::XBLK;       // NB B buffers
  unsigned char* raw = bs + 2 * C::NB * C::BELEM;        // R raw slots
  const int RAWB = C::raw_bytes(NR);
  // rows of missing right-hand sides are never written: clear the blocks once
  for (int q = tid; q < 3 * NCOL * C::XBLK / 8; q += C::THREADS)
    ((uint4*)xs)[q] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&tmem_sh, C::TCOLS);
  if (tid == 0) {
    tc::mbar_init(&full[0], C::PRODUCERS);
    tc::mbar_init(&full[1], C::PRODUCERS);
    tc::mbar_init(&done[0], 1);
    tc::mbar_init(&done[1], 1);
    for (int q = 0; q < 4; ++q) {
      tc::mbar_init(&rawbar[q], 1);
      tc::mbar_init(&empty[q], C::PRODUCERS);
    }
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  bool ok = true;

  if (warp == 8) {
    // ---- MMA warp: the sites of this CTA in order
    int g = 0;
    for (int sidx = blockIdx.x; sidx < NS && ok; sidx += gridDim.x) {
      const int len = min(SL, Lx - (sidx % spr) * SL);
      for (int i = 0; i < len; ++i, ++g) {
        ok = tc::mbar_wait(&full[g & 1], (uint32_t)((g >> 1) & 1), &g_coarse_tc_err);
        if (!ok) break;
        if (lane == 0) {
          tc::fence_after_sync();
          const uint32_t x0a = tc::saddr(xs), b0 = tc::saddr(bs + (g % C::NB) * C::BELEM * 2);
          const uint32_t d = tmem + (uint32_t)((g & 1) * C::NC);
#pragma unroll
          for (int dd = 0; dd < 9; ++dd) {
            const int slot = (i + dd % 3) % NCOL, tr = dd / 3;   // column i + dd % 3 of the strip
            const uint32_t blk = x0a + (uint32_t)((slot * 3 + tr) * C::XBLK * 2);
#pragma unroll
            for (int kk = 0; kk < C::BSTEPS; ++kk) {
              const uint64_t da = tc::desc(blk + 256 * kk, 128, (KB / 8) * 128);
              const uint64_t db = tc::desc(b0 + 256 * (dd * C::BSTEPS + kk), 128, (KA / 8) * 128);
              tc::mma_bf16(d, da, db, C::IDESC, (dd | kk) ? 1u : 0u);
            }
          }
          tc::commit(&done[g & 1]);
        }
        __syncwarp();
      }
    }
  } else if (warp == 9) {
    // ---- load warp: the loads of this CTA in order.  Load k of a strip (k =
    // 0 .. len + 1) is column x0 - 1 + k of rows t - 1, t, t + 1 and, for k >= 2,
    // the blocks of site x0 + k - 2.  Load q uses raw slot q % R.
    if (lane == 0) {
      int q = 0;
      for (int sidx = blockIdx.x; sidx < NS && ok; sidx += gridDim.x) {
        const int t = sidx / spr, x0 = (sidx % spr) * SL;
        const int len = min(SL, Lx - x0);
        for (int k = 0; k < len + 2; ++k, ++q) {
          const int slot = q % R;
          if (q >= R) {              // the converting threads are done with load q - R
            ok = tc::mbar_wait(&empty[slot], (uint32_t)((q / R - 1) & 1), &g_coarse_tc_err);
            if (!ok) break;
          }
          const uint32_t rb = tc::saddr(raw + slot * RAWB);
          const int xw = wrap(x0 - 1 + k, Lx);
          const uint32_t xbytes = 3u * NR * P * 16;
          mbar_expect_tx(&rawbar[slot], xbytes + (k >= 2 ? C::ACH * 16u : 0u));
#pragma unroll
          for (int tr = 0; tr < 3; ++tr) {
            const int site = xw + Lx * wrap(t + tr - 1, Lt);
            tma_load_2d(rb + tr * NR * P * 16, &xmap, site * 2 * n, 0, &rawbar[slot]);
          }
          if (k >= 2) {
            const int j = x0 + k - 2 + Lx * t;
            bulk_load(rb + xbytes, A + (long long)j * 9 * n * n, C::ACH * 16u, &rawbar[slot]);
          }
        }
      }
    }
    __syncwarp();
  } else {
    // conversion of a raw column into ring column `slot`.  X item e: r = 4 (..)
    // + (e & 3), combo = (tr, 8-column group); lanes 4k..4k+3 write the high
    // rows first and lanes 4k+4..4k+7 the low rows first (8 distinct rows of a
    // core matrix: no bank conflicts).
    auto convert_col = [&](const unsigned char* rs, int slot) {
      unsigned char* colb = xs + slot * 3 * C::XBLK * 2;
#pragma unroll
      for (int i = 0; i < C::XI; ++i) {
        const int e = tid + C::PRODUCERS * i, u = e >> 2;
        const int combo = u % (3 * C8), r = (u / (3 * C8)) * 4 + (e & 3);
        if (e >= C::XITEMS || r >= nrhs) continue;
        const int tr = combo % 3, c8 = combo / 3;
        const bool flip = (u & 1) != 0;
        const unsigned char* rrow = rs + (tr * NR + r) * P * 16;
        const int sw = C::SWZ ? (r & 7) : 0;       // the tensor load's 128-byte swizzle
        uint32_t hre[4], him[4], lre[4], lim[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 v = *(const float4*)(rrow + ((4 * c8 + k) ^ sw) * 16);
          const __nv_bfloat162 hr = __floats2bfloat162_rn(v.x, v.z);
          const __nv_bfloat162 hi = __floats2bfloat162_rn(v.y, v.w);
          const float2 fr = __bfloat1622float2(hr), fi = __bfloat1622float2(hi);
          hre[k] = bf2u(hr);
          him[k] = bf2u(hi);
          lre[k] = bf2u(__floats2bfloat162_rn(v.x - fr.x, v.z - fr.y));
          lim[k] = bf2u(__floats2bfloat162_rn(v.y - fi.x, v.w - fi.y));
        }
        unsigned char* p = colb + tr * C::XBLK * 2 + op_byte<KB>(2 * r + (flip ? 1 : 0), 8 * c8);
        const int other = flip ? -16 : 16;           // the other part's row
        const uint4 Hre = make_uint4(hre[0], hre[1], hre[2], hre[3]);
        const uint4 Him = make_uint4(him[0], him[1], him[2], him[3]);
        const uint4 Lre = make_uint4(lre[0], lre[1], lre[2], lre[3]);
        const uint4 Lim = make_uint4(lim[0], lim[1], lim[2], lim[3]);
        *(uint4*)p = flip ? Lre : Hre;
        *(uint4*)(p + n * 16) = flip ? Lim : Him;
        *(uint4*)(p + other) = flip ? Hre : Lre;
        *(uint4*)(p + other + n * 16) = flip ? Him : Lim;
      }
    };
    // B item e: block row 8 (..) + (e & 7), (d, 8-column group) from e >> 3
    auto convert_B = [&](const unsigned char* rs, int buf) {
      const unsigned char* ab = rs + 3 * NR * P * 16;
      unsigned char* Bop = bs + buf * C::BELEM * 2;
#pragma unroll
      for (int i = 0; i < C::BI; ++i) {
        const int e = tid + C::PRODUCERS * i, u = e >> 3;
        if (e >= C::BITEMS) continue;
        const int ih = u % C8, c8 = (u / C8) % C8, d = u / (C8 * C8);
        const int row = ih * 8 + (e & 7);
        const int q0 = ((d * n + row) * n + 8 * c8) / 4;   // chunk of columns 8 c8 .. 8 c8 + 3
        const uint4 w0 = *(const uint4*)(ab + q0 * 16);
        const uint4 w1 = *(const uint4*)(ab + (q0 + 1) * 16);
        const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        uint32_t re[4], im[4], nim[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {                // (re, im) words of columns 2k, 2k+1
          re[k] = __byte_perm(w[2 * k], w[2 * k + 1], 0x5410);
          im[k] = __byte_perm(w[2 * k], w[2 * k + 1], 0x7632);
          nim[k] = im[k] ^ 0x80008000u;
        }
        unsigned char* p = Bop + op_byte<KA>(row, d * KB + 8 * c8);
        const int lower = (n / 8) * (KA / 8) * 128;  // rows n + i: n / 8 groups of 8 rows further
        *(uint4*)p = make_uint4(re[0], re[1], re[2], re[3]);
        *(uint4*)(p + n * 16) = make_uint4(nim[0], nim[1], nim[2], nim[3]);
        *(uint4*)(p + lower) = make_uint4(im[0], im[1], im[2], im[3]);
        *(uint4*)(p + lower + n * 16) = make_uint4(re[0], re[1], re[2], re[3]);
      }
    };
    // outputs of site j from accumulator buf (its MMAs have completed)
    auto epilogue = [&](int j, int buf) {
      tc::fence_after_sync();
      constexpr int H = n / 2;                     // block rows of this warp's half
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
      // the even lane writes the first half of the row's H outputs, the odd lane the second
      const int r = 16 * qd + (lane >> 1), half = lane & 1;
      if (r < nrhs) {
        const long long o = ((long long)r * V + j) * n + hh * H + half * (H / 2);
        const float ca = (float)ep.ca, cu = (float)ep.cu, cw = (float)ep.cw;
#pragma unroll
        for (int i = 0; i < H / 2; i += 2) {      // two complex outputs per 16-byte store
          float4 y;
          y.x = ca * (half ? vre[H / 2 + i] : vre[i]);
          y.y = ca * (half ? vim[H / 2 + i] : vim[i]);
          y.z = ca * (half ? vre[H / 2 + i + 1] : vre[i + 1]);
          y.w = ca * (half ? vim[H / 2 + i + 1] : vim[i + 1]);
          if (ep.U) {
            const float4 w = *(const float4*)((const float2*)ep.U + o + i);
            y.x += cu * w.x; y.y += cu * w.y; y.z += cu * w.z; y.w += cu * w.w;
          }
          if (ep.W) {
            const float4 w = *(const float4*)((const float2*)ep.W + o + i);
            y.x += cw * w.x; y.y += cw * w.y; y.z += cw * w.z; y.w += cw * w.w;
          }
          *(float4*)(out + o + i) = y;
        }
      }
    };
    auto wait_done = [&](int site) -> bool {
      return tc::mbar_wait(&done[site & 1], (uint32_t)((site >> 1) & 1), &g_coarse_tc_err);
    };

    int g = 0;                     // sites handed to the MMA warp; site g uses accumulator g & 1
    int q = 0;                     // loads consumed
    for (int sidx = blockIdx.x; sidx < NS && ok; sidx += gridDim.x) {
      const int t = sidx / spr, x0 = (sidx % spr) * SL;
      const int len = min(SL, Lx - x0);
      for (int k = 0; k < len + 2; ++k, ++q) {
        // the MMAs that may still read the ring slot (and B buffer) about to be
        // replaced: at a strip's first load every earlier site, then the site
        // that last used the column NCOL loads back
        if (k == 0 && g > 0) ok = wait_done(g - 1);
        else if (k >= 2 && g - (NCOL - 2) >= 0) ok = wait_done(g - (NCOL - 2));
        const int slot = q % R;
        ok = ok && tc::mbar_wait(&rawbar[slot], (uint32_t)((q / R) & 1), &g_coarse_tc_err);
        if (!ok) break;
        const unsigned char* rs = raw + slot * RAWB;
        convert_col(rs, k % NCOL);
        if (k >= 2) convert_B(rs, g % C::NB);
        mbar_arrive(&empty[slot]);   // the raw slot may be refilled
        if (k >= 2) {
          tc::fence_proxy_async();
          mbar_arrive(&full[g & 1]);   // operands of site g in place
        }
        if (k >= 3) {                // outputs of the previous site of this strip
          ok = wait_done(g - 1);
          if (!ok) break;
          epilogue(x0 + k - 3 + Lx * t, (g - 1) & 1);
        }
        if (k >= 2) ++g;
      }
      if (ok && len > 0) {           // the strip's last site
        ok = wait_done(g - 1);
        if (ok) epilogue(x0 + len - 1 + Lx * t, (g - 1) & 1);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

template <int NDOF>
cudaError_t launch_tc(const void* in, void* out, const void* A, int Lx, int Lt, int nrhs,
                      const Epilogue& ep, cudaStream_t s) {
  using C = CoarseTC<NDOF>;
  static int sms = 0, dyn_max = 0;
  if (!sms) {
    // the largest dynamic shared memory a block may opt in to, less the static part
    int dev = 0, m = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, k_coarse_apply_tc<NDOF>);
    if (e != cudaSuccess) return e;
    const int dm = optin - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(k_coarse_apply_tc<NDOF>, cudaFuncAttributeMaxDynamicSharedMemorySize, dm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_coarse_apply_tc<NDOF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dyn_max = dm;
    sms = m > 0 ? m : 1;
  }
  EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  // X as a 2D FP32 tensor [nrhs][V * 2n]: a box is one site's nrhs rows (NR
  // rows, the ones past nrhs read as zero) of 2n floats
  const int NR = (nrhs + 7) & ~7;
  const long long V = (long long)Lx * Lt;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)V * 2 * NDOF, (cuuint64_t)nrhs};
  const cuuint64_t strides[1] = {(cuuint64_t)V * 2 * NDOF * 4};
  const cuuint32_t box[2] = {2 * NDOF, (cuuint32_t)NR};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(in), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE,
          C::SWZ ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  // raw ring depth: as many loads ahead as shared memory allows, at most 4
  const int avail = dyn_max - C::FIXED - 1024;
  int R = avail / C::raw_bytes(NR);
  R = R > 4 ? 4 : R;
  if (R < 1) return cudaErrorInvalidValue;
  const int smem = C::FIXED + R * C::raw_bytes(NR) + 1024;
  // one CTA per SM; strips of SL sites, short enough that every CTA gets one, at most 8
  int SL = (int)((V + sms - 1) / sms);
  SL = SL < 2 ? 2 : (SL > 8 ? 8 : SL);
  if (SL > Lx) SL = Lx;
  const long long NS = (long long)((Lx + SL - 1) / SL) * Lt;
  const int grid = (int)(NS < sms ? NS : sms);
  k_coarse_apply_tc<NDOF><<<grid, C::THREADS, smem, s>>>(map, (float2*)out,
                                                        (const __nv_bfloat162*)A, Lx, Lt, nrhs, SL,
                                                        R, ep);
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
