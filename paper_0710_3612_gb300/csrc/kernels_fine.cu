// Fine-lattice Wilson-Dirac operator D and D^dagger (Sec. 1 of the paper,
// display after Eq. 1), 2D, U(1) links, gamma_1 = sigma_1 (x), gamma_2 =
// sigma_2 (t), diagonal 4 + m, t antiperiodic (sign folded into the t link at
// t = Lt - 1 by fold_links).
//
// Spin projection: (1 - s sigma_1) phi = (phi0 - s phi1) (1, -s)^T and
// (1 - s sigma_2) phi = (phi0 + i s phi1) (1, -i s)^T, so each hop is one
// complex projection, one link multiply and a rank-1 reconstruction.
// D uses s = +1 forward (x + mu) and s = -1 backward; D^dagger swaps them.
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "kernels.h"

namespace mgk {

template <typename R, bool DAG>
__device__ __forceinline__ void wilson_site(const cplx_t<R>* __restrict__ in,
                                            const cplx_t<R>* __restrict__ U, R diag, int x, int t,
                                            int Lx, int Lt, cplx_t<R>& o0, cplx_t<R>& o1) {
  using C = cplx_t<R>;
  const int V = Lx * Lt;
  const int site = x + Lx * t;
  const int xp = (x + 1 == Lx) ? site - x : site + 1;
  const int xm = (x == 0) ? site + Lx - 1 : site - 1;
  const int tp = (t + 1 == Lt) ? x : site + Lx;
  const int tm = (t == 0) ? site + (Lt - 1) * Lx : site - Lx;
  const R sf = DAG ? (R)-1 : (R)1;   // projector sign of the forward hop
  C a0 = mk((R)0, (R)0), a1 = mk((R)0, (R)0);
  hop_x<R>(a0, a1, U[site], in[2 * xp], in[2 * xp + 1], sf);
  hop_x<R>(a0, a1, cconj(U[xm]), in[2 * xm], in[2 * xm + 1], -sf);
  hop_t<R>(a0, a1, U[V + site], in[2 * tp], in[2 * tp + 1], sf);
  hop_t<R>(a0, a1, cconj(U[V + tm]), in[2 * tm], in[2 * tm + 1], -sf);
  C p0 = in[2 * site], p1 = in[2 * site + 1];
  o0 = mk(diag * p0.x - (R)0.5 * a0.x, diag * p0.y - (R)0.5 * a0.y);
  o1 = mk(diag * p1.x - (R)0.5 * a1.x, diag * p1.y - (R)0.5 * a1.y);
}

template <typename R, bool DAG>
__global__ void __launch_bounds__(256) k_wilson_D(const cplx_t<R>* __restrict__ in,
                                                  cplx_t<R>* __restrict__ out,
                                                  const cplx_t<R>* __restrict__ U, R diag, int Lx,
                                                  int Lt) {
  const int V = Lx * Lt;
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= V) return;
  const long long off = (long long)blockIdx.y * V * 2;
  cplx_t<R> o0, o1;
  wilson_site<R, DAG>(in + off, U, diag, site % Lx, site / Lx, Lx, Lt, o0, o1);
  out[off + 2 * site] = o0;
  out[off + 2 * site + 1] = o1;
}

template <typename R>
cudaError_t wilson_D(const void* in, void* out, const void* U, double diag, int Lx, int Lt,
                     int nrhs, bool dagger, cudaStream_t s) {
  const int V = Lx * Lt;
  dim3 grid((V + 255) / 256, nrhs);
  if (dagger)
    k_wilson_D<R, true><<<grid, 256, 0, s>>>((const cplx_t<R>*)in, (cplx_t<R>*)out,
                                             (const cplx_t<R>*)U, (R)diag, Lx, Lt);
  else
    k_wilson_D<R, false><<<grid, 256, 0, s>>>((const cplx_t<R>*)in, (cplx_t<R>*)out,
                                              (const cplx_t<R>*)U, (R)diag, Lx, Lt);
  count_launch();
  return cudaGetLastError();
}

// Fused A = D^dagger D.  A CTA of TX x TY threads owns a TX x (TY * RPT) tile
// of output sites (each thread RPT sites of one column).  It stages psi on the
// tile plus a 2-site halo and the links on the tile plus a 2-site halo below /
// 1-site halo above in shared memory, forms D psi on the tile plus a 1-site
// halo, and applies D^dagger to it -- one pass over psi and the links.
// Coordinates wrap periodically (the antiperiodic sign sits in the links), so
// lattices that are not multiples of the tile work unchanged.
// Tile geometry: TX x (TY * RPT) sites per CTA of TX x TY threads.  Large
// lattices use 32 x 16 (FP32, two rows per thread) or 32 x 8 (FP64, shared
// memory below 48 KB); lattices with fewer than two tiles per SM use 16 x 8
// tiles so that every SM gets work.

template <typename R> struct spinor_t;              // both spin components of a site
template <> struct spinor_t<float> { using type = float4; };
template <> struct spinor_t<double> { using type = double4_32a; };

__device__ __forceinline__ void split(const float4& v, float2& a, float2& b) {
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void split(const double4_32a& v, double2& a, double2& b) {
  a = make_double2(v.x, v.y);
  b = make_double2(v.z, v.w);
}
__device__ __forceinline__ float4 join(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ double4_32a join(double2 a, double2 b) {
  double4_32a r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}
__device__ __forceinline__ float4 ld_spinor(const float2* p) { return *(const float4*)p; }
__device__ __forceinline__ double4_32a ld_spinor(const double2* p) {
  const double2 a = p[0], b = p[1];
  return join(a, b);
}
__device__ __forceinline__ void st_spinor(float2* p, float4 v) { *(float4*)p = v; }
__device__ __forceinline__ void st_spinor(double2* p, double4_32a v) {
  p[0] = make_double2(v.x, v.y);
  p[1] = make_double2(v.z, v.w);
}

__device__ __forceinline__ int wrap(int g, int L) { return g < 0 ? g + L : (g >= L ? g - L : g); }

template <typename R, int TX, int TY, int RPT>
__global__ void __launch_bounds__(TX* TY) k_wilson_A(const cplx_t<R>* __restrict__ in,
                                                     cplx_t<R>* out,
                                                     const cplx_t<R>* __restrict__ U, R diag,
                                                     int Lx, int Lt, Epilogue ep) {
  constexpr int TT = TY * RPT;
  constexpr int PW = TX + 4, PH = TT + 4;     // psi region [-2, TX+1] x [-2, TT+1]
  constexpr int DW = TX + 2, DH = TT + 2;     // D psi region [-1, TX] x [-1, TT]
  constexpr int UW = TX + 3, UH = TT + 3;     // link region [-2, TX] x [-2, TT]
  using C = cplx_t<R>;
  using S = typename spinor_t<R>::type;
  __shared__ S sp[PH * PW];
  __shared__ S sd[DH * DW];
  __shared__ C su[UH * UW][2];
  const int V = Lx * Lt;
  const int x0 = blockIdx.x * TX, t0 = blockIdx.y * TT;
  const long long off = (long long)blockIdx.z * V * 2;
  const int tid = threadIdx.x;
  for (int q = tid; q < PH * PW; q += TX * TY) {
    const int gx = wrap(x0 + q % PW - 2, Lx), gt = wrap(t0 + q / PW - 2, Lt);
    sp[q] = ld_spinor(in + off + 2LL * (gx + Lx * gt));
  }
  for (int q = tid; q < UH * UW; q += TX * TY) {
    const int gx = wrap(x0 + q % UW - 2, Lx), gt = wrap(t0 + q / UW - 2, Lt);
    const int g = gx + Lx * gt;
    su[q][0] = U[g];
    su[q][1] = U[V + g];
  }
  __syncthreads();
  // D psi on [-1, TX] x [-1, TT]
  for (int q = tid; q < DH * DW; q += TX * TY) {
    const int lx = q % DW - 1, lt = q / DW - 1;
    const int pc = (lt + 2) * PW + (lx + 2);
    const int uc = (lt + 2) * UW + (lx + 2);
    C a0 = mk((R)0, (R)0), a1 = mk((R)0, (R)0), f0, f1;
    split(sp[pc + 1], f0, f1);
    hop_x<R>(a0, a1, su[uc][0], f0, f1, (R)1);
    split(sp[pc - 1], f0, f1);
    hop_x<R>(a0, a1, cconj(su[uc - 1][0]), f0, f1, (R)-1);
    split(sp[pc + PW], f0, f1);
    hop_t<R>(a0, a1, su[uc][1], f0, f1, (R)1);
    split(sp[pc - PW], f0, f1);
    hop_t<R>(a0, a1, cconj(su[uc - UW][1]), f0, f1, (R)-1);
    split(sp[pc], f0, f1);
    sd[q] = join(mk(diag * f0.x - (R)0.5 * a0.x, diag * f0.y - (R)0.5 * a0.y),
                 mk(diag * f1.x - (R)0.5 * a1.x, diag * f1.y - (R)0.5 * a1.y));
  }
  __syncthreads();
  // D^dagger on the tile, then the epilogue
  const int lx = tid % TX;
  const int gx = x0 + lx;
  const R ca = (R)ep.ca, cu = (R)ep.cu, cw = (R)ep.cw;
  const C* EU = (const C*)ep.U;
  const C* EW = (const C*)ep.W;
  R dre = (R)0, dim = (R)0;     // per-thread partials in the stencil's precision
  double zq = 0.0, rz = 0.0;     // the flexible-CG pair (FP64 operands)
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int lt = tid / TX + TY * k;
    const int gt = t0 + lt;
    if (gx >= Lx || gt >= Lt) continue;
    const int dc = (lt + 1) * DW + (lx + 1);
    const int uc = (lt + 2) * UW + (lx + 2);
    C a0 = mk((R)0, (R)0), a1 = mk((R)0, (R)0), f0, f1;
    split(sd[dc + 1], f0, f1);
    hop_x<R>(a0, a1, su[uc][0], f0, f1, (R)-1);
    split(sd[dc - 1], f0, f1);
    hop_x<R>(a0, a1, cconj(su[uc - 1][0]), f0, f1, (R)1);
    split(sd[dc + DW], f0, f1);
    hop_t<R>(a0, a1, su[uc][1], f0, f1, (R)-1);
    split(sd[dc - DW], f0, f1);
    hop_t<R>(a0, a1, cconj(su[uc - UW][1]), f0, f1, (R)1);
    split(sd[dc], f0, f1);
    C y0 = mk(diag * f0.x - (R)0.5 * a0.x, diag * f0.y - (R)0.5 * a0.y);
    C y1 = mk(diag * f1.x - (R)0.5 * a1.x, diag * f1.y - (R)0.5 * a1.y);
    const long long g = off + 2LL * (gx + Lx * gt);
    if (ep.dot_out && !ep.zq_q) {
      C p0, p1;
      split(sp[(lt + 2) * PW + (lx + 2)], p0, p1);
      dre += p0.x * y0.x + p0.y * y0.y + p1.x * y1.x + p1.y * y1.y;
      dim += p0.x * y0.y - p0.y * y0.x + p1.x * y1.y - p1.y * y1.x;
    }
    y0 = mk(ca * y0.x, ca * y0.y);
    y1 = mk(ca * y1.x, ca * y1.y);
    if (EU) {
      const S u = ld_spinor(EU + g);
      C u0, u1;
      split(u, u0, u1);
      y0 = mk(y0.x + cu * u0.x, y0.y + cu * u0.y);
      y1 = mk(y1.x + cu * u1.x, y1.y + cu * u1.y);
    }
    if (EW) {
      const S w = ld_spinor(EW + g);
      C w0, w1;
      split(w, w0, w1);
      y0 = mk(y0.x + cw * w0.x, y0.y + cw * w0.y);
      y1 = mk(y1.x + cw * w1.x, y1.y + cw * w1.y);
    }
    if (ep.zq_q) {
      const double2* Q = (const double2*)ep.zq_q + g;
      const double2* Rv = (const double2*)ep.zq_r + g;
      const double2 q0 = Q[0], q1 = Q[1], r0 = Rv[0], r1 = Rv[1];
      zq += (double)y0.x * q0.x + (double)y0.y * q0.y + (double)y1.x * q1.x + (double)y1.y * q1.y;
      rz += r0.x * (double)y0.x + r0.y * (double)y0.y + r1.x * (double)y1.x + r1.y * (double)y1.y;
    }
    st_spinor(out + g, join(y0, y1));
  }
  if (ep.dot_out) {
    __shared__ double sh[64];
    if (ep.zq_q) {
      finish_reduction_g(zq, rz, ep.dot_ws, ep.dot_out, sh, blockIdx.z,
                         blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
      return;
    }
    finish_reduction_g((double)dre, (double)dim, ep.dot_ws, ep.dot_out, sh, blockIdx.z,
                       blockIdx.y * gridDim.x + blockIdx.x, gridDim.x * gridDim.y);
  }
}

// Register-streaming A = D^dagger D for large lattices.  A warp owns a strip
// of 32 consecutive x sites (lanes 2..29 produce output, lanes 0, 1, 30, 31
// are halo) and marches along t over SROWS output rows, keeping three rows of
// psi, two rows of D psi and the needed link rows in registers; x neighbours
// come from warp shuffles, t neighbours from the row window.  No shared
// memory and no block barriers: every loaded byte is used from registers.
// Row r + 2 of psi and the links of row r + 1 are prefetched one step ahead.
static constexpr int SROWS = 32;
static constexpr int SOUT = 28;            // output lanes per warp

template <typename C>
__device__ __forceinline__ C shfl_c(C v, int delta, bool up) {
  C r;
  if (up) {
    r.x = __shfl_up_sync(0xffffffffu, v.x, delta);
    r.y = __shfl_up_sync(0xffffffffu, v.y, delta);
  } else {
    r.x = __shfl_down_sync(0xffffffffu, v.x, delta);
    r.y = __shfl_down_sync(0xffffffffu, v.y, delta);
  }
  return r;
}

// D (sf = +1) or D^dagger (sf = -1) at this lane's site for one row: (f0, f1)
// the row's spinor, fu / fd the rows t+1 / t-1 at this x, ux and ut the links
// here, utm the t link one row below; the x-hop terms come from the adjacent
// lanes.
template <typename R>
__device__ __forceinline__ void dslash_row(cplx_t<R> f0, cplx_t<R> f1, cplx_t<R> fu0,
                                           cplx_t<R> fu1, cplx_t<R> fd0, cplx_t<R> fd1,
                                           cplx_t<R> ux, cplx_t<R> ut, cplx_t<R> utm, R diag,
                                           R sf, cplx_t<R>& o0, cplx_t<R>& o1) {
  using C = cplx_t<R>;
  // x hops: each lane forms the projections of its own site and the lane
  // x - 1 also applies its link, so only one complex per direction moves.
  const C q = mk(f0.x - sf * f1.x, f0.y - sf * f1.y);               // (1 - sf s1) projection
  const C g = cmul(cconj(ux), mk(f0.x + sf * f1.x, f0.y + sf * f1.y));
  const C qn = shfl_c(q, 1, false);                                 // from x + 1
  const C gp = shfl_c(g, 1, true);                                  // U_x(x-1)^* (...)(x - 1)
  const C hf = cmul(ux, qn);
  C a0 = cadd(hf, gp);
  C a1 = mk(-sf * hf.x + sf * gp.x, -sf * hf.y + sf * gp.y);
  hop_t<R>(a0, a1, ut, fu0, fu1, sf);
  hop_t<R>(a0, a1, cconj(utm), fd0, fd1, -sf);
  o0 = mk(diag * f0.x - (R)0.5 * a0.x, diag * f0.y - (R)0.5 * a0.y);
  o1 = mk(diag * f1.x - (R)0.5 * a1.x, diag * f1.y - (R)0.5 * a1.y);
}

// Asynchronous row prefetch for the streaming stencil: each lane copies its
// own spinor and links of a future row into a per-warp ring of SNB slots in
// shared memory (cp.async), SNB - 1 iterations ahead of use.
static constexpr int SNB = 4;

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 7 : 3) k_wilson_A_stream(
    const cplx_t<R>* __restrict__ in, cplx_t<R>* out, const cplx_t<R>* __restrict__ U, R diag,
    int Lx, int Lt, Epilogue ep) {
  using C = cplx_t<R>;
  using S = typename spinor_t<R>::type;
  __shared__ S ring_psi[4][SNB][32];           // [warp][slot][lane]
  __shared__ C ring_u[4][SNB][32][2];
  const int V = Lx * Lt;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int strips = (Lx + SOUT - 1) / SOUT;
  const int w = blockIdx.x * (blockDim.x >> 5) + wl;
  const int row_blocks = (Lt + SROWS - 1) / SROWS;
  if (w >= strips * row_blocks) return;                  // whole warp
  const int strip = w % strips, t0 = (w / strips) * SROWS;
  const int xu = strip * SOUT - 2 + lane;                // unwrapped x
  const int x = wrap(xu, Lx);
  const bool writer = lane >= 2 && lane < 30 && xu < Lx;
  const long long off = (long long)blockIdx.y * V * 2;
  const int t1 = min(t0 + SROWS, Lt);                    // output rows [t0, t1)
  auto ld_psi = [&](int t, C& a, C& b) {
    split(ld_spinor(in + off + 2LL * (x + Lx * wrap(t, Lt))), a, b);
  };
  auto ld_u = [&](int t, C& ux, C& ut) {
    const int g = x + Lx * wrap(t, Lt);
    ux = U[g];
    ut = U[V + g];
  };
  // group for loop step r: psi(r + 2) and links(r + 1), into slot
  // (r - t0 + 1) mod SNB; empty past the last step that reads one
  auto issue = [&](int r) {
    if (r < t1) {
      const int slot = (r - t0 + 1 + SNB) % SNB;
      const C* ps = in + off + 2LL * (x + Lx * wrap(r + 2, Lt));
      char* dst = (char*)&ring_psi[wl][slot][lane];
      if (sizeof(S) == 16) {
        cp_async(dst, ps, 16);
      } else {
        cp_async(dst, ps, 16);
        cp_async(dst + 16, ps + 1, 16);
      }
      const int g = x + Lx * wrap(r + 1, Lt);
      cp_async(&ring_u[wl][slot][lane][0], U + g, (int)sizeof(C));
      cp_async(&ring_u[wl][slot][lane][1], U + V + g, (int)sizeof(C));
    }
    cp_commit();
  };
  C pm0, pm1, pc0, pc1, pp0, pp1;          // psi rows r-1, r, r+1
  C dm0, dm1, dc0, dc1;                    // D psi rows r-2, r-1
  C uxc, utc, utm;                         // U_x(r), U_t(r), U_t(r-1)
  C uxo, uto, utmo;                        // the same one row earlier (for D^dagger)
  C dummy;
  ld_psi(t0 - 2, pm0, pm1);
  ld_psi(t0 - 1, pc0, pc1);
  ld_psi(t0, pp0, pp1);
  ld_u(t0 - 2, dummy, utm);
  ld_u(t0 - 1, uxc, utc);
  for (int k = 0; k < SNB - 1; ++k) issue(t0 - 1 + k);
  dm0 = dm1 = dc0 = dc1 = mk((R)0, (R)0);
  uxo = uto = utmo = mk((R)0, (R)0);
  const R ca = (R)ep.ca, cu = (R)ep.cu, cw = (R)ep.cw;
  const C* EU = (const C*)ep.U;
  const C* EW = (const C*)ep.W;
  for (int r = t0 - 1; r <= t1; ++r) {
    C e0, e1;                                            // D psi at row r
    dslash_row<R>(pc0, pc1, pp0, pp1, pm0, pm1, uxc, utc, utm, diag, (R)1, e0, e1);
    if (r >= t0 + 1) {                                   // output row r - 1
      C o0, o1;
      dslash_row<R>(dc0, dc1, e0, e1, dm0, dm1, uxo, uto, utmo, diag, (R)-1, o0, o1);
      if (writer) {
        const long long g = off + 2LL * (x + Lx * (r - 1));
        o0 = mk(ca * o0.x, ca * o0.y);
        o1 = mk(ca * o1.x, ca * o1.y);
        if (EU) {
          C u0, u1;
          split(ld_spinor(EU + g), u0, u1);
          o0 = mk(o0.x + cu * u0.x, o0.y + cu * u0.y);
          o1 = mk(o1.x + cu * u1.x, o1.y + cu * u1.y);
        }
        if (EW) {
          C w0, w1;
          split(ld_spinor(EW + g), w0, w1);
          o0 = mk(o0.x + cw * w0.x, o0.y + cw * w0.y);
          o1 = mk(o1.x + cw * w1.x, o1.y + cw * w1.y);
        }
        st_spinor(out + g, join(o0, o1));
      }
    }
    dm0 = dc0; dm1 = dc1; dc0 = e0; dc1 = e1;            // shift: row r becomes r - 1
    uxo = uxc; uto = utc; utmo = utm;
    pm0 = pc0; pm1 = pc1; pc0 = pp0; pc1 = pp1;
    utm = utc;
    if (r + 1 <= t1) {                                   // psi(r + 2), links(r + 1)
      cp_wait<SNB - 2>();
      const int slot = (r - t0 + 1 + SNB) % SNB;
      split(ring_psi[wl][slot][lane], pp0, pp1);
      uxc = ring_u[wl][slot][lane][0];
      utc = ring_u[wl][slot][lane][1];
    }
    issue(r + SNB - 1);
  }
  cp_wait<0>();
}

// The streaming kernel serves lattices with enough strips to fill the GPU.
bool wilson_A_streamed(int Lx, int Lt) {
  const long long warps = (long long)((Lx + SOUT - 1) / SOUT) * ((Lt + SROWS - 1) / SROWS);
  return Lx >= 64 && Lt >= 2 * SROWS && warps >= 4LL * 152;
}

// Tile choice of the fused kernel: 32 x 8 (FP64) or 32 x 16 (FP32) when that
// gives two CTAs per SM, else 16 x 8 (smaller tiles measured slower: more halo).
int wilson_A_ctas(int Lx, int Lt, bool f64) {
  const int big = ((Lx + 31) / 32) * ((Lt + (f64 ? 7 : 15)) / (f64 ? 8 : 16));
  if (big >= 2 * 152) return big;
  return ((Lx + 15) / 16) * ((Lt + 7) / 8);
}

template <typename R, int TX, int TY, int RPT>
static void launch_wilson_A(const void* in, void* out, const void* U, double diag, int Lx, int Lt,
                            int nrhs, const Epilogue& ep, cudaStream_t s) {
  static_assert(sizeof(R) * 4 * ((TY * RPT + 4) * (TX + 4) + (TY * RPT + 2) * (TX + 2)) +
                        sizeof(R) * 4 * (TY * RPT + 3) * (TX + 3) <= 48 * 1024,
                "tile above the static shared-memory limit");
  dim3 grid((Lx + TX - 1) / TX, (Lt + TY * RPT - 1) / (TY * RPT), nrhs);
  k_wilson_A<R, TX, TY, RPT><<<grid, TX * TY, 0, s>>>((const cplx_t<R>*)in, (cplx_t<R>*)out,
                                                      (const cplx_t<R>*)U, (R)diag, Lx, Lt, ep);
}

// ---------------------------------------------------------------------------
// Launch shapes of the fused A and their autotuner.  Every shape runs the same
// per-site arithmetic (wilson_site order), so a shape is admitted by the
// tuner only if it reproduces the default shape's output bit for bit; the
// tuner then keeps the fastest admitted shape per (precision, Lx, Lt, nrhs)
// when it beats the default shape by more than 3%.
// Launches with the fused <in, A in> epilogue keep the default shape (their
// partial sums depend on the tiling).
// ---------------------------------------------------------------------------
enum { WV_STREAM = 0, WV_16x8, WV_32x8, WV_32x8x2, WV_16x16, WV_64x4, WV_64x4x2, WV_COUNT };
static const int WV_SHAPE[WV_COUNT][3] = {{0, 0, 0}, {16, 8, 1}, {32, 8, 1}, {32, 8, 2},
                                          {16, 16, 1}, {64, 4, 1}, {64, 4, 2}};

// The default shape (the choice made before any tuning).
template <typename R>
static int wilson_default_variant(int Lx, int Lt, bool dot) {
  const bool f64 = sizeof(R) == 8;
  if (!dot && wilson_A_streamed(Lx, Lt)) return WV_STREAM;
  const bool big = ((Lx + 31) / 32) * ((Lt + (f64 ? 7 : 15)) / (f64 ? 8 : 16)) >= 2 * 152;
  if (!big) return WV_16x8;
  return f64 ? WV_32x8 : WV_32x8x2;
}

template <typename R>
static bool wilson_variant_ok(int v, int Lx, int Lt) {
  if (v == WV_STREAM) return wilson_A_streamed(Lx, Lt);
  if (sizeof(R) == 8 && (v == WV_32x8x2 || v == WV_64x4x2)) return false;   // shared memory
  return true;
}

template <typename R>
static void launch_variant(int v, const void* in, void* out, const void* U, double diag, int Lx,
                           int Lt, int nrhs, const Epilogue& ep, cudaStream_t s) {
  switch (v) {
    case WV_STREAM: {
      const long long warps = (long long)((Lx + SOUT - 1) / SOUT) * ((Lt + SROWS - 1) / SROWS);
      k_wilson_A_stream<R><<<dim3((unsigned)((warps + 3) / 4), nrhs), 128, 0, s>>>(
          (const cplx_t<R>*)in, (cplx_t<R>*)out, (const cplx_t<R>*)U, (R)diag, Lx, Lt, ep);
      break;
    }
    case WV_16x8: launch_wilson_A<R, 16, 8, 1>(in, out, U, diag, Lx, Lt, nrhs, ep, s); break;
    case WV_32x8: launch_wilson_A<R, 32, 8, 1>(in, out, U, diag, Lx, Lt, nrhs, ep, s); break;
    case WV_16x16: launch_wilson_A<R, 16, 16, 1>(in, out, U, diag, Lx, Lt, nrhs, ep, s); break;
    case WV_64x4: launch_wilson_A<R, 64, 4, 1>(in, out, U, diag, Lx, Lt, nrhs, ep, s); break;
    default:
      if constexpr (sizeof(R) == 4) {
        if (v == WV_32x8x2) launch_wilson_A<R, 32, 8, 2>(in, out, U, diag, Lx, Lt, nrhs, ep, s);
        else launch_wilson_A<R, 64, 4, 2>(in, out, U, diag, Lx, Lt, nrhs, ep, s);
      }
      break;
  }
}

struct TuneKey {
  int prec, Lx, Lt, nrhs;
  bool operator<(const TuneKey& o) const {
    return std::tie(prec, Lx, Lt, nrhs) < std::tie(o.prec, o.Lx, o.Lt, o.nrhs);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, StencilTuning> g_tune;

template <typename R>
static int tuned_variant(int Lx, int Lt, int nrhs) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find({(int)sizeof(R), Lx, Lt, nrhs});
  return it == g_tune.end() ? -1 : it->second.variant;
}

__global__ void k_count_diff(const unsigned long long* __restrict__ a,
                             const unsigned long long* __restrict__ b, long long n, int* diff) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (a[i] != b[i]) atomicAdd(diff, 1);
}

template <typename R>
cudaError_t wilson_A_tune(const void* in, void* out, void* ref, const void* U, double diag,
                          int Lx, int Lt, int nrhs, int* dflag, cudaStream_t s) {
  const TuneKey key{(int)sizeof(R), Lx, Lt, nrhs};
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    if (g_tune.count(key)) return cudaSuccess;
  }
  const Epilogue none{};
  const int def = wilson_default_variant<R>(Lx, Lt, false);
  const long long words = (long long)Lx * Lt * nrhs * 2 * sizeof(cplx_t<R>) / 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  StencilTuning t{};
  t.precision = sizeof(R) == 8 ? 0 : 1;
  t.Lx = Lx; t.Lt = Lt; t.nrhs = nrhs;
  t.variant = def;
  float best = 0.f;
  launch_variant<R>(def, in, ref, U, diag, Lx, Lt, nrhs, none, s);
  for (int v = 0; v < WV_COUNT; ++v) {
    if (!wilson_variant_ok<R>(v, Lx, Lt)) continue;
    ++t.tried;
    launch_variant<R>(v, in, out, U, diag, Lx, Lt, nrhs, none, s);
    int diff = 0;
    cudaMemsetAsync(dflag, 0, sizeof(int), s);
    k_count_diff<<<152, 256, 0, s>>>((const unsigned long long*)out,
                                     (const unsigned long long*)ref, words, dflag);
    cudaMemcpyAsync(&diff, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return err;
    }
    if (diff) continue;                                    // not bit-identical: never used
    ++t.admitted;
    for (int w = 0; w < 2; ++w) launch_variant<R>(v, in, out, U, diag, Lx, Lt, nrhs, none, s);
    constexpr int REPS = 10;
    cudaEventRecord(e0, s);
    for (int w = 0; w < REPS; ++w) launch_variant<R>(v, in, out, U, diag, Lx, Lt, nrhs, none, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = 1000.0 * ms / REPS;
    if (v == def) t.us_default = us;
    if (t.admitted == 1 || ms < best) {
      best = ms;
      t.variant = v;
      t.us_best = us;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // a timing difference inside the noise of isolated launches does not carry
  // over to launches inside a solve: keep the default unless 3% faster
  if (t.variant != def && !(t.us_best < 0.97 * t.us_default)) {
    t.variant = def;
    t.us_best = t.us_default;
  }
  t.tx = WV_SHAPE[t.variant][0];
  t.ty = WV_SHAPE[t.variant][1];
  t.rpt = WV_SHAPE[t.variant][2];
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = t;
  }
  return cudaGetLastError();
}

int stencil_tunings(StencilTuning* out, int max) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  int k = 0;
  for (const auto& kv : g_tune) {
    if (k < max && out) out[k] = kv.second;
    ++k;
  }
  return k;
}

template <typename R>
cudaError_t wilson_A(const void* in, void* out, const void* U, double diag, int Lx, int Lt,
                     int nrhs, const Epilogue& ep, cudaStream_t s) {
  const bool dot = ep.dot_out != nullptr;
  if (dot && (nrhs > 64 || wilson_A_ctas(Lx, Lt, sizeof(R) == 8) > 608)) return cudaErrorInvalidValue;
  int v = dot ? -1 : tuned_variant<R>(Lx, Lt, nrhs);
  if (v < 0) v = wilson_default_variant<R>(Lx, Lt, dot);
  launch_variant<R>(v, in, out, U, diag, Lx, Lt, nrhs, ep, s);
  count_launch();
  return cudaGetLastError();
}

// out = sigma_3 in on V two-spinors (FP64): spin component 1 negated.
__global__ void k_sigma3(const double2* __restrict__ in, double2* out, long long V) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double2 a = in[2 * i], b = in[2 * i + 1];
  out[2 * i] = a;
  out[2 * i + 1] = make_double2(-b.x, -b.y);
}

cudaError_t sigma3_mul(const void* in, void* out, long long V, cudaStream_t s) {
  k_sigma3<<<(unsigned)((V + 255) / 256), 256, 0, s>>>((const double2*)in, (double2*)out, V);
  count_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void k_fold_links(const double2* __restrict__ g, cplx_t<R>* __restrict__ U, int Lx,
                             int Lt) {
  const int V = Lx * Lt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * V) return;
  const int mu = i / V, site = i % V;
  const double sg = (mu == 1 && site / Lx == Lt - 1) ? -1.0 : 1.0;
  double2 u = g[i];
  U[i] = mk((R)(sg * u.x), (R)(sg * u.y));
}

template <typename R>
cudaError_t fold_links(const void* gauge, void* U, int Lx, int Lt, cudaStream_t s) {
  const int n = 2 * Lx * Lt;
  k_fold_links<R><<<(n + 255) / 256, 256, 0, s>>>((const double2*)gauge, (cplx_t<R>*)U, Lx, Lt); count_launch();
  return cudaGetLastError();
}

__global__ void k_link_unitarity(const double2* __restrict__ g, long long count, double* out) {
  double m = 0.0;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) {
    double2 u = g[i];
    double d = fabs(sqrt(u.x * u.x + u.y * u.y) - 1.0);
    m = (d > m || d != d) ? d : m;   // NaN propagates
  }
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_down_sync(0xffffffffu, m, o);
    m = (v > m || v != v) ? v : m;
  }
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = (sh[w] > r || sh[w] != sh[w]) ? sh[w] : r;
    *out = r;
  }
}

cudaError_t link_unitarity(const void* gauge, long long count, double* out, cudaStream_t s) {
  k_link_unitarity<<<1, 1024, 0, s>>>((const double2*)gauge, count, out); count_launch();
  return cudaGetLastError();
}

#define INST(R)                                                                               \
  template cudaError_t wilson_D<R>(const void*, void*, const void*, double, int, int, int,    \
                                   bool, cudaStream_t);                                       \
  template cudaError_t wilson_A<R>(const void*, void*, const void*, double, int, int, int,    \
                                   const Epilogue&, cudaStream_t);                            \
  template cudaError_t wilson_A_tune<R>(const void*, void*, void*, const void*, double, int,   \
                                        int, int, int*, cudaStream_t);                        \
  template cudaError_t fold_links<R>(const void*, void*, int, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace mgk
