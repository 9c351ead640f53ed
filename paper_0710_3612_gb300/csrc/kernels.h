// Host-side launchers of the CUDA kernels (one declaration per kernel family).
// Vectors are [nrhs][count] complex arrays (count = sites * dof), precision R
// (double -> complex128, float -> complex64).  Every launcher enqueues on the
// given stream and returns the launch error.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mgk {

// Kernel launches made by this library so far (counted at every launch site).
unsigned long long launch_count();
void count_launch();
// Adjusts the count (kernels recorded into a graph run later, once per replay).
void add_launches(long long n);

// ---- deterministic reductions -------------------------------------------
// Number of partial sums a reduction over `count` complex entries produces.
int reduce_blocks(long long count);
// Reductions take a workspace ws of (64 + 2 * 608 * nrhs) doubles whose first
// 64 doubles (tickets) are zero before the first call (they are left zero);
// nrhs <= 64.  One launch: the last block adds the partials in fixed order.

// out[rhs] (double2) = sum conj(a) b.
template <typename R>
cudaError_t dot(const void* a, const void* b, long long count, int nrhs, double* partials,
                double* out, cudaStream_t s);
// out[rhs] = sum |a|^2 (stored as double2 {norm2, 0}).
template <typename R>
cudaError_t norm2(const void* a, long long count, int nrhs, double* partials, double* out,
                  cudaStream_t s);

// ---- BLAS-1 --------------------------------------------------------------
// y = a x + b y (host real scalars).
template <typename R>
cudaError_t axpby(double a, const void* x, double b, void* y, long long count, int nrhs,
                  cudaStream_t s);
// y = x * (1 / sqrt(nrm[rhs].x))  (power iteration normalisation)
template <typename R>
cudaError_t scale_inv_sqrt(const void* x, void* y, const double* nrm, long long count, int nrhs,
                           cudaStream_t s);
// Loop control of k_cg_control run by cg_xr itself (graph loops): the block
// that completes the last right-hand side's |r|^2 takes the decisions; tick is
// one unsigned, zero between launches.
struct CgControl {
  int* ctrl = nullptr;
  const double* stop = nullptr;
  unsigned* tick = nullptr;
  cudaGraphConditionalHandle cond = 0;
};
// CG step on per-RHS device scalars (double2 arrays, real part used):
//   alpha = rz / pq (0 when frozen[rhs]); x += alpha p; r -= alpha q;
//   rr[rhs] = |r|^2 (one launch, reduction workspace ws); cc: see CgControl.
template <typename R>
cudaError_t cg_xr(void* x, void* r, const void* p, const void* q, const double* rz,
                  const double* pq, const int* frozen, long long count, int nrhs, double* ws,
                  double* rr, cudaStream_t s, void* r32 = nullptr,
                  const CgControl* cc = nullptr);
//   beta = rz_new / rz_old; p = z + beta p; then rz_old <- rz_new is done by the caller.
template <typename R>
cudaError_t cg_p(void* p, const void* z, const double* rz_new, const double* rz_old,
                 const int* frozen, long long count, int nrhs, cudaStream_t s);
// Graph-resident CG loop control for nrhs right-hand sides (nrhs <= 64):
// ctrl = {iterations, status, limit, nrhs, frozen[nrhs], it_done[nrhs]};
// status 0 running, 1 all converged, 2 breakdown, 3 limit reached.
cudaError_t cg_control(const double* rr, const double* pq, const double* stop, int* ctrl,
                       cudaGraphConditionalHandle cond, cudaStream_t s);
// ctrl init and stop[rhs] = tol2 * bn[rhs] (double2 slots); b = 0 starts frozen.
cudaError_t set_control(int* ctrl, int maxiter, int nrhs, const double* bn, double tol2,
                        double* stop, cudaStream_t s);
// Flexible CG (FP64 vectors, FP32 preconditioned residual z32) per rhs:
// zr = {Re<z32, q>, Re<r, z32>} (one launch), then beta = -zr[0] / Re(pq),
// p = z32 + beta p, and rz <- zr[1] for the next step length.
cudaError_t dot2_zq_rz(const void* z32, const void* q, const void* r, long long count, int nrhs,
                       double* ws, double* zr, cudaStream_t s);
cudaError_t cg_p_pr(void* p, const void* z32, const double* zr, const double* pq, double* rz,
                    const int* frozen, long long count, int nrhs, cudaStream_t s);
// Reliable-update flexible CG: every vector of the iteration in FP32 (per-
// thread FP32 partial sums, FP64 across blocks); the solution increment x32
// and the true residual are carried over to FP64 by ru_fold / ru_residual.
cudaError_t rdot(const void* a, const void* b, long long count, int nrhs, double* ws, double* out,
                 cudaStream_t s);
cudaError_t rcg_xr(void* x32, void* r32, const void* p32, const void* q32, const double* rz,
                   const double* pq, const int* frozen, long long count, int nrhs, double* ws,
                   double* rr, cudaStream_t s);
cudaError_t rdot2_zq_rz(const void* z32, const void* q32, const void* r32, long long count,
                        int nrhs, double* ws, double* zr, cudaStream_t s);
cudaError_t rcg_p(void* p32, const void* z32, const double* zr, const double* pq, double* rz,
                  const int* frozen, long long count, int nrhs, cudaStream_t s);
// rmax = max(rmax, rr) over running right-hand sides; *due = some rr < delta2 rmax
// (then ++*count); with cond_set the IF condition of the graph node follows *due.
cudaError_t ru_check(const double* rr, double* rmax, const int* ctrl, double delta2, int* due,
                     int* count, cudaGraphConditionalHandle cond, bool cond_set, cudaStream_t s);
// x64 += x32 and x32 = 0 over count entries.
cudaError_t ru_fold(void* x64, void* x32, long long count, cudaStream_t s);
// r32 = (float) r64, rr = |r64|^2 per rhs, and rmax = rr when rmax is given.
cudaError_t ru_residual(const void* r64, void* r32, long long count, int nrhs, double* ws,
                        double* rr, double* rmax, cudaStream_t s);
// out(FP32) = in(FP64) * (1/sqrt(nrm[rhs].x)) ; in==0 norm -> 0.
cudaError_t f64_to_f32_scaled(const void* in, void* out, const double* nrm, long long count,
                              int nrhs, cudaStream_t s);
// x(FP64) += in(FP32) * sqrt(nrm[rhs].x)   (scale 1 when nrm is null)
cudaError_t f32_accumulate_scaled(const void* in, void* x, const double* nrm, long long count,
                                  int nrhs, cudaStream_t s);
// out = in (precision convert, no scaling)
cudaError_t convert_f64_f32(const void* in, void* out, long long count, cudaStream_t s);
cudaError_t convert_f32_f64(const void* in, void* out, long long count, cudaStream_t s);
// out = a u + b v (+ c w when w != nullptr); out may alias u, v or w.
template <typename R>
cudaError_t lincomb(void* out, double a, const void* u, double b, const void* v, double c,
                    const void* w, long long count, int nrhs, cudaStream_t s);
// r = b - r  (in place: r holds A x on entry)
template <typename R>
cudaError_t sub_from(const void* b, void* r, long long count, cudaStream_t s);

// ---- fused epilogue of the operator kernels -------------------------------
// out = ca * (Op x) + cu * U + cw * W (U, W optional, same precision and layout
// as out; out may alias W).  When dot_out is set (fine A only, one RHS), the
// kernel also forms <x, Op x> (double2, deterministic, workspace dot_ws as
// for the reductions).
struct Epilogue {
  double ca = 1.0, cu = 0.0, cw = 0.0;
  const void* U = nullptr;
  const void* W = nullptr;
  double* dot_ws = nullptr;
  double* dot_out = nullptr;     // <in, out> per rhs (fine stencil; needs <= 608 blocks)
  // with dot_out, instead of <in, out>: {Re<out, zq_q>, Re<zq_r, out>} per rhs,
  // zq_q and zq_r complex128 vectors shaped like out (the flexible-CG pair)
  const void* zq_q = nullptr;
  const void* zq_r = nullptr;
};

// ---- fine Wilson operator ------------------------------------------------
// U: [2][V] complex of precision R with the antiperiodic sign folded into the
// t links at t = Lt - 1.  diag = 4 + m.
template <typename R>
cudaError_t wilson_D(const void* in, void* out, const void* U, double diag, int Lx, int Lt,
                     int nrhs, bool dagger, cudaStream_t s);
template <typename R>
cudaError_t wilson_A(const void* in, void* out, const void* U, double diag, int Lx, int Lt,
                     int nrhs, const Epilogue& ep, cudaStream_t s);

// out = sigma_3 in for V fine two-spinors (FP64); out may alias in.
cudaError_t sigma3_mul(const void* in, void* out, long long V, cudaStream_t s);

// Launch shape chosen by the autotuner for one (precision, Lx, Lt, nrhs):
// tile tx x ty with rpt rows per thread (0 x 0: the streaming kernel), timed
// against the default shape; only shapes whose output is bit-identical to
// the default's are admitted.
struct StencilTuning {
  int precision;        // 0 = FP64, 1 = FP32
  int Lx, Lt, nrhs;
  int variant, tx, ty, rpt;
  int tried, admitted;
  double us_best, us_default;
};
// Times every launch shape of the fused A on (in, U) once per process and
// shape, writing into out and ref (nrhs fine vectors each) and using dflag (one
// device int); later wilson_A launches without the dot epilogue use the
// fastest admitted shape.
template <typename R>
cudaError_t wilson_A_tune(const void* in, void* out, void* ref, const void* U, double diag,
                          int Lx, int Lt, int nrhs, int* dflag, cudaStream_t s);
// Copies up to max tuned shapes into out; returns how many exist.
int stencil_tunings(StencilTuning* out, int max);
// Thread blocks wilson_A launches per right-hand side (the fused <x, A x>
// needs at most 608).
int wilson_A_ctas(int Lx, int Lt, bool f64);
// links: gauge complex128 [2][V] -> folded links of precision R
template <typename R>
cudaError_t fold_links(const void* gauge, void* U, int Lx, int Lt, cudaStream_t s);
// max_i ||U_i| - 1| into *out (device double), single block reduction
cudaError_t link_unitarity(const void* gauge, long long count, double* out, cudaStream_t s);

// ---- coarse operator -----------------------------------------------------
// y(j) = sum_d A[j][d] x(j + d); A element type: double2 (R=double), float2
// (R=float, W=float) or bf16x2 (R=float, W=bf16).
enum CoarseWeights { W_F64 = 0, W_F32 = 1, W_BF16 = 2 };
cudaError_t coarse_apply(const void* in, void* out, const void* A, int weights, int Lx, int Lt,
                         int n, int nrhs, const Epilogue& ep, cudaStream_t s);
// Multi-RHS BF16 coarse apply on tcgen05 tensor cores (TMEM accumulator):
// n in {16, 24}, 1 <= nrhs <= 64, FP32 vectors [nrhs][V][n], bf16x2 blocks.
bool coarse_apply_tcgen05_ok(int n, int nrhs);
cudaError_t coarse_apply_tcgen05(const void* in, void* out, const void* A, int Lx, int Lt, int n,
                                 int nrhs, const Epilogue& ep, cudaStream_t s);
// Reads and clears the process-wide flag set when a bounded completion wait
// of the tcgen05 coarse apply ran out (its results are then invalid).
cudaError_t coarse_tc_take_error(int* flag);
// Tensor-core kernel of coarse_apply for BF16 blocks and >= 8 right-hand
// sides: 0 = tcgen05 where the shape allows it (default), 1 = mma.sync.
void set_coarse_tensor_kernel(int kind);
// A (complex128) -> float2 or bf16x2 copy
// out = a X + b Y + c I for coarse operators of `sites` sites and n dof (FP64).
cudaError_t coarse_lincomb(double a, const void* X, double b, const void* Y, double c, void* out,
                           long long sites, int n, cudaStream_t s);
cudaError_t coarse_convert(const void* A64, void* out, int weights, long long count,
                           cudaStream_t s);

// ---- column probing (smoothed Galerkin products) ---------------------------
// Probe vectors: out[s][j][r] = 1 if r == s and site j has colour (cx, ct) =
// (x mod Kx, t mod Kt), else 0 (nc vectors of Lxc x Ltc sites, nc dof,
// complex128).  Scatter: Ac[j][d][r][s] = y[s][j][r] for every site j and
// displacement d whose neighbour j + d has that colour (Ac complex128
// [Vc][9][nc][nc]).  With Kx, Kt >= 3 dividing the extents and an operator
// reaching one block, each entry is written by exactly one colour.
cudaError_t probe_vectors(void* out, int Lxc, int Ltc, int nc, int Kx, int Kt, int cx, int ct,
                          cudaStream_t s);
cudaError_t probe_scatter(const void* y, void* Ac, int Lxc, int Ltc, int nc, int Kx, int Kt, int cx,
                          int ct, cudaStream_t s);

// ---- transfer ------------------------------------------------------------
// Vst: [V_f][2][Nv][h] complex (h = n_f / 2), the per-site storage of P.
template <typename R>
cudaError_t restrict_op(const void* fine, void* coarse, const void* Vst, int Lx, int Lt, int bx,
                        int bt, int h, int Nv, int nrhs, cudaStream_t s);
template <typename R>
cudaError_t prolong_op(const void* coarse, void* fine, const void* Vst, int Lx, int Lt, int bx,
                       int bt, int h, int Nv, int nrhs, bool accumulate, cudaStream_t s);

// ---- setup ---------------------------------------------------------------
// Chirality-split block modified Gram-Schmidt (two passes) of Nv relaxed
// vectors E [Nv][V_f][n] (complex128) into Vst [V_f][2][Nv][h] (complex128).
// flag (device int) is set to 1 on breakdown.
cudaError_t block_gram_schmidt(const void* E, void* Vst, int Lx, int Lt, int bx, int bt, int h,
                               int Nv, double breakdown_tol, int* flag, cudaStream_t s);
// Level-1 Galerkin: W = D P on the extended blocks, then A_c = W^dagger W
// overlaps.  Wbuf: [Vc][2Nv][(bx+2)(bt+2)][2] complex128 scratch.
cudaError_t galerkin_fine(const void* U64, double diag, const void* Vst, void* Wbuf, void* Ac,
                          int Lx, int Lt, int bx, int bt, int Nv, cudaStream_t s);
// Level >= 2 Galerkin: A_{l+1}[j][d] = sum P(i)^dagger A_l[i][e] P(i+e).
cudaError_t galerkin_coarse(const void* Af, const void* Vst, void* Ac, int Lx, int Lt, int bx,
                            int bt, int nf, int Nv, cudaStream_t s);
// Dense coarsest matrix (complex64, row-major, leading dimension ld >= N) from
// the stencil (complex128); rows/columns N..ld-1 are set to the identity.
cudaError_t coarse_to_dense_f32(const void* A, void* dense, int Lx, int Lt, int n, long long ld,
                                cudaStream_t s);
// In-place blocked Gauss-Jordan inversion of a Hermitian positive definite
// complex64 N x N matrix (N multiple of 64), lower triangle kept (the upper
// halves of diagonal 64 x 64 tiles are rebuilt by pack_hermitian).
// work: 3 * N * 64 + 2 * 64 * 64 complex64.  Launch sequence: begin (inverts
// the first pivot block), then for k = 0 .. N/64 - 1: panel(k), update(k).
cudaError_t gauss_jordan_begin(void* M, int N, void* work, cudaStream_t s);
cudaError_t gauss_jordan_panel(void* M, int N, int k, void* work, cudaStream_t s);
cudaError_t gauss_jordan_update(void* M, int N, int k, void* work, cudaStream_t s);
// The same update on tcgen05 tensor cores (TMEM accumulator); needs 16 more
// bytes of work: an int error flag after the row panel, zero before the first
// call, set if a completion wait runs out (the inverse is then invalid).
cudaError_t gauss_jordan_update_tc(void* M, int N, int k, void* work, cudaStream_t s);
// y = B x, or y += B x when accumulate (complex64 B, leading dimension ld);
// x complex128 (N) -> y complex128 (N); FP32 products and accumulation, result
// widened to FP64.  xtmp: ld complex64.
cudaError_t dense_gemv_f32(const void* B, const void* x, void* y, int N, int ld, void* xtmp,
                           bool accumulate, cudaStream_t s);

// Packed Hermitian matrix: the lower-triangular 64 x 64 tiles (I >= J, stored
// at I (I + 1) / 2 + J) of a dense ld x ld complex64 matrix (ld multiple of
// 64); diagonal tiles are made Hermitian from their lower halves.
cudaError_t pack_hermitian(const void* M, void* P, int ld, cudaStream_t s);
// y = B x (or y += B x) with B Hermitian in packed tiles, for nrhs vectors;
// x, y complex128 [nrhs][N]; part: nrhs * 2 * 64 * ntiles complex64 scratch.
// FP32 products and accumulation; each tile is read once for all vectors.
cudaError_t hermitian_gemv_f32(const void* P, const void* x, void* y, int N, int ld, int nrhs,
                               void* part, bool accumulate, cudaStream_t s);
// The two launches of hermitian_gemv_f32: partial products per stored tile,
// then their fixed-order sum per row into y.
// xscratch (optional, nrhs * ld complex64): with 16..64 vectors the tile
// products run on tensor cores from an FP32 copy of x held there.
cudaError_t hermitian_gemv_tiles(const void* P, const void* x, int N, int ld, int nrhs,
                                 void* part, cudaStream_t s, void* xscratch = nullptr);
// hermitian_gemv_tiles for 1 to 4 vectors given in FP32 (x32, complex64
// [nrhs][N]); the diagonal tiles also write the exact FP64 copy of x32 into
// x64 (complex128 [nrhs][N]).
bool hermitian_gemv_f32in_ok(int nrhs);
cudaError_t hermitian_gemv_tiles_f32in(const void* P, const void* x32, int N, int ld, int nrhs,
                                       void* part, void* x64, cudaStream_t s);
// y32 (optional, complex64 [nrhs][N]) receives an FP32 copy of y.
cudaError_t hermitian_gemv_reduce(const void* part, void* y, int N, int ld, int nrhs,
                                  bool accumulate, cudaStream_t s, void* y32 = nullptr);

// index map for tests
cudaError_t block_map(int Lx, int Lt, int bx, int bt, int32_t* coarse, int32_t* offset,
                      cudaStream_t s);

// Checkerboard Metropolis sweeps first_sweep .. first_sweep + sweeps - 1 of the
// U(1) plaquette action on angles theta[2][Lt][Lx] (counter-based uniforms
// keyed by seed); accepted (device, may be NULL) accumulates the accepted
// proposals.  U = exp(i theta) for n angles.
cudaError_t gauge_metropolis(double* theta, int Lx, int Lt, double beta, double eps, int sweeps,
                             long long first_sweep, unsigned long long seed,
                             unsigned long long* accepted, cudaStream_t s);
cudaError_t links_from_angles(const double* theta, void* U, long long n, cudaStream_t s);

}  // namespace mgk
