// C ABI of the solver (declared in include/mg.h) and the host orchestration
// of the method: adaptive setup (Sec. 3), Galerkin hierarchy (Eq. Galerkin),
// frozen MR smoother (Sec. 4), five-step V-cycle (Sec. 2), MG-CG (Sec. 4).
// All arithmetic runs in the kernels of this library; the host only sequences
// launches and reads back the few scalars the Krylov loops branch on.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mg.h"
#include "kernels.h"

using namespace mgk;

namespace {

thread_local std::string g_last_error;

struct Level {
  int Lx = 0, Lt = 0, V = 0, n = 0;      // geometry; n = dof per site
  long long count() const { return (long long)V * n; }
  // operator blocks of this level (index >= 1): FP64 master, FP32, BF16 copies
  double2* A64 = nullptr;
  float2* A32 = nullptr;
  void* A16 = nullptr;
  double2* G0 = nullptr;                 // A(m) = G0 + m G1 + m^2 I (remass_quadratic)
  double2* G1 = nullptr;
  // transfer to the next level
  int bx = 0, bt = 0, Nv = 0;
  double2* Vst64 = nullptr;
  float2* Vst32 = nullptr;
  double c0 = 0, c1 = 0, lambda_max = 0, omega_relax = 0;
  double2* eta = nullptr;                // MR start vector (kept for re-massing)
  // V-cycle work vectors, [prec][4]: b (input copy for level > 0), x, r, t
  void* w64[4] = {nullptr, nullptr, nullptr, nullptr};
  void* w32[4] = {nullptr, nullptr, nullptr, nullptr};
};

}  // namespace

struct mg_handle {
  mg_params p{};
  cudaStream_t s = nullptr;
  double mass = 0.0;
  int L = 0;
  std::vector<Level> lv;
  double2* U64 = nullptr;
  float2* U32 = nullptr;
  // coarsest level
  int Nc = 0, ldc = 0;
  float2* Binv = nullptr;
  float2* gj_work = nullptr;
  float2* gemv_x = nullptr;
  float2* Bpk = nullptr;        // packed Hermitian tiles of the inverse
  float2* gemv_part = nullptr;  // partial products of the packed GEMV
  int n_refine = 0;
  int n_inner = 1;              // refinement steps of the FP32 V-cycle's coarsest solve
  bool inverse_ok = false;      // Binv / Bpk hold an FP32 inverse (of some mass)
  int inverse_reuses = 0;       // re-masses that kept the previous inverse
  double2 *cb = nullptr, *cx = nullptr, *cr = nullptr;   // coarsest FP64 scratch
  bool dense = true;            // dense inverse (else CG on the coarsest stencil)
  int ccg_iters = 0;            // CG iterations of one coarsest solve (fixed at set-up)
  double coarsest_test_res = 0; // worst relative residual of the set-up's test vectors
  double smooth = 0.0;          // omega of the smoothed first coarsening in use (0: off)
  double smooth_cond = 0.0;     // condition number of level 2 found by the omega search
  bool poisoned = false;        // a bounded device wait ran out: device state undefined
  double2 *cp = nullptr, *cq = nullptr;                  // coarsest CG vectors
  // CUDA graphs of the Krylov loop (one per preconditioner mode), launched on
  // the internal stream gs and fenced to the user's stream with events
  cudaStream_t gs = nullptr;
  cudaEvent_t fence[2] = {nullptr, nullptr};
  static constexpr int MAXR = 64;
  cudaGraphExec_t loop_exec[4 * MAXR] = {};     // per (preconditioner mode, nrhs)
  long long loop_kernels[4] = {0, 0, 0, 0};   // kernels per loop-body iteration
  long long ru_kernels = 0;                   // kernels of one reliable update
  int* ru = nullptr;            // reliable updates: {due, count since the loop started}
  unsigned* cg_tick = nullptr;  // ticket of the loop control fused into cg_xr
  int* dctrl = nullptr;         // loop control (see k_cg_control)
  int* hctrl = nullptr;         // pinned host mirror of dctrl
  int R = 1;                    // right-hand sides per batch (max_rhs)
  bool use_graphs = true;
  // solver vectors (one RHS), FP64 and FP32: x r p q z t
  void* sv64[6] = {};
  void* sv32[6] = {};
  // setup scratch
  void* Wbuf = nullptr;
  // scalars
  double* partials = nullptr;   // 2 * 608 * max_rhs doubles
  int partial_rhs = 0;
  double* scal = nullptr;       // device scalar slots (double2 each)
  double* hscal = nullptr;      // pinned host mirror
  int* dflag = nullptr;
  std::vector<void*> allocs;
  long long bytes = 0;          // device bytes currently allocated by the handle
  long long peak_bytes = 0;     // largest value of `bytes` so far
  bool dry = false;             // size-only pass: dalloc counts bytes, allocates nothing
  std::string err;
  long long fine_applies = 0, vcycles = 0;
  std::vector<double> refine_rho;   // rho of each adaptive pass made by mg_setup
  bool g_built = false;             // G0, G1 of every coarse level hold the current vectors
  // optional per-family event timing
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev[MG_KF_COUNT];
  size_t prof_used[MG_KF_COUNT] = {};
};

namespace {

// Largest coarsest level the dense inverse may take (FP32 N x N: 4.5 GiB).
constexpr long long MG_DENSE_MAX = 24576;

// scalar slots (each a double2)
// scalar slots: slot k holds one double2 per right-hand side
enum { S_RZ = 0, S_RZN, S_PQ, S_RR, S_T0, S_T1, S_BN, S_NR, S_STOP, S_CA, S_CB, S_CPQ, S_RMAX,
       S_COUNT };

struct Fail {
  mg_status st;
};

void fail(mg_handle* h, mg_status st, const std::string& msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  throw Fail{st};
}

void ck(mg_handle* h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(h, MG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T = void>
T* dalloc(mg_handle* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  h->bytes += (long long)bytes;
  h->peak_bytes = std::max(h->peak_bytes, h->bytes);
  if (h->dry) return (T*)(uintptr_t)256;        // never dereferenced in a size-only pass
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->bytes -= (long long)bytes;
    fail(h, MG_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  h->allocs.push_back(p);
  return (T*)p;
}

void sync(mg_handle* h) { ck(h, cudaStreamSynchronize(h->s), "stream synchronize"); }

double* slot(mg_handle* h, int k) { return h->scal + (size_t)k * 2 * h->R; }

// First double of a slot (right-hand side 0), read synchronously.
double read_scalar(mg_handle* h, int k) {
  ck(h, cudaMemcpyAsync(h->hscal, slot(h, k), 2 * sizeof(double), cudaMemcpyDeviceToHost,
                        h->s),
     "scalar readback");
  sync(h);
  return h->hscal[0];
}

void ensure_partials(mg_handle* h, int nrhs) {
  if (h->partial_rhs >= nrhs) return;
  h->partials = dalloc<double>(h, sizeof(double) * (64 + 2 * 608 * (size_t)nrhs));
  if (!h->dry) ck(h, cudaMemsetAsync(h->partials, 0, sizeof(double) * 64, h->s), "memset tickets");
  h->partial_rhs = nrhs;
}

// Brackets one call of a kernel family with CUDA events when profiling is on.
struct ProfScope {
  mg_handle* h;
  int fam;
  cudaEvent_t end = nullptr;
  ProfScope(mg_handle* h_, int fam_) : h(h_), fam(fam_) {
    if (!h->prof_on) return;
    auto& ev = h->prof_ev[fam];
    size_t& u = h->prof_used[fam];
    while (ev.size() < 2 * (u + 1)) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    cudaEventRecord(ev[2 * u], h->s);
    end = ev[2 * u + 1];
    ++u;
  }
  ~ProfScope() {
    if (end) cudaEventRecord(end, h->s);
  }
};

// ----- level operator ------------------------------------------------------
// weights for coarse levels: 0 = F64, 1 = F32, 2 = BF16
// out = ca (A_l in) + cu U + cw W per the epilogue (default: out = A_l in).
template <typename R>
void apply_level(mg_handle* h, int l, const void* in, void* out, int nrhs, int weights,
                 const Epilogue& ep = Epilogue()) {
  Level& L = h->lv[l];
  ProfScope prof(h, l == 0 ? (sizeof(R) == 8 ? MG_KF_FINE_A64 : MG_KF_FINE_A)
                          : (weights == W_F64 ? MG_KF_COARSE64 : MG_KF_COARSE));
  if (l == 0) {
    const double diag = 4.0 + h->mass;
    const void* U = sizeof(R) == 8 ? (const void*)h->U64 : (const void*)h->U32;
    ck(h, wilson_A<R>(in, out, U, diag, L.Lx, L.Lt, nrhs, ep, h->s), "wilson_A");
  } else {
    const void* A = weights == W_F64 ? (const void*)L.A64
                    : weights == W_F32 ? (const void*)L.A32 : L.A16;
    ck(h, coarse_apply(in, out, A, weights, L.Lx, L.Lt, L.n, nrhs, ep, h->s), "coarse_apply");
  }
}

Epilogue ep_lincomb(double ca, const void* U, double cu, const void* W = nullptr, double cw = 0.0) {
  Epilogue e;
  e.ca = ca;
  e.U = U;
  e.cu = cu;
  e.W = W;
  e.cw = cw;
  return e;
}

// ----- coarsest solve ---------------------------------------------------------
// Coarsest levels above coarsest_dense_max unknowns: CG on the coarsest
// stencil in FP64, x0 = 0, a fixed number `iters` of iterations (chosen at
// set-up so that a test vector reaches coarsest_tol), so that the whole solve
// can be captured in a graph.  The two r.r slots alternate between iterations.
void coarsest_cg(mg_handle* h, const double2* b, double2* x, int iters, int nrhs) {
  const long long n = h->Nc;
  double* rz = slot(h, S_CA);
  double* rn = slot(h, S_CB);
  ck(h, cudaMemsetAsync(x, 0, n * nrhs * sizeof(double2), h->s), "memset");
  ck(h, cudaMemcpyAsync(h->cr, b, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  ck(h, cudaMemcpyAsync(h->cp, b, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  ck(h, norm2<double>(h->cr, n, nrhs, h->partials, rz, h->s), "norm");
  for (int it = 0; it < iters; ++it) {
    apply_level<double>(h, h->L - 1, h->cp, h->cq, nrhs, W_F64);
    ck(h, dot<double>(h->cp, h->cq, n, nrhs, h->partials, slot(h, S_CPQ), h->s), "dot");
    ck(h, cg_xr<double>(x, h->cr, h->cp, h->cq, rz, slot(h, S_CPQ), nullptr, n, nrhs,
                        h->partials, rn, h->s), "cg update");
    if (it + 1 < iters)
      ck(h, cg_p<double>(h->cp, h->cr, rn, rz, nullptr, n, nrhs, h->s), "cg direction");
    std::swap(rz, rn);
  }
}

// Dense path: FP32 explicit inverse refined in FP64.  x = B b; then `steps`
// times: r = b - A_L x (FP64 stencil), x += B r; for nrhs vectors [nrhs][N].
// x32 (optional): an FP32 copy of the result, written by the last step.
// b32 (optional): the right-hand side in FP32; b then receives its FP64 copy
// (for 1 to 4 vectors written by the first GEMV's tile kernel itself).
void coarsest_solve64(mg_handle* h, const double2* b, double2* x, int steps, int nrhs,
                      void* x32 = nullptr, const float2* b32 = nullptr) {
  ProfScope prof(h, MG_KF_COARSEST);
  const long long c = (long long)h->Nc * nrhs;
  const bool in32 = b32 && h->dense && hermitian_gemv_f32in_ok(nrhs);
  if (b32 && !in32) ck(h, convert_f32_f64(b32, (void*)b, c, h->s), "coarsest in");
  if (!h->dense) {
    coarsest_cg(h, b, x, h->ccg_iters, nrhs);
    if (x32) ck(h, convert_f64_f32(x, x32, c, h->s), "coarsest out");
    return;
  }
  auto gemv = [&](const double2* in, bool accumulate, void* out32) {
    {
      ProfScope pd(h, MG_KF_DENSE);
      if (in32 && in == b)
        ck(h, hermitian_gemv_tiles_f32in(h->Bpk, b32, h->Nc, h->ldc, nrhs, h->gemv_part, (void*)b,
                                         h->s), "coarsest gemv");
      else
        ck(h, hermitian_gemv_tiles(h->Bpk, in, h->Nc, h->ldc, nrhs, h->gemv_part, h->s, h->gemv_x),
           "coarsest gemv");
    }
    ck(h, hermitian_gemv_reduce(h->gemv_part, x, h->Nc, h->ldc, nrhs, accumulate, h->s, out32),
       "coarsest gemv reduce");
  };
  gemv(b, false, steps == 0 ? x32 : nullptr);
  for (int it = 0; it < steps; ++it) {
    apply_level<double>(h, h->L - 1, x, h->cr, nrhs, W_F64, ep_lincomb(-1.0, b, 1.0));
    gemv(h->cr, true, it + 1 == steps ? x32 : nullptr);
  }
}

// ----- V-cycle (Sec. 2, five steps), recursive ------------------------------
// Reads b, writes x (both level-l vectors of precision R, nrhs of them).
// tail (optional, level 0): reductions fused into the cycle's last stencil
// application (the flexible-CG pair of Epilogue::zq_q / zq_r).
template <typename R>
void vcycle(mg_handle* h, int l, const void* b, void* x, int nrhs = 1,
            const Epilogue* tail = nullptr) {
  const bool f64 = sizeof(R) == 8;
  const int weights = f64 ? W_F64 : (h->p.vcycle_coarse_bf16 ? W_BF16 : W_F32);
  if (l == h->L - 1) {
    if (f64) {
      coarsest_solve64(h, (const double2*)b, (double2*)x, h->n_refine, nrhs);
    } else {
      coarsest_solve64(h, h->cb, h->cx, h->n_inner, nrhs, x, (const float2*)b);
    }
    return;
  }
  Level& L = h->lv[l];
  Level& C = h->lv[l + 1];
  void** w = f64 ? L.w64 : L.w32;
  void** wc = f64 ? C.w64 : C.w32;
  void* r = w[2];
  // 1. x = R b = c0 b + c1 A b
  apply_level<R>(h, l, b, x, nrhs, weights, ep_lincomb(L.c1, b, L.c0));
  // 2. r_c = P^dagger (b - A x); smoothed first coarsening: P_s^dagger r = P^dagger (r - omega A r)
  apply_level<R>(h, l, x, r, nrhs, weights, ep_lincomb(-1.0, b, 1.0));
  const bool smoothed = l == 0 && h->smooth != 0.0;
  if (smoothed) apply_level<R>(h, 0, r, w[3], nrhs, weights, ep_lincomb(-h->smooth, r, 1.0));
  const void* Vst = f64 ? (const void*)L.Vst64 : (const void*)L.Vst32;
  {
    ProfScope prof(h, MG_KF_TRANSFER);
    ck(h, restrict_op<R>(smoothed ? w[3] : r, wc[0], Vst, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv,
                         nrhs, h->s),
       "restrict");
  }
  // 3. e_c = V_{l+1} r_c
  vcycle<R>(h, l + 1, wc[0], wc[1], nrhs);
  // 4. x = x + P e_c; smoothed: x = x + p - omega A p with p = P e_c
  {
    ProfScope prof(h, MG_KF_TRANSFER);
    ck(h, prolong_op<R>(wc[1], smoothed ? w[3] : x, Vst, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv,
                        nrhs, !smoothed, h->s),
       "prolong");
  }
  if (smoothed)
    apply_level<R>(h, 0, w[3], x, nrhs, weights, ep_lincomb(-h->smooth, w[3], 1.0, x, 1.0));
  // 5. x = x + R (b - A x):  r = b - A x, then x = x + c0 r + c1 A r
  apply_level<R>(h, l, x, r, nrhs, weights, ep_lincomb(-1.0, b, 1.0));
  Epilogue e5 = ep_lincomb(L.c1, r, L.c0, x, 1.0);
  if (tail && l == 0) {
    e5.dot_ws = tail->dot_ws;
    e5.dot_out = tail->dot_out;
    e5.zq_q = tail->zq_q;
    e5.zq_r = tail->zq_r;
  }
  apply_level<R>(h, l, r, x, nrhs, weights, e5);
}

// ----- setup pieces ---------------------------------------------------------
double power_lambda_max(mg_handle* h, int l, const double2* start, void* v, void* w) {
  Level& L = h->lv[l];
  const long long n = L.count();
  ck(h, norm2<double>(start, n, 1, h->partials, slot(h, S_T0), h->s), "norm");
  ck(h, scale_inv_sqrt<double>(start, v, slot(h, S_T0), n, 1, h->s), "scale");
  for (int it = 0; it < h->p.power_iters; ++it) {
    apply_level<double>(h, l, v, w, 1, W_F64);
    if (it == h->p.power_iters - 1) ck(h, dot<double>(v, w, n, 1, h->partials, slot(h, S_T1), h->s), "dot");
    ck(h, norm2<double>(w, n, 1, h->partials, slot(h, S_T0), h->s), "norm");
    ck(h, scale_inv_sqrt<double>(w, v, slot(h, S_T0), n, 1, h->s), "scale");
  }
  return read_scalar(h, S_T1);
}

void smoother_coefficients(mg_handle* h, int l, void* q, void* r1) {
  // Two under-relaxed MR steps from r0 = eta (Sec. 4); R = c0 + c1 A frozen.
  Level& L = h->lv[l];
  const long long n = L.count();
  const double om = h->p.omega_mr;
  apply_level<double>(h, l, L.eta, q, 1, W_F64);
  ck(h, dot<double>(q, L.eta, n, 1, h->partials, slot(h, S_T0), h->s), "dot");
  ck(h, norm2<double>(q, n, 1, h->partials, slot(h, S_T1), h->s), "norm");
  const double num0 = read_scalar(h, S_T0), den0 = read_scalar(h, S_T1);
  if (!(den0 > 0.0)) fail(h, MG_ERR_BREAKDOWN, "MR smoother: A eta = 0");
  const double a0 = num0 / den0;
  ck(h, lincomb<double>(r1, 1.0, L.eta, -om * a0, q, 0.0, nullptr, n, 1, h->s), "mr");
  apply_level<double>(h, l, r1, q, 1, W_F64);
  ck(h, dot<double>(q, r1, n, 1, h->partials, slot(h, S_T0), h->s), "dot");
  ck(h, norm2<double>(q, n, 1, h->partials, slot(h, S_T1), h->s), "norm");
  const double num1 = read_scalar(h, S_T0), den1 = read_scalar(h, S_T1);
  if (!(den1 > 0.0)) fail(h, MG_ERR_BREAKDOWN, "MR smoother: A r1 = 0");
  const double a1 = num1 / den1;
  L.c0 = om * (a0 + a1);
  L.c1 = -om * om * a0 * a1;
}

// G0 and G1 of every coarse level from the vectors: on level 2, G0 = the
// Galerkin product at m = 0 and G1 = (the product at m = 1) - G0 - I; below,
// both pass through P^dagger . P like the operator itself.
void build_quadratic(mg_handle* h) {
  for (int l = 0; l + 1 < h->L; ++l) {
    Level& L = h->lv[l];
    Level& C = h->lv[l + 1];
    ProfScope prof(h, MG_KF_GALERKIN);
    if (l == 0) {
      ck(h, galerkin_fine(h->U64, 4.0, L.Vst64, h->Wbuf, C.G0, L.Lx, L.Lt, L.bx, L.bt, L.Nv, h->s), "galerkin G0");
      ck(h, galerkin_fine(h->U64, 5.0, L.Vst64, h->Wbuf, C.G1, L.Lx, L.Lt, L.bx, L.bt, L.Nv, h->s), "galerkin A(1)");
      ck(h, coarse_lincomb(1.0, C.G1, -1.0, C.G0, -1.0, C.G1, C.V, C.n, h->s), "G1");
    } else {
      ck(h, galerkin_coarse(L.G0, L.Vst64, C.G0, L.Lx, L.Lt, L.bx, L.bt, L.n, L.Nv, h->s), "galerkin G0");
      ck(h, galerkin_coarse(L.G1, L.Vst64, C.G1, L.Lx, L.Lt, L.bx, L.bt, L.n, L.Nv, h->s), "galerkin G1");
    }
  }
  h->g_built = true;
}

void galerkin_next(mg_handle* h, int l);

void build_coarse_ops(mg_handle* h) {
  if (h->p.remass_quadratic) {
    if (!h->g_built) build_quadratic(h);
    const double m = h->mass;
    for (int l = 1; l < h->L; ++l) {
      Level& C = h->lv[l];
      ProfScope prof(h, MG_KF_GALERKIN);
      ck(h, coarse_lincomb(1.0, C.G0, m, C.G1, m * m, C.A64, C.V, C.n, h->s), "A(m)");
      const long long cnt = (long long)C.V * 9 * C.n * C.n;
      ck(h, coarse_convert(C.A64, C.A32, W_F32, cnt, h->s), "convert f32");
      ck(h, coarse_convert(C.A64, C.A16, W_BF16, cnt, h->s), "convert bf16");
    }
    return;
  }
  for (int l = 0; l + 1 < h->L; ++l) {
    Level& L = h->lv[l];
    Level& C = h->lv[l + 1];
    ProfScope prof(h, MG_KF_GALERKIN);
    galerkin_next(h, l);
    const long long cnt = (long long)C.V * 9 * C.n * C.n;
    ck(h, coarse_convert(C.A64, C.A32, W_F32, cnt, h->s), "convert f32");
    ck(h, coarse_convert(C.A64, C.A16, W_BF16, cnt, h->s), "convert bf16");
  }
}

// Test vectors of the coarsest solve's set-up: complex Gaussian entries (Re,
// Im ~ N(0, 1/2)) from splitmix64 (Steele, Lea, Flood, OOPSLA'14) by the
// Box-Muller transform, seeded per vector.  A random vector has components on
// every eigenvector, so the iteration counts fixed with it hold for other
// right-hand sides too (an all-ones vector can miss the slow modes).
constexpr int COARSEST_TEST_VECTORS = 2;

std::vector<double2> coarsest_test_vector(long long n, uint64_t seed) {
  uint64_t st = 0x5eed0000c0a25e57ULL ^ (seed * 0x9E3779B97F4A7C15ULL);
  auto next = [&st]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  std::vector<double2> v(n);
  for (long long i = 0; i < n; ++i) {
    const double u1 = ((next() >> 11) + 1.0) * 0x1.0p-53;     // (0, 1]
    const double u2 = (next() >> 11) * 0x1.0p-53;             // [0, 1)
    const double r = std::sqrt(-std::log(u1));                // E|z|^2 = 1
    v[i] = make_double2(r * std::cos(6.283185307179586 * u2), r * std::sin(6.283185307179586 * u2));
  }
  return v;
}

// Iterations of the coarsest CG: the largest count at which a test vector
// reaches coarsest_tol, times 1.25 plus 4 for other right-hand sides; at most
// COARSEST_CG_MAX (MG_ERR_NOCONV beyond).
constexpr int COARSEST_CG_MAX = 5000;

void build_coarsest_cg(mg_handle* h) {
  const long long n = h->Nc;
  int worst = 0;
  for (int tv = 0; tv < COARSEST_TEST_VECTORS; ++tv) {
    std::vector<double2> tvec = coarsest_test_vector(n, (uint64_t)tv + 1);
    ck(h, cudaMemcpyAsync(h->cb, tvec.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, h->s),
       "upload");
    ck(h, norm2<double>(h->cb, n, 1, h->partials, slot(h, S_T1), h->s), "norm");
    const double bn = read_scalar(h, S_T1);
    const double stop = h->p.coarsest_tol * h->p.coarsest_tol * bn;
    double* rz = slot(h, S_CA);
    double* rn = slot(h, S_CB);
    ck(h, cudaMemsetAsync(h->cx, 0, n * sizeof(double2), h->s), "memset");
    ck(h, cudaMemcpyAsync(h->cr, h->cb, n * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
    ck(h, cudaMemcpyAsync(h->cp, h->cb, n * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
    ck(h, norm2<double>(h->cr, n, 1, h->partials, rz, h->s), "norm");
    int it = 0;
    for (; it < COARSEST_CG_MAX; ++it) {
      apply_level<double>(h, h->L - 1, h->cp, h->cq, 1, W_F64);
      ck(h, dot<double>(h->cp, h->cq, n, 1, h->partials, slot(h, S_CPQ), h->s), "dot");
      ck(h, cg_xr<double>(h->cx, h->cr, h->cp, h->cq, rz, slot(h, S_CPQ), nullptr, n, 1,
                          h->partials, rn, h->s), "cg update");
      ck(h, cg_p<double>(h->cp, h->cr, rn, rz, nullptr, n, 1, h->s), "cg direction");
      std::swap(rz, rn);
      double rr = 0.0;
      ck(h, cudaMemcpyAsync(&rr, rz, sizeof(double), cudaMemcpyDeviceToHost, h->s), "read");
      sync(h);
      if (!(rr == rr)) fail(h, MG_ERR_BREAKDOWN, "coarsest CG is not finite");
      if (rr <= stop) {
        h->coarsest_test_res = std::max(h->coarsest_test_res, std::sqrt(rr / bn));
        break;
      }
    }
    if (it == COARSEST_CG_MAX) fail(h, MG_ERR_NOCONV, "coarsest CG did not reach coarsest_tol");
    worst = std::max(worst, it + 1);
  }
  h->ccg_iters = std::min(COARSEST_CG_MAX, worst + worst / 4 + 4);
}

// Refinement with the FP32 inverse in hand on the current coarsest operator,
// one step at a time: x = B b, then x += B (b - A x) until every test vector
// reaches coarsest_tol within kmax steps.  On success *steps and *inner are the
// largest step counts that reached coarsest_tol and 1e-6.
bool refinement_test(mg_handle* h, int kmax, int* steps, int* inner, double* worst_rel) {
  *steps = 0;
  *inner = 0;
  *worst_rel = 0.0;
  for (int tv = 0; tv < COARSEST_TEST_VECTORS; ++tv) {
    std::vector<double2> tvec = coarsest_test_vector(h->Nc, (uint64_t)tv + 1);
    ck(h, cudaMemcpyAsync(h->cb, tvec.data(), sizeof(double2) * h->Nc, cudaMemcpyHostToDevice,
                          h->s),
       "upload");
    ck(h, norm2<double>(h->cb, h->Nc, 1, h->partials, slot(h, S_T1), h->s), "norm");
    const double bn = read_scalar(h, S_T1);
    ck(h, hermitian_gemv_tiles(h->Bpk, h->cb, h->Nc, h->ldc, 1, h->gemv_part, h->s), "gemv");
    ck(h, hermitian_gemv_reduce(h->gemv_part, h->cx, h->Nc, h->ldc, 1, false, h->s), "gemv");
    int s = 0, s6 = -1;
    double rel = 0.0;
    for (;; ++s) {
      apply_level<double>(h, h->L - 1, h->cx, h->cr, 1, W_F64, ep_lincomb(-1.0, h->cb, 1.0));
      ck(h, norm2<double>(h->cr, h->Nc, 1, h->partials, slot(h, S_T0), h->s), "norm");
      const double rr = read_scalar(h, S_T0);
      if (!(rr == rr)) return false;
      rel = std::sqrt(rr / bn);
      if (s6 < 0 && rel <= 1e-6) s6 = s;
      if (rel <= h->p.coarsest_tol) break;
      if (s == kmax) return false;
      ck(h, hermitian_gemv_tiles(h->Bpk, h->cr, h->Nc, h->ldc, 1, h->gemv_part, h->s), "gemv");
      ck(h, hermitian_gemv_reduce(h->gemv_part, h->cx, h->Nc, h->ldc, 1, true, h->s), "gemv");
    }
    *steps = std::max(*steps, s);
    *inner = std::max(*inner, s6);
    *worst_rel = std::max(*worst_rel, rel);
  }
  return true;
}

// remass: called for a new mass of an existing hierarchy (mg_set_mass).
void build_coarsest(mg_handle* h, bool remass = false) {
  h->coarsest_test_res = 0.0;
  if (!h->dense) {
    build_coarsest_cg(h);
    return;
  }
  if (remass && h->inverse_ok && h->p.coarsest_reuse > 0) {
    int steps = 0, inner = 0;
    double rel = 0.0;
    const int kmax = std::min(h->p.coarsest_reuse, h->p.coarsest_refine_max - 1);
    if (refinement_test(h, kmax, &steps, &inner, &rel)) {
      h->coarsest_test_res = rel;
      h->n_refine = std::min(steps + 1, h->p.coarsest_refine_max);
      h->n_inner = std::max(h->p.inner_coarsest_refine, inner);
      ++h->inverse_reuses;
      return;
    }
    h->coarsest_test_res = 0.0;
  }
  h->inverse_ok = false;
  Level& L = h->lv[h->L - 1];
  ck(h, coarse_to_dense_f32(L.A64, h->Binv, L.Lx, L.Lt, L.n, h->ldc, h->s), "dense");
  {
    ProfScope prof(h, MG_KF_INVERSE);
    const bool tc = h->p.coarsest_gj_tcgen05 != 0;
    int* gj_err = (int*)(h->gj_work + (size_t)3 * h->ldc * 64 + 2 * 64 * 64);
    if (tc) ck(h, cudaMemsetAsync(gj_err, 0, sizeof(int), h->s), "memset");
    ck(h, gauss_jordan_begin(h->Binv, h->ldc, h->gj_work, h->s), "gauss-jordan");
    for (int k = 0; k < h->ldc / 64; ++k) {
      ck(h, gauss_jordan_panel(h->Binv, h->ldc, k, h->gj_work, h->s), "gauss-jordan panel");
      ProfScope pu(h, MG_KF_GJ_UPDATE);
      ck(h, tc ? gauss_jordan_update_tc(h->Binv, h->ldc, k, h->gj_work, h->s)
               : gauss_jordan_update(h->Binv, h->ldc, k, h->gj_work, h->s), "gauss-jordan update");
    }
    if (tc) {
      int e = 0;
      ck(h, cudaMemcpyAsync(&e, gj_err, sizeof(int), cudaMemcpyDeviceToHost, h->s), "read");
      sync(h);
      if (e) {
        // the CTA that gave up may have left tensor-core work in flight: no
        // later result of this handle can be trusted
        h->poisoned = true;
        fail(h, MG_ERR_TIMEOUT, "tensor-core Gauss-Jordan update: completion wait ran out");
      }
    }
    ck(h, pack_hermitian(h->Binv, h->Bpk, h->ldc, h->s), "pack");
  }
  // Refinement count: the smallest number of FP64 correction steps that brings
  // every test vector to coarsest_tol, plus one (at most coarsest_refine_max).
  // If a test vector does not get there within coarsest_refine_max steps the
  // FP32 inverse is too inaccurate for this operator (condition number near
  // 1/eps_FP32): MG_ERR_NOCONV, with the residual reached in the message.
  int worst = 0;
  for (int tv = 0; tv < COARSEST_TEST_VECTORS; ++tv) {
    std::vector<double2> tvec = coarsest_test_vector(h->Nc, (uint64_t)tv + 1);
    ck(h, cudaMemcpyAsync(h->cb, tvec.data(), sizeof(double2) * h->Nc, cudaMemcpyHostToDevice,
                          h->s),
       "upload");
    ck(h, norm2<double>(h->cb, h->Nc, 1, h->partials, slot(h, S_T1), h->s), "norm");
    const double bn = read_scalar(h, S_T1);
    int steps = 0;
    double rel = 0.0;
    for (; steps <= h->p.coarsest_refine_max; ++steps) {
      coarsest_solve64(h, h->cb, h->cx, steps, 1);
      apply_level<double>(h, h->L - 1, h->cx, h->cr, 1, W_F64);
      ck(h, sub_from<double>(h->cb, h->cr, h->Nc, h->s), "residual");
      ck(h, norm2<double>(h->cr, h->Nc, 1, h->partials, slot(h, S_T0), h->s), "norm");
      const double rr = read_scalar(h, S_T0);
      if (!(rr == rr)) fail(h, MG_ERR_BREAKDOWN, "coarsest inverse is not finite");
      rel = std::sqrt(rr / bn);
      if (rel <= h->p.coarsest_tol) break;
    }
    h->coarsest_test_res = std::max(h->coarsest_test_res, rel);
    if (steps > h->p.coarsest_refine_max) {
      char msg[200];
      std::snprintf(msg, sizeof msg,
                    "coarsest solve: FP64 refinement of the FP32 inverse reached %.3g, not "
                    "coarsest_tol %.3g, in %d steps (operator too ill-conditioned for FP32)",
                    rel, h->p.coarsest_tol, h->p.coarsest_refine_max);
      fail(h, MG_ERR_NOCONV, msg);
    }
    worst = std::max(worst, steps);
  }
  h->n_refine = std::min(worst + 1, h->p.coarsest_refine_max);
  h->n_inner = h->p.inner_coarsest_refine;
  h->inverse_ok = true;
}

void drop_graphs(mg_handle* h) {
  for (auto& e : h->loop_exec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
}

void set_mass_internal(mg_handle* h, double mass) {
  drop_graphs(h);
  h->mass = mass;
  build_coarse_ops(h);
  for (int l = 0; l + 1 < h->L; ++l)
    smoother_coefficients(h, l, h->lv[l].w64[3], h->lv[l].w64[2]);
  if (h->L > 1) build_coarsest(h, true);
  sync(h);
}

// Adaptive passes asked for by p (refine_levels up to the first 0).
// Parameters as the handle uses them: smoothed aggregation probes every mass
// anew, so it keeps no quadratic re-mass coefficients.
mg_params normalized(const mg_params& p) {
  mg_params q = p;
  if (q.smooth_omega != 0.0) q.remass_quadratic = 0;
  return q;
}

int refine_count(const mg_params* p) {
  int k = 0;
  while (k < MG_MAX_REFINE && p->refine_levels[k] != 0) ++k;
  return k;
}

// Complex entries of one level-l vector (geometry already validated).
long long level_size(const mg_params* p, int l) {
  long long lx = p->Lx, lt = p->Lt, n = 2;
  for (int k = 0; k < l; ++k) {
    lx /= p->block[k][0];
    lt /= p->block[k][1];
    n = 2 * p->Nv[k];
  }
  return lx * lt * n;
}

// Entries of the random starts of levels first .. nlevels - 2.
size_t noise_len_from(const mg_params* p, int first) {
  size_t t = 0;
  for (int l = first; l + 1 < p->nlevels; ++l) t += (size_t)(p->Nv[l] + 2) * level_size(p, l);
  return t;
}

// The parameters after the first `passes` adaptive passes, with no plan left.
mg_params after_passes(const mg_params* p, int passes) {
  mg_params q = *p;
  for (int k = 0; k < passes; ++k) q.Nv[p->refine_levels[k] - 1] += 1;
  std::memset(q.refine_levels, 0, sizeof(q.refine_levels));
  return q;
}

mg_status validate(const mg_params* p, std::string& msg) {
  if (!p) { msg = "params is NULL"; return MG_ERR_ARG; }
  if (p->Lx < 4 || p->Lt < 4 || p->Lx % 2 || p->Lt % 2) { msg = "Lx, Lt must be even and >= 4"; return MG_ERR_ARG; }
  if (p->nlevels < 1 || p->nlevels > MG_MAX_LEVELS) { msg = "nlevels out of range"; return MG_ERR_ARG; }
  int lx = p->Lx, lt = p->Lt, n = 2;
  for (int l = 0; l + 1 < p->nlevels; ++l) {
    const int bx = p->block[l][0], bt = p->block[l][1], nv = p->Nv[l];
    if (bx < 2 || bt < 2) { msg = "blocks must be at least 2 x 2"; return MG_ERR_ARG; }
    if (lx % bx || lt % bt) { msg = "lattice extent not divisible by block at level " + std::to_string(l + 1); return MG_ERR_ARG; }
    if (lx / bx < 2 || lt / bt < 2) { msg = "coarse extent below 2 at level " + std::to_string(l + 2); return MG_ERR_ARG; }
    if (nv < 1 || nv > bx * bt * n / 2) { msg = "Nv must be in [1, bx*bt*n/2]"; return MG_ERR_ARG; }
    if (bx * bt * n / 2 > 256) { msg = "block-chirality dimension above 256"; return MG_ERR_ARG; }
    if (2 * nv > 64) { msg = "Nv above 32"; return MG_ERR_ARG; }
    lx /= bx; lt /= bt; n = 2 * nv;
  }
  if (p->setup_sweeps < 0 || p->power_iters < 1) { msg = "setup_sweeps >= 0 and power_iters >= 1 required"; return MG_ERR_ARG; }
  if (p->max_rhs < 1 || p->max_rhs > 64) { msg = "max_rhs must be in [1, 64]"; return MG_ERR_ARG; }
  if (p->coarsest_reuse < 0) {
    msg = "coarsest_reuse must be >= 0";
    return MG_ERR_ARG;
  }
  if (!(p->reliable_delta > 0.0 && p->reliable_delta < 1.0)) {
    msg = "reliable_delta must be in (0, 1)";
    return MG_ERR_ARG;
  }
  if (p->nlevels > 1 && !p->setup_noise) { msg = "setup_noise is NULL"; return MG_ERR_ARG; }
  if (p->coarsest_dense_max < 0 || p->coarsest_dense_max > MG_DENSE_MAX) {
    msg = "coarsest_dense_max must be in [0, " + std::to_string(MG_DENSE_MAX) + "]";
    return MG_ERR_ARG;
  }
  if (p->smooth_omega != 0.0) {
    if (!std::isfinite(p->smooth_omega) || p->nlevels < 2) {
      msg = "smooth_omega needs a finite value and nlevels >= 2";
      return MG_ERR_ARG;
    }
    if (p->block[0][0] < 4 || p->block[0][1] < 4 || p->Lx / p->block[0][0] < 3 ||
        p->Lt / p->block[0][1] < 3) {
      msg = "smoothed aggregation needs level-1 blocks of at least 4 x 4 and coarse extents of at least 3";
      return MG_ERR_ARG;
    }
    if (refine_count(p)) { msg = "smoothed aggregation excludes refine_levels"; return MG_ERR_ARG; }
    if (p->smooth_omega < 0.0 &&
        (p->nlevels != 2 || (long long)(p->Lx / p->block[0][0]) * (p->Lt / p->block[0][1]) * 2 *
                                    p->Nv[0] > p->coarsest_dense_max)) {
      msg = "the omega search needs two levels with a dense coarsest level";
      return MG_ERR_ARG;
    }
  }
  const int np = refine_count(p);
  if (np) {
    if (p->refine_cycles < 1) { msg = "refine_cycles must be >= 1"; return MG_ERR_ARG; }
    for (int k = 0; k < np; ++k) {
      const int lv = p->refine_levels[k];
      if (lv < 1 || lv >= p->nlevels || (k && lv < p->refine_levels[k - 1])) {
        msg = "refine_levels must be in [1, nlevels - 1] and not decrease";
        return MG_ERR_ARG;
      }
    }
    // Nv only grows, so the limits hold after every pass if they hold after the last
    const mg_params q = after_passes(p, np);
    if (validate(&q, msg) != MG_OK) { msg = "after the adaptive passes: " + msg; return MG_ERR_ARG; }
  }
  return MG_OK;
}

template <typename F>
mg_status guarded(mg_handle* h, F&& f) {
  if (h && h->poisoned) {
    h->err = "handle unusable: a bounded device-side wait ran out earlier (device state undefined)";
    return MG_ERR_CUDA;
  }
  try {
    f();
    return MG_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    if (h) h->err = "host allocation failed";
    g_last_error = "host allocation failed";
    return MG_ERR_NOMEM;
  } catch (...) {
    if (h) h->err = "unexpected exception";
    g_last_error = "unexpected exception";
    return MG_ERR_CUDA;
  }
}

void free_all(mg_handle* h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->gs) cudaStreamSynchronize(h->gs);
  drop_graphs(h);
  for (auto& e : h->fence)
    if (e) cudaEventDestroy(e);
  if (h->gs) cudaStreamDestroy(h->gs);
  h->gs = nullptr;
  for (auto& v : h->prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  for (void* p : h->allocs)
    if (p) cudaFree(p);
  h->allocs.clear();
  if (h->hscal) cudaFreeHost(h->hscal);
  h->hscal = nullptr;
  if (h->hctrl) cudaFreeHost(h->hctrl);
  h->hctrl = nullptr;
}

// ----- Krylov solvers ---------------------------------------------------------
// All loops below run nrhs right-hand sides in lockstep (nrhs <= max_rhs):
// vectors are [nrhs][count], every scalar slot holds one double2 per rhs, and
// a right-hand side whose residual has reached its target is frozen (the CG
// updates skip it; the V-cycle still processes it, harmlessly).
int* frozen_of(mg_handle* h) { return h->dctrl + 4; }

// q = A p and <p, q> per rhs (fused when the kernel's block count allows it).
// pmode 3: p, q and the product in FP32 (sv32[0], sv32[2]).
void apply_pq(mg_handle* h, int nrhs, int pmode) {
  const long long n = h->lv[0].count();
  const Level& F = h->lv[0];
  Epilogue ep;
  if (pmode == 3) {
    if (wilson_A_ctas(F.Lx, F.Lt, false) <= 608) {
      ep.dot_ws = h->partials;
      ep.dot_out = slot(h, S_PQ);
    }
    apply_level<float>(h, 0, h->sv32[0], h->sv32[2], nrhs, W_F32, ep);
    if (!ep.dot_out)
      ck(h, rdot(h->sv32[0], h->sv32[2], n, nrhs, h->partials, slot(h, S_PQ), h->s), "dot");
    return;
  }
  if (wilson_A_ctas(F.Lx, F.Lt, true) <= 608) {
    ep.dot_ws = h->partials;
    ep.dot_out = slot(h, S_PQ);
  }
  apply_level<double>(h, 0, h->sv64[2], h->sv64[3], nrhs, W_F64, ep);
  if (!ep.dot_out)
    ck(h, dot<double>(h->sv64[2], h->sv64[3], n, nrhs, h->partials, slot(h, S_PQ), h->s), "dot");
}

// x += alpha p, r -= alpha q, |r|^2 (and the FP32 copy of r for pmode 2);
// cc: the loop control taken in the same kernel (graph loops, pmode 0-2).
void pcg_update(mg_handle* h, void* x, int pmode, int nrhs, const CgControl* cc = nullptr) {
  const long long n = h->lv[0].count();
  if (pmode == 3) {           // x32 += alpha p32, r32 -= alpha q32, |r32|^2
    ck(h, rcg_xr(h->sv32[3], h->sv32[1], h->sv32[0], h->sv32[2], slot(h, S_RZ), slot(h, S_PQ),
                 frozen_of(h), n, nrhs, h->partials, slot(h, S_RR), h->s),
       "cg_xr");
    return;
  }
  ck(h, cg_xr<double>(x, h->sv64[1], h->sv64[2], h->sv64[3], slot(h, S_RZ), slot(h, S_PQ),
                      frozen_of(h), n, nrhs, h->partials, slot(h, S_RR), h->s,
                      pmode == 2 ? h->sv32[1] : nullptr, cc),
     "cg_xr");
}

// Preconditioned residual and new search direction.
//   pmode 0: p = r + (|r+|^2/|r|^2) p
//   pmode 1: z = V64 r, p = z + (<r+,z+>/<r,z>) p
//   pmode 2: z32 = V32 r32, p = z32 - (Re<z32, q>/<p, q>) p  (flexible)
void pcg_direction(mg_handle* h, int pmode, int nrhs) {
  const long long n = h->lv[0].count();
  void *r = h->sv64[1], *p = h->sv64[2], *q = h->sv64[3], *z = h->sv64[4];
  const size_t sb = 2 * sizeof(double) * nrhs;
  if (pmode == 3) {
    vcycle<float>(h, 0, h->sv32[1], h->sv32[4], nrhs);
    ck(h, rdot2_zq_rz(h->sv32[4], h->sv32[2], h->sv32[1], n, nrhs, h->partials, slot(h, S_T0),
                      h->s), "dot2");
    ck(h, rcg_p(h->sv32[0], h->sv32[4], slot(h, S_T0), slot(h, S_PQ), slot(h, S_RZ), frozen_of(h),
                n, nrhs, h->s), "cg_p");
  } else if (pmode == 2) {
    // {Re<z, q>, Re<r, z>} in the V-cycle's last fine stencil for batches (when its
    // block count allows); one right-hand side keeps the separate reduction, which
    // measured as fast and leaves the stencil without FP64 operands
    const Level& F = h->lv[0];
    Epilogue tail;
    tail.dot_ws = h->partials;
    tail.dot_out = slot(h, S_T0);
    tail.zq_q = q;
    tail.zq_r = r;
    const bool fused = nrhs > 1 && wilson_A_ctas(F.Lx, F.Lt, false) <= 608;
    vcycle<float>(h, 0, h->sv32[1], h->sv32[4], nrhs, fused ? &tail : nullptr);
    if (!fused)
      ck(h, dot2_zq_rz(h->sv32[4], q, r, n, nrhs, h->partials, slot(h, S_T0), h->s), "dot2");
    ck(h, cg_p_pr(p, h->sv32[4], slot(h, S_T0), slot(h, S_PQ), slot(h, S_RZ), frozen_of(h), n,
                  nrhs, h->s), "cg_p");
  } else if (pmode == 1) {
    vcycle<double>(h, 0, r, z, nrhs);
    ck(h, dot<double>(r, z, n, nrhs, h->partials, slot(h, S_RZN), h->s), "dot");
    ck(h, cg_p<double>(p, z, slot(h, S_RZN), slot(h, S_RZ), frozen_of(h), n, nrhs, h->s), "cg_p");
    ck(h, cudaMemcpyAsync(slot(h, S_RZ), slot(h, S_RZN), sb, cudaMemcpyDeviceToDevice, h->s), "copy");
  } else {
    ck(h, cg_p<double>(p, r, slot(h, S_RR), slot(h, S_RZ), frozen_of(h), n, nrhs, h->s), "cg_p");
    ck(h, cudaMemcpyAsync(slot(h, S_RZ), slot(h, S_RR), sb, cudaMemcpyDeviceToDevice, h->s), "copy");
  }
}

// First direction: p = z0 = M r0, rz = <r0, z0>.
void pcg_start(mg_handle* h, int pmode, int nrhs) {
  const long long n = h->lv[0].count();
  void *r = h->sv64[1], *p = h->sv64[2], *z = h->sv64[4];
  if (pmode == 3) {           // r32 = r, rmax = |r|^2, x32 = 0, p32 = z32 = V r32, rz = <r32, z32>
    ck(h, ru_residual(r, h->sv32[1], n, nrhs, h->partials, slot(h, S_RR), slot(h, S_RMAX), h->s),
       "residual");
    ck(h, cudaMemsetAsync(h->sv32[3], 0, n * nrhs * sizeof(float2), h->s), "memset");
    vcycle<float>(h, 0, h->sv32[1], h->sv32[4], nrhs);
    ck(h, cudaMemcpyAsync(h->sv32[0], h->sv32[4], n * nrhs * sizeof(float2),
                          cudaMemcpyDeviceToDevice, h->s), "copy");
    ck(h, rdot(h->sv32[1], h->sv32[4], n, nrhs, h->partials, slot(h, S_RZ), h->s), "dot");
    return;
  }
  if (pmode == 2) {
    ck(h, convert_f64_f32(r, h->sv32[1], n * nrhs, h->s), "to f32");
    vcycle<float>(h, 0, h->sv32[1], h->sv32[4], nrhs);
    ck(h, convert_f32_f64(h->sv32[4], p, n * nrhs, h->s), "to f64");
  } else if (pmode == 1) {
    vcycle<double>(h, 0, r, z, nrhs);
    ck(h, cudaMemcpyAsync(p, z, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  } else {
    ck(h, cudaMemcpyAsync(p, r, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  }
  ck(h, dot<double>(r, p, n, nrhs, h->partials, slot(h, S_RZ), h->s), "dot");
}

// Reliable update (pmode 3): the FP32 increment joins the FP64 solution and
// the residual is recomputed from it in FP64: x += x32, x32 = 0,
// r = b - A x (FP64 stencil), r32 = r, rr = rmax = |r|^2.
void ru_update(mg_handle* h, const void* b, void* x, int nrhs) {
  const long long n = h->lv[0].count();
  void* r = h->sv64[1];
  ck(h, ru_fold(x, h->sv32[3], n * nrhs, h->s), "fold");
  apply_level<double>(h, 0, x, r, nrhs, W_F64, ep_lincomb(-1.0, b, 1.0));
  ck(h, ru_residual(r, h->sv32[1], n, nrhs, h->partials, slot(h, S_RR), slot(h, S_RMAX), h->s),
     "residual");
}

double ru_delta2(const mg_handle* h) { return h->p.reliable_delta * h->p.reliable_delta; }

// Captures the CG loop body into the body of a conditional WHILE node: the
// control kernel at the end of each iteration decides on the device whether
// to run another iteration, so the whole loop is one graph launch.  pmode 3
// adds a conditional IF node after the residual update whose body is the
// reliable update; the test kernel before it sets its condition.
cudaGraphExec_t build_loop_graph(mg_handle* h, const void* b, void* x, int pmode, int nrhs) {
  const unsigned long long launches0 = launch_count();
  cudaGraph_t g = nullptr;
  ck(h, cudaGraphCreate(&g, 0), "graph create");
  cudaGraphConditionalHandle cond;
  ck(h, cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault), "conditional handle");
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  ck(h, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np), "conditional node");
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaGraphConditionalHandle ifc{};
  if (pmode == 3)
    ck(h, cudaGraphConditionalHandleCreate(&ifc, body, 0, cudaGraphCondAssignDefault),
       "conditional handle");
  cudaStream_t saved = h->s;
  h->s = h->gs;
  ck(h, cudaStreamBeginCaptureToGraph(h->gs, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal), "begin capture");
  long long ru_kern = 0;
  try {
    apply_pq(h, nrhs, pmode);
    CgControl cc;
    cc.ctrl = h->dctrl;
    cc.stop = slot(h, S_STOP);
    cc.tick = h->cg_tick;
    cc.cond = cond;
    pcg_update(h, x, pmode, nrhs, pmode == 3 ? nullptr : &cc);
    if (pmode == 3) {
      ck(h, ru_check(slot(h, S_RR), slot(h, S_RMAX), h->dctrl, ru_delta2(h), h->ru, h->ru + 1, ifc,
                     true, h->s), "reliable-update test");
      // close this segment, add the IF node after its last node, capture the
      // update into the IF body, then continue the loop body after the IF node
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      ck(h, cudaStreamGetCaptureInfo(h->gs, &cs, nullptr, nullptr, &deps, nullptr, &nd),
         "capture info");
      std::vector<cudaGraphNode_t> dv(deps, deps + nd);
      cudaGraph_t seg;
      ck(h, cudaStreamEndCapture(h->gs, &seg), "end capture");
      alignas(cudaGraphNodeParams) unsigned char raw_if[sizeof(cudaGraphNodeParams)] = {};
      cudaGraphNodeParams& ip = *reinterpret_cast<cudaGraphNodeParams*>(raw_if);
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = ifc;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t ifnode;
      ck(h, cudaGraphAddNode(&ifnode, body, dv.data(), nullptr, dv.size(), &ip), "IF node");
      ck(h, cudaStreamBeginCaptureToGraph(h->gs, ip.conditional.phGraph_out[0], nullptr, nullptr,
                                          0, cudaStreamCaptureModeThreadLocal), "begin capture");
      const unsigned long long u0 = launch_count();
      ru_update(h, b, x, nrhs);
      ru_kern = (long long)(launch_count() - u0);
      ck(h, cudaStreamEndCapture(h->gs, &seg), "end capture");
      ck(h, cudaStreamBeginCaptureToGraph(h->gs, body, &ifnode, nullptr, 1,
                                          cudaStreamCaptureModeThreadLocal), "begin capture");
    }
    pcg_direction(h, pmode, nrhs);
    if (pmode == 3)
      ck(h, cg_control(slot(h, S_RR), slot(h, S_PQ), slot(h, S_STOP), h->dctrl, cond, h->s),
         "control");
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(h->gs, &dummy);
    h->s = saved;
    cudaGraphDestroy(g);
    throw;
  }
  h->s = saved;
  // captured kernels did not run; they are counted once per executed iteration
  const long long kern = (long long)(launch_count() - launches0);
  add_launches(-kern);
  ck(h, cudaStreamEndCapture(h->gs, &body), "end capture");
  cudaGraphExec_t exec = nullptr;
  ck(h, cudaGraphInstantiate(&exec, g, 0), "graph instantiate");
  cudaGraphDestroy(g);
  h->loop_kernels[pmode] = kern - ru_kern;
  if (pmode == 3) h->ru_kernels = ru_kern;
  return exec;
}

// PCG on A x = b in FP64 for nrhs right-hand sides, x0 = 0.  Right-hand side
// k stops when |r_k|^2 <= tol2 * ref[k] (recursive residual; ref is the slot
// S_BN, |b_original|^2).  pmode 0: no preconditioner (plain CG); 1: FP64
// V-cycle, standard PCG (beta = <r+, z+>/<r, z>); 2: FP32 V-cycle (FP32
// vectors, FP32 or BF16 coarse blocks, FP64 coarsest solve) on the FP64
// residual, flexible CG: beta = -Re<z+, A p>/<p, A p> (Polak-Ribiere with
// r+ = r - alpha A p), so that rounding in the low-precision preconditioner
// does not break the recursion.  The iteration loop runs as one CUDA graph
// with a device-side WHILE condition (or eagerly, with the same control
// evaluated on the host, while per-kernel profiling is on).  iters[k]
// receives the iterations of right-hand side k; returns the loop length.  x
// must be the handle's solver vector sv64[5]; b is read only here.
int pcg(mg_handle* h, const void* b, void* x, double tol2, int maxiter, int pmode, int nrhs,
        std::vector<int>& iters, mg_status& st) {
  Level& F = h->lv[0];
  const long long n = F.count();
  void* r = h->sv64[1];
  st = MG_OK;
  ck(h, cudaMemsetAsync(x, 0, n * nrhs * sizeof(double2), h->s), "memset");
  ck(h, cudaMemcpyAsync(r, b, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  ck(h, set_control(h->dctrl, maxiter, nrhs, slot(h, S_BN), tol2, slot(h, S_STOP), h->s), "control init");
  if (pmode == 3) ck(h, cudaMemsetAsync(h->ru, 0, 2 * sizeof(int), h->s), "memset");
  pcg_start(h, pmode, nrhs);
  if (pmode) {
    h->vcycles++;
    h->fine_applies += 4;
  }
  const int per_it_fine = 1 + (pmode ? 4 : 0);
  int it = 0, status = 0;
  int hru[2] = {0, 0};
  if (h->use_graphs && !h->prof_on) {
    const int key = pmode + 4 * (nrhs - 1);
    auto& exec = h->loop_exec[key];
    if (!exec) exec = build_loop_graph(h, b, x, pmode, nrhs);
    ck(h, cudaEventRecord(h->fence[0], h->s), "event");
    ck(h, cudaStreamWaitEvent(h->gs, h->fence[0], 0), "wait");
    ck(h, cudaGraphLaunch(exec, h->gs), "graph launch");
    ck(h, cudaEventRecord(h->fence[1], h->gs), "event");
    ck(h, cudaStreamWaitEvent(h->s, h->fence[1], 0), "wait");
    ck(h, cudaMemcpyAsync(h->hctrl, h->dctrl, (4 + 2 * nrhs) * sizeof(int), cudaMemcpyDeviceToHost, h->s), "rb");
    if (pmode == 3)
      ck(h, cudaMemcpyAsync(hru, h->ru, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s), "rb");
    sync(h);
    it = h->hctrl[0];
    status = h->hctrl[1];
    add_launches((long long)it * h->loop_kernels[pmode]);
    h->fine_applies += (long long)it * per_it_fine;
    if (pmode) h->vcycles += it;
  } else {
    // eager loop: the control decisions of k_cg_control, taken on the host
    std::vector<int> ctrl(4 + 2 * nrhs);
    ck(h, cudaMemcpyAsync(ctrl.data(), h->dctrl, ctrl.size() * sizeof(int), cudaMemcpyDeviceToHost, h->s), "rb");
    sync(h);
    std::vector<double> pq(2 * nrhs), rr(2 * nrhs), stop(2 * nrhs);
    ck(h, cudaMemcpyAsync(stop.data(), slot(h, S_STOP), stop.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
    sync(h);
    status = 0;
    while (status == 0) {
      apply_pq(h, nrhs, pmode);
      h->fine_applies++;
      pcg_update(h, x, pmode, nrhs);
      if (pmode == 3) {         // the reliable-update test of the graph, decided on the host
        ck(h, ru_check(slot(h, S_RR), slot(h, S_RMAX), h->dctrl, ru_delta2(h), h->ru, h->ru + 1,
                       cudaGraphConditionalHandle{}, false, h->s), "reliable-update test");
        ck(h, cudaMemcpyAsync(hru, h->ru, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->s), "rb");
        sync(h);
        if (hru[0]) ru_update(h, b, x, nrhs);
      }
      ck(h, cudaMemcpyAsync(pq.data(), slot(h, S_PQ), pq.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
      ck(h, cudaMemcpyAsync(rr.data(), slot(h, S_RR), rr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
      sync(h);
      ++it;
      int running = 0, broken = 0;
      for (int k = 0; k < nrhs; ++k) {
        int& fr = ctrl[4 + k];
        if (fr) continue;
        if (!(pq[2 * k] > 0.0) || !(rr[2 * k] == rr[2 * k])) { fr = 2; ctrl[4 + nrhs + k] = it; broken = 1; }
        else if (rr[2 * k] <= stop[2 * k]) { fr = 1; ctrl[4 + nrhs + k] = it; }
        else ++running;
      }
      status = running ? 0 : 1;
      if (broken) status = 2;
      else if (running && it >= maxiter) status = 3;
      if (status == 3)
        for (int k = 0; k < nrhs; ++k)
          if (!ctrl[4 + k]) ctrl[4 + nrhs + k] = it;
      ck(h, cudaMemcpyAsync(h->dctrl + 4, ctrl.data() + 4, nrhs * sizeof(int), cudaMemcpyHostToDevice, h->s), "frozen");
      sync(h);
      if (status != 0) break;
      pcg_direction(h, pmode, nrhs);
      if (pmode) {
        h->vcycles++;
        h->fine_applies += 4;
      }
    }
    std::memcpy(h->hctrl, ctrl.data(), ctrl.size() * sizeof(int));
  }
  if (pmode == 3) {             // updates made in the loop, then the last FP32 increment
    if (h->use_graphs && !h->prof_on) add_launches((long long)hru[1] * h->ru_kernels);
    h->fine_applies += hru[1];
    ck(h, ru_fold(x, h->sv32[3], n * nrhs, h->s), "fold");
  }
  for (int k = 0; k < nrhs; ++k) iters[k] += h->hctrl[4 + nrhs + k];
  if (status == 2) {
    st = MG_ERR_BREAKDOWN;
    h->err = "CG breakdown: <p, A p> <= 0 or non-finite residual";
  } else if (status == 3) {
    st = MG_ERR_NOCONV;
    h->err = "maximum iterations reached";
  }
  return it;
}

// True residuals |b - A x|^2 of nrhs vectors into slot S_NR (r receives b - A x).
void true_residuals(mg_handle* h, const void* b, const void* x, void* r, int nrhs) {
  const long long n = h->lv[0].count();
  apply_level<double>(h, 0, x, r, nrhs, W_F64, ep_lincomb(-1.0, b, 1.0));
  h->fine_applies++;
  ck(h, norm2<double>(r, n, nrhs, h->partials, slot(h, S_NR), h->s), "norm");
}

// Solves nrhs <= max_rhs right-hand sides together; restarts from the true
// residual when the recursive one has drifted from it.
mg_status solve_batch(mg_handle* h, const void* b, void* x, int nrhs, double tol, int maxiter,
                      int solver, mg_solve_info* info) {
  const long long n = h->lv[0].count();
  const int pmode = solver == MG_SOLVER_MGCG_FP64 ? 1 : solver == MG_SOLVER_MGCG_MIXED ? 2
                    : solver == MG_SOLVER_MGCG_RELIABLE ? 3 : 0;
  if (solver != MG_SOLVER_MGCG_FP64 && solver != MG_SOLVER_CG_FP64 && solver != MG_SOLVER_MGCG_MIXED &&
      solver != MG_SOLVER_MGCG_RELIABLE)
    fail(h, MG_ERR_ARG, "unknown solver");
  h->fine_applies = 0;
  h->vcycles = 0;
  std::vector<double> hb(2 * nrhs), hr(2 * nrhs);
  ck(h, norm2<double>(b, n, nrhs, h->partials, slot(h, S_BN), h->s), "norm");
  ck(h, cudaMemcpyAsync(hb.data(), slot(h, S_BN), hb.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
  sync(h);
  for (int k = 0; k < nrhs; ++k)
    if (!(hb[2 * k] == hb[2 * k]) || std::isinf(hb[2 * k]))
      fail(h, MG_ERR_BREAKDOWN, "non-finite right-hand side");
  ck(h, cudaMemsetAsync(x, 0, n * nrhs * sizeof(double2), h->s), "memset");
  void* xc = h->sv64[5];
  void* rt = h->sv64[0];
  ck(h, cudaMemcpyAsync(rt, b, n * nrhs * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  std::vector<int> iters(nrhs, 0);
  mg_status st = MG_OK;
  int total = 0, restarts = 0;
  for (int cycle = 0; cycle < 8; ++cycle) {
    // target |r|^2 <= tol2 |b|^2: tol^2 first, then half of it on restarts
    const double tol2 = cycle == 0 ? tol * tol : 0.25 * tol * tol;
    total += pcg(h, rt, xc, tol2, maxiter - total, pmode, nrhs, iters, st);
    ck(h, lincomb<double>(x, 1.0, x, 1.0, xc, 0.0, nullptr, n * nrhs, 1, h->s), "accumulate");
    if (st != MG_OK && st != MG_ERR_NOCONV) break;
    true_residuals(h, b, x, rt, nrhs);
    ck(h, cudaMemcpyAsync(hr.data(), slot(h, S_NR), hr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
    sync(h);
    bool done = true;
    for (int k = 0; k < nrhs; ++k)
      if (hr[2 * k] > tol * tol * hb[2 * k]) done = false;
    if (done) { st = MG_OK; break; }
    if (total >= maxiter) { st = MG_ERR_NOCONV; h->err = "maximum iterations reached"; break; }
    restarts++;
  }
  if (info) {
    true_residuals(h, b, x, h->sv64[0], nrhs);
    ck(h, cudaMemcpyAsync(hr.data(), slot(h, S_NR), hr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->s), "rb");
    sync(h);
    for (int k = 0; k < nrhs; ++k) {
      info[k].iterations = iters[k];
      info[k].refinements = restarts;
      info[k].true_residual = hb[2 * k] > 0 ? std::sqrt(hr[2 * k] / hb[2 * k]) : 0.0;
      info[k].fine_applies = h->fine_applies;
      info[k].vcycles = h->vcycles;
    }
  }
  return st;
}

// Level geometry from the parameters (no device work).
void set_geometry(mg_handle* h) {
  const mg_params& P = h->p;
    h->lv.resize(h->L);
    int lx = P.Lx, lt = P.Lt, n = 2;
    for (int l = 0; l < h->L; ++l) {
      Level& L = h->lv[l];
      L.Lx = lx; L.Lt = lt; L.V = lx * lt; L.n = n;
      if (l + 1 < h->L) {
        L.bx = P.block[l][0]; L.bt = P.block[l][1]; L.Nv = P.Nv[l];
        lx /= L.bx; lt /= L.bt; n = 2 * L.Nv;
      }
    }
}

// Every device allocation that outlives mg_setup, in one place, so that a
// size-only pass (h->dry) gives the handle's device footprint exactly.
void allocate_storage(mg_handle* h) {
  const mg_params& P = h->p;
  h->scal = dalloc<double>(h, (size_t)S_COUNT * 2 * h->R * sizeof(double));
  h->dflag = dalloc<int>(h, sizeof(int));
  h->dctrl = dalloc<int>(h, (4 + 2 * h->R) * sizeof(int));
  h->ru = dalloc<int>(h, 2 * sizeof(int));
  h->cg_tick = dalloc<unsigned>(h, sizeof(unsigned));
  if (!h->dry) ck(h, cudaMemsetAsync(h->cg_tick, 0, sizeof(unsigned), h->s), "memset ticket");
  int max_nv = h->R;
  for (int l = 0; l + 1 < h->L; ++l) max_nv = std::max(max_nv, h->lv[l].Nv);
  ensure_partials(h, max_nv);
  const long long V = h->lv[0].V;
  h->U64 = dalloc<double2>(h, 2 * V * sizeof(double2));
  h->U32 = dalloc<float2>(h, 2 * V * sizeof(float2));
  // per-level storage
  for (int l = 0; l < h->L; ++l) {
    Level& L = h->lv[l];
    const size_t c = (size_t)L.count();
    for (int k = 0; k < 4; ++k) {
      L.w64[k] = dalloc(h, c * h->R * sizeof(double2));
      L.w32[k] = dalloc(h, c * h->R * sizeof(float2));
    }
    if (l > 0) {
      const size_t ab = (size_t)L.V * 9 * L.n * L.n;
      L.A64 = dalloc<double2>(h, ab * sizeof(double2));
      L.A32 = dalloc<float2>(h, ab * sizeof(float2));
      L.A16 = dalloc(h, ab * 4);
      if (h->p.remass_quadratic) {
        L.G0 = dalloc<double2>(h, ab * sizeof(double2));
        L.G1 = dalloc<double2>(h, ab * sizeof(double2));
      }
    }
    if (l + 1 < h->L) {
      L.Vst64 = dalloc<double2>(h, (size_t)L.V * 2 * L.Nv * (L.n / 2) * sizeof(double2));
      L.Vst32 = dalloc<float2>(h, (size_t)L.V * 2 * L.Nv * (L.n / 2) * sizeof(float2));
      L.eta = dalloc<double2>(h, c * sizeof(double2));
    }
  }
  for (int k = 0; k < 6; ++k) {
    h->sv64[k] = dalloc(h, (size_t)h->lv[0].count() * h->R * sizeof(double2));
    h->sv32[k] = dalloc(h, (size_t)h->lv[0].count() * h->R * sizeof(float2));
  }
  if (h->L > 1) {
    const Level& L0 = h->lv[0];
    const size_t Vc = (size_t)(L0.Lx / L0.bx) * (L0.Lt / L0.bt);
    h->Wbuf = dalloc(h, Vc * 2 * L0.Nv * (L0.bx + 2) * (L0.bt + 2) * 2 * sizeof(double2));
  }
  // coarsest dense storage
  if (h->L > 1) {
    const Level& C = h->lv[h->L - 1];
    h->Nc = (int)C.count();
    h->ldc = (h->Nc + 63) / 64 * 64;
    h->dense = h->Nc <= P.coarsest_dense_max;
    if (h->dense) {
      h->Binv = dalloc<float2>(h, (size_t)h->ldc * h->ldc * sizeof(float2));
      h->gj_work = dalloc<float2>(h, ((size_t)3 * h->ldc * 64 + 2 * 64 * 64 + 2) * sizeof(float2));
      h->gemv_x = dalloc<float2>(h, (size_t)h->ldc * h->R * sizeof(float2));
      const size_t nt = h->ldc / 64, ntiles = nt * (nt + 1) / 2;
      h->Bpk = dalloc<float2>(h, ntiles * 64 * 64 * sizeof(float2));
      h->gemv_part = dalloc<float2>(h, ntiles * 2 * 64 * h->R * sizeof(float2));
    } else {
      h->cp = dalloc<double2>(h, (size_t)h->Nc * h->R * sizeof(double2));
      h->cq = dalloc<double2>(h, (size_t)h->Nc * h->R * sizeof(double2));
    }
    h->cb = dalloc<double2>(h, (size_t)h->Nc * h->R * sizeof(double2));
    h->cx = dalloc<double2>(h, (size_t)h->Nc * h->R * sizeof(double2));
    h->cr = dalloc<double2>(h, (size_t)h->Nc * h->R * sizeof(double2));
  }
}

// Pinned host mirrors, the internal graph stream and its fences.
void init_runtime(mg_handle* h) {
  ck(h, cudaMallocHost((void**)&h->hscal, 64 * sizeof(double)), "pinned alloc");
  ck(h, cudaMallocHost((void**)&h->hctrl, (4 + 2 * h->R) * sizeof(int)), "pinned alloc");
  ck(h, cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking), "stream create");
  ck(h, cudaEventCreateWithFlags(&h->fence[0], cudaEventDisableTiming), "event create");
  ck(h, cudaEventCreateWithFlags(&h->fence[1], cudaEventDisableTiming), "event create");
  if (const char* e = std::getenv("MG_NO_GRAPHS")) h->use_graphs = e[0] == '0';
}

// Device bytes of the set-up's temporary relaxation vectors (E and T of the
// largest level), allocated and freed inside mg_setup.
long long setup_temp_bytes(const mg_handle* h) {
  long long t = 0;
  for (int l = 0; l + 1 < h->L; ++l)
    t = std::max(t, 2LL * h->lv[l].Nv * h->lv[l].count() * (long long)sizeof(double2));
  if (h->p.smooth_omega != 0.0 && h->L > 1) {   // column probing of the smoothed level 2
    const Level& L = h->lv[0];
    const Level& C = h->lv[1];
    const long long nc = 2LL * L.Nv;
    t = std::max(t, (3 * nc * L.count() + 2 * nc * C.count() + 3LL * C.V * 9 * C.n * C.n) *
                        (long long)sizeof(double2));
  }
  return t;
}

// ----- smoothed aggregation of the first coarsening (Sec. 3) ----------------
// Colour period of the column probing along an axis of `L` coarse sites: the
// smallest divisor >= 3 (sites of one colour are then at least 3 apart).
int probe_period(int L) {
  for (int k = 3; k < L; ++k)
    if (L % k == 0) return k;
  return L;
}

// G_k = P^dagger A^(k+1) P (k = 0, 1, 2) on level 2, by column probing: for
// each colour, the 2 Nv probe vectors are prolonged, A is applied three times,
// and the restrictions of A w, A^2 w, A^3 w are scattered into G_0, G_1, G_2.
// The level-2 operator of P_s = (1 - omega A) P is then
// P_s^dagger A P_s = G_0 - 2 omega G_1 + omega^2 G_2.
void smoothed_products(mg_handle* h, double2* G[3]) {
  Level& L = h->lv[0];
  Level& C = h->lv[1];
  const int nc = 2 * L.Nv;
  const long long c = L.count(), cc = C.count();
  ProfScope prof(h, MG_KF_GALERKIN);
  void* W = dalloc(h, (size_t)nc * c * sizeof(double2));
  void* T1 = dalloc(h, (size_t)nc * c * sizeof(double2));
  void* T2 = dalloc(h, (size_t)nc * c * sizeof(double2));
  void* E = dalloc(h, (size_t)nc * cc * sizeof(double2));
  void* Y = dalloc(h, (size_t)nc * cc * sizeof(double2));
  const int Kx = probe_period(C.Lx), Kt = probe_period(C.Lt);
  for (int ct = 0; ct < Kt; ++ct)
    for (int cx = 0; cx < Kx; ++cx) {
      ck(h, probe_vectors(E, C.Lx, C.Lt, nc, Kx, Kt, cx, ct, h->s), "probe vectors");
      ck(h, prolong_op<double>(E, W, L.Vst64, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nc, false, h->s),
         "probe prolong");
      const void* in = W;
      void* outs[3] = {T1, T2, T1};
      for (int k = 0; k < 3; ++k) {
        apply_level<double>(h, 0, in, outs[k], nc, W_F64);
        ck(h, restrict_op<double>(outs[k], Y, L.Vst64, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nc, h->s),
           "probe restrict");
        ck(h, probe_scatter(Y, G[k], C.Lx, C.Lt, nc, Kx, Kt, cx, ct, h->s), "probe scatter");
        in = outs[k];
      }
    }
  sync(h);
  for (void* q : {W, T1, T2, E, Y}) {
    for (auto& a : h->allocs)
      if (a == q) a = nullptr;
    cudaFree(q);
  }
  h->bytes -= (3LL * nc * c + 2LL * nc * cc) * (long long)sizeof(double2);
}

void smoothed_combination(mg_handle* h, double2* const G[3], double omega) {
  Level& C = h->lv[1];
  ck(h, coarse_lincomb(1.0, G[0], -2.0 * omega, G[1], 0.0, C.A64, C.V, C.n, h->s), "A_c(omega)");
  ck(h, coarse_lincomb(1.0, C.A64, omega * omega, G[2], 0.0, C.A64, C.V, C.n, h->s), "A_c(omega)");
}

// Largest eigenvalue of a Hermitian positive operator on n entries by
// `iters` power iterations from v (overwritten), with w as scratch: the
// Rayleigh quotient <v, apply(v)> of the last normalised iterate.
template <typename F>
double power_rq(mg_handle* h, long long n, void* v, void* w, int iters, F apply) {
  ck(h, norm2<double>(v, n, 1, h->partials, slot(h, S_T0), h->s), "norm");
  ck(h, scale_inv_sqrt<double>(v, v, slot(h, S_T0), n, 1, h->s), "scale");
  for (int it = 0; it < iters; ++it) {
    apply(v, w);
    if (it == iters - 1) ck(h, dot<double>(v, w, n, 1, h->partials, slot(h, S_T1), h->s), "dot");
    ck(h, norm2<double>(w, n, 1, h->partials, slot(h, S_T0), h->s), "norm");
    ck(h, scale_inv_sqrt<double>(w, v, slot(h, S_T0), n, 1, h->s), "scale");
  }
  return read_scalar(h, S_T1);
}

// Condition number of the two-level hierarchy's level 2 (its coarsest level,
// with the dense inverse built): lambda_max from power iterations on A_2,
// lambda_min as 1 / lambda_max(A_2^-1) from power iterations on the coarsest
// solve, both from fixed Gaussian starts.
constexpr int SMOOTH_POWER_ITERS = 200;

double coarse_condition(mg_handle* h) {
  Level& C = h->lv[1];
  const long long n = C.count();
  void* v = C.w64[0];
  void* w = C.w64[1];
  std::vector<double2> st = coarsest_test_vector(n, 11);
  ck(h, cudaMemcpyAsync(v, st.data(), n * sizeof(double2), cudaMemcpyHostToDevice, h->s), "upload");
  const double lmax = power_rq(h, n, v, w, SMOOTH_POWER_ITERS, [&](void* a, void* b) {
    apply_level<double>(h, 1, a, b, 1, W_F64);
  });
  st = coarsest_test_vector(n, 12);
  ck(h, cudaMemcpyAsync(v, st.data(), n * sizeof(double2), cudaMemcpyHostToDevice, h->s), "upload");
  const double mu = power_rq(h, n, v, w, SMOOTH_POWER_ITERS, [&](void* a, void* b) {
    coarsest_solve64(h, (const double2*)a, (double2*)b, h->n_refine, 1);
  });
  if (!(lmax > 0.0) || !(mu > 0.0)) return INFINITY;
  return lmax * mu;
}

// omega in [0, 2 / lambda~max(A)] minimising the condition number of level 2
// (Sec. 3: the damping of the smoothing step), the best of an even grid of 41
// points refined by 40 golden-section steps on the bracket around it.  An omega
// for which the dense coarsest inverse cannot be refined to coarsest_tol
// counts as infinitely ill-conditioned.
double smoothed_search(mg_handle* h, double2* const G[3], double* cond_out) {
  const double lam = h->lv[0].lambda_max;
  auto f = [&](double w) {
    smoothed_combination(h, G, w);
    try {
      build_coarsest(h);
    } catch (const Fail&) {
      return (double)INFINITY;
    }
    return coarse_condition(h);
  };
  const int samples = 41, refine = 40;
  std::vector<double> grid(samples), vals(samples);
  for (int k = 0; k < samples; ++k) {
    grid[k] = 2.0 / lam * k / (samples - 1);
    vals[k] = f(grid[k]);
  }
  int kb = 0;
  for (int k = 1; k < samples; ++k)
    if (vals[k] < vals[kb]) kb = k;
  double a = grid[std::max(kb - 1, 0)], b = grid[std::min(kb + 1, samples - 1)];
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double c = b - g * (b - a), d = a + g * (b - a);
  double fc = f(c), fd = f(d);
  for (int it = 0; it < refine; ++it) {
    if (fc < fd) {
      b = d; d = c; fd = fc;
      c = b - g * (b - a);
      fc = f(c);
    } else {
      a = c; c = d; fc = fd;
      d = a + g * (b - a);
      fd = f(d);
    }
  }
  double best = grid[kb], fb = vals[kb];
  if (fc < fb) { best = c; fb = fc; }
  if (fd < fb) { best = d; fb = fd; }
  if (!std::isfinite(fb)) fail(h, MG_ERR_NOCONV, "smoothed aggregation: no omega gives a usable level 2");
  *cond_out = fb;
  return best;
}

// Level 2 from the smoothed prolongator: omega in use, else the given one, else searched.
void galerkin_smoothed(mg_handle* h) {
  Level& C = h->lv[1];
  const size_t ab = (size_t)C.V * 9 * C.n * C.n * sizeof(double2);
  double2* G[3];
  for (auto& q : G) q = dalloc<double2>(h, ab);
  smoothed_products(h, G);
  if (h->smooth == 0.0) {
    if (h->p.smooth_omega > 0.0) {
      h->smooth = h->p.smooth_omega;
    } else {
      double cond = 0.0;
      h->smooth = smoothed_search(h, G, &cond);
      h->smooth_cond = cond;
    }
  }
  smoothed_combination(h, G, h->smooth);
  sync(h);
  for (double2* q : G) {
    for (auto& a : h->allocs)
      if (a == q) a = nullptr;
    cudaFree(q);
  }
  h->bytes -= 3LL * (long long)ab;
}

// Galerkin operator of level l + 1 from the vectors of level l (FP64 master only).
void galerkin_next(mg_handle* h, int l) {
  Level& L = h->lv[l];
  Level& C = h->lv[l + 1];
  if (l == 0 && h->p.smooth_omega != 0.0)
    galerkin_smoothed(h);
  else if (l == 0)
    ck(h, galerkin_fine(h->U64, 4.0 + h->mass, L.Vst64, h->Wbuf, C.A64, L.Lx, L.Lt, L.bx, L.bt, L.Nv, h->s), "galerkin_fine");
  else
    ck(h, galerkin_coarse(L.A64, L.Vst64, C.A64, L.Lx, L.Lt, L.bx, L.bt, L.n, L.Nv, h->s), "galerkin_coarse");
}

// One level of the adaptive setup (Sec. 3): with E = NULL, Nv random starts
// from `noise` (then the power-iteration start and the smoother start) are
// relaxed with Eq. relax; with E given (Nv full level vectors), the level takes
// them as they are and keeps the relaxation step and smoother start it holds.
// The vectors are split by chirality and block-orthonormalised (FP64), and the
// Galerkin operator of the next level is built from them.
void build_level(mg_handle* h, int l, const double2* noise, const void* Egiven) {
  Level& L = h->lv[l];
  const long long c = L.count();
  void* E = nullptr;
  void* T = nullptr;
  if (!Egiven) {
    const double2* starts = noise;
    const double2* pw = noise + (size_t)L.Nv * c;
    ck(h, cudaMemcpyAsync(L.eta, pw + c, c * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy eta");
    // relaxation step from lambda_max (power iteration)
    L.lambda_max = power_lambda_max(h, l, pw, L.w64[1], L.w64[2]);
    if (!(L.lambda_max > 0.0)) fail(h, MG_ERR_BREAKDOWN, "power iteration gave lambda_max <= 0");
    L.omega_relax = 1.0 / L.lambda_max;
    // Eq. relax: e <- (1 - omega A) e, nu sweeps, all Nv vectors at once
    E = dalloc(h, (size_t)L.Nv * c * sizeof(double2));
    T = dalloc(h, (size_t)L.Nv * c * sizeof(double2));
    ck(h, cudaMemcpyAsync(E, starts, (size_t)L.Nv * c * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
    for (int sw = 0; sw < h->p.setup_sweeps; ++sw) {
      apply_level<double>(h, l, E, T, L.Nv, W_F64);
      ck(h, axpby<double>(-L.omega_relax, T, 1.0, E, c, L.Nv, h->s), "relax");
    }
  }
  // chirality split + block Gram-Schmidt (FP64)
  ck(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->s), "memset");
  ck(h, block_gram_schmidt(Egiven ? Egiven : E, L.Vst64, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, 1e-14,
                           h->dflag, h->s), "gram-schmidt");
  int flag = 0;
  ck(h, cudaMemcpyAsync(h->hscal, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->s), "rb");
  sync(h);
  std::memcpy(&flag, h->hscal, sizeof(int));
  if (flag) fail(h, MG_ERR_BREAKDOWN, "block Gram-Schmidt breakdown at level " + std::to_string(l + 1));
  ck(h, convert_f64_f32(L.Vst64, L.Vst32, (long long)L.V * 2 * L.Nv * (L.n / 2), h->s), "convert");
  // Galerkin operator of the next level (needed before relaxing on it)
  galerkin_next(h, l);
  sync(h);
  if (E) {
    for (auto& a : h->allocs)
      if (a == E || a == T) a = nullptr;
    cudaFree(E);
    cudaFree(T);
    h->bytes -= 2LL * L.Nv * c * (long long)sizeof(double2);
  }
}

// Autotuning of the fused fine A for this handle's launches (FP32 and FP64,
// 1 and max_rhs right-hand sides), on the idle solver vectors.  The input is
// the link field read as a fine vector (2 V unit-modulus entries, the size of
// one fine vector), repeated.
void autotune_fine(mg_handle* h) {
  const Level& F = h->lv[0];
  const long long c = F.count();
  const double diag = 4.0 + h->mass;
  for (int k = 0; k < h->R; ++k)
    ck(h, cudaMemcpyAsync((double2*)h->sv64[0] + k * c, h->U64, c * sizeof(double2),
                          cudaMemcpyDeviceToDevice, h->s), "tune input");
  ck(h, convert_f64_f32(h->sv64[0], h->sv32[0], c * h->R, h->s), "tune input");
  for (int nrhs : {1, h->R}) {
    ck(h, wilson_A_tune<double>(h->sv64[0], h->sv64[1], h->sv64[2], h->U64, diag, F.Lx, F.Lt,
                                nrhs, h->dflag, h->s), "tune f64");
    ck(h, wilson_A_tune<float>(h->sv32[0], h->sv32[1], h->sv32[2], h->U32, diag, F.Lx, F.Lt,
                               nrhs, h->dflag, h->s), "tune f32");
    if (h->R == 1) break;
  }
  sync(h);
}

// ----- critical mass (the mass gap m - m_crit of Sec. 4) ----------------------
struct EigH {
  double lam = 0.0, slope = 0.0;
  int its = 0;
};

// Eigenvalue of the Hermitian H(m) = sigma_3 D(m) nearest zero, by inverse
// iteration with H^-1 = A^-1 D^dagger sigma_3 (one MG-CG solve per step,
// warm-started from v, which holds the unit eigenvector on return): lam =
// <v, sigma_3 D v>, and its derivative dlam/dm = <v, sigma_3 v> (dH/dm =
// sigma_3, first-order perturbation theory).  w, t: scratch fine vectors.
EigH nearest_eig_H(mg_handle* h, double m, void* v, void* w, void* t, int solver, double solve_tol,
                   int max_inv, double conv) {
  if (m != h->mass) set_mass_internal(h, m);
  const Level& F = h->lv[0];
  const long long c = F.count();
  const double diag = 4.0 + m;
  EigH e;
  double prev = 0.0;
  for (int k = 0; k < max_inv; ++k) {
    ck(h, sigma3_mul(v, t, F.V, h->s), "sigma3");
    ck(h, wilson_D<double>(t, w, h->U64, diag, F.Lx, F.Lt, 1, true, h->s), "D dagger");
    mg_solve_info info{};
    solve_batch(h, w, t, 1, solve_tol, 100000, solver, &info);   // an inexact solve still iterates
    ck(h, norm2<double>(t, c, 1, h->partials, slot(h, S_T0), h->s), "norm");
    ck(h, scale_inv_sqrt<double>(t, v, slot(h, S_T0), c, 1, h->s), "normalise");
    ck(h, wilson_D<double>(v, w, h->U64, diag, F.Lx, F.Lt, 1, false, h->s), "D");
    ck(h, sigma3_mul(w, w, F.V, h->s), "sigma3");
    ck(h, dot<double>(v, w, c, 1, h->partials, slot(h, S_T1), h->s), "dot");
    e.lam = read_scalar(h, S_T1);
    e.its = k + 1;
    if (k && std::fabs(e.lam - prev) <= conv * std::fabs(e.lam)) break;
    prev = e.lam;
  }
  ck(h, sigma3_mul(v, w, F.V, h->s), "sigma3");
  ck(h, dot<double>(v, w, c, 1, h->partials, slot(h, S_T1), h->s), "dot");
  e.slope = read_scalar(h, S_T1);
  return e;
}

// Eigenvalue of D(m) nearest zero, by inverse iteration with D^-1 =
// A^-1 D^dagger (warm-started from v, which holds the unit right eigenvector
// on return): lam = <v, D v>.  Since D(m) = D_0 + m, an eigenvalue of D(m) is
// lam_0 + m exactly, so a real one gives the mass at which it vanishes.
double2 nearest_eig_D(mg_handle* h, double m, void* v, void* w, void* t, int solver,
                      double solve_tol, int max_inv, double conv) {
  if (m != h->mass) set_mass_internal(h, m);
  const Level& F = h->lv[0];
  const long long c = F.count();
  const double diag = 4.0 + m;
  double2 lam = make_double2(0.0, 0.0), prev = lam;
  for (int k = 0; k < max_inv; ++k) {
    ck(h, wilson_D<double>(v, w, h->U64, diag, F.Lx, F.Lt, 1, true, h->s), "D dagger");
    mg_solve_info info{};
    solve_batch(h, w, t, 1, solve_tol, 100000, solver, &info);
    ck(h, norm2<double>(t, c, 1, h->partials, slot(h, S_T0), h->s), "norm");
    ck(h, scale_inv_sqrt<double>(t, v, slot(h, S_T0), c, 1, h->s), "normalise");
    ck(h, wilson_D<double>(v, w, h->U64, diag, F.Lx, F.Lt, 1, false, h->s), "D");
    ck(h, dot<double>(v, w, c, 1, h->partials, slot(h, S_T1), h->s), "dot");
    lam.x = read_scalar(h, S_T1);
    lam.y = h->hscal[1];
    if (k && std::hypot(lam.x - prev.x, lam.y - prev.y) <= conv * std::hypot(lam.x, lam.y)) break;
    prev = lam;
  }
  return lam;
}

// Root of the cubic Hermite interpolant of (m0, f0, d0), (m1, f1, d1) nearest
// m1 (Newton on the cubic from the Newton step of the second point).
double hermite_root(double m0, double f0, double d0, double m1, double f1, double d1) {
  const double hh = m1 - m0;
  auto p = [&](double x, double* dp) {
    const double u = (x - m0) / hh, u2 = u * u, u3 = u2 * u;
    const double h00 = 2 * u3 - 3 * u2 + 1, h10 = u3 - 2 * u2 + u, h01 = -2 * u3 + 3 * u2,
                 h11 = u3 - u2;
    const double g00 = 6 * u2 - 6 * u, g10 = 3 * u2 - 4 * u + 1, g01 = -6 * u2 + 6 * u,
                 g11 = 3 * u2 - 2 * u;
    *dp = (g00 * f0 + g01 * f1) / hh + g10 * d0 + g11 * d1;
    return h00 * f0 + hh * h10 * d0 + h01 * f1 + hh * h11 * d1;
  };
  double x = m1 - f1 / d1;
  for (int k = 0; k < 60; ++k) {
    double dp = 0.0;
    const double f = p(x, &dp);
    if (!(dp != 0.0)) break;
    const double dx = f / dp;
    x -= dx;
    if (std::fabs(dx) <= 1e-16 * std::fabs(x)) break;
  }
  return x;
}

// One adaptive pass on level lr of src (Sec. 3; the contract is mg_refine's).
// noise: the random starts of the levels below lr for the refined Nv.  The
// arguments are validated by the caller.
mg_status refine_core(mg_handle* src, int lr, const void* e0, int ncycles, const double2* noise,
                      cudaStream_t stream, mg_handle** out, double* rho, void* e_out) {
  *out = nullptr;
  mg_params P = src->p;
  P.Nv[lr] += 1;
  std::memset(P.refine_levels, 0, sizeof(P.refine_levels));
  const Level& S = src->lv[lr];
  const long long c = S.count();
  const int nv0 = S.Nv;
  const Level& SC = src->lv[lr + 1];
  const long long cc = SC.count();
  // scratch: E = the nv0 current vectors of the level, then the surviving
  // error e''; then two level vectors, then nv0 coarse indicator vectors
  void* E = nullptr;
  if (cudaMalloc(&E, ((size_t)(nv0 + 3) * c + (size_t)nv0 * cc) * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "device allocation failed (refine scratch)";
    return MG_ERR_NOMEM;
  }
  double2* Ek = (double2*)E;
  double2* e = Ek + (size_t)nv0 * c;
  double2* t = e + c;
  double2* z = t + c;
  double2* dind = z + c;
  // 1. V-cycles of the level on the error, no source (Sec. 3)
  double a0 = 0.0, a1 = 0.0;
  mg_status st = guarded(src, [&]() {
    ck(src, cudaMemcpyAsync(e, e0, c * sizeof(double2), cudaMemcpyDeviceToDevice, src->s), "copy e0");
    apply_level<double>(src, lr, e, t, 1, W_F64);
    ck(src, dot<double>(e, t, c, 1, src->partials, slot(src, S_T0), src->s), "dot");
    a0 = read_scalar(src, S_T0);
    for (int k = 0; k < ncycles; ++k) {
      if (k) apply_level<double>(src, lr, e, t, 1, W_F64);
      vcycle<double>(src, lr, t, z, 1);
      ck(src, axpby<double>(-1.0, z, 1.0, e, c, 1, src->s), "e -= V A e");
    }
    apply_level<double>(src, lr, e, t, 1, W_F64);
    ck(src, dot<double>(e, t, c, 1, src->partials, slot(src, S_T0), src->s), "dot");
    a1 = read_scalar(src, S_T0);
    if (!(a0 > 0.0) || !(a1 == a1)) fail(src, MG_ERR_BREAKDOWN, "refine: |e0|_A = 0 or non-finite error");
    if (e_out) ck(src, cudaMemcpyAsync(e_out, e, c * sizeof(double2), cudaMemcpyDeviceToDevice, src->s), "copy e''");
    // the level's current vectors as full level vectors: v_k = P (1_{s=k} + 1_{s=Nv+k})
    std::vector<double2> ind((size_t)nv0 * cc, make_double2(0.0, 0.0));
    for (int k = 0; k < nv0; ++k)
      for (long long j = 0; j < SC.V; ++j) {
        ind[(size_t)k * cc + j * SC.n + k] = make_double2(1.0, 0.0);
        ind[(size_t)k * cc + j * SC.n + nv0 + k] = make_double2(1.0, 0.0);
      }
    ck(src, cudaMemcpyAsync(dind, ind.data(), ind.size() * sizeof(double2), cudaMemcpyHostToDevice, src->s), "upload");
    ck(src, prolong_op<double>(dind, Ek, S.Vst64, S.Lx, S.Lt, S.bx, S.bt, S.n / 2, nv0, nv0, false, src->s), "unpack");
    sync(src);
  });
  if (st != MG_OK) {
    g_last_error = src->err;
    cudaFree(E);
    return st;
  }
  if (rho) *rho = std::pow(std::sqrt(a1 / a0), 1.0 / ncycles);
  // 2. the refined hierarchy: finer levels copied, this level from E, coarser
  //    levels set up again on the new coarse operators
  mg_handle* h = new (std::nothrow) mg_handle();
  if (!h) { cudaFree(E); g_last_error = "host allocation failed"; return MG_ERR_NOMEM; }
  h->p = P;
  h->s = stream;
  h->L = src->L;
  h->R = src->R;
  h->prof_on = src->prof_on;
  st = guarded(h, [&]() {
    set_geometry(h);
    init_runtime(h);
    allocate_storage(h);
    h->mass = src->mass;
    const long long V = h->lv[0].V;
    auto copy = [&](void* d, const void* sp, size_t bytes) {
      ck(h, cudaMemcpyAsync(d, sp, bytes, cudaMemcpyDeviceToDevice, h->s), "refine copy");
    };
    copy(h->U64, src->U64, 2 * V * sizeof(double2));
    copy(h->U32, src->U32, 2 * V * sizeof(float2));
    size_t pos = 0;
    for (int l = 0; l + 1 < h->L; ++l) {
      Level& L = h->lv[l];
      const Level& Sl = src->lv[l];
      if (l <= lr) {
        copy(L.eta, Sl.eta, (size_t)L.count() * sizeof(double2));
        L.lambda_max = Sl.lambda_max;
        L.omega_relax = Sl.omega_relax;
      }
      if (l < lr) {
        const size_t nvs = (size_t)L.V * 2 * L.Nv * (L.n / 2);
        copy(L.Vst64, Sl.Vst64, nvs * sizeof(double2));
        copy(L.Vst32, Sl.Vst32, nvs * sizeof(float2));
        galerkin_next(h, l);
      } else if (l == lr) {
        build_level(h, l, nullptr, E);
      } else {
        build_level(h, l, noise + pos, nullptr);
        pos += (size_t)(L.Nv + 2) * L.count();
      }
    }
    set_mass_internal(h, src->mass);
  });
  cudaFree(E);
  if (st != MG_OK) {
    g_last_error = h->err;
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return MG_OK;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

mg_status mg_params_default(mg_params* p, int Lx, int Lt) {
  if (!p) return MG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->Lx = Lx;
  p->Lt = Lt;
  p->nlevels = 2;
  p->block[0][0] = p->block[0][1] = 4;
  p->Nv[0] = 4;
  p->setup_sweeps = 8;
  p->power_iters = 30;
  p->omega_mr = 0.8;
  p->coarsest_tol = 1e-13;
  p->coarsest_refine_max = 12;
  p->inner_coarsest_refine = 1;
  p->vcycle_coarse_bf16 = 1;
  p->max_rhs = 1;
  p->reliable_delta = 0.1;
  p->coarsest_reuse = 0;
  p->profile = 0;
  p->coarsest_dense_max = 16384;
  p->coarsest_gj_tcgen05 = 0;
  p->refine_cycles = 30;
  p->autotune = 1;
  p->remass_quadratic = 1;
  return MG_OK;
}

size_t mg_setup_noise_len(const mg_params* p) {
  if (!p || p->nlevels < 1 || p->nlevels > MG_MAX_LEVELS) return 0;
  long long lx = p->Lx, lt = p->Lt;
  for (int l = 0; l + 1 < p->nlevels; ++l) {
    const int bx = p->block[l][0], bt = p->block[l][1];
    if (bx <= 0 || bt <= 0 || lx % bx || lt % bt) return 0;
    lx /= bx; lt /= bt;
  }
  size_t tot = noise_len_from(p, 0);
  const int np = refine_count(p);
  for (int k = 0; k < np; ++k) {
    const int lr = p->refine_levels[k] - 1;
    if (lr < 0 || lr + 1 >= p->nlevels) return 0;
    const mg_params q = after_passes(p, k + 1);
    tot += (size_t)level_size(&q, lr) + noise_len_from(&q, lr + 1);
  }
  return tot;
}

mg_status mg_setup(const void* gauge, double mass, const mg_params* params, void* stream,
                   mg_handle** out) {
  if (!out) { g_last_error = "out is NULL"; return MG_ERR_ARG; }
  *out = nullptr;
  std::string msg;
  mg_status v = validate(params, msg);
  if (v != MG_OK) { g_last_error = msg; return v; }
  if (!gauge) { g_last_error = "gauge is NULL"; return MG_ERR_ARG; }
  mg_handle* h = new (std::nothrow) mg_handle();
  if (!h) { g_last_error = "host allocation failed"; return MG_ERR_NOMEM; }
  h->p = normalized(*params);
  h->s = (cudaStream_t)stream;
  h->L = params->nlevels;
  h->R = params->max_rhs;
  h->prof_on = params->profile != 0;
  mg_status st = guarded(h, [&]() {
    const mg_params& P = h->p;
    set_geometry(h);
    init_runtime(h);
    allocate_storage(h);
    // links
    const long long V = h->lv[0].V;
    ck(h, link_unitarity(gauge, 2 * V, slot(h, S_T0), h->s), "unitarity");
    const double dev = read_scalar(h, S_T0);
    if (!(dev <= 1e-12)) fail(h, MG_ERR_ARG, "gauge links are not unit modulus (|U|-1 = " + std::to_string(dev) + ")");
    ck(h, fold_links<double>(gauge, h->U64, P.Lx, P.Lt, h->s), "fold");
    ck(h, fold_links<float>(gauge, h->U32, P.Lx, P.Lt, h->s), "fold");
    h->mass = mass;
    // adaptive setup, level by level (Sec. 3)
    const double2* noise = (const double2*)P.setup_noise;
    size_t pos = 0;
    for (int l = 0; l + 1 < h->L; ++l) {
      build_level(h, l, noise + pos, nullptr);
      pos += (size_t)(h->lv[l].Nv + 2) * h->lv[l].count();
    }
    set_mass_internal(h, mass);
    // adaptive passes (Sec. 3), each replacing the hierarchy in place
    std::vector<double> rhos;
    const int np = refine_count(params);
    for (int k = 0; k < np; ++k) {
      const int lr = params->refine_levels[k] - 1;
      const mg_params q = after_passes(params, k + 1);
      const double2* e0 = noise + pos;
      pos += (size_t)level_size(&q, lr);
      const double2* tail = noise + pos;
      pos += noise_len_from(&q, lr + 1);
      mg_handle* nh = nullptr;
      double rho = 0.0;
      const mg_status rs = refine_core(h, lr, e0, params->refine_cycles, tail, h->s, &nh, &rho, nullptr);
      if (rs != MG_OK) fail(h, rs, "adaptive pass " + std::to_string(k + 1) + ": " + g_last_error);
      std::swap(*h, *nh);
      free_all(nh);
      delete nh;
      rhos.push_back(rho);
    }
    h->refine_rho = rhos;
    if (params->autotune) autotune_fine(h);
  });
  if (st != MG_OK) {
    g_last_error = h->err;
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return MG_OK;
}

mg_status mg_setup_bytes(const mg_params* params, long long* resident, long long* peak) {
  std::string msg;
  mg_status v = validate(params, msg);
  if (v != MG_OK) { g_last_error = msg; return v; }
  auto dry = [](const mg_params& q, long long* temp) {
    mg_handle tmp;
    tmp.p = q;
    tmp.L = q.nlevels;
    tmp.R = q.max_rhs;
    tmp.dry = true;
    set_geometry(&tmp);
    allocate_storage(&tmp);
    *temp = setup_temp_bytes(&tmp);
    return tmp.bytes;
  };
  long long temp = 0;
  long long res = dry(normalized(after_passes(params, 0)), &temp);
  long long top = res + temp;
  const int np = refine_count(params);
  for (int k = 0; k < np; ++k) {
    // the pass holds the previous hierarchy, the new one with its set-up
    // temporaries, and its scratch (Nv + 3 level vectors, Nv coarse vectors)
    const int lr = params->refine_levels[k] - 1;
    const mg_params prev = after_passes(params, k);
    const long long res_k = dry(after_passes(params, k + 1), &temp);
    const long long scratch = ((long long)(prev.Nv[lr] + 3) * level_size(&prev, lr) +
                               (long long)prev.Nv[lr] * level_size(&prev, lr + 1)) * 16;
    top = std::max(top, res + res_k + temp + scratch);
    res = res_k;
  }
  if (resident) *resident = res;
  if (peak) *peak = top;
  return MG_OK;
}

mg_status mg_device_bytes(const mg_handle* h, long long* bytes) {
  if (!h || !bytes) return MG_ERR_ARG;
  *bytes = h->bytes;
  return MG_OK;
}

mg_status mg_clone(const mg_handle* src, double mass, void* stream, mg_handle** out) {
  if (!src || !out) return MG_ERR_ARG;
  *out = nullptr;
  mg_handle* h = new (std::nothrow) mg_handle();
  if (!h) { g_last_error = "host allocation failed"; return MG_ERR_NOMEM; }
  h->p = src->p;
  h->p.profile = 0;
  h->s = (cudaStream_t)stream;
  h->L = src->L;
  h->R = src->R;
  mg_status st = guarded(h, [&]() {
    set_geometry(h);
    init_runtime(h);
    allocate_storage(h);
    const long long V = h->lv[0].V;
    auto copy = [&](void* d, const void* sp, size_t bytes) {
      ck(h, cudaMemcpyAsync(d, sp, bytes, cudaMemcpyDeviceToDevice, h->s), "clone copy");
    };
    copy(h->U64, src->U64, 2 * V * sizeof(double2));
    copy(h->U32, src->U32, 2 * V * sizeof(float2));
    for (int l = 0; l + 1 < h->L; ++l) {
      Level& L = h->lv[l];
      const Level& S = src->lv[l];
      const size_t nv = (size_t)L.V * 2 * L.Nv * (L.n / 2);
      copy(L.Vst64, S.Vst64, nv * sizeof(double2));
      copy(L.Vst32, S.Vst32, nv * sizeof(float2));
      copy(L.eta, S.eta, (size_t)L.count() * sizeof(double2));
      L.lambda_max = S.lambda_max;
      L.omega_relax = S.omega_relax;
    }
    h->smooth = src->smooth;           // the damping found for the source is kept
    h->smooth_cond = src->smooth_cond;
    if (h->p.remass_quadratic && src->g_built) {
      for (int l = 1; l < h->L; ++l) {
        const size_t ab = (size_t)h->lv[l].V * 9 * h->lv[l].n * h->lv[l].n * sizeof(double2);
        copy(h->lv[l].G0, src->lv[l].G0, ab);
        copy(h->lv[l].G1, src->lv[l].G1, ab);
      }
      h->g_built = true;
    }
    set_mass_internal(h, mass);
  });
  if (st != MG_OK) {
    g_last_error = h->err;
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return MG_OK;
}

mg_status mg_refine(mg_handle* src, int level, const void* e0, int ncycles, const void* noise,
                    void* stream, mg_handle** out, double* rho, void* e_out) {
  if (src && src->smooth != 0.0) {
    src->err = "mg_refine: not available with smoothed aggregation";
    return MG_ERR_ARG;
  }
  if (!out) { g_last_error = "out is NULL"; return MG_ERR_ARG; }
  *out = nullptr;
  if (!src || !e0 || ncycles < 1 || level < 1 || level >= src->L) {
    g_last_error = "invalid refine arguments (level must be in [1, nlevels - 1], ncycles >= 1)";
    return MG_ERR_ARG;
  }
  const int lr = level - 1;
  if (!noise && lr + 2 < src->L) { g_last_error = "noise is NULL but coarser levels are relaxed"; return MG_ERR_ARG; }
  mg_params P = src->p;
  P.Nv[lr] += 1;
  std::memset(P.refine_levels, 0, sizeof(P.refine_levels));
  P.setup_noise = noise ? noise : (const void*)src;   // a non-NULL placeholder when nothing is read
  std::string msg;
  mg_status v = validate(&P, msg);
  if (v != MG_OK) { g_last_error = msg; return v; }
  return refine_core(src, lr, e0, ncycles, (const double2*)noise, (cudaStream_t)stream, out, rho,
                     e_out);
}

mg_status mg_gauge_metropolis(double* theta, int Lx, int Lt, double beta, double eps, int sweeps,
                              long long first_sweep, unsigned long long seed, void* stream,
                              long long* accepted) {
  if (!theta || Lx < 2 || Lt < 2 || Lx % 2 || Lt % 2 || sweeps < 0 || first_sweep < 0 ||
      !(eps > 0.0) || (long long)Lx * Lt > (1LL << 31)) {
    g_last_error = "invalid Metropolis arguments";
    return MG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "device allocation failed";
    return MG_ERR_NOMEM;
  }
  unsigned long long n = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(n), s);
  if (e == cudaSuccess) e = gauge_metropolis(theta, Lx, Lt, beta, eps, sweeps, first_sweep, seed, d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, d, sizeof(n), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) {
    g_last_error = std::string("Metropolis: ") + cudaGetErrorString(e);
    return MG_ERR_CUDA;
  }
  if (accepted) *accepted = (long long)n;
  return MG_OK;
}

mg_status mg_gauge_links(const double* theta, void* U, int Lx, int Lt, void* stream) {
  if (!theta || !U || Lx < 1 || Lt < 1) { g_last_error = "invalid arguments"; return MG_ERR_ARG; }
  cudaError_t e = links_from_angles(theta, U, 2LL * Lx * Lt, (cudaStream_t)stream);
  if (e != cudaSuccess) { g_last_error = cudaGetErrorString(e); return MG_ERR_CUDA; }
  return MG_OK;
}

mg_status mg_critical_mass(mg_handle* h, double m_hi, double m_lo, const void* v0, double safety,
                           double newton_below, double newton_floor, int max_evals,
                           double* m_crit, double* slope, int* evals) {
  if (!h || !v0 || !m_crit || !(m_hi > m_lo) || !(safety > 0.0 && safety < 1.0) ||
      !(newton_below > newton_floor && newton_floor > 0.0) || max_evals < 1 || h->L < 2) {
    if (h) h->err = "invalid critical-mass arguments";
    g_last_error = "invalid critical-mass arguments";
    return MG_ERR_ARG;
  }
  const long long c = h->lv[0].count();
  void* buf = nullptr;
  if (cudaMalloc(&buf, 3 * c * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "device allocation failed (critical-mass scratch)";
    return MG_ERR_NOMEM;
  }
  double2* v = (double2*)buf;
  double2* w = v + c;
  double2* t = w + c;
  int n_ev = 0;
  bool found = false;
  double root = 0.0, root_slope = 0.0;
  const int solver = MG_SOLVER_MGCG_FP64;
  const double solve_tol = 1e-9, conv = 1e-10;
  const int max_inv = 60;
  mg_status st = guarded(h, [&]() {
    ck(h, norm2<double>(v0, c, 1, h->partials, slot(h, S_T0), h->s), "norm");
    ck(h, scale_inv_sqrt<double>(v0, v, slot(h, S_T0), c, 1, h->s), "normalise");
    double m = m_hi;
    while (m > m_lo && n_ev < max_evals && !found) {
      const EigH e = nearest_eig_H(h, m, v, w, t, solver, solve_tol, max_inv, conv);
      ++n_ev;
      const double mu = std::fabs(e.lam);
      if (mu < newton_below && std::fabs(e.slope) > 1e-3) {
        // Newton steps aimed at |lam| = newton_floor on the same side (no
        // solve closer to the singular point), then the root of the cubic
        // Hermite interpolant of the last two points
        double pm = m, pl = e.lam, ps = e.slope, qm = m, ql = e.lam, qs = e.slope;
        int npts = 1;
        bool ok = true;
        for (int k = 0; k < 40 && std::fabs(ql) > 1.5 * newton_floor && n_ev < max_evals; ++k) {
          const double target = ql > 0 ? newton_floor : -newton_floor;
          const double mn = qm - (ql - target) / qs;
          if (!(m - 4.0 * mu / std::fabs(e.slope) <= mn && mn <= m + 1e-15)) { ok = false; break; }
          const EigH f = nearest_eig_H(h, mn, v, w, t, solver, solve_tol, max_inv, conv);
          ++n_ev;
          if (std::fabs(f.lam) > 0.75 * std::fabs(ql) || std::fabs(f.slope) < 1e-3) { ok = false; break; }
          const bool crossed = (f.lam > 0) != (ql > 0);   // the root is now bracketed
          pm = qm; pl = ql; ps = qs;
          qm = mn; ql = f.lam; qs = f.slope;
          ++npts;
          if (crossed) break;
        }
        if (ok) {
          root = npts >= 2 ? hermite_root(pm, pl, ps, qm, ql, qs) : qm - ql / qs;
          root_slope = qs;
          // the exact shift: a real eigenvalue lam_D of D(qm) vanishes at qm - lam_D
          const double2 ld = nearest_eig_D(h, qm, v, w, t, solver, solve_tol, max_inv, 1e-13);
          ++n_ev;
          if (std::fabs(ld.y) <= 1e-8 * std::fabs(ld.x) + 1e-13 &&
              std::fabs(qm - ld.x - root) <= 0.5 * std::fabs(qm - root) + 1e-12)
            root = qm - ld.x;
          found = root <= m + 1e-15 && root >= m - 4.0 * mu / std::fabs(e.slope);
          if (found) break;
        }
      }
      m -= safety * mu;
    }
  });
  cudaFree(buf);
  if (evals) *evals = n_ev;
  if (st != MG_OK) { g_last_error = h->err; return st; }
  if (!found) {
    h->err = "no crossing above m_lo within max_evals";
    g_last_error = h->err;
    return MG_ERR_NOCONV;
  }
  *m_crit = root;
  if (slope) *slope = root_slope;
  return MG_OK;
}

int mg_stencil_tunings(mg_stencil_tuning* out, int max) {
  std::vector<StencilTuning> t(std::max(0, max));
  const int n = stencil_tunings(t.data(), max);
  for (int k = 0; k < n && k < max && out; ++k) {
    mg_stencil_tuning& o = out[k];
    o.precision = t[k].precision == 0 ? MG_PREC_F64 : MG_PREC_F32;
    o.Lx = t[k].Lx; o.Lt = t[k].Lt; o.nrhs = t[k].nrhs;
    o.tx = t[k].tx; o.ty = t[k].ty; o.rows_per_thread = t[k].rpt;
    o.tried = t[k].tried; o.admitted = t[k].admitted;
    o.us_chosen = t[k].us_best; o.us_default = t[k].us_default;
  }
  return n;
}

mg_status mg_get_refine_rho(const mg_handle* h, double* rho, int max, int* count) {
  if (!h || (max > 0 && !rho)) return MG_ERR_ARG;
  const int n = (int)h->refine_rho.size();
  for (int k = 0; k < n && k < max; ++k) rho[k] = h->refine_rho[k];
  if (count) *count = n;
  return MG_OK;
}

mg_status mg_set_mass(mg_handle* h, double mass) {
  if (!h) return MG_ERR_ARG;
  return guarded(h, [&]() { set_mass_internal(h, mass); });
}

// Bounded device-side waits of the tensor-core kernels report through a flag;
// one that ran out leaves the results invalid and the device state undefined.
void check_device_waits(mg_handle* h) {
  int flag = 0;
  ck(h, coarse_tc_take_error(&flag), "read the wait flag");
  if (flag) {
    h->poisoned = true;
    fail(h, MG_ERR_TIMEOUT, "tcgen05 coarse apply: a completion wait ran out (results invalid)");
  }
}

mg_status mg_solve(mg_handle* h, const void* b, void* x, int nrhs, double tol, int maxiter,
                   int solver, mg_solve_info* info) {
  if (!h) return MG_ERR_ARG;
  if (!b || !x || nrhs < 1 || !(tol > 0.0) || maxiter < 1) { h->err = "invalid solve arguments"; return MG_ERR_ARG; }
  if (h->L < 2 && solver != MG_SOLVER_CG_FP64) { h->err = "multigrid solvers need nlevels >= 2"; return MG_ERR_ARG; }
  mg_status worst = MG_OK;
  mg_status st = guarded(h, [&]() {
    const long long n = h->lv[0].count();
    for (int k0 = 0; k0 < nrhs; k0 += h->R) {
      const int nb = std::min(h->R, nrhs - k0);
      auto t0 = std::chrono::steady_clock::now();
      mg_status one = solve_batch(h, (const double2*)b + k0 * n, (double2*)x + k0 * n, nb, tol,
                                  maxiter, solver, info ? info + k0 : nullptr);
      sync(h);
      auto t1 = std::chrono::steady_clock::now();
      if (info)
        for (int k = 0; k < nb; ++k)
          info[k0 + k].milliseconds = std::chrono::duration<double, std::milli>(t1 - t0).count();
      if (one != MG_OK && worst == MG_OK) worst = one;
    }
    check_device_waits(h);
  });
  return st != MG_OK ? st : worst;
}

mg_status mg_apply_D(mg_handle* h, const void* in, void* out, int nrhs, int dagger, int precision) {
  if (!h) return MG_ERR_ARG;
  if (!in || !out || nrhs < 1 || (precision != MG_PREC_F64 && precision != MG_PREC_F32)) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    const Level& F = h->lv[0];
    if (precision == MG_PREC_F64)
      ck(h, wilson_D<double>(in, out, h->U64, 4.0 + h->mass, F.Lx, F.Lt, nrhs, dagger != 0, h->s), "wilson_D");
    else
      ck(h, wilson_D<float>(in, out, h->U32, 4.0 + h->mass, F.Lx, F.Lt, nrhs, dagger != 0, h->s), "wilson_D");
  });
}

mg_status mg_apply_A(mg_handle* h, const void* in, void* out, int nrhs, int precision) {
  if (!h) return MG_ERR_ARG;
  if (!in || !out || nrhs < 1 || (precision != MG_PREC_F64 && precision != MG_PREC_F32)) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    if (precision == MG_PREC_F64) apply_level<double>(h, 0, in, out, nrhs, W_F64);
    else apply_level<float>(h, 0, in, out, nrhs, W_F32);
  });
}

mg_status mg_apply_coarse(mg_handle* h, int level, const void* in, void* out, int nrhs, int precision) {
  if (!h) return MG_ERR_ARG;
  if (level < 2 || level > h->L || !in || !out || nrhs < 1 || precision < 0 || precision > 2) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    if (precision == MG_PREC_F64) apply_level<double>(h, level - 1, in, out, nrhs, W_F64);
    else apply_level<float>(h, level - 1, in, out, nrhs, precision == MG_PREC_F32 ? W_F32 : W_BF16);
  });
}

mg_status mg_set_coarse_tensor_kernel(int kind) {
  if (kind != 0 && kind != 1) return MG_ERR_ARG;
  set_coarse_tensor_kernel(kind);
  return MG_OK;
}

mg_status mg_restrict(mg_handle* h, int level, const void* fine_in, void* coarse_out, int nrhs, int precision) {
  if (!h) return MG_ERR_ARG;
  if (level < 1 || level >= h->L || !fine_in || !coarse_out || nrhs < 1 || (precision != MG_PREC_F64 && precision != MG_PREC_F32)) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  const bool sm = level == 1 && h->smooth != 0.0;
  if (sm && nrhs > h->R) { h->err = "smoothed restriction: nrhs above max_rhs"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    Level& L = h->lv[level - 1];
    const void* in = fine_in;
    if (precision == MG_PREC_F64) {
      if (sm) {                        // P_s^dagger r = P^dagger (r - omega A r)
        apply_level<double>(h, 0, fine_in, L.w64[3], nrhs, W_F64, ep_lincomb(-h->smooth, fine_in, 1.0));
        in = L.w64[3];
      }
      ck(h, restrict_op<double>(in, coarse_out, L.Vst64, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nrhs, h->s), "restrict");
    } else {
      if (sm) {
        apply_level<float>(h, 0, fine_in, L.w32[3], nrhs, W_F32, ep_lincomb(-h->smooth, fine_in, 1.0));
        in = L.w32[3];
      }
      ck(h, restrict_op<float>(in, coarse_out, L.Vst32, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nrhs, h->s), "restrict");
    }
  });
}

mg_status mg_prolong(mg_handle* h, int level, const void* coarse_in, void* fine_out, int nrhs, int precision) {
  if (!h) return MG_ERR_ARG;
  if (level < 1 || level >= h->L || !coarse_in || !fine_out || nrhs < 1 || (precision != MG_PREC_F64 && precision != MG_PREC_F32)) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  const bool sm = level == 1 && h->smooth != 0.0;
  if (sm && nrhs > h->R) { h->err = "smoothed prolongation: nrhs above max_rhs"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    Level& L = h->lv[level - 1];
    if (precision == MG_PREC_F64) {
      void* p = sm ? L.w64[3] : fine_out;
      ck(h, prolong_op<double>(coarse_in, p, L.Vst64, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nrhs, false, h->s), "prolong");
      if (sm)                          // P_s e = p - omega A p
        apply_level<double>(h, 0, p, fine_out, nrhs, W_F64, ep_lincomb(-h->smooth, p, 1.0));
    } else {
      void* p = sm ? L.w32[3] : fine_out;
      ck(h, prolong_op<float>(coarse_in, p, L.Vst32, L.Lx, L.Lt, L.bx, L.bt, L.n / 2, L.Nv, nrhs, false, h->s), "prolong");
      if (sm)
        apply_level<float>(h, 0, p, fine_out, nrhs, W_F32, ep_lincomb(-h->smooth, p, 1.0));
    }
  });
}

mg_status mg_vcycle(mg_handle* h, const void* in, void* out, int precision) {
  if (!h) return MG_ERR_ARG;
  if (!in || !out || h->L < 2 || (precision != MG_PREC_F64 && precision != MG_PREC_F32)) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  return guarded(h, [&]() {
    if (precision == MG_PREC_F64) vcycle<double>(h, 0, in, out);
    else vcycle<float>(h, 0, in, out);
  });
}

mg_status mg_coarsest_solve(mg_handle* h, const void* in, void* out) {
  if (!h) return MG_ERR_ARG;
  if (!in || !out || h->L < 2) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  return guarded(h, [&]() { coarsest_solve64(h, (const double2*)in, (double2*)out, h->n_refine, 1); });
}

mg_status mg_get_smoothing(const mg_handle* h, double* omega, double* cond) {
  if (!h) return MG_ERR_ARG;
  if (omega) *omega = h->smooth;
  if (cond) *cond = h->smooth_cond;
  return MG_OK;
}

mg_status mg_get_coarsest_info(const mg_handle* h, int* dense, int* steps, double* test_residual) {
  if (!h || h->L < 2) return MG_ERR_ARG;
  if (dense) *dense = h->dense ? 1 : 0;
  if (steps) *steps = h->dense ? h->n_refine : h->ccg_iters;
  if (test_residual) *test_residual = h->coarsest_test_res;
  return MG_OK;
}

mg_status mg_get_coarsest_reuse(const mg_handle* h, int* inner, int* reuses) {
  if (!h || h->L < 2) return MG_ERR_ARG;
  if (inner) *inner = h->n_inner;
  if (reuses) *reuses = h->inverse_reuses;
  return MG_OK;
}

mg_status mg_get_level(const mg_handle* h, int level, int* Lx, int* Lt, int* ndof, int* Nv) {
  if (!h || level < 1 || level > h->L) return MG_ERR_ARG;
  const Level& L = h->lv[level - 1];
  if (Lx) *Lx = L.Lx;
  if (Lt) *Lt = L.Lt;
  if (ndof) *ndof = L.n;
  if (Nv) *Nv = level < h->L ? L.Nv : 0;
  return MG_OK;
}

}  // extern "C"

// ----- allocation-free fused A with <x, A x> -----------------------------------
// Reduction scratch for mg_apply_A_dot_noalloc: 64 tickets (as doubles) plus
// 2 x 608 partial sums -- the layout of the handle's reduction workspace.
namespace {
constexpr int NOALLOC_BLOCKS = 608;
constexpr int NOALLOC_DOUBLES = 64 + 2 * NOALLOC_BLOCKS;
constexpr int NOALLOC_MAX_DEVICES = 64;
// device address of the array per device ordinal; threads that make their first
// call on a device at the same time both look it up and store the same value
std::atomic<double*> g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

extern "C" mg_status mg_apply_A_dot_noalloc(mg_handle* h, const void* in, void* out,
                                            double* xAx) {
  if (!h) return MG_ERR_ARG;
  if (!in || !out || !xAx) { h->err = "invalid arguments"; return MG_ERR_ARG; }
  const Level& F = h->lv[0];
  if (wilson_A_ctas(F.Lx, F.Lt, true) > NOALLOC_BLOCKS) {
    h->err = "mg_apply_A_dot_noalloc: lattice needs " + std::to_string(wilson_A_ctas(F.Lx, F.Lt, true)) +
             " thread blocks, more than the " + std::to_string(NOALLOC_BLOCKS) +
             " the library-held scratch holds";
    return MG_ERR_ARG;
  }
  return guarded(h, [&]() {
    int dev = 0;
    ck(h, cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(h, MG_ERR_ARG, "device ordinal out of range");
    double* ws = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!ws) {
      // once per device, with that device current: the device address of the array
      void* p = nullptr;
      ck(h, cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
      ws = (double*)p;
      g_noalloc_ptr[dev].store(ws, std::memory_order_release);
    }
    // the tickets must start at zero (the last block of a reduction clears them,
    // but a previous kernel may have been interrupted)
    ck(h, cudaMemsetAsync(ws, 0, 64 * sizeof(double), h->s), "clear tickets");
    Epilogue ep;
    ep.dot_ws = ws;
    ep.dot_out = xAx;
    ck(h, wilson_A<double>(in, out, h->U64, 4.0 + h->mass, F.Lx, F.Lt, 1, ep, h->s), "wilson_A");
  });
}

// Gather of Vst [V][2][Nv][h] into [Nv][V][2h] (complex128).
__global__ void k_vst_to_vectors(const double2* __restrict__ Vst, double2* __restrict__ out, int V,
                                 int Nv, int h) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)V * 2 * Nv * h;
  if (idx >= tot) return;
  const int a = (int)(idx % h), k = (int)((idx / h) % Nv), c = (int)((idx / ((long long)h * Nv)) % 2);
  const long long i = idx / (2LL * Nv * h);
  out[((long long)k * V + i) * 2 * h + c * h + a] = Vst[idx];
}

extern "C" {

mg_status mg_get_null_vectors(const mg_handle* hc, int level, void* out) {
  mg_handle* h = const_cast<mg_handle*>(hc);
  if (!h || level < 1 || level >= h->L || !out) return MG_ERR_ARG;
  return guarded(h, [&]() {
    const Level& L = h->lv[level - 1];
    const long long tot = (long long)L.V * 2 * L.Nv * (L.n / 2);
    k_vst_to_vectors<<<(unsigned)((tot + 255) / 256), 256, 0, h->s>>>(L.Vst64, (double2*)out, L.V, L.Nv, L.n / 2); count_launch();
    ck(h, cudaGetLastError(), "gather");
  });
}

mg_status mg_get_coarse_op(const mg_handle* hc, int level, void* out) {
  mg_handle* h = const_cast<mg_handle*>(hc);
  if (!h || level < 2 || level > h->L || !out) return MG_ERR_ARG;
  return guarded(h, [&]() {
    const Level& L = h->lv[level - 1];
    ck(h, cudaMemcpyAsync(out, L.A64, (size_t)L.V * 9 * L.n * L.n * sizeof(double2), cudaMemcpyDeviceToDevice, h->s), "copy");
  });
}

mg_status mg_get_smoother(const mg_handle* h, int level, double* out4) {
  if (!h || level < 1 || level >= h->L || !out4) return MG_ERR_ARG;
  const Level& L = h->lv[level - 1];
  out4[0] = L.c0;
  out4[1] = L.c1;
  out4[2] = L.lambda_max;
  out4[3] = L.omega_relax;
  return MG_OK;
}

mg_status mg_block_map(int Lx, int Lt, int bx, int bt, int32_t* coarse, int32_t* offset, void* stream) {
  if (Lx < 1 || Lt < 1 || bx < 1 || bt < 1 || Lx % bx || Lt % bt || !coarse || !offset) {
    g_last_error = "invalid block map arguments";
    return MG_ERR_ARG;
  }
  cudaError_t e = block_map(Lx, Lt, bx, bt, coarse, offset, (cudaStream_t)stream);
  if (e != cudaSuccess) { g_last_error = cudaGetErrorString(e); return MG_ERR_CUDA; }
  return MG_OK;
}

unsigned long long mg_kernel_launches(void) { return launch_count(); }

mg_status mg_profile_enable(mg_handle* h, int on) {
  if (!h) return MG_ERR_ARG;
  h->prof_on = on != 0;
  for (int f = 0; f < MG_KF_COUNT; ++f) h->prof_used[f] = 0;
  return MG_OK;
}

mg_status mg_profile_read(mg_handle* h, int family, double* total_ms, long long* calls) {
  if (!h || family < 0 || family >= MG_KF_COUNT) return MG_ERR_ARG;
  return guarded(h, [&]() {
    sync(h);
    double tot = 0.0;
    for (size_t u = 0; u < h->prof_used[family]; ++u) {
      float ms = 0.f;
      ck(h, cudaEventElapsedTime(&ms, h->prof_ev[family][2 * u], h->prof_ev[family][2 * u + 1]), "event time");
      tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (calls) *calls = (long long)h->prof_used[family];
  });
}

const char* mg_last_error(const mg_handle* h) {
  return h ? h->err.c_str() : g_last_error.c_str();
}

void mg_destroy(mg_handle* h) {
  if (!h) return;
  free_all(h);
  delete h;
}

}  // extern "C"
