// Quenched U(1) gauge fields on the device: the checkerboard Metropolis update
// of the Wilson plaquette action S = -beta sum_p Re U_p (the paper's gauge
// ensembles, Sec. 4), with counter-based uniforms so that a host program
// drawing the same counters makes the same decisions.
//
// Uniforms: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11) at counter (site, half-sweep low,
// half-sweep high, 0) and key (seed low, seed high), half-sweep = 4 sweep +
// 2 mu + parity; u_prop from words 0 and 1, u_acc from words 2 and 3, each a
// double in [0, 1) made exactly from 27 + 26 bits.  Angle arithmetic is
// rounded operation by operation (no contraction), in the order of the host
// generator, so both sides accept from the same values (up to the last bit of
// cos and exp).
#include "common.cuh"
#include "kernels.h"

namespace mgk {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double uniform53(unsigned hi, unsigned lo) {
  return __dmul_rn(__dadd_rn(__dmul_rn((double)(hi >> 5), 67108864.0), (double)(lo >> 6)),
                   1.1102230246251565e-16);   // 2^-53
}

// One half-sweep: every link of direction mu whose other coordinate has the
// given parity (they share no plaquette).  theta: [2][Lt][Lx] angles.
__global__ void k_metropolis_half(double* __restrict__ theta, int Lx, int Lt, double beta,
                                  double eps, int mu, int parity, unsigned long long half,
                                  uint2 key, unsigned long long* accepted) {
  constexpr double PI = 3.141592653589793, TWO_PI = 6.283185307179586;
  const int n = Lx * Lt / 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < n;
  bool acc = false;
  if (active) {
    int x, t;
    if (mu == 0) {
      t = 2 * (i / Lx) + parity;
      x = i % Lx;
    } else {
      const int hx = Lx / 2;
      t = i / hx;
      x = 2 * (i % hx) + parity;
    }
    const int V = Lx * Lt;
    const double* th0 = theta;
    const double* th1 = theta + V;
    const int xp = x + 1 == Lx ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
    const int tp = t + 1 == Lt ? 0 : t + 1, tm = t == 0 ? Lt - 1 : t - 1;
    double a, b, cur;
    if (mu == 0) {   // theta0(x,t) enters p(x,t) = theta0 + a and p(x,t-1) = b - theta0
      a = __dsub_rn(__dsub_rn(th1[t * Lx + xp], th0[tp * Lx + x]), th1[t * Lx + x]);
      b = __dsub_rn(__dadd_rn(th0[tm * Lx + x], th1[tm * Lx + xp]), th1[tm * Lx + x]);
      cur = th0[t * Lx + x];
    } else {         // theta1(x,t) enters p(x,t) = a - theta1 and p(x-1,t) = b + theta1
      a = __dadd_rn(__dsub_rn(th0[t * Lx + x], th0[tp * Lx + x]), th1[t * Lx + xp]);
      b = __dsub_rn(__dsub_rn(th0[t * Lx + xm], th0[tp * Lx + xm]), th1[t * Lx + xm]);
      cur = th1[t * Lx + x];
    }
    const uint4 r = philox4x32_10(
        make_uint4((unsigned)(t * Lx + x), (unsigned)half, (unsigned)(half >> 32), 0u), key);
    const double up = uniform53(r.x, r.y), ua = uniform53(r.z, r.w);
    const double nw = __dadd_rn(cur, __dmul_rn(eps, __dsub_rn(__dmul_rn(2.0, up), 1.0)));
    double so, sn;
    if (mu == 0) {
      so = __dadd_rn(cos(__dadd_rn(cur, a)), cos(__dsub_rn(b, cur)));
      sn = __dadd_rn(cos(__dadd_rn(nw, a)), cos(__dsub_rn(b, nw)));
    } else {
      so = __dadd_rn(cos(__dsub_rn(a, cur)), cos(__dadd_rn(b, cur)));
      sn = __dadd_rn(cos(__dsub_rn(a, nw)), cos(__dadd_rn(b, nw)));
    }
    const double ds = __dmul_rn(-beta, __dsub_rn(sn, so));
    acc = ua < exp(fmin(-ds, 0.0));
    if (acc) {   // map to [-pi, pi): fmod, shifted into [0, 2 pi) like a floored modulo
      double m = fmod(__dadd_rn(nw, PI), TWO_PI);
      if (m != 0.0) {
        if (m < 0.0) m = __dadd_rn(m, TWO_PI);
      } else {
        m = 0.0;
      }
      theta[mu * V + t * Lx + x] = __dsub_rn(m, PI);
    }
  }
  const unsigned votes = __ballot_sync(0xffffffffu, acc);
  if (accepted && (threadIdx.x & 31) == 0 && votes)
    atomicAdd(accepted, (unsigned long long)__popc(votes));
}

__global__ void k_links_from_angles(const double* __restrict__ theta, double2* __restrict__ U,
                                    long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s, c;
  sincos(theta[i], &s, &c);
  U[i] = make_double2(c, s);
}

cudaError_t gauge_metropolis(double* theta, int Lx, int Lt, double beta, double eps, int sweeps,
                             long long first_sweep, unsigned long long seed,
                             unsigned long long* accepted, cudaStream_t s) {
  const int n = Lx * Lt / 2;
  const uint2 key = make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32));
  for (long long sw = first_sweep; sw < first_sweep + sweeps; ++sw)
    for (int mu = 0; mu < 2; ++mu)
      for (int parity = 0; parity < 2; ++parity) {
        k_metropolis_half<<<(n + 255) / 256, 256, 0, s>>>(
            theta, Lx, Lt, beta, eps, mu, parity, (unsigned long long)(4 * sw + 2 * mu + parity),
            key, accepted);
        count_launch();
      }
  return cudaGetLastError();
}

cudaError_t links_from_angles(const double* theta, void* U, long long n, cudaStream_t s) {
  k_links_from_angles<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, (double2*)U, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgk
