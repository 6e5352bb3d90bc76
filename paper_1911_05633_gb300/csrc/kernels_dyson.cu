// Eq. G_1 (Dyson equation) on the device, G(k, tau) through Appendix A's inverse
// transform, and the particle number from G(k, beta-).  Declarations in dyson.h.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "dyson.h"
#include "kernels.h"
#include "ktimer.h"
#include "smem_limit.h"

namespace gw {

namespace {

__device__ __forceinline__ double2 cfma_d(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// [(i w_n + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, i w_n)] for block b = k n_w + n.
__global__ void k_dyson_build(const double2* __restrict__ H, const double2* __restrict__ Sx,
                              const double2* __restrict__ Sc, const double* __restrict__ w, double mu, int N, int n_w,
                              double2* __restrict__ M) {
  const long long b = blockIdx.x;
  const long long k = b / n_w;
  const int n = (int)(b - k * n_w);
  const long long NN = (long long)N * N;
  for (long long x = threadIdx.x; x < NN; x += blockDim.x) {
    const double2 h = H[k * NN + x];
    double re = -h.x, im = -h.y;
    if (Sx) {
      const double2 s = Sx[k * NN + x];
      re -= s.x;
      im -= s.y;
    }
    if (Sc) {
      const double2 c = Sc[b * NN + x];
      re -= c.x;
      im -= c.y;
    }
    if (x / N == x % N) {
      re += mu;
      im += w[n];
    }
    M[b * NN + x] = make_double2(re, im);
  }
}

// M1 = H + Sigma_x - mu of element x of momentum k
__device__ __forceinline__ double2 tail_m1(const double2* __restrict__ H, const double2* __restrict__ Sx, long long k,
                                           long long NN, long long x, bool diag, double mu) {
  const double2 h = H[k * NN + x];
  double2 m = make_double2(h.x - (diag ? mu : 0.0), h.y);
  if (Sx) {
    const double2 s = Sx[k * NN + x];
    m.x += s.x;
    m.y += s.y;
  }
  return m;
}

// G - 1/(i w) - M1/(i w)^2 = G + i/w + M1/w^2 (diagonal for the first term)
__device__ __forceinline__ double2 tail_rem(double2 g, double2 m1, double wn, bool diag) {
  const double iw2 = 1.0 / (wn * wn);
  return make_double2(fma(m1.x, iw2, g.x), fma(m1.y, iw2, g.y) + (diag ? 1.0 / wn : 0.0));
}

// G(k, tau_i) = sum_n T[i][n] rem(k, n) - 1/2 + M1 (2 tau_i - beta)/4; grid (k, chunk of
// 64 elements), each thread's remainders over n staged in shared memory.
__global__ void __launch_bounds__(64) k_green_tau(const double2* __restrict__ G, const double2* __restrict__ H,
                                                  const double2* __restrict__ Sx, const double* __restrict__ w,
                                                  const double2* __restrict__ T, const double* __restrict__ tau,
                                                  double beta, double mu, int N, int n_w, int n_tau,
                                                  double2* __restrict__ out) {
  extern __shared__ double2 rem[];  // [n_w][64]
  const long long k = blockIdx.x;
  const long long NN = (long long)N * N;
  const long long x = (long long)blockIdx.y * 64 + threadIdx.x;
  if (x >= NN) return;
  const bool diag = x / N == x % N;
  const double2 m1 = tail_m1(H, Sx, k, NN, x, diag, mu);
  for (int n = 0; n < n_w; ++n) rem[n * 64 + threadIdx.x] = tail_rem(G[(k * n_w + n) * NN + x], m1, w[n], diag);
  for (int i = 0; i < n_tau; ++i) {
    const double2* Ti = T + (long long)i * n_w;
    double2 acc = make_double2(0.0, 0.0);
    for (int n = 0; n < n_w; ++n) acc = cfma_d(Ti[n], rem[n * 64 + threadIdx.x], acc);
    const double f = (2.0 * tau[i] - beta) * 0.25;
    out[(k * n_tau + i) * NN + x] = make_double2(fma(m1.x, f, acc.x) - (diag ? 0.5 : 0.0), fma(m1.y, f, acc.y));
  }
}

// part[k] = Re Tr[-G(k, beta-)]: the last row of the inverse transform on the diagonal
// remainders, plus the tail at beta, -1/2 + M1 beta/4.  One block of 256 per k.
__global__ void __launch_bounds__(256) k_density_trace(const double2* __restrict__ G, const double2* __restrict__ H,
                                                       const double2* __restrict__ Sx, const double* __restrict__ w,
                                                       const double2* __restrict__ Tlast, double beta, double mu,
                                                       int N, int n_w, double* __restrict__ part) {
  __shared__ double red[8];
  const long long k = blockIdx.x;
  const long long NN = (long long)N * N;
  double acc = 0.0;
  for (int q = threadIdx.x; q < n_w * N; q += blockDim.x) {
    const int n = q / N, i = q - (q / N) * N;
    const long long x = (long long)i * N + i;
    const double2 r = tail_rem(G[(k * n_w + n) * NN + x], tail_m1(H, Sx, k, NN, x, true, mu), w[n], true);
    const double2 t = Tlast[n];
    acc += t.x * r.x - t.y * r.y;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const long long x = (long long)i * N + i;
    acc += fma(tail_m1(H, Sx, k, NN, x, true, mu).x, 0.25 * beta, -0.5);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    part[k] = -s;
  }
}

gw_status launch_ok(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace

gw_status dyson_init(DysonPlan& d, const HostPlan& h) {
  if (d.ready) return GW_OK;
  d.N = h.n_orb_total();
  d.n_w = h.n_omega;
  d.n_k = h.n_k;
  d.n_tau = h.n_tau;
  const size_t nb = (size_t)d.n_k * d.n_w;
  std::vector<double> w(d.n_w);
  for (int n = 0; n < d.n_w; ++n) w[n] = (2.0 * h.omega_idx[n] + 1.0) * M_PI / h.beta;
  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    d.bytes += bytes;
    return !src || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  const bool good = up((void**)&d.M, nullptr, nb * d.N * d.N * sizeof(double2)) &&
                    up((void**)&d.perm, nullptr, nb * d.N * sizeof(int)) &&
                    up((void**)&d.w, w.data(), w.size() * sizeof(double)) &&
                    up((void**)&d.tau, h.tau.data(), h.tau.size() * sizeof(double)) &&
                    up((void**)&d.part, nullptr, (size_t)d.n_k * sizeof(double)) &&
                    up((void**)&d.ainv, nullptr, (size_t)d.n_k * d.N * d.N * sizeof(double2));
  if (!good) {
    dyson_free(d);
    set_last_error("Dyson scratch allocation failed");
    return GW_ERR_OOM;
  }
  if ((size_t)d.n_w * 64 * sizeof(double2) > 227 * 1024 ||
      raise_smem_limit(k_green_tau, (int)((size_t)d.n_w * 64 * sizeof(double2))) != cudaSuccess) {
    dyson_free(d);
    set_last_error("Dyson transform: too many fermionic frequencies for shared memory");
    return GW_ERR_UNSUPPORTED;
  }
  if (uploads_landed() != cudaSuccess) {
    dyson_free(d);
    set_last_error("Dyson tables did not reach the device");
    return GW_ERR_CUDA;
  }
  d.ready = true;
  return GW_OK;
}

void dyson_free(DysonPlan& d) {
  void* ptrs[] = {d.M, d.perm, d.w, d.tau, d.part, d.ainv, d.cont, d.spec};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  d = DysonPlan{};
}

gw_status dyson_solve(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, const double2* Sigc,
                      double mu, int* d_status, cudaStream_t st) {
  (void)h;
  const int nb = d.n_k * d.n_w;
  {
    TimedLaunch tl_("k_dyson_build", st);
    k_dyson_build<<<nb, 256, 0, st>>>(H, Sigx, Sigc, d.w, mu, d.N, d.n_w, d.M);
  }
  gw_status s = launch_ok("k_dyson_build");
  if (s != GW_OK) return s;
  {
    TimedLaunch tl_("k_gj_inverse", st);
    k_gj_inverse<<<nb, 512, 2 * (size_t)d.N * sizeof(double2), st>>>(d.M, d.perm, d.N, (long long)d.N * d.N,
                                                                       d_status);
  }
  return launch_ok("k_gj_inverse");
}

gw_status dyson_to_tau(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, double mu,
                       const double2* T, double2* G_tau, cudaStream_t st) {
  const long long NN = (long long)d.N * d.N;
  dim3 g((unsigned)d.n_k, (unsigned)((NN + 63) / 64));
  {
    TimedLaunch tl_("k_green_tau", st);
    k_green_tau<<<g, 64, (size_t)d.n_w * 64 * sizeof(double2), st>>>(d.M, H, Sigx, d.w, T, d.tau, h.beta, mu, d.N,
                                                                      d.n_w, d.n_tau, G_tau);
  }
  return launch_ok("k_green_tau");
}

gw_status dyson_density(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, double mu,
                        const double2* Tlast, cudaStream_t st) {
  {
    TimedLaunch tl_("k_density_trace", st);
    k_density_trace<<<d.n_k, 256, 0, st>>>(d.M, H, Sigx, d.w, Tlast, h.beta, mu, d.N, d.n_w, d.part);
  }
  return launch_ok("k_density_trace");
}

}  // namespace gw
