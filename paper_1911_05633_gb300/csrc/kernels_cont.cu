// Eq. sf_9 on the device: the continued fraction through Sigma(k, i w_n) on the stored
// grid's non-negative sampled frequencies, evaluated at real frequencies w + i delta.
// One thread per (k, element).  Declarations in dyson.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dyson.h"
#include "kernels.h"
#include "ktimer.h"

namespace gw {

namespace {

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a / b with the scaling of Smith's method (the larger component of b divides first)
__device__ __forceinline__ double2 cdivc(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

// g_0(z_i) = Sigma(z_i); g_p(z_i) = (g_{p-1}(z_{p-1}) - g_{p-1}(z_i)) / ((z_i - z_{p-1}) g_{p-1}(z_i)),
// a_p = g_p(z_p), z_i = i w_i; then a_0 / (1 + a_1 (w - z_0) / (1 + ... a_M (w - z_{M-1}) / 1)).
__global__ void k_continue_sigma(const double2* __restrict__ S, const int* __restrict__ slot,
                                 const double* __restrict__ zw, int P, int n_w, long long NN, int n_k,
                                 const double* __restrict__ wr, int n_real, double delta, double2* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_k * NN) return;
  const long long k = t / NN, x = t - (t / NN) * NN;
  double2 g[kContMax];
  for (int p = 0; p < P; ++p) g[p] = S[(k * n_w + slot[p]) * NN + x];
  for (int p = 1; p < P; ++p) {
    const double2 gp = g[p - 1];
    for (int i = p; i < P; ++i) {
      const double2 num = make_double2(gp.x - g[i].x, gp.y - g[i].y);
      const double dz = zw[i] - zw[p - 1];  // z_i - z_{p-1} = i (w_i - w_{p-1})
      g[i] = cdivc(num, make_double2(-dz * g[i].y, dz * g[i].x));
    }
  }
  for (int r = 0; r < n_real; ++r) {
    double2 A = make_double2(1.0, 0.0);
    for (int p = P - 1; p >= 1; --p) {
      const double2 d = make_double2(wr[r], delta - zw[p - 1]);  // w + i delta - i w_{p-1}
      const double2 q = cdivc(cmulc(g[p], d), A);
      A = make_double2(1.0 + q.x, q.y);
    }
    out[(k * n_real + r) * NN + x] = cdivc(g[0], A);
  }
}

// [(w_r + i delta + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, w_r)] for block b = k n_real + r.
__global__ void k_retarded_build(const double2* __restrict__ H, const double2* __restrict__ Sx,
                                 const double2* __restrict__ Sc, const double* __restrict__ wr, double delta,
                                 double mu, int N, int n_real, double2* __restrict__ M) {
  const long long b = blockIdx.x;
  const long long k = b / n_real;
  const int r = (int)(b - k * n_real);
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
      re += wr[r] + mu;
      im += delta;
    }
    M[b * NN + x] = make_double2(re, im);
  }
}

// A[b] = -(1/pi) Im Tr M_b^{-1}, one warp per block b.
__global__ void k_trace_spectral(const double2* __restrict__ G, int N, long long n_b, double* __restrict__ A) {
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= n_b) return;
  const int lane = threadIdx.x & 31;
  const long long NN = (long long)N * N;
  double t = 0.0;
  for (int i = lane; i < N; i += 32) t += G[b * NN + (long long)i * N + i].y;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) A[b] = -t / M_PI;
}

}  // namespace

gw_status spectral_function(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx,
                            const double2* Sigc_w, int n_real, const double* w_real_host, double delta, double mu,
                            double* A, int* d_status, cudaStream_t st) {
  const int N = h.n_orb_total();
  const long long nb = (long long)h.n_k * n_real, NN = (long long)N * N;
  const size_t need = (size_t)nb * NN * sizeof(double2) + (size_t)nb * N * sizeof(int) + (size_t)n_real * sizeof(double) + 256;
  if (need > d.spec_bytes) {
    if (d.spec) cudaFree(d.spec);
    d.spec = nullptr;
    d.spec_bytes = 0;
    if (cudaMalloc(&d.spec, need) != cudaSuccess) {
      set_last_error("spectral function: scratch allocation failed");
      return GW_ERR_OOM;
    }
    d.spec_bytes = need;
  }
  double2* M = static_cast<double2*>(d.spec);
  int* perm = reinterpret_cast<int*>(M + nb * NN);
  double* d_wr = reinterpret_cast<double*>(perm + nb * N + (((nb * N) & 1) ? 1 : 0));
  cudaError_t e = cudaMemcpyAsync(d_wr, w_real_host, n_real * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // w_real is the caller's host memory
  if (e != cudaSuccess) {
    set_last_error(std::string("spectral function: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  {
    TimedLaunch tl_("k_retarded_build", st);
    k_retarded_build<<<(unsigned)nb, 256, 0, st>>>(H, Sigx, Sigc_w, d_wr, delta, mu, N, n_real, M);
  }
  {
    TimedLaunch tl_("k_gj_inverse", st);
    k_gj_inverse<<<(unsigned)nb, 512, 2 * (size_t)N * sizeof(double2), st>>>(M, perm, N, NN, d_status);
  }
  {
    TimedLaunch tl_("k_trace_spectral", st);
    k_trace_spectral<<<(unsigned)((nb + 7) / 8), 256, 0, st>>>(M, N, nb, A);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("spectral function: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

gw_status continue_sigma(DysonPlan& d, const HostPlan& h, const double2* S, int n_real, const double* w_real_host,
                         double delta, double2* out, cudaStream_t st) {
  // the non-negative sampled frequencies, ascending
  std::vector<std::pair<int, int>> pts;
  for (int n = 0; n < h.n_omega; ++n)
    if (h.omega_idx[n] >= 0) pts.push_back({h.omega_idx[n], n});
  std::sort(pts.begin(), pts.end());
  const int P = (int)pts.size();
  if (P < 1 || P > kContMax) {
    set_last_error("continued fraction: 1 to 64 non-negative sampled frequencies needed");
    return GW_ERR_UNSUPPORTED;
  }
  std::vector<int> slot(P);
  std::vector<double> zw(P);
  for (int p = 0; p < P; ++p) {
    slot[p] = pts[p].second;
    zw[p] = (2.0 * pts[p].first + 1.0) * M_PI / h.beta;
  }
  // small per-call tables in one device buffer: slots, point frequencies, real frequencies
  const size_t need = (size_t)P * sizeof(int) + (size_t)(P + n_real) * sizeof(double) + 64;
  if (need > d.cont_bytes) {
    if (d.cont) cudaFree(d.cont);
    d.cont = nullptr;
    d.cont_bytes = 0;
    if (cudaMalloc(&d.cont, need) != cudaSuccess) {
      set_last_error("continued fraction: scratch allocation failed");
      return GW_ERR_OOM;
    }
    d.cont_bytes = need;
  }
  unsigned char* base = static_cast<unsigned char*>(d.cont);
  double* d_zw = reinterpret_cast<double*>(base);
  double* d_wr = d_zw + P;
  int* d_slot = reinterpret_cast<int*>(d_wr + n_real);
  cudaError_t e = cudaMemcpyAsync(d_zw, zw.data(), P * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_wr, w_real_host, n_real * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_slot, slot.data(), P * sizeof(int), cudaMemcpyHostToDevice, st);
  // the host vectors go out of scope on return: wait for the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_last_error(std::string("continued fraction: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  const int N = h.n_orb_total();
  const long long NN = (long long)N * N, tot = (long long)h.n_k * NN;
  {
    TimedLaunch tl_("k_continue_sigma", st);
    k_continue_sigma<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(S, d_slot, d_zw, P, h.n_omega, NN, h.n_k, d_wr,
                                                                     n_real, delta, out);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("k_continue_sigma: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
