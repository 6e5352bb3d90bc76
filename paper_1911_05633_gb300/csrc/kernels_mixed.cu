// Mixed-precision contractions of Eqs. P_MM and S_MM: the same three stages as
// the FP64 kernels, computed in FP32 with FP32 accumulation from FP64 inputs and
// written back as FP64 (complex128).  The surrounding rows of the sweep (lattice
// and tau transforms, the W solve, the exchange term) stay in FP64.
#include <cuda_runtime.h>

#include "kernels.h"
#include "smem_limit.h"
#include "mixed.h"
#include "ktimer.h"

namespace gw {

namespace {

__device__ __forceinline__ float2 f2(double2 z) { return make_float2((float)z.x, (float)z.y); }
// c + a * b
__device__ __forceinline__ float2 cfmaf_(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// c + a * conj(b)
__device__ __forceinline__ float2 cfmacf_(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.y, b.x, fmaf(-a.x, b.y, c.y)));
}
__device__ __forceinline__ float2 rfmaf_(float r, float2 b, float2 c) {
  return make_float2(fmaf(r, b.x, c.x), fmaf(r, b.y, c.y));
}

constexpr int kKCm = 16;

// P contraction (Eq. P_MM) in FP32; one block per (entry, tau node), mirrored node
// written as the conjugate when C is symmetric in (L, L'').
__global__ void k_polarizability_f32(const DevEntry* __restrict__ ent, const float* __restrict__ C,
                                     const double2* __restrict__ G, double2* __restrict__ out, int n_tau, int spin,
                                     int mirror_tau) {
  extern __shared__ float2 smf[];
  const int e = blockIdx.x;
  const int it = blockIdx.y;
  const DevEntry E = ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  const int im = n_tau - 1 - it;
  float2* G1 = smf;
  float2* G2 = G1 + na * nb;
  float2* X = G2 + na * nb;
  float2* Y = X + kKCm * na * nb;
  const double2* Gin = G + E.off_orb * n_tau;
  for (int x = threadIdx.x; x < na * nb; x += blockDim.x) {
    G1[x] = f2(Gin[(long long)it * na * nb + x]);
    G2[x] = f2(Gin[(long long)im * na * nb + x]);
  }
  __syncthreads();
  const float* Ca = C + E.ca;
  const float* Cb = C + E.cb;
  double2* Pout = out + E.off_pb * n_tau;
  const float ms = -(float)spin;
  const bool mirror = mirror_tau && (im != it);
  for (int k0 = 0; k0 < Ka; k0 += kKCm) {
    const int kc = min(kKCm, Ka - k0);
    for (int x = threadIdx.x; x < kc * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;
      const float* c = Ca + (long long)(k0 + K) * na * na;
      float2 acc = make_float2(0.f, 0.f);
      for (int L = 0; L < na; ++L) acc = rfmaf_(c[L * na + L2], G1[L * nb + L1], acc);
      X[x] = acc;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kc * nb * nb; x += blockDim.x) {
      const int K = x / (nb * nb);
      const int r = x - K * nb * nb;
      const int L1 = r / nb, L3 = r - L1 * nb;
      const float2* xk = X + K * na * nb;
      float2 acc = make_float2(0.f, 0.f);
      for (int L2 = 0; L2 < na; ++L2) acc = cfmacf_(xk[L2 * nb + L1], G2[L2 * nb + L3], acc);
      Y[x] = acc;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kc * Kb; x += blockDim.x) {
      const int K = x / Kb, Kp = x - (x / Kb) * Kb;
      const float2* y = Y + K * nb * nb;
      const float* c = Cb + (long long)Kp * nb * nb;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 0; j < nb * nb; ++j) acc = rfmaf_(c[j], y[j], acc);
      const long long o = (long long)(k0 + K) * Kb + Kp;
      const double2 r = make_double2(ms * acc.x, ms * acc.y);
      Pout[(long long)it * Ka * Kb + o] = r;
      if (mirror) Pout[(long long)im * Ka * Kb + o] = make_double2(r.x, -r.y);
    }
    __syncthreads();
  }
}

// Sigma contraction (Eq. S_MM, dynamic part) in FP32; one block per (entry, tau node).
__global__ void k_self_energy_f32(const DevEntry* __restrict__ ent, const float* __restrict__ C,
                                  const double2* __restrict__ G, const double2* __restrict__ W,
                                  double2* __restrict__ out, int n_tau) {
  extern __shared__ float2 smf[];
  const int e = blockIdx.x;
  const int s = blockIdx.y;
  const DevEntry E = ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  float2* Gs = smf;
  float2* B = Gs + na * nb;
  float2* D = B + kKCm * nb * nb;
  float2* Ws = D + kKCm * na * nb;  // [kKCm][Kb]
  const double2* Gin = G + E.off_orb * n_tau + (long long)s * na * nb;
  for (int x = threadIdx.x; x < na * nb; x += blockDim.x) Gs[x] = f2(Gin[x]);
  const double2* Wg = W + E.off_pb * n_tau + (long long)s * Ka * Kb;
  const float* Ca = C + E.ca;
  const float* Cb = C + E.cb;
  float2 acc = make_float2(0.f, 0.f);
  const int own = threadIdx.x;
  for (int k0 = 0; k0 < Ka; k0 += kKCm) {
    const int kc = min(kKCm, Ka - k0);
    __syncthreads();
    for (int x = threadIdx.x; x < kc * Kb; x += blockDim.x) Ws[x] = f2(Wg[(long long)k0 * Kb + x]);
    __syncthreads();
    for (int x = threadIdx.x; x < kc * nb * nb; x += blockDim.x) {
      const int K = x / (nb * nb);
      const int j = x - K * nb * nb;
      const float2* w = Ws + K * Kb;
      float2 t = make_float2(0.f, 0.f);
      for (int Kp = 0; Kp < Kb; ++Kp) t = rfmaf_(Cb[(long long)Kp * nb * nb + j], w[Kp], t);
      B[x] = t;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kc * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;
      const float2* bk = B + K * nb * nb + L1 * nb;
      float2 t = make_float2(0.f, 0.f);
      for (int L3 = 0; L3 < nb; ++L3) t = cfmaf_(Gs[L2 * nb + L3], bk[L3], t);
      D[x] = t;
    }
    __syncthreads();
    if (own < na * nb) {
      const int L = own / nb, L1 = own - (own / nb) * nb;
      for (int K = 0; K < kc; ++K) {
        const float* c = Ca + (long long)(k0 + K) * na * na + L * na;
        const float2* dk = D + K * na * nb;
        for (int L2 = 0; L2 < na; ++L2) acc = rfmaf_(c[L2], dk[L2 * nb + L1], acc);
      }
    }
  }
  if (own < na * nb) {
    double2* o = out + E.off_orb * n_tau + (long long)s * na * nb;
    o[own] = make_double2(-(double)acc.x, -(double)acc.y);
  }
}

size_t smem_p32(const HostPlan& h) {
  size_t m = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      size_t na = h.n_orb[s], nb = h.n_orb[t];
      m = std::max(m, (2 * na * nb + kKCm * na * nb + kKCm * nb * nb) * sizeof(float2));
    }
  return m;
}

size_t smem_s32(const HostPlan& h) {
  size_t m = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      size_t na = h.n_orb[s], nb = h.n_orb[t], Kb = h.n_prod[t];
      m = std::max(m, (na * nb + kKCm * nb * nb + kKCm * na * nb + kKCm * Kb) * sizeof(float2));
    }
  return m;
}

}  // namespace

gw_status mixed_init(MixedPlan& m, const HostPlan& h, const std::vector<DevEntry>&) {
  std::vector<float> Cf(h.C_packed.begin(), h.C_packed.end());
  cudaError_t e = cudaMalloc((void**)&m.d_Cf, Cf.size() * sizeof(float));
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return GW_ERR_OOM;
  }
  e = cudaMemcpy(m.d_Cf, Cf.data(), Cf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  m.smem_P = smem_p32(h);
  m.smem_S = smem_s32(h);
  if (gw::raise_smem_limit(k_polarizability_f32, (int)m.smem_P) !=
          cudaSuccess ||
      gw::raise_smem_limit(k_self_energy_f32, (int)m.smem_S) !=
          cudaSuccess) {
    set_last_error("cudaFuncSetAttribute failed for the mixed kernels");
    return GW_ERR_UNSUPPORTED;
  }
  m.ready = true;
  return GW_OK;
}

void mixed_free(MixedPlan& m) {
  if (m.d_Cf) cudaFree(m.d_Cf);
  m.d_Cf = nullptr;
  m.ready = false;
}

gw_status mixed_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double*,
                               const double2* G_R, double2* P_R, int* d_status, cudaStream_t st) {
  if (!m.ready) { set_last_error("mixed path not initialised"); return GW_ERR_ARG; }
  const int nt_eff = h.c_symmetric ? (h.n_tau + 1) / 2 : h.n_tau;
  dim3 grid(h.n_entries(), nt_eff);
  {
    gw::TimedLaunch tl_("k_polarizability_f32", st);
    k_polarizability_f32<<<grid, 256, m.smem_P, st>>>(d_ent, m.d_Cf, G_R, P_R, h.n_tau, h.spin, h.c_symmetric);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_last_error(std::string("k_polarizability_f32: ") + cudaGetErrorString(e)); return GW_ERR_CUDA; }
  return GW_OK;
}

gw_status mixed_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double*,
                            const double2* G_R, const double2* Wt_R, double2* Sig_R, int* d_status, cudaStream_t st) {
  if (!m.ready) { set_last_error("mixed path not initialised"); return GW_ERR_ARG; }
  dim3 grid(h.n_entries(), h.n_tau);
  {
    gw::TimedLaunch tl_("k_self_energy_f32", st);
    k_self_energy_f32<<<grid, 256, m.smem_S, st>>>(d_ent, m.d_Cf, G_R, Wt_R, Sig_R, h.n_tau);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_last_error(std::string("k_self_energy_f32: ") + cudaGetErrorString(e)); return GW_ERR_CUDA; }
  return GW_OK;
}

}  // namespace gw
