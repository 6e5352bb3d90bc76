// Eq. G_1 on the device: G(k, i w_n) = [(i w_n + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, i w_n)]^{-1}
// for the sampled fermionic frequencies, G(k, tau) through the inverse transform of
// Appendix A with the two leading tail terms taken out, and the particle number from
// G(k, beta-).  Kernels in kernels_dyson.cu.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gw {

struct DysonPlan {
  bool ready = false;
  int N = 0, n_w = 0, n_k = 0, n_tau = 0;
  double2* M = nullptr;    // [n_k][n_w][N][N]: the matrices, then G(k, i w_n)
  int* perm = nullptr;     // [n_k * n_w][N] pivot rows of the inverse
  double* w = nullptr;     // [n_w] w_n = (2n + 1) pi / beta
  double* tau = nullptr;   // [n_tau]
  double* part = nullptr;  // [n_k] per-k traces for the particle number
  double2* ainv = nullptr;  // [n_k][N][N] scratch of the quasiparticle energies
  void* cont = nullptr;      // small tables of the continued fraction
  size_t cont_bytes = 0;
  void* spec = nullptr;      // matrices, pivots and frequencies of the spectral function
  size_t spec_bytes = 0;
  size_t bytes = 0;
};

gw_status dyson_init(DysonPlan& d, const HostPlan& h);
void dyson_free(DysonPlan& d);
// G(k, i w_n) into d.M (H, Sigx: [n_k][N][N]; Sigc: [n_k][n_w][N][N]; Sigx and Sigc may be null).
gw_status dyson_solve(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, const double2* Sigc,
                      double mu, int* d_status, cudaStream_t st);
// G(k, tau) [n_k][n_tau][N][N] from d.M; T: the inverse fermionic transform [n_tau][n_w].
gw_status dyson_to_tau(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, double mu,
                       const double2* T, double2* G_tau, cudaStream_t st);
// d.part[k] = Re Tr[-G(k, beta-)] from d.M; Tlast: the last row of the inverse transform.
gw_status dyson_density(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx, double mu,
                        const double2* Tlast, cudaStream_t st);

// Linearised quasiparticle energies E [n_k][N] ascending (kernels_qp.cu): Sigma_c from
// the sampled frequencies n = 0 and n = 1; ainv_scratch: [n_k][N][N] complex.  N <= kQpMaxN.
constexpr int kQpMaxN = 80;
gw_status qp_energies(const HostPlan& h, const double2* H, const double2* Sigx, const double2* Sigc, double mu,
                      double2* ainv_scratch, double* E, cudaStream_t st);

// Eq. sf_9: Sigma(k, w_r + i delta) [n_k][n_real][N][N] from Sigma(k, i w_n) [n_k][n_w][N][N]
// through the non-negative sampled frequencies (kernels_cont.cu); w_real on the host.
constexpr int kContMax = 64;
gw_status continue_sigma(DysonPlan& d, const HostPlan& h, const double2* S, int n_real, const double* w_real_host,
                         double delta, double2* out, cudaStream_t st);

// Eqs. sf_1, sf_7: A [n_k][n_real] = -(1/pi) Im Tr [(w + i delta + mu) - H - Sigma_x - Sigma_c(w)]^{-1}
// (kernels_cont.cu); Sigc_w [n_k][n_real][N][N] or null; w_real on the host.
gw_status spectral_function(DysonPlan& d, const HostPlan& h, const double2* H, const double2* Sigx,
                            const double2* Sigc_w, int n_real, const double* w_real_host, double delta, double mu,
                            double* A, int* d_status, cudaStream_t st);

}  // namespace gw
