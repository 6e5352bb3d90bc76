// Linearised quasiparticle energies on the device: Sigma_c(i w) ~ S0 + i w S1 through the
// two lowest positive fermionic frequencies, then the eigenvalues of
// A^{-1} (H + Sigma_x^h + S0^h - mu) A^{-1} + mu with A = (I - S1^h)^{1/2} (h: Hermitian part).
// One block per momentum; the Hermitian eigenproblems by cyclic Jacobi in shared memory.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "dyson.h"
#include "ktimer.h"
#include "smem_limit.h"

namespace gw {

namespace {

__device__ __forceinline__ double2 cmulq(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 conjq(double2 a) { return make_double2(a.x, -a.y); }

// Sum over the block, returned to every thread.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

struct Rot {
  int p, q;
  double c, s;
  double2 e;  // a_pq / |a_pq|
};

// Hermitian a (N x N at stride Np, Np = N rounded up to even) -> J^H a J diagonal by cyclic
// Jacobi: per sweep Np - 1 rounds of Np / 2 disjoint pairs (the round-robin order), each
// round one rotation per pair, J_pq = D P with D = diag(1, e^{-i phi}) making a_pq real
// and P the real Jacobi rotation of the 2 x 2 block.  v <- v J when v is given.  Stops when
// the off-diagonal squared norm is below 1e-30 of the total (at most max_sweeps sweeps).
__device__ void jacobi_heev(double2* a, double2* v, int N, int Np, int max_sweeps, Rot* rot, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x, half = Np / 2;
  double t = 0.0;
  for (int x = tid; x < N * N; x += nt) {
    const double2 z = a[(x / N) * Np + x % N];
    t += z.x * z.x + z.y * z.y;
  }
  const double total = block_sum(t, red);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    double o = 0.0;
    for (int x = tid; x < N * N; x += nt) {
      const int i = x / N, j = x % N;
      if (i != j) {
        const double2 z = a[i * Np + j];
        o += z.x * z.x + z.y * z.y;
      }
    }
    if (!(block_sum(o, red) > 1e-30 * total)) break;
    for (int r = 0; r < Np - 1; ++r) {
      if (tid < half) {
        Rot R;
        if (tid == 0) { R.p = Np - 1; R.q = r; }
        else { R.p = (r + tid) % (Np - 1); R.q = (r - tid + Np - 1) % (Np - 1); }
        R.c = 1.0;
        R.s = 0.0;
        R.e = make_double2(1.0, 0.0);
        if (R.p < N && R.q < N) {
          const double2 apq = a[R.p * Np + R.q];
          const double m = hypot(apq.x, apq.y);
          if (m > 0.0) {
            R.e = make_double2(apq.x / m, apq.y / m);
            const double zeta = (a[R.q * Np + R.q].x - a[R.p * Np + R.p].x) / (2.0 * m);
            const double tt = fabs(zeta) > 1e150 ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            R.c = 1.0 / sqrt(1.0 + tt * tt);
            R.s = tt * R.c;
          }
        }
        rot[tid] = R;
      }
      __syncthreads();
      // rows p, q: a <- J^H a
      for (int x = tid; x < half * Np; x += nt) {
        const Rot R = rot[x / Np];
        if (R.s == 0.0) continue;
        const int j = x % Np;
        const double2 ap = a[R.p * Np + j], eq = cmulq(R.e, a[R.q * Np + j]);
        a[R.p * Np + j] = make_double2(R.c * ap.x - R.s * eq.x, R.c * ap.y - R.s * eq.y);
        a[R.q * Np + j] = make_double2(R.s * ap.x + R.c * eq.x, R.s * ap.y + R.c * eq.y);
      }
      __syncthreads();
      // columns p, q: a <- a J, v <- v J
      for (int x = tid; x < half * Np; x += nt) {
        const Rot R = rot[x / Np];
        if (R.s == 0.0) continue;
        const int i = x % Np;
        const double2 eb = conjq(R.e);
        double2 ap = a[i * Np + R.p], eq = cmulq(eb, a[i * Np + R.q]);
        a[i * Np + R.p] = make_double2(R.c * ap.x - R.s * eq.x, R.c * ap.y - R.s * eq.y);
        a[i * Np + R.q] = make_double2(R.s * ap.x + R.c * eq.x, R.s * ap.y + R.c * eq.y);
        if (v) {
          ap = v[i * Np + R.p];
          eq = cmulq(eb, v[i * Np + R.q]);
          v[i * Np + R.p] = make_double2(R.c * ap.x - R.s * eq.x, R.c * ap.y - R.s * eq.y);
          v[i * Np + R.q] = make_double2(R.s * ap.x + R.c * eq.x, R.s * ap.y + R.c * eq.y);
        }
      }
      __syncthreads();
    }
  }
}

// Hermitian part of element (i, j) of M (row-major N x N) at offset base.
__device__ __forceinline__ double2 herm_el(const double2* __restrict__ M, long long base, int N, int i, int j) {
  const double2 x = M[base + (long long)i * N + j], y = M[base + (long long)j * N + i];
  return make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
}

// One block per momentum k; Ainv: global scratch [N_k][N][N].
__global__ void __launch_bounds__(256) k_qp_energies(const double2* __restrict__ H, const double2* __restrict__ Sx,
                                                     const double2* __restrict__ Sc, int n_w, int i0, int i1,
                                                     double w0, double w1, double mu, int N, int max_sweeps,
                                                     double2* __restrict__ Ainv, double* __restrict__ E) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Np = (N + 1) & ~1;
  double2* a = reinterpret_cast<double2*>(smraw);  // [Np][Np]
  double2* v = a + (size_t)Np * Np;                // [Np][Np]
  __shared__ Rot rot[kQpMaxN / 2];
  __shared__ double red[8];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long k = blockIdx.x;
  const long long NN = (long long)N * N;
  const long long b0 = (k * n_w + i0) * NN, b1 = (k * n_w + i1) * NN;
  // S1 = (Sc(i w1) - Sc(i w0)) / (i (w1 - w0)); S0 = Sc(i w0) - i w0 S1
  auto s1 = [&](int i, int j) -> double2 {
    if (!Sc) return make_double2(0.0, 0.0);
    const double2 d1 = Sc[b1 + (long long)i * N + j], d0 = Sc[b0 + (long long)i * N + j];
    const double f = 1.0 / (w1 - w0);
    return make_double2((d1.y - d0.y) * f, -(d1.x - d0.x) * f);  // (d1 - d0) / i
  };
  auto s0 = [&](int i, int j) -> double2 {
    if (!Sc) return make_double2(0.0, 0.0);
    const double2 d0 = Sc[b0 + (long long)i * N + j], m = s1(i, j);
    return make_double2(d0.x + w0 * m.y, d0.y - w0 * m.x);  // d0 - i w0 S1
  };
  // B = I - S1^h, V = I (padding rows and columns zero)
  for (int x = tid; x < Np * Np; x += nt) {
    const int i = x / Np, j = x % Np;
    double2 z = make_double2(0.0, 0.0);
    if (i < N && j < N) {
      const double2 p = s1(i, j), q = s1(j, i);
      z = make_double2((i == j ? 1.0 : 0.0) - 0.5 * (p.x + q.x), -0.5 * (p.y - q.y));
    }
    a[x] = z;
    v[x] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  jacobi_heev(a, v, N, Np, max_sweeps, rot, red);
  // Ainv = U diag(lambda^{-1/2}) U^H
  for (int x = tid; x < N * N; x += nt) {
    const int i = x / N, j = x % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) {
      const double f = rsqrt(a[l * Np + l].x);
      acc = make_double2(fma(f, cmulq(v[i * Np + l], conjq(v[j * Np + l])).x, acc.x),
                         fma(f, cmulq(v[i * Np + l], conjq(v[j * Np + l])).y, acc.y));
    }
    Ainv[k * NN + x] = acc;
  }
  __syncthreads();
  // X = H^h + Sx^h + S0^h - mu into v, T = Ainv X into a, Y = T Ainv into v, then a = Y^h
  for (int x = tid; x < N * N; x += nt) {
    const int i = x / N, j = x % N;
    double2 z = herm_el(H, k * NN, N, i, j);
    if (Sx) {
      const double2 y = herm_el(Sx, k * NN, N, i, j);
      z.x += y.x;
      z.y += y.y;
    }
    const double2 p = s0(i, j), q = s0(j, i);
    z.x += 0.5 * (p.x + q.x) - (i == j ? mu : 0.0);
    z.y += 0.5 * (p.y - q.y);
    v[i * Np + j] = z;
  }
  __syncthreads();
  for (int x = tid; x < N * N; x += nt) {
    const int i = x / N, j = x % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) {
      const double2 m = cmulq(Ainv[k * NN + (long long)i * N + l], v[l * Np + j]);
      acc.x += m.x;
      acc.y += m.y;
    }
    a[i * Np + j] = acc;
  }
  __syncthreads();
  for (int x = tid; x < N * N; x += nt) {
    const int i = x / N, j = x % N;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < N; ++l) {
      const double2 m = cmulq(a[i * Np + l], Ainv[k * NN + (long long)l * N + j]);
      acc.x += m.x;
      acc.y += m.y;
    }
    v[i * Np + j] = acc;
  }
  __syncthreads();
  for (int x = tid; x < Np * Np; x += nt) {
    const int i = x / Np, j = x % Np;
    double2 z = make_double2(0.0, 0.0);
    if (i < N && j < N) {
      const double2 p = v[i * Np + j], q = v[j * Np + i];
      z = make_double2(0.5 * (p.x + q.x), 0.5 * (p.y - q.y));
    }
    a[x] = z;
  }
  __syncthreads();
  jacobi_heev(a, nullptr, N, Np, max_sweeps, rot, red);
  // ascending order: rank of each eigenvalue (ties by index)
  for (int i = tid; i < N; i += nt) {
    const double li = a[i * Np + i].x;
    int r = 0;
    for (int j = 0; j < N; ++j) {
      const double lj = a[j * Np + j].x;
      r += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    E[k * N + r] = li + mu;
  }
}

}  // namespace

gw_status qp_energies(const HostPlan& h, const double2* H, const double2* Sigx, const double2* Sigc, double mu,
                      double2* ainv_scratch, double* E, cudaStream_t st) {
  const int N = h.n_orb_total();
  int i0 = -1, i1 = -1;
  for (int n = 0; n < h.n_omega; ++n) {
    if (h.omega_idx[n] == 0) i0 = n;
    if (h.omega_idx[n] == 1) i1 = n;
  }
  if (i0 < 0 || i1 < 0) {
    set_last_error("the sampled fermionic frequencies do not include n = 0 and n = 1");
    return GW_ERR_ARG;
  }
  if (N > kQpMaxN) {
    set_last_error("quasiparticle energies: more orbitals than the compiled limit");
    return GW_ERR_UNSUPPORTED;
  }
  const int Np = (N + 1) & ~1;
  const size_t smem = 2 * (size_t)Np * Np * sizeof(double2);
  cudaError_t e = raise_smem_limit(k_qp_energies, smem);
  if (e != cudaSuccess) {
    set_last_error(std::string("quasiparticle energies: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  {
    TimedLaunch tl_("k_qp_energies", st);
    k_qp_energies<<<h.n_k, 256, smem, st>>>(H, Sigx, Sigc, h.n_omega, i0, i1, M_PI / h.beta, 3.0 * M_PI / h.beta, mu,
                                            N, 60, ainv_scratch, E);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("k_qp_energies: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
