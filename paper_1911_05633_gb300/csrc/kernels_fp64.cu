// FP64 kernels of the sweep: lattice Fourier gather/scatter over the pair list
// (Sec. 2), tau <-> i omega transforms (Appendix A grid), the P and Sigma
// contractions of Eqs. P_MM and S_MM, and the batched W solve of Eq. W_1.
//
// Complex numbers are double2 (re, im).  Every kernel is bounds-checked against
// the sizes it is given; launch shapes are computed by the C ABI in capi.cu.
#include <cuda_runtime.h>

#include "kernels.h"

namespace gw {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c + a * conj(b)
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.y, b.x, fma(-a.x, b.y, c.y)));
}
// c + conj(a) * b
__device__ __forceinline__ double2 cfma_conj_a(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + r * b (r real)
__device__ __forceinline__ double2 rfma(double r, double2 b, double2 c) {
  return make_double2(fma(r, b.x, c.x), fma(r, b.y, c.y));
}

// i^c v for a quarter-turn code c (0..3): a swap and sign flips of the bit patterns, no
// arithmetic (c = 1: (-y, x), 2: (-x, -y), 3: (y, -x)).
__device__ __forceinline__ double neg_if(double x, bool n) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)n << 63));
}
__device__ __forceinline__ double2 qmul(int c, double2 v) {
  const bool sw = c & 1;
  return make_double2(neg_if(sw ? v.y : v.x, c == 1 || c == 2), neg_if(sw ? v.x : v.y, c >= 2));
}

constexpr int kHoldK = 8;  // k points held in registers by the gather and scatter

// ---------------------------------------------------------------------------
// k -> R gather:  F_R[e][s][i][j] = scale * sum_k conj(ph[e][k]) (F_k - F_sub)[k][s][oa+i][ob+j]
// grid: (row atom a, slice); the block sweeps the band of rows of atom a across every
// column of the dense matrix, so that consecutive threads read consecutive columns; an
// element whose atom pair has no entry is skipped; an entry with a reduced product basis
// keeps its top-left K_a(e) x K_b(e).  With at most kHoldK k points the element's values
// are read once for all its entries; with quarter-turn phases each term is two additions.
// ---------------------------------------------------------------------------
template <bool MANY_K>
__global__ void k_gather_k_to_R(GatherArgs g) {
  const int a = blockIdx.x, s = blockIdx.y;
  const int ro = g.row_off[a];
  const int rows = g.row_off[a + 1] - ro;
  const int n_el = rows * g.ld;
  const bool hold = g.n_k_in <= kHoldK;
  for (int x = threadIdx.x + blockIdx.z * blockDim.x; x < n_el; x += blockDim.x * gridDim.z) {
    const int i = x / g.ld, col = x - i * g.ld;
    const int b = g.col_atom[col];
    const int j = col - g.row_off[b];
    const int p = a * g.n_atoms + b;
    const int e0 = g.pair_start[p], e1 = g.pair_start[p + 1];
    if (e0 == e1) continue;
    const long long in_el = (long long)(ro + i) * g.ld + col;
    auto value = [&](int kk) -> double2 {
      const int k = g.k_list ? g.k_list[kk] : kk;
      double2 v = g.F_k[(long long)kk * g.k_stride + (long long)s * g.s_stride + in_el];
      if (g.F_sub) {
        const double2 w = g.F_sub[(long long)k * g.sub_k_stride + (long long)s * g.sub_s_stride + in_el];
        v.x -= w.x;
        v.y -= w.y;
      }
      if (g.k_weight) {
        const double wk = g.k_weight[kk];
        v.x *= wk;
        v.y *= wk;
      }
      return v;
    };
    // conj(ph[e][k]) v added to acc (real part only for real_only)
    auto term_e = [&](int e, int kk, double2 v, double2& acc) {
      const int k = g.k_list ? g.k_list[kk] : kk;
      if (g.pcode) {  // conj(i^c) v = i^(4 - c) v
        const double2 t = qmul((4 - g.pcode[(long long)e * g.n_k + k]) & 3, v);
        acc.x += t.x;
        if (!g.real_only) acc.y += t.y;
      } else {
        const double2 c = g.phase[(long long)e * g.n_k + k];
        if (g.real_only) acc.x = fma(c.x, v.x, fma(c.y, v.y, acc.x));
        else acc = cfma_conj_a(c, v, acc);
      }
    };
    auto store = [&](int e, double2 acc) {
      const DevEntry& E = g.ent[e];
      const long long off = g.pb ? E.off_pb : E.off_orb;
      const int ce = g.pb ? E.Kb : E.nb, be = (g.pb ? E.Ka : E.na) * ce;
      if (g.scale != 1.0) {
        acc.x *= g.scale;
        acc.y *= g.scale;
      }
      g.F_R[off * g.out_n_slices + (long long)(g.out_slice0 + s) * be + i * ce + j] =
          make_double2(acc.x, g.real_only ? 0.0 : acc.y);
    };
    auto keeps = [&](int e) {
      const DevEntry& E = g.ent[e];
      return i < (g.pb ? E.Ka : E.na) && j < (g.pb ? E.Kb : E.nb);
    };
    if (MANY_K && !hold && e1 - e0 <= kHoldK) {
      // many k points: the element's values streamed once, in chunks, for all its entries
      double2 acc[kHoldK];
#pragma unroll
      for (int q = 0; q < kHoldK; ++q) acc[q] = make_double2(0.0, 0.0);
      for (int k0 = 0; k0 < g.n_k_in; k0 += kHoldK) {
        double2 vc[kHoldK];
#pragma unroll
        for (int u = 0; u < kHoldK; ++u)
          if (k0 + u < g.n_k_in) vc[u] = value(k0 + u);
#pragma unroll
        for (int q = 0; q < kHoldK; ++q)
          if (q < e1 - e0 && keeps(e0 + q))
#pragma unroll
            for (int u = 0; u < kHoldK; ++u)
              if (k0 + u < g.n_k_in) term_e(e0 + q, k0 + u, vc[u], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kHoldK; ++q)
        if (q < e1 - e0 && keeps(e0 + q)) store(e0 + q, acc[q]);
      continue;
    }
    double2 vh[kHoldK];
    if (hold)
#pragma unroll
      for (int kk = 0; kk < kHoldK; ++kk)
        if (kk < g.n_k_in) vh[kk] = value(kk);
    // one sum over k per entry that keeps (i, j) (runtime loops: the FP64 work is
    // proportional to the entries, not to a fixed unrolled count)
    for (int e = e0; e < e1; ++e) {
      const DevEntry& E = g.ent[e];
      if (i >= (g.pb ? E.Ka : E.na) || j >= (g.pb ? E.Kb : E.nb)) continue;
      const double2* ph = g.phase + (long long)e * g.n_k;
      const signed char* pc = g.pcode ? g.pcode + (long long)e * g.n_k : nullptr;
      double2 acc = make_double2(0.0, 0.0);
      auto term = [&](int kk, double2 v) {
        const int k = g.k_list ? g.k_list[kk] : kk;
        if (pc) {  // conj(i^c) v = i^(4 - c) v
          const double2 t = qmul((4 - pc[k]) & 3, v);
          acc.x += t.x;
          if (!g.real_only) acc.y += t.y;
        } else {
          const double2 c = ph[k];
          if (g.real_only) acc.x = fma(c.x, v.x, fma(c.y, v.y, acc.x));  // Re(conj(ph) v) only
          else acc = cfma_conj_a(c, v, acc);
        }
      };
      if (hold) {
#pragma unroll
        for (int kk = 0; kk < kHoldK; ++kk)
          if (kk < g.n_k_in) term(kk, vh[kk]);
      } else {
        for (int kk = 0; kk < g.n_k_in; ++kk) term(kk, value(kk));
      }
      const long long off = g.pb ? E.off_pb : E.off_orb;
      const int ce = g.pb ? E.Kb : E.nb, be = (g.pb ? E.Ka : E.na) * ce;
      if (g.scale != 1.0) {
        acc.x *= g.scale;
        acc.y *= g.scale;
      }
      g.F_R[off * g.out_n_slices + (long long)(g.out_slice0 + s) * be + i * ce + j] =
          make_double2(acc.x, g.real_only ? 0.0 : acc.y);
    }
  }
}

// The gather on `grid` x 256 threads: the form that streams each element's values once for
// all its entries when there are more k points than registers hold.
void launch_gather_kernel(dim3 grid, cudaStream_t st, const GatherArgs& g) {
  if (g.n_k_in > kHoldK) k_gather_k_to_R<true><<<grid, 256, 0, st>>>(g);
  else k_gather_k_to_R<false><<<grid, 256, 0, st>>>(g);
}

// ---------------------------------------------------------------------------
// R -> k scatter:  F_k[k][s][oa+i][ob+j] = sum_{e in (a,b)} ph[e][k] F_R[e][s][i][j]
// grid: (row atom a, slice); the block writes the band of rows of atom a across every
// column (zeros where the atom pair has no entry), consecutive threads on consecutive
// columns.  With at most kHoldK k points the sums of all k are kept in registers and each
// entry's value is read once; with quarter-turn phases each term is two additions.
// ---------------------------------------------------------------------------
__global__ void k_scatter_R_to_k(ScatterArgs g) {
  const int a = blockIdx.x, s = blockIdx.y;
  const int ro = g.row_off[a];
  const int rows = g.row_off[a + 1] - ro;
  const int n_el = rows * g.ld;
  const bool hold = g.n_k_out <= kHoldK;
  for (int x = threadIdx.x + blockIdx.z * blockDim.x; x < n_el; x += blockDim.x * gridDim.z) {
    const int i = x / g.ld, col = x - i * g.ld;
    const int b = g.col_atom[col];
    const int j = col - g.row_off[b];
    const int p = a * g.n_atoms + b;
    const int e0 = g.pair_start[p], e1 = g.pair_start[p + 1];
    const long long out_el = (long long)(ro + i) * g.ld + col;
    // ph[e][k] v (or ph Re(v) for a real input) added to acc
    auto term = [&](int e, int k, double2 v, double2& acc) {
      if (g.pcode) {
        const int c = g.pcode[(long long)e * g.n_k + k];
        const double2 t = qmul(c, g.real_in ? make_double2(v.x, 0.0) : v);
        acc.x += t.x;
        acc.y += t.y;
      } else {
        const double2 c = g.phase[(long long)e * g.n_k + k];
        acc = g.real_in ? rfma(v.x, c, acc) : cfma(c, v, acc);
      }
    };
    auto finish = [&](int kk, double2 acc) {
      if (g.coef != 1.0) {
        acc.x *= g.coef;
        acc.y *= g.coef;
      }
      if (g.base) acc = cadd(acc, g.base[(long long)kk * g.ld * g.ld + out_el]);
      g.F_k[(long long)kk * g.k_stride + (long long)s * g.s_stride + out_el] = acc;
    };
    if (hold) {
      double2 acc[kHoldK];
#pragma unroll
      for (int kk = 0; kk < kHoldK; ++kk) acc[kk] = make_double2(0.0, 0.0);
      // the entries of the pair whose kept block holds (i, j); runtime loop, so the FP64
      // work is proportional to them
      for (int e = e0; e < e1; ++e) {
        const DevEntry& E = g.ent[e];
        const int re = g.pb ? E.Ka : E.na, ce = g.pb ? E.Kb : E.nb;
        if (i >= re || j >= ce) continue;
        const long long off = g.pb ? E.off_pb : E.off_orb;
        const double2 v = g.F_R[off * g.in_n_slices + (long long)(g.in_slice0 + s) * re * ce + i * ce + j];
#pragma unroll
        for (int kk = 0; kk < kHoldK; ++kk)
          if (kk < g.n_k_out) term(e, g.k_list ? g.k_list[kk] : kk, v, acc[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < kHoldK; ++kk)
        if (kk < g.n_k_out) finish(kk, acc[kk]);
    } else if (e1 - e0 <= kHoldK) {
      // many k points: the entries' values read once and held
      double2 vq[kHoldK];
      bool on[kHoldK];
#pragma unroll
      for (int q = 0; q < kHoldK; ++q) {
        on[q] = false;
        vq[q] = make_double2(0.0, 0.0);
        if (q < e1 - e0) {
          const DevEntry& E = g.ent[e0 + q];
          const int re = g.pb ? E.Ka : E.na, ce = g.pb ? E.Kb : E.nb;
          if (i < re && j < ce) {
            const long long off = g.pb ? E.off_pb : E.off_orb;
            vq[q] = g.F_R[off * g.in_n_slices + (long long)(g.in_slice0 + s) * re * ce + i * ce + j];
            on[q] = true;
          }
        }
      }
      for (int kk = 0; kk < g.n_k_out; ++kk) {
        const int k = g.k_list ? g.k_list[kk] : kk;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < kHoldK; ++q)
          if (on[q]) term(e0 + q, k, vq[q], acc);
        finish(kk, acc);
      }
    } else {
      for (int kk = 0; kk < g.n_k_out; ++kk) {
        const int k = g.k_list ? g.k_list[kk] : kk;
        double2 acc = make_double2(0.0, 0.0);
        for (int e = e0; e < e1; ++e) {
          const DevEntry& E = g.ent[e];
          const int re = g.pb ? E.Ka : E.na, ce = g.pb ? E.Kb : E.nb;
          if (i >= re || j >= ce) continue;
          const long long off = g.pb ? E.off_pb : E.off_orb;
          term(e, k, g.F_R[off * g.in_n_slices + (long long)(g.in_slice0 + s) * re * ce + i * ce + j], acc);
        }
        finish(kk, acc);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tau <-> i omega:  out[e][m][c] = sum_i T[m][i] in[e][i][c]
// grid: (entry, column chunk of 32); block (32, 8); input tile staged in smem.
// ---------------------------------------------------------------------------
__global__ void k_transform(TransformArgs g) {
  extern __shared__ double2 tile[];  // [n_in][32]
  const int e = blockIdx.x;
  const DevEntry E = g.ent[e];
  const int blk = g.pb ? E.Ka * E.Kb : E.na * E.nb;
  const long long off = g.pb ? E.off_pb : E.off_orb;
  const int c0 = blockIdx.y * 32;
  if (c0 >= blk) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = c0 + tx;
  const double2* in = g.in + off * g.in_stride;
  double2* out = g.out + off * g.n_out;
  for (int i = ty; i < g.n_in; i += blockDim.y)
    tile[i * 32 + tx] = (c < blk) ? in[(long long)i * blk + c] : make_double2(0.0, 0.0);
  __syncthreads();
  if (c >= blk) return;
  for (int m = g.m_begin + ty; m < g.n_out; m += blockDim.y) {
    const double2* Tm = g.T + (long long)m * g.n_in;
    double2 acc = make_double2(0.0, 0.0);
    if (g.mode == 1) {  // Re out = sum a Re F + b Im F over the paired nodes; Im out = 0
      for (int i = 0; i < g.n_in; ++i) {
        const double2 t = Tm[i], f = tile[i * 32 + tx];
        acc.x = fma(t.x, f.x, fma(t.y, f.y, acc.x));
      }
    } else if (g.mode == 2) {  // real input
      for (int i = 0; i < g.n_in; ++i) {
        const double2 t = Tm[i];
        const double f = tile[i * 32 + tx].x;
        acc.x = fma(t.x, f, acc.x);
        acc.y = fma(t.y, f, acc.y);
      }
    } else {
      for (int i = 0; i < g.n_in; ++i) acc = cfma(Tm[i], tile[i * 32 + tx], acc);
    }
    out[(long long)m * blk + c] = acc;
  }
}

// ---------------------------------------------------------------------------
// Eq. P_MM, FP64.  One block per (entry, tau node i); with C symmetric in
// (L, L'') the block also writes the mirrored node N-1-i as the conjugate.
//   X[K][L''][L'] = sum_L C^a[K][L][L''] G(tau_i)[L][L']
//   Y[K][L'][L''']= sum_L'' X[K][L''][L'] conj(G(beta - tau_i)[L''][L'''])
//   P[K][K']      = -s sum_{L' L'''} Y[K][L'][L'''] C^b[K'][L'][L''']
// ---------------------------------------------------------------------------
constexpr int kKC = 16;  // product functions of atom a per pass

__global__ void k_polarizability_fp64(ContractArgs g) {
  extern __shared__ double2 sm[];
  const int e = blockIdx.x;
  const int it = g.Ypre ? g.s0 + (int)blockIdx.y : (int)blockIdx.y;
  const DevEntry E = g.ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  const int N = g.n_tau;
  const int im = N - 1 - it;
  double2* G1 = sm;                 // [na][nb]
  double2* G2 = G1 + na * nb;       // [na][nb]
  double2* X = G2 + na * nb;        // [kKC][na][nb]
  double2* Y = X + kKC * na * nb;   // [kKC][nb][nb]
  const double2* Gin = g.G + E.off_orb * N;
  for (int x = threadIdx.x; x < na * nb; x += blockDim.x) {
    G1[x] = Gin[(long long)it * na * nb + x];
    G2[x] = Gin[(long long)im * na * nb + x];
  }
  __syncthreads();
  const double* Ca = g.C + E.ca;
  const double* Cb = g.C + E.cb;
  double2* Pout = g.out + E.off_pb * N;
  const double ms = -(double)g.spin;
  const bool mirror = g.mirror_tau && (im != it);
  for (int k0 = 0; k0 < Ka; k0 += kKC) {
    const int kc = min(kKC, Ka - k0);
    for (int x = threadIdx.x; x < kc * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;  // X[K][L''=L2][L'=L1]
      const double* c = Ca + (long long)(k0 + K) * na * na;
      double2 acc = make_double2(0.0, 0.0);
      for (int L = 0; L < na; ++L) acc = rfma(c[L * na + L2], G1[L * nb + L1], acc);
      X[x] = acc;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kc * nb * nb; x += blockDim.x) {
      const int K = x / (nb * nb);
      const int r = x - K * nb * nb;
      const int L1 = r / nb, L3 = r - L1 * nb;  // Y[K][L'=L1][L'''=L3]
      const double2* xk = X + K * na * nb;
      double2 acc = make_double2(0.0, 0.0);
      for (int L2 = 0; L2 < na; ++L2) acc = cfmac(xk[L2 * nb + L1], G2[L2 * nb + L3], acc);
      Y[x] = acc;
      if (g.Ypre)  // stage 3 runs on the tensor cores
        g.Ypre[g.offB[e] * g.tau_c + ((long long)blockIdx.y * Ka + k0) * nb * nb + x] = acc;
    }
    __syncthreads();
    if (g.Ypre) continue;
    for (int x = threadIdx.x; x < kc * Kb; x += blockDim.x) {
      const int K = x / Kb, Kp = x - (x / Kb) * Kb;
      const double2* y = Y + K * nb * nb;
      const double* c = Cb + (long long)Kp * nb * nb;
      double2 acc = make_double2(0.0, 0.0);
      for (int j = 0; j < nb * nb; ++j) acc = rfma(c[j], y[j], acc);
      acc.x *= ms;
      acc.y *= ms;
      const long long o = (long long)(k0 + K) * Kb + Kp;
      Pout[(long long)it * Ka * Kb + o] = acc;
      if (mirror) Pout[(long long)im * Ka * Kb + o] = make_double2(acc.x, -acc.y);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Eq. S_MM, FP64.  One block per (entry, slice).
//   B[K][L'][L''']  = sum_K' W[K][K'] C^b[K'][L'][L''']
//   D[K][L''][L']   = sum_L''' G[L''][L'''] B[K][L'][L''']
//   S[L][L']       += sum_{K, L''} C^a[K][L][L''] D[K][L''][L']
// out = sign * S  (sign -1: dynamic part; +1 with G(beta-) and v: exchange)
// ---------------------------------------------------------------------------
__global__ void k_self_energy_fp64(ContractArgs g) {
  extern __shared__ double2 sm[];
  const int e = blockIdx.x;
  const int s = blockIdx.y;
  const DevEntry E = g.ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  double2* Gs = sm;                  // [na][nb]
  double2* B = Gs + na * nb;         // [kKC][nb][nb]
  double2* D = B + kKC * nb * nb;    // [kKC][na][nb]
  const int so = g.Bpre ? g.s0 + s : s;  // slice of G and of the output
  const int gs = (g.g_slice >= 0) ? g.g_slice : so;
  const double2* Gin = g.G + E.off_orb * g.g_n_slices + (long long)gs * na * nb;
  for (int x = threadIdx.x; x < na * nb; x += blockDim.x) Gs[x] = Gin[x];
  const double2* W = g.W + E.off_pb * g.w_n_slices + (long long)s * Ka * Kb;
  const double* Ca = g.C + E.ca;
  const double* Cb = g.C + E.cb;
  double2 acc = make_double2(0.0, 0.0);
  const int own = threadIdx.x;  // output (L, L') owned by this thread
  __syncthreads();
  for (int k0 = 0; k0 < Ka; k0 += kKC) {
    const int kc = min(kKC, Ka - k0);
    if (g.Bpre) {  // stage A done on the tensor cores
      const double2* bp = g.Bpre + g.offB[e] * g.tau_c + ((long long)s * Ka + k0) * nb * nb;
      for (int x = threadIdx.x; x < kc * nb * nb; x += blockDim.x) B[x] = bp[x];
    } else {
      for (int x = threadIdx.x; x < kc * nb * nb; x += blockDim.x) {
        const int K = x / (nb * nb);
        const int j = x - K * nb * nb;
        const double2* w = W + (long long)(k0 + K) * Kb;
        double2 t = make_double2(0.0, 0.0);
        for (int Kp = 0; Kp < Kb; ++Kp) t = rfma(Cb[(long long)Kp * nb * nb + j], w[Kp], t);
        B[x] = t;
      }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < kc * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;  // D[K][L''=L2][L'=L1]
      const double2* bk = B + K * nb * nb + L1 * nb;
      double2 t = make_double2(0.0, 0.0);
      for (int L3 = 0; L3 < nb; ++L3) t = cfma(Gs[L2 * nb + L3], bk[L3], t);
      D[x] = t;
    }
    __syncthreads();
    if (own < na * nb) {
      const int L = own / nb, L1 = own - (own / nb) * nb;
      for (int K = 0; K < kc; ++K) {
        const double* c = Ca + (long long)(k0 + K) * na * na + L * na;
        const double2* dk = D + K * na * nb;
        for (int L2 = 0; L2 < na; ++L2) acc = rfma(c[L2], dk[L2 * nb + L1], acc);
      }
    }
    __syncthreads();
  }
  if (own < na * nb) {
    double2* o = g.out + E.off_orb * g.out_n_slices + (long long)so * na * nb;
    o[own] = make_double2(g.sign * acc.x, g.sign * acc.y);
  }
}

// ---------------------------------------------------------------------------
// W solve (Eq. W_1): W = (v^{-1} - P)^{-1} per (q, nu), by in-place Gauss-Jordan
// ---------------------------------------------------------------------------

// In-place Gauss-Jordan inverse with partial pivoting (|re| + |im| measure), one
// block per matrix.  Row exchanges are recorded in perm and undone on the columns
// at the end.  A zero pivot sets *status and leaves the matrix undefined.
__global__ void k_gj_inverse(double2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                             int* status) {
  extern __shared__ unsigned char smraw[];
  double2* rowk = reinterpret_cast<double2*>(smraw);  // [N] scaled pivot row
  double2* colk = rowk + N;                            // [N] multipliers
  __shared__ double rv[32];
  __shared__ int ri[32];
  const int b = blockIdx.x;
  double2* M = A + (long long)b * mat_stride;
  int* pm = perm + (long long)b * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k = 0; k < N; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < N; i += nt) {
      double2 z = M[(long long)i * N + k];
      double m = fabs(z.x) + fabs(z.y);
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
    __syncthreads();
    if (wid == 0) {
      best = (lane < nw) ? rv[lane] : -1.0;
      bi = (lane < nw) ? ri[lane] : N;
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        ri[0] = bi;
        pm[k] = bi;
        if (!(best > 0.0)) atomicExch(status, 1);
      }
    }
    __syncthreads();
    const int p = ri[0];
    // exchange rows k and p; the pivot row goes to shared memory
    for (int j = tid; j < N; j += nt) {
      double2 zk = M[(long long)k * N + j];
      double2 zp = M[(long long)p * N + j];
      if (p != k) M[(long long)p * N + j] = zk;
      rowk[j] = (p != k) ? zp : zk;
    }
    for (int i = tid; i < N; i += nt) {
      const int src = (i == p) ? k : i;  // row p now holds the old row k
      colk[i] = (i == k) ? make_double2(0.0, 0.0) : M[(long long)src * N + k];
    }
    __syncthreads();
    const double2 d = rowk[k];
    const double den = d.x * d.x + d.y * d.y;
    const double2 inv = (den > 0.0) ? make_double2(d.x / den, -d.y / den) : make_double2(0.0, 0.0);
    __syncthreads();
    // scaled pivot row: r_j = a_kj / d (j != k), r_k = 1 / d
    for (int j = tid; j < N; j += nt) {
      double2 r = (j == k) ? inv : cmul(rowk[j], inv);
      rowk[j] = r;
      M[(long long)k * N + j] = r;
    }
    __syncthreads();
    // every other row: a_ij <- (j == k ? 0 : a_ij) - f_i r_j   (one warp per row, lanes along j)
    for (int i = wid; i < N; i += nw) {
      if (i == k) continue;
      const double2 f = colk[i];
      const double2 mf = make_double2(-f.x, -f.y);
      double2* Mi = M + (long long)i * N;
      for (int j = lane; j < N; j += 32) {
        const double2 z = (j == k) ? make_double2(0.0, 0.0) : Mi[j];
        Mi[j] = cfma(mf, rowk[j], z);
      }
    }
    __syncthreads();
  }
  // undo the row exchanges on the columns of the inverse, last exchange first
  for (int k = N - 1; k >= 0; --k) {
    const int p = pm[k];
    if (p != k) {
      for (int i = tid; i < N; i += nt) {
        double2 t = M[(long long)i * N + k];
        M[(long long)i * N + k] = M[(long long)i * N + p];
        M[(long long)i * N + p] = t;
      }
    }
    __syncthreads();
  }
}

// Blocked form of the same in-place Gauss-Jordan inverse, panels of kGJB columns.
// The panel's elementary steps (pivot, row exchange, scaling, elimination) run in
// shared memory on the N x kGJB panel only; their product is I + Z with Z nonzero
// in the panel columns, so the rest of the matrix is updated once per panel by
// the row exchanges followed by the rank-kGJB product A[:, T] += Z A[panel rows, T].
// Same pivot choice and result as k_gj_inverse; the matrix is read and written
// once per panel instead of once per column.  Requires 2 N kGJB complex values of
// shared memory (N <= 430).
__global__ void k_gj_inverse_blocked(double2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                                     int* status) {
  extern __shared__ unsigned char smraw[];
  double2* Pan = reinterpret_cast<double2*>(smraw);  // [N][kGJB] panel columns
  double2* Prow = Pan + (size_t)N * kGJB;            // [kGJB][N] pivot rows (pre-update)
  double2* colk = Prow + (size_t)N * kGJB;           // [N]
  __shared__ double2 rowk[kGJB];
  __shared__ int pmk[kGJB];
  __shared__ double rv[32];
  __shared__ int ri[32];
  const int b = blockIdx.x;
  double2* M = A + (long long)b * mat_stride;
  int* pm = perm + (long long)b * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k0 = 0; k0 < N; k0 += kGJB) {
    const int bb = min(kGJB, N - k0);
    // load the panel
    for (int x = tid; x < N * bb; x += nt) {
      const int i = x / bb, m = x - (x / bb) * bb;
      Pan[i * kGJB + m] = M[(long long)i * N + k0 + m];
    }
    __syncthreads();
    for (int m = 0; m < bb; ++m) {
      const int k = k0 + m;
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < N; i += nt) {
        const double2 z = Pan[i * kGJB + m];
        const double a = fabs(z.x) + fabs(z.y);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
      __syncthreads();
      if (wid == 0) {
        best = (lane < nw) ? rv[lane] : -1.0;
        bi = (lane < nw) ? ri[lane] : N;
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          ri[0] = bi;
          pm[k] = bi;
          pmk[m] = bi;
          if (!(best > 0.0)) atomicExch(status, 1);
        }
      }
      __syncthreads();
      const int p = ri[0];
      if (p != k && tid < bb) {
        const double2 t = Pan[k * kGJB + tid];
        Pan[k * kGJB + tid] = Pan[p * kGJB + tid];
        Pan[p * kGJB + tid] = t;
      }
      __syncthreads();
      const double2 d = Pan[k * kGJB + m];
      const double den = d.x * d.x + d.y * d.y;
      const double2 inv = (den > 0.0) ? make_double2(d.x / den, -d.y / den) : make_double2(0.0, 0.0);
      for (int i = tid; i < N; i += nt) colk[i] = (i == k) ? make_double2(0.0, 0.0) : Pan[i * kGJB + m];
      if (tid < bb) rowk[tid] = (tid == m) ? inv : cmul(Pan[k * kGJB + tid], inv);
      __syncthreads();
      for (int x = tid; x < N * bb; x += nt) {
        const int i = x / bb, j = x - (x / bb) * bb;
        if (i == k) {
          Pan[i * kGJB + j] = rowk[j];
        } else {
          const double2 f = colk[i];
          const double2 z = (j == m) ? make_double2(0.0, 0.0) : Pan[i * kGJB + j];
          Pan[i * kGJB + j] = cfma(make_double2(-f.x, -f.y), rowk[j], z);
        }
      }
      __syncthreads();
    }
    // row exchanges on the other columns, then the pivot rows (pre-update) to shared memory
    for (int j = tid; j < N; j += nt) {
      if (j >= k0 && j < k0 + bb) continue;
      for (int m = 0; m < bb; ++m) {
        const int k = k0 + m, p = pmk[m];
        if (p != k) {
          const double2 t = M[(long long)k * N + j];
          M[(long long)k * N + j] = M[(long long)p * N + j];
          M[(long long)p * N + j] = t;
        }
      }
      for (int m = 0; m < bb; ++m) Prow[m * N + j] = M[(long long)(k0 + m) * N + j];
    }
    __syncthreads();
    // A[:, T] += (Pan - I[:, panel]) Prow   (one warp per row, lanes along j)
    for (int i = wid; i < N; i += nw) {
      double2 z[kGJB];
#pragma unroll
      for (int m = 0; m < kGJB; ++m) {
        z[m] = (m < bb) ? Pan[i * kGJB + m] : make_double2(0.0, 0.0);
        if (i == k0 + m) z[m].x -= 1.0;
      }
      double2* Mi = M + (long long)i * N;
      for (int j = lane; j < N; j += 32) {
        if (j >= k0 && j < k0 + bb) continue;
        double2 acc = Mi[j];
#pragma unroll
        for (int m = 0; m < kGJB; ++m)
          if (m < bb) acc = cfma(z[m], Prow[m * N + j], acc);
        Mi[j] = acc;
      }
    }
    // the panel itself
    for (int x = tid; x < N * bb; x += nt) {
      const int i = x / bb, m = x - (x / bb) * bb;
      M[(long long)i * N + k0 + m] = Pan[i * kGJB + m];
    }
    __syncthreads();
  }
  for (int k = N - 1; k >= 0; --k) {
    const int p = pm[k];
    if (p != k) {
      for (int i = tid; i < N; i += nt) {
        const double2 t = M[(long long)i * N + k];
        M[(long long)i * N + k] = M[(long long)i * N + p];
        M[(long long)i * N + p] = t;
      }
    }
    __syncthreads();
  }
}

__global__ void k_copy_mats(const double2* __restrict__ src, const int* __restrict__ map, double2* __restrict__ dst,
                            long long NN) {
  const int b = blockIdx.y;
  const double2* s = src + (long long)map[b] * NN;
  double2* d = dst + (long long)b * NN;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < NN; x += (long long)gridDim.x * blockDim.x)
    d[x] = s[x];
}

// One block per (entry, negative-frequency slot j): copy the transposed block of the
// mirror entry at the mirrored (non-negative) frequency.  Blocks are K_a x K_b.
__global__ void k_mirror_nu(const DevEntry* __restrict__ ent, const int* __restrict__ nu_mirror, int n_neg, int n_nu,
                            double2* __restrict__ W) {
  const int e = blockIdx.x;
  const int j = blockIdx.y;
  if (j >= n_neg) return;
  const DevEntry E = ent[e];
  const DevEntry F = ent[E.mirror];
  const int Ka = E.Ka, Kb = E.Kb;  // mirror block is Kb x Ka
  const int jm = nu_mirror[j];
  const double2* src = W + F.off_pb * n_nu + (long long)jm * Kb * Ka;
  double2* dst = W + E.off_pb * n_nu + (long long)j * Ka * Kb;
  for (int x = threadIdx.x; x < Ka * Kb; x += blockDim.x) {
    const int r = x / Kb, c = x - (x / Kb) * Kb;
    dst[x] = src[c * Ka + r];
  }
}

}  // namespace gw
