// Tensor-core (tcgen05) form of the P contraction of Eq. P_MM for the mixed path.
//
// Per (entry, tau node) the first two stages run in FP32 on the CUDA cores:
//   X[K][L''][L'] = sum_L C^a[K][L][L''] G(tau)[L][L']
//   Y[K][j]       = sum_L'' X[K][L''][L'] conj(G(beta - tau)[L''][L''']),  j = (L', L''')
// and the dense third stage, P[K][K'] = -s sum_j Y[K][j] C^b[K'][j], runs on the
// tensor cores: the rows (Re Y; Im Y) form the 128-row A operand, C^b the B
// operand, both split into three BF16 terms (x = hi + mid + lo, 24 significant
// bits) and multiplied as the six products with i + j <= 2, accumulated in FP32
// in tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "kernels.h"
#include "smem_limit.h"
#include "mixed.h"
#include "ktimer.h"
#include "umma.h"
#include "fpbits.h"

namespace gw {

namespace {

using namespace umma;

constexpr uint64_t kWaitNs = 200ull * 1000ull * 1000ull;  // 200 ms per wait

__device__ __forceinline__ void split3(float y, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(y);
  const float r1 = y - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

struct TcLayout {
  int KD;      // padded reduction length (n_b^2 rounded up to 16)
  int NP;      // padded N (K_b rounded up to 16)
  uint32_t offA, offB, offX, offG, offP, offBar, total;
};

__host__ __device__ inline TcLayout tc_layout(int na, int nb, int Ka, int Kb) {
  TcLayout L;
  L.KD = ((nb * nb + 15) / 16) * 16;
  L.NP = ((Kb + 15) / 16) * 16;
  uint32_t o = 0;
  L.offA = o; o += 3u * 128u * L.KD * 2u;
  L.offB = o; o += 3u * (uint32_t)L.NP * L.KD * 2u;
  L.offX = o; o += (uint32_t)Ka * na * nb * 8u;
  L.offG = o; o += 2u * na * nb * 8u;
  L.offP = o; o += (uint32_t)Ka * Kb * 8u;
  o = (o + 15u) & ~15u;
  L.offBar = o; o += 16u;
  L.total = o;
  return L;
}

// grid (entry, tau chunk); 512 threads.  taus: the computed nodes it = 0 .. n_eff-1.
__global__ void __launch_bounds__(512, 1)
k_polarizability_tc(const DevEntry* __restrict__ ent, const float* __restrict__ C, const uint16_t* __restrict__ Bsplit,
                    const int* __restrict__ Bsplit_off, const int* __restrict__ species_of_atom,
                    const double2* __restrict__ G, double2* __restrict__ out, int n_tau, int n_eff, int tau_per_cta,
                    int spin, int mirror_tau, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  const int e = blockIdx.x;
  const DevEntry E = ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  const TcLayout L = tc_layout(na, nb, Ka, Kb);
  unsigned char* Ap = sm + L.offA;
  unsigned char* Bp = sm + L.offB;
  float2* X = reinterpret_cast<float2*>(sm + L.offX);
  float2* G1 = reinterpret_cast<float2*>(sm + L.offG);
  float2* G2 = G1 + na * nb;
  float2* Ps = reinterpret_cast<float2*>(sm + L.offP);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.offBar);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // tensor-memory accumulators: one of 128 lanes x NP columns per 16-wide K step when they
  // fit the 512 columns (the tensor core truncates as it accumulates, so fewer additions
  // per accumulator keep the sum closer; the epilogue adds them with rounding to nearest),
  // else one for all (allocation: power of two >= 32)
  const int nks = L.KD / 16;
  const bool per_step = nks * L.NP <= 512;
  uint32_t ncols = 32;
  while ((int)ncols < (per_step ? nks * L.NP : L.NP)) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  // B operand (C^b split in three planes, canonical layout) and a zeroed A operand
  const int sb = species_of_atom[E.b];
  // the planes of C^b for this entry's product-basis size (full, or reduced beyond sphere B)
  const uint4* bsrc = reinterpret_cast<const uint4*>(Bsplit + Bsplit_off[2 * sb + E.far]);
  uint4* bdst = reinterpret_cast<uint4*>(Bp);
  const int nb16 = (int)(3u * L.NP * L.KD * 2u / 16u);
  for (int x = tid; x < nb16; x += blockDim.x) bdst[x] = bsrc[x];
  uint4* az = reinterpret_cast<uint4*>(Ap);
  const int na16 = (int)(3u * 128u * L.KD * 2u / 16u);
  for (int x = tid; x < na16; x += blockDim.x) az[x] = make_uint4(0, 0, 0, 0);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const uint32_t idesc = idesc_bf16_f32(128, L.NP);
  const uint32_t aBase = smem_u32(Ap), bBase = smem_u32(Bp);
  const uint32_t aPlane = 128u * L.KD * 2u, bPlane = (uint32_t)L.NP * L.KD * 2u;
  const float* Ca = C + E.ca;
  const double2* Gin = G + E.off_orb * n_tau;
  double2* Pout = out + E.off_pb * n_tau;
  const float msf = -(float)spin;
  const int t0 = blockIdx.y * tau_per_cta;
  const int t1 = min(n_eff, t0 + tau_per_cta);
  bool ok = true;
  uint32_t phase = 0;
  for (int it = t0; it < t1 && ok; ++it) {
    const int im = n_tau - 1 - it;
    for (int x = tid; x < na * nb; x += blockDim.x) {
      const double2 g1 = Gin[(long long)it * na * nb + x];
      const double2 g2 = Gin[(long long)im * na * nb + x];
      G1[x] = make_float2(d2f(g1.x), d2f(g1.y));
      G2[x] = make_float2(d2f(g2.x), d2f(g2.y));
    }
    __syncthreads();
    // stage 1: X[K][L''][L']
    for (int x = tid; x < Ka * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;
      const float* c = Ca + (long long)K * na * na;
      float ax = 0.f, ay = 0.f;
      for (int l = 0; l < na; ++l) {
        const float cv = c[l * na + L2];
        const float2 g = G1[l * nb + L1];
        ax = fmaf(cv, g.x, ax);
        ay = fmaf(cv, g.y, ay);
      }
      X[x] = make_float2(ax, ay);
    }
    __syncthreads();
    // stage 2 + split: rows K (Re) and Ka + K (Im), columns j = L' nb + L''' in groups of
    // 8 (one 16-byte core-matrix row per plane; the padding columns j >= nb^2 are zeros)
    const int ngj = L.KD / 8;
    for (int x = tid; x < Ka * ngj; x += blockDim.x) {
      const int K = x / ngj;
      const int j0 = (x - K * ngj) * 8;
      const float2* xk = X + K * na * nb;
      uint32_t pk[6][4];  // (hi, mid, lo) x (Re, Im), 8 BF16 each
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) pk[q][w] = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        float yr = 0.f, yi = 0.f;
        if (j < nb * nb) {
          const int L1 = j / nb, L3 = j - L1 * nb;
          for (int L2 = 0; L2 < na; ++L2) {
            const float2 a = xk[L2 * nb + L1];
            const float2 b = G2[L2 * nb + L3];
            // a * conj(b)
            yr = fmaf(a.x, b.x, fmaf(a.y, b.y, yr));
            yi = fmaf(a.y, b.x, fmaf(-a.x, b.y, yi));
          }
        }
        __nv_bfloat16 h, m, l;
        const uint32_t sh = (uint32_t)(u & 1) * 16u;
        split3(yr, h, m, l);
        pk[0][u >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << sh;
        pk[1][u >> 1] |= (uint32_t)__bfloat16_as_ushort(m) << sh;
        pk[2][u >> 1] |= (uint32_t)__bfloat16_as_ushort(l) << sh;
        split3(yi, h, m, l);
        pk[3][u >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << sh;
        pk[4][u >> 1] |= (uint32_t)__bfloat16_as_ushort(m) << sh;
        pk[5][u >> 1] |= (uint32_t)__bfloat16_as_ushort(l) << sh;
      }
      const uint32_t o_r = kmajor_offset(128, K, j0), o_i = kmajor_offset(128, Ka + K, j0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        *reinterpret_cast<uint4*>(Ap + q * aPlane + o_r) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
        *reinterpret_cast<uint4*>(Ap + q * aPlane + o_i) =
            make_uint4(pk[3 + q][0], pk[3 + q][1], pk[3 + q][2], pk[3 + q][3]);
      }
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
      uint32_t acc = 0;
      for (int s = 0; s < nks; ++s) {
        const uint32_t ao = (uint32_t)s * 128u * 32u, bo = (uint32_t)s * (uint32_t)L.NP * 32u;
        const uint32_t td = tm + (per_step ? (uint32_t)(s * L.NP) : 0u);
        if (per_step) acc = 0;
        // the six split products with i + j <= 2 (0 = hi, 1 = mid, 2 = lo)
        const int pa[6] = {0, 0, 1, 0, 1, 2};
        const int pb[6] = {0, 1, 0, 2, 1, 0};
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = smem_desc(aBase + pa[q] * aPlane + ao, 128, 256);
          const uint64_t db = smem_desc(bBase + pb[q] * bPlane + bo, 128, 256);
          mma_bf16(td, da, db, idesc, acc);
          acc = 1;
        }
      }
      mma_commit(bar);
    }
    // every thread waits; the block acts on one common outcome
    ok = __syncthreads_and(mbar_wait(bar, phase, kWaitNs, status) ? 1 : 0) != 0;
    phase ^= 1u;
    fence_after_sync();
    if (!ok) {
      if (tid == 0) atomicExch(status, 2);
      // give the tensor core a second bounded chance to finish before the
      // accumulator is released
      mbar_wait(bar, phase ^ 1u, kWaitNs, nullptr);
      break;
    }
    // epilogue: TMEM rows (Re | Im) -> Ps[K][K'] -> P(tau) and its mirror
    if (warp < 4) {
      const int r = 32 * warp + lane;
      for (int c0 = 0; c0 < L.NP; c0 += 16) {
        float v[16], t[16];
        tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        for (int s = 1; per_step && s < nks; ++s) {
          tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)(s * L.NP + c0), t);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += t[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int Kp = c0 + i;
          if (Kp < Kb) {
            if (r < Ka) Ps[r * Kb + Kp].x = v[i];
            else if (r < 2 * Ka) Ps[(r - Ka) * Kb + Kp].y = v[i];
          }
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    const bool mirror = mirror_tau && (im != it);
    for (int x = tid; x < Ka * Kb; x += blockDim.x) {
      const float2 p = Ps[x];
      const float zr = msf * p.x, zi = msf * p.y;  // -s is a power of two: exact in FP32
      Pout[(long long)it * Ka * Kb + x] = make_double2(f2d(zr), f2d(zi));
      if (mirror) Pout[(long long)im * Ka * Kb + x] = make_double2(f2d(zr), f2d(-zi));
    }
    __syncthreads();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, ncols);
}

struct TcLayoutS {
  int KK;      // padded reduction length (K_b rounded up to 16)
  int NJ;      // padded N (n_b^2 rounded up to 16)
  uint32_t offA, offB, offBm, offD, offG, offRed, offBar, total;
};

constexpr int kSGroups = 8;  // thread groups splitting the K sum of stage C

__host__ __device__ inline TcLayoutS tc_layout_s(int na, int nb, int Ka, int Kb) {
  TcLayoutS L;
  L.KK = ((Kb + 15) / 16) * 16;
  L.NJ = ((nb * nb + 15) / 16) * 16;
  uint32_t o = 0;
  L.offA = o; o += 3u * 128u * L.KK * 2u;
  L.offB = o; o += 3u * (uint32_t)L.NJ * L.KK * 2u;
  L.offBm = o; o += (uint32_t)Ka * nb * nb * 8u;
  L.offD = o; o += (uint32_t)Ka * na * nb * 8u;
  L.offG = o; o += (uint32_t)na * nb * 8u;
  L.offRed = o; o += (uint32_t)kSGroups * na * nb * 8u;
  o = (o + 15u) & ~15u;
  L.offBar = o; o += 16u;
  L.total = o;
  return L;
}

// Sigma contraction (Eq. S_MM, dynamic part), mixed path.  Stage A on the tensor
// cores: Bm[(Re|Im) K][j] = sum_K2 W~[K][K2] C^b[K2][j] (A = W~ split in three
// BF16 terms, B = (C^b)^T split likewise, six products); stages B and C in FP32:
//   D[K][L2][L1]  = sum_L3 G[L2][L3] Bm[K][L1 nb + L3]
//   Sigma[L][L1]  = -sum_{K, L2} C^a[K][L][L2] D[K][L2][L1]
// grid (entry, tau chunk); 512 threads.
__global__ void __launch_bounds__(512, 1)
k_self_energy_tc(const DevEntry* __restrict__ ent, const float* __restrict__ C, const uint16_t* __restrict__ BsplitT,
                 const int* __restrict__ BsplitT_off, const int* __restrict__ species_of_atom,
                 const double2* __restrict__ G, const double2* __restrict__ W, double2* __restrict__ out, int n_tau,
                 int tau_per_cta, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  const int e = blockIdx.x;
  const DevEntry E = ent[e];
  const int na = E.na, nb = E.nb, Ka = E.Ka, Kb = E.Kb;
  const TcLayoutS L = tc_layout_s(na, nb, Ka, Kb);
  unsigned char* Ap = sm + L.offA;
  unsigned char* Bp = sm + L.offB;
  float2* Bm = reinterpret_cast<float2*>(sm + L.offBm);
  float2* D = reinterpret_cast<float2*>(sm + L.offD);
  float2* Gs = reinterpret_cast<float2*>(sm + L.offG);
  float2* Red = reinterpret_cast<float2*>(sm + L.offRed);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.offBar);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // one accumulator of NJ columns per 16-wide K step when they fit the 512 columns (as in
  // the P kernel: fewer truncating additions per accumulator), else one for all
  const int nks = L.KK / 16;
  const bool per_step = nks * L.NJ <= 512;
  uint32_t ncols = 32;
  while ((int)ncols < (per_step ? nks * L.NJ : L.NJ)) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_base, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  const int sb = species_of_atom[E.b];
  const uint4* bsrc = reinterpret_cast<const uint4*>(BsplitT + BsplitT_off[2 * sb + E.far]);
  uint4* bdst = reinterpret_cast<uint4*>(Bp);
  const int nb16 = (int)(3u * L.NJ * L.KK * 2u / 16u);
  for (int x = tid; x < nb16; x += blockDim.x) bdst[x] = bsrc[x];
  uint4* az = reinterpret_cast<uint4*>(Ap);
  const int na16 = (int)(3u * 128u * L.KK * 2u / 16u);
  for (int x = tid; x < na16; x += blockDim.x) az[x] = make_uint4(0, 0, 0, 0);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const uint32_t idesc = idesc_bf16_f32(128, L.NJ);
  const uint32_t aBase = smem_u32(Ap), bBase = smem_u32(Bp);
  const uint32_t aPlane = 128u * L.KK * 2u, bPlane = (uint32_t)L.NJ * L.KK * 2u;
  const float* Ca = C + E.ca;
  const int t0 = blockIdx.y * tau_per_cta;
  const int t1 = min(n_tau, t0 + tau_per_cta);
  bool ok = true;
  uint32_t phase = 0;
  for (int it = t0; it < t1 && ok; ++it) {
    const double2* Gin = G + E.off_orb * n_tau + (long long)it * na * nb;
    const double2* Win = W + E.off_pb * n_tau + (long long)it * Ka * Kb;
    for (int x = tid; x < na * nb; x += blockDim.x) {
      const double2 g = Gin[x];
      Gs[x] = make_float2(d2f(g.x), d2f(g.y));
    }
    // A operand: rows K (Re W~) and Ka + K (Im W~), reduction index K2 in groups of 8
    // (one 16-byte core-matrix row per plane; the padding K2 >= Kb stays zero)
    const int ngk = (Kb + 7) / 8;
    for (int x = tid; x < Ka * ngk; x += blockDim.x) {
      const int K = x / ngk;
      const int k0 = (x - K * ngk) * 8;
      uint32_t pk[6][4];
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) pk[q][w] = 0u;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (k0 + u < Kb) {
          const double2 w = Win[(long long)K * Kb + k0 + u];
          const uint32_t sh = (uint32_t)(u & 1) * 16u;
          __nv_bfloat16 h, m, l;
          split3(d2f(w.x), h, m, l);
          pk[0][u >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << sh;
          pk[1][u >> 1] |= (uint32_t)__bfloat16_as_ushort(m) << sh;
          pk[2][u >> 1] |= (uint32_t)__bfloat16_as_ushort(l) << sh;
          split3(d2f(w.y), h, m, l);
          pk[3][u >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << sh;
          pk[4][u >> 1] |= (uint32_t)__bfloat16_as_ushort(m) << sh;
          pk[5][u >> 1] |= (uint32_t)__bfloat16_as_ushort(l) << sh;
        }
      }
      const uint32_t o_r = kmajor_offset(128, K, k0), o_i = kmajor_offset(128, Ka + K, k0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        *reinterpret_cast<uint4*>(Ap + q * aPlane + o_r) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
        *reinterpret_cast<uint4*>(Ap + q * aPlane + o_i) =
            make_uint4(pk[3 + q][0], pk[3 + q][1], pk[3 + q][2], pk[3 + q][3]);
      }
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid == 0) {
      uint32_t acc = 0;
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      for (int s2 = 0; s2 < nks; ++s2) {
        const uint32_t ao = (uint32_t)s2 * 128u * 32u, bo = (uint32_t)s2 * (uint32_t)L.NJ * 32u;
        const uint32_t td = tm + (per_step ? (uint32_t)(s2 * L.NJ) : 0u);
        if (per_step) acc = 0;
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = smem_desc(aBase + pa[q] * aPlane + ao, 128, 256);
          const uint64_t db = smem_desc(bBase + pb[q] * bPlane + bo, 128, 256);
          mma_bf16(td, da, db, idesc, acc);
          acc = 1;
        }
      }
      mma_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait(bar, phase, kWaitNs, status) ? 1 : 0) != 0;
    phase ^= 1u;
    fence_after_sync();
    if (!ok) {
      if (tid == 0) atomicExch(status, 2);
      mbar_wait(bar, phase ^ 1u, kWaitNs, nullptr);
      break;
    }
    // TMEM -> Bm[K][j] (complex FP32)
    if (warp < 4) {
      const int r = 32 * warp + lane;
      for (int c0 = 0; c0 < L.NJ; c0 += 16) {
        float v[16], t[16];
        tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        for (int s2 = 1; per_step && s2 < nks; ++s2) {
          tmem_ld16(tm + ((uint32_t)(32 * warp) << 16) + (uint32_t)(s2 * L.NJ + c0), t);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += t[i];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = c0 + i;
          if (j < nb * nb) {
            if (r < Ka) Bm[r * nb * nb + j].x = v[i];
            else if (r < 2 * Ka) Bm[(r - Ka) * nb * nb + j].y = v[i];
          }
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    // stage B: D[K][L2][L1] = sum_L3 G[L2][L3] Bm[K][L1 nb + L3]
    for (int x = tid; x < Ka * na * nb; x += blockDim.x) {
      const int K = x / (na * nb);
      const int r = x - K * na * nb;
      const int L2 = r / nb, L1 = r - L2 * nb;
      const float2* bk = Bm + K * nb * nb + L1 * nb;
      float tx = 0.f, ty = 0.f;
      for (int L3 = 0; L3 < nb; ++L3) {
        const float2 g = Gs[L2 * nb + L3];
        const float2 bv = bk[L3];
        tx = fmaf(g.x, bv.x, fmaf(-g.y, bv.y, tx));
        ty = fmaf(g.x, bv.y, fmaf(g.y, bv.x, ty));
      }
      D[x] = make_float2(tx, ty);
    }
    __syncthreads();
    // stage C: output (L, L1) summed over K in kSGroups slices of the threads, then reduced
    {
      const int no = na * nb;
      const int per_g = blockDim.x / kSGroups;
      const int g = tid / per_g, t = tid - g * per_g;
      const int kchunk = (Ka + kSGroups - 1) / kSGroups;
      const int K0 = g * kchunk, K1 = min(Ka, K0 + kchunk);
      for (int o = t; o < no; o += per_g) {
        const int Lr = o / nb, L1 = o - (o / nb) * nb;
        float ax = 0.f, ay = 0.f;
        for (int K = K0; K < K1; ++K) {
          const float* c = Ca + (long long)K * na * na + Lr * na;
          const float2* dk = D + K * na * nb;
          for (int L2 = 0; L2 < na; ++L2) {
            const float cv = c[L2];
            const float2 d = dk[L2 * nb + L1];
            ax = fmaf(cv, d.x, ax);
            ay = fmaf(cv, d.y, ay);
          }
        }
        Red[g * no + o] = make_float2(ax, ay);
      }
    }
    __syncthreads();
    for (int o = tid; o < na * nb; o += blockDim.x) {
      float ax = 0.f, ay = 0.f;
      for (int g = 0; g < kSGroups; ++g) {
        const float2 r2 = Red[g * na * nb + o];
        ax += r2.x;
        ay += r2.y;
      }
      double2* op = out + E.off_orb * n_tau + (long long)it * na * nb;
      op[o] = make_double2(f2d(-ax), f2d(-ay));
    }
    __syncthreads();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, ncols);
}

}  // namespace

// Host side: eligibility, B-operand planes per species, launch.
bool tc_eligible(const HostPlan& h, size_t* smem_out) {
  size_t smax = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      const int na = h.n_orb[s], nb = h.n_orb[t], Ka = h.n_prod[s], Kb = h.n_prod[t];
      if (2 * Ka > 128 || nb * nb > 128 || Kb > 128) return false;
      smax = std::max<size_t>(smax, tc_layout(na, nb, Ka, Kb).total);
    }
  if (smax > 200 * 1024) return false;
  *smem_out = smax;
  return true;
}

static bool tc_eligible_s(const HostPlan& h, size_t* smem_out) {
  size_t smax = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      const int na = h.n_orb[s], nb = h.n_orb[t], Ka = h.n_prod[s], Kb = h.n_prod[t];
      if (2 * Ka > 128 || nb * nb > 256 || Kb > 128) return false;
      smax = std::max<size_t>(smax, tc_layout_s(na, nb, Ka, Kb).total);
    }
  if (smax > 200 * 1024) return false;
  *smem_out = smax;
  return true;
}

// Round to BF16 (nearest even) on the host; returns the bits and the rounded value.
static uint16_t bf16_round(double c, double* rounded) {
  float f = (float)c;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t rb = ((u >> 16) & 1u) + 0x7FFFu;
  u = (u + rb) & 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  *rounded = (double)r;
  return (uint16_t)(u >> 16);
}

gw_status tc_init(MixedPlan& m, const HostPlan& h) {
  m.tc_ready = false;
  size_t smem = 0;
  if (!tc_eligible(h, &smem)) return GW_OK;
  // C^b in three BF16 planes per species and product-basis size (full, then the reduced
  // size of entries beyond sphere B), canonical K-major layout of an NP x KD operand
  std::vector<uint16_t> planes;
  std::vector<int> off;
  for (int sv = 0; sv < 2 * h.n_species; ++sv) {
    const int s = sv / 2;
    const int nb = h.n_orb[s], Kb = (sv & 1) ? h.n_prod_far[s] : h.n_prod[s];
    const TcLayout L = tc_layout(nb, nb, Kb, Kb);
    off.push_back((int)planes.size());
    const size_t plane = (size_t)L.NP * L.KD;
    std::vector<uint16_t> buf(3 * plane, 0);
    for (int Kp = 0; Kp < Kb; ++Kp)
      for (int j = 0; j < nb * nb; ++j) {
        double c = h.C[s][(size_t)Kp * nb * nb + j];
        const uint32_t byte_off = umma::kmajor_offset(L.NP, Kp, j);
        for (int q = 0; q < 3; ++q) {
          double r;
          buf[q * plane + byte_off / 2] = bf16_round(c, &r);
          c -= r;
        }
      }
    planes.insert(planes.end(), buf.begin(), buf.end());
  }
  cudaError_t e = cudaMalloc((void**)&m.d_Bsplit, planes.size() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(m.d_Bsplit, planes.data(), planes.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m.d_Bsplit_off, off.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(m.d_Bsplit_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m.d_species, h.species.size() * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(m.d_species, h.species.data(), h.species.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = gw::raise_smem_limit(k_polarizability_tc, (int)smem);
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core setup: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  m.smem_tc = smem;
  m.tc_ready = true;

  // Sigma: (C^b)^T, rows j = (L1, L3), reduction K2, three BF16 planes per species and
  // product-basis size as above
  size_t smem_s = 0;
  if (!tc_eligible_s(h, &smem_s)) return GW_OK;
  std::vector<uint16_t> tplanes;
  std::vector<int> toff;
  for (int sv = 0; sv < 2 * h.n_species; ++sv) {
    const int s = sv / 2;
    const int nb = h.n_orb[s], Kb = (sv & 1) ? h.n_prod_far[s] : h.n_prod[s];
    const TcLayoutS L = tc_layout_s(nb, nb, Kb, Kb);
    toff.push_back((int)tplanes.size());
    const size_t plane = (size_t)L.NJ * L.KK;
    std::vector<uint16_t> buf(3 * plane, 0);
    for (int Kp = 0; Kp < Kb; ++Kp)
      for (int j = 0; j < nb * nb; ++j) {
        double c = h.C[s][(size_t)Kp * nb * nb + j];
        const uint32_t byte_off = umma::kmajor_offset(L.NJ, j, Kp);
        for (int q = 0; q < 3; ++q) {
          double r;
          buf[q * plane + byte_off / 2] = bf16_round(c, &r);
          c -= r;
        }
      }
    tplanes.insert(tplanes.end(), buf.begin(), buf.end());
  }
  e = cudaMalloc((void**)&m.d_BsplitT, tplanes.size() * sizeof(uint16_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(m.d_BsplitT, tplanes.data(), tplanes.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m.d_BsplitT_off, toff.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(m.d_BsplitT_off, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = gw::raise_smem_limit(k_self_energy_tc, (int)smem_s);
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core setup (Sigma): ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  m.smem_tc_s = smem_s;
  m.tc_s_ready = true;
  return GW_OK;
}

gw_status tc_self_energy(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double2* G_R,
                         const double2* Wt_R, double2* Sig_R, int* d_status, cudaStream_t st) {
  const int per = 4;
  dim3 grid(h.n_entries(), (h.n_tau + per - 1) / per);
  {
    gw::TimedLaunch tl_("k_self_energy_tc", st);
    k_self_energy_tc<<<grid, 512, m.smem_tc_s, st>>>(d_ent, m.d_Cf, m.d_BsplitT, m.d_BsplitT_off, m.d_species, G_R,
                                                     Wt_R, Sig_R, h.n_tau, per, d_status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("k_self_energy_tc: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

void tc_free(MixedPlan& m) {
  if (m.d_BsplitT) cudaFree(m.d_BsplitT);
  if (m.d_BsplitT_off) cudaFree(m.d_BsplitT_off);
  m.d_BsplitT = nullptr;
  m.d_BsplitT_off = nullptr;
  m.tc_s_ready = false;
  if (m.d_Bsplit) cudaFree(m.d_Bsplit);
  if (m.d_Bsplit_off) cudaFree(m.d_Bsplit_off);
  if (m.d_species) cudaFree(m.d_species);
  m.d_Bsplit = nullptr;
  m.d_Bsplit_off = nullptr;
  m.d_species = nullptr;
  m.tc_ready = false;
}

gw_status tc_polarizability(MixedPlan& m, const HostPlan& h, const DevEntry* d_ent, const double2* G_R, double2* P_R,
                            int* d_status, cudaStream_t st) {
  const int n_eff = h.c_symmetric ? (h.n_tau + 1) / 2 : h.n_tau;
  const int per = 4;
  dim3 grid(h.n_entries(), (n_eff + per - 1) / per);
  {
    gw::TimedLaunch tl_("k_polarizability_tc", st);
    k_polarizability_tc<<<grid, 512, m.smem_tc, st>>>(d_ent, m.d_Cf, m.d_Bsplit, m.d_Bsplit_off, m.d_species, G_R, P_R,
                                                      h.n_tau, n_eff, per, h.spin, h.c_symmetric, d_status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("k_polarizability_tc: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
