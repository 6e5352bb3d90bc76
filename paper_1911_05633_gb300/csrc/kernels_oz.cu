// Stage A of the Sigma contraction of Eq. S_MM, B = W~ C^b, to FP64 accuracy on the
// tensor cores.  Each row (entry, tau, K, Re/Im) of W~ is scaled by a power of two and
// cut into kOzDigits signed base-2^7 digits (exact in BF16), the columns j of C^b the
// same way once per plan; the digit products a_s b_t with s + t <= kOzLmax are summed
// in FP32 tensor-memory accumulators per level L = s + t.  For a reduction length
// K_b <= 64 the sums of levels 0 .. 4 stay below 2^24 of their unit (2^-7(L+2)), so
// they are exact whatever rounding the tensor core applies; levels >= 5 share one
// accumulator.  The epilogue adds the levels as one exact 64-bit integer in units of
// 2^-52 and rounds once to FP64.  The error is that of an FP64 dot product: ~2^-52 K
// of sum |W~| |C|.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "kernels.h"
#include "ktimer.h"
#include "oz.h"
#include "ozaki.h"
#include "smem_limit.h"
#include "umma.h"

namespace gw {

namespace {

using namespace umma;

constexpr uint64_t kWaitNs = 500ull * 1000ull * 1000ull;

// Digits of W~.  One thread per row of a 128-row tile: row rho = (sl K_a + K) 2 + c of
// the tile's entry, values W~[s0 + sl][K][k].c for k < K_b (zeros beyond, and for the
// padding rows past the entry's last one).  Per 8 consecutive k one 16-byte core-matrix
// row per digit plane.
__global__ void __launch_bounds__(128)
k_oz_slice_w(const DevEntry* __restrict__ ent, const int* __restrict__ tile_e, const int* __restrict__ tile_r0,
             const double2* __restrict__ W, int n_tau, int s0, int tau_eff, int KS, uint16_t* __restrict__ Adig,
             int* __restrict__ eA) {
  const int t = blockIdx.x, r = threadIdx.x;
  const DevEntry E = ent[tile_e[t]];
  const int Ka = E.Ka, Kb = E.Kb;
  const int rho = tile_r0[t] + r;
  const bool valid = rho < tau_eff * Ka * 2;
  const double* src = nullptr;
  if (valid) {
    const int c = rho & 1, q = rho >> 1;
    const int sl = q / Ka, K = q - (q / Ka) * Ka;
    src = reinterpret_cast<const double*>(W + E.off_pb * n_tau + (long long)(s0 + sl) * Ka * Kb + (long long)K * Kb) + c;
  }
  int m = 0;
  if (valid)
    for (int k = 0; k < Kb; ++k) m = max(m, exp_field(src[2 * k]));
  const int e = m > 0 ? m - 1022 : 0;
  eA[t * 128 + r] = e;
  uint16_t* tile = Adig + (long long)t * KS * (kOzAChunk / 2);
  for (int ks = 0; ks < KS; ++ks) {
    for (int h = 0; h < 2; ++h) {
      long long mv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = ks * 16 + 8 * h + u;
        mv[u] = (valid && k < Kb) ? fixed56(src[2 * k], e) : 0ll;
      }
      uint16_t* chunk = tile + (long long)ks * (kOzAChunk / 2);
      const uint32_t off = kmajor_offset(128, r, 8 * h) / 2;
#pragma unroll
      for (int s = 0; s < kOzDigits; ++s) {
        uint32_t p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          p[u] = digit_bf16(next_digit(mv[2 * u], s), s) | (digit_bf16(next_digit(mv[2 * u + 1], s), s) << 16);
        *reinterpret_cast<uint4*>(chunk + s * (128 * 16) + off) = make_uint4(p[0], p[1], p[2], p[3]);
      }
    }
  }
}

// Accumulator of level L (levels >= 5 together).
__host__ __device__ constexpr int oz_bucket(int L) { return L < kOzBuckets - 1 ? L : kOzBuckets - 1; }

// One 128-row tile x NT columns per block (128 threads): all K steps of both operands
// are loaded into shared memory by two bulk copies, then one thread issues the digit
// products; the epilogue writes B to FP64.
__global__ void __launch_bounds__(128, 1)
k_oz_gemm(const DevEntry* __restrict__ ent, const int* __restrict__ tile_e, const int* __restrict__ tile_r0,
          const int* __restrict__ species, const uint16_t* __restrict__ Adig, const int* __restrict__ eA,
          const uint16_t* __restrict__ Bdig, const long long* __restrict__ Boff, const int* __restrict__ eB,
          const int* __restrict__ eBoff, int KS, int NT, int tau_c, int tau_eff, double2* __restrict__ Bpre,
          const long long* __restrict__ offB, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar;
  const int t = blockIdx.x, nt = blockIdx.y;
  const int e = tile_e[t];
  const DevEntry E = ent[e];
  const int nb2 = E.nb * E.nb;
  if (nt * NT >= nb2) return;  // this entry has fewer column tiles (uniform over the block)
  const int sb = species[E.b];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const uint32_t AB = (uint32_t)KS * kOzAChunk, BB = (uint32_t)KS * oz_bchunk(NT);
  bool ok = true;
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar, AB + BB);
    bulk_g2s(sm, reinterpret_cast<const unsigned char*>(Adig) + (long long)t * AB, AB, &bar);
    bulk_g2s(sm + AB, reinterpret_cast<const unsigned char*>(Bdig + Boff[sb]) + (long long)nt * BB, BB, &bar);
    ok = mbar_wait(&bar, 0, kWaitNs, status);
    if (ok) {
      fence_after_sync();
      const uint32_t id = idesc_bf16_f32(128, NT);
      const uint32_t a0 = smem_u32(sm), b0 = a0 + AB;
      const uint32_t PA = 128 * 16 * 2, PB = (uint32_t)NT * 16 * 2;
      uint32_t used = 0;
      for (int ks = 0; ks < KS; ++ks)
        for (int tt = 0; tt < kOzDigits; ++tt)
          for (int s = 0; s + tt <= kOzLmax && s < kOzDigits; ++s) {
            const int q = oz_bucket(s + tt);
            const uint32_t acc = (used >> q) & 1u;
            used |= 1u << q;
            mma_bf16(tm + (uint32_t)(q * NT), smem_desc(a0 + ks * kOzAChunk + s * PA, 128, 256),
                     smem_desc(b0 + ks * oz_bchunk(NT) + tt * PB, 128, 256), id, acc);
          }
      mma_commit(&bar);
    }
  }
  const bool done = __syncthreads_and(ok ? 1 : 0) != 0 && mbar_wait(&bar, 1, kWaitNs, status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 2);
  } else {
    const int Ka = E.Ka;
    const int r = 32 * warp + lane;
    const int rho = tile_r0[t] + r;
    const bool valid = rho < tau_eff * Ka * 2;
    const int c = rho & 1, q = rho >> 1;
    const int sl = q / Ka, K = q - (q / Ka) * Ka;
    const int ea = eA[t * 128 + r];
    double* orow = reinterpret_cast<double*>(Bpre + offB[e] * tau_c + ((long long)sl * Ka + K) * nb2) + c;
    const int* eb = eB + eBoff[sb] + nt * NT;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int n0 = 0; n0 < NT; n0 += 16) {
      long long S[16];
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) S[i] = 0;
#pragma unroll 1
      for (int b = 0; b < kOzBuckets; ++b) {
        tmem_ld16(tm + lane_base + (uint32_t)(b * NT + n0), v);
        // levels 0 .. 4: exact multiples of 2^-7(L+2) below 2^24 of them; levels >= 5: rounded
#pragma unroll
        for (int i = 0; i < 16; ++i)
          S[i] += b < kOzBuckets - 1
                      ? (long long)__float2int_rn(v[i] * __int_as_float((127 + 7 * (b + 2)) << 23)) << (38 - 7 * b)
                      : __float2ll_rn(v[i] * 0x1p52f);
      }
      if (valid) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = nt * NT + n0 + i;
          if (j < nb2) orow[2 * (long long)j] = i2d_scaled(S[i], ea + eb[n0 + i] - 52);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// Host digits with the device's rules (scale exponent from the exponent field, rounding
// half up at 2^-56 of the scale, top-down signed digits).
int host_exp_field(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return (int)((u >> 52) & 0x7FF);
}
long long host_fixed56(double x, int e) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = E - 1019 - e;
  long long r = sh >= 0 ? (m << sh) : (sh > -63 ? (m + (1ll << (-sh - 1))) >> (-sh) : 0);
  return (u >> 63) ? -r : r;
}
uint16_t host_digit_bf16(long long& m, int s) {
  const int sh = 49 - 7 * s;
  long long d;
  if (sh > 0) {
    const long long t = m + (1ll << (sh - 1));
    d = t >= 0 ? (t >> sh) : -((-t + (1ll << sh) - 1) >> sh);  // floor division by 2^sh
  } else {
    d = m;
  }
  m -= d * (1ll << sh);
  const float f = std::ldexp((float)d, -7 * (s + 1));
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

}  // namespace

gw_status oz_sigma_init(OzSigma& o, const HostPlan& h, size_t cap) {
  o.ready = false;
  int KS = 0, max_nb2 = 0;
  for (int s = 0; s < h.n_species; ++s) {
    if (h.n_prod[s] > 16 * kOzMaxKS) return GW_OK;  // reduction too long for the resident design
    KS = std::max(KS, (h.n_prod[s] + 15) / 16);
    max_nb2 = std::max(max_nb2, h.n_orb[s] * h.n_orb[s]);
  }
  // column tile: the multiple of 16 up to 80 (6 accumulators fit the 512 tensor-memory
  // columns) with the least padding of the widest n_b^2, the wider on ties
  int NT = 16, best = 1 << 30;
  for (int c = 16; c <= 80; c += 16) {
    const int padded = ((max_nb2 + c - 1) / c) * c;
    if (padded <= best) { best = padded; NT = c; }
  }
  o.KS = KS;
  o.NT = NT;
  o.max_nt = (max_nb2 + NT - 1) / NT;
  o.smem = (size_t)KS * kOzAChunk + (size_t)KS * oz_bchunk(NT);
  const int E = h.n_entries();
  // stage-A output per tau slice and entry: K_a n_b^2 complex values
  std::vector<long long> offB(E + 1, 0);
  std::vector<int> Ka(E), rows1(E);
  for (int e = 0; e < E; ++e) {
    const int a = (int)h.entries[8 * e], b = (int)h.entries[8 * e + 1];
    Ka[e] = h.n_prod[h.species[a]];
    const int nb = h.n_orb[h.species[b]];
    offB[e + 1] = offB[e] + (long long)Ka[e] * nb * nb;
    rows1[e] = 2 * Ka[e];
  }
  // tau slices per pass within the cap (stage-A output + digits of W~)
  long long rows_all = 0;
  for (int e = 0; e < E; ++e) rows_all += rows1[e];
  const double per_slice = (double)offB[E] * 16.0 + (double)rows_all * KS * 16 * kOzDigits * 2.0;
  int tau_c = std::max(1, std::min(h.n_tau, (int)((double)cap / std::max(per_slice, 1.0))));
  o.tau_c = tau_c;
  std::vector<int> te, tr;
  for (int e = 0; e < E; ++e)
    for (int r0 = 0; r0 < tau_c * rows1[e]; r0 += 128) {
      te.push_back(e);
      tr.push_back(r0);
    }
  o.n_tiles = (int)te.size();
  // digits of C^b per species: B[n = j][k = K2] = C[K2][j]
  std::vector<uint16_t> bd;
  std::vector<long long> boff;
  std::vector<int> eb, eboff;
  for (int s = 0; s < h.n_species; ++s) {
    const int nb = h.n_orb[s], Kb = h.n_prod[s], nb2 = nb * nb;
    const int nts = (nb2 + NT - 1) / NT;
    boff.push_back((long long)bd.size());
    eboff.push_back((int)eb.size());
    const size_t base = bd.size();
    bd.resize(base + (size_t)nts * KS * (oz_bchunk(NT) / 2), 0);
    for (int n = 0; n < nts * NT; ++n) {
      int m = 0;
      if (n < nb2)
        for (int k = 0; k < Kb; ++k) m = std::max(m, host_exp_field(h.C[s][(size_t)k * nb2 + n]));
      const int e = m > 0 ? m - 1022 : 0;
      eb.push_back(e);
      if (n >= nb2) continue;
      const int ntile = n / NT, nl = n % NT;
      for (int k = 0; k < Kb; ++k) {
        long long mv = host_fixed56(h.C[s][(size_t)k * nb2 + n], e);
        const int ks = k / 16;
        const size_t chunk = base + ((size_t)ntile * KS + ks) * (oz_bchunk(NT) / 2);
        const uint32_t off = umma::kmajor_offset(NT, nl, k % 16) / 2;
        for (int d = 0; d < kOzDigits; ++d) bd[chunk + (size_t)d * NT * 16 + off] = host_digit_bf16(mv, d);
      }
    }
  }
  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    o.bytes += bytes;
    return !src || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  const bool good =
      up((void**)&o.d_tile_e, te.data(), te.size() * sizeof(int)) &&
      up((void**)&o.d_tile_r0, tr.data(), tr.size() * sizeof(int)) &&
      up((void**)&o.d_Adig, nullptr, (size_t)o.n_tiles * KS * kOzAChunk) &&
      up((void**)&o.d_eA, nullptr, (size_t)o.n_tiles * 128 * sizeof(int)) &&
      up((void**)&o.d_Bdig, bd.data(), bd.size() * sizeof(uint16_t)) &&
      up((void**)&o.d_Boff, boff.data(), boff.size() * sizeof(long long)) &&
      up((void**)&o.d_eB, eb.data(), eb.size() * sizeof(int)) &&
      up((void**)&o.d_eBoff, eboff.data(), eboff.size() * sizeof(int)) &&
      up((void**)&o.d_species, h.species.data(), h.species.size() * sizeof(int)) &&
      up((void**)&o.d_Bpre, nullptr, (size_t)offB[E] * tau_c * sizeof(double2)) &&
      up((void**)&o.d_offB, offB.data(), offB.size() * sizeof(long long));
  if (!good) {
    set_last_error("device allocation for the tensor-core Sigma stage failed");
    oz_sigma_free(o);
    return GW_ERR_OOM;
  }
  if (raise_smem_limit(k_oz_gemm, o.smem) != cudaSuccess) {
    set_last_error("cudaFuncSetAttribute (tensor-core Sigma stage)");
    oz_sigma_free(o);
    return GW_ERR_UNSUPPORTED;
  }
  o.ready = true;
  return GW_OK;
}

void oz_sigma_free(OzSigma& o) {
  void* ptrs[] = {o.d_tile_e, o.d_tile_r0, o.d_Adig, o.d_eA, o.d_Bdig, o.d_Boff, o.d_eB,
                  o.d_eBoff, o.d_species, o.d_Bpre, o.d_offB};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  o = OzSigma{};
}

gw_status oz_sigma_stage_a(OzSigma& o, const HostPlan& h, const DevEntry* d_ent, const double2* W, int s0,
                           int tau_eff, int* d_status, cudaStream_t st) {
  {
    TimedLaunch tl_("k_oz_slice_w", st);
    k_oz_slice_w<<<o.n_tiles, 128, 0, st>>>(d_ent, o.d_tile_e, o.d_tile_r0, W, h.n_tau, s0, tau_eff, o.KS, o.d_Adig,
                                           o.d_eA);
  }
  {
    TimedLaunch tl_("k_oz_gemm", st);
    k_oz_gemm<<<dim3((unsigned)o.n_tiles, (unsigned)o.max_nt), 128, o.smem, st>>>(
        d_ent, o.d_tile_e, o.d_tile_r0, o.d_species, o.d_Adig, o.d_eA, o.d_Bdig, o.d_Boff, o.d_eB, o.d_eBoff, o.KS,
        o.NT, o.tau_c, tau_eff, o.d_Bpre, o.d_offB, d_status);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core Sigma stage: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
