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

// One 128-row tile x NT columns per block (128 threads).  The K steps of both operands
// pass through kOzStages shared-memory stages (one bulk copy of each per step; while
// step ks runs, the stage of step ks - 1 is refilled with step ks - 1 + kOzStages); one
// thread issues the digit products; the epilogue writes the FP64 result where the mode
// puts it.
__global__ void __launch_bounds__(128, 1) k_oz_gemm(OzGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[kOzStages];
  __shared__ __align__(8) uint64_t mmad[kOzStages];
  const int t = blockIdx.x, nt = blockIdx.y;
  const int e = g.tile_e[t];
  const DevEntry E = g.ent[e];
  const int NT = g.NT, KS = g.KS;
  // columns of this entry's output rows
  const int ncols = g.mode == kOzOutSigmaB ? E.nb * E.nb
                    : g.mode == kOzOutP    ? E.Kb
                    : (g.mode == kOzOutRealToComplex ? 2 * g.n_out : g.n_out);
  if (nt * NT >= ncols) return;  // this entry has fewer column tiles (uniform over the block)
  const int sb = g.species ? g.species[E.b] : 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int st = 0; st < kOzStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&mmad[st], 1);
    }
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base;
  const uint32_t BC = oz_bchunk(NT), SB = kOzAChunk + BC;  // bytes per stage
  const unsigned char* Ab = reinterpret_cast<const unsigned char*>(g.Adig) + (long long)t * KS * kOzAChunk;
  const unsigned char* Bb = reinterpret_cast<const unsigned char*>(g.Bdig + g.Boff[sb]) + (long long)nt * KS * BC;
  auto load = [&](int ks, int st) {
    mbar_arrive_expect_tx(&full[st], SB);
    bulk_g2s(sm + st * SB, Ab + (long long)ks * kOzAChunk, kOzAChunk, &full[st]);
    bulk_g2s(sm + st * SB + kOzAChunk, Bb + (long long)ks * BC, BC, &full[st]);
  };
  bool ok = true;
  if (tid == 0) {
    const uint32_t id = idesc_bf16_f32(128, NT);
    const uint32_t s0 = smem_u32(sm);
    const uint32_t PA = 128 * 16 * 2, PB = (uint32_t)NT * 16 * 2;
    for (int st = 0; st < kOzStages && st < KS; ++st) load(st, st);
    uint32_t used = 0;
    for (int ks = 0; ks < KS; ++ks) {
      const int st = ks % kOzStages;
      if (!mbar_wait(&full[st], (uint32_t)(ks / kOzStages) & 1u, kWaitNs, g.status)) { ok = false; break; }
      fence_after_sync();
      const uint32_t a0 = s0 + st * SB, b0 = a0 + kOzAChunk;
      for (int tt = 0; tt < kOzDigits; ++tt)
        for (int s = 0; s + tt <= kOzLmax && s < kOzDigits; ++s) {
          const int q = oz_bucket(s + tt);
          const uint32_t acc = (used >> q) & 1u;
          used |= 1u << q;
          mma_bf16(tm + (uint32_t)(q * NT), smem_desc(a0 + s * PA, 128, 256), smem_desc(b0 + tt * PB, 128, 256), id,
                   acc);
        }
      mma_commit(&mmad[st]);
      if (ks >= 1 && ks - 1 + kOzStages < KS) {
        // the products of step ks - 1 are done once its commit arrives: refill its stage
        const int so = (ks - 1) % kOzStages;
        if (!mbar_wait(&mmad[so], (uint32_t)((ks - 1) / kOzStages) & 1u, kWaitNs, g.status)) { ok = false; break; }
        load(ks - 1 + kOzStages, so);
      }
    }
  }
  const int last = KS - 1;
  const bool done = __syncthreads_and(ok ? 1 : 0) != 0 &&
                    mbar_wait(&mmad[last % kOzStages], (uint32_t)(last / kOzStages) & 1u, kWaitNs, g.status);
  ok = __syncthreads_and(done ? 1 : 0) != 0;
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(g.status, 2);
  } else {
    const int r = 32 * warp + lane;
    const int rho = g.tile_r0[t] + r;
    const int ea = g.eA[t * 128 + r];
    const int* eb = g.eB + g.eBoff[sb] + nt * NT;
    // the destination of this row: one double per column, at stride `cstride` doubles
    bool valid;
    double* orow;
    long long cstride;
    bool zero_im = false;
    long long moff = 0;  // P: offset of the mirrored node (0: none)
    bool mneg = false;  // P: the mirrored node's imaginary part changes sign
    if (g.mode == kOzOutSigmaB) {
      const int Ka = E.Ka, nb2 = E.nb * E.nb;
      valid = rho < g.tau_eff * Ka * 2;
      const int c = rho & 1, q = rho >> 1;
      const int sl = q / Ka, K = q - (q / Ka) * Ka;
      orow = reinterpret_cast<double*>(g.out + g.offB[e] * g.tau_c + ((long long)sl * Ka + K) * nb2) + c;
      cstride = 2;
    } else if (g.mode == kOzOutP) {
      const int Ka = E.Ka, Kb = E.Kb;
      valid = rho < g.tau_eff * Ka * 2;
      const int c = rho & 1, q = rho >> 1;
      const int sl = q / Ka, K = q - (q / Ka) * Ka;
      const int it = g.s0 + sl, im = g.n_tau - 1 - it;
      orow = reinterpret_cast<double*>(g.out + E.off_pb * g.n_tau + ((long long)it * Ka + K) * Kb) + c;
      cstride = 2;
      if (g.mirror && im != it) {  // the mirrored node is the conjugate
        moff = 2LL * (im - it) * Ka * Kb;
        mneg = c != 0;
      }
    } else {
      const int blk = E.Ka * E.Kb;  // transforms on the product-basis layout
      valid = rho < blk;
      orow = reinterpret_cast<double*>(g.out + E.off_pb * g.n_out + rho);
      cstride = 2LL * blk;  // next output slice (tau or nu) of the same element
      zero_im = g.mode == kOzOutReal;
    }
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int ms_shift = g.ms < -1.5 ? 1 : 0;  // P: s = 2 doubles the value
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
          if (j >= ncols || j < g.n_skip) continue;
          if (g.mode == kOzOutP) {
            // -s (s = 1 or 2) folded into the integer and the exponent: exact, no FP64 arithmetic
            const double pv = i2d_scaled(-S[i], ea + eb[n0 + i] - 52 + ms_shift);
            orow[(long long)j * cstride] = pv;
            if (moff) orow[(long long)j * cstride + moff] = mneg ? dneg(pv) : pv;
            continue;
          }
          const double val = i2d_scaled(S[i], ea + eb[n0 + i] - 52);
          if (g.mode == kOzOutRealToComplex) {
            // columns 0 .. n_out-1: Re of slice j; n_out .. 2 n_out-1: Im of slice j - n_out
            const int sl = j < g.n_out ? j : j - g.n_out;
            orow[(long long)sl * cstride + (j < g.n_out ? 0 : 1)] = val;
          } else if (zero_im) {
            reinterpret_cast<double2*>(orow)[(long long)j * (cstride / 2)] = make_double2(val, 0.0);
          } else {
            orow[(long long)j * cstride] = val;
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// Digits of Y (stage 2 of the P contraction).  One thread per row of a 128-row tile:
// row rho = (sl K_a + K) 2 + c of the tile's entry, values Y[sl][K][j].c for j < n_b^2
// from the pass buffer (entry e at offB[e] tau_c, [sl][K_a][n_b^2] complex).
__global__ void __launch_bounds__(128)
k_oz_slice_y(const DevEntry* __restrict__ ent, const int* __restrict__ tile_e, const int* __restrict__ tile_r0,
             const double2* __restrict__ Y, const long long* __restrict__ offB, int tau_c, int tau_eff, int KS,
             uint16_t* __restrict__ Adig, int* __restrict__ eA) {
  const int t = blockIdx.x, r = threadIdx.x;
  const int ei = tile_e[t];
  const DevEntry E = ent[ei];
  const int Ka = E.Ka, nb2 = E.nb * E.nb;
  const int rho = tile_r0[t] + r;
  const bool valid = rho < tau_eff * Ka * 2;
  const double* src = nullptr;
  if (valid) {
    const int c = rho & 1, q = rho >> 1;
    const int sl = q / Ka, K = q - (q / Ka) * Ka;
    src = reinterpret_cast<const double*>(Y + offB[ei] * tau_c + ((long long)sl * Ka + K) * nb2) + c;
  }
  int m = 0;
  if (valid)
    for (int k = 0; k < nb2; ++k) m = max(m, exp_field(src[2 * k]));
  const int e = m > 0 ? m - 1022 : 0;
  eA[t * 128 + r] = e;
  uint16_t* tile = Adig + (long long)t * KS * (kOzAChunk / 2);
  for (int ks = 0; ks < KS; ++ks) {
    for (int h = 0; h < 2; ++h) {
      long long mv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = ks * 16 + 8 * h + u;
        mv[u] = (valid && k < nb2) ? fixed56(src[2 * k], e) : 0ll;
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

// Digits of the rows of a tau <-> i nu transform input on the product-basis layout: row x
// of entry e (x < K_a K_b), value k from slice k (GW_IN_REAL: Re in[k]) or, for the
// mirror-paired form, Re in[k] for k < nh and Im in[k - nh] for nh <= k < 2 nh.
__global__ void __launch_bounds__(128)
k_oz_slice_elem(const DevEntry* __restrict__ ent, const int* __restrict__ tile_e, const int* __restrict__ tile_r0,
                const double2* __restrict__ in, int n_slices, int K, int nh, int KS, uint16_t* __restrict__ Adig,
                int* __restrict__ eA) {
  const int t = blockIdx.x, r = threadIdx.x;
  const DevEntry E = ent[tile_e[t]];
  const int blk = E.Ka * E.Kb;
  const int x = tile_r0[t] + r;
  const bool valid = x < blk;
  const double* base = reinterpret_cast<const double*>(in + E.off_pb * n_slices + x);
  auto value = [&](int k) -> double {
    if (nh > 0 && k >= nh) return base[2LL * (k - nh) * blk + 1];
    return base[2LL * k * blk];
  };
  int m = 0;
  if (valid)
    for (int k = 0; k < K; ++k) m = max(m, exp_field(value(k)));
  const int e = m > 0 ? m - 1022 : 0;
  eA[t * 128 + r] = e;
  uint16_t* tile = Adig + (long long)t * KS * (kOzAChunk / 2);
  for (int ks = 0; ks < KS; ++ks) {
    for (int h = 0; h < 2; ++h) {
      long long mv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = ks * 16 + 8 * h + u;
        mv[u] = (valid && k < K) ? fixed56(value(k), e) : 0ll;
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

// Host digits with the device's rules (top-down signed digits, as next_digit).
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

// Digit chunks [nt][KS] of kOzDigits planes of NT x 16 and the column exponents of a
// column operand B[n][k] (n < n_cols, k < K) given by value(n, k).
struct OzMatrix {
  int NT = 0, n_nt = 0, KS = 0;
  std::vector<uint16_t> dig;
  std::vector<int> e;
};
template <typename F>
OzMatrix oz_matrix(int n_cols, int K, int NT, int KS, F value) {
  OzMatrix m;
  m.NT = NT;
  m.KS = KS;
  m.n_nt = (n_cols + NT - 1) / NT;
  m.dig.assign((size_t)m.n_nt * KS * (oz_bchunk(NT) / 2), 0);
  for (int n = 0; n < m.n_nt * NT; ++n) {
    int mx = 0;
    if (n < n_cols)
      for (int k = 0; k < K; ++k) mx = std::max(mx, host_exp_field(value(n, k)));
    const int e = mx > 0 ? mx - 1022 : 0;
    m.e.push_back(e);
    if (n >= n_cols) continue;
    const int ntile = n / NT, nl = n % NT;
    for (int k = 0; k < K; ++k) {
      long long mv = host_fixed56(value(n, k), e);
      const size_t chunk = ((size_t)ntile * KS + k / 16) * (oz_bchunk(NT) / 2);
      const uint32_t off = umma::kmajor_offset(NT, nl, k % 16) / 2;
      for (int d = 0; d < kOzDigits; ++d) m.dig[chunk + (size_t)d * NT * 16 + off] = host_digit_bf16(mv, d);
    }
  }
  return m;
}
// The multiple of 16 up to 80 (six accumulators fit the 512 tensor-memory columns) with
// the least padding of n_cols, the wider on ties.
int oz_pick_nt(int n_cols) {
  int NT = 16, best = 1 << 30;
  for (int c = 16; c <= 80; c += 16) {
    const int padded = ((n_cols + c - 1) / c) * c;
    if (padded <= best) { best = padded; NT = c; }
  }
  return NT;
}

}  // namespace

gw_status oz_sigma_init(OzSigma& o, const HostPlan& h, size_t cap) {
  o.ready = false;
  int KS = 0, max_nb2 = 0;
  for (int s = 0; s < h.n_species; ++s) {
    if (h.n_prod[s] > 16 * kOzMaxKS) return GW_OK;  // levels 0-4 exact up to 384 terms only
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
  o.smem = oz_smem(KS, NT);
  const int E = h.n_entries();
  // stage-A output per tau slice and entry: K_a n_b^2 complex values
  std::vector<long long> offB(E + 1, 0);
  std::vector<int> Ka(E), rows1(E);
  for (int e = 0; e < E; ++e) {
    const int b = (int)h.entries[8 * e + 1];
    Ka[e] = h.Ka_e[e];  // product functions of a kept by this entry
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
    OzGemmArgs g{};
    g.ent = d_ent;
    g.tile_e = o.d_tile_e;
    g.tile_r0 = o.d_tile_r0;
    g.Adig = o.d_Adig;
    g.eA = o.d_eA;
    g.KS = o.KS;
    g.Bdig = o.d_Bdig;
    g.Boff = o.d_Boff;
    g.eB = o.d_eB;
    g.eBoff = o.d_eBoff;
    g.species = o.d_species;
    g.NT = o.NT;
    g.mode = kOzOutSigmaB;
    g.out = o.d_Bpre;
    g.offB = o.d_offB;
    g.tau_c = o.tau_c;
    g.tau_eff = tau_eff;
    g.status = d_status;
    TimedLaunch tl_("k_oz_gemm", st);
    k_oz_gemm<<<dim3((unsigned)o.n_tiles, (unsigned)o.max_nt), 128, o.smem, st>>>(g);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core Sigma stage: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

gw_status oz_transform_init(OzTransform& o, const HostPlan& h) {
  o = OzTransform{};
  const int N = h.n_tau, nh = (N + 1) / 2, nn = h.n_nu;
  const bool w_ok = nn <= 16 * kOzMaxKS;      // reduction over the nu slices
  const bool p_ok = 2 * nh <= 16 * kOzMaxKS;  // reduction over (Re, Im) of the paired nodes
  if (!w_ok && !p_ok) return GW_OK;
  // row tiles: the K_a K_b elements of every entry, 128 per tile
  std::vector<int> te, tr;
  for (int e = 0; e < h.n_entries(); ++e) {
    const int blk = h.Ka_e[e] * h.Kb_e[e];
    for (int r0 = 0; r0 < blk; r0 += 128) {
      te.push_back(e);
      tr.push_back(r0);
    }
  }
  o.n_tiles = (int)te.size();
  // W: B[n][k] = Re T_inv[n][k] (n < N), Im T_inv[n - N][k]; P: B[m][k] = a (k < nh), b (k >= nh)
  o.KS_w = (nn + 15) / 16;
  o.KS_p = (2 * nh + 15) / 16;
  o.NT_w = oz_pick_nt(2 * N);
  o.NT_p = oz_pick_nt(nn);
  const std::vector<double>& Ti = h.Tb_inv;  // [N][nn] complex
  const std::vector<double>& Tm = h.Tb_mirror;  // [nn][nh] (a, b)
  OzMatrix mw = oz_matrix(2 * N, nn, o.NT_w, o.KS_w, [&](int n, int k) {
    return n < N ? Ti[2 * ((size_t)n * nn + k)] : Ti[2 * ((size_t)(n - N) * nn + k) + 1];
  });
  OzMatrix mp = oz_matrix(nn, 2 * nh, o.NT_p, o.KS_p, [&](int n, int k) {
    return k < nh ? Tm[2 * ((size_t)n * nh + k)] : Tm[2 * ((size_t)n * nh + (k - nh)) + 1];
  });
  o.nt_w = mw.n_nt;
  o.nt_p = mp.n_nt;
  o.KSmax = std::max(w_ok ? o.KS_w : 0, p_ok ? o.KS_p : 0);
  const long long zero64 = 0;
  const int zero32 = 0;
  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    o.bytes += bytes;
    return !src || cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up((void**)&o.d_tile_e, te.data(), te.size() * sizeof(int)) ||
      !up((void**)&o.d_tile_r0, tr.data(), tr.size() * sizeof(int))) {
    set_last_error("device allocation for the tensor-core transforms failed");
    oz_transform_free(o);
    return GW_ERR_OOM;
  }
  // row tiles of the orbital blocks, for the general transforms of the orbital layout
  {
    std::vector<int> te2, tr2;
    for (int e = 0; e < h.n_entries(); ++e) {
      const int a = (int)h.entries[8 * e], b = (int)h.entries[8 * e + 1];
      const int blk = h.n_orb[h.species[a]] * h.n_orb[h.species[b]];
      for (int r0 = 0; r0 < blk; r0 += 128) {
        te2.push_back(e);
        tr2.push_back(r0);
      }
    }
    o.n_tiles_orb = (int)te2.size();
    if (!up((void**)&o.d_tile_e_orb, te2.data(), te2.size() * sizeof(int)) ||
        !up((void**)&o.d_tile_r0_orb, tr2.data(), tr2.size() * sizeof(int))) {
      set_last_error("device allocation for the tensor-core transforms failed");
      oz_transform_free(o);
      return GW_ERR_OOM;
    }
  }
  // the fused kernels need only the row tiles; the digit planes serve the forms they cannot take
  const gw_status fs = oz_fused_init(o, h);
  if (fs != GW_OK) {
    oz_transform_free(o);
    return fs;
  }
  if ((!w_ok || o.fw.ready) && (!p_ok || o.fp.ready)) {
    o.ready_w = w_ok;
    o.ready_p = p_ok;
    return GW_OK;
  }
  const bool good = up((void**)&o.d_Adig, nullptr, (size_t)o.n_tiles * o.KSmax * kOzAChunk) &&
                    up((void**)&o.d_eA, nullptr, (size_t)o.n_tiles * 128 * sizeof(int)) &&
                    up((void**)&o.d_Bw, mw.dig.data(), mw.dig.size() * sizeof(uint16_t)) &&
                    up((void**)&o.d_ew, mw.e.data(), mw.e.size() * sizeof(int)) &&
                    up((void**)&o.d_Bp, mp.dig.data(), mp.dig.size() * sizeof(uint16_t)) &&
                    up((void**)&o.d_ep, mp.e.data(), mp.e.size() * sizeof(int)) &&
                    up((void**)&o.d_zero64, &zero64, sizeof(long long)) &&
                    up((void**)&o.d_zero32, &zero32, sizeof(int));
  if (!good) {
    set_last_error("device allocation for the tensor-core transforms failed");
    oz_transform_free(o);
    return GW_ERR_OOM;
  }
  o.smem = std::max(w_ok ? oz_smem(o.KS_w, o.NT_w) : 0, p_ok ? oz_smem(o.KS_p, o.NT_p) : 0);
  if (raise_smem_limit(k_oz_gemm, o.smem) != cudaSuccess) {
    set_last_error("cudaFuncSetAttribute (tensor-core transforms)");
    oz_transform_free(o);
    return GW_ERR_UNSUPPORTED;
  }
  o.ready_w = w_ok;
  o.ready_p = p_ok;
  return GW_OK;
}

void oz_transform_free(OzTransform& o) {
  oz_fused_free(o);
  void* ptrs[] = {o.d_tile_e, o.d_tile_r0, o.d_Adig, o.d_eA, o.d_Bw, o.d_ew, o.d_Bp, o.d_ep, o.d_zero64, o.d_zero32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  o = OzTransform{};
}

gw_status oz_transform(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int structure, const double2* in,
                       double2* out, int* d_status, cudaStream_t st) {
  const bool w = structure == GW_IN_REAL;
  if (structure == (GW_IN_MIRROR | GW_OUT_NONNEG) && o.fph.ready)
    return oz_fused_run(o, h, d_ent, structure, in, out, d_status, st);
  // the forms below: GW_OUT_NONNEG skips the output slices of the negative frequencies
  int n_skip = 0;
  if (structure & GW_OUT_NONNEG) {
    bool ascending = true;
    for (int j = 1; j < h.n_nu; ++j) ascending = ascending && h.nu_idx[j] > h.nu_idx[j - 1];
    while (ascending && n_skip < h.n_nu && h.nu_idx[n_skip] < 0) ++n_skip;
    structure &= ~GW_OUT_NONNEG;
  }
  if (n_skip == 0 && (w ? o.fw.ready : o.fp.ready)) return oz_fused_run(o, h, d_ent, structure, in, out, d_status, st);
  const int N = h.n_tau, nh = (N + 1) / 2, nn = h.n_nu;
  const int KS = w ? o.KS_w : o.KS_p, NT = w ? o.NT_w : o.NT_p, nts = w ? o.nt_w : o.nt_p;
  {
    TimedLaunch tl_("k_oz_slice_elem", st);
    k_oz_slice_elem<<<o.n_tiles, 128, 0, st>>>(d_ent, o.d_tile_e, o.d_tile_r0, in, w ? nn : N, w ? nn : 2 * nh,
                                               w ? 0 : nh, KS, o.d_Adig, o.d_eA);
  }
  {
    OzGemmArgs g{};
    g.ent = d_ent;
    g.tile_e = o.d_tile_e;
    g.tile_r0 = o.d_tile_r0;
    g.Adig = o.d_Adig;
    g.eA = o.d_eA;
    g.KS = KS;
    g.Bdig = w ? o.d_Bw : o.d_Bp;
    g.Boff = o.d_zero64;
    g.eB = w ? o.d_ew : o.d_ep;
    g.eBoff = o.d_zero32;
    g.species = nullptr;
    g.NT = NT;
    g.mode = w ? kOzOutRealToComplex : kOzOutReal;
    g.out = out;
    g.n_out = w ? N : nn;
    g.n_skip = w ? 0 : n_skip;
    g.status = d_status;
    TimedLaunch tl_("k_oz_gemm", st);
    k_oz_gemm<<<dim3((unsigned)o.n_tiles, (unsigned)nts), 128, oz_smem(KS, NT), st>>>(g);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core transform: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

gw_status oz_pol_init(OzPol& o, const HostPlan& h, size_t cap) {
  o = OzPol{};
  int KS = 0, max_Kb = 0;
  for (int s = 0; s < h.n_species; ++s) {
    const int nb2 = h.n_orb[s] * h.n_orb[s];
    if (nb2 > 16 * kOzMaxKS) return GW_OK;  // levels 0-4 exact up to 384 terms only
    KS = std::max(KS, (nb2 + 15) / 16);
    max_Kb = std::max(max_Kb, h.n_prod[s]);
  }
  const int NT = oz_pick_nt(max_Kb);
  o.KS = KS;
  o.NT = NT;
  o.max_nt = (max_Kb + NT - 1) / NT;
  o.smem = oz_smem(KS, NT);
  const int E = h.n_entries();
  const int n_eff = h.c_symmetric ? (h.n_tau + 1) / 2 : h.n_tau;
  std::vector<long long> offB(E + 1, 0);
  std::vector<int> rows1(E);
  long long rows_all = 0;
  for (int e = 0; e < E; ++e) {
    const int b = (int)h.entries[8 * e + 1];
    const int Ka = h.Ka_e[e], nb = h.n_orb[h.species[b]];
    offB[e + 1] = offB[e] + (long long)Ka * nb * nb;
    rows1[e] = 2 * Ka;
    rows_all += rows1[e];
  }
  const double per_slice = (double)offB[E] * 16.0 + (double)rows_all * KS * 16 * kOzDigits * 2.0;
  o.tau_c = std::max(1, std::min(n_eff, (int)((double)cap / std::max(per_slice, 1.0))));
  std::vector<int> te, tr;
  for (int e = 0; e < E; ++e)
    for (int r0 = 0; r0 < o.tau_c * rows1[e]; r0 += 128) {
      te.push_back(e);
      tr.push_back(r0);
    }
  o.n_tiles = (int)te.size();
  std::vector<uint16_t> bd;
  std::vector<long long> boff;
  std::vector<int> eb, eboff;
  for (int s = 0; s < h.n_species; ++s) {
    const int nb2 = h.n_orb[s] * h.n_orb[s], Kb = h.n_prod[s];
    const std::vector<double>& C = h.C[s];  // [K'][j]
    OzMatrix m = oz_matrix(Kb, nb2, NT, KS, [&](int n, int k) { return C[(size_t)n * nb2 + k]; });
    boff.push_back((long long)bd.size());
    eboff.push_back((int)eb.size());
    bd.insert(bd.end(), m.dig.begin(), m.dig.end());
    eb.insert(eb.end(), m.e.begin(), m.e.end());
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
      up((void**)&o.d_Ypre, nullptr, (size_t)offB[E] * o.tau_c * sizeof(double2)) &&
      up((void**)&o.d_offB, offB.data(), offB.size() * sizeof(long long));
  if (!good) {
    set_last_error("device allocation for the tensor-core P stage failed");
    oz_pol_free(o);
    return GW_ERR_OOM;
  }
  if (raise_smem_limit(k_oz_gemm, o.smem) != cudaSuccess) {
    set_last_error("cudaFuncSetAttribute (tensor-core P stage)");
    oz_pol_free(o);
    return GW_ERR_UNSUPPORTED;
  }
  o.ready = true;
  return GW_OK;
}

void oz_pol_free(OzPol& o) {
  void* ptrs[] = {o.d_tile_e, o.d_tile_r0, o.d_Adig, o.d_eA, o.d_Bdig, o.d_Boff, o.d_eB,
                  o.d_eBoff, o.d_species, o.d_Ypre, o.d_offB};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  o = OzPol{};
}

gw_status oz_pol_stage3(OzPol& o, const HostPlan& h, const DevEntry* d_ent, int s0, int tau_eff, double2* P_R,
                        int* d_status, cudaStream_t st) {
  {
    TimedLaunch tl_("k_oz_slice_y", st);
    k_oz_slice_y<<<o.n_tiles, 128, 0, st>>>(d_ent, o.d_tile_e, o.d_tile_r0, o.d_Ypre, o.d_offB, o.tau_c, tau_eff,
                                            o.KS, o.d_Adig, o.d_eA);
  }
  {
    OzGemmArgs g{};
    g.ent = d_ent;
    g.tile_e = o.d_tile_e;
    g.tile_r0 = o.d_tile_r0;
    g.Adig = o.d_Adig;
    g.eA = o.d_eA;
    g.KS = o.KS;
    g.Bdig = o.d_Bdig;
    g.Boff = o.d_Boff;
    g.eB = o.d_eB;
    g.eBoff = o.d_eBoff;
    g.species = o.d_species;
    g.NT = o.NT;
    g.mode = kOzOutP;
    g.out = P_R;
    g.tau_eff = tau_eff;
    g.s0 = s0;
    g.n_tau = h.n_tau;
    g.mirror = h.c_symmetric;
    g.ms = -(double)h.spin;
    g.status = d_status;
    TimedLaunch tl_("k_oz_gemm", st);
    k_oz_gemm<<<dim3((unsigned)o.n_tiles, (unsigned)o.max_nt), 128, o.smem, st>>>(g);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("tensor-core P stage: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
