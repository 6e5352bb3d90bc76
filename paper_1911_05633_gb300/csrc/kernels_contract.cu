// Persistent tensor-core contractions of Eq. P_MM (with the sign and tau pairing of
// Eq. P_II) and Eq. S_MM for the mixed-precision path, over a queue of work units.
//
// Polarizability, per unit (entry e = (a, b, R), computed node tau), per row tile of 64 K:
//   X[K][L''](L') = sum_L C^a[K][L][L''] G(tau)[L][L']                     CUDA cores, FP32
//   Y[K][j]       = sum_L'' X[K][L''](L') conj(G(beta - tau)[L''][L'''])    j = (L', L''')
//   P[K][K']      = -s sum_j Y[K][j] C^b[K'][j]                            tensor cores
// Self-energy, per unit (entry, node), over the row tiles of K:
//   Bm[K][j]      = sum_K' W~[K][K'] C^b[K'][j]                            tensor cores
//   h_K[L][L''']  = sum_L'' C^a[K][L][L''] G(tau)[L''][L''']                CUDA cores, FP32
//   Sigma[L][L']  = -sum_K sum_L''' h_K[L][L'''] Bm[K][(L', L''')]
//
// The dense stage runs as BF16 three-term split products (x = hi + mid + lo, the six
// products with i + j <= 2) with FP32 accumulation in tensor memory.  The tensor core
// truncates as it accumulates, so the large hi x hi products go to accumulators of
// their own (the K steps spread over several) and the five small correction products to
// one more; the epilogue adds the accumulators with rounding to nearest.
//
// Each resident block (one per SM) runs two independent groups of 256 threads (one
// group when the Sigma stage is wider than 128 columns); a group takes units from the
// queue with an atomic counter and owns its operand buffers, tensor-memory columns and
// barriers, so one group's CUDA-core stages overlap the other's tensor-core products and
// stores.  Every wait on the tensor core or on a bulk copy is bounded: after the limit
// the group records the failure (status 2) and waits once more, bounded, for its
// products in flight before the block releases its tensor memory and ends.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "contract.h"
#include "fpbits.h"
#include "ozaki.h"
#include "ktimer.h"
#include "smem_limit.h"
#include "umma.h"

namespace gw {

namespace {

using namespace umma;

constexpr int kTG = 256;                                  // threads per group
constexpr uint64_t kWaitNs = 500ull * 1000ull * 1000ull;  // 500 ms per wait

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(kTG) : "memory");
}

// Barrier of the group that also returns whether `v` holds for every thread of it.
__device__ __forceinline__ bool group_all(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r) : "r"((uint32_t)v), "r"(1 + g), "r"(kTG) : "memory");
  return r != 0;
}

// Bounded wait for an mbarrier phase; gives up after kWaitNs or as soon as another
// block has reported a timeout (status 2).
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t parity, const volatile int* status) {
  const uint32_t a = smem_u32(mbar);
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(a, parity)) return true;
    if (status && *status == 2) return false;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// Wait for a phase with the whole group; on failure record it and wait once more
// (bounded) so that no product or copy is left writing or reading the group's buffers.
__device__ __forceinline__ bool group_wait(uint64_t* bar, uint32_t& phase, int* status, int g) {
  const bool ok = group_all(g, wait_phase(bar, phase, status));
  if (!ok) {
    if ((threadIdx.x % kTG) == 0) atomicExch(status, 2);
    wait_phase(bar, phase, nullptr);
  }
  phase ^= 1u;
  return ok;
}

// Three-term BF16 split of two values, packed in pairs: (x0, x1) -> hi, mid, lo words.
__device__ __forceinline__ void split3x2(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
  __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
  const float r0 = x0 - __low2float(hh), r1 = x1 - __high2float(hh);
  __nv_bfloat162 mm = __floats2bfloat162_rn(r0, r1);
  const float s0 = r0 - __low2float(mm), s1 = r1 - __high2float(mm);
  __nv_bfloat162 ll = __floats2bfloat162_rn(s0, s1);
  h = *reinterpret_cast<uint32_t*>(&hh);
  m = *reinterpret_cast<uint32_t*>(&mm);
  l = *reinterpret_cast<uint32_t*>(&ll);
}

// Shared-memory layout of one group (byte offsets from the group's base).
struct GLayout {
  uint32_t a, b, g, total;
};

__host__ __device__ inline GLayout glayout(int kc, int n_cols) {
  GLayout L;
  uint32_t o = 0;
  L.a = o; o += 3u * 128u * (uint32_t)kc * 2u;              // A: 3 planes x 128 rows x kc
  L.b = o; o += 3u * (uint32_t)n_cols * (uint32_t)kc * 2u;  // B: 3 planes x n_cols rows x kc
  L.g = o; o += 2u * kCMaxOrb * kCMaxOrb * 8u;               // G(tau), G(beta - tau) as float2
  o = (o + 127u) & ~127u;
  L.total = o;
  return L;
}

struct GroupState {
  CUnit u;
  int bkey;  // the B operand held in the group's buffer (system, species, size), -1: none
  int stop;
  int next;  // the unit claimed after u (its input already on its way into L2), -1: none yet
};

// What a group works with: its buffers, barriers and tensor-memory columns.
struct GCtx {
  int g, t, warp, lane;
  unsigned char* A;
  unsigned char* B;
  float2* Gs;
  uint32_t aPlane, bPlane, a_bytes;
  uint32_t col_corr, col_hh, n_cols;
  int n_hh, kc;
  uint64_t* bar_mma;
  uint64_t* bar_b;
  uint32_t* ph_mma;
  uint32_t* ph_b;
  GroupState* gs;
  int* status;
};

// Accumulators of the hi x hi products for a dense stage N columns wide: as many as fit
// next to acc_corr in 256 columns (512 when N > 128, which runs one group per block).
// It depends on the unit's own N only, so a system gets the same arithmetic alone and
// in a batch.
__device__ __forceinline__ int unit_n_hh(int N) {
  return (N > 128 ? 512 : 256) / N - 1;
}

// The dense stage of one chunk: the five correction products of each K step into
// acc_corr and its hi x hi product into one of the unit's n_hh accumulators (one
// issuing thread); accumulator i starts at column (1 + i) N.
__device__ __forceinline__ void issue_chunk(const GCtx& c, int NP, int ns, int s_global0) {
  const uint32_t idesc = idesc_bf16_f32(128, NP);
  const uint32_t aBase = smem_u32(c.A), bBase = smem_u32(c.B);
  // products (i, j) of the splits with 0 < i + j <= 2 (0 = hi, 1 = mid, 2 = lo)
  const int pa[5] = {0, 1, 0, 1, 2};
  const int pb[5] = {1, 0, 2, 1, 0};
  for (int s = 0; s < ns; ++s) {
    const int sg = s_global0 + s;
    const uint32_t ao = (uint32_t)s * 128u * 32u, bo = (uint32_t)s * (uint32_t)NP * 32u;
    for (int q = 0; q < 5; ++q) {
      const uint64_t da = smem_desc(aBase + pa[q] * c.aPlane + ao, 128, 256);
      const uint64_t db = smem_desc(bBase + pb[q] * c.bPlane + bo, 128, 256);
      mma_bf16(c.col_corr, da, db, idesc, (sg > 0 || q > 0) ? 1u : 0u);
    }
    const int n_hh = unit_n_hh(NP);
    const uint64_t da = smem_desc(aBase + ao, 128, 256);
    const uint64_t db = smem_desc(bBase + bo, 128, 256);
    mma_bf16(c.col_corr + (uint32_t)(1 + sg % n_hh) * (uint32_t)NP, da, db, idesc, sg >= n_hh ? 1u : 0u);
  }
}

// Bring the B planes of K steps [s0, s0 + ns) of a plane set (n_rows rows per K step)
// into the group's B buffer: three bulk copies completing on the group's barrier.
__device__ __forceinline__ void load_b(const GCtx& c, const uint16_t* src, long long plane_elems, int n_rows, int s0,
                                       int ns) {
  const uint32_t bytes = (uint32_t)ns * (uint32_t)n_rows * 32u;
  mbar_arrive_expect_tx(c.bar_b, 3u * bytes);
  for (int p = 0; p < 3; ++p)
    bulk_g2s(c.B + p * c.bPlane, src + p * plane_elems + (long long)s0 * n_rows * 16, bytes, c.bar_b);
}

// One chunk of the dense stage after the group has written its A operand: the B planes
// (unless resident), the products, and the wait for them.  Returns false on a timeout.
__device__ __forceinline__ bool run_chunk(const GCtx& c, bool need_b, int bkey, const uint16_t* bsrc,
                                          long long plane_elems, int NP, int s0, int ns) {
  if (c.t == 0 && need_b) load_b(c, bsrc, plane_elems, NP, s0, ns);
  fence_smem_to_async();
  fence_before_sync();
  group_sync(c.g);
  fence_after_sync();
  if (need_b) {
    const bool ok = group_wait(c.bar_b, *c.ph_b, c.status, c.g);
    if (c.t == 0) c.gs->bkey = ok ? bkey : -1;
    if (!ok) return false;
  }
  if (c.t == 0) {
    issue_chunk(c, NP, ns, s0);
    mma_commit(c.bar_mma);
  }
  const bool ok = group_wait(c.bar_mma, *c.ph_mma, c.status, c.g);
  fence_after_sync();
  return ok;
}

// Sum of the accumulators for 16 columns of this thread's tensor-memory lane (a dense
// stage N columns wide with n_used accumulators of hi x hi products).
__device__ __forceinline__ void acc_sum16(const GCtx& c, uint32_t lane_off, int c0, int N, int n_used, float* v) {
  float w[16];
  tmem_ld16(c.col_corr + lane_off + (uint32_t)c0, v);
  for (int i = 0; i < n_used; ++i) {
    tmem_ld16(c.col_corr + (uint32_t)(1 + i) * (uint32_t)N + lane_off + (uint32_t)c0, w);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] += w[k];
  }
}

// ---------------------------------------------------------------------------------------
// P: one unit.  NA, NB: compile-time orbital counts (EXACT) or upper bounds.
// ---------------------------------------------------------------------------------------
template <int NA, int NB, bool EXACT>
__device__ bool p_unit(const GCtx& c, const CSys& S, const DevEntry& E, int it, int sys) {
  const int na = EXACT ? NA : E.na, nb = EXACT ? NB : E.nb, Ka = E.Ka, Kb = E.Kb;
  const int nt = S.n_tau, im = nt - 1 - it;
  const int nbb = nb * nb;
  const int KD = (nbb + 15) & ~15, NP = (Kb + 15) & ~15;
  const int sa = S.species[E.a], sb = S.species[E.b];
  const float* Ca = S.Cp + S.cp_off[sa];  // [L][L''][K], K fastest
  const int ldk = S.cp_ld[sa];
  const uint16_t* bsrc = S.Bp + S.bp_off[3 * sb + E.tier];
  const long long plane_elems = (long long)NP * KD;
  const int n_chunks = (KD + c.kc - 1) / c.kc;
  const int bkey = (sys << 12) | (sb << 2) | E.tier;
  const int t = c.t;
  // G(tau) and conj(G(beta - tau)) transposed, in FP32
  float2* G1 = c.Gs;
  float2* G2t = c.Gs + kCMaxOrb * kCMaxOrb;
  {
    const double2* Gin = S.G + E.off_orb * nt;
    for (int x = t; x < na * nb; x += kTG) {
      const double2 g1 = __ldg(Gin + (long long)it * na * nb + x);
      const double2 g2 = __ldg(Gin + (long long)im * na * nb + x);
      G1[x] = make_float2(d2f(g1.x), d2f(g1.y));
      const int L2 = x / nb, L3 = x - L2 * nb;
      G2t[L3 * na + L2] = make_float2(d2f(g2.x), -d2f(g2.y));
    }
  }
  group_sync(c.g);
  double2* Pout = S.out + E.off_pb * nt;
  const float msf = -(float)S.spin;
  const bool mirror = S.mirror && im != it;
  const int n_tiles = (Ka + 63) / 64;
  for (int tile = 0; tile < n_tiles; ++tile) {
    const int K0 = 64 * tile, KL = min(64, Ka - K0);
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int j0 = ch * c.kc, jn = min(c.kc, KD - j0), ns = jn / 16;
      const bool need_b = n_chunks > 1 || c.gs->bkey != bkey;
      // A operand: rows kl (Re Y) and 64 + kl (Im Y) for K = K0 + kl; thread (kl, quarter q)
      // writes columns [q jn/4, (q + 1) jn/4) of the chunk, 4 at a time
      const int kl = t & 63, q = t >> 6;
      const int jq = jn / 4;
      const int ja = j0 + q * jq, jb = ja + jq;
      if (kl < KL) {
        const float* CK = Ca + K0 + kl;  // C^a[K][L][L''] at CK[(L na + L'') ldk]
        float xr[NA], xi[NA];
        int cur = -1;
        for (int j4 = ja; j4 < jb; j4 += 4) {
          uint32_t pk[6][2];
#pragma unroll
          for (int u2 = 0; u2 < 2; ++u2) {
            float yr2[2], yi2[2];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
              const int j = j4 + 2 * u2 + w;
              float yr = 0.f, yi = 0.f;
              if (j < nbb) {
                const int L1 = j / nb, L3 = j - L1 * nb;
                if (L1 != cur) {
#pragma unroll
                  for (int L2 = 0; L2 < NA; ++L2) { xr[L2] = 0.f; xi[L2] = 0.f; }
#pragma unroll
                  for (int L = 0; L < NA; ++L) {
                    if (EXACT || L < na) {
                      const float2 gv = G1[L * nb + L1];
                      const float* cr = CK + (long long)L * na * ldk;
#pragma unroll
                      for (int L2 = 0; L2 < NA; ++L2) {
                        if (EXACT || L2 < na) {
                          const float cv = __ldg(cr + (long long)L2 * ldk);
                          xr[L2] = fmaf(cv, gv.x, xr[L2]);
                          xi[L2] = fmaf(cv, gv.y, xi[L2]);
                        }
                      }
                    }
                  }
                  cur = L1;
                }
                const float2* g2 = G2t + L3 * na;
#pragma unroll
                for (int L2 = 0; L2 < NA; ++L2) {
                  if (EXACT || L2 < na) {
                    const float2 b = g2[L2];  // conj(G(beta - tau)[L''][L'''])
                    yr = fmaf(xr[L2], b.x, fmaf(-xi[L2], b.y, yr));
                    yi = fmaf(xr[L2], b.y, fmaf(xi[L2], b.x, yi));
                  }
                }
              }
              yr2[w] = yr;
              yi2[w] = yi;
            }
            split3x2(yr2[0], yr2[1], pk[0][u2], pk[1][u2], pk[2][u2]);
            split3x2(yi2[0], yi2[1], pk[3][u2], pk[4][u2], pk[5][u2]);
          }
          const int jl = j4 - j0;
          const uint32_t o_r = kmajor_offset(128, kl, jl), o_i = kmajor_offset(128, 64 + kl, jl);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            *reinterpret_cast<uint2*>(c.A + p * c.aPlane + o_r) = make_uint2(pk[p][0], pk[p][1]);
            *reinterpret_cast<uint2*>(c.A + p * c.aPlane + o_i) = make_uint2(pk[3 + p][0], pk[3 + p][1]);
          }
        }
      }
      if (!run_chunk(c, need_b, bkey, bsrc, plane_elems, NP, j0 / 16, ns)) return false;
    }
    // epilogue: tensor memory -> FP32 staging [kl][K'] over the A buffer (and the B buffer
    // when wider) -> FP64 P(tau) and, for a mirrored node, its conjugate at beta - tau
    const int n_used = min(unit_n_hh(NP), KD / 16);
    float2* Ps = reinterpret_cast<float2*>(c.A);
    const int ldp = NP + 1;
    {
      const int wq = c.warp & 3, half = (c.warp >> 2) & 1;
      const int r = 32 * wq + c.lane;
      const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
      const int n16 = NP / 16;
      for (int s16 = half; s16 < n16; s16 += 2) {
        const int c0 = 16 * s16;
        float v[16];
        acc_sum16(c, lane_off, c0, NP, n_used, v);
        const int klr = r & 63;
        if (klr < KL) {
          float* dst = reinterpret_cast<float*>(Ps + klr * ldp + c0) + (r >> 6);
#pragma unroll
          for (int k = 0; k < 16; ++k) dst[2 * k] = v[k];
        }
      }
    }
    fence_before_sync();
    group_sync(c.g);
    {
      double2* Pt = Pout + (long long)it * Ka * Kb + (long long)K0 * Kb;
      double2* Pm = Pout + (long long)im * Ka * Kb + (long long)K0 * Kb;
      // rows over the group's warps, columns over the lanes (consecutive stores)
      for (int klx = t >> 5; klx < KL; klx += kTG / 32)
        for (int Kp = t & 31; Kp < Kb; Kp += 32) {
          const float2 p = Ps[klx * ldp + Kp];
          const float zr = msf * p.x, zi = msf * p.y;  // -s is a power of two: exact
          const double dr = f2d(zr), di = f2d(zi);
          const int x = klx * Kb + Kp;
          Pt[x] = make_double2(dr, di);
          if (mirror) Pm[x] = make_double2(dr, dneg(di));
        }
    }
    // a staging wider than the A buffer overwrote the B operand
    if (t == 0 && (uint32_t)(64 * ldp * 8) > c.a_bytes) c.gs->bkey = -1;
    group_sync(c.g);
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Sigma: one unit.
// ---------------------------------------------------------------------------------------
template <int NA, int NB, bool EXACT>
__device__ bool s_unit(const GCtx& c, const CSys& S, const DevEntry& E, int it, int sys) {
  const int na = EXACT ? NA : E.na, nb = EXACT ? NB : E.nb, Ka = E.Ka, Kb = E.Kb;
  const int nbb = nb * nb;
  const int KD = (Kb + 15) & ~15, NJ = (nbb + 15) & ~15;
  const int sa = S.species[E.a], sb = S.species[E.b];
  const float* Ca = S.Cp + S.cp_off[sa];  // [L][L''][K], K fastest
  const int ldk = S.cp_ld[sa];
  const uint16_t* bsrc = S.Bp + S.bp_off[3 * sb + E.tier];
  const long long plane_elems = (long long)NJ * KD;
  const int n_chunks = (KD + c.kc - 1) / c.kc;
  const int bkey = (sys << 12) | (sb << 2) | E.tier;
  const int t = c.t;
  const double2* Win = S.W + E.off_pb * S.w_slices + (long long)it * Ka * Kb;
  {
    const int gs = S.g_fixed >= 0 ? S.g_fixed : it;
    const double2* Gin = S.G + E.off_orb * S.g_slices + (long long)gs * na * nb;
    for (int x = t; x < na * nb; x += kTG) {
      const double2 gv = __ldg(Gin + x);
      c.Gs[x] = make_float2(d2f(gv.x), d2f(gv.y));
    }
  }
  group_sync(c.g);
  // stage-C thread mapping: thread (L, ks) sums over K = ks, ks + nks_t, ...
  const int nks_t = kTG / na;
  const int Lr = t / nks_t, ks = t - Lr * nks_t;
  const bool sc_on = Lr < na;
  float accr[NB], acci[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) { accr[i] = 0.f; acci[i] = 0.f; }
  const int n_tiles = (Ka + 63) / 64;
  for (int tile = 0; tile < n_tiles; ++tile) {
    const int K0 = 64 * tile, KL = min(64, Ka - K0);
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int k0 = ch * c.kc, kn = min(c.kc, KD - k0), ns = kn / 16;
      const bool need_b = n_chunks > 1 || c.gs->bkey != bkey;
      // A operand: rows kl (Re W~) and 64 + kl (Im W~), reduction K' in groups of 8
      const int n8 = kn / 8;
      for (int x = t; x < 64 * n8; x += kTG) {
        const int kl = x / n8, q8 = x - kl * n8;
        if (kl >= KL) continue;
        const int kk = k0 + 8 * q8;
        uint32_t pk[6][4];
        const double2* wrow = Win + (long long)(K0 + kl) * Kb;
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
          float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
          const int k = kk + 2 * u2;
          if (k < Kb) { const double2 w = __ldg(wrow + k); a0 = d2f(w.x); b0 = d2f(w.y); }
          if (k + 1 < Kb) { const double2 w = __ldg(wrow + k + 1); a1 = d2f(w.x); b1 = d2f(w.y); }
          split3x2(a0, a1, pk[0][u2], pk[1][u2], pk[2][u2]);
          split3x2(b0, b1, pk[3][u2], pk[4][u2], pk[5][u2]);
        }
        const uint32_t o_r = kmajor_offset(128, kl, kk - k0), o_i = kmajor_offset(128, 64 + kl, kk - k0);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          *reinterpret_cast<uint4*>(c.A + p * c.aPlane + o_r) = make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
          *reinterpret_cast<uint4*>(c.A + p * c.aPlane + o_i) =
              make_uint4(pk[3 + p][0], pk[3 + p][1], pk[3 + p][2], pk[3 + p][3]);
        }
      }
      if (!run_chunk(c, need_b, bkey, bsrc, plane_elems, NJ, k0 / 16, ns)) return false;
    }
    // Bm[kl][L'][L'''] (complex FP32) from tensor memory into the A buffer, in passes over L'
    const int n_used = min(unit_n_hh(NJ), KD / 16);
    float2* Bm = reinterpret_cast<float2*>(c.A);
    const int ldb = (nb + 1) & ~1;  // padded L''' stride (float2): rows 16-byte aligned
    const int cap = (int)(c.a_bytes / 8u) / (64 * ldb);
    const int per_pass = max(1, min(nb, cap));
    for (int l0 = 0; l0 < nb; l0 += per_pass) {
      const int l1 = min(nb, l0 + per_pass), np_ = l1 - l0;
      const int jlo = l0 * nb, jhi = l1 * nb;
      {
        const int wq = c.warp & 3, wsub = (c.warp >> 2) & 1;
        const int r = 32 * wq + c.lane;
        const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
        for (int s16 = (jlo >> 4) + wsub; 16 * s16 < jhi; s16 += 2) {
          const int c0 = 16 * s16;
          float v[16];
          acc_sum16(c, lane_off, c0, NJ, n_used, v);
          const int kl = r & 63;
          if (kl < KL) {
            float* dst = reinterpret_cast<float*>(Bm + kl * (np_ * ldb)) + (r >> 6);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int j = c0 + k;
              if (j >= jlo && j < jhi) {
                const int L1 = j / nb, L3 = j - L1 * nb;
                dst[2 * ((L1 - l0) * ldb + L3)] = v[k];
              }
            }
          }
        }
      }
      fence_before_sync();
      group_sync(c.g);
      if (sc_on) {
        for (int kl = ks; kl < KL; kl += nks_t) {
          const float* CK = Ca + (long long)Lr * na * ldk + K0 + kl;  // C^a[K][L][L''] at CK[L'' ldk]
          float hr[NB], hi[NB];
#pragma unroll
          for (int L3 = 0; L3 < NB; ++L3) { hr[L3] = 0.f; hi[L3] = 0.f; }
#pragma unroll
          for (int L2 = 0; L2 < NA; ++L2) {
            if (EXACT || L2 < na) {
              const float cv = __ldg(CK + (long long)L2 * ldk);
              const float2* gr = c.Gs + L2 * nb;
#pragma unroll
              for (int L3 = 0; L3 < NB; ++L3) {
                if (EXACT || L3 < nb) {
                  const float2 gv = gr[L3];
                  hr[L3] = fmaf(cv, gv.x, hr[L3]);
                  hi[L3] = fmaf(cv, gv.y, hi[L3]);
                }
              }
            }
          }
          const float2* bk = Bm + kl * (np_ * ldb);
#pragma unroll
          for (int L1 = 0; L1 < NB; ++L1) {
            if (L1 >= l0 && L1 < l1) {
              const float2* b = bk + (L1 - l0) * ldb;
              float sr = 0.f, si = 0.f;
#pragma unroll
              for (int L3 = 0; L3 < NB; ++L3) {
                if (EXACT || L3 < nb) {
                  const float2 bv = b[L3];
                  sr = fmaf(hr[L3], bv.x, fmaf(-hi[L3], bv.y, sr));
                  si = fmaf(hr[L3], bv.y, fmaf(hi[L3], bv.x, si));
                }
              }
              accr[L1] += sr;
              acci[L1] += si;
            }
          }
        }
      }
      group_sync(c.g);
    }
  }
  // partial sums over ks -> the A buffer, then the sum per (L, L') and the store
  float2* part = reinterpret_cast<float2*>(c.A);
  if (sc_on) {
#pragma unroll
    for (int L1 = 0; L1 < NB; ++L1)
      if (EXACT || L1 < nb) part[(Lr * nks_t + ks) * kCMaxOrb + L1] = make_float2(accr[L1], acci[L1]);
  }
  group_sync(c.g);
  double2* op = S.out + E.off_orb * S.out_slices + (long long)it * na * nb;
  const float sgn = (float)S.sign;  // +-1: exact
  for (int o = t; o < na * nb; o += kTG) {
    const int L = o / nb, L1 = o - L * nb;
    float sr = 0.f, si = 0.f;
    for (int k2 = 0; k2 < nks_t; ++k2) {
      const float2 p = part[(L * nks_t + k2) * kCMaxOrb + L1];
      sr += p.x;
      si += p.y;
    }
    op[o] = make_double2(f2d(sgn * sr), f2d(sgn * si));
  }
  group_sync(c.g);
  return true;
}

// Take the next unit of the queue for the group (one thread fetches, the group reads).
// Bring a unit's inputs into L2 (bulk prefetches of 16-byte aligned, whole-block ranges):
// the slices of G it reads and, for Sigma, its block of W~.
__device__ __forceinline__ void prefetch_unit(const CBatch& batch, const CUnit& u, bool sigma) {
  const CSys& S = batch.s[u.sys];
  const DevEntry E = S.ent[u.e];
  const uint32_t gb = (uint32_t)(E.na * E.nb) * 16u;
  const int gs = S.g_fixed >= 0 ? S.g_fixed : u.tau;
  const double2* G = S.G + E.off_orb * S.g_slices;
  prefetch_l2(G + (long long)gs * E.na * E.nb, gb);
  if (!sigma) {
    prefetch_l2(G + (long long)(S.n_tau - 1 - u.tau) * E.na * E.nb, gb);
    return;
  }
  const char* w = reinterpret_cast<const char*>(S.W + E.off_pb * S.w_slices + (long long)u.tau * E.Ka * E.Kb);
  const long long wb = (long long)E.Ka * E.Kb * 16;
  for (long long o = 0; o < wb; o += 32768) prefetch_l2(w + o, (uint32_t)min(32768ll, wb - o));
}

// The group's next unit: the one claimed on the previous call (or a fresh claim).  After
// the group has it, one thread of the second warp claims the unit after it and prefetches
// that unit's input, off the path of the others, so that it streams in during this one.
__device__ __forceinline__ bool next_unit(GroupState* gs, const CBatch& batch, const CUnit* units, int n_units,
                                          int* counter, const volatile int* status, int g, bool sigma) {
  if ((threadIdx.x % kTG) == 0) {
    int i = n_units;
    if (!(*status == 2 || gs->stop)) i = gs->next >= 0 ? gs->next : atomicAdd(counter, 1);
    if (i < n_units) gs->u = units[i];
    else gs->stop = 1;
  }
  group_sync(g);
  if ((threadIdx.x % kTG) == 32 && !gs->stop) {
    // read again by thread 0 only at the next call, after this unit's group barriers
    const int j = atomicAdd(counter, 1);
    gs->next = j;
    if (j < n_units) prefetch_unit(batch, units[j], sigma);
  }
  return !gs->stop;
}

template <bool SIGMA>
__global__ void __launch_bounds__(2 * kTG, 1)
k_contract(const __grid_constant__ CBatch batch, const CUnit* __restrict__ units, int n_units, int* counter, int kc,
           int n_cols, int n_hh, int n_groups, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tmem_base;
  __shared__ GroupState gst[2];
  __shared__ __align__(8) uint64_t bars[2][2];  // per group: products done, B loaded
  const int g = threadIdx.x / kTG;
  const GLayout GL = glayout(kc, n_cols);
  GCtx c;
  c.g = g;
  c.t = threadIdx.x % kTG;
  c.warp = threadIdx.x >> 5;
  c.lane = threadIdx.x & 31;
  unsigned char* base = sm + (size_t)g * GL.total;
  c.A = base + GL.a;
  c.B = base + GL.b;
  c.Gs = reinterpret_cast<float2*>(base + GL.g);
  c.aPlane = 128u * (uint32_t)kc * 2u;
  c.bPlane = (uint32_t)n_cols * (uint32_t)kc * 2u;
  c.a_bytes = 3u * c.aPlane;
  c.n_cols = (uint32_t)n_cols;
  c.n_hh = n_hh;
  c.kc = kc;
  c.bar_mma = &bars[g][0];
  c.bar_b = &bars[g][1];
  c.gs = &gst[g];
  c.status = status;
  uint32_t ph_mma = 0, ph_b = 0;
  c.ph_mma = &ph_mma;
  c.ph_b = &ph_b;
  if (c.warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (c.t == 0) {
    mbar_init(c.bar_mma, 1);
    mbar_init(c.bar_b, 1);
    fence_mbar_init();
    gst[g].bkey = -1;
    gst[g].stop = 0;
    gst[g].next = -1;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = tmem_base + (512u / (uint32_t)n_groups) * (uint32_t)g;
  c.col_corr = tm;
  c.col_hh = tm + (uint32_t)n_cols;
  while (next_unit(c.gs, batch, units, n_units, counter, status, g, SIGMA)) {
    const CUnit u = c.gs->u;
    const CSys& S = batch.s[u.sys];
    const DevEntry E = S.ent[u.e];
    bool ok;
    if (SIGMA) {
      if (E.na == 9 && E.nb == 9) ok = s_unit<9, 9, true>(c, S, E, u.tau, u.sys);
      else if (E.na == 4 && E.nb == 4) ok = s_unit<4, 4, true>(c, S, E, u.tau, u.sys);
      else ok = s_unit<kCMaxOrb, kCMaxOrb, false>(c, S, E, u.tau, u.sys);
    } else {
      if (E.na == 9 && E.nb == 9) ok = p_unit<9, 9, true>(c, S, E, u.tau, u.sys);
      else if (E.na == 4 && E.nb == 4) ok = p_unit<4, 4, true>(c, S, E, u.tau, u.sys);
      else ok = p_unit<kCMaxOrb, kCMaxOrb, false>(c, S, E, u.tau, u.sys);
    }
    if (!ok && c.t == 0) c.gs->stop = 1;
    group_sync(g);
  }
  fence_before_sync();
  __syncthreads();
  if (c.warp == 0) tmem_dealloc(tmem_base, 512);
}

// Round to BF16 (nearest even) on the host; returns the bits and the rounded value.
uint16_t bf16_round_host(double c, double* rounded) {
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

// Three BF16 terms of c at element (r, k) of the three planes of an R-row operand.
void put_split(std::vector<uint16_t>& buf, size_t plane, int R, int r, int k, double c) {
  const uint32_t off = umma::kmajor_offset(R, r, k) / 2;
  for (int q = 0; q < 3; ++q) {
    double rd;
    buf[q * plane + off] = bf16_round_host(c, &rd);
    c -= rd;
  }
}

template <typename T>
cudaError_t upload_vec(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

gw_status ctables_init(CTables& t, const HostPlan& h) {
  t.ready = false;
  for (int s = 0; s < h.n_species; ++s)
    if (h.n_orb[s] > kCMaxOrb || h.n_prod[s] > kCMaxProd) return GW_OK;  // outside the kernels' limits
  // C in FP32 as [L][L''][K] (K fastest, so that threads of consecutive K read
  // consecutive words), K padded to a multiple of 4
  std::vector<float> Cp;
  std::vector<int> cp_off, cp_ld;
  for (int s = 0; s < h.n_species; ++s) {
    const int n = h.n_orb[s], K = h.n_prod[s], ld = (K + 3) & ~3;
    cp_off.push_back((int)Cp.size());
    cp_ld.push_back(ld);
    for (int x = 0; x < n * n; ++x)
      for (int k = 0; k < ld; ++k) Cp.push_back(k < K ? (float)h.C[s][(size_t)k * n * n + x] : 0.f);
  }
  // B planes per (species, size): P rows K' and reduction j; Sigma rows j and reduction K'
  std::vector<uint16_t> bpP, bpS;
  std::vector<long long> offP, offS;
  t.np_max = t.kd_max = t.nj_max = t.kds_max = 0;
  for (int sv = 0; sv < 3 * h.n_species; ++sv) {
    const int s = sv / 3, tier = sv % 3;
    const int n = h.n_orb[s], K = tier == 0 ? h.n_prod[s] : tier == 1 ? h.n_prod_near[s] : h.n_prod_far[s];
    const int nn = n * n;
    const int KD = (nn + 15) & ~15, NP = (K + 15) & ~15;
    t.np_max = std::max(t.np_max, NP);
    t.kd_max = std::max(t.kd_max, KD);
    t.nj_max = std::max(t.nj_max, KD);
    t.kds_max = std::max(t.kds_max, NP);
    offP.push_back((long long)bpP.size());
    {
      const size_t plane = (size_t)NP * KD;
      std::vector<uint16_t> buf(3 * plane, 0);
      for (int Kp = 0; Kp < K; ++Kp)
        for (int j = 0; j < nn; ++j) put_split(buf, plane, NP, Kp, j, h.C[s][(size_t)Kp * nn + j]);
      bpP.insert(bpP.end(), buf.begin(), buf.end());
    }
    offS.push_back((long long)bpS.size());
    {
      const size_t plane = (size_t)KD * NP;  // rows j (KD of them), reduction K' (NP)
      std::vector<uint16_t> buf(3 * plane, 0);
      for (int Kp = 0; Kp < K; ++Kp)
        for (int j = 0; j < nn; ++j) put_split(buf, plane, KD, j, Kp, h.C[s][(size_t)Kp * nn + j]);
      bpS.insert(bpS.end(), buf.begin(), buf.end());
    }
  }
  cudaError_t e = upload_vec(&t.d_Cp, Cp);
  if (e == cudaSuccess) e = upload_vec(&t.d_cp_off, cp_off);
  if (e == cudaSuccess) e = upload_vec(&t.d_cp_ld, cp_ld);
  if (e == cudaSuccess) e = upload_vec(&t.d_BpP, bpP);
  if (e == cudaSuccess) e = upload_vec(&t.d_bpP_off, offP);
  if (e == cudaSuccess) e = upload_vec(&t.d_BpS, bpS);
  if (e == cudaSuccess) e = upload_vec(&t.d_bpS_off, offS);
  if (e == cudaSuccess) e = upload_vec(&t.d_species, h.species);
  if (e != cudaSuccess) {
    set_last_error(std::string("contraction tables: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  t.ready = true;
  return GW_OK;
}

void ctables_free(CTables& t) {
  cudaFree(t.d_Cp);
  cudaFree(t.d_cp_off);
  cudaFree(t.d_cp_ld);
  cudaFree(t.d_BpP);
  cudaFree(t.d_bpP_off);
  cudaFree(t.d_BpS);
  cudaFree(t.d_bpS_off);
  cudaFree(t.d_species);
  t = CTables();
}

std::vector<CUnit> contract_units(const HostPlan& h, int sys, bool sigma, int n_nodes) {
  const int E = h.n_entries();
  const int ne = n_nodes > 0 ? n_nodes : (!sigma && h.c_symmetric) ? (h.n_tau + 1) / 2 : h.n_tau;
  std::vector<int> order(E);
  for (int e = 0; e < E; ++e) order[e] = e;
  auto key = [&](int e) {
    const int a = (int)h.entries[8 * e], b = (int)h.entries[8 * e + 1];
    return (h.species[b] * 3 + h.tier_e[e]) * 64 + h.species[a];
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
  std::vector<CUnit> u;
  u.reserve((size_t)E * ne);
  for (int e : order)
    for (int i = 0; i < ne; ++i) u.push_back({sys, e, i, 0});
  return u;
}

long long contract_unit_cost(const HostPlan& h, int e, bool sigma) {
  const int a = (int)h.entries[8 * e], b = (int)h.entries[8 * e + 1];
  const long long na = h.n_orb[h.species[a]], nb = h.n_orb[h.species[b]];
  const long long Ka = h.Ka_e[e], Kb = h.Kb_e[e];
  (void)sigma;
  return 2 * Ka * na * na * nb + 4 * Ka * na * nb * nb + 2 * Ka * Kb * nb * nb;
}

gw_status contract_config(bool sigma, int n_cols_max, int kd_max, CConfig& c, int device, int groups_req,
                          int kc_req) {
  c.n_cols = n_cols_max;
  c.groups = (sigma && n_cols_max > 128) ? 1 : 2;
  if (groups_req == 1 || (groups_req == 2 && c.groups == 2)) c.groups = groups_req;
  const int cols_g = 512 / c.groups;
  c.n_hh = cols_g / n_cols_max - 1;
  if (c.n_hh < 1 || n_cols_max > 256) {
    set_last_error("contraction: dense-stage width beyond the tensor-memory budget");
    return GW_ERR_UNSUPPORTED;
  }
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (smem_max <= 0) smem_max = 227 * 1024;
  const size_t budget = (size_t)smem_max - 1024;  // static shared memory and alignment
  // the epilogue stages its results over the operand buffers: P 64 rows of up to
  // n_cols + 1 FP32 pairs over A and B, Sigma 256 threads x 16 FP32 pairs over A; the
  // chunk is at least what these need (a chunk longer than the reduction only costs space)
  auto fits_epilogue = [&](int k) {
    const GLayout L = glayout(k, n_cols_max);
    return sigma ? (size_t)kTG * kCMaxOrb * 8 <= L.b : (size_t)64 * (n_cols_max + 1) * 8 <= L.g;
  };
  int kc_min = 16;
  while (kc_min <= 256 && !fits_epilogue(kc_min)) kc_min += 16;
  int kc = std::max(kc_min, (kd_max + 15) & ~15);
  if (kc_req > 0) kc = std::max(kc_min, std::min(kc, kc_req & ~15));
  for (; kc >= kc_min; kc -= 16)
    if ((size_t)c.groups * glayout(kc, n_cols_max).total <= budget) break;
  if (kc < kc_min || kc_min > 256) {
    set_last_error("contraction: no reduction chunk fits shared memory");
    return GW_ERR_UNSUPPORTED;
  }
  const GLayout L = glayout(kc, n_cols_max);
  c.kc = kc;
  // more than half of the SM's shared memory: one block per SM, so that no two blocks
  // compete for the 512 tensor-memory columns each allocates
  c.smem = std::max((size_t)c.groups * L.total, (size_t)smem_max / 2 + 1024);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  c.grid = std::max(1, sms);
  cudaError_t e = sigma ? raise_smem_limit(k_contract<true>, c.smem) : raise_smem_limit(k_contract<false>, c.smem);
  if (e != cudaSuccess) {
    set_last_error(std::string("contraction: shared-memory opt-in: ") + cudaGetErrorString(e));
    return GW_ERR_UNSUPPORTED;
  }
  return GW_OK;
}

gw_status contract_launch(bool sigma, const CConfig& c, const CBatch& b, const CUnit* d_units, int n_units,
                          int* d_counter, int* d_status, cudaStream_t st) {
  if (n_units <= 0) return GW_OK;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  const int grid = std::min(c.grid, (n_units + c.groups - 1) / c.groups);
  if (e == cudaSuccess) {
    gw::TimedLaunch tl_(sigma ? "k_contract_s_tc" : "k_contract_p_tc", st);
    if (sigma)
      k_contract<true><<<grid, c.groups * kTG, c.smem, st>>>(b, d_units, n_units, d_counter, c.kc, c.n_cols, c.n_hh,
                                                              c.groups, d_status);
    else
      k_contract<false><<<grid, c.groups * kTG, c.smem, st>>>(b, d_units, n_units, d_counter, c.kc, c.n_cols, c.n_hh,
                                                               c.groups, d_status);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string(sigma ? "k_contract_s_tc: " : "k_contract_p_tc: ") + cudaGetErrorString(e));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
