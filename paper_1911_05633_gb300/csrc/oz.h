// FP64-accurate stage A of the Sigma contraction (Eq. S_MM) on the tensor cores:
//   B[e][tau][K][j] = sum_K2 W~[e][tau][K][K2] C^b[K2][j],  j = (L', L''')
// as a row GEMM over rows (entry, tau, K, Re/Im) from exact BF16 digits of W~ (sliced
// per call) and of C^b (sliced once per plan).  Kernels in kernels_oz.cu; stages B and C
// of the contraction then run in FP64 on B (k_self_energy_fp64 with Bpre set).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace gw {

constexpr int kOzDigits = 8;   // base-2^7 digits per value
constexpr int kOzLmax = 7;     // digit products a_s b_t with s + t <= kOzLmax
constexpr int kOzBuckets = 6;  // accumulators: levels 0 .. 4 exactly, levels >= 5 together
constexpr int kOzMaxKS = 24;   // reduction length up to 384 (K steps of 16): levels 0-4 stay exact
constexpr int kOzStages = 4;   // shared-memory stages of one K step of both operands
constexpr uint32_t kOzAChunk = kOzDigits * 128 * 16 * 2;  // bytes of A digits per (row tile, K step)
__host__ __device__ constexpr uint32_t oz_bchunk(int NT) { return (uint32_t)kOzDigits * NT * 16 * 2; }
// dynamic shared memory of k_oz_gemm for KS K steps and NT columns
__host__ __device__ constexpr size_t oz_smem(int KS, int NT) {
  return (size_t)(KS < kOzStages ? KS : kOzStages) * (kOzAChunk + oz_bchunk(NT));
}

// Where k_oz_gemm writes its rows: Sigma stage A (B of one pass of tau slices), or a
// tau <-> i nu transform on the product-basis layout with a real input (columns:
// Re then Im of each output slice) or a real output (imaginary parts written as 0).
constexpr int kOzOutSigmaB = 0;
constexpr int kOzOutRealToComplex = 1;
constexpr int kOzOutReal = 2;
constexpr int kOzOutP = 3;  // P stage 3: P[e][s0 + sl][K][K'] = -s value (and the mirrored node)

struct OzGemmArgs {
  const DevEntry* ent;
  const int* tile_e;       // [tiles] entry of a 128-row tile
  const int* tile_r0;      // [tiles] its first row within the entry
  const uint16_t* Adig;    // [tiles][KS] digit chunks of the rows
  const int* eA;           // [tiles][128] row scale exponents
  int KS;                  // 16-wide K steps
  const uint16_t* Bdig;    // digit chunks of the column operand, [nt][KS] per matrix
  const long long* Boff;   // offset of each matrix in Bdig (uint16 units)
  const int* eB;           // column scale exponents
  const int* eBoff;        // offset of each matrix in eB
  const int* species;      // Sigma: species of each atom selects the matrix (else matrix 0)
  int NT;                  // columns per tile
  int mode;                // kOzOut*
  double2* out;
  const long long* offB;   // Sigma: [E] prefix sums of K_a n_b^2
  int tau_c, tau_eff;      // Sigma: slices per pass, slices in this pass
  int n_out;               // transforms: output slices
  int s0, n_tau, mirror;   // P: first computed node of the pass, N_tau, write the mirrored nodes
  double ms;               // P: -s
  int n_skip;              // transforms (real output): columns before it are not written
  int* status;
};

// Column operand of the fused transform kernel (k_oz_transform, kernels_oztf.cu): balanced
// digits d_s 2^-7s of B[n][k], [KS][kOzDigits][NT x 16] in the K-major layout, and the
// column scale exponents.
struct OzFused {
  bool ready = false;
  int K = 0, KS = 0;        // reduction length, 16-wide steps (<= 8)
  int n_cols = 0, NT = 0;   // columns, and columns per tile (a multiple of 16, <= 80)
  int n_ct = 0;             // column tiles
  bool wide = false;        // level sums may pass 2^22 (K > 102)
  bool stage = false;       // the epilogue stages its sums in shared memory (KS <= 5)
  uint16_t* d_B = nullptr;  // per column tile [KS][kOzDigits][NT x 16]
  int* d_e = nullptr;       // [n_ct NT]
  size_t smem = 0;          // dynamic shared memory of the kernel
};

// FP64-accurate structured tau <-> i nu transforms of the product-basis layout.
struct OzTransform {
  bool ready_w = false;  // bosonic i nu -> tau of a real input
  bool ready_p = false;  // bosonic tau -> i nu of a mirror-paired input
  int n_tiles = 0, KSmax = 0;
  int* d_tile_e = nullptr;
  int* d_tile_r0 = nullptr;
  uint16_t* d_Adig = nullptr;
  int* d_eA = nullptr;
  // the two column operands
  int KS_w = 0, NT_w = 0, nt_w = 0, KS_p = 0, NT_p = 0, nt_p = 0;
  uint16_t* d_Bw = nullptr;
  int* d_ew = nullptr;
  uint16_t* d_Bp = nullptr;
  int* d_ep = nullptr;
  long long* d_zero64 = nullptr;  // {0}: offset of the single matrix
  int* d_zero32 = nullptr;
  size_t smem = 0;
  size_t bytes = 0;
  // the fused kernels (reduction <= 80 terms, <= 80 output columns); when both are ready
  // the digit planes above are not allocated
  OzFused fw, fp;
  OzFused fph;           // fp for the frequencies nu >= 0 only (GW_OUT_NONNEG)
  int nu_nonneg0 = 0;    // slice of the first sampled nu >= 0
  // the general complex transforms (reduction <= 128 terms, <= 256 output columns):
  // [fermionic tau -> i w, i w -> tau, bosonic tau -> i nu, i nu -> tau]
  OzFused fg[4];
  int* d_tile_e_orb = nullptr;   // row tiles of the orbital blocks (n_a n_b per entry)
  int* d_tile_r0_orb = nullptr;
  int n_tiles_orb = 0;
  int n_sm = 0;
};

gw_status oz_transform_init(OzTransform& o, const HostPlan& h);
// Plans the fused kernels for the plan's grids (needs the row tiles of o); fills o.fw, o.fp.
gw_status oz_fused_init(OzTransform& o, const HostPlan& h);
void oz_fused_free(OzTransform& o);
// A general (complex input) transform on the fused kernel: ready, and run.
bool oz_general_ready(const OzTransform& o, int fermion, int to_tau, bool pb);
gw_status oz_general_run(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int fermion, int to_tau, bool pb,
                         const double2* in, double2* out, int* d_status, cudaStream_t st);
// One fused transform (structure GW_IN_REAL or GW_IN_MIRROR) when its kernel is ready.
gw_status oz_fused_run(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int structure, const double2* in,
                       double2* out, int* d_status, cudaStream_t st);
void oz_transform_free(OzTransform& o);
// structure: GW_IN_REAL (bosonic i nu -> tau) or GW_IN_MIRROR (bosonic tau -> i nu), with
// GW_OUT_NONNEG the latter for the frequencies nu >= 0 only
gw_status oz_transform(OzTransform& o, const HostPlan& h, const DevEntry* d_ent, int structure, const double2* in,
                       double2* out, int* d_status, cudaStream_t st);

// FP64-accurate stage 3 of the P contraction (Eq. P_MM) on the tensor cores:
//   P[e][tau][K][K'] = -s sum_j Y[e][tau][K][j] C^b[K'][j],  j = (L', L''')
// with Y from the FP64 stages 1 and 2 (k_polarizability_fp64 with Ypre set).
struct OzPol {
  bool ready = false;
  int KS = 0, NT = 0, max_nt = 0;
  int tau_c = 0;       // computed nodes per pass
  int n_tiles = 0;
  size_t smem = 0;
  int* d_tile_e = nullptr;
  int* d_tile_r0 = nullptr;
  uint16_t* d_Adig = nullptr;
  int* d_eA = nullptr;
  uint16_t* d_Bdig = nullptr;   // per species: B[K'][j] = C[K'][j]
  long long* d_Boff = nullptr;
  int* d_eB = nullptr;
  int* d_eBoff = nullptr;
  int* d_species = nullptr;
  double2* d_Ypre = nullptr;    // [sum_e K_a n_b^2][tau_c]
  long long* d_offB = nullptr;  // [E] prefix sums of K_a n_b^2
  size_t bytes = 0;
};
gw_status oz_pol_init(OzPol& o, const HostPlan& h, size_t cap);
void oz_pol_free(OzPol& o);
// Stage 3 for the computed nodes s0 .. s0 + tau_eff - 1, Y in o.d_Ypre, into P_R (PB layout).
gw_status oz_pol_stage3(OzPol& o, const HostPlan& h, const DevEntry* d_ent, int s0, int tau_eff, double2* P_R,
                        int* d_status, cudaStream_t st);

struct OzSigma {
  bool ready = false;
  int KS = 0;          // K steps: max over species of ceil(K_b / 16)
  int NT = 0;          // output columns per tile (multiple of 16)
  int max_nt = 0;      // column tiles of the widest n_b^2
  int tau_c = 0;       // tau slices per pass
  int n_tiles = 0;     // 128-row tiles per pass
  size_t smem = 0;     // dynamic shared memory of the product kernel
  int* d_tile_e = nullptr;        // [n_tiles] entry of the tile
  int* d_tile_r0 = nullptr;       // [n_tiles] first row of the tile within its entry
  uint16_t* d_Adig = nullptr;     // [n_tiles][KS] chunks of kOzDigits planes of 128 x 16
  int* d_eA = nullptr;            // [n_tiles][128] row scale exponents
  uint16_t* d_Bdig = nullptr;     // per species [nt][KS] chunks of kOzDigits planes of NT x 16
  long long* d_Boff = nullptr;    // [n_species] offset of a species in d_Bdig (uint16 units)
  int* d_eB = nullptr;            // per species [nt * NT] column scale exponents
  int* d_eBoff = nullptr;         // [n_species]
  int* d_species = nullptr;       // [n_atoms]
  double2* d_Bpre = nullptr;      // [sum_e K_a n_b^2][tau_c]: stage A of one pass
  long long* d_offB = nullptr;    // [E] prefix sums of K_a n_b^2
  size_t bytes = 0;               // device memory held
};

// Plans the tensor-core stage A when every species fits (K_b <= 64) and allocates its
// scratch within `cap` bytes; leaves o.ready false otherwise.
gw_status oz_sigma_init(OzSigma& o, const HostPlan& h, size_t cap);
void oz_sigma_free(OzSigma& o);
// Stage A for slices s0 .. s0 + tau_eff - 1 of W~ (PB entry layout, n_tau slices) into o.d_Bpre.
gw_status oz_sigma_stage_a(OzSigma& o, const HostPlan& h, const DevEntry* d_ent, const double2* W, int s0,
                           int tau_eff, int* d_status, cudaStream_t st);

}  // namespace gw
