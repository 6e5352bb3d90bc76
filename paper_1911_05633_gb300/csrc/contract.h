// Persistent tensor-core contractions of Eqs. P_MM and S_MM (the mixed-precision path)
// over a queue of work units, for one system or a batch of systems of uneven sizes.
//
// A unit is (system, pair entry, tau node, row tile): the P or Sigma block of one
// entry at one imaginary-time node, restricted to 64 product functions K of atom a
// (entries with K_a > 64 have two row tiles).  One launch drains the whole queue with
// one resident block per SM; each block runs two independent thread groups, so that
// one group's CUDA-core stages overlap the other's tensor-core products and stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"

namespace gw {

// One system of a launch (device-visible; all pointers are device pointers).
struct CSys {
  const DevEntry* ent;       // the plan's entry table
  const float* Cp;           // C^s[K][L][L''] in FP32, stored [L][L''][K] (K fastest)
  const int* cp_off;         // [n_species] first float of species s in Cp
  const int* cp_ld;          // [n_species] K stride of species s (n_prod padded to a multiple of 4)
  const uint16_t* Bp;        // BF16 three-term planes of the dense-stage B operand, per (species, size)
  const long long* bp_off;   // [3 n_species] first element of the plane set of (species, level)
  const int* species;        // [n_atoms]
  const double2* G;          // G(R, tau): orbital entry layout, n_tau slices
  const double2* W;          // W~(R, tau): product entry layout, n_tau slices (Sigma only)
  double2* out;              // P (product layout) or Sigma (orbital layout), n_tau slices
  int n_tau;
  // Sigma: slices of G, W~ and the output per entry, a fixed G slice (-1: the unit's node)
  // and the sign of the result (-1: Eq. S_MM; +1: the exchange term with W~ -> v and
  // G(tau) -> G(beta-), one slice each of W and of the output)
  int g_slices, w_slices, out_slices, g_fixed;
  double sign;
  int spin;                  // P: spin degeneracy s
  int mirror;                // P: the nodes i < ceil(n_tau/2) are computed, the node n_tau-1-i written
                             // as the conjugate (C symmetric in (L, L''))
};

struct CUnit {
  int sys, e, tau, tile;
};

// The systems of one launch, passed by value as a kernel parameter (no host-to-device
// copy per call, so a launch can be captured in a CUDA graph).
constexpr int kMaxBatch = 24;
struct CBatch {
  int n;
  CSys s[kMaxBatch];
};

// Shape limits of the contraction kernels (the library's compiled maxima).
constexpr int kCMaxOrb = 16;
constexpr int kCMaxProd = 128;

// Host-side description of one system's tables for the contraction kernels.
struct CTables {
  float* d_Cp = nullptr;
  int* d_cp_off = nullptr;
  int* d_cp_ld = nullptr;
  uint16_t* d_BpP = nullptr;   // P: rows K' (N = K_b padded to 16), reduction j = (L', L''') (padded to 16)
  long long* d_bpP_off = nullptr;
  uint16_t* d_BpS = nullptr;   // Sigma: rows j = (L', L''') (N = n_b^2 padded to 16), reduction K' (padded to 16)
  long long* d_bpS_off = nullptr;
  int* d_species = nullptr;
  int np_max = 0, kd_max = 0;    // P: largest padded N and reduction length
  int nj_max = 0, kds_max = 0;   // Sigma: the same
  bool ready = false;
};

gw_status ctables_init(CTables& t, const HostPlan& h);
void ctables_free(CTables& t);

// The queue of one system's units for P (computed nodes only) or Sigma (n_nodes nodes:
// N_tau, or 1 for the exchange term), grouped by (species a, species b, reduced size) so
// that consecutive units share their B operand.
std::vector<CUnit> contract_units(const HostPlan& h, int sys, bool sigma, int n_nodes = -1);

// Launch configuration (per batch): reduction chunk, accumulators, thread groups and
// dynamic shared memory, from the largest shapes of the batch.
struct CConfig {
  int kc = 0;        // reduction chunk (multiple of 16)
  int n_hh = 1;      // accumulators of the hi x hi products
  int n_cols = 0;    // N of the dense stage (largest padded N of the batch)
  int groups = 2;    // thread groups per block (1 when the Sigma stage is wider than 128)
  size_t smem = 0;
  int grid = 0;
};

// groups_req: 0 automatic (two groups unless the Sigma stage is wider than 128 columns),
// else 1 or 2; kc_req: 0 the longest chunk that fits, else that chunk (clamped to what fits).
gw_status contract_config(bool sigma, int np_or_nj_max, int kd_max, CConfig& c, int device, int groups_req = 0,
                          int kc_req = 0);

// Estimated work of a unit (for ordering the queue heaviest first).
long long contract_unit_cost(const HostPlan& h, int e, bool sigma);

// Queue launch: d_units [n_units] CUnit; d_counter one int (reset here, on the stream);
// d_status the error word (2 = a bounded wait gave up).
gw_status contract_launch(bool sigma, const CConfig& c, const CBatch& b, const CUnit* d_units, int n_units,
                          int* d_counter, int* d_status, cudaStream_t st);

}  // namespace gw
