// Internal declarations shared by the host plan builder, the C ABI and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gw.h"

namespace gw {

constexpr int kMaxOrb = 16;    // orbitals per atom
constexpr int kMaxProd = 128;  // product functions per atom
constexpr int kMaxTau = 128;   // imaginary-time nodes

// Per-entry table used by every kernel (one pair entry e = (a, b, R)).
struct DevEntry {
  int a, b;            // atoms
  int na, nb;          // orbitals of a, b
  int Ka, Kb;          // product functions of a, b
  int oa, ob;          // first orbital of a, b in the dense k-space matrices
  int pa, pb;          // first product function of a, b
  int ca, cb;          // offset of C^{species(a)}, C^{species(b)} in the packed C array
  long long off_orb;   // prefix sum of na*nb over earlier entries
  long long off_pb;    // prefix sum of Ka*Kb over earlier entries
  int mirror;          // entry index of (b, a, -R)
  int tier;            // product-basis level (Sec. 2, Fig. 2): 0 one sphere, 1 within sphere B, 2 beyond
};

// Host-side tables of a plan (no CUDA types; built by build_host_plan()).
struct HostPlan {
  double lat[9];
  int n_atoms = 0;
  std::vector<double> frac;
  std::vector<int> species;
  int n_species = 0;
  std::vector<int> n_orb, n_prod;
  std::vector<int> n_prod_far;          // per species: product functions kept beyond r_b
  std::vector<int> n_prod_near;         // per species: kept by two spheres within r_b
  double r_b = 0;                       // radius of sphere B (<= 0: no reduced tier)
  std::vector<std::vector<double>> C;  // per species [K][n][n]
  int kmesh[3];
  int n_k = 0;
  double beta = 0;
  int n_tau = 0, n_omega = 0, n_nu = 0;
  std::vector<double> tau;
  std::vector<int> omega_idx, nu_idx;
  double cutoff = 0;
  int spin = 2;

  // derived
  std::vector<int> orb_off, pb_off;       // [n_atoms + 1]
  std::vector<int64_t> entries;           // [E][8]
  std::vector<int64_t> off_orb, off_pb;   // [E + 1]
  std::vector<int> Ka_e, Kb_e;            // [E] product functions of a and b kept by entry e
  std::vector<int> tier_e;                // [E] product-basis level: 0 sphere A, 1 B, 2 C
  int n_far = 0;                          // entries beyond sphere B
  int n_near = 0;                         // entries within sphere B keeping n_prod_near < n_prod
  std::vector<int> pair_start;            // [n_atoms^2 + 1] entry range per ordered atom pair
  std::vector<int> mirror;                // [E]
  std::vector<double> phase;              // [E][N_k] complex e^{+i k.R}
  std::vector<signed char> phase_code;    // [E][N_k] c with e^{+i k.R} = i^c, when every phase is one (else empty)
  std::vector<double> Tf_fwd, Tf_inv, Tb_fwd, Tb_inv;  // complex matrices
  // bosonic tau -> i nu for inputs with F(beta - tau) = conj(F(tau)): coefficients
  // (a, b) per (frequency, node i < ceil(N_tau / 2)) with Re out = sum a Re F + b Im F
  std::vector<double> Tb_mirror;
  std::vector<int> c_off;                 // per species offset into packed C
  std::vector<double> C_packed;
  int kmesh_required[3] = {0, 0, 0};
  int c_symmetric = 1;
  double cond_f = 0, cond_b = 0;

  int n_entries() const { return (int)(entries.size() / 8); }
  int n_orb_total() const { return orb_off.back(); }
  int n_pb_total() const { return pb_off.back(); }
};

// Builds every host table; returns GW_OK or an error with a message.
gw_status build_host_plan(const gw_cell* cell, const gw_basis* basis, const int kmesh[3],
                          const gw_grid* grid, double cutoff, const gw_options* opt,
                          HostPlan& hp, std::string& err);

std::vector<DevEntry> make_dev_entries(const HostPlan& hp);

void set_last_error(const std::string& msg);

}  // namespace gw
