// Host-side plan tables: pair list (Sec. 2), lattice phases, packed product-basis
// coefficients and the tau <-> i omega matrices of the sparse Matsubara grid
// (Appendix A).  Plain C++17, no CUDA; runs once per plan.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <sstream>

#include "internal.h"

namespace gw {

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

double det3(const double* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Spacing of the lattice planes crossed by a_i: V / |a_j x a_k|.
double plane_spacing(const double* A, int i) {
  const double* u = A + 3 * ((i + 1) % 3);
  const double* v = A + 3 * ((i + 2) % 3);
  double c0 = u[1] * v[2] - u[2] * v[1];
  double c1 = u[2] * v[0] - u[0] * v[2];
  double c2 = u[0] * v[1] - u[1] * v[0];
  return std::fabs(det3(A)) / std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term recurrence).
void gauss_legendre(int M, std::vector<double>& x, std::vector<double>& w) {
  x.assign(M, 0.0);
  w.assign(M, 0.0);
  for (int k = 0; k < (M + 1) / 2; ++k) {
    long double z = std::cos(kPi * (k + 0.75) / (M + 0.5));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int n = 2; n <= M; ++n) {
        long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = M * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-18) break;
    }
    long double p0 = 1, p1 = z;
    for (int n = 2; n <= M; ++n) {
      long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    dp = M * (z * p1 - p0) / (z * z - 1);
    double wk = (double)(2.0L / ((1 - z * z) * dp * dp));
    x[k] = -(double)z;
    x[M - 1 - k] = (double)z;
    w[k] = wk;
    w[M - 1 - k] = wk;
  }
}

// Inverse of a real n x n matrix by Gauss-Jordan with partial pivoting (long double).
bool invert_real(int n, const std::vector<long double>& A_in, std::vector<long double>& Ainv) {
  std::vector<long double> A(A_in);
  Ainv.assign((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + i] = 1.0L;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs((double)A[(size_t)i * n + k]) > std::fabs((double)A[(size_t)p * n + k])) p = i;
    if (A[(size_t)p * n + k] == 0.0L) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
        std::swap(Ainv[(size_t)k * n + j], Ainv[(size_t)p * n + j]);
      }
    long double d = A[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) {
      A[(size_t)k * n + j] /= d;
      Ainv[(size_t)k * n + j] /= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      long double f = A[(size_t)i * n + k];
      if (f == 0.0L) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        Ainv[(size_t)i * n + j] -= f * Ainv[(size_t)k * n + j];
      }
    }
  }
  return true;
}

// Forward matrix T[r][i] = int_0^beta e^{i w_r tau} l_i(tau) dtau, with l_i the
// Lagrange polynomial of the tau nodes, expanded in Chebyshev polynomials of
// x = 2 tau / beta - 1 and integrated term by term by Gauss-Legendre quadrature.
std::vector<cd> fourier_matrix(double beta, const std::vector<double>& tau, const std::vector<int>& idx,
                               bool fermion, std::string& err) {
  const int N = (int)tau.size();
  const int R = (int)idx.size();
  std::vector<long double> V((size_t)N * N), Vinv;
  for (int j = 0; j < N; ++j) {
    long double x = 2.0L * tau[j] / beta - 1.0L;
    if (j == 0) x = -1.0L;
    if (j == N - 1) x = 1.0L;
    long double t0 = 1, t1 = x;
    for (int l = 0; l < N; ++l) {
      long double tl = (l == 0) ? t0 : (l == 1 ? t1 : 0);
      if (l >= 2) {
        long double t2 = 2 * x * t1 - t0;
        t0 = t1;
        t1 = t2;
        tl = t2;
      }
      V[(size_t)j * N + l] = tl;
    }
  }
  if (!invert_real(N, V, Vinv)) {
    err = "tau nodes are not distinct";
    return {};
  }
  double amax = 0;
  std::vector<double> a(R);
  for (int r = 0; r < R; ++r) {
    a[r] = fermion ? (2.0 * idx[r] + 1.0) * kPi / 2.0 : idx[r] * kPi;
    amax = std::max(amax, std::fabs(a[r]));
  }
  const int M = N + (int)std::ceil(amax) + 40;
  std::vector<double> xg, wg;
  gauss_legendre(M, xg, wg);
  // T_l(x_g) table
  std::vector<double> Tl((size_t)M * N);
  for (int g = 0; g < M; ++g) {
    double x = xg[g], t0 = 1, t1 = x;
    for (int l = 0; l < N; ++l) {
      double tl;
      if (l == 0) tl = 1;
      else if (l == 1) tl = x;
      else { double t2 = 2 * x * t1 - t0; t0 = t1; t1 = t2; tl = t2; }
      Tl[(size_t)g * N + l] = tl;
    }
  }
  std::vector<cd> out((size_t)R * N);
  std::vector<cd> Il(N);
  for (int r = 0; r < R; ++r) {
    std::fill(Il.begin(), Il.end(), cd(0, 0));
    for (int g = 0; g < M; ++g) {
      cd e = std::polar(wg[g], a[r] * xg[g]);
      const double* t = &Tl[(size_t)g * N];
      for (int l = 0; l < N; ++l) Il[l] += e * t[l];
    }
    cd pre = 0.5 * beta * std::polar(1.0, a[r]);
    for (int i = 0; i < N; ++i) {
      cd s(0, 0);
      for (int l = 0; l < N; ++l) s += Il[l] * (double)Vinv[(size_t)l * N + i];
      out[(size_t)r * N + i] = pre * s;
    }
  }
  return out;
}

// Least-squares inverse (pseudo-inverse) of a full-column-rank m x n complex
// matrix, m >= n, by Householder QR: U = R^{-1} Q^H (n x m).
bool pinv_qr(int m, int n, const std::vector<cd>& T, std::vector<cd>& U) {
  std::vector<cd> A(T);                   // row-major m x n, overwritten by R
  std::vector<cd> Q((size_t)m * m, 0.0);  // accumulate Q^H applied to I
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<cd> v(m);
  for (int k = 0; k < n; ++k) {
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += std::norm(A[(size_t)i * n + k]);
    nrm = std::sqrt(nrm);
    if (nrm == 0) return false;
    cd akk = A[(size_t)k * n + k];
    cd alpha = (std::abs(akk) > 0) ? -akk / std::abs(akk) * nrm : cd(-nrm, 0);
    for (int i = 0; i < m; ++i) v[i] = 0;
    v[k] = akk - alpha;
    for (int i = k + 1; i < m; ++i) v[i] = A[(size_t)i * n + k];
    double vn = 0;
    for (int i = k; i < m; ++i) vn += std::norm(v[i]);
    if (vn == 0) continue;
    // H = I - 2 v v^H / (v^H v); apply to A (columns k..n-1) and to Q (all columns)
    for (int j = k; j < n; ++j) {
      cd s = 0;
      for (int i = k; i < m; ++i) s += std::conj(v[i]) * A[(size_t)i * n + j];
      s *= 2.0 / vn;
      for (int i = k; i < m; ++i) A[(size_t)i * n + j] -= s * v[i];
    }
    for (int j = 0; j < m; ++j) {
      cd s = 0;
      for (int i = k; i < m; ++i) s += std::conj(v[i]) * Q[(size_t)i * m + j];
      s *= 2.0 / vn;
      for (int i = k; i < m; ++i) Q[(size_t)i * m + j] -= s * v[i];
    }
  }
  // Now A = R (upper n x n in the first n rows), Q holds Q^H (m x m).  U = R^{-1} (Q^H)[0:n, :]
  U.assign((size_t)n * m, 0.0);
  for (int j = 0; j < m; ++j) {
    for (int i = n - 1; i >= 0; --i) {
      cd s = Q[(size_t)i * m + j];
      for (int l = i + 1; l < n; ++l) s -= A[(size_t)i * n + l] * U[(size_t)l * m + j];
      if (std::abs(A[(size_t)i * n + i]) == 0) return false;
      U[(size_t)i * m + j] = s / A[(size_t)i * n + i];
    }
  }
  return true;
}

// Largest singular value of a complex r x c matrix by power iteration on M^H M.
double sigma_max(int r, int c, const std::vector<cd>& M) {
  std::vector<cd> x(c, 1.0), y(r);
  double s = 0;
  for (int it = 0; it < 300; ++it) {
    for (int i = 0; i < r; ++i) {
      cd t = 0;
      for (int j = 0; j < c; ++j) t += M[(size_t)i * c + j] * x[j];
      y[i] = t;
    }
    for (int j = 0; j < c; ++j) {
      cd t = 0;
      for (int i = 0; i < r; ++i) t += std::conj(M[(size_t)i * c + j]) * y[i];
      x[j] = t;
    }
    double n = 0;
    for (auto& z : x) n += std::norm(z);
    n = std::sqrt(n);
    if (n == 0) return 0;
    for (auto& z : x) z /= n;
    s = std::sqrt(n);
  }
  return s;
}

std::vector<double> to_interleaved(const std::vector<cd>& v) {
  std::vector<double> o(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    o[2 * i] = v[i].real();
    o[2 * i + 1] = v[i].imag();
  }
  return o;
}

}  // namespace

gw_status build_host_plan(const gw_cell* cell, const gw_basis* basis, const int kmesh[3],
                          const gw_grid* grid, double cutoff, const gw_options* opt,
                          HostPlan& hp, std::string& err) {
  if (!cell || !basis || !kmesh || !grid) { err = "null argument"; return GW_ERR_ARG; }
  if (cell->n_atoms <= 0 || !cell->frac || !cell->species) { err = "bad cell"; return GW_ERR_ARG; }
  if (basis->n_species <= 0 || !basis->n_orb || !basis->n_prod || !basis->C) { err = "bad basis"; return GW_ERR_ARG; }
  if (kmesh[0] <= 0 || kmesh[1] <= 0 || kmesh[2] <= 0) { err = "bad k-mesh"; return GW_ERR_ARG; }
  if (grid->n_tau < 2 || !grid->tau || grid->beta <= 0) { err = "bad tau grid"; return GW_ERR_ARG; }
  if (grid->n_omega < grid->n_tau || grid->n_nu < grid->n_tau || !grid->omega_idx || !grid->nu_idx) {
    err = "need n_omega >= n_tau and n_nu >= n_tau";
    return GW_ERR_ARG;
  }
  if (grid->n_tau > kMaxTau) { err = "n_tau above the compiled limit"; return GW_ERR_UNSUPPORTED; }
  if (std::fabs(det3(cell->lattice)) < 1e-12) { err = "singular lattice"; return GW_ERR_ARG; }

  std::memcpy(hp.lat, cell->lattice, sizeof(hp.lat));
  hp.n_atoms = cell->n_atoms;
  hp.frac.assign(cell->frac, cell->frac + 3 * cell->n_atoms);
  hp.species.assign(cell->species, cell->species + cell->n_atoms);
  hp.n_species = basis->n_species;
  hp.n_orb.assign(basis->n_orb, basis->n_orb + basis->n_species);
  hp.n_prod.assign(basis->n_prod, basis->n_prod + basis->n_species);
  for (int s = 0; s < hp.n_species; ++s) {
    if (hp.n_orb[s] < 1 || hp.n_prod[s] < 1 || !basis->C[s]) { err = "bad species"; return GW_ERR_ARG; }
    if (hp.n_orb[s] > kMaxOrb || hp.n_prod[s] > kMaxProd) { err = "species above the compiled limits"; return GW_ERR_UNSUPPORTED; }
    size_t n = (size_t)hp.n_prod[s] * hp.n_orb[s] * hp.n_orb[s];
    hp.C.emplace_back(basis->C[s], basis->C[s] + n);
  }
  for (int a = 0; a < hp.n_atoms; ++a)
    if (hp.species[a] < 0 || hp.species[a] >= hp.n_species) { err = "species index out of range"; return GW_ERR_ARG; }
  for (int i = 0; i < 3; ++i) hp.kmesh[i] = kmesh[i];
  hp.n_k = kmesh[0] * kmesh[1] * kmesh[2];
  hp.beta = grid->beta;
  hp.n_tau = grid->n_tau;
  hp.n_omega = grid->n_omega;
  hp.n_nu = grid->n_nu;
  hp.tau.assign(grid->tau, grid->tau + grid->n_tau);
  hp.omega_idx.assign(grid->omega_idx, grid->omega_idx + grid->n_omega);
  hp.nu_idx.assign(grid->nu_idx, grid->nu_idx + grid->n_nu);
  hp.cutoff = cutoff;
  hp.spin = opt ? opt->spin : 2;
  // reduced product basis beyond sphere B (Sec. 2, Fig. 2)
  hp.r_b = (opt && basis->n_prod_far) ? opt->r_b : 0.0;
  hp.n_prod_far = hp.n_prod;
  hp.n_prod_near = hp.n_prod;
  if (hp.r_b > 0)
    for (int s = 0; s < hp.n_species; ++s) {
      const int f = basis->n_prod_far[s];
      if (f < 1 || f > hp.n_prod[s]) { err = "n_prod_far must be in [1, n_prod]"; return GW_ERR_ARG; }
      hp.n_prod_far[s] = f;
      if (basis->n_prod_near) {
        const int nr = basis->n_prod_near[s];
        if (nr < f || nr > hp.n_prod[s]) { err = "n_prod_near must be in [n_prod_far, n_prod]"; return GW_ERR_ARG; }
        hp.n_prod_near[s] = nr;
      }
    }
  if (hp.spin != 1 && hp.spin != 2) { err = "spin must be 1 or 2"; return GW_ERR_ARG; }

  // tau grid: ascending, ends at 0 and beta, mirror symmetric
  const int N = hp.n_tau;
  if (hp.tau[0] != 0.0 || std::fabs(hp.tau[N - 1] - hp.beta) > 1e-12 * hp.beta) { err = "tau must run from 0 to beta"; return GW_ERR_ARG; }
  for (int i = 1; i < N; ++i)
    if (!(hp.tau[i] > hp.tau[i - 1])) { err = "tau must be ascending"; return GW_ERR_ARG; }
  for (int i = 0; i < N; ++i)
    if (std::fabs(hp.beta - hp.tau[i] - hp.tau[N - 1 - i]) > 1e-12 * hp.beta) { err = "tau grid not mirror symmetric"; return GW_ERR_ARG; }

  // offsets
  hp.orb_off.assign(hp.n_atoms + 1, 0);
  hp.pb_off.assign(hp.n_atoms + 1, 0);
  for (int a = 0; a < hp.n_atoms; ++a) {
    hp.orb_off[a + 1] = hp.orb_off[a] + hp.n_orb[hp.species[a]];
    hp.pb_off[a + 1] = hp.pb_off[a] + hp.n_prod[hp.species[a]];
  }

  // k-mesh rule (Sec. 2, Fig. 1)
  if (cutoff > 0) {
    for (int i = 0; i < 3; ++i)
      hp.kmesh_required[i] = (int)std::ceil(2.0 * cutoff / plane_spacing(hp.lat, i) - 1e-12) + 1;
    if (opt && opt->strict_kmesh)
      for (int i = 0; i < 3; ++i)
        if (hp.kmesh[i] < hp.kmesh_required[i]) {
          std::ostringstream os;
          os << "k-mesh below the rule along axis " << i << ": " << hp.kmesh[i] << " < " << hp.kmesh_required[i];
          err = os.str();
          return GW_ERR_KMESH_ALIAS;
        }
  }

  // pair list: minimum image per class, ties to the lexicographically smallest R
  const double* A = hp.lat;
  std::vector<double> dist2;  // squared minimum-image distance of each kept entry
  hp.entries.clear();
  hp.pair_start.assign((size_t)hp.n_atoms * hp.n_atoms + 1, 0);
  for (int a = 0; a < hp.n_atoms; ++a) {
    for (int b = 0; b < hp.n_atoms; ++b) {
      hp.pair_start[(size_t)a * hp.n_atoms + b] = hp.n_entries();
      double d0[3];
      for (int j = 0; j < 3; ++j) d0[j] = hp.frac[3 * b + j] - hp.frac[3 * a + j];
      for (int c1 = 0; c1 < kmesh[0]; ++c1)
        for (int c2 = 0; c2 < kmesh[1]; ++c2)
          for (int c3 = 0; c3 < kmesh[2]; ++c3) {
            double best = 1e300;
            long long bR[3] = {0, 0, 0};
            for (int m1 = -2; m1 <= 2; ++m1)
              for (int m2 = -2; m2 <= 2; ++m2)
                for (int m3 = -2; m3 <= 2; ++m3) {
                  long long R[3] = {c1 + (long long)kmesh[0] * m1, c2 + (long long)kmesh[1] * m2,
                                    c3 + (long long)kmesh[2] * m3};
                  double f[3] = {R[0] + d0[0], R[1] + d0[1], R[2] + d0[2]};
                  double x[3];
                  for (int j = 0; j < 3; ++j) x[j] = f[0] * A[j] + f[1] * A[3 + j] + f[2] * A[6 + j];
                  double d2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                  bool better = d2 < best - 1e-9;
                  bool tie = std::fabs(d2 - best) <= 1e-9 &&
                             std::lexicographical_compare(R, R + 3, bR, bR + 3);
                  if (better || tie) {
                    best = d2;
                    bR[0] = R[0]; bR[1] = R[1]; bR[2] = R[2];
                  }
                }
            if (cutoff <= 0 || std::sqrt(best) <= cutoff) {
              int64_t row[8] = {a, b, c1, c2, c3, bR[0], bR[1], bR[2]};
              hp.entries.insert(hp.entries.end(), row, row + 8);
              dist2.push_back(best);
            }
          }
    }
  }
  hp.pair_start[(size_t)hp.n_atoms * hp.n_atoms] = hp.n_entries();
  const int E = hp.n_entries();
  if (E == 0) { err = "no pair entry inside the cutoff"; return GW_ERR_ARG; }

  // product functions per entry at its level (Sec. 2, Fig. 2): every function when both
  // arguments are in one sphere (A), the first n_prod_near within sphere B, the first
  // n_prod_far beyond it
  hp.Ka_e.assign(E, 0);
  hp.Kb_e.assign(E, 0);
  hp.tier_e.assign(E, 0);
  hp.n_far = hp.n_near = 0;
  for (int e = 0; e < E; ++e) {
    const int a = (int)hp.entries[8 * e], b = (int)hp.entries[8 * e + 1];
    const int sa = hp.species[a], sb = hp.species[b];
    int tier = 1;
    if (a == b && dist2[e] <= 1e-9) tier = 0;
    else if (hp.r_b > 0 && dist2[e] > hp.r_b * hp.r_b + 1e-9) tier = 2;
    const std::vector<int>& n = tier == 0 ? hp.n_prod : tier == 1 ? hp.n_prod_near : hp.n_prod_far;
    hp.Ka_e[e] = n[sa];
    hp.Kb_e[e] = n[sb];
    hp.tier_e[e] = tier;
    hp.n_far += tier == 2 ? 1 : 0;
    hp.n_near += (tier == 1 && (n[sa] < hp.n_prod[sa] || n[sb] < hp.n_prod[sb])) ? 1 : 0;
  }

  // block offsets
  hp.off_orb.assign(E + 1, 0);
  hp.off_pb.assign(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    int sa = hp.species[hp.entries[8 * e]], sb = hp.species[hp.entries[8 * e + 1]];
    hp.off_orb[e + 1] = hp.off_orb[e] + (int64_t)hp.n_orb[sa] * hp.n_orb[sb];
    hp.off_pb[e + 1] = hp.off_pb[e] + (int64_t)hp.Ka_e[e] * hp.Kb_e[e];
  }

  // mirror entry (b, a, -R mod N)
  hp.mirror.assign(E, -1);
  for (int e = 0; e < E; ++e) {
    int a = (int)hp.entries[8 * e], b = (int)hp.entries[8 * e + 1];
    int mc[3];
    for (int j = 0; j < 3; ++j) mc[j] = (int)((kmesh[j] - hp.entries[8 * e + 2 + j]) % kmesh[j]);
    for (int f = hp.pair_start[(size_t)b * hp.n_atoms + a]; f < hp.pair_start[(size_t)b * hp.n_atoms + a + 1]; ++f)
      if (hp.entries[8 * f + 2] == mc[0] && hp.entries[8 * f + 3] == mc[1] && hp.entries[8 * f + 4] == mc[2]) hp.mirror[e] = f;
  }

  // phases e^{+i k.R} = exp(2 pi i sum_j m_j c_j / N_j), reduced exactly in integers
  const long long L = (long long)kmesh[0] * kmesh[1] * kmesh[2];
  hp.phase.assign((size_t)2 * E * hp.n_k, 0.0);
  // when every phase is a quarter turn (4 r = 0 mod L: Gamma-centred meshes of 1, 2 or 4
  // points per axis) it is i^code exactly, and the lattice sums need no multiplications
  hp.phase_code.assign((size_t)E * hp.n_k, 0);
  bool quarter = true;
  for (int e = 0; e < E; ++e) {
    int k = 0;
    for (int m1 = 0; m1 < kmesh[0]; ++m1)
      for (int m2 = 0; m2 < kmesh[1]; ++m2)
        for (int m3 = 0; m3 < kmesh[2]; ++m3, ++k) {
          long long r = ((m1 * hp.entries[8 * e + 2]) % kmesh[0]) * (L / kmesh[0]) +
                        ((m2 * hp.entries[8 * e + 3]) % kmesh[1]) * (L / kmesh[1]) +
                        ((m3 * hp.entries[8 * e + 4]) % kmesh[2]) * (L / kmesh[2]);
          r %= L;
          long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)r / (long double)L;
          hp.phase[2 * ((size_t)e * hp.n_k + k)] = (double)std::cos(th);
          hp.phase[2 * ((size_t)e * hp.n_k + k) + 1] = (double)std::sin(th);
          if ((4 * r) % L == 0) hp.phase_code[(size_t)e * hp.n_k + k] = (signed char)(4 * r / L);
          else quarter = false;
        }
  }
  if (!quarter) hp.phase_code.clear();

  // packed C and its (L, L'') symmetry
  hp.c_off.assign(hp.n_species + 1, 0);
  for (int s = 0; s < hp.n_species; ++s) hp.c_off[s + 1] = hp.c_off[s] + (int)hp.C[s].size();
  hp.C_packed.clear();
  hp.c_symmetric = 1;
  for (int s = 0; s < hp.n_species; ++s) {
    hp.C_packed.insert(hp.C_packed.end(), hp.C[s].begin(), hp.C[s].end());
    int n = hp.n_orb[s];
    for (int K = 0; K < hp.n_prod[s]; ++K)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          if (hp.C[s][((size_t)K * n + i) * n + j] != hp.C[s][((size_t)K * n + j) * n + i]) hp.c_symmetric = 0;
  }

  // transform matrices
  std::vector<cd> Tf = fourier_matrix(hp.beta, hp.tau, hp.omega_idx, true, err);
  if (Tf.empty()) return GW_ERR_ARG;
  std::vector<cd> Tb = fourier_matrix(hp.beta, hp.tau, hp.nu_idx, false, err);
  if (Tb.empty()) return GW_ERR_ARG;
  std::vector<cd> Uf, Ub;
  if (!pinv_qr(hp.n_omega, N, Tf, Uf) || !pinv_qr(hp.n_nu, N, Tb, Ub)) {
    err = "Matsubara sampling does not determine the tau polynomial (rank deficient)";
    return GW_ERR_ARG;
  }
  hp.cond_f = sigma_max(hp.n_omega, N, Tf) * sigma_max(N, hp.n_omega, Uf);
  hp.cond_b = sigma_max(hp.n_nu, N, Tb) * sigma_max(N, hp.n_nu, Ub);
  hp.Tf_fwd = to_interleaved(Tf);
  hp.Tf_inv = to_interleaved(Uf);
  hp.Tb_fwd = to_interleaved(Tb);
  hp.Tb_inv = to_interleaved(Ub);
  // F(tau_{N-1-i}) = conj(F(tau_i)) pairs node i with its mirror: T F + T' conj(F) has the
  // real part (Re T + Re T') Re F + (Im T' - Im T) Im F; the self-mirrored middle node of
  // an odd grid keeps (Re T, -Im T).  The imaginary part vanishes for bosonic frequencies.
  const int nh = (N + 1) / 2;
  hp.Tb_mirror.assign((size_t)2 * hp.n_nu * nh, 0.0);
  for (int m = 0; m < hp.n_nu; ++m)
    for (int i = 0; i < nh; ++i) {
      const cd t = Tb[(size_t)m * N + i], tm = Tb[(size_t)m * N + (N - 1 - i)];
      const bool mid = (N - 1 - i) == i;
      hp.Tb_mirror[2 * ((size_t)m * nh + i)] = mid ? t.real() : t.real() + tm.real();
      hp.Tb_mirror[2 * ((size_t)m * nh + i) + 1] = mid ? -t.imag() : tm.imag() - t.imag();
    }
  return GW_OK;
}

std::vector<DevEntry> make_dev_entries(const HostPlan& hp) {
  const int E = hp.n_entries();
  std::vector<DevEntry> out(E);
  for (int e = 0; e < E; ++e) {
    DevEntry d{};
    d.a = (int)hp.entries[8 * e];
    d.b = (int)hp.entries[8 * e + 1];
    int sa = hp.species[d.a], sb = hp.species[d.b];
    d.na = hp.n_orb[sa];
    d.nb = hp.n_orb[sb];
    d.Ka = hp.Ka_e[e];
    d.Kb = hp.Kb_e[e];
    d.oa = hp.orb_off[d.a];
    d.ob = hp.orb_off[d.b];
    d.pa = hp.pb_off[d.a];
    d.pb = hp.pb_off[d.b];
    d.ca = hp.c_off[sa];
    d.cb = hp.c_off[sb];
    d.off_orb = hp.off_orb[e];
    d.off_pb = hp.off_pb[e];
    d.mirror = hp.mirror[e];
    d.tier = hp.tier_e[e];
    out[e] = d;
  }
  return out;
}

}  // namespace gw
