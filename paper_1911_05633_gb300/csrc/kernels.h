// Kernel argument blocks and kernel declarations (device code only).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gw {

// The library's tables go up with cudaMemcpy from pageable host memory (and flags are
// cleared with cudaMemset) on the legacy default stream.  Such a copy can return before it
// has landed, and the callers' streams (created non-blocking) are not ordered after the
// legacy stream: wait for it before any kernel on another stream may read what was
// uploaded.  Called once at the end of each setup that uploads.
inline cudaError_t uploads_landed() { return cudaStreamSynchronize(cudaStreamLegacy); }


struct GatherArgs {
  const DevEntry* ent;
  const int* pair_start;   // [n_atoms^2 + 1] entry range of each ordered atom pair
  const int* col_atom;     // [N] atom of each dense row / column
  int n_atoms;
  const double2* phase;    // [E][N_k] e^{+i k.R}
  const signed char* pcode;  // optional [E][N_k]: e^{+i k.R} = i^pcode exactly (quarter turns)
  int n_k;                 // mesh size (phase row length)
  const int* k_list;       // optional: input k index kk -> mesh k (n_k_in entries)
  const double* k_weight;  // optional: weight per input k index
  int n_k_in;              // number of input k indices summed over
  int real_only;           // keep the real part of the result
  const double2* F_k;      // dense input
  long long k_stride, s_stride;
  int ld;
  int pb;                  // 1: product-basis blocks, 0: orbital blocks
  const int* row_off;      // [n_atoms + 1] orbital or product offsets (the full pair block)
  const double2* F_sub;    // optional dense input subtracted from F_k
  long long sub_k_stride, sub_s_stride;
  double2* F_R;            // entry layout output
  int out_n_slices, out_slice0;
  double scale;
};

struct ScatterArgs {
  const DevEntry* ent;
  const int* pair_start;   // [n_atoms^2 + 1]
  const int* col_atom;     // [N] atom of each dense row / column
  const int* row_off;      // [n_atoms + 1] orbital or product offsets
  int n_atoms;
  const double2* phase;
  const signed char* pcode;  // optional [E][N_k]: e^{+i k.R} = i^pcode exactly (quarter turns)
  int n_k;                 // mesh size (phase row length)
  const int* k_list;       // optional: output k index kk -> mesh k (n_k_out entries)
  int n_k_out;
  const double2* base;     // optional dense [n_k_out][N][N] added to the result
  double coef;             // result = base + coef * sum
  int real_in;             // imaginary parts of F_R are zero: not read
  const double2* F_R;      // entry layout input
  int in_n_slices, in_slice0;
  int pb;
  double2* F_k;            // dense output
  long long k_stride, s_stride;
  int ld;
};

struct TransformArgs {
  const DevEntry* ent;
  const double2* T;        // [n_out][n_in]
  int n_in, n_out;
  int pb;
  const double2* in;
  double2* out;
  // 0: general complex; 1: mirror-paired input, n_in = the first ceil(N/2) nodes of an
  // in-stride of in_stride slices, T = (a, b) coefficients, real output; 2: real input
  int mode;
  int in_stride;
  int m_begin;             // first output slice written (the ones before keep their contents)
};

struct ContractArgs {
  const DevEntry* ent;
  const double* C;         // packed per-species coefficients
  const double2* G;        // orbital entry layout
  const double2* W;        // product entry layout (Sigma only)
  double2* out;
  int n_tau;
  int spin;
  int mirror_tau;          // P: write the mirrored node as the conjugate
  int g_n_slices, g_slice; // Sigma: slices of G and a fixed slice (or -1: = blockIdx.y)
  int w_n_slices;
  int out_n_slices;
  double sign;
  // Sigma with stage A precomputed (B[e][sl][K][j] at Bpre + offB[e] tau_c + (sl K_a + K) n_b^2 + j):
  // block y = sl is slice s0 + sl of G and of the output
  const double2* Bpre;
  const long long* offB;
  int tau_c, s0;
  // P with stage 3 on the tensor cores: block y = sl is computed node s0 + sl; stage 2 (Y)
  // goes to Ypre + offB[e] tau_c + (sl K_a + K) n_b^2 + j instead of stage 3
  double2* Ypre;
};

void launch_gather_kernel(dim3 grid, cudaStream_t st, const GatherArgs& g);
__global__ void k_scatter_R_to_k(ScatterArgs g);
__global__ void k_transform(TransformArgs g);
__global__ void k_polarizability_fp64(ContractArgs g);
__global__ void k_self_energy_fp64(ContractArgs g);
// In-place Gauss-Jordan inverse of a batch of N x N complex matrices (partial pivoting).
__global__ void k_gj_inverse(double2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                             int* status);
constexpr int kGJB = 16;  // panel width of the blocked Gauss-Jordan inverse
__global__ void k_gj_inverse_blocked(double2* __restrict__ A, int* __restrict__ perm, int N, long long mat_stride,
                                     int* status);
// dst[b] = src[map[b]] for dense N x N matrices (used to stage v(q) before inversion).
__global__ void k_copy_mats(const double2* __restrict__ src, const int* __restrict__ map, double2* __restrict__ dst,
                            long long NN);
// W~(R, -nu_j) = W~(mirror(R), nu_{mirror j})^T for the negative frequencies (real blocks).
__global__ void k_mirror_nu(const DevEntry* __restrict__ ent, const int* __restrict__ nu_mirror, int n_neg, int n_nu,
                            double2* __restrict__ W);

constexpr int kKCHost = 16;  // must match kKC in kernels_fp64.cu

}  // namespace gw
