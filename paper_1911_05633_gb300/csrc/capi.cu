// The C ABI declared in include/gw.h: plan lifetime, queries and the entry
// points of the sweep.  Host orchestration only; the arithmetic runs in the
// kernels of kernels_fp64.cu and kernels_mixed.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "smem_limit.h"
#include "mixed.h"
#include "contract.h"
#include "wtc.h"
#include "oz.h"
#include "ktimer.h"
#include "dyson.h"

struct gw_plan_s {
  gw::HostPlan h;
  bool host_only = true;
  int device = 0;
  gw::DevEntry* d_ent = nullptr;
  int* d_pair_start = nullptr;  // [n_atoms^2 + 1]
  int* d_pair_first = nullptr;  // [n_active + 1]
  int n_active = 0;
  int* d_orb_off = nullptr;
  int* d_pb_off = nullptr;
  int* d_orb_atom = nullptr;  // [N_orb] atom of each orbital row / column
  int* d_pb_atom = nullptr;   // [N_PB] atom of each product-basis row / column
  double2* d_phase = nullptr;
  signed char* d_pcode = nullptr;  // quarter-turn codes of the phases, when every phase is one
  double* d_C = nullptr;
  double2* d_Tf_fwd = nullptr;
  double2* d_Tf_inv = nullptr;
  double2* d_Tb_fwd = nullptr;
  double2* d_Tb_mirror = nullptr;  // [n_nu][ceil(N_tau/2)] mirror-pair coefficients
  double2* d_Tb_inv = nullptr;
  // W solve: momenta and frequencies solved, and scratch
  bool w_sym = false;
  int n_qh = 0;                 // momenta solved per frequency
  int* d_qh = nullptr;          // [n_qh] mesh index of each solved momentum
  double* d_qw = nullptr;       // [n_qh] weight (2 for a (q, -q) pair, else 1); symmetric mode only
  int nu_start = 0;             // first solved bosonic slot (the nu >= 0 ones in symmetric mode)
  int n_neg = 0;                // negative-frequency slots filled by symmetry
  int* d_numirror = nullptr;    // [n_neg] slot of -nu for each negative slot
  double2* d_wsV = nullptr;     // [n_qh][N][N] v(q)^{-1}
  double2* d_wsA = nullptr;     // [nu_chunk][n_qh][N][N]
  int* d_perm = nullptr;        // [nu_chunk * n_qh][N]
  int* d_status = nullptr;
  int nu_chunk = 0;
  size_t ws_bytes = 0;
  size_t ws_cap = 0;            // cap on the W-solve scratch
  // scratch left for the first call that needs it (gw_options.defer_scratch)
  bool w_pending = false, oz_pending = false, ozp_pending = false;
  size_t smem_P = 0, smem_S = 0, smem_T = 0, smem_GJ = 0;
  bool gj_blocked = false;
  // tensor-core inverse (FP32 Gauss-Jordan + sliced FP64-accurate residual)
  bool w_tensor = false;
  size_t smem_GJ32 = 0;
  float2* t_X32 = nullptr;
  float2* t_lo = nullptr;
  float2* t_R = nullptr;
  uint16_t* t_PX = nullptr;
  uint16_t* t_Asl = nullptr;
  uint16_t* t_Xsl = nullptr;
  int* t_eA = nullptr;
  int* t_eX = nullptr;
  // block Gauss-Jordan for N_PB beyond the tensor-core inverse (pivot blocks of w_bs,
  // each inverted by the tensor-core inverse; the t_* buffers above sized for them)
  bool w_block = false;
  int w_bs = 0;
  double2* b_D = nullptr;
  double2* b_Rp = nullptr;
  uint16_t* b_Asl = nullptr;
  uint16_t* b_Bsl = nullptr;
  int* b_eA = nullptr;
  int* b_eB = nullptr;
  gw::MixedPlan mixed;
  // mixed-precision contractions as persistent tensor-core kernels over a unit queue
  gw::CTables ct;
  gw::CConfig cfgP, cfgS;
  bool contract_p = false, contract_s = false;
  gw::CUnit* d_unitsP = nullptr;
  gw::CUnit* d_unitsS = nullptr;
  gw::CUnit* d_unitsX = nullptr;  // the exchange term: one node per entry
  int n_unitsP = 0, n_unitsS = 0, n_unitsX = 0;
  int* d_counter = nullptr;
  bool sigma_tensor = false;  // FP64 Sigma stage A by tensor-core digit products
  gw::OzSigma oz;
  gw::OzTransform ozt;  // FP64-accurate structured transforms on the tensor cores
  gw::OzPol ozp;        // FP64-accurate stage 3 of P on the tensor cores
  gw::KernelTimer timer;  // optional per-kernel event timing (gw_timing_*)
  gw::DysonPlan dyson;    // Eq. G_1 scratch, allocated by the first Dyson call
};

namespace gw {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

KernelTimer*& current_timer() {
  static thread_local KernelTimer* t = nullptr;
  return t;
}

}  // namespace gw

namespace {

using gw::set_last_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

gw_status cuda_fail(cudaError_t e, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return GW_ERR_CUDA;
}

#define GW_CUDA(call)                                         \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);       \
  } while (0)

template <typename T>
gw_status upload(T** dst, const void* src, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) {
    set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;
  }
  if (src) GW_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return GW_OK;
}

void free_device(gw_plan_s* p) {
  void* ptrs[] = {p->d_ent, p->d_pair_start, p->d_pair_first, p->d_orb_off, p->d_pb_off, p->d_orb_atom,
                  p->d_pb_atom, p->d_phase, p->d_pcode,
                  p->d_C, p->d_Tf_fwd, p->d_Tf_inv, p->d_Tb_fwd, p->d_Tb_mirror, p->d_Tb_inv, p->d_qh, p->d_qw,
                  p->d_numirror, p->d_wsV, p->d_wsA, p->d_perm, p->d_status, p->t_X32, p->t_lo, p->t_R, p->t_PX, p->t_Asl,
                  p->t_Xsl, p->t_eA, p->t_eX, p->d_unitsP, p->d_unitsS, p->d_unitsX, p->d_counter,
                  p->b_D, p->b_Rp, p->b_Asl, p->b_Bsl, p->b_eA, p->b_eB};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  gw::mixed_free(p->mixed);
  gw::ctables_free(p->ct);
  gw::oz_sigma_free(p->oz);
  gw::oz_transform_free(p->ozt);
  gw::oz_pol_free(p->ozp);
  gw::dyson_free(p->dyson);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

gw_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return GW_OK;
}

gw_status need_device(gw_plan_t p) {
  if (!p) { set_last_error("null plan"); return GW_ERR_ARG; }
  if (p->host_only) { set_last_error("plan was built with host_only"); return GW_ERR_NO_DEVICE; }
  return GW_OK;
}

// Dense k-space leading dimension and entry-layout kind
int dense_n(const gw_plan_s* p, gw_block kind) {
  return kind == GW_BLOCK_PB ? p->h.n_pb_total() : p->h.n_orb_total();
}

// Blocks per (atom, slice) row band of the gather and scatter: enough for about four
// blocks per SM, and no more than one per 256 elements of the widest band.
unsigned band_splits(const gw_plan_s* p, gw_block kind, int n_slices) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const std::vector<int>& off = kind == GW_BLOCK_PB ? p->h.pb_off : p->h.orb_off;
  int band = 0;
  for (int a = 0; a < p->h.n_atoms; ++a) band = std::max(band, off[a + 1] - off[a]);
  const long long el = (long long)band * off[p->h.n_atoms];
  const long long base = (long long)p->h.n_atoms * std::max(1, n_slices);
  const long long want = (4LL * std::max(1, sms) + base - 1) / base;
  return (unsigned)std::max<long long>(1, std::min<long long>({want, (el + 255) / 256, 65535}));
}

gw_status launch_gather(gw_plan_s* p, gw_block kind, int n_slices, const double2* F_k, long long k_stride,
                        long long s_stride, const double2* F_sub, long long sub_k_stride, long long sub_s_stride,
                        double2* F_R, int out_n_slices, int out_slice0, double scale, cudaStream_t st,
                        const int* k_list = nullptr, const double* k_weight = nullptr, int n_k_in = -1,
                        int real_only = 0) {
  gw::GatherArgs g{};
  g.ent = p->d_ent;
  g.pair_start = p->d_pair_start;
  g.col_atom = kind == GW_BLOCK_PB ? p->d_pb_atom : p->d_orb_atom;
  g.n_atoms = p->h.n_atoms;
  g.phase = p->d_phase;
  g.pcode = p->d_pcode;
  g.n_k = p->h.n_k;
  g.k_list = k_list;
  g.k_weight = k_weight;
  g.n_k_in = n_k_in < 0 ? p->h.n_k : n_k_in;
  g.real_only = real_only;
  g.F_k = F_k;
  g.k_stride = k_stride;
  g.s_stride = s_stride;
  g.ld = dense_n(p, kind);
  g.pb = kind == GW_BLOCK_PB;
  g.row_off = kind == GW_BLOCK_PB ? p->d_pb_off : p->d_orb_off;
  g.F_sub = F_sub;
  g.sub_k_stride = sub_k_stride;
  g.sub_s_stride = sub_s_stride;
  g.F_R = F_R;
  g.out_n_slices = out_n_slices;
  g.out_slice0 = out_slice0;
  g.scale = scale;
  dim3 grid(p->h.n_atoms, n_slices, band_splits(p, kind, n_slices));
  {
    gw::TimedLaunch tl_("k_gather_k_to_R", st);
    gw::launch_gather_kernel(grid, st, g);
  }
  return check_launch("k_gather_k_to_R");
}

gw_status launch_scatter(gw_plan_s* p, gw_block kind, int n_slices, const double2* F_R, int in_n_slices,
                         int in_slice0, double2* F_k, long long k_stride, long long s_stride, cudaStream_t st,
                         const int* k_list = nullptr, int n_k_out = -1, const double2* base = nullptr,
                         double coef = 1.0, bool real_in = false) {
  gw::ScatterArgs g{};
  g.real_in = real_in ? 1 : 0;
  g.ent = p->d_ent;
  g.pair_start = p->d_pair_start;
  g.col_atom = kind == GW_BLOCK_PB ? p->d_pb_atom : p->d_orb_atom;
  g.row_off = kind == GW_BLOCK_PB ? p->d_pb_off : p->d_orb_off;
  g.n_atoms = p->h.n_atoms;
  g.phase = p->d_phase;
  g.pcode = p->d_pcode;
  g.n_k = p->h.n_k;
  g.k_list = k_list;
  g.n_k_out = n_k_out < 0 ? p->h.n_k : n_k_out;
  g.base = base;
  g.coef = coef;
  g.F_R = F_R;
  g.in_n_slices = in_n_slices;
  g.in_slice0 = in_slice0;
  g.pb = kind == GW_BLOCK_PB;
  g.F_k = F_k;
  g.k_stride = k_stride;
  g.s_stride = s_stride;
  g.ld = dense_n(p, kind);
  dim3 grid(p->h.n_atoms, n_slices, band_splits(p, kind, n_slices));
  {
    gw::TimedLaunch tl_("k_scatter_R_to_k", st);
    gw::k_scatter_R_to_k<<<grid, 256, 0, st>>>(g);
  }
  return check_launch("k_scatter_R_to_k");
}

// Batched in-place inverse of `batch` dense N x N matrices (perm and status from the plan).
gw_status launch_gj(gw_plan_s* p, double2* mats, int batch, long long N, cudaStream_t st) {
  if (p->gj_blocked) {
    gw::TimedLaunch tl_("k_gj_inverse_blocked", st);
    gw::k_gj_inverse_blocked<<<batch, 512, p->smem_GJ, st>>>(mats, p->d_perm, (int)N, N * N, p->d_status);
  } else {
    gw::TimedLaunch tl_("k_gj_inverse", st);
    gw::k_gj_inverse<<<batch, 512, p->smem_GJ, st>>>(mats, p->d_perm, (int)N, N * N, p->d_status);
  }
  return check_launch("k_gj_inverse");
}

// In place: mats[b] (FP64, N x N) -> its inverse by the tensor-core refinement (kernels_wtc.cu).
gw_status launch_tensor_inverse(gw_plan_s* p, double2* mats, int batch, long long N, cudaStream_t st) {
  gw::WtcBuffers w{};  // by name: the buffers differ in size per element
  w.X32 = p->t_X32;
  w.lo = p->t_lo;
  w.R = p->t_R;
  w.Asl = p->t_Asl;
  w.Xsl = p->t_Xsl;
  w.PX = p->t_PX;
  w.eA = p->t_eA;
  w.eX = p->t_eX;
  w.status = p->d_status;
  gw::wtc_inverse(w, mats, batch, (int)N, p->smem_GJ32, st);
  return check_launch("tensor-core inverse");
}

gw_status launch_block_inverse(gw_plan_s* p, double2* mats, int batch, long long N, cudaStream_t st) {
  gw::WblkBuffers w{};
  w.D = p->b_D;
  w.Rp = p->b_Rp;
  w.Asl = p->b_Asl;
  w.Bsl = p->b_Bsl;
  w.eA = p->b_eA;
  w.eB = p->b_eB;
  w.inner.X32 = p->t_X32;
  w.inner.lo = p->t_lo;
  w.inner.R = p->t_R;
  w.inner.Asl = p->t_Asl;
  w.inner.Xsl = p->t_Xsl;
  w.inner.PX = p->t_PX;
  w.inner.eA = p->t_eA;
  w.inner.eX = p->t_eX;
  w.inner.status = p->d_status;
  gw::wblk_inverse(w, mats, batch, (int)N, p->w_bs, p->smem_GJ32, st);
  return check_launch("block inverse");
}

size_t smem_polar(const gw::HostPlan& h) {
  size_t m = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      size_t na = h.n_orb[s], nb = h.n_orb[t];
      m = std::max(m, (2 * na * nb + gw::kKCHost * na * nb + gw::kKCHost * nb * nb) * sizeof(double2));
    }
  return m;
}

size_t smem_sigma(const gw::HostPlan& h) {
  size_t m = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t) {
      size_t na = h.n_orb[s], nb = h.n_orb[t];
      m = std::max(m, (na * nb + gw::kKCHost * nb * nb + gw::kKCHost * na * nb) * sizeof(double2));
    }
  return m;
}

}  // namespace

// The W-solve scratch: v(q)^-1 of the solved momenta and a chunk of bosonic frequencies
// sized to the cap, plus the tensor-core inverse's planes.
static gw_status alloc_w_scratch(gw_plan_s* p) {
  const gw::HostPlan& h = p->h;
  const size_t npb = (size_t)h.n_pb_total();
  const size_t mat = npb * npb * sizeof(double2);
  // bytes per inverted matrix: FP64 matrix, pivots, and (tensor path) the FP32 inverse,
  // its correction and the residual, the BF16 digit planes of both operands, the term
  // planes of X0 and the scale exponents
  // the tensor-core inverse's scratch per inverted matrix of order ni (the matrix itself,
  // or the pivot block of the block Gauss-Jordan)
  const size_t ni = p->w_block ? (size_t)p->w_bs : npb;
  const size_t tc_per = ni * ni * (3 * sizeof(float2) + 2 * (gw::kWSA + gw::kWSX1) * 2 + 6 * 2) + 2 * ni * sizeof(int);
  // block Gauss-Jordan: the pivot block, the row panel, the digits of a column and a row
  // panel (2 kWSA, 2 kWSX1 BF16 planes per element) and 2 npb exponents
  const size_t bs = (size_t)p->w_bs;
  const size_t blk_per = p->w_block ? bs * bs * sizeof(double2) + bs * npb * sizeof(double2) +
                                          npb * bs * 2 * (gw::kWSA + gw::kWSX1) * 2 + 2 * npb * sizeof(int)
                                    : 0;
  const size_t per_mat = mat + npb * sizeof(int) + (p->w_tensor || p->w_block ? tc_per : 0) + blk_per;
  const size_t per_nu = (size_t)p->n_qh * per_mat;
  const size_t cap = p->ws_cap;
  const int n_work_nu = h.n_nu - p->nu_start;
  const size_t base_bytes = (size_t)p->n_qh * mat;
  const int nch = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_work_nu, cap > base_bytes ? (cap - base_bytes) / per_nu : 1));
  p->nu_chunk = nch;
  auto up = [&](void** dst, size_t bytes) -> gw_status {
    if (cudaMalloc(dst, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("device allocation for the W-solve scratch failed");
      return GW_ERR_OOM;
    }
    return GW_OK;
  };
  gw_status st;
  if ((st = up((void**)&p->d_wsV, (size_t)p->n_qh * mat)) != GW_OK) return st;
  if ((st = up((void**)&p->d_wsA, (size_t)nch * p->n_qh * mat)) != GW_OK) return st;
  if ((st = up((void**)&p->d_perm, (size_t)nch * p->n_qh * npb * sizeof(int))) != GW_OK) return st;
  p->ws_bytes = (size_t)p->n_qh * mat + (size_t)nch * per_nu;
  if (p->w_tensor || p->w_block) {
    const size_t nm = (size_t)nch * p->n_qh;
    if ((st = up((void**)&p->t_X32, nm * ni * ni * sizeof(float2))) != GW_OK) return st;
    if ((st = up((void**)&p->t_lo, nm * ni * ni * sizeof(float2))) != GW_OK) return st;
    if ((st = up((void**)&p->t_R, nm * ni * ni * sizeof(float2))) != GW_OK) return st;
    if ((st = up((void**)&p->t_PX, nm * ni * ni * 6 * 2)) != GW_OK) return st;
    if ((st = up((void**)&p->t_Asl, nm * ni * ni * 2 * gw::kWSA * 2)) != GW_OK) return st;
    if ((st = up((void**)&p->t_Xsl, nm * ni * ni * 2 * gw::kWSX1 * 2)) != GW_OK) return st;
    if ((st = up((void**)&p->t_eA, nm * ni * sizeof(int))) != GW_OK) return st;
    if ((st = up((void**)&p->t_eX, nm * ni * sizeof(int))) != GW_OK) return st;
  }
  if (p->w_block) {
    const size_t nm = (size_t)nch * p->n_qh;
    if ((st = up((void**)&p->b_D, nm * bs * bs * sizeof(double2))) != GW_OK) return st;
    if ((st = up((void**)&p->b_Rp, nm * bs * npb * sizeof(double2))) != GW_OK) return st;
    if ((st = up((void**)&p->b_Asl, nm * npb * bs * 2 * gw::kWSA * 2)) != GW_OK) return st;
    if ((st = up((void**)&p->b_Bsl, nm * npb * bs * 2 * gw::kWSX1 * 2)) != GW_OK) return st;
    if ((st = up((void**)&p->b_eA, nm * npb * sizeof(int))) != GW_OK) return st;
    if ((st = up((void**)&p->b_eB, nm * npb * sizeof(int))) != GW_OK) return st;
  }
  p->w_pending = false;
  return GW_OK;
}

// The FP64 digit-GEMM scratch of the Sigma stage W~ C^b and of the P stage Y C^b.
static gw_status alloc_oz_sigma(gw_plan_s* p) {
  const gw_status st = gw::oz_sigma_init(p->oz, p->h, (size_t)4 << 30);
  p->oz_pending = false;
  if (st != GW_OK) return st;
  if (gw::uploads_landed() != cudaSuccess) return GW_ERR_CUDA;
  p->sigma_tensor = p->oz.ready;
  return GW_OK;
}
static gw_status alloc_oz_pol(gw_plan_s* p) {
  const gw_status st = gw::oz_pol_init(p->ozp, p->h, (size_t)4 << 30);
  p->ozp_pending = false;
  if (st == GW_OK && gw::uploads_landed() != cudaSuccess) return GW_ERR_CUDA;
  return st;
}

extern "C" {

const char* gw_status_string(gw_status s) {
  switch (s) {
    case GW_OK: return "ok";
    case GW_ERR_ARG: return "invalid argument";
    case GW_ERR_OOM: return "out of memory";
    case GW_ERR_CUDA: return "CUDA error";
    case GW_ERR_KMESH_ALIAS: return "k-mesh below the cutoff rule";
    case GW_ERR_NOT_HERMITIAN: return "input not Hermitian";
    case GW_ERR_SINGULAR: return "singular matrix in the W solve";
    case GW_ERR_TIMEOUT: return "device wait timed out";
    case GW_ERR_NAN: return "NaN detected";
    case GW_ERR_NO_DEVICE: return "plan has no device state";
    case GW_ERR_UNSUPPORTED: return "unsupported size or mode";
  }
  return "unknown status";
}

const char* gw_last_error(void) { return gw::g_last_error.c_str(); }

gw_status gw_plan_create(const gw_cell* cell, const gw_basis* basis, const int kmesh[3], const gw_grid* grid,
                         double cutoff, const gw_options* opt, gw_plan_t* out) {
  if (!out) { set_last_error("null output"); return GW_ERR_ARG; }
  *out = nullptr;
  gw_plan_s* p = new (std::nothrow) gw_plan_s();
  if (!p) return GW_ERR_OOM;
  std::string err;
  std::vector<int> qh, numirror;
  std::vector<double> qw;
  gw_status st = gw::build_host_plan(cell, basis, kmesh, grid, cutoff, opt, p->h, err);
  if (st != GW_OK) {
    set_last_error(err);
    delete p;
    return st;
  }
  p->host_only = opt ? (opt->host_only != 0) : false;
  const gw::HostPlan& hh = p->h;
  // W solve: which momenta and frequencies are solved, and the scratch
  {
    bool nu_sym = true;
    for (int j = 0; j < hh.n_nu; ++j) {
      bool found = false;
      for (int l = 0; l < hh.n_nu; ++l) found |= (hh.nu_idx[l] == -hh.nu_idx[j]);
      nu_sym &= found;
    }
    for (int j = 1; j < hh.n_nu; ++j) nu_sym &= (hh.nu_idx[j] > hh.nu_idx[j - 1]);
    p->w_sym = p->h.c_symmetric && nu_sym && !(opt && opt->no_symmetry);
  }
    for (int q = 0, q1 = 0; q1 < hh.kmesh[0]; ++q1)
    for (int q2 = 0; q2 < hh.kmesh[1]; ++q2)
      for (int q3 = 0; q3 < hh.kmesh[2]; ++q3, ++q) {
        const int m1 = (hh.kmesh[0] - q1) % hh.kmesh[0], m2 = (hh.kmesh[1] - q2) % hh.kmesh[1],
                  m3 = (hh.kmesh[2] - q3) % hh.kmesh[2];
        const int mq = (m1 * hh.kmesh[1] + m2) * hh.kmesh[2] + m3;
        if (!p->w_sym) { qh.push_back(q); qw.push_back(1.0); }
        else if (q <= mq) { qh.push_back(q); qw.push_back(q == mq ? 1.0 : 2.0); }
      }
  p->n_qh = (int)qh.size();
  if (p->w_sym) {
    int n_neg = 0;
    while (n_neg < hh.n_nu && hh.nu_idx[n_neg] < 0) ++n_neg;
    p->n_neg = n_neg;
    p->nu_start = n_neg;
    for (int j = 0; j < n_neg; ++j)
      for (int l = 0; l < hh.n_nu; ++l)
        if (hh.nu_idx[l] == -hh.nu_idx[j]) numirror.push_back(l);
  }
  {
    // tensor-core inverse: N a multiple of 128, at most 384 (the bound under which the
    // FP32 level accumulators of the residual are exact)
    const size_t n = (size_t)hh.n_pb_total();
    p->w_tensor = !(opt && opt->w_solver == 1) && n % 128 == 0 && n > 0 && n <= (size_t)gw::kWNmax;
    // beyond it: block Gauss-Jordan over pivot blocks that the tensor-core inverse takes
    p->w_bs = !(opt && opt->w_solver == 1) && !p->w_tensor ? gw::wblk_block_size((int)n) : 0;
    p->w_block = p->w_bs > 0;
    bool k_ok = true;  // the tensor-core Sigma stage sums levels 0-4 exactly for K_b <= 384
    for (int s = 0; s < hh.n_species; ++s) k_ok = k_ok && hh.n_prod[s] <= 16 * gw::kOzMaxKS;
    p->sigma_tensor = !(opt && opt->fp64_products == 1) && k_ok;
  }
  p->device = opt ? opt->device : 0;
  if (p->host_only) {
    *out = p;
    return GW_OK;
  }
  DeviceGuard guard(p->device);
  const gw::HostPlan& h = p->h;
  auto fail = [&](gw_status s) {
    free_device(p);
    delete p;
    return s;
  };
  std::vector<gw::DevEntry> de = gw::make_dev_entries(h);
  std::vector<int> pair_first;
  for (size_t q = 0; q + 1 < h.pair_start.size(); ++q)
    if (h.pair_start[q + 1] > h.pair_start[q]) pair_first.push_back(h.pair_start[q]);
  pair_first.push_back(h.n_entries());
  p->n_active = (int)pair_first.size() - 1;
  if ((st = upload(&p->d_ent, de.data(), de.size() * sizeof(gw::DevEntry))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_pair_start, h.pair_start.data(), h.pair_start.size() * sizeof(int))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_pair_first, pair_first.data(), pair_first.size() * sizeof(int))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_orb_off, h.orb_off.data(), h.orb_off.size() * sizeof(int))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_pb_off, h.pb_off.data(), h.pb_off.size() * sizeof(int))) != GW_OK) return fail(st);
  {
    std::vector<int> oa(h.n_orb_total()), pa(h.n_pb_total());
    for (int a = 0; a < h.n_atoms; ++a) {
      for (int i = h.orb_off[a]; i < h.orb_off[a + 1]; ++i) oa[i] = a;
      for (int i = h.pb_off[a]; i < h.pb_off[a + 1]; ++i) pa[i] = a;
    }
    if ((st = upload(&p->d_orb_atom, oa.data(), oa.size() * sizeof(int))) != GW_OK) return fail(st);
    if ((st = upload(&p->d_pb_atom, pa.data(), pa.size() * sizeof(int))) != GW_OK) return fail(st);
  }
  if ((st = upload(&p->d_phase, h.phase.data(), h.phase.size() * sizeof(double))) != GW_OK) return fail(st);
  if (!h.phase_code.empty() &&
      (st = upload(&p->d_pcode, h.phase_code.data(), h.phase_code.size())) != GW_OK)
    return fail(st);
  if ((st = upload(&p->d_C, h.C_packed.data(), h.C_packed.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_Tf_fwd, h.Tf_fwd.data(), h.Tf_fwd.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_Tf_inv, h.Tf_inv.data(), h.Tf_inv.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_Tb_fwd, h.Tb_fwd.data(), h.Tb_fwd.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_Tb_mirror, h.Tb_mirror.data(), h.Tb_mirror.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_Tb_inv, h.Tb_inv.data(), h.Tb_inv.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_status, nullptr, 16)) != GW_OK) return fail(st);
  if (cudaMemset(p->d_status, 0, 16) != cudaSuccess) return fail(GW_ERR_CUDA);

  // W-solve scratch
  const size_t npb = (size_t)h.n_pb_total();
  if ((st = upload(&p->d_qh, qh.data(), qh.size() * sizeof(int))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_qw, qw.data(), qw.size() * sizeof(double))) != GW_OK) return fail(st);
  if ((st = upload(&p->d_numirror, numirror.data(), numirror.size() * sizeof(int))) != GW_OK) return fail(st);
  p->ws_cap = (opt && opt->workspace_bytes) ? opt->workspace_bytes
                                            : (p->w_tensor || p->w_block ? ((size_t)24 << 30) : ((size_t)4 << 30));
  if (p->w_tensor || p->w_block) {
    p->smem_GJ32 = gw::gj32_smem(p->w_block ? p->w_bs : (int)npb);
    if ((p->w_block ? gw::wblk_setup(p->smem_GJ32) : gw::wtc_setup(p->smem_GJ32)) != cudaSuccess) {
      cudaError_t e = cudaGetLastError();
      set_last_error(std::string("cudaFuncSetAttribute (tensor W): ") + cudaGetErrorString(e));
      return fail(GW_ERR_UNSUPPORTED);
    }
  }
  const bool defer = opt && opt->defer_scratch;
  if (defer) p->w_pending = true;
  else if ((st = alloc_w_scratch(p)) != GW_OK) return fail(st);

  // dynamic shared memory opt-ins
  p->smem_P = smem_polar(h);
  p->smem_S = smem_sigma(h);
  p->smem_T = (size_t)std::max(std::max(h.n_tau, h.n_omega), h.n_nu) * 32 * sizeof(double2);
  // Gauss-Jordan form: blocked (panel in shared memory) when the panel fits, else unblocked
  p->gj_blocked = npb >= 64 && (2 * npb * gw::kGJB + npb) * sizeof(double2) <= 220 * 1024;
  p->smem_GJ = p->gj_blocked ? (2 * npb * gw::kGJB + npb) * sizeof(double2) : 2 * npb * sizeof(double2);
  if (p->smem_GJ > 227 * 1024) {
    set_last_error("product basis too large for the single-block Gauss-Jordan solve");
    return fail(GW_ERR_UNSUPPORTED);
  }
  if (gw::raise_smem_limit(gw::k_polarizability_fp64, (int)p->smem_P) != cudaSuccess ||
      gw::raise_smem_limit(gw::k_self_energy_fp64, (int)p->smem_S) != cudaSuccess ||
      gw::raise_smem_limit(gw::k_transform, (int)p->smem_T) != cudaSuccess ||
      gw::raise_smem_limit(p->gj_blocked ? gw::k_gj_inverse_blocked : gw::k_gj_inverse, (int)p->smem_GJ) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    set_last_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return fail(GW_ERR_UNSUPPORTED);
  }
  if ((st = gw::mixed_init(p->mixed, h, de)) != GW_OK) return fail(st);
  if ((st = gw::ctables_init(p->ct, h)) != GW_OK) return fail(st);
  if (p->ct.ready) {
    // the queue kernels where their configuration fits this device; otherwise the
    // mixed path keeps its per-entry kernels
    p->contract_p = gw::contract_config(false, p->ct.np_max, p->ct.kd_max, p->cfgP, p->device) == GW_OK;
    p->contract_s = gw::contract_config(true, p->ct.nj_max, p->ct.kds_max, p->cfgS, p->device) == GW_OK;
    const std::vector<gw::CUnit> uP = gw::contract_units(h, 0, false), uS = gw::contract_units(h, 0, true);
    p->n_unitsP = (int)uP.size();
    p->n_unitsS = (int)uS.size();
    if ((st = upload(&p->d_unitsP, uP.data(), uP.size() * sizeof(gw::CUnit))) != GW_OK) return fail(st);
    if ((st = upload(&p->d_unitsS, uS.data(), uS.size() * sizeof(gw::CUnit))) != GW_OK) return fail(st);
    const std::vector<gw::CUnit> uX = gw::contract_units(h, 0, true, 1);
    p->n_unitsX = (int)uX.size();
    if ((st = upload(&p->d_unitsX, uX.data(), uX.size() * sizeof(gw::CUnit))) != GW_OK) return fail(st);
    if ((st = upload(&p->d_counter, nullptr, 16)) != GW_OK) return fail(st);
    gw::set_last_error("");
  }
  if (p->sigma_tensor) {
    if (defer) p->oz_pending = true;
    else if ((st = alloc_oz_sigma(p)) != GW_OK) return fail(st);
  }
  if (!(opt && opt->fp64_products == 1)) {
    if ((st = gw::oz_transform_init(p->ozt, h)) != GW_OK) return fail(st);
    if (defer) p->ozp_pending = true;
    else if ((st = alloc_oz_pol(p)) != GW_OK) return fail(st);
  }
  if (gw::uploads_landed() != cudaSuccess) {
    set_last_error("plan tables did not reach the device");
    return fail(GW_ERR_CUDA);
  }
  *out = p;
  return GW_OK;
}

gw_status gw_plan_destroy(gw_plan_t p) {
  if (!p) return GW_OK;
  if (!p->host_only) {
    DeviceGuard guard(p->device);
    p->timer.release();
    free_device(p);
  }
  delete p;
  return GW_OK;
}

gw_status gw_plan_query(gw_plan_t p, gw_plan_info* info) {
  if (!p || !info) { set_last_error("null argument"); return GW_ERR_ARG; }
  const gw::HostPlan& h = p->h;
  std::memset(info, 0, sizeof(*info));
  info->n_atoms = h.n_atoms;
  info->n_entries = h.n_entries();
  info->n_k = h.n_k;
  info->n_tau = h.n_tau;
  info->n_omega = h.n_omega;
  info->n_nu = h.n_nu;
  info->n_orb_total = h.n_orb_total();
  info->n_pb_total = h.n_pb_total();
  for (int i = 0; i < 3; ++i) {
    info->kmesh[i] = h.kmesh[i];
    info->kmesh_required[i] = h.kmesh_required[i];
  }
  info->c_symmetric = h.c_symmetric;
  info->len_orb = h.off_orb.back();
  info->len_pb = h.off_pb.back();
  info->n_entries_far = h.n_far;
  info->n_entries_near = h.n_near;
  info->workspace_bytes = p->ws_bytes;
  info->nu_chunk = p->nu_chunk;
  info->cond_fermion = h.cond_f;
  info->cond_boson = h.cond_b;
  info->w_symmetric = p->w_sym ? 1 : 0;
  info->w_tensor = p->w_tensor ? 1 : 0;
  info->w_block = p->w_bs;
  info->sigma_tensor = p->sigma_tensor ? 1 : 0;
  info->p_tensor = (p->ozp.ready || p->ozp_pending) ? 1 : 0;  // pending: planned at the first call
  info->mixed_queue = (p->contract_p ? 1 : 0) | (p->contract_s ? 2 : 0);
  info->transform_tensor = (p->ozt.ready_w ? 1 : 0) | (p->ozt.ready_p ? 2 : 0);
  info->n_q_solved = p->n_qh;
  return GW_OK;
}

gw_status gw_plan_entries(gw_plan_t p, int64_t* rows) {
  if (!p || !rows) { set_last_error("null argument"); return GW_ERR_ARG; }
  std::memcpy(rows, p->h.entries.data(), p->h.entries.size() * sizeof(int64_t));
  return GW_OK;
}

gw_status gw_plan_offsets(gw_plan_t p, gw_block kind, int64_t* off) {
  if (!p || !off) { set_last_error("null argument"); return GW_ERR_ARG; }
  const std::vector<int64_t>& v = (kind == GW_BLOCK_PB) ? p->h.off_pb : p->h.off_orb;
  std::memcpy(off, v.data(), v.size() * sizeof(int64_t));
  return GW_OK;
}

gw_status gw_plan_entry_dims(gw_plan_t p, gw_block kind, int32_t* rows, int32_t* cols) {
  if (!p || !rows || !cols) { set_last_error("null argument"); return GW_ERR_ARG; }
  const gw::HostPlan& h = p->h;
  for (int e = 0; e < h.n_entries(); ++e) {
    if (kind == GW_BLOCK_PB) {
      rows[e] = h.Ka_e[e];
      cols[e] = h.Kb_e[e];
    } else {
      rows[e] = h.n_orb[h.species[h.entries[8 * e]]];
      cols[e] = h.n_orb[h.species[h.entries[8 * e + 1]]];
    }
  }
  return GW_OK;
}

gw_status gw_plan_transform_matrix(gw_plan_t p, gw_statistics st, gw_direction dir, double* out) {
  if (!p || !out) { set_last_error("null argument"); return GW_ERR_ARG; }
  const std::vector<double>* m;
  if (st == GW_FERMION) m = (dir == GW_TAU_TO_IW) ? &p->h.Tf_fwd : &p->h.Tf_inv;
  else m = (dir == GW_TAU_TO_IW) ? &p->h.Tb_fwd : &p->h.Tb_inv;
  std::memcpy(out, m->data(), m->size() * sizeof(double));
  return GW_OK;
}

gw_status gw_fourier_k_to_R(gw_plan_t p, gw_block kind, int n_slices, const void* F_k, void* F_R, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!F_k || !F_R || n_slices <= 0) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const long long N = dense_n(p, kind);
  return launch_gather(p, kind, n_slices, (const double2*)F_k, (long long)n_slices * N * N, N * N, nullptr, 0, 0,
                       (double2*)F_R, n_slices, 0, 1.0 / p->h.n_k, S(stream));
}

gw_status gw_green_k_to_R(gw_plan_t p, const void* G_k, void* G_R, void* stream) {
  if (!p) { set_last_error("null plan"); return GW_ERR_ARG; }
  return gw_fourier_k_to_R(p, GW_BLOCK_ORB, p->h.n_tau, G_k, G_R, stream);
}

gw_status gw_fourier_R_to_k(gw_plan_t p, gw_block kind, int n_slices, const void* F_R, void* F_k, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!F_k || !F_R || n_slices <= 0) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const long long N = dense_n(p, kind);
  return launch_scatter(p, kind, n_slices, (const double2*)F_R, n_slices, 0, (double2*)F_k,
                        (long long)n_slices * N * N, N * N, S(stream));
}

gw_status gw_transform_tau_iw_ex(gw_plan_t p, gw_statistics stt, gw_direction dir, gw_block kind, int structure,
                                 const void* in, void* out, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!in || !out) { set_last_error("bad argument"); return GW_ERR_ARG; }
  if (structure != 0 && structure != GW_IN_MIRROR && structure != GW_IN_REAL &&
      structure != (GW_IN_MIRROR | GW_OUT_NONNEG)) {
    set_last_error("unknown input structure");
    return GW_ERR_ARG;
  }
  if ((structure & GW_IN_MIRROR) && !(stt == GW_BOSON && dir == GW_TAU_TO_IW)) {
    set_last_error("GW_IN_MIRROR applies to the bosonic tau -> i nu transform only");
    return GW_ERR_UNSUPPORTED;
  }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const gw::HostPlan& h = p->h;
  if (kind == GW_BLOCK_PB && stt == GW_BOSON &&
      ((structure == GW_IN_REAL && dir == GW_IW_TO_TAU && p->ozt.ready_w) ||
       ((structure & GW_IN_MIRROR) && p->ozt.ready_p)))
    return gw::oz_transform(p->ozt, h, p->d_ent, structure, (const double2*)in, (double2*)out, p->d_status,
                            S(stream));
  // GW_OUT_NONNEG: the slices of the frequencies nu >= 0 only (ascending sampled indices)
  int m_begin = 0;
  if (structure & GW_OUT_NONNEG) {
    bool ascending = true;
    for (int j = 1; j < h.n_nu; ++j) ascending = ascending && h.nu_idx[j] > h.nu_idx[j - 1];
    while (ascending && m_begin < h.n_nu && h.nu_idx[m_begin] < 0) ++m_begin;
    structure &= ~GW_OUT_NONNEG;
  }
  if (structure == 0 && gw::oz_general_ready(p->ozt, stt == GW_FERMION, dir == GW_IW_TO_TAU, kind == GW_BLOCK_PB))
    return gw::oz_general_run(p->ozt, h, p->d_ent, stt == GW_FERMION, dir == GW_IW_TO_TAU, kind == GW_BLOCK_PB,
                              (const double2*)in, (double2*)out, p->d_status, S(stream));
  gw::TransformArgs g{};
  g.m_begin = m_begin;
  g.ent = p->d_ent;
  const int nfreq = (stt == GW_FERMION) ? h.n_omega : h.n_nu;
  if (dir == GW_TAU_TO_IW) {
    g.T = (stt == GW_FERMION) ? p->d_Tf_fwd : p->d_Tb_fwd;
    g.n_in = h.n_tau;
    g.n_out = nfreq;
  } else {
    g.T = (stt == GW_FERMION) ? p->d_Tf_inv : p->d_Tb_inv;
    g.n_in = nfreq;
    g.n_out = h.n_tau;
  }
  g.in_stride = g.n_in;
  g.mode = 0;
  if (structure == GW_IN_MIRROR) {
    g.T = p->d_Tb_mirror;
    g.n_in = (h.n_tau + 1) / 2;
    g.mode = 1;
  } else if (structure == GW_IN_REAL) {
    g.mode = 2;
  }
  g.pb = kind == GW_BLOCK_PB;
  g.in = (const double2*)in;
  g.out = (double2*)out;
  int maxblk = 0;
  for (int s = 0; s < h.n_species; ++s)
    for (int t = 0; t < h.n_species; ++t)
      maxblk = std::max(maxblk, g.pb ? h.n_prod[s] * h.n_prod[t] : h.n_orb[s] * h.n_orb[t]);
  dim3 grid(h.n_entries(), (maxblk + 31) / 32);
  dim3 block(32, 8);
  {
    gw::TimedLaunch tl_("k_transform", S(stream));
    gw::k_transform<<<grid, block, (size_t)g.n_in * 32 * sizeof(double2), S(stream)>>>(g);
  }
  return check_launch("k_transform");
}

gw_status gw_transform_tau_iw(gw_plan_t p, gw_statistics stt, gw_direction dir, gw_block kind, const void* in,
                              void* out, void* stream) {
  return gw_transform_tau_iw_ex(p, stt, dir, kind, 0, in, out, stream);
}

// One plan's entry in a queue launch of the contraction kernels.
static gw::CSys contract_sys(const gw_plan_s* p, const double2* G, const double2* W, double2* out) {
  gw::CSys s{};
  s.ent = p->d_ent;
  s.Cp = p->ct.d_Cp;
  s.cp_off = p->ct.d_cp_off;
  s.cp_ld = p->ct.d_cp_ld;
  s.Bp = W ? p->ct.d_BpS : p->ct.d_BpP;
  s.bp_off = W ? p->ct.d_bpS_off : p->ct.d_bpP_off;
  s.species = p->ct.d_species;
  s.G = G;
  s.W = W;
  s.out = out;
  s.n_tau = p->h.n_tau;
  s.g_slices = s.w_slices = s.out_slices = p->h.n_tau;
  s.g_fixed = -1;
  s.sign = -1.0;
  s.spin = p->h.spin;
  s.mirror = p->h.c_symmetric;
  return s;
}

gw_status gw_polarizability_tau(gw_plan_t p, const void* G_R, void* P_R, gw_precision prec, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!G_R || !P_R) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const gw::HostPlan& h = p->h;
  if (prec == GW_MIXED) {
    if (p->contract_p) {
      gw::CBatch b{};
      b.n = 1;
      b.s[0] = contract_sys(p, (const double2*)G_R, nullptr, (double2*)P_R);
      return gw::contract_launch(false, p->cfgP, b, p->d_unitsP, p->n_unitsP, p->d_counter, p->d_status, S(stream));
    }
    return gw::mixed_polarizability(p->mixed, h, p->d_ent, p->d_C, (const double2*)G_R, (double2*)P_R, p->d_status,
                                    S(stream));
  }
  if (prec != GW_FP64) { set_last_error("unknown precision"); return GW_ERR_ARG; }
  gw::ContractArgs g{};
  g.ent = p->d_ent;
  g.C = p->d_C;
  g.G = (const double2*)G_R;
  g.out = (double2*)P_R;
  g.n_tau = h.n_tau;
  g.spin = h.spin;
  g.mirror_tau = h.c_symmetric;
  const int nt_eff = h.c_symmetric ? (h.n_tau + 1) / 2 : h.n_tau;
  if (p->ozp_pending && (st = alloc_oz_pol(p)) != GW_OK) return st;
  if (p->ozp.ready) {
    // stages 1 and 2 in FP64 (Y to the pass buffer), stage 3 on the tensor cores, per pass
    for (int s0 = 0; s0 < nt_eff; s0 += p->ozp.tau_c) {
      const int te = std::min(p->ozp.tau_c, nt_eff - s0);
      g.Ypre = p->ozp.d_Ypre;
      g.offB = p->ozp.d_offB;
      g.tau_c = p->ozp.tau_c;
      g.s0 = s0;
      {
        gw::TimedLaunch tl_("k_polarizability_fp64", S(stream));
        gw::k_polarizability_fp64<<<dim3(h.n_entries(), te), 256, p->smem_P, S(stream)>>>(g);
      }
      if ((st = check_launch("k_polarizability_fp64")) != GW_OK) return st;
      if ((st = gw::oz_pol_stage3(p->ozp, h, p->d_ent, s0, te, (double2*)P_R, p->d_status, S(stream))) != GW_OK)
        return st;
    }
    return GW_OK;
  }
  dim3 grid(h.n_entries(), nt_eff);
  {
    gw::TimedLaunch tl_("k_polarizability_fp64", S(stream));
    gw::k_polarizability_fp64<<<grid, 256, p->smem_P, S(stream)>>>(g);
  }
  return check_launch("k_polarizability_fp64");
}

gw_status gw_self_energy_tau(gw_plan_t p, const void* G_R, const void* Wt_R, const void* v_R, void* Sig_R,
                             void* Sigx_R, gw_precision prec, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!G_R || !Wt_R || !Sig_R) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const gw::HostPlan& h = p->h;
  if (prec == GW_MIXED) {
    if (p->contract_s) {
      gw::CBatch b{};
      b.n = 1;
      b.s[0] = contract_sys(p, (const double2*)G_R, (const double2*)Wt_R, (double2*)Sig_R);
      st = gw::contract_launch(true, p->cfgS, b, p->d_unitsS, p->n_unitsS, p->d_counter, p->d_status, S(stream));
    } else {
      st = gw::mixed_self_energy(p->mixed, h, p->d_ent, p->d_C, (const double2*)G_R, (const double2*)Wt_R,
                                 (double2*)Sig_R, p->d_status, S(stream));
    }
    if (st != GW_OK) return st;
  } else if (prec == GW_FP64) {
    gw::ContractArgs g{};
    g.ent = p->d_ent;
    g.C = p->d_C;
    g.G = (const double2*)G_R;
    g.W = (const double2*)Wt_R;
    g.out = (double2*)Sig_R;
    g.n_tau = h.n_tau;
    g.g_n_slices = h.n_tau;
    g.g_slice = -1;
    g.w_n_slices = h.n_tau;
    g.out_n_slices = h.n_tau;
    g.sign = -1.0;
    if (p->oz_pending && (st = alloc_oz_sigma(p)) != GW_OK) return st;
    if (p->sigma_tensor) {
      // stage A (W~ C^b) on the tensor cores per pass of tau slices, stages B and C in FP64
      for (int s0 = 0; s0 < h.n_tau; s0 += p->oz.tau_c) {
        const int te = std::min(p->oz.tau_c, h.n_tau - s0);
        if ((st = gw::oz_sigma_stage_a(p->oz, h, p->d_ent, (const double2*)Wt_R, s0, te, p->d_status, S(stream))) !=
            GW_OK)
          return st;
        g.Bpre = p->oz.d_Bpre;
        g.offB = p->oz.d_offB;
        g.tau_c = p->oz.tau_c;
        g.s0 = s0;
        dim3 grid(h.n_entries(), te);
        {
          gw::TimedLaunch tl_("k_self_energy_fp64", S(stream));
          gw::k_self_energy_fp64<<<grid, 256, p->smem_S, S(stream)>>>(g);
        }
        if ((st = check_launch("k_self_energy_fp64")) != GW_OK) return st;
      }
    } else {
      dim3 grid(h.n_entries(), h.n_tau);
      {
        gw::TimedLaunch tl_("k_self_energy_fp64", S(stream));
        gw::k_self_energy_fp64<<<grid, 256, p->smem_S, S(stream)>>>(g);
      }
      if ((st = check_launch("k_self_energy_fp64")) != GW_OK) return st;
    }
  } else {
    set_last_error("unknown precision");
    return GW_ERR_ARG;
  }
  if (v_R && Sigx_R && prec == GW_MIXED && p->contract_s) {
    // exchange: W~ -> v, G(tau) -> -G(beta-): +C G(beta-) v C, one node per entry through the
    // same queue kernel (reduced precision like the dynamic part)
    gw::CBatch b{};
    b.n = 1;
    b.s[0] = contract_sys(p, (const double2*)G_R, (const double2*)v_R, (double2*)Sigx_R);
    b.s[0].w_slices = b.s[0].out_slices = 1;
    b.s[0].g_fixed = h.n_tau - 1;
    b.s[0].sign = +1.0;
    return gw::contract_launch(true, p->cfgS, b, p->d_unitsX, p->n_unitsX, p->d_counter, p->d_status, S(stream));
  }
  if (v_R && Sigx_R) {
    // exchange: W~ -> v, G(tau) -> -G(beta-): +C G(beta-) v C in FP64
    gw::ContractArgs g{};
    g.ent = p->d_ent;
    g.C = p->d_C;
    g.G = (const double2*)G_R;
    g.W = (const double2*)v_R;
    g.out = (double2*)Sigx_R;
    g.n_tau = h.n_tau;
    g.g_n_slices = h.n_tau;
    g.g_slice = h.n_tau - 1;
    g.w_n_slices = 1;
    g.out_n_slices = 1;
    g.sign = +1.0;
    dim3 grid(h.n_entries(), 1);
    {
      gw::TimedLaunch tl_("k_self_energy_fp64", S(stream));
      gw::k_self_energy_fp64<<<grid, 256, p->smem_S, S(stream)>>>(g);
    }
    if ((st = check_launch("k_self_energy_fp64 (exchange)")) != GW_OK) return st;
  }
  return GW_OK;
}

gw_status gw_screened_W_iw(gw_plan_t p, const void* P_R_iw, const void* v_q, void* Wt_R_iw, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!P_R_iw || !v_q || !Wt_R_iw) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer timing(&p->timer);
  const gw::HostPlan& h = p->h;
  cudaStream_t s = S(stream);
  if (p->w_pending && (st = alloc_w_scratch(p)) != GW_OK) return st;
  const long long N = h.n_pb_total();
  const long long NN = N * N;
  const int nq = p->n_qh;
  const double2* v = (const double2*)v_q;
  // v(q)^{-1} for the solved momenta
  {
    dim3 g((unsigned)std::min<long long>((NN + 255) / 256, 1024), (unsigned)nq);
    {
      gw::TimedLaunch tl_("k_copy_mats", s);
      gw::k_copy_mats<<<g, 256, 0, s>>>(v, p->d_qh, p->d_wsV, NN);
    }
    if ((st = check_launch("k_copy_mats")) != GW_OK) return st;
    if (p->w_tensor) st = launch_tensor_inverse(p, p->d_wsV, nq, N, s);
    else if (p->w_block) st = launch_block_inverse(p, p->d_wsV, nq, N, s);
    else st = launch_gj(p, p->d_wsV, nq, N, s);
    if (st != GW_OK) return st;
  }
  const int n_work = h.n_nu - p->nu_start;
  for (int c0 = 0; c0 < n_work; c0 += p->nu_chunk) {
    const int nc = std::min(p->nu_chunk, n_work - c0);
    const int slot0 = p->nu_start + c0;
    // A = v(q)^{-1} - P(q, nu) for the chunk, [nu][q][N][N]
    // symmetric mode: P(R, i nu) is real (the imaginary parts are not read)
    if ((st = launch_scatter(p, GW_BLOCK_PB, nc, (const double2*)P_R_iw, h.n_nu, slot0, p->d_wsA, NN,
                             (long long)nq * NN, s, p->d_qh, nq, p->d_wsV, -1.0, p->w_sym)) != GW_OK)
      return st;
    if (p->w_tensor) st = launch_tensor_inverse(p, p->d_wsA, nc * nq, N, s);
    else if (p->w_block) st = launch_block_inverse(p, p->d_wsA, nc * nq, N, s);
    else st = launch_gj(p, p->d_wsA, nc * nq, N, s);
    if (st != GW_OK) return st;
    // W~(R) = (1/N_k) sum_q e^{-iqR} (W(q) - v(q)); in symmetric mode the sum runs over
    // one momentum of each (q, -q) pair with weight 2 and keeps the (exactly real) real part
    if ((st = launch_gather(p, GW_BLOCK_PB, nc, p->d_wsA, NN, (long long)nq * NN, v, NN, 0, (double2*)Wt_R_iw,
                            h.n_nu, slot0, 1.0 / h.n_k, s, p->d_qh, p->w_sym ? p->d_qw : nullptr, nq,
                            p->w_sym ? 1 : 0)) != GW_OK)
      return st;
  }
  if (p->w_sym && p->n_neg > 0) {
    dim3 g((unsigned)h.n_entries(), (unsigned)p->n_neg);
    {
      gw::TimedLaunch tl_("k_mirror_nu", s);
      gw::k_mirror_nu<<<g, 256, 0, s>>>(p->d_ent, p->d_numirror, p->n_neg, h.n_nu, (double2*)Wt_R_iw);
    }
    if ((st = check_launch("k_mirror_nu")) != GW_OK) return st;
  }
  return GW_OK;
}

gw_status gw_sync(gw_plan_t p, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  DeviceGuard guard(p->device);
  GW_CUDA(cudaStreamSynchronize(S(stream)));
  int flag = 0;
  GW_CUDA(cudaMemcpyAsync(&flag, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
  GW_CUDA(cudaStreamSynchronize(S(stream)));
  if (flag) {
    // cleared on the caller's stream, ordered before any later launch on it
    GW_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), S(stream)));
    GW_CUDA(cudaStreamSynchronize(S(stream)));
    if (flag == 2) {
      set_last_error("a tensor-core wait gave up (bounded wait)");
      return GW_ERR_TIMEOUT;
    }
    set_last_error("zero pivot in the W solve");
    return GW_ERR_SINGULAR;
  }
  return GW_OK;
}

gw_status gw_timing_enable(gw_plan_t p, int enable) {
  if (!p) { set_last_error("null plan"); return GW_ERR_ARG; }
  p->timer.on = enable != 0;
  return GW_OK;
}

gw_status gw_timing_read(gw_plan_t p, int index, const char** name, double* total_ms, long long* launches) {
  if (!p || index < 0) { set_last_error("bad argument"); return GW_ERR_ARG; }
  if (!p->host_only) {
    DeviceGuard guard(p->device);
    cudaError_t e = p->timer.collect();
    if (e != cudaSuccess) return cuda_fail(e, "gw_timing_read");
  }
  if (index >= (int)p->timer.totals.size()) { set_last_error("no such timing entry"); return GW_ERR_ARG; }
  const gw::KernelTimer::Total& t = p->timer.totals[(size_t)index];
  if (name) *name = t.name.c_str();
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.launches;
  return GW_OK;
}

gw_status gw_timing_reset(gw_plan_t p) {
  if (!p) { set_last_error("null plan"); return GW_ERR_ARG; }
  if (!p->host_only) {
    DeviceGuard guard(p->device);
    p->timer.reset();
  } else {
    p->timer.totals.clear();
  }
  return GW_OK;
}

gw_status gw_dyson_green_tau(gw_plan_t p, const void* H_k, const void* Sigx_k, const void* Sig_k_iw, double mu,
                             void* G_k_tau, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!H_k || !G_k_tau || !std::isfinite(mu)) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer at_(&p->timer);
  if ((st = gw::dyson_init(p->dyson, p->h)) != GW_OK) return st;
  cudaStream_t s = S(stream);
  const double2* H = (const double2*)H_k;
  const double2* Sx = (const double2*)Sigx_k;
  if ((st = gw::dyson_solve(p->dyson, p->h, H, Sx, (const double2*)Sig_k_iw, mu, p->d_status, s)) != GW_OK) return st;
  return gw::dyson_to_tau(p->dyson, p->h, H, Sx, mu, p->d_Tf_inv, (double2*)G_k_tau, s);
}

gw_status gw_chemical_potential(gw_plan_t p, const void* H_k, const void* Sigx_k, const void* Sig_k_iw,
                                double n_electrons, double mu_lo, double mu_hi, double tol, double* mu_out,
                                double* n_out, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!H_k || !mu_out || !(mu_lo < mu_hi) || !(tol > 0.0) || !std::isfinite(n_electrons)) {
    set_last_error("bad argument");
    return GW_ERR_ARG;
  }
  DeviceGuard guard(p->device);
  gw::ActiveTimer at_(&p->timer);
  if ((st = gw::dyson_init(p->dyson, p->h)) != GW_OK) return st;
  const gw::HostPlan& h = p->h;
  cudaStream_t s = S(stream);
  const double2* H = (const double2*)H_k;
  const double2* Sx = (const double2*)Sigx_k;
  const double2* Tlast = p->d_Tf_inv + (size_t)(h.n_tau - 1) * h.n_omega;  // the row of tau = beta-
  std::vector<double> part(h.n_k);
  // N(mu) = s (1/N_k) sum_k Re Tr[-G(k, beta-)], one Dyson solve per evaluation
  auto count = [&](double mu, double* n) -> gw_status {
    gw_status e = gw::dyson_solve(p->dyson, h, H, Sx, (const double2*)Sig_k_iw, mu, p->d_status, s);
    if (e == GW_OK) e = gw::dyson_density(p->dyson, h, H, Sx, mu, Tlast, s);
    if (e != GW_OK) return e;
    GW_CUDA(cudaMemcpyAsync(part.data(), p->dyson.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    int flag = 0;
    GW_CUDA(cudaMemcpyAsync(&flag, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    if (flag) {
      GW_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
      GW_CUDA(cudaStreamSynchronize(s));
      set_last_error("zero pivot in the Dyson solve");
      return GW_ERR_SINGULAR;
    }
    double t = 0.0;
    for (double v : part) t += v;
    *n = h.spin * t / h.n_k;
    return GW_OK;
  };
  double lo = mu_lo, hi = mu_hi, n = 0.0;
  for (int it = 0; it < 200 && hi - lo > tol; ++it) {
    const double mid = 0.5 * (lo + hi);
    if ((st = count(mid, &n)) != GW_OK) return st;
    if (n < n_electrons) lo = mid;
    else hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  if ((st = count(mu, &n)) != GW_OK) return st;
  *mu_out = mu;
  if (n_out) *n_out = n;
  return GW_OK;
}

gw_status gw_qp_energies(gw_plan_t p, const void* H_k, const void* Sigx_k, const void* Sig_k_iw, double mu,
                         void* E_k, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!H_k || !E_k || !std::isfinite(mu)) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  gw::ActiveTimer at_(&p->timer);
  if ((st = gw::dyson_init(p->dyson, p->h)) != GW_OK) return st;
  return gw::qp_energies(p->h, (const double2*)H_k, (const double2*)Sigx_k, (const double2*)Sig_k_iw, mu,
                         p->dyson.ainv, (double*)E_k, S(stream));
}

gw_status gw_continue_sigma(gw_plan_t p, const void* Sig_k_iw, int n_real, const double* w_real, double delta,
                            void* Sig_k_w, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!Sig_k_iw || !Sig_k_w || !w_real || n_real < 1 || !(delta >= 0.0)) {
    set_last_error("bad argument");
    return GW_ERR_ARG;
  }
  DeviceGuard guard(p->device);
  gw::ActiveTimer at_(&p->timer);
  if ((st = gw::dyson_init(p->dyson, p->h)) != GW_OK) return st;
  return gw::continue_sigma(p->dyson, p->h, (const double2*)Sig_k_iw, n_real, w_real, delta, (double2*)Sig_k_w,
                            S(stream));
}

gw_status gw_spectral_function(gw_plan_t p, const void* H_k, const void* Sigx_k, const void* Sig_k_w, int n_real,
                               const double* w_real, double delta, double mu, void* A_kw, void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!H_k || !A_kw || !w_real || n_real < 1 || !(delta > 0.0) || !std::isfinite(mu)) {
    set_last_error("bad argument");
    return GW_ERR_ARG;
  }
  DeviceGuard guard(p->device);
  gw::ActiveTimer at_(&p->timer);
  if ((st = gw::dyson_init(p->dyson, p->h)) != GW_OK) return st;
  return gw::spectral_function(p->dyson, p->h, (const double2*)H_k, (const double2*)Sigx_k, (const double2*)Sig_k_w,
                               n_real, w_real, delta, mu, (double*)A_kw, p->d_status, S(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free W solve (gw_screened_W_iw_noalloc; no counterpart in the paper)
// ---------------------------------------------------------------------------
// Its scratch is a fixed array in the library's device image instead of the plan's
// workspace, for callers that cannot allocate device memory while they run.

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB on every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device: a host-side name of a
// __device__ array is not a device address, so it is looked up once per device.
gw_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_last_error("device ordinal out of range for the fixed scratch");
    return GW_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return GW_OK;
}

// Zero the bosonic slots [slot0, n_slots) of every entry (PB blocks).
__global__ void k_zero_slots(const gw::DevEntry* __restrict__ ent, int n_slots, int slot0, double2* __restrict__ W) {
  const gw::DevEntry E = ent[blockIdx.x];
  const int blk = E.Ka * E.Kb;
  double2* w = W + E.off_pb * n_slots + (long long)(slot0 + blockIdx.y) * blk;
  for (int x = threadIdx.x; x < blk; x += blockDim.x) w[x] = make_double2(0.0, 0.0);
}

// W~_R[e][slot0 + s] += scale w conj(e^{iq.R}) (W(q) - v(q)) for one momentum q, taking the
// real part in symmetric mode; grid (active pair, slice, element chunk).
__global__ void k_gather_one_q(const gw::DevEntry* __restrict__ ent, const int* __restrict__ pair_first,
                               const int* __restrict__ pb_off, const double2* __restrict__ phase, int n_k, int q,
                               double w, const double2* __restrict__ Wq, long long s_stride,
                               const double2* __restrict__ vq, int ld, double2* __restrict__ out, int n_slots,
                               int slot0, double scale, int real_only) {
  const int p = blockIdx.x;
  const int s = blockIdx.y;
  const int e0 = pair_first[p], e1 = pair_first[p + 1];
  const gw::DevEntry E0 = ent[e0];
  // the pair's full block; an entry beyond sphere B keeps its top-left K_a(e) x K_b(e)
  const int cols = pb_off[E0.b + 1] - pb_off[E0.b];
  const int blk = (pb_off[E0.a + 1] - pb_off[E0.a]) * cols;
  const int idx = blockIdx.z * blockDim.x + threadIdx.x;
  if (idx >= blk) return;
  const int i = idx / cols, j = idx - (idx / cols) * cols;
  const long long el = (long long)(E0.pa + i) * ld + (E0.pb + j);
  const double2 a = Wq[(long long)s * s_stride + el];
  const double2 b = vq[(long long)q * ld * ld + el];
  const double vr = (a.x - b.x) * w * scale, vi = (a.y - b.y) * w * scale;
  for (int e = e0; e < e1; ++e) {
    const gw::DevEntry& E = ent[e];
    if (i >= E.Ka || j >= E.Kb) continue;
    const double2 ph = phase[(long long)e * n_k + q];
    const double rr = ph.x * vr + ph.y * vi;
    const double ri = real_only ? 0.0 : ph.x * vi - ph.y * vr;
    double2* o = out + E.off_pb * n_slots + (long long)(slot0 + s) * E.Ka * E.Kb + i * E.Kb + j;
    const double2 t = *o;
    *o = make_double2(t.x + rr, t.y + ri);
  }
}

}  // namespace

extern "C" gw_status gw_screened_W_iw_noalloc(gw_plan_t p, const void* P_R_iw, const void* v_q, void* Wt_R_iw,
                                              void* stream) {
  gw_status st = need_device(p);
  if (st != GW_OK) return st;
  if (!P_R_iw || !v_q || !Wt_R_iw) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(p->device);
  const gw::HostPlan& h = p->h;
  const long long N = h.n_pb_total();
  const long long NN = N * N;
  const size_t mat = (size_t)NN * sizeof(double2);
  const size_t perm_bytes = ((size_t)N * sizeof(int) + 255) & ~(size_t)255;
  // v(q)^-1 and at least one (q, nu) matrix, each with its pivot record
  if (2 * (mat + perm_bytes) > kNoAllocScratchBytes) {
    set_last_error("product basis too large for the fixed 32 MiB scratch of gw_screened_W_iw_noalloc "
                   "(needs 2 N_PB^2 complex values)");
    return GW_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  if ((st = noalloc_scratch(p->device, &base)) != GW_OK) return st;
  cudaStream_t s = S(stream);
  const int n_work = h.n_nu - p->nu_start;
  const int n_slots = (int)std::min<size_t>((size_t)n_work, kNoAllocScratchBytes / (mat + perm_bytes) - 1);
  unsigned char* bytes = static_cast<unsigned char*>(base);
  double2* vinv = reinterpret_cast<double2*>(bytes);
  double2* slots = reinterpret_cast<double2*>(bytes + mat);
  int* perm = reinterpret_cast<int*>(bytes + (size_t)(1 + n_slots) * mat);
  const double2* v = (const double2*)v_q;
  // the momenta solved (one of each (q, -q) pair in symmetric mode) and their weights
  std::vector<int> qh;
  std::vector<double> qw;
  for (int q = 0, q1 = 0; q1 < h.kmesh[0]; ++q1)
    for (int q2 = 0; q2 < h.kmesh[1]; ++q2)
      for (int q3 = 0; q3 < h.kmesh[2]; ++q3, ++q) {
        const int mq = (((h.kmesh[0] - q1) % h.kmesh[0]) * h.kmesh[1] + (h.kmesh[1] - q2) % h.kmesh[1]) * h.kmesh[2] +
                       (h.kmesh[2] - q3) % h.kmesh[2];
        if (!p->w_sym) { qh.push_back(q); qw.push_back(1.0); }
        else if (q <= mq) { qh.push_back(q); qw.push_back(q == mq ? 1.0 : 2.0); }
      }
  // the solved slots accumulate over momenta: they start from zero (the array keeps the
  // previous call's contents, and so does the output)
  {
    dim3 g((unsigned)h.n_entries(), (unsigned)n_work);
    k_zero_slots<<<g, 256, 0, s>>>(p->d_ent, h.n_nu, p->nu_start, (double2*)Wt_R_iw);
    if ((st = check_launch("k_zero_slots")) != GW_OK) return st;
  }
  int maxblk = 0;
  for (int a = 0; a < h.n_species; ++a)
    for (int b2 = 0; b2 < h.n_species; ++b2) maxblk = std::max(maxblk, h.n_prod[a] * h.n_prod[b2]);
  for (size_t qi = 0; qi < qh.size(); ++qi) {
    dim3 gc((unsigned)std::min<long long>((NN + 255) / 256, 1024), 1);
    gw::k_copy_mats<<<gc, 256, 0, s>>>(v, p->d_qh + qi, vinv, NN);
    if ((st = check_launch("k_copy_mats")) != GW_OK) return st;
    if (p->gj_blocked) gw::k_gj_inverse_blocked<<<1, 512, p->smem_GJ, s>>>(vinv, perm, (int)N, NN, p->d_status);
    else gw::k_gj_inverse<<<1, 512, p->smem_GJ, s>>>(vinv, perm, (int)N, NN, p->d_status);
    if ((st = check_launch("k_gj_inverse")) != GW_OK) return st;
    for (int c0 = 0; c0 < n_work; c0 += n_slots) {
      const int nc = std::min(n_slots, n_work - c0);
      const int slot0 = p->nu_start + c0;
      if ((st = launch_scatter(p, GW_BLOCK_PB, nc, (const double2*)P_R_iw, h.n_nu, slot0, slots, NN, NN, s,
                               p->d_qh + qi, 1, vinv, -1.0)) != GW_OK)
        return st;
      if (p->gj_blocked) gw::k_gj_inverse_blocked<<<nc, 512, p->smem_GJ, s>>>(slots, perm, (int)N, NN, p->d_status);
      else gw::k_gj_inverse<<<nc, 512, p->smem_GJ, s>>>(slots, perm, (int)N, NN, p->d_status);
      if ((st = check_launch("k_gj_inverse")) != GW_OK) return st;
      dim3 gg((unsigned)p->n_active, (unsigned)nc, (unsigned)((maxblk + 127) / 128));
      k_gather_one_q<<<gg, 128, 0, s>>>(p->d_ent, p->d_pair_first, p->d_pb_off, p->d_phase, h.n_k, qh[qi], qw[qi], slots, NN, v,
                                         (int)N, (double2*)Wt_R_iw, h.n_nu, slot0, 1.0 / h.n_k, p->w_sym ? 1 : 0);
      if ((st = check_launch("k_gather_one_q")) != GW_OK) return st;
    }
  }
  if (p->w_sym && p->n_neg > 0) {
    dim3 g((unsigned)h.n_entries(), (unsigned)p->n_neg);
    gw::k_mirror_nu<<<g, 256, 0, s>>>(p->d_ent, p->d_numirror, p->n_neg, h.n_nu, (double2*)Wt_R_iw);
    if ((st = check_launch("k_mirror_nu")) != GW_OK) return st;
  }
  return GW_OK;
}

// ---------------------------------------------------------------------------------------
// Batches of systems: the GW_MIXED contractions of several plans in one queue launch
// ---------------------------------------------------------------------------------------

// One shape class of a batch: the plans whose contractions take the same launch shape
// (thread groups and hi x hi accumulators of each stage), with their own unit queues and
// configurations; a batch launch is one kernel launch per class.
struct BatchClass {
  std::vector<int> sys;  // plan indices of the batch
  int ncols_p = 0, kd_p = 0, ncols_s = 0, kd_s = 0;
  gw::CConfig cfgP, cfgS;
  int orderP = 0, orderS = 0;
  gw::CUnit* d_unitsP = nullptr;
  gw::CUnit* d_unitsS = nullptr;
  int nP = 0, nS = 0;
};

struct gw_batch_s {
  std::vector<gw_plan_s*> plans;
  int device = 0;
  std::vector<BatchClass> cls;
  int* d_counter = nullptr;
  int* d_status = nullptr;
  bool tuned = false;
};

namespace {

// The class's units of one contraction in the given order: 0 grouped by shape (species
// pair and basis size, so that consecutive units share their B operand), 1 the heaviest
// first (so that the queue's tail is made of light units).
std::vector<gw::CUnit> batch_units(const gw_batch_s* b, const BatchClass& k, bool sigma, int order) {
  std::vector<gw::CUnit> u;
  std::vector<long long> key;
  for (int i : k.sys) {
    const gw::HostPlan& h = b->plans[i]->h;
    for (const gw::CUnit& x : gw::contract_units(h, i, sigma)) {
      u.push_back(x);
      if (order == 1) {
        key.push_back(-gw::contract_unit_cost(h, x.e, sigma));
      } else {
        const int a = (int)h.entries[8 * x.e], bb = (int)h.entries[8 * x.e + 1];
        const long long na = h.n_orb[h.species[a]], nb = h.n_orb[h.species[bb]];
        key.push_back((((na * 32 + nb) * 256 + h.Ka_e[x.e]) * 256 + h.Kb_e[x.e]) * 32 + i);
      }
    }
  }
  std::vector<size_t> idx(u.size());
  for (size_t q = 0; q < idx.size(); ++q) idx[q] = q;
  std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return key[x] < key[y]; });
  std::vector<gw::CUnit> out(u.size());
  for (size_t q = 0; q < idx.size(); ++q) out[q] = u[idx[q]];
  return out;
}

gw_status batch_upload_units(gw_batch_s* b, BatchClass& k, bool sigma, int order) {
  const std::vector<gw::CUnit> u = batch_units(b, k, sigma, order);
  gw::CUnit*& d = sigma ? k.d_unitsS : k.d_unitsP;
  if (!d) {
    gw_status st = upload(&d, nullptr, u.size() * sizeof(gw::CUnit));
    if (st != GW_OK) return st;
  }
  GW_CUDA(cudaMemcpy(d, u.data(), u.size() * sizeof(gw::CUnit), cudaMemcpyHostToDevice));
  GW_CUDA(gw::uploads_landed());
  (sigma ? k.nS : k.nP) = (int)u.size();
  (sigma ? k.orderS : k.orderP) = order;
  return GW_OK;
}

gw::CBatch batch_systems(const gw_batch_s* b, const void* const* G_R, const void* const* Wt_R, void* const* out) {
  gw::CBatch cb{};
  cb.n = (int)b->plans.size();
  for (int i = 0; i < cb.n; ++i)
    cb.s[i] = contract_sys(b->plans[i], (const double2*)G_R[i], Wt_R ? (const double2*)Wt_R[i] : nullptr,
                           (double2*)out[i]);
  return cb;
}

}  // namespace

gw_status gw_batch_create(const gw_plan_t* plans, int n_plans, gw_batch_t* out) {
  if (!plans || !out || n_plans < 1 || n_plans > GW_BATCH_MAX) {
    set_last_error("gw_batch_create: need 1 .. GW_BATCH_MAX plans");
    return GW_ERR_ARG;
  }
  *out = nullptr;
  gw_batch_s* b = new (std::nothrow) gw_batch_s();
  if (!b) return GW_ERR_OOM;
  for (int i = 0; i < n_plans; ++i) {
    gw_plan_s* p = plans[i];
    if (!p || p->host_only || (i > 0 && p->device != plans[0]->device)) {
      delete b;
      set_last_error("gw_batch_create: device plans on one device only");
      return GW_ERR_ARG;
    }
    if (!p->ct.ready) {
      delete b;
      set_last_error("gw_batch_create: a plan is outside the contraction kernels' limits");
      return GW_ERR_UNSUPPORTED;
    }
    b->plans.push_back(p);
  }
  b->device = plans[0]->device;
  DeviceGuard guard(b->device);
  // shape classes: plans whose own configurations agree on the thread groups and the hi x hi
  // accumulators of both stages share a class (and one launch per contraction); a wide plan
  // then no longer sets the shape of every other plan's launch
  gw_status st = GW_OK;
  std::vector<std::array<int, 4>> keys;
  for (int i = 0; i < n_plans && st == GW_OK; ++i) {
    const gw_plan_s* p = plans[i];
    gw::CConfig cp, cs;
    st = gw::contract_config(false, p->ct.np_max, p->ct.kd_max, cp, b->device);
    if (st == GW_OK) st = gw::contract_config(true, p->ct.nj_max, p->ct.kds_max, cs, b->device);
    if (st != GW_OK) break;
    const std::array<int, 4> key{cp.groups, cp.n_hh, cs.groups, cs.n_hh};
    size_t c = 0;
    while (c < keys.size() && keys[c] != key) ++c;
    if (c == keys.size()) {
      keys.push_back(key);
      b->cls.emplace_back();
    }
    BatchClass& k = b->cls[c];
    k.sys.push_back(i);
    k.ncols_p = std::max(k.ncols_p, p->ct.np_max);
    k.kd_p = std::max(k.kd_p, p->ct.kd_max);
    k.ncols_s = std::max(k.ncols_s, p->ct.nj_max);
    k.kd_s = std::max(k.kd_s, p->ct.kds_max);
  }
  for (BatchClass& k : b->cls) {
    if (st == GW_OK) st = gw::contract_config(false, k.ncols_p, k.kd_p, k.cfgP, b->device);
    if (st == GW_OK) st = gw::contract_config(true, k.ncols_s, k.kd_s, k.cfgS, b->device);
    if (st == GW_OK) st = batch_upload_units(b, k, false, 0);
    if (st == GW_OK) st = batch_upload_units(b, k, true, 0);
  }
  if (st == GW_OK) st = upload(&b->d_counter, nullptr, 16);
  if (st == GW_OK) st = upload(&b->d_status, nullptr, 16);
  if (st == GW_OK && cudaMemset(b->d_status, 0, 16) != cudaSuccess) st = GW_ERR_CUDA;
  if (st == GW_OK && gw::uploads_landed() != cudaSuccess) st = GW_ERR_CUDA;
  if (st != GW_OK) {
    gw_batch_destroy(b);
    return st;
  }
  *out = b;
  return GW_OK;
}

gw_status gw_batch_destroy(gw_batch_t b) {
  if (!b) return GW_OK;
  {
    DeviceGuard guard(b->device);
    for (BatchClass& k : b->cls) {
      cudaFree(k.d_unitsP);
      cudaFree(k.d_unitsS);
    }
    cudaFree(b->d_counter);
    cudaFree(b->d_status);
  }
  delete b;
  return GW_OK;
}

gw_status gw_batch_query(gw_batch_t b, gw_batch_info* info) {
  if (!b || !info) return GW_ERR_ARG;
  info->n_plans = (int)b->plans.size();
  info->n_units_p = info->n_units_s = 0;
  for (const BatchClass& k : b->cls) {
    info->n_units_p += k.nP;
    info->n_units_s += k.nS;
  }
  const BatchClass& k0 = b->cls[0];
  info->groups_p = k0.cfgP.groups;
  info->groups_s = k0.cfgS.groups;
  info->kc_p = k0.cfgP.kc;
  info->kc_s = k0.cfgS.kc;
  info->order_p = k0.orderP;
  info->order_s = k0.orderS;
  info->tuned = b->tuned ? 1 : 0;
  info->n_classes = (int)b->cls.size();
  return GW_OK;
}

gw_status gw_batch_polarizability_tau(gw_batch_t b, const void* const* G_R, void* const* P_R, void* stream) {
  if (!b || !G_R || !P_R) return GW_ERR_ARG;
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (!G_R[i] || !P_R[i]) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(b->device);
  gw::ActiveTimer timing(&b->plans[0]->timer);
  const gw::CBatch cb = batch_systems(b, G_R, nullptr, P_R);
  for (const BatchClass& k : b->cls) {
    const gw_status st = gw::contract_launch(false, k.cfgP, cb, k.d_unitsP, k.nP, b->d_counter, b->d_status, S(stream));
    if (st != GW_OK) return st;
  }
  return GW_OK;
}

gw_status gw_batch_self_energy_tau(gw_batch_t b, const void* const* G_R, const void* const* Wt_R,
                                   void* const* Sig_R, void* stream) {
  if (!b || !G_R || !Wt_R || !Sig_R) return GW_ERR_ARG;
  for (size_t i = 0; i < b->plans.size(); ++i)
    if (!G_R[i] || !Wt_R[i] || !Sig_R[i]) { set_last_error("bad argument"); return GW_ERR_ARG; }
  DeviceGuard guard(b->device);
  gw::ActiveTimer timing(&b->plans[0]->timer);
  const gw::CBatch cb = batch_systems(b, G_R, Wt_R, Sig_R);
  for (const BatchClass& k : b->cls) {
    const gw_status st = gw::contract_launch(true, k.cfgS, cb, k.d_unitsS, k.nS, b->d_counter, b->d_status, S(stream));
    if (st != GW_OK) return st;
  }
  return GW_OK;
}

gw_status gw_batch_sync(gw_batch_t b, void* stream) {
  if (!b) return GW_ERR_ARG;
  DeviceGuard guard(b->device);
  GW_CUDA(cudaStreamSynchronize(S(stream)));
  int flag = 0;
  GW_CUDA(cudaMemcpyAsync(&flag, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
  GW_CUDA(cudaStreamSynchronize(S(stream)));
  if (flag) {
    GW_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int), S(stream)));
    GW_CUDA(cudaStreamSynchronize(S(stream)));
    set_last_error("a tensor-core wait gave up (bounded wait)");
    return GW_ERR_TIMEOUT;
  }
  return GW_OK;
}

gw_status gw_batch_tune(gw_batch_t b, const void* const* G_R, void* const* P_R, const void* const* Wt_R,
                        void* const* Sig_R, int reps, void* stream) {
  if (!b || !G_R || !P_R || !Wt_R || !Sig_R || reps < 1) return GW_ERR_ARG;
  DeviceGuard guard(b->device);
  cudaStream_t st = S(stream);
  // the unit tables are rewritten between candidates: nothing on the stream may read them
  GW_CUDA(cudaStreamSynchronize(st));
  cudaEvent_t e0, e1;
  GW_CUDA(cudaEventCreate(&e0));
  GW_CUDA(cudaEventCreate(&e1));
  gw_status result = GW_OK;
  for (int sig = 0; sig < 2 && result == GW_OK; ++sig) {
    const bool sigma = sig == 1;
    const gw::CBatch cb = sigma ? batch_systems(b, G_R, Wt_R, Sig_R) : batch_systems(b, G_R, nullptr, P_R);
    // each class on its own: its launch is timed alone with every candidate
    for (size_t ci = 0; ci < b->cls.size() && result == GW_OK; ++ci) {
      BatchClass& k = b->cls[ci];
      const int ncols = sigma ? k.ncols_s : k.ncols_p, kd = sigma ? k.kd_s : k.kd_p;
      float best = 1e30f;
      gw::CConfig best_cfg = sigma ? k.cfgS : k.cfgP;
      int best_order = 0;
      for (int order = 0; order < 2 && result == GW_OK; ++order) {
        if ((result = batch_upload_units(b, k, sigma, order)) != GW_OK) break;
        for (int groups = 1; groups <= 2; ++groups) {
          // the longest chunk that fits, and half of it
          for (int half = 0; half < 2; ++half) {
            gw::CConfig c;
            if (gw::contract_config(sigma, ncols, kd, c, b->device, groups) != GW_OK || c.groups != groups) continue;
            if (half) {
              const int kc2 = (c.kc / 2) & ~15;
              gw::CConfig c2;
              if (kc2 < 16 || gw::contract_config(sigma, ncols, kd, c2, b->device, groups, kc2) != GW_OK ||
                  c2.kc == c.kc)
                continue;
              c = c2;
            }
            const gw::CUnit* du = sigma ? k.d_unitsS : k.d_unitsP;
            const int nu = sigma ? k.nS : k.nP;
            if ((result = gw::contract_launch(sigma, c, cb, du, nu, b->d_counter, b->d_status, st)) != GW_OK) break;
            GW_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < reps && result == GW_OK; ++r)
              result = gw::contract_launch(sigma, c, cb, du, nu, b->d_counter, b->d_status, st);
            GW_CUDA(cudaEventRecord(e1, st));
            GW_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            GW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (result == GW_OK && ms < best) {
              best = ms;
              best_cfg = c;
              best_order = order;
            }
          }
        }
      }
      if (result != GW_OK) break;
      (sigma ? k.cfgS : k.cfgP) = best_cfg;
      // the chosen configuration's shared-memory opt-in (raised for every candidate already)
      result = batch_upload_units(b, k, sigma, best_order);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result == GW_OK) {
    b->tuned = true;
    result = gw_batch_sync(b, stream);
  }
  return result;
}
