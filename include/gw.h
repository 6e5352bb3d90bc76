/*
 * gw.h -- C ABI of the real-space / imaginary-time GW sweep (arXiv:1911.05633).
 *
 * One GB300 (sm_103a), one process.  Every data buffer is owned by the caller
 * and is a DEVICE pointer unless stated otherwise; the plan owns its tables
 * (pair list, lattice phases, product-basis coefficients, transform matrices)
 * and the scratch of the W solve.  Complex numbers are interleaved
 * (re, im) doubles, i.e. C99 double complex / numpy complex128.  All compute
 * calls are asynchronous on the given stream (a cudaStream_t passed as
 * void*; NULL is the legacy default stream).  Errors are returned by value;
 * nothing crosses the ABI by exception.  A call that returns an error has
 * launched nothing.
 *
 * Notation: atoms a, b; orbitals L (n_a per atom), product-basis functions K
 * (K_a per atom); a pair entry e = (a, b, R) is one atom pair and one lattice
 * class R kept by the distance cutoff; N_k k-points; N_tau imaginary-time
 * nodes; N_omega fermionic and N_nu bosonic sampled Matsubara frequencies.
 *
 * Ragged "entry" layouts.  A buffer with n_slices slices per entry holds the
 * entries back to back, entry e as a row-major [n_slices][rows_e][cols_e]
 * block starting at element n_slices * off[e], where off[] is the prefix sum
 * of rows_e * cols_e returned by gw_plan_offsets():
 *   GW_BLOCK_ORB: rows_e = n_a, cols_e = n_b   (G, Sigma)
 *   GW_BLOCK_PB : rows_e = K_a(e), cols_e = K_b(e)   (P, W~, v)
 * K_a(e) is the product-basis size of atom a for entry e at the entry's level of
 * Sec. 2, Fig. 2: n_prod of its species when both arguments are in one sphere
 * (the onsite entry, sphere A), n_prod_near for two spheres within the radius r_b
 * of sphere B, n_prod_far beyond it; an entry keeps the FIRST K_a(e) product
 * functions of each atom.  gw_plan_entry_dims() returns the
 * per-entry shapes.
 * Dense k-space buffers are [N_k][n_slices][N][N] with N = total orbitals
 * (ORB) or total product functions (PB), atoms in order.
 */
#ifndef GW_H
#define GW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_plan_s* gw_plan_t;

typedef enum {
  GW_OK = 0,
  GW_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad grid) */
  GW_ERR_OOM = 2,            /* device or host allocation failed */
  GW_ERR_CUDA = 3,           /* a CUDA call failed (message in gw_last_error()) */
  GW_ERR_KMESH_ALIAS = 4,    /* strict mode: the k-mesh is below the rule of Sec. 2 */
  GW_ERR_NOT_HERMITIAN = 5,  /* reserved */
  GW_ERR_SINGULAR = 6,       /* a zero pivot in the W solve (reported by gw_sync) */
  GW_ERR_TIMEOUT = 7,        /* reserved (bounded device waits) */
  GW_ERR_NAN = 8,            /* reserved */
  GW_ERR_NO_DEVICE = 9,      /* compute call on a plan built with host_only */
  GW_ERR_UNSUPPORTED = 10    /* size outside the compiled limits (see gw_plan_create) */
} gw_status;

/* GW_MIXED: the P and Sigma contractions in reduced precision with FP32
 * accumulation (everything else stays FP64); target 1e-6 relative error. */
typedef enum { GW_FP64 = 0, GW_MIXED = 1 } gw_precision;
typedef enum { GW_FERMION = 0, GW_BOSON = 1 } gw_statistics;
typedef enum { GW_TAU_TO_IW = 0, GW_IW_TO_TAU = 1 } gw_direction;
typedef enum { GW_BLOCK_ORB = 0, GW_BLOCK_PB = 1 } gw_block;

/* Crystal: lattice rows a_1, a_2, a_3 in bohr; atoms in fractional coordinates. */
typedef struct {
  double lattice[9];
  int n_atoms;
  const double* frac;     /* host [n_atoms][3] */
  const int* species;     /* host [n_atoms], 0 <= species < n_species */
} gw_cell;

/* Per-species orbital and product basis.  C[s] is the one-centre coefficient
 * tensor <M_K | phi_L phi_L''> of Eq. P_MM, host [n_prod][n_orb][n_orb], real. */
typedef struct {
  int n_species;
  const int* n_orb;       /* host [n_species], 1..16 */
  const int* n_prod;      /* host [n_species], 1..128 */
  const double* const* C; /* host [n_species] pointers */
  const int* n_prod_far;  /* host [n_species], 1..n_prod, or NULL: product functions kept for
                             pair entries beyond gw_options.r_b (Sec. 2, the pairs between
                             spheres B and C); NULL keeps n_prod for every entry */
  const int* n_prod_near; /* host [n_species], n_prod_far..n_prod, or NULL (n_prod): product
                             functions kept for the entries of two distinct spheres within r_b
                             (sphere B); the onsite entries (one sphere, sphere A) keep n_prod.
                             Read only together with n_prod_far and r_b > 0 */
} gw_basis;

/* Imaginary-time nodes and sampled Matsubara indices (Appendix A grid).
 * tau: ascending, tau[0] = 0 (read as 0+), tau[n_tau-1] = beta (read as beta-),
 * mirror-symmetric beta - tau_i = tau_{n_tau-1-i} to 1e-12 beta.
 * omega_idx: fermionic n, w_n = (2n+1) pi / beta; nu_idx: bosonic m, v_m = 2 m pi / beta.
 * n_omega >= n_tau and n_nu >= n_tau (least-squares inverse transforms). */
typedef struct {
  double beta;
  int n_tau;   const double* tau;
  int n_omega; const int* omega_idx;
  int n_nu;    const int* nu_idx;
} gw_grid;

typedef struct {
  int spin;               /* spin degeneracy s of Eq. P_MM (sum over alpha): 1 or 2 */
  int strict_kmesh;       /* 1: reject a k-mesh below the rule of Sec. 2 */
  int host_only;          /* 1: build host tables only; compute calls fail with GW_ERR_NO_DEVICE */
  int device;             /* CUDA device ordinal used by the plan */
  size_t workspace_bytes; /* cap on the W-solve scratch (0: 24 GiB for the tensor-core and the block
                             inverse, 4 GiB otherwise) */
  int no_symmetry;        /* 1: never use the frequency / momentum symmetries in the W solve */
  int w_solver;           /* 0: automatic (tensor-core inverse when N_PB is 128, 256 or 384;
                             block Gauss-Jordan over pivot blocks of 384, 256 or 128 that the
                             tensor-core inverse takes when N_PB is a larger multiple of 128),
                             1: FP64 Gauss-Jordan inverse always */
  int fp64_products;      /* 0 automatic: FP64-accurate digit products on the tensor cores for
                             the W~ C^b stage of the GW_FP64 Sigma (every K <= 384), the Y C^b
                             stage of the GW_FP64 P (every n^2 <= 384) and the structured
                             bosonic transforms (reduction <= 384);
                             1: FP64 arithmetic only */
  double r_b;             /* radius of sphere B in bohr (Sec. 2, Fig. 2): an entry whose
                             minimum-image distance |R + t_b - t_a| exceeds r_b by more than
                             1e-9 bohr^2 in the square keeps n_prod_far product functions per
                             atom, an entry of two spheres within it n_prod_near, an onsite
                             entry n_prod; <= 0 (or n_prod_far NULL): every entry keeps n_prod */
  int defer_scratch;      /* 1: allocate the W-solve scratch (gw_screened_W_iw) and the FP64
                             digit-product scratch (GW_FP64 gw_polarizability_tau and
                             gw_self_energy_tau) at the first call that needs them instead of at
                             plan creation, so that plans used for the mixed contractions alone
                             hold none of it; such a first call allocates device memory and so
                             must not be inside a stream capture.  0: allocate at creation */
} gw_options;

typedef struct {
  int n_atoms, n_entries, n_k, n_tau, n_omega, n_nu;
  int n_orb_total, n_pb_total;
  int kmesh[3];
  int kmesh_required[3];      /* the rule of Sec. 2 for the given cutoff (0 if cutoff <= 0) */
  int c_symmetric;            /* every C[s] symmetric in (L, L'') */
  int64_t len_orb;            /* sum over entries of n_a n_b (one slice) */
  int64_t len_pb;             /* sum over entries of K_a K_b (one slice) */
  size_t workspace_bytes;     /* device scratch the plan holds */
  int nu_chunk;               /* bosonic frequencies per W-solve pass */
  double cond_fermion;        /* 2-norm condition numbers of the forward matrices */
  double cond_boson;
  int w_symmetric;            /* the W solve runs on nu >= 0 and half of the q mesh (see gw_screened_W_iw) */
  int n_q_solved;             /* momenta solved per frequency */
  int w_tensor;               /* inverses by FP32 Gauss-Jordan + two tensor-core refinements */
  int sigma_tensor;           /* GW_FP64 Sigma: stage W~ C^b by FP64-accurate tensor-core products */
  int p_tensor;               /* GW_FP64 P: stage Y C^b by FP64-accurate tensor-core products (device plans) */
  int transform_tensor;       /* bit 0: GW_IN_REAL bosonic i nu -> tau, bit 1: GW_IN_MIRROR bosonic
                                 tau -> i nu of the product-basis layout by FP64-accurate
                                 tensor-core products (device plans) */
  int n_entries_far;          /* entries with the reduced product basis (beyond r_b) */
  int n_entries_near;         /* entries of two distinct spheres within r_b that keep n_prod_near
                                 (0 when n_prod_near is NULL) */
  int mixed_queue;            /* GW_MIXED contractions as persistent tensor-core kernels over a queue
                                 of (entry, tau) units: bit 0 P, bit 1 Sigma (device plans) */
  int w_block;                /* pivot block size of the block Gauss-Jordan W inverse (0: not used) */
} gw_plan_info;

/* ---- plan ------------------------------------------------------------------ */

/* Build the plan: the pair list of Sec. 2 (every ordered atom pair (a, b) and
 * lattice class R modulo the k-mesh supercell whose minimum-image distance
 * |R + t_b - t_a| is <= cutoff; cutoff <= 0 keeps every class; ties go to the
 * lexicographically smallest R), the phases e^{ik.R}, and the tau <-> i omega
 * matrices of Appendix A (exact Fourier integrals of the polynomial through
 * the tau nodes and their least-squares inverses).  Host inputs are copied.
 * Returns GW_ERR_ARG on invalid input, GW_ERR_KMESH_ALIAS in strict mode,
 * GW_ERR_UNSUPPORTED beyond n_orb <= 16, n_prod <= 128, n_tau <= 128. */
gw_status gw_plan_create(const gw_cell* cell, const gw_basis* basis, const int kmesh[3],
                         const gw_grid* grid, double cutoff, const gw_options* opt,
                         gw_plan_t* out);
gw_status gw_plan_destroy(gw_plan_t plan);
gw_status gw_plan_query(gw_plan_t plan, gw_plan_info* info);

/* Host copy of the entry list, [n_entries][8] int64 rows (a, b, c1, c2, c3, R1, R2, R3):
 * class c in [0, N_i) and its minimum-image representative R.  Sorted by (a, b, c). */
gw_status gw_plan_entries(gw_plan_t plan, int64_t* rows);

/* Host copy of the per-entry block offsets, [n_entries + 1] int64 (see the layout note). */
gw_status gw_plan_offsets(gw_plan_t plan, gw_block kind, int64_t* off);

/* Host copy of the per-entry block shapes, rows[e] x cols[e] ([n_entries] int32 each):
 * (n_a, n_b) for GW_BLOCK_ORB, (K_a(e), K_b(e)) for GW_BLOCK_PB (see the layout note). */
gw_status gw_plan_entry_dims(gw_plan_t plan, gw_block kind, int32_t* rows, int32_t* cols);

/* Host copy of a transform matrix, complex [n_out][n_in] interleaved doubles:
 * (FERMION, TAU_TO_IW) n_omega x n_tau, (FERMION, IW_TO_TAU) n_tau x n_omega,
 * (BOSON, TAU_TO_IW) n_nu x n_tau, (BOSON, IW_TO_TAU) n_tau x n_nu. */
gw_status gw_plan_transform_matrix(gw_plan_t plan, gw_statistics st, gw_direction dir, double* out);

/* ---- the sweep (Sec. 2: "one follows Eqs. P_old - G_1" in real space) ---------- */

/* F_ab(R) = (1/N_k) sum_k e^{-i k.R} F_ab(k) for the kept entries (Sec. 2, R <-> k
 * transforms over the pair list).  F_k dense [N_k][n_slices][N][N] -> F_R entry layout. */
gw_status gw_fourier_k_to_R(gw_plan_t plan, gw_block kind, int n_slices,
                            const void* F_k, void* F_R, void* stream);

/* G(R, tau) from G(k, tau): gw_fourier_k_to_R with GW_BLOCK_ORB and n_slices = N_tau. */
gw_status gw_green_k_to_R(gw_plan_t plan, const void* G_k, void* G_R, void* stream);

/* P_{aK,bK'}(R, tau_i) = -s sum C^a_{K;L L''} G_{aL,bL'}(R, tau_i)
 *      conj(G_{aL'',bL'''}(R, beta - tau_i)) C^b_{K';L' L'''}
 * (Eq. P_MM with the sign and tau pairing of Eq. P_II; conj from the Hermiticity
 * of G).  G_R: ORB layout, N_tau slices.  P_R: PB layout, N_tau slices. */
gw_status gw_polarizability_tau(gw_plan_t plan, const void* G_R, void* P_R,
                                gw_precision prec, void* stream);

/* out[e][m] = sum_i T[m][i] in[e][i] per entry and block element, with T the
 * matrix named by (st, dir) (Appendix A grid).  Layout of `kind` on both sides;
 * slices: N_tau on the tau side, N_omega (FERMION) or N_nu (BOSON) on the other. */
gw_status gw_transform_tau_iw(gw_plan_t plan, gw_statistics st, gw_direction dir,
                              gw_block kind, const void* in, void* out, void* stream);

/* Input structure for gw_transform_tau_iw_ex.
 * GW_IN_MIRROR: in(tau_{N-1-i}) = conj(in(tau_i)) for every block element, i.e. F(beta - tau)
 *   = F(tau)* on the mirror-symmetric grid (P from gw_polarizability_tau when the plan
 *   reports c_symmetric).  Bosonic tau -> i nu only: the output is real (F(i nu) =
 *   sum over mirror pairs of 2 Re(T F)), so only the nodes i < ceil(N_tau / 2) are read,
 *   the imaginary parts are written as 0, and it takes a quarter of the general flops.
 * GW_IN_REAL: the imaginary parts of `in` are zero (W~(R, i nu) from gw_screened_W_iw when
 *   the plan reports w_symmetric); they are not read, and it takes half the flops.
 * GW_OUT_NONNEG (with GW_IN_MIRROR): only the output slices of the sampled frequencies
 *   nu >= 0 are written; the others keep what they held.  With the mirror-symmetric
 *   frequency set of a w_symmetric plan these are all gw_screened_W_iw reads (it fills the
 *   negative ones from the mirror entries, P_ab(R, -i nu) = P_ba(-R, i nu)^T); half the
 *   columns and half the bytes written. */
enum { GW_IN_GENERAL = 0, GW_IN_MIRROR = 1, GW_IN_REAL = 2, GW_OUT_NONNEG = 4 };

/* gw_transform_tau_iw for inputs of a known structure (the symmetries of the tau grid
 * and of Eq. P_MM with symmetric product coefficients).  GW_ERR_ARG for an unknown
 * `structure`; GW_ERR_UNSUPPORTED for GW_IN_MIRROR with fermionic statistics or the
 * i omega -> tau direction.  The input is trusted to have the stated structure. */
gw_status gw_transform_tau_iw_ex(gw_plan_t plan, gw_statistics st, gw_direction dir,
                                 gw_block kind, int structure, const void* in, void* out,
                                 void* stream);

/* W~(R, i nu) on the kept entries from P(R, i nu) (Eq. W_1 with W = v + W~):
 * P(q) = sum_{kept R} e^{iq.R} P(R); W(q) = (I - v(q) P(q))^{-1} v(q), computed as
 * (v(q)^{-1} - P(q))^{-1}, each inverse either by FP64 Gauss-Jordan with partial
 * pivoting or (w_tensor) by FP32 Gauss-Jordan refined twice with a residual
 * I - A X evaluated to FP64 accuracy on the tensor cores (exact BF16 slices), or
 * (w_block, N_PB beyond 384) by Gauss-Jordan over pivot blocks of w_block rows without
 * pivoting across blocks, each pivot block inverted as in w_tensor and every block
 * product (w_block terms) taken to FP64 accuracy from exact BF16 slices: it needs the
 * leading blocks well conditioned, as they are for v(q) and v(q)^{-1} - P(q, i nu)
 * (Hermitian positive definite when P comes from a Hermitian G), and reports
 * GW_ERR_SINGULAR from gw_sync for a singular pivot block;
 * W~(R) = (1/N_k) sum_q e^{-iq.R} (W(q) - v(q)).
 * P_R_iw, Wt_R_iw: PB layout, N_nu slices.  v_q: dense [N_k][N_PB][N_PB].
 * When the plan reports w_symmetric (C symmetric in (L, L''), a symmetric bosonic
 * set, option no_symmetry unset) the solve runs on nu >= 0 and on one momentum of
 * each pair (q, -q) only, and the rest follows from the symmetries that P obtained
 * from a Hermitian G(tau) has: P(R, i nu) real and P_ab(R, -i nu) = P_ba(-R, i nu)^T,
 * with v(-q) = v(q)^*.  Inputs without these symmetries need no_symmetry.
 * Uses the plan's scratch; calls on one plan must not overlap on the GPU. */
gw_status gw_screened_W_iw(gw_plan_t plan, const void* P_R_iw, const void* v_q,
                           void* Wt_R_iw, void* stream);

/* Sigma_{aL,bL'}(R, tau_i) = -sum C^a_{K;L L''} G_{aL'',bL'''}(R, tau_i)
 *      W~_{aK,bK'}(R, tau_i) C^b_{K';L' L'''}                     (Eq. S_MM)
 * and, when v_R and Sigx_R are both non-NULL, the static exchange of the same
 * contraction with W~ -> v and G(tau) -> -G(beta-) (the rule after Eq. P_II):
 *   Sigx = + sum C^a G(R, beta-) v(R) C^b
 * (in the precision `prec` asks for, like the dynamic part).
 * G_R: ORB, N_tau slices; Wt_R: PB, N_tau slices; v_R: PB, 1 slice;
 * Sig_R: ORB, N_tau slices; Sigx_R: ORB, 1 slice. */
gw_status gw_self_energy_tau(gw_plan_t plan, const void* G_R, const void* Wt_R,
                             const void* v_R, void* Sig_R, void* Sigx_R,
                             gw_precision prec, void* stream);

/* F_ab(k) = sum_{kept R} e^{+i k.R} F_ab(R) (Sec. 2), entry layout -> dense
 * [N_k][n_slices][N][N]; blocks of atom pairs without entries are zero. */
gw_status gw_fourier_R_to_k(gw_plan_t plan, gw_block kind, int n_slices,
                            const void* F_R, void* F_k, void* stream);

/* Allocation-free variant of gw_screened_W_iw (no counterpart in the paper).
 * For callers that cannot allocate device memory once they run -- for example a code
 * that hands all device memory to its own pool at start-up, or one that runs under a
 * memory manager that refuses new allocations: the scratch of this call is a fixed
 * 32 MiB array in the library's device image (held on every GPU that loads the
 * library until the process exits), not the plan's workspace.  Same inputs, output
 * and arithmetic as gw_screened_W_iw with the FP64 Gauss-Jordan inverse.
 * Limit: 2 N_PB^2 complex values must fit (N_PB <= 1024); a larger plan gets
 * GW_ERR_UNSUPPORTED and nothing is launched.  The call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress): make that first call
 * before any stream capture.  Every call shares the array, which keeps the last
 * call's contents; calls that overlap on the GPU (other streams, threads or plans on
 * the same device) race and give wrong results. */
gw_status gw_screened_W_iw_noalloc(gw_plan_t plan, const void* P_R_iw, const void* v_q, void* Wt_R_iw,
                                   void* stream);

/* Per-kernel device timing (an instrumentation aid; no counterpart in the paper).
 * gw_timing_enable(plan, 1) makes every later kernel launch of this plan's entry points
 * record a CUDA event before and after it on the launching stream (off by default;
 * keep it off while a stream is being captured into a graph).  gw_timing_read waits for
 * the recorded events, adds their elapsed times per kernel name and reports entry
 * `index` (GW_ERR_ARG past the last one): `*name` stays valid until the next
 * gw_timing_reset or gw_plan_destroy, `*total_ms` is the summed device time and
 * `*launches` the number of launches.  gw_timing_reset clears the totals. */
gw_status gw_timing_enable(gw_plan_t plan, int enable);
gw_status gw_timing_read(gw_plan_t plan, int index, const char** name, double* total_ms, long long* launches);
gw_status gw_timing_reset(gw_plan_t plan);

/* Wait for the stream and report any deferred device-side error of the plan. */
gw_status gw_sync(gw_plan_t plan, void* stream);

const char* gw_status_string(gw_status s);
/* Text of the last error on this thread (empty if none). */
const char* gw_last_error(void);

/* ---- batches of systems of uneven sizes in one launch -------------------------- */

/* A batch of up to GW_BATCH_MAX plans (device plans on one device, each within the
 * contraction kernels' limits: n_orb <= 16, n_prod <= 128) whose GW_MIXED P and Sigma
 * contractions (Eqs. P_MM and S_MM) run as ONE persistent launch each: a queue of
 * (system, pair entry, tau node) units drained by one resident block per SM, so that
 * systems with different atom counts, pair lists and basis sizes share the GPU without
 * one launch per system.  Plans whose contractions take the same launch shape (thread
 * groups, hi x hi accumulators) form a class; each class has its own unit queue and
 * launch configuration, and a batch call is one launch per class.  The plans must
 * outlive the batch.  Results are those of gw_polarizability_tau and
 * gw_self_energy_tau (without exchange) with GW_MIXED on each plan alone. */
#define GW_BATCH_MAX 24
typedef struct gw_batch_s* gw_batch_t;

typedef struct {
  int n_plans;
  long long n_units_p, n_units_s;  /* queue lengths */
  int groups_p, groups_s;          /* thread groups per block */
  int kc_p, kc_s;                  /* reduction chunk (product-basis or orbital-pair columns) */
  int order_p, order_s;            /* unit order: 0 by shape class, 1 heaviest first */
  int tuned;                       /* 1 after gw_batch_tune */
  int n_classes;                   /* launch classes (launches per contraction); the groups, kc and
                                      order fields above are the first class's */
} gw_batch_info;

/* GW_ERR_ARG for n_plans outside [1, GW_BATCH_MAX], plans on different devices or host-only
 * plans; GW_ERR_UNSUPPORTED for a plan outside the kernels' limits. */
gw_status gw_batch_create(const gw_plan_t* plans, int n_plans, gw_batch_t* out);
gw_status gw_batch_destroy(gw_batch_t b);
gw_status gw_batch_query(gw_batch_t b, gw_batch_info* info);

/* P of every plan of the batch in one launch.  G_R, P_R: HOST arrays of n_plans DEVICE
 * pointers, each in the layout of gw_polarizability_tau for its plan.  Asynchronous;
 * capturable in a CUDA graph (no host-to-device copy, no allocation). */
gw_status gw_batch_polarizability_tau(gw_batch_t b, const void* const* G_R, void* const* P_R, void* stream);

/* The dynamic Sigma of every plan in one launch (layouts of gw_self_energy_tau). */
gw_status gw_batch_self_energy_tau(gw_batch_t b, const void* const* G_R, const void* const* Wt_R,
                                   void* const* Sig_R, void* stream);

/* Autotuner: times each candidate launch configuration (thread groups per block, reduction
 * chunk, unit order) of both contractions on these buffers with CUDA events on `stream`,
 * `reps` launches per candidate, and keeps the fastest.  Overwrites P_R and Sig_R;
 * synchronous.  Call before capturing the batch's launches in a graph. */
gw_status gw_batch_tune(gw_batch_t b, const void* const* G_R, void* const* P_R, const void* const* Wt_R,
                        void* const* Sig_R, int reps, void* stream);

/* Wait for the stream and report a deferred device error of the batch's launches. */
gw_status gw_batch_sync(gw_batch_t b, void* stream);

/* ---- Eq. G_1: the Dyson equation and the chemical potential ------------------- */

/* G(k, tau) from Eq. G_1, G = G0 + G0 Sigma G with G0 = (i w + mu - H)^{-1} the Green
 * function of the fixed (Hartree) Hamiltonian: per momentum k and sampled fermionic
 * frequency w_n (the plan's omega indices), the FP64 inverse
 *   G(k, i w_n) = [(i w_n + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, i w_n)]^{-1},
 * then G(k, tau_i) = sum_n T[i][n] (G - 1/(i w_n) - M1/(i w_n)^2) - I/2 + M1 (2 tau_i - beta)/4
 * with T the inverse fermionic transform of Appendix A (gw_plan_transform_matrix) and
 * M1 = H + Sigma_x - mu: the two leading terms of G at large frequency are taken out
 * before the transform and added back as their exact tau functions.
 * H_k, Sigx_k: device [N_k][N][N] (N = total orbitals; Sigx_k NULL reads as zero);
 * Sig_k_iw: device [N_k][n_omega][N][N] (the layout gw_fourier_R_to_k writes) or NULL;
 * G_k_tau: device [N_k][n_tau][N][N], the layout gw_green_k_to_R reads.  The plan
 * allocates N_k n_omega N^2 complex values of scratch on the first call.  A zero pivot
 * is reported by gw_sync (GW_ERR_SINGULAR). */
gw_status gw_dyson_green_tau(gw_plan_t plan, const void* H_k, const void* Sigx_k, const void* Sig_k_iw, double mu,
                             void* G_k_tau, void* stream);

/* The chemical potential mu in [mu_lo, mu_hi] at which the electrons per cell,
 * N(mu) = s (1/N_k) sum_k Re Tr[-G(k, beta-)] with G from gw_dyson_green_tau at tau = beta-,
 * equal n_electrons: bisection until the bracket is narrower than tol (at most 200
 * steps; N grows with mu).  Each step is one Dyson solve on the device; the call is
 * synchronous on `stream`.  Writes mu and, if n_out is not NULL, N(mu).  Returns
 * GW_ERR_ARG for mu_lo >= mu_hi or tol <= 0, GW_ERR_SINGULAR for a zero pivot. */
gw_status gw_chemical_potential(gw_plan_t plan, const void* H_k, const void* Sigx_k, const void* Sig_k_iw,
                                double n_electrons, double mu_lo, double mu_hi, double tol, double* mu_out,
                                double* n_out, void* stream);

/* Linearised quasiparticle energies (the procedure behind the paper's band plots: the
 * value and the frequency derivative of Sigma at zero frequency).  Sigma_c(i w) ~ S0 + i w S1
 * through the sampled frequencies n = 0 and n = 1 (w_0 = pi/beta, w_1 = 3 pi/beta); with
 * Hermitian parts (h) and A = (I - S1^h)^{1/2}, E(k) are the eigenvalues of
 * A^{-1} (H(k) + Sigma_x^h(k) + S0^h - mu) A^{-1}, plus mu, in ascending order.
 * H_k, Sigx_k, Sig_k_iw as for gw_dyson_green_tau (Sigx_k, Sig_k_iw may be NULL);
 * E_k: device double [N_k][N].  FP64 throughout (Hermitian eigenproblems by cyclic
 * Jacobi, one block per momentum).  GW_ERR_ARG if the sampled set lacks n = 0 or 1,
 * GW_ERR_UNSUPPORTED for more than 80 orbitals in total. */
gw_status gw_qp_energies(gw_plan_t plan, const void* H_k, const void* Sigx_k, const void* Sig_k_iw, double mu,
                         void* E_k, void* stream);

/* Eq. sf_9: the continued fraction through Sigma on the stored Matsubara grid, per
 * element, continued to the real frequencies w_r + i delta (w measured from mu):
 *   Sigma(w) = a_0 / (1 + a_1 (w - z_0) / (1 + ... a_M (w - z_{M-1}) / 1)),
 * with z_i = i w_i the non-negative sampled fermionic frequencies of the plan (ascending,
 * at most 64) and a_p from the recursion of the fraction's reference (Vidberg and Serene).
 * Sig_k_iw: device [N_k][n_omega][N][N]; w_real: HOST [n_real]; Sig_k_w: device
 * [N_k][n_real][N][N].  The continuation from the imaginary axis is ill-conditioned by
 * nature: results near poles close to the real axis carry rounding amplified accordingly.
 * Synchronous with respect to the copy of w_real; the kernel is asynchronous. */
gw_status gw_continue_sigma(gw_plan_t plan, const void* Sig_k_iw, int n_real, const double* w_real, double delta,
                            void* Sig_k_w, void* stream);

/* Eqs. sf_1 and sf_7: the k-resolved spectral function A(k, w) = -(1/pi) Im Tr G^R(k, w) with
 *   G^R = [(w + i delta + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, w)]^{-1}
 * (Eq. sf_7 in the band states of H + Sigma_x; the trace is basis independent), FP64
 * inverses on the device.  Sig_k_w: device [N_k][n_real][N][N], e.g. from
 * gw_continue_sigma with the same w_real and delta, or NULL; H_k, Sigx_k as for
 * gw_dyson_green_tau; w_real: HOST [n_real] (from mu); delta > 0; A_kw: device double
 * [N_k][n_real].  Allocates N_k n_real N^2 complex values of scratch on first use (kept). */
gw_status gw_spectral_function(gw_plan_t plan, const void* H_k, const void* Sigx_k, const void* Sig_k_w, int n_real,
                               const double* w_real, double delta, double mu, void* A_kw, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GW_H */
