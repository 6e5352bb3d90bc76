"""FP64 CPU oracle for the real-space / imaginary-time GW sweep (arXiv:1911.05633).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library and its
Python binding never call it, and it shares no code with them: its inputs come
from the seeded generator ``synth`` only.

Plain NumPy / SciPy in float64 (complex128), written for clarity, not speed.
Every function follows one statement of the paper, cited in its docstring:

* Sec. 2, "basic approximation" (Fig. 1): two-point functions F^R_{rr'} are kept
  only for |R + r - r'| <= R_max, and the k-mesh must be at least the number of
  cells the R_max sphere encloses or crosses.  -> ``kmesh_rule``, ``pair_list``
* Sec. 2, the three product-basis levels (Fig. 2): both arguments in one sphere
  (A) keep the whole basis, pairs within the radius of sphere B a smaller one, pairs
  beyond it the smallest (the first n_prod_near / n_prod_far functions of each atom
  here) -> ``entry_tier``, ``entry_far``, ``entry_pb_dims``; every product-basis
  function below takes its block shapes from its inputs
* Sec. 2, transformations between R and k spaces over the kept pairs
  -> ``fourier_k_to_R``, ``fourier_R_to_k``
* Eq. P_MM with the sign and the tau pairing of Eq. P_II -> ``polarizability_R``
  and the momentum route of Eq. P_old -> ``polarizability_q_kspace``
* Eq. W_1 (W = V + V P W, with W~ = W - V) -> ``screened_W``
* Eq. S_MM (dynamic part) and the exchange rule stated after Eq. P_II
  (W~(tau) -> V, G(tau) -> -G(beta)) -> ``self_energy_R``, ``exchange_R``,
  and the momentum route of Eq. S_old -> ``self_energy_k_kspace``
* Appendix A, the sparse Matsubara grid: tau <-> i omega transforms, read as
  exact Fourier integrals of the polynomial that interpolates the tau nodes
  -> ``fourier_matrix``, ``inverse_matrix``
* Eq. G_1 (Dyson equation) with the Hartree G0, the particle number from
  G(beta-) and the chemical potential by bisection -> ``dyson_green_iw``,
  ``green_iw_to_tau``, ``particle_number``, ``chemical_potential``
* the linearisation of Sigma at zero frequency behind the paper's band plots
  (quasiparticle energies) -> ``qp_energies``
* Eq. sf_9, the continued fraction through Sigma on the stored Matsubara grid
  (analytic continuation to w + i delta) -> ``continued_fraction_coefficients``,
  ``continued_fraction_value``, ``continue_sigma``
* Eqs. sf_1 and sf_7, the spectral function from the retarded G -> ``spectral_function``

Readings where the paper is silent or garbled (each listed in the design notes):
P(x, x'; tau) = -s G(x, x'; tau) G(x', x; beta - tau) and G(x', x) = G(x, x')^*;
Sigma(x, x'; tau) = -G(x, x'; tau) W~(x, x'; tau) (the G_{tL;t'L'} of Eq. S_MM
is read as G_{tL'';t'L'''}); pair classes are taken modulo the k-mesh
supercell with minimum-image distances.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np
from numpy.polynomial.legendre import leggauss

__all__ = [
    "kmesh_rule",
    "pair_list",
    "entry_tier",
    "entry_far",
    "entry_pb_dims",
    "green0_k_tau",
    "fourier_k_to_R",
    "fourier_R_to_k",
    "polarizability_R",
    "polarizability_q_kspace",
    "fourier_matrix",
    "inverse_matrix",
    "transform",
    "screened_W",
    "self_energy_R",
    "exchange_R",
    "self_energy_k_kspace",
    "dyson_green_iw",
    "green_iw_to_tau",
    "particle_number",
    "chemical_potential",
    "qp_energies",
    "continued_fraction_coefficients",
    "continued_fraction_value",
    "continue_sigma",
    "spectral_function",
    "OracleSystem",
]


# ----------------------------------------------------------------------------
# Sec. 2: cutoff sphere, k-mesh rule and the pair list
# ----------------------------------------------------------------------------

def kmesh_rule(lattice: np.ndarray, rmax: float) -> Tuple[int, int, int]:
    """Smallest k-mesh with no periodic image inside the R_max sphere (Sec. 2, Fig. 1).

    Along a_i the sphere (diameter 2 R_max) can meet at most ceil(2 R_max / d_i) + 1
    cells, d_i = V / |a_j x a_k| being the spacing of the lattice planes that a_i
    crosses; the mesh needs at least that many points along b_i.
    """
    A = np.asarray(lattice, dtype=np.float64)
    vol = abs(float(np.linalg.det(A)))
    out = []
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        d = vol / float(np.linalg.norm(np.cross(A[j], A[k])))
        out.append(int(math.ceil(2.0 * rmax / d - 1e-12)) + 1)
    return tuple(out)


def pair_list(lattice: np.ndarray, frac: np.ndarray, kmesh: Sequence[int], cutoff: float) -> np.ndarray:
    """Kept pair entries (a, b, class) with their minimum-image lattice vector.

    For every ordered atom pair (a, b) and every lattice class c (R modulo the
    k-mesh supercell, c_i in [0, N_i)), the image R = c + N*m closest to the
    pair, |R + t_b - t_a| minimal, represents the class; the entry is kept when
    that distance is <= cutoff (every class is kept when cutoff <= 0).  Ties
    (squared distances within 1e-9 bohr^2) go to the lexicographically smallest
    R.  Rows: (a, b, c1, c2, c3, R1, R2, R3), sorted by (a, b, c).
    """
    A = np.asarray(lattice, dtype=np.float64)
    frac = np.asarray(frac, dtype=np.float64)
    N = np.asarray(kmesh, dtype=np.int64)
    rows = []
    for a in range(len(frac)):
        for b in range(len(frac)):
            d0 = frac[b] - frac[a]
            for c in np.ndindex(*[int(x) for x in N]):
                best = None
                for m in np.ndindex(5, 5, 5):
                    R = np.array(c, dtype=np.int64) + N * (np.array(m, dtype=np.int64) - 2)
                    x = (R.astype(np.float64) + d0) @ A
                    d2 = float(x @ x)
                    key = (d2, tuple(int(v) for v in R))
                    if best is None or d2 < best[0] - 1e-9 or (abs(d2 - best[0]) <= 1e-9 and key[1] < best[1]):
                        best = key
                if cutoff <= 0.0 or math.sqrt(best[0]) <= cutoff:
                    rows.append((a, b) + tuple(int(v) for v in c) + best[1])
    return np.array(rows, dtype=np.int64).reshape(-1, 8)


def _class_phase(kint: np.ndarray, kmesh: Sequence[int], cls: np.ndarray) -> np.ndarray:
    """e^{+i k.R} on the mesh, k = sum (m_i/N_i) b_i, for integer k-indices and classes."""
    N = np.asarray(kmesh, dtype=np.float64)
    arg = 2.0 * np.pi * ((kint.astype(np.float64) / N) @ cls.astype(np.float64).T)
    return np.exp(1j * arg)


# ----------------------------------------------------------------------------
# the non-interacting input, written independently of the generator
# ----------------------------------------------------------------------------

def green0_k_tau(H_k: np.ndarray, mu: float, beta: float, tau: np.ndarray) -> np.ndarray:
    """G0(k, tau) = -e^{-(H - mu) tau} (1 + e^{-beta (H - mu)})^{-1}, 0+ <= tau <= beta-.

    (The Hartree-level G0 entering Eq. G_1.)  Evaluated in the eigenbasis with
    both exponentials combined into one bounded factor per level; valid for
    tau in (-beta, beta) too, where G0(tau) = -G0(tau + beta) for tau < 0.
    """
    e, U = np.linalg.eigh(H_k)
    xi = e - mu
    out = np.empty((H_k.shape[0], len(tau)) + H_k.shape[1:], np.complex128)
    for i, t in enumerate(np.asarray(tau, dtype=np.float64)):
        if t < 0.0:
            d = +_occ_factor(xi, t + beta, beta)   # G0(tau) = -G0(tau + beta)
        else:
            d = -_occ_factor(xi, t, beta)
        out[:, i] = np.einsum("kij,kj,klj->kil", U, d, U.conj())
    return out


def _occ_factor(xi: np.ndarray, t: float, beta: float) -> np.ndarray:
    # e^{-xi t}/(1+e^{-beta xi}) = 1/(e^{xi t} + e^{xi (t - beta)})
    a = np.clip(xi * t, -700, 700)
    b = np.clip(xi * (t - beta), -700, 700)
    return 1.0 / (np.exp(a) + np.exp(b))


# ----------------------------------------------------------------------------
# Sec. 2: R <-> k transforms restricted to the kept entries
# ----------------------------------------------------------------------------

def entry_tier(lattice: np.ndarray, frac: np.ndarray, entries: np.ndarray, r_b: float) -> np.ndarray:
    """The product-basis level of each entry (Sec. 2, Fig. 2, three levels): 0 when both
    arguments are in the same sphere (a = b and minimum-image distance 0: sphere A), 1 when
    the distance |R + t_b - t_a| is within the radius r_b of sphere B (its square at most
    r_b^2 + 1e-9 bohr^2), 2 beyond it (up to the cutoff, sphere C).  r_b <= 0: no level 2."""
    A = np.asarray(lattice, dtype=np.float64)
    frac = np.asarray(frac, dtype=np.float64)
    tier = np.zeros(len(entries), dtype=np.int64)
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        x = (np.asarray(row[5:8], dtype=np.float64) + frac[b] - frac[a]) @ A
        d2 = float(x @ x)
        if a == b and d2 <= 1e-9:
            tier[e] = 0
        elif r_b > 0.0 and d2 > r_b * r_b + 1e-9:
            tier[e] = 2
        else:
            tier[e] = 1
    return tier


def entry_far(lattice: np.ndarray, frac: np.ndarray, entries: np.ndarray, r_b: float) -> np.ndarray:
    """Entries beyond sphere B (level 2 of entry_tier)."""
    return entry_tier(lattice, frac, entries, r_b) == 2


def entry_pb_dims(entries: np.ndarray, tier, n_prod_atom, n_prod_far_atom, n_prod_near_atom=None) \
        -> List[Tuple[int, int]]:
    """(K_a(e), K_b(e)) per entry: the first functions of each atom's product basis kept at
    the entry's level -- all of them in sphere A, n_prod_near within sphere B (default: all),
    n_prod_far beyond it.  `tier` is the level per entry (entry_tier) or a boolean "far"."""
    near = n_prod_atom if n_prod_near_atom is None else n_prod_near_atom
    out = []
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        t = int(tier[e]) if np.asarray(tier).dtype != bool else (2 if tier[e] else 0)
        src = (n_prod_atom, near, n_prod_far_atom)[t]
        out.append((int(src[a]), int(src[b])))
    return out


def fourier_k_to_R(F_k: np.ndarray, entries: np.ndarray, kmesh, row_off, col_off, dims=None) -> List[np.ndarray]:
    """F_ab(R) = (1/N_k) sum_k e^{-i k.R} F_ab(k) for each kept entry (brute force).

    F_k: [N_k][n_slices][N][N].  Returns a list over entries of [n_slices][rows][cols]:
    the atoms' full blocks, or the top-left dims[e] of them (an entry beyond sphere B).
    """
    kint = np.array(list(np.ndindex(*kmesh)), dtype=np.int64)
    ph = _class_phase(kint, kmesh, entries[:, 2:5])  # [N_k][E]
    nk = len(kint)
    out = []
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        r, c = (row_off[a + 1] - row_off[a], col_off[b + 1] - col_off[b]) if dims is None else dims[e]
        blk = F_k[:, :, row_off[a]:row_off[a] + r, col_off[b]:col_off[b] + c]
        out.append(np.einsum("k,ksij->sij", np.conj(ph[:, e]), blk) / nk)
    return out


def fourier_R_to_k(F_R: Sequence[np.ndarray], entries: np.ndarray, kmesh, row_off, col_off) -> np.ndarray:
    """F_ab(k) = sum_{kept R} e^{+i k.R} F_ab(R) (brute force), dense [N_k][n_slices][N][N]."""
    kint = np.array(list(np.ndindex(*kmesh)), dtype=np.int64)
    ph = _class_phase(kint, kmesh, entries[:, 2:5])
    ns = F_R[0].shape[0]
    out = np.zeros((len(kint), ns, row_off[-1], col_off[-1]), np.complex128)
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        r, c = F_R[e].shape[1:]  # the full block, or the kept top-left part of it
        out[:, :, row_off[a]:row_off[a] + r, col_off[b]:col_off[b] + c] += (
            ph[:, e][:, None, None, None] * F_R[e][None])
    return out


# ----------------------------------------------------------------------------
# Eq. P_MM (MT-MT polarizability) and Eq. P_old (momentum route)
# ----------------------------------------------------------------------------

def polarizability_R(G_R: Sequence[np.ndarray], entries: np.ndarray, C_atom: Sequence[np.ndarray],
                     spin: int = 2, kdims=None) -> List[np.ndarray]:
    """P_{aK, bK'}(R, tau_i) per kept entry (Eq. P_MM, sign and pairing of Eq. P_II).

    P = -s sum_{L L'' L' L'''} C^a_{K; L L''} G_{aL, bL'}(R, tau_i)
            conj(G_{aL'', bL'''}(R, beta - tau_i)) C^b_{K'; L' L'''},
    beta - tau_i being the mirrored node tau_{N-1-i}; K < K_a(e), K' < K_b(e) when
    kdims gives the entry's product-basis sizes (the reduced basis beyond sphere B).
    """
    out = []
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        Ka, Kb = (len(C_atom[a]), len(C_atom[b])) if kdims is None else kdims[e]
        out.append(-spin * _p_block(C_atom[a][:Ka], G_R[e], np.conj(G_R[e][::-1]), C_atom[b][:Kb]))
    return out


def _contract(spec, *ops):
    """np.einsum of the whole sum, with the pairwise order that NumPy's own path search
    picks when intermediates may be as large as 2^27 elements (its default limit, the size
    of the largest operand, would leave a loop over all indices at once)."""
    path = np.einsum_path(spec, *ops, optimize=("greedy", 2 ** 27))[0]
    return np.einsum(spec, *ops, optimize=path)


def _p_block(Ca, G1, G2c, Cb):
    """The sum of Eq. P_MM as one contraction: sum over A, B, C, D of
    Ca[k,A,B] G1[t,A,C] G2c[t,B,D] Cb[q,C,D] -> [t,k,q] (A = L, B = L'', C = L', D = L''')."""
    return _contract("kAB,tAC,tBD,qCD->tkq", Ca, G1, G2c, Cb)


def _s_block(Ca, G, W, Cb):
    """The sum of Eq. S_MM as one contraction: sum over K, M, N, Q of
    Ca[K,L,M] G[t,M,N] W[t,K,Q] Cb[Q,P,N] -> [t,L,P] (M = L'', N = L''', Q = K', P = L')."""
    return _contract("KLM,tMN,tKQ,QPN->tLP", Ca, G, W, Cb)


def polarizability_q_kspace(G_k: np.ndarray, C_atom, orb_off, pb_off, kmesh, spin: int = 2) -> np.ndarray:
    """P_ab(q, tau_i) = -(s/N_k) sum_k C^a [G_ab(k, tau_i) (x) conj G_ab(k - q, beta - tau_i)] C^b.

    The momentum-space convolution of Eq. P_old, evaluated at the tau nodes
    (every pair class included).  Returns dense [N_k][N_tau][N_PB][N_PB].
    """
    kint = np.array(list(np.ndindex(*kmesh)), dtype=np.int64)
    N = np.asarray(kmesh, dtype=np.int64)
    index = {tuple(k): i for i, k in enumerate(kint)}
    nk, nt = G_k.shape[0], G_k.shape[1]
    nat = len(orb_off) - 1
    out = np.zeros((nk, nt, pb_off[-1], pb_off[-1]), np.complex128)
    for iq, q in enumerate(kint):
        for ik, k in enumerate(kint):
            ikq = index[tuple(int(v) for v in np.mod(k - q, N))]
            for a in range(nat):
                for b in range(nat):
                    G1 = G_k[ik, :, orb_off[a]:orb_off[a + 1], orb_off[b]:orb_off[b + 1]]
                    G2 = np.conj(G_k[ikq, ::-1, orb_off[a]:orb_off[a + 1], orb_off[b]:orb_off[b + 1]])
                    out[iq, :, pb_off[a]:pb_off[a + 1], pb_off[b]:pb_off[b + 1]] += _p_block(
                        C_atom[a], G1, G2, C_atom[b])
    return -spin * out / nk


# ----------------------------------------------------------------------------
# Appendix A: tau <-> i omega on the sparse Matsubara grid
# ----------------------------------------------------------------------------

def _barycentric_weights(x: np.ndarray) -> np.ndarray:
    n = len(x)
    w = np.ones(n)
    for i in range(n):
        for j in range(n):
            if i != j:
                w[i] /= (x[i] - x[j])
    return w


def _lagrange_at(xn: np.ndarray, w: np.ndarray, x: np.ndarray) -> np.ndarray:
    """l_i(x) for the interpolation nodes xn (second barycentric form), [len(x)][n]."""
    d = x[:, None] - xn[None, :]
    hit = d == 0.0
    d[hit] = 1.0
    t = w[None, :] / d
    L = t / t.sum(axis=1, keepdims=True)
    r, c = np.nonzero(hit)
    L[r] = 0.0
    L[r, c] = 1.0
    return L


def fourier_matrix(beta: float, tau: np.ndarray, idx: np.ndarray, statistics: str) -> np.ndarray:
    """T[n, i] = int_0^beta e^{i w_n tau} l_i(tau) d tau, l_i the Lagrange polynomial
    of the tau nodes; w_n = (2n+1) pi/beta ('F') or 2n pi/beta ('B').

    A function known at the nodes is read as the polynomial through them, and
    its transform is that polynomial's exact Fourier integral, evaluated by
    composite Gauss-Legendre quadrature (exact up to rounding for this entire
    integrand).
    """
    tau = np.asarray(tau, dtype=np.float64)
    x_n = 2.0 * tau / beta - 1.0
    w = _barycentric_weights(x_n)
    idx = np.asarray(idx, dtype=np.int64)
    if statistics == "F":
        a = (2 * idx + 1) * np.pi / 2.0
    elif statistics == "B":
        a = idx * np.pi * 1.0
    else:
        raise ValueError(statistics)
    out = np.empty((len(idx), len(tau)), np.complex128)
    # composite Gauss-Legendre: panels short enough that e^{iax} turns by at most
    # ~4 radians on each, 48 nodes per panel (exact to rounding for l_i e^{iax});
    # short panels keep the node positions, hence the phases, accurate.
    t48, w48 = leggauss(48)
    for r, ar in enumerate(a):
        S = int(math.ceil(abs(ar) / 4.0)) + 1
        edges = np.linspace(-1.0, 1.0, S + 1)
        c = 0.5 * (edges[1:] + edges[:-1])
        h = 0.5 * (edges[1:] - edges[:-1])
        xg = (c[:, None] + h[:, None] * t48[None, :]).reshape(-1)
        wg = (h[:, None] * w48[None, :]).reshape(-1)
        L = _lagrange_at(x_n, w, xg)  # [M][N]
        # tau = beta (x + 1)/2 ; e^{i w tau} = e^{i a} e^{i a x}
        out[r] = (0.5 * beta) * np.exp(1j * ar) * ((wg * np.exp(1j * ar * xg)) @ L)
    return out


def inverse_matrix(T: np.ndarray) -> np.ndarray:
    """The least-squares inverse of T (its Moore-Penrose pseudo-inverse): the
    polynomial on the tau nodes whose transform best fits the sampled values."""
    return np.linalg.pinv(T, rcond=1e-15)


def transform(T: np.ndarray, F: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Apply a tau/frequency matrix to each entry: out[e][m] = sum_i T[m, i] F[e][i]."""
    return [np.einsum("mi,i...->m...", T, f) for f in F]


# ----------------------------------------------------------------------------
# Eq. W_1: screened interaction, W~ = (1 - v P)^{-1} v - v per (q, nu)
# ----------------------------------------------------------------------------

def screened_W(P_R_iw: Sequence[np.ndarray], entries: np.ndarray, v_q: np.ndarray, kmesh, pb_off,
               nu_subset=None, q_subset=None):
    """W~(R, i nu) on the kept entries (Eq. W_1 with W = V + W~).

    P(q, i nu) = sum_{kept R} e^{+i q.R} P(R, i nu); W(q) solves
    (I - v(q) P(q)) W = v(q) (Eq. W_1 rearranged), W~ = W - v; and
    W~(R) = (1/N_k) sum_q e^{-i q.R} W~(q).  ``nu_subset``/``q_subset``
    restrict the returned W~(q) (for sampled checks); W~(R) needs all q.
    """
    nk = v_q.shape[0]
    n_nu = P_R_iw[0].shape[0]
    dims = [blk.shape[1:] for blk in P_R_iw]  # the entries' product-basis blocks
    P_q = fourier_R_to_k(P_R_iw, entries, kmesh, pb_off, pb_off)  # [N_k][N_nu][N][N]
    I = np.eye(v_q.shape[1])
    if q_subset is not None or nu_subset is not None:
        qs = range(nk) if q_subset is None else q_subset
        ns = range(n_nu) if nu_subset is None else nu_subset
        return {(q, n): np.linalg.solve(I - v_q[q] @ P_q[q, n], v_q[q]) - v_q[q] for q in qs for n in ns}
    Wt_q = np.empty_like(P_q)
    for q in range(nk):
        for n in range(n_nu):
            Wt_q[q, n] = np.linalg.solve(I - v_q[q] @ P_q[q, n], v_q[q]) - v_q[q]
    return fourier_k_to_R(Wt_q, entries, kmesh, pb_off, pb_off, dims), Wt_q


# ----------------------------------------------------------------------------
# Eq. S_MM (dynamic part), the exchange rule, and Eq. S_old (momentum route)
# ----------------------------------------------------------------------------

def self_energy_R(G_R, Wt_R, entries, C_atom) -> List[np.ndarray]:
    """Sigma_{aL, bL'}(R, tau_i) = -sum C^a_{K; L L''} G_{aL'', bL'''}(R, tau_i)
    W~_{aK, bK'}(R, tau_i) C^b_{K'; L' L'''}  (Eq. S_MM, indices as read above), K and K'
    over the entry's product basis (the shape of its W~ block)."""
    out = []
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        Ka, Kb = Wt_R[e].shape[1:]
        out.append(-_s_block(C_atom[a][:Ka], G_R[e], Wt_R[e], C_atom[b][:Kb]))
    return out


def exchange_R(G_R, v_R, entries, C_atom) -> List[np.ndarray]:
    """Static exchange: Eq. S_MM with W~(tau) -> v and G(tau) -> -G(beta-):
    Sigma_x = +sum C^a G(R, beta-) v(R) C^b  (= -rho o v, the Fock term)."""
    out = []
    for e, row in enumerate(entries):
        a, b = int(row[0]), int(row[1])
        Ka, Kb = v_R[e].shape
        out.append(_s_block(C_atom[a][:Ka], G_R[e][-1:], v_R[e][None], C_atom[b][:Kb])[0])
    return out


def self_energy_k_kspace(G_k: np.ndarray, Wt_q_tau: np.ndarray, C_atom, orb_off, pb_off, kmesh) -> np.ndarray:
    """Sigma_ab(k, tau_i) = -(1/N_k) sum_q C^a [G_ab(k - q, tau_i) (x) W~_ab(q, tau_i)] C^b
    (the momentum route of Eq. S_old, at the tau nodes, every pair class included)."""
    kint = np.array(list(np.ndindex(*kmesh)), dtype=np.int64)
    N = np.asarray(kmesh, dtype=np.int64)
    index = {tuple(k): i for i, k in enumerate(kint)}
    nk, nt = G_k.shape[0], G_k.shape[1]
    nat = len(orb_off) - 1
    out = np.zeros((nk, nt, orb_off[-1], orb_off[-1]), np.complex128)
    for ik, k in enumerate(kint):
        for iq, q in enumerate(kint):
            ikq = index[tuple(int(v) for v in np.mod(k - q, N))]
            for a in range(nat):
                for b in range(nat):
                    G = G_k[ikq, :, orb_off[a]:orb_off[a + 1], orb_off[b]:orb_off[b + 1]]
                    W = Wt_q_tau[iq, :, pb_off[a]:pb_off[a + 1], pb_off[b]:pb_off[b + 1]]
                    out[ik, :, orb_off[a]:orb_off[a + 1], orb_off[b]:orb_off[b + 1]] -= _s_block(
                        C_atom[a], G, W, C_atom[b])
    return out / nk


# ----------------------------------------------------------------------------
# Eq. G_1 (Dyson equation), the particle number and the chemical potential
# ----------------------------------------------------------------------------

def dyson_green_iw(H_k: np.ndarray, Sigx_k: np.ndarray, Sig_k_iw, mu: float, beta: float, omega_idx) -> np.ndarray:
    """G(k, i w_n) from Eq. G_1, G = G0 + G0 Sigma G, with G0 = (i w_n + mu - H)^{-1} the
    Green function of the fixed (Hartree) Hamiltonian H and Sigma = Sigma_x + Sigma_c:
    one inverse G = [(i w_n + mu) I - H(k) - Sigma_x(k) - Sigma_c(k, i w_n)]^{-1} per
    (k, n), w_n = (2n + 1) pi / beta.  H_k, Sigx_k: [N_k][N][N]; Sig_k_iw: [N_k][n_w][N][N]
    or None (Sigma_c = 0).  Returns [N_k][n_w][N][N]."""
    nk, N = H_k.shape[0], H_k.shape[1]
    w = (2 * np.asarray(omega_idx, dtype=np.float64) + 1) * np.pi / beta
    I = np.eye(N)
    out = np.empty((nk, len(w), N, N), np.complex128)
    for k in range(nk):
        for n, wn in enumerate(w):
            S = Sigx_k[k] + (Sig_k_iw[k, n] if Sig_k_iw is not None else 0.0)
            out[k, n] = np.linalg.inv((1j * wn + mu) * I - H_k[k] - S)
    return out


def green_iw_to_tau(G_iw: np.ndarray, H_k: np.ndarray, Sigx_k: np.ndarray, mu: float, beta: float, tau,
                    omega_idx, F_inv: np.ndarray) -> np.ndarray:
    """G(k, tau_i) from G(k, i w_n) by the inverse transform of Appendix A.  The two leading
    terms of G at large frequency, 1/(i w) and M1/(i w)^2 with M1 = H + Sigma_x - mu, are
    taken out before the transform and added back as their tau functions over [0, beta]:
    -1/2 and M1 (2 tau - beta)/4 (each the function whose fermionic Matsubara integral is
    that term).  Returns [N_k][N_tau][N][N]."""
    w = (2 * np.asarray(omega_idx, dtype=np.float64) + 1) * np.pi / beta
    N = G_iw.shape[-1]
    I = np.eye(N)
    M1 = H_k + Sigx_k - mu * I
    iw = 1j * w
    rem = G_iw - I[None, None] / iw[None, :, None, None] - M1[:, None] / (iw * iw)[None, :, None, None]
    out = np.einsum("tn,knij->ktij", F_inv, rem)
    t = np.asarray(tau, dtype=np.float64)
    return out - 0.5 * I[None, None] + M1[:, None] * ((2.0 * t - beta) / 4.0)[None, :, None, None]


def particle_number(G_k_tau: np.ndarray, spin: int = 2) -> float:
    """Electrons per cell, N = s (1/N_k) sum_k Tr[-G(k, beta-)] (the last tau node):
    -G(beta-) is the one-particle density matrix."""
    return float(spin * np.real(np.trace(-G_k_tau[:, -1], axis1=1, axis2=2)).sum() / G_k_tau.shape[0])


def chemical_potential(H_k, Sigx_k, Sig_k_iw, n_electrons: float, beta: float, tau, omega_idx, F_inv,
                       spin: int = 2, lo: float = -5.0, hi: float = 5.0, tol: float = 1e-12):
    """mu with N(mu) = n_electrons, by bisection on [lo, hi] (N grows with mu); N(mu)
    from G(k, beta-) of Eq. G_1 through the inverse transform above.  Returns (mu, N(mu))."""
    def count(m):
        G = green_iw_to_tau(dyson_green_iw(H_k, Sigx_k, Sig_k_iw, m, beta, omega_idx), H_k, Sigx_k, m, beta,
                            tau, omega_idx, F_inv)
        return particle_number(G, spin)
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if count(mid) < n_electrons:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return mu, count(mu)


def qp_energies(H_k: np.ndarray, Sigx_k: np.ndarray, Sig_k_iw, mu: float, beta: float, omega_idx) -> np.ndarray:
    """Linearised quasiparticle energies (the procedure the paper uses for its band
    plots: the value and the frequency derivative of Sigma at zero frequency).  Through
    the two lowest positive fermionic frequencies w_0 = pi/beta and w_1 = 3 pi/beta,
    Sigma_c(i w) ~ S0 + i w S1 with S1 = (Sigma_c(i w_1) - Sigma_c(i w_0)) / (i (w_1 - w_0)) and
    S0 = Sigma_c(i w_0) - i w_0 S1.  The poles of [i w (I - S1) - (H + Sigma_x + S0 - mu)]^{-1}
    continued to the real axis, with Hermitian parts (h), are the eigenvalues of
    A^{-1} (H + Sigma_x^h + S0^h - mu) A^{-1} with A = (I - S1^h)^{1/2}, plus mu.
    Returns [N_k][N] ascending."""
    idx = [int(n) for n in omega_idx]
    i0, i1 = idx.index(0), idx.index(1)
    w0, w1 = np.pi / beta, 3.0 * np.pi / beta
    nk, N = H_k.shape[0], H_k.shape[1]
    I = np.eye(N)
    herm = lambda M: 0.5 * (M + M.conj().T)
    out = np.empty((nk, N))
    for k in range(nk):
        if Sig_k_iw is None:
            S0 = S1 = np.zeros((N, N), np.complex128)
        else:
            S1 = (Sig_k_iw[k, i1] - Sig_k_iw[k, i0]) / (1j * (w1 - w0))
            S0 = Sig_k_iw[k, i0] - 1j * w0 * S1
        lam, U = np.linalg.eigh(I - herm(S1))
        Ainv = (U / np.sqrt(lam)) @ U.conj().T
        X = herm(H_k[k]) + herm(Sigx_k[k]) + herm(S0) - mu * I
        out[k] = np.linalg.eigvalsh(herm(Ainv @ X @ Ainv)) + mu
    return out


def continued_fraction_coefficients(z: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Coefficients a_0..a_M of the continued fraction of Eq. sf_9 through the points
    (z_i, f_i), i = 0..M (the recursion of its reference, Vidberg and Serene): g_0(z_i) = f_i,
    g_p(z_i) = (g_{p-1}(z_{p-1}) - g_{p-1}(z_i)) / ((z_i - z_{p-1}) g_{p-1}(z_i)) for i >= p,
    a_p = g_p(z_p).  f: [M+1][...] (any trailing shape, one fraction per element)."""
    z = np.asarray(z, dtype=np.complex128)
    g = np.array(f, dtype=np.complex128, copy=True)
    a = np.empty_like(g)
    a[0] = g[0]
    shape = (-1,) + (1,) * (g.ndim - 1)
    for p in range(1, len(z)):
        g[p:] = (g[p - 1] - g[p:]) / ((z[p:] - z[p - 1]).reshape(shape) * g[p:])
        a[p] = g[p]
    return a


def continued_fraction_value(a: np.ndarray, z: np.ndarray, w) -> np.ndarray:
    """Eq. sf_9 at the complex frequencies w: a_0 / (1 + a_1 (w - z_0) / (1 + ... a_M (w - z_{M-1}) / 1)),
    evaluated from the innermost level out.  Returns [len(w)][...]."""
    z = np.asarray(z, dtype=np.complex128)
    w = np.asarray(w, dtype=np.complex128)
    M = len(z) - 1
    out = []
    for x in w:
        A = np.ones_like(a[0])
        for p in range(M, 0, -1):
            A = 1.0 + a[p] * (x - z[p - 1]) / A
        out.append(a[0] / A)
    return np.array(out)


def continue_sigma(Sig_k_iw: np.ndarray, omega_idx, beta: float, w_real, delta: float) -> np.ndarray:
    """Sigma(k, w + i delta) per element from Sigma(k, i w_n) on the stored grid's non-negative
    sampled frequencies (the paper feeds the continuation the self-consistent grid itself),
    by the continued fraction of Eq. sf_9.  Sig_k_iw: [N_k][n_w][N][N]; returns
    [N_k][len(w_real)][N][N]."""
    idx = np.asarray(omega_idx)
    pos = np.nonzero(idx >= 0)[0]
    pos = pos[np.argsort(idx[pos])]
    z = 1j * (2 * idx[pos] + 1) * np.pi / beta
    w = np.asarray(w_real, dtype=np.float64) + 1j * delta
    out = np.empty((Sig_k_iw.shape[0], len(w)) + Sig_k_iw.shape[2:], np.complex128)
    for k in range(Sig_k_iw.shape[0]):
        a = continued_fraction_coefficients(z, Sig_k_iw[k, pos])
        out[k] = continued_fraction_value(a, z, w)
    return out


def spectral_function(H_k: np.ndarray, Sigx_k: np.ndarray, Sig_k_w, mu: float, w_real, delta: float) -> np.ndarray:
    """Eq. sf_1 with the retarded Green function of Eq. sf_7: A(k, w) = -(1/pi) Im Tr G^R(k, w),
    G^R = [(w + i delta + mu) I - H - Sigma_x - Sigma_c^R(w)]^{-1}.  Eq. sf_7 writes it in the
    band states of H + Sigma_x (its eigenvalues on the diagonal); the trace is the same in
    any basis.  Sig_k_w: [N_k][n_w][N][N] continued Sigma_c (or None); returns [N_k][n_w]."""
    nk, N = H_k.shape[0], H_k.shape[1]
    w = np.asarray(w_real, dtype=np.float64)
    I = np.eye(N)
    out = np.empty((nk, len(w)))
    for k in range(nk):
        for r, x in enumerate(w):
            S = Sigx_k[k] + (Sig_k_w[k, r] if Sig_k_w is not None else 0.0)
            out[k, r] = -np.trace(np.linalg.inv((x + 1j * delta + mu) * I - H_k[k] - S)).imag / np.pi
    return out


# ----------------------------------------------------------------------------
# convenience: one whole sweep on a synthetic cell
# ----------------------------------------------------------------------------

class OracleSystem:
    """Holds one synthetic cell's inputs and runs the oracle's steps in order."""

    def __init__(self, cell, entries: np.ndarray = None):
        self.cell = cell
        self.kmesh = tuple(int(x) for x in cell.kmesh)
        self.entries = pair_list(cell.lattice, cell.frac, self.kmesh, cell.cutoff) if entries is None else entries
        self.orb_off = cell.orb_offsets
        self.pb_off = cell.pb_offsets
        self.C_atom = [cell.species[s].C for s in cell.species_of_atom]
        self.spin = cell.spin
        self.beta = cell.beta
        self.tau = cell.tau
        self.F_fwd = fourier_matrix(cell.beta, self.tau, cell.omega_idx, "F")
        self.B_fwd = fourier_matrix(cell.beta, self.tau, cell.nu_idx, "B")
        self.F_inv = inverse_matrix(self.F_fwd)
        self.B_inv = inverse_matrix(self.B_fwd)
        # the product-basis levels of Sec. 2, Fig. 2 (spheres A, B, C), when the cell has them
        r_b = float(getattr(cell, "r_b", 0.0) or 0.0)
        self.tier = entry_tier(cell.lattice, cell.frac, self.entries, r_b)
        self.far = self.tier == 2
        n_full = [len(C) for C in self.C_atom]
        sp = [cell.species[s] for s in cell.species_of_atom]
        n_far = [x.n_prod_far or x.n_prod for x in sp] if r_b > 0 else n_full
        n_near = [getattr(x, "n_prod_near", None) or x.n_prod for x in sp] if r_b > 0 else n_full
        self.kdims = entry_pb_dims(self.entries, self.tier, n_full, n_far, n_near)

    def v_R(self, v_class: np.ndarray) -> List[np.ndarray]:
        out = []
        for e, row in enumerate(self.entries):
            a, b = int(row[0]), int(row[1])
            c = int(np.ravel_multi_index(tuple(row[2:5]), self.kmesh))
            Ka, Kb = self.kdims[e]
            out.append(v_class[a, b, c, :Ka, :Kb].astype(np.complex128))
        return out

    def sweep(self, G_k: np.ndarray, v_q: np.ndarray, v_class: np.ndarray) -> dict:
        r = {}
        r["G_R"] = fourier_k_to_R(G_k, self.entries, self.kmesh, self.orb_off, self.orb_off)
        r["P_R"] = polarizability_R(r["G_R"], self.entries, self.C_atom, self.spin, self.kdims)
        r["P_iw"] = transform(self.B_fwd, r["P_R"])
        r["Wt_iw"], r["Wt_q"] = screened_W(r["P_iw"], self.entries, v_q, self.kmesh, self.pb_off)
        r["Wt_R"] = transform(self.B_inv, r["Wt_iw"])
        r["v_R"] = self.v_R(v_class)
        r["Sig_R"] = self_energy_R(r["G_R"], r["Wt_R"], self.entries, self.C_atom)
        r["Sigx_R"] = exchange_R(r["G_R"], r["v_R"], self.entries, self.C_atom)
        r["Sig_iw"] = transform(self.F_fwd, r["Sig_R"])
        r["Sig_k"] = fourier_R_to_k(r["Sig_iw"], self.entries, self.kmesh, self.orb_off, self.orb_off)
        r["Sigx_k"] = fourier_R_to_k([s[None] for s in r["Sigx_R"]], self.entries, self.kmesh,
                                     self.orb_off, self.orb_off)[:, 0]
        return r
