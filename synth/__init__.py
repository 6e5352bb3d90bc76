"""Seeded synthetic inputs for the real-space / imaginary-time GW sweep.

This module builds the *inputs* of one GW iteration on tight-binding stand-ins
for the paper's silicon and oxide supercells (Sec. 4 and Sec. 5 of
arXiv:1911.05633 use FLAPW inputs that are not reproduced here):

* the cell (lattice, atoms, species), the k-mesh and the distance cutoff;
* the per-species one-centre product-basis coefficients C[K][L][L'']
  (the <M_K | phi_L phi_L''> of Eq. P_MM), real and symmetric in (L, L'');
* the seeded tight-binding hoppings, the Bloch Hamiltonian H(k), the
  chemical potential and the non-interacting Green's function G(k, tau) that
  an iteration takes as its input (the paper starts each iteration from "some
  approximate Green's function", Sec. 2);
* the bare interaction v in the product basis, both per lattice class v(R)
  and on the mesh v(q), an exact discrete Fourier pair;
* the imaginary-time nodes and the sampled Matsubara index sets.

It holds none of the arithmetic of the method itself (no P, W, Sigma, no
tau <-> i omega transform and no pair list).  Both the oracle and the CUDA
path take their inputs from here; neither imports the other.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Species",
    "SynthCell",
    "make_config",
    "batch_family",
    "perovskite_cell",
    "f_rich_cell",
    "chain_cell",
    "mixed_species_cell",
    "tau_nodes",
    "matsubara_sets",
    "fermi",
]

# ----------------------------------------------------------------------------
# geometry helpers (plain crystallography, no GW arithmetic)
# ----------------------------------------------------------------------------

_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_DIAMOND8 = np.vstack([_FCC, _FCC + 0.25])


@dataclasses.dataclass
class Species:
    name: str
    n_orb: int
    n_prod: int
    C: np.ndarray  # [n_prod][n_orb][n_orb] float64, symmetric in the last two
    n_prod_far: Optional[int] = None   # product functions kept by pairs beyond sphere B
    n_prod_near: Optional[int] = None  # product functions kept by other pairs within sphere B


@dataclasses.dataclass
class SynthCell:
    """One synthetic system: geometry, basis, grids and seeded model inputs."""

    name: str
    lattice: np.ndarray          # [3][3] rows a_1, a_2, a_3 (bohr)
    frac: np.ndarray             # [n_atoms][3] fractional coordinates
    species_of_atom: np.ndarray  # [n_atoms] int32
    species: List[Species]
    kmesh: Tuple[int, int, int]
    beta: float
    n_tau: int
    cutoff: float                # <= 0 : keep every pair class
    seed: int
    gap: Optional[float] = None  # target on-mesh gap (Ha) or None
    hop_cutoff: float = 10.0
    spin: int = 2
    r_b: float = 0.0             # radius of sphere B (bohr); <= 0: one product basis for every pair
    # filled by build()
    hoppings: Optional[list] = None
    H_k: Optional[np.ndarray] = None
    mu: Optional[float] = None
    X_coul: Optional[np.ndarray] = None
    delta_coul: float = 0.0

    # -- derived sizes ---------------------------------------------------------
    @property
    def n_atoms(self) -> int:
        return int(len(self.frac))

    @property
    def n_k(self) -> int:
        return int(np.prod(self.kmesh))

    def n_orb_of(self, a: int) -> int:
        return self.species[self.species_of_atom[a]].n_orb

    def n_prod_of(self, a: int) -> int:
        return self.species[self.species_of_atom[a]].n_prod

    @property
    def orb_offsets(self) -> np.ndarray:
        n = [self.n_orb_of(a) for a in range(self.n_atoms)]
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    @property
    def pb_offsets(self) -> np.ndarray:
        n = [self.n_prod_of(a) for a in range(self.n_atoms)]
        return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    @property
    def n_orb_total(self) -> int:
        return int(self.orb_offsets[-1])

    @property
    def n_pb_total(self) -> int:
        return int(self.pb_offsets[-1])

    @property
    def tau(self) -> np.ndarray:
        return tau_nodes(self.beta, self.n_tau)

    @property
    def omega_idx(self) -> np.ndarray:
        return matsubara_sets(self.n_tau)[0]

    @property
    def nu_idx(self) -> np.ndarray:
        return matsubara_sets(self.n_tau)[1]

    def kpoints_frac(self) -> np.ndarray:
        """Gamma-centred mesh, k = sum_i (m_i / N_i) b_i; rows are (m_i / N_i)."""
        n1, n2, n3 = self.kmesh
        m = np.array(list(np.ndindex(n1, n2, n3)), dtype=np.int64)
        return m / np.array(self.kmesh, dtype=np.float64)

    def kpoints_int(self) -> np.ndarray:
        n1, n2, n3 = self.kmesh
        return np.array(list(np.ndindex(n1, n2, n3)), dtype=np.int64)

    # -- model construction ------------------------------------------------------
    def build(self) -> "SynthCell":
        rng = np.random.default_rng(self.seed)
        self._draw_basis(rng)
        self._draw_hoppings(rng)
        self._draw_coulomb(rng)
        if self.gap is not None:
            self._fit_gap(self.gap)
        self.H_k = self.bloch_hamiltonian()
        self.mu = self._chemical_potential()
        return self

    def _draw_basis(self, rng: np.random.Generator) -> None:
        for sp in self.species:
            if sp.C is None or sp.C.size == 0:
                x = rng.standard_normal((sp.n_prod, sp.n_orb, sp.n_orb))
                sp.C = (0.5 * (x + x.transpose(0, 2, 1)) / sp.n_orb).astype(np.float64)

    def _images(self, a: int, b: int, rmax: float):
        """All lattice vectors R (integer) with |R + t_b - t_a| <= rmax."""
        A = self.lattice
        d0 = self.frac[b] - self.frac[a]
        # bound on |n_i| from the plane spacings
        vol = abs(np.linalg.det(A))
        spans = []
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            h = vol / np.linalg.norm(np.cross(A[j], A[k]))
            spans.append(int(math.ceil(rmax / h)) + 1)
        out = []
        for n1 in range(-spans[0], spans[0] + 1):
            for n2 in range(-spans[1], spans[1] + 1):
                for n3 in range(-spans[2], spans[2] + 1):
                    R = np.array([n1, n2, n3], dtype=np.float64)
                    dist = float(np.linalg.norm((R + d0) @ A))
                    if dist <= rmax + 1e-9:
                        out.append(((n1, n2, n3), dist))
        return out

    def _draw_hoppings(self, rng: np.random.Generator) -> None:
        """h(a L, b L', R) = <a,0| H |b,R>, Hermitian by construction.

        Onsite levels U[-0.5, 0.5] Ha; every other element within hop_cutoff has
        magnitude 0.1 exp(-|d| / 2 bohr) and a uniform random phase.  Only the
        canonical half is drawn; h(b, a, -R) = h(a, b, R)^dagger.
        """
        hops = []
        for a in range(self.n_atoms):
            for b in range(a, self.n_atoms):
                for R, dist in self._images(a, b, self.hop_cutoff):
                    if a == b and R < (0, 0, 0):
                        continue
                    na, nb = self.n_orb_of(a), self.n_orb_of(b)
                    mag = 0.1 * math.exp(-dist / 2.0)
                    ph = np.exp(2j * np.pi * rng.random((na, nb)))
                    blk = mag * ph
                    if a == b and R == (0, 0, 0):
                        lev = rng.uniform(-0.5, 0.5, na)
                        blk = np.triu(blk, 1)
                        blk = blk + blk.conj().T + np.diag(lev)
                    hops.append((a, b, R, blk))
        self.hoppings = hops

    def bloch_hamiltonian(self, kfrac: Optional[np.ndarray] = None) -> np.ndarray:
        """H(k) = sum_R e^{+i k.R} h(a, b, R) over the infinite lattice."""
        if kfrac is None:
            kfrac = self.kpoints_frac()
        oo = self.orb_offsets
        H = np.zeros((len(kfrac), self.n_orb_total, self.n_orb_total), np.complex128)
        for a, b, R, blk in self.hoppings:
            ph = np.exp(2j * np.pi * (kfrac @ np.array(R, dtype=np.float64)))
            sa = slice(oo[a], oo[a + 1])
            sb = slice(oo[b], oo[b + 1])
            if a == b and R == (0, 0, 0):
                H[:, sa, sb] += blk[None]
                continue
            H[:, sa, sb] += ph[:, None, None] * blk[None]
            # the Hermitian partner h(b, a, -R) = blk^dagger
            H[:, sb, sa] += np.conj(ph)[:, None, None] * blk.conj().T[None]
        return H

    def _fit_gap(self, target: float) -> None:
        """Shift the lower/upper half of the sorted onsite levels by -+D/2 so that
        the on-mesh gap at half filling equals `target` (bisection on D)."""
        oo = self.orb_offsets
        onsite = [(i, h) for i, h in enumerate(self.hoppings) if h[0] == h[1] and h[2] == (0, 0, 0)]
        levels = []
        for i, (a, _, _, blk) in onsite:
            for L in range(blk.shape[0]):
                levels.append((blk[L, L].real, i, L))
        order = sorted(range(len(levels)), key=lambda j: levels[j][0])
        half = len(order) // 2
        sign = np.zeros(len(levels))
        sign[order[:half]] = -1.0
        sign[order[half:]] = +1.0
        base = [blk.copy() for (_, (_, _, _, blk)) in onsite]

        def apply(D):
            for n, (i, (a, b, R, _)) in enumerate(onsite):
                blk = base[n].copy()
                for j, (lev, ii, L) in enumerate(levels):
                    if ii == i:
                        blk[L, L] += 0.5 * D * sign[j]
                self.hoppings[i] = (a, b, R, blk)

        def gap_of(D):
            apply(D)
            e = np.linalg.eigvalsh(self.bloch_hamiltonian())
            nh = self.n_orb_total // 2
            return float(e[:, nh].min() - e[:, nh - 1].max())

        if gap_of(0.0) >= target:
            apply(0.0)
            return
        lo, hi = 0.0, 1.0
        while gap_of(hi) < target:
            hi *= 2.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if gap_of(mid) < target:
                lo = mid
            else:
                hi = mid
        apply(hi)

    def _chemical_potential(self) -> float:
        """Half filling: N_orb electrons per cell with spin degeneracy 2."""
        e = np.linalg.eigvalsh(self.H_k)
        target = float(self.n_orb_total) / self.spin
        lo, hi = float(e.min()) - 1.0, float(e.max()) + 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            n = float(fermi(e - mid, self.beta).sum()) / self.n_k
            if n < target:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    # -- the input Green's function ---------------------------------------------------
    def green_k_tau(self, tau: Optional[np.ndarray] = None) -> np.ndarray:
        """Input G(k, tau_i) = -U diag(e^{-xi tau} / (1 + e^{-beta xi})) U^dagger.

        tau = 0 is read as 0+, tau = beta as beta-.  Layout [N_k][N_tau][N_orb][N_orb].
        """
        if tau is None:
            tau = self.tau
        e, U = np.linalg.eigh(self.H_k)
        xi = e - self.mu
        out = np.empty((self.n_k, len(tau), self.n_orb_total, self.n_orb_total), np.complex128)
        for k in range(self.n_k):
            for i, t in enumerate(tau):
                g = _g0_diag(xi[k], t, self.beta)
                out[k, i] = (U[k] * g[None, :]) @ U[k].conj().T
        return out

    # -- bare interaction in the product basis ---------------------------------------
    def _draw_coulomb(self, rng: np.random.Generator) -> None:
        kmax = max(sp.n_prod for sp in self.species)
        A = rng.standard_normal((kmax, kmax))
        self.X_coul = A @ A.T / kmax + 0.1 * np.eye(kmax)

    def class_min_distance(self, a: int, b: int) -> np.ndarray:
        """Minimum-image distance |R + t_b - t_a| for every class R mod the mesh."""
        n = np.array(self.kmesh)
        A = self.lattice
        d0 = self.frac[b] - self.frac[a]
        out = np.empty(self.n_k)
        shifts = np.array(list(np.ndindex(5, 5, 5))) - 2
        for ci, c in enumerate(self.kpoints_int()):
            R = c[None, :] + shifts * n[None, :]
            out[ci] = np.min(np.linalg.norm((R + d0) @ A, axis=1))
        return out

    def coulomb_class(self) -> np.ndarray:
        """v_{aK, bK'}(c) for every class c, [n_atoms][n_atoms][N_k][Kmax][Kmax].

        v = X_{KK'} / (1 + d_min) plus delta I on the onsite (a = a, R = 0) block;
        blocks of atoms with fewer product functions use the leading sub-block.
        """
        na, nk = self.n_atoms, self.n_k
        kmax = self.X_coul.shape[0]
        out = np.zeros((na, na, nk, kmax, kmax))
        for a in range(na):
            for b in range(na):
                f = 1.0 / (1.0 + self.class_min_distance(a, b))
                out[a, b] = f[:, None, None] * self.X_coul[None]
        return out

    def coulomb(self) -> Tuple[np.ndarray, np.ndarray]:
        """(v_q [N_k][N_PB][N_PB], v_class) with v_q = sum_c e^{i q.R_c} v(c) + delta I.

        delta >= 0 is the smallest shift that makes every v(q) >= 0.05 I.  The same
        delta is added to v_class on the onsite blocks, so the pair stays exact.
        """
        vc = self.coulomb_class()
        po = self.pb_offsets
        kint = self.kpoints_int()
        nk = self.n_k
        npb = self.n_pb_total
        # phase[q][c] = exp(2 pi i sum_j q_j c_j / N_j)
        qf = self.kpoints_frac()
        ph = np.exp(2j * np.pi * (qf @ kint.T.astype(np.float64)))
        vq = np.zeros((nk, npb, npb), np.complex128)
        for a in range(self.n_atoms):
            for b in range(self.n_atoms):
                Ka, Kb = self.n_prod_of(a), self.n_prod_of(b)
                blk = np.einsum("qc,cij->qij", ph, vc[a, b, :, :Ka, :Kb])
                vq[:, po[a]:po[a + 1], po[b]:po[b + 1]] = blk
        vq = 0.5 * (vq + vq.conj().transpose(0, 2, 1))
        lam = min(float(np.linalg.eigvalsh(vq[q]).min()) for q in range(nk))
        delta = max(0.0, 0.05 - lam)
        self.delta_coul = delta
        vq += delta * np.eye(npb)[None]
        for a in range(self.n_atoms):
            vc[a, a, 0] += delta * np.eye(vc.shape[-1])
        return vq, vc


def _g0_diag(xi: np.ndarray, t: float, beta: float) -> np.ndarray:
    """-e^{-xi t}/(1+e^{-beta xi}) for 0 <= t <= beta, written without overflow."""
    out = np.empty_like(xi)
    pos = xi >= 0
    out[pos] = -np.exp(-xi[pos] * t) / (1.0 + np.exp(-beta * xi[pos]))
    neg = ~pos
    out[neg] = -np.exp(xi[neg] * (beta - t)) / (np.exp(beta * xi[neg]) + 1.0)
    return out


def fermi(xi: np.ndarray, beta: float) -> np.ndarray:
    """Fermi function 1/(1+e^{beta xi}), overflow-safe."""
    x = np.clip(beta * np.asarray(xi, dtype=np.float64), -700.0, 700.0)
    return 0.5 * (1.0 - np.tanh(0.5 * x))


# ----------------------------------------------------------------------------
# imaginary-time / Matsubara grids (inputs of the plan)
# ----------------------------------------------------------------------------

def tau_nodes(beta: float, n: int) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto nodes tau_i = (beta/2)(1 - cos(pi i/(n-1))).

    Clustered at 0 and beta and mirror-symmetric: beta - tau_i = tau_{n-1-i}.
    The end points are read as the one-sided limits 0+ and beta-.
    """
    i = np.arange(n, dtype=np.float64)
    t = 0.5 * beta * (1.0 - np.cos(np.pi * i / (n - 1)))
    t[0] = 0.0
    t[-1] = beta
    # enforce exact mirror symmetry in floating point
    half = n // 2
    t[n - 1 - np.arange(half)] = beta - t[np.arange(half)]
    return t


def matsubara_sets(n_tau: int) -> Tuple[np.ndarray, np.ndarray]:
    """Sampled Matsubara indices (fermionic n: (2n+1)pi/beta, bosonic m: 2m pi/beta).

    The lowest round(3 N/8) non-negative fermionic indices are equidistant, the
    rest of the ceil(N/2) non-negative ones grow geometrically up to 3N (the
    sparse, progressively spaced shape of the paper's appendix A).  The
    fermionic set is symmetric (n <-> -n-1, 2 ceil(N/2) indices); the bosonic
    set is {0, +-(n+1)} (2 ceil(N/2) + 1 indices).  Ascending order.
    """
    npos = (n_tau + 1) // 2
    neq = max(1, int(round(0.375 * n_tau)))
    nmax = 3 * n_tau
    idx = list(range(min(neq, npos)))
    if npos > len(idx):
        geo = np.geomspace(max(neq, 1), nmax, npos - len(idx))
        for g in geo:
            g = max(int(round(g)), idx[-1] + 1)
            idx.append(g)
    idx = np.array(idx[:npos], dtype=np.int64)
    fer = np.sort(np.concatenate([idx, -idx - 1]))
    bos = np.sort(np.concatenate([[0], idx + 1, -(idx + 1)]))
    return fer.astype(np.int64), bos.astype(np.int64)


# ----------------------------------------------------------------------------
# named configurations
# ----------------------------------------------------------------------------

def _diamond_supercell(mult: Sequence[int], a: float = 10.26) -> Tuple[np.ndarray, np.ndarray]:
    m = np.array(mult)
    frac = []
    for s in np.ndindex(*m):
        for f in _DIAMOND8:
            frac.append((f + np.array(s)) / m)
    return np.diag(a * m.astype(np.float64)), np.array(frac)


def make_config(idx: int, atoms: Optional[int] = None, build: bool = True, **over) -> SynthCell:
    """The synthetic workloads.

    0: simple-cubic a = 5 bohr, 2 atoms, 4 orbitals, 8 product functions,
       2x2x2 mesh, beta = 50, 24 tau nodes, every pair class kept.
    1: diamond 8-atom cell a = 10.26 bohr, 9 orbitals, 48 product functions,
       4x4x4 mesh, beta = 1000, 48 tau nodes, cutoff 12 bohr, gap 0.04 Ha.
    2: diamond supercell (3x3x1 of the 8-atom cell: 72 atoms; `atoms` picks
       8/16/32/48/72 along 1x1x1, 2x1x1, 2x2x1, 3x2x1, 3x3x1), 9 orbitals,
       64 product functions, 2x2x2 mesh, beta = 1000, 64 tau nodes, cutoff 12.
    """
    if idx == 0:
        lat = np.eye(3) * 5.0
        frac = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
        sp = [Species("sp", 4, 8, None)]
        cell = SynthCell("sc2-n4-K8", lat, frac, np.zeros(2, np.int32), sp, (2, 2, 2),
                         50.0, 24, 0.0, seed=0, gap=None, hop_cutoff=8.0)
    elif idx == 1:
        lat, frac = _diamond_supercell((1, 1, 1))
        sp = [Species("spd", 9, 48, None)]
        cell = SynthCell("diamond8-n9-K48", lat, frac, np.zeros(8, np.int32), sp, (4, 4, 4),
                         1000.0, 48, 12.0, seed=1000, gap=0.04, hop_cutoff=12.0)
    elif idx == 2:
        series = {8: (1, 1, 1), 16: (2, 1, 1), 32: (2, 2, 1), 48: (3, 2, 1), 72: (3, 3, 1)}
        nat = 72 if atoms is None else int(atoms)
        lat, frac = _diamond_supercell(series[nat])
        sp = [Species("spd", 9, 64, None)]
        cell = SynthCell(f"diamond{nat}-n9-K64", lat, frac, np.zeros(len(frac), np.int32), sp,
                         (2, 2, 2), 1000.0, 64, 12.0, seed=2000 + nat, gap=0.04, hop_cutoff=12.0)
    else:
        raise ValueError(f"unknown configuration {idx}")
    for k, v in over.items():
        setattr(cell, k, v)
    return cell.build() if build else cell


# the layered perovskite of the large-cell runs (K2NiF4 type, as La2CuO4): body-centred
# tetragonal conventional cell of 14 atoms, a = 7.14 bohr, c = 24.85 bohr
_K2NIF4_14 = np.array([
    [0.0, 0.0, 0.0], [0.5, 0.5, 0.5],                                        # transition-metal sites
    [0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5],      # in-plane anions
    [0.0, 0.0, 0.182], [0.0, 0.0, 0.818], [0.5, 0.5, 0.318], [0.5, 0.5, 0.682],  # apical anions
    [0.0, 0.0, 0.362], [0.0, 0.0, 0.638], [0.5, 0.5, 0.138], [0.5, 0.5, 0.862],  # A-site cations
])
_K2NIF4_SPECIES = np.array([0, 0, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1], np.int32)


def perovskite_cell(mult=(2, 2, 1), kmesh=(2, 2, 2), n_tau: int = 48, cutoff: float = 12.0, seed: int = 3000,
                    beta: float = 1000.0) -> SynthCell:
    """Layered perovskite-like cell (K2NiF4 type, the structure of La2CuO4): 14 atoms per
    conventional cell, `mult` cells (2x2x1: 56 atoms).  Species: transition-metal sites with
    14 orbitals (s, p, d and a second d-like shell) and 96 product functions, A-site cations
    with 9 orbitals and 64, anions with 9 orbitals and 40."""
    m = np.array(mult)
    frac, spec = [], []
    for sft in np.ndindex(*m):
        for f, sp in zip(_K2NIF4_14, _K2NIF4_SPECIES):
            frac.append((f + np.array(sft)) / m)
            spec.append(sp)
    lat = np.diag([7.14 * m[0], 7.14 * m[1], 24.85 * m[2]])
    sp = [Species("tm", 14, 96, None), Species("a", 9, 64, None), Species("x", 9, 40, None)]
    n = len(frac)
    return SynthCell(f"perovskite{n}-n14/9-K96/64/40", lat, np.array(frac), np.array(spec, np.int32), sp,
                     tuple(kmesh), beta, n_tau, cutoff, seed=seed, gap=None, hop_cutoff=cutoff).build()


def f_rich_cell(kmesh=(2, 2, 2), n_tau: int = 48, cutoff: float = 10.0, seed: int = 4000,
                beta: float = 1000.0) -> SynthCell:
    """Cubic cell of 64 atoms rich in f orbitals (as the SmB6 runs): 8 heavy sites on a 2x2x2
    simple-cubic sublattice with 16 orbitals (s, p, d and f shells: 1 + 3 + 5 + 7) and 112
    product functions, and 56 light atoms with 9 orbitals and 48 (an octahedron of six around
    each cube centre and eight on the x-edge midpoints of the heavy sublattice)."""
    a = 7.8  # bohr per heavy-atom cube
    frac = []
    for c in np.ndindex(2, 2, 2):
        frac.append(np.array(c) / 2.0)
    spec = [0] * 8
    u = 0.2
    for c in np.ndindex(2, 2, 2):
        ctr = (np.array(c) + 0.5) / 2.0
        for d in np.vstack([np.eye(3), -np.eye(3)]):
            frac.append(ctr + u * d / 2.0)
            spec.append(1)
    for c in np.ndindex(2, 2, 2):  # the x-edge midpoints of the heavy sublattice
        frac.append(np.array([0.25 + c[0] / 2.0, c[1] / 2.0, c[2] / 2.0]))
        spec.append(1)
    frac = np.mod(np.array(frac), 1.0)
    lat = np.eye(3) * 2 * a
    sp = [Species("f", 16, 112, None), Species("light", 9, 48, None)]
    return SynthCell("frich64-n16/9-K112/48", lat, frac, np.array(spec, np.int32), sp, tuple(kmesh), beta, n_tau,
                     cutoff, seed=seed, gap=None, hop_cutoff=cutoff).build()


# the batch of uneven systems: (diamond multiples, k-mesh, cutoff) and the perovskite
_BATCH3 = [((1, 1, 1), (4, 4, 4), 12.0), ((1, 1, 1), (3, 3, 3), 10.0), ((2, 1, 1), (2, 2, 2), 12.0),
           ((2, 1, 1), (3, 3, 3), 14.0), ((3, 1, 1), (2, 2, 2), 10.0), ((1, 1, 1), (4, 4, 4), 14.0),
           ((2, 2, 1), (2, 2, 2), 12.0), ((3, 1, 1), (3, 3, 3), 12.0), ((4, 1, 1), (2, 2, 2), 10.0),
           ((2, 1, 1), (4, 4, 4), 10.0), ((5, 1, 1), (2, 2, 2), 12.0), ((3, 2, 1), (2, 2, 2), 10.0),
           ((2, 2, 1), (3, 3, 3), 14.0), ((6, 1, 1), (2, 2, 2), 10.0), ((7, 1, 1), (2, 2, 2), 12.0)]


def batch_family(n: int = 16, n_tau: int = 48) -> List[SynthCell]:
    """The batch of uneven systems: 15 diamond-like supercells of 8 to 56 atoms (9 orbitals,
    48 product functions per atom; k-meshes 2x2x2 to 4x4x4, cutoffs 10 to 14 bohr) and the
    56-atom layered perovskite-like cell (perovskite_cell).  Seeds 3000 + index."""
    cells = []
    for i, (mult, km, rc) in enumerate(_BATCH3[:max(0, n - 1)]):
        lat, frac = _diamond_supercell(mult)
        sp = [Species("spd", 9, 48, None)]
        cells.append(SynthCell(f"diamond{len(frac)}-n9-K48-k{km[0]}-rc{rc:g}", lat, frac,
                               np.zeros(len(frac), np.int32), sp, km, 1000.0, n_tau, rc, seed=3000 + i, gap=None,
                               hop_cutoff=rc).build())
    if n >= 16:
        cells.append(perovskite_cell(n_tau=n_tau, seed=3015))
    return cells


def with_far_basis(cell: SynthCell, r_b: float, n_prod_far: Sequence[int],
                   n_prod_near: Optional[Sequence[int]] = None) -> SynthCell:
    """The same cell with reduced product bases for pairs of distinct spheres (inputs only):
    n_prod_far[s] functions per atom of species s beyond a sphere of radius r_b (bohr) and,
    when given, n_prod_near[s] within it (the onsite pairs keep every function)."""
    cell.r_b = float(r_b)
    for sp, f in zip(cell.species, n_prod_far):
        sp.n_prod_far = int(f)
    if n_prod_near is not None:
        for sp, f in zip(cell.species, n_prod_near):
            sp.n_prod_near = int(f)
    cell.name = f"{cell.name}-rb{r_b:g}-K" + "/".join(str(int(f)) for f in n_prod_far) + (
        "" if n_prod_near is None else "-near" + "/".join(str(int(f)) for f in n_prod_near))
    return cell


def chain_cell(n_cells_k: int = 8, t_hop: float = 0.25, beta: float = 20.0, n_tau: int = 24,
               eps0: float = 0.1, seed: int = 7) -> SynthCell:
    """One-band, one-atom chain along x (n = 1, K = 1, C = 1) with nearest-neighbour
    hopping -t: the Lindhard / Fock closed-form test system."""
    lat = np.diag([3.0, 50.0, 50.0])
    sp = [Species("s", 1, 1, np.ones((1, 1, 1)))]
    cell = SynthCell("chain", lat, np.zeros((1, 3)), np.zeros(1, np.int32), sp,
                     (n_cells_k, 1, 1), beta, n_tau, 0.0, seed=seed, gap=None, hop_cutoff=3.5)
    rng = np.random.default_rng(seed)
    cell.hoppings = [(0, 0, (0, 0, 0), np.array([[eps0]], np.complex128)),
                     (0, 0, (1, 0, 0), np.array([[-t_hop]], np.complex128))]
    cell.X_coul = np.array([[1.0]])
    cell.H_k = cell.bloch_hamiltonian()
    e = np.linalg.eigvalsh(cell.H_k)[:, 0]
    cell.mu = float(np.median(e)) + 0.013  # a metal: mu inside the band
    del rng
    return cell


def mixed_species_cell(n_tau: int = 15, kmesh=(2, 2, 2), cutoff: float = 0.0, seed: int = 31,
                       n_orb=(4, 5), n_prod=(8, 19), symmetric_C: bool = True) -> SynthCell:
    """Two species on a simple-cubic a = 5 bohr two-atom cell: ragged blocks
    (n_a != n_b, K_a != K_b, K not a multiple of 16), an odd tau count (the middle
    node is its own mirror) and, optionally, coefficients C not symmetric in (L, L'')."""
    lat = np.eye(3) * 5.0
    frac = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    sp = [Species("A", n_orb[0], n_prod[0], None), Species("B", n_orb[1], n_prod[1], None)]
    cell = SynthCell("mixed2", lat, frac, np.array([0, 1], np.int32), sp, tuple(kmesh), 30.0, n_tau,
                     cutoff, seed=seed, gap=None, hop_cutoff=8.0)
    cell.build()
    if not symmetric_C:
        rng = np.random.default_rng(seed + 1)
        for spc in cell.species:
            spc.C = rng.standard_normal(spc.C.shape) / spc.n_orb
    return cell
