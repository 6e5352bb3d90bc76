"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks one oracle function against something other than itself:
printed worked values, closed forms, an independent library routine, a second
route through the same physics, or an invariant.  No GPU is needed.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# k-mesh rule and pair list (Sec. 2, Fig. 1; worked values in Sec. 3 and Sec. 4)
# ----------------------------------------------------------------------------

def _fcc(a=10.26):
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def test_kmesh_rule_printed_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "kmesh_rule.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        m = np.array([int(x) for x in r[:3]])
        rmax = float(r[3])
        want = tuple(int(x) for x in r[4:7])
        lat = _fcc() * m[:, None]
        assert oracle.kmesh_rule(lat, rmax) == want
    # the totals printed in the paper
    assert np.prod(oracle.kmesh_rule(_fcc(), 14.0)) == 216
    assert np.prod(oracle.kmesh_rule(_fcc(), 10.0)) == 125
    assert np.prod(oracle.kmesh_rule(_fcc() * np.array([4, 3, 3])[:, None], 10.0)) == 18


def _brute_pairs(lat, frac, cutoff, span=4):
    out = set()
    for a in range(len(frac)):
        for b in range(len(frac)):
            for R in np.ndindex(2 * span + 1, 2 * span + 1, 2 * span + 1):
                R = np.array(R) - span
                if np.linalg.norm((R + frac[b] - frac[a]) @ lat) <= cutoff:
                    out.add((a, b) + tuple(int(x) for x in R))
    return out


def test_pair_list_equals_brute_force_when_mesh_obeys_rule():
    # simple cubic a = 5, two atoms, cutoff 9: rule gives ceil(18/5)+1 = 5 -> 5x5x5 is alias free
    lat = np.eye(3) * 5.0
    frac = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])
    assert oracle.kmesh_rule(lat, 9.0) == (5, 5, 5)
    ent = oracle.pair_list(lat, frac, (5, 5, 5), 9.0)
    got = {(int(r[0]), int(r[1]), int(r[5]), int(r[6]), int(r[7])) for r in ent}
    assert got == _brute_pairs(lat, frac, 9.0)
    assert len(got) == len(ent)
    # class of the representative is the stored class
    assert np.all(np.mod(ent[:, 5:8], 5) == ent[:, 2:5])


def test_pair_list_diamond_count_and_symmetry():
    cell = synth.make_config(1, build=False)
    ent = oracle.pair_list(cell.lattice, cell.frac, cell.kmesh, cell.cutoff)
    brute = _brute_pairs(cell.lattice, cell.frac, cell.cutoff, span=2)
    assert len(ent) == len(brute) == 376
    keys = {(int(r[0]), int(r[1]), int(r[5]), int(r[6]), int(r[7])) for r in ent}
    for a, b, r1, r2, r3 in keys:
        assert (b, a, -r1, -r2, -r3) in keys


def test_pair_list_keeps_all_classes_without_cutoff():
    cell = synth.make_config(0, build=False)
    ent = oracle.pair_list(cell.lattice, cell.frac, cell.kmesh, 0.0)
    assert len(ent) == 2 * 2 * 8
    # a tie: classes at distance a from the same atom have two images (+-5); the smaller R wins
    same = ent[(ent[:, 0] == 0) & (ent[:, 1] == 0)]
    row = same[(same[:, 2] == 1) & (same[:, 3] == 0) & (same[:, 4] == 0)][0]
    assert tuple(row[5:8]) == (-1, 0, 0)


# ----------------------------------------------------------------------------
# G0(k, tau): closed form against the matrix exponential, invariants
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cell0():
    return synth.make_config(0)


def test_green0_against_expm(cell0):
    H = cell0.H_k
    mu, beta = cell0.mu, 8.0  # moderate beta so that expm stays well scaled
    tau = np.array([0.0, 0.7, 3.1, 8.0])
    G = oracle.green0_k_tau(H, mu, beta, tau)
    I = np.eye(H.shape[1])
    for k in range(H.shape[0]):
        h = H[k] - mu * I
        inv = np.linalg.inv(I + expm(-beta * h))
        for i, t in enumerate(tau):
            ref = -expm(-t * h) @ inv
            assert np.abs(G[k, i] - ref).max() < 1e-12


def test_green0_invariants(cell0):
    c = cell0
    tau = c.tau
    G = oracle.green0_k_tau(c.H_k, c.mu, c.beta, tau)
    I = np.eye(c.n_orb_total)
    # jump G(0+) + G(beta-) = -S^{-1} = -I
    assert np.abs(G[:, 0] + G[:, -1] + I[None]).max() < 1e-13
    # Hermitian at every tau
    assert np.abs(G - G.conj().transpose(0, 1, 3, 2)).max() < 1e-14
    # antiperiodicity G(tau - beta) = -G(tau)
    t = np.array([3.3, 17.0, 41.2])
    Gp = oracle.green0_k_tau(c.H_k, c.mu, c.beta, t)
    Gm = oracle.green0_k_tau(c.H_k, c.mu, c.beta, t - c.beta)
    assert np.abs(Gp + Gm).max() < 1e-13
    # particle number: s * (1/N_k) sum_k tr rho(k) = N_e with rho = -G(beta-), half filling
    n = c.spin * np.real(np.trace(-G[:, -1], axis1=1, axis2=2)).sum() / c.n_k
    e = np.linalg.eigvalsh(c.H_k)
    nref = c.spin * synth.fermi(e - c.mu, c.beta).sum() / c.n_k
    assert abs(n - nref) < 1e-12
    assert abs(n - c.n_orb_total) < 1e-6
    # the generator's input G is this G0
    assert np.abs(c.green_k_tau() - G).max() < 1e-13


# ----------------------------------------------------------------------------
# R <-> k transforms against numpy's FFT and a round trip
# ----------------------------------------------------------------------------

def test_fourier_matches_fft_and_round_trips(cell0):
    c = cell0
    ent = oracle.pair_list(c.lattice, c.frac, c.kmesh, 0.0)
    G = oracle.green0_k_tau(c.H_k, c.mu, c.beta, c.tau[:3])
    oo = c.orb_offsets
    GR = oracle.fourier_k_to_R(G, ent, c.kmesh, oo, oo)
    # numpy FFT of the (a, b) = (0, 1) block: F(R) = (1/N) sum_k e^{-ikR} F(k) = ifftn over k
    blk = G[:, :, oo[0]:oo[1], oo[1]:oo[2]].reshape(c.kmesh + (3, 4, 4))
    ref = np.fft.ifftn(blk, axes=(0, 1, 2))
    for e, row in enumerate(ent):
        if row[0] == 0 and row[1] == 1:
            assert np.abs(GR[e] - ref[tuple(row[2:5])]).max() < 1e-15
    back = oracle.fourier_R_to_k(GR, ent, c.kmesh, oo, oo)
    assert np.abs(back - G).max() < 1e-14
    # Hermiticity in R: G_ba(-R) = G_ab(R)^dagger
    key = {(int(r[0]), int(r[1]), tuple(int(x) for x in r[2:5])): e for e, r in enumerate(ent)}
    for e, r in enumerate(ent):
        mc = tuple(int(x) for x in np.mod(-r[2:5], c.kmesh))
        e2 = key[(int(r[1]), int(r[0]), mc)]
        assert np.abs(GR[e2] - GR[e].conj().transpose(0, 2, 1)).max() < 1e-15


# ----------------------------------------------------------------------------
# polarizability: Lindhard closed form, second route, invariants
# ----------------------------------------------------------------------------

def test_polarizability_lindhard_chain_tau():
    ch = synth.chain_cell(n_cells_k=8, beta=20.0, n_tau=24)
    ent = oracle.pair_list(ch.lattice, ch.frac, ch.kmesh, 0.0)
    G = oracle.green0_k_tau(ch.H_k, ch.mu, ch.beta, ch.tau)
    GR = oracle.fourier_k_to_R(G, ent, ch.kmesh, [0, 1], [0, 1])
    PR = oracle.polarizability_R(GR, ent, [np.ones((1, 1, 1))], spin=2)
    Pq = oracle.fourier_R_to_k(PR, ent, ch.kmesh, [0, 1], [0, 1])[:, :, 0, 0]
    xi = np.linalg.eigvalsh(ch.H_k)[:, 0] - ch.mu
    f = synth.fermi(xi, ch.beta)
    N = ch.n_k
    for q in range(N):
        for i, t in enumerate(ch.tau):
            ref = 0.0
            for k in range(N):
                kq = (k - q) % N
                # (1 - f_k) e^{-xi_k t} f_kq e^{+xi_kq t}, each factor in its bounded form
                ref += (1.0 / (math.exp(xi[k] * t) + math.exp(xi[k] * (t - ch.beta)))
                        / (math.exp(xi[kq] * (ch.beta - t)) + math.exp(-xi[kq] * t)))
            ref *= -2.0 / N
            assert abs(Pq[q, i] - ref) < 1e-14 * max(1.0, abs(ref)) * 4


def test_polarizability_real_space_equals_kspace_route(cell0):
    c = cell0
    ent = oracle.pair_list(c.lattice, c.frac, c.kmesh, 0.0)
    G = c.green_k_tau()
    oo, po = c.orb_offsets, c.pb_offsets
    C = [c.species[s].C for s in c.species_of_atom]
    PR = oracle.polarizability_R(oracle.fourier_k_to_R(G, ent, c.kmesh, oo, oo), ent, C)
    Pq_real = oracle.fourier_R_to_k(PR, ent, c.kmesh, po, po)
    Pq_k = oracle.polarizability_q_kspace(G, C, oo, po, c.kmesh)
    assert np.abs(Pq_real - Pq_k).max() < 1e-14 * np.abs(Pq_k).max() * 10


def test_polarizability_invariants(cell0):
    c = cell0
    ent = oracle.pair_list(c.lattice, c.frac, c.kmesh, 0.0)
    G = c.green_k_tau()
    oo, po = c.orb_offsets, c.pb_offsets
    C = [c.species[s].C for s in c.species_of_atom]
    PR = oracle.polarizability_R(oracle.fourier_k_to_R(G, ent, c.kmesh, oo, oo), ent, C)
    scale = max(np.abs(p).max() for p in PR)
    key = {(int(r[0]), int(r[1]), tuple(int(x) for x in r[2:5])): e for e, r in enumerate(ent)}
    for e, r in enumerate(ent):
        # P(beta - tau) = P(tau)^* for C symmetric in (L, L'')
        assert np.abs(PR[e][::-1] - PR[e].conj()).max() < 1e-14 * scale
        # P_ba(-R) = P_ab(R)^dagger
        e2 = key[(int(r[1]), int(r[0]), tuple(int(x) for x in np.mod(-r[2:5], c.kmesh)))]
        assert np.abs(PR[e2] - PR[e].conj().transpose(0, 2, 1)).max() < 1e-14 * scale
    # P(q, i nu = 0) is Hermitian negative semidefinite
    B = oracle.fourier_matrix(c.beta, c.tau, np.array([0]), "B")
    P0 = oracle.fourier_R_to_k(oracle.transform(B, PR), ent, c.kmesh, po, po)[:, 0]
    for q in range(c.n_k):
        assert np.abs(P0[q] - P0[q].conj().T).max() < 1e-12 * np.abs(P0[q]).max()
        assert np.linalg.eigvalsh(0.5 * (P0[q] + P0[q].conj().T)).max() < 1e-10 * np.abs(P0[q]).max()


def test_polarizability_complete_product_basis():
    # K = n^2 and C_{(L1 L2); L L''} = delta_{L1 L} delta_{L2 L''}: P is the orbital product
    rng = np.random.default_rng(3)
    n, nt = 3, 6
    G = rng.standard_normal((nt, n, n)) + 1j * rng.standard_normal((nt, n, n))
    C = np.zeros((n * n, n, n))
    for L1 in range(n):
        for L2 in range(n):
            C[L1 * n + L2, L1, L2] = 1.0
    ent = np.array([[0, 0, 0, 0, 0, 0, 0, 0]])
    P = oracle.polarizability_R([G], ent, [C], spin=2)[0]
    for t in range(nt):
        assert np.abs(P[t] + 2.0 * np.kron(G[t], np.conj(G[nt - 1 - t]))).max() < 1e-14


# ----------------------------------------------------------------------------
# tau <-> i omega matrices: exactness on polynomials, high precision, round trip
# ----------------------------------------------------------------------------

def _poly_moment(m, w, beta):
    """int_0^beta tau^m e^{i w tau} d tau by repeated integration by parts (w != 0)."""
    iw = 1j * w
    s = 0.0
    for j in range(m + 1):
        s += (-1) ** j * math.factorial(m) / math.factorial(m - j) * beta ** (m - j) / iw ** (j + 1)
    val = np.exp(iw * beta) * s - (-1) ** m * math.factorial(m) / iw ** (m + 1)
    return val


@pytest.mark.parametrize("stat", ["F", "B"])
def test_transform_exact_on_polynomials(stat):
    beta, N = 37.0, 24
    tau = synth.tau_nodes(beta, N)
    fer, bos = synth.matsubara_sets(N)
    idx = fer if stat == "F" else bos
    T = oracle.fourier_matrix(beta, tau, idx, stat)
    for m in range(5):
        g = tau ** m
        got = T @ g
        for r, n in enumerate(idx):
            w = (2 * n + 1) * np.pi / beta if stat == "F" else 2 * n * np.pi / beta
            ref = beta ** (m + 1) / (m + 1) if w == 0 else _poly_moment(m, w, beta)
            assert abs(got[r] - ref) < 1e-12 * beta ** (m + 1)


def test_transform_matrix_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    beta, N = 50.0, 24
    tau = synth.tau_nodes(beta, N)
    fer, _ = synth.matsubara_sets(N)
    idx = np.array([fer[0], 0, 40])  # includes the largest |n| of the set
    T = oracle.fourier_matrix(beta, tau, idx, "F")
    tmax = np.abs(oracle.fourier_matrix(beta, tau, fer, "F")).max()
    # the nodes as the oracle holds them (x = 2 tau / beta - 1 in float64): the Lagrange
    # basis is sensitive to node rounding at the ~N^2 eps level, the quadrature is not
    xs = [mp.mpf(float(v)) for v in 2.0 * tau / beta - 1.0]
    for r, n in enumerate(idx):
        a = mp.mpf(2 * int(n) + 1) * mp.pi / 2
        for i in (0, N // 2, N - 1):
            def li(x, i=i):
                p = mp.mpf(1)
                for j in range(N):
                    if j != i:
                        p *= (x - xs[j]) / (xs[i] - xs[j])
                return p
            val = mp.quad(lambda x: mp.expj(a * x) * li(x), mp.linspace(-1, 1, 81))
            ref = complex(mp.mpf(beta) / 2 * mp.expj(a) * val)
            # float64 floor: rounded quadrature nodes meet Lagrange slopes ~N^2 and the
            # phase a*x, so agreement is ~eps (N^2 + |a|) relative to max |T|
            assert abs(T[r, i] - ref) < 2.3e-16 * (N * N + abs(float(a))) * tmax


def test_transform_round_trip_and_conditioning():
    for N in (24, 48, 64):
        tau = synth.tau_nodes(1000.0, N)
        fer, bos = synth.matsubara_sets(N)
        for idx, st in ((fer, "F"), (bos, "B")):
            T = oracle.fourier_matrix(1000.0, tau, idx, st)
            U = oracle.inverse_matrix(T)
            assert np.abs(U @ T - np.eye(N)).max() < 1e-11
            assert np.linalg.cond(T) < 1e4


def test_transform_converges_to_single_pole():
    # g(tau) = -e^{-xi tau}/(1+e^{-beta xi}) has g(i w_n) = 1/(i w_n - xi)
    beta, xi = 10.0, 0.3
    for N, tol in ((24, 1e-3), (48, 1e-6), (64, 1e-9)):
        tau = synth.tau_nodes(beta, N)
        fer, _ = synth.matsubara_sets(N)
        T = oracle.fourier_matrix(beta, tau, fer, "F")
        g = -np.exp(-xi * tau) / (1 + np.exp(-beta * xi))
        w = (2 * fer + 1) * np.pi / beta
        err = np.abs(T @ g - 1.0 / (1j * w - xi)).max()
        assert err < tol, (N, err)


# ----------------------------------------------------------------------------
# screened interaction
# ----------------------------------------------------------------------------

def _one_entry_system(v, P):
    """One atom, one pair class, K x K blocks: P(q) = P(R=0), W~(R=0) = W~(q)."""
    ent = np.array([[0, 0, 0, 0, 0, 0, 0, 0]])
    return ent, [P[None]], v[None]


def test_screened_W_scalar_closed_form():
    v, p = 0.7, -0.35
    ent, PR, vq = _one_entry_system(np.array([[v]], complex), np.array([[p]], complex))
    WR, _ = oracle.screened_W(PR, ent, vq, (1, 1, 1), [0, 1])
    assert abs(WR[0][0, 0, 0] - v * v * p / (1 - v * p)) < 1e-15


def test_screened_W_neumann_series():
    rng = np.random.default_rng(5)
    K = 6
    A = rng.standard_normal((K, K))
    v = (A @ A.T / K + np.eye(K)).astype(complex)
    P = 1e-4 * (rng.standard_normal((K, K)) + 1j * rng.standard_normal((K, K)))
    ent, PR, vq = _one_entry_system(v, P)
    WR, _ = oracle.screened_W(PR, ent, vq, (1, 1, 1), [0, K])
    ref = v @ P @ v + v @ P @ v @ P @ v
    assert np.abs(WR[0][0] - ref).max() < 10 * np.abs(v @ P @ v @ P @ v @ P @ v).max()
    # the leading term alone misses the second order by its size
    assert np.abs(WR[0][0] - v @ P @ v).max() > 0.5 * np.abs(v @ P @ v @ P @ v).max()


def test_screened_W_screens_static(cell0):
    # P(q, 0) <= 0 and v > 0 give W(q, 0) = v + W~ <= v  (screening)
    c = cell0
    ent = oracle.pair_list(c.lattice, c.frac, c.kmesh, 0.0)
    sysm = oracle.OracleSystem(c, ent)
    vq, vc = c.coulomb()
    G = c.green_k_tau()
    PR = oracle.polarizability_R(oracle.fourier_k_to_R(G, ent, c.kmesh, c.orb_offsets, c.orb_offsets), ent, sysm.C_atom)
    i0 = int(np.nonzero(c.nu_idx == 0)[0][0])
    Piw = [x[i0:i0 + 1] for x in oracle.transform(sysm.B_fwd, PR)]
    _, Wq = oracle.screened_W(Piw, ent, vq, c.kmesh, c.pb_offsets)
    for q in range(c.n_k):
        Wt = Wq[q, 0]
        assert np.linalg.eigvalsh(0.5 * (Wt + Wt.conj().T)).max() < 1e-12


# ----------------------------------------------------------------------------
# self-energy: Fock closed form, second route, invariants
# ----------------------------------------------------------------------------

def test_exchange_fock_chain():
    ch = synth.chain_cell(n_cells_k=8, beta=20.0, n_tau=12)
    ent = oracle.pair_list(ch.lattice, ch.frac, ch.kmesh, 0.0)
    G = oracle.green0_k_tau(ch.H_k, ch.mu, ch.beta, ch.tau)
    GR = oracle.fourier_k_to_R(G, ent, ch.kmesh, [0, 1], [0, 1])
    N = ch.n_k
    vcls = np.array([1.0 / (1.0 + abs(min(c, N - c)) * 3.0) for c in range(N)])
    vR = [np.array([[vcls[int(r[2])]]], complex) for r in ent]
    SxR = oracle.exchange_R(GR, vR, ent, [np.ones((1, 1, 1))])
    Sxk = oracle.fourier_R_to_k([s[None] for s in SxR], ent, ch.kmesh, [0, 1], [0, 1])[:, 0, 0, 0]
    vq = np.array([sum(vcls[c] * np.exp(2j * np.pi * q * c / N) for c in range(N)) for q in range(N)])
    f = synth.fermi(np.linalg.eigvalsh(ch.H_k)[:, 0] - ch.mu, ch.beta)
    for k in range(N):
        ref = -sum(vq[q] * f[(k - q) % N] for q in range(N)) / N
        assert abs(Sxk[k] - ref) < 1e-14


def _complete_basis(n):
    """K = n^2 product functions with C_{(L1 L2); L L''} = delta_{L1 L} delta_{L2 L''} (not
    symmetric in (L, L''))."""
    C = np.zeros((n * n, n, n))
    for L1 in range(n):
        for L2 in range(n):
            C[L1 * n + L2, L1, L2] = 1.0
    return C


def test_self_energy_complete_product_basis():
    """Eq. S_MM with a complete product basis on both atoms reduces to the orbital-pair
    form of Eq. S_II: Sigma_{L L'}(tau) = -sum_{L'' L'''} G_{L'' L'''}(tau) W~_{(L L''), (L' L''')}(tau).
    Atoms with different orbital counts, a non-Hermitian W~ and coefficients that are not
    symmetric in (L, L''), so a transposed W~ block or a C contracted on the wrong index shows."""
    rng = np.random.default_rng(17)
    na, nb, nt = 2, 3, 5
    G = rng.standard_normal((nt, na, nb)) + 1j * rng.standard_normal((nt, na, nb))
    W = rng.standard_normal((nt, na * na, nb * nb)) + 1j * rng.standard_normal((nt, na * na, nb * nb))
    ent = np.array([[0, 1, 0, 0, 0, 0, 0, 0]])
    S = oracle.self_energy_R([G], [W], ent, [_complete_basis(na), _complete_basis(nb)])[0]
    ref = np.zeros((nt, na, nb), complex)
    for t in range(nt):
        for L in range(na):
            for Lp in range(nb):
                s = 0j
                for L2 in range(na):
                    for L3 in range(nb):
                        s += G[t, L2, L3] * W[t, L * na + L2, Lp * nb + L3]
                ref[t, L, Lp] = -s
    assert np.abs(S - ref).max() < 1e-14 * np.abs(ref).max()


def test_exchange_complete_product_basis():
    """The exchange rule (W~ -> v, G(tau) -> -G(beta-)) in a complete product basis:
    Sigma_x,{L L'} = +sum_{L'' L'''} G_{L'' L'''}(beta-) v_{(L L''), (L' L''')}."""
    rng = np.random.default_rng(19)
    na, nb, nt = 3, 2, 4
    G = rng.standard_normal((nt, na, nb)) + 1j * rng.standard_normal((nt, na, nb))
    v = rng.standard_normal((na * na, nb * nb)) + 1j * rng.standard_normal((na * na, nb * nb))
    ent = np.array([[0, 1, 0, 0, 0, 0, 0, 0]])
    Sx = oracle.exchange_R([G], [v], ent, [_complete_basis(na), _complete_basis(nb)])[0]
    ref = np.zeros((na, nb), complex)
    for L in range(na):
        for Lp in range(nb):
            for L2 in range(na):
                for L3 in range(nb):
                    ref[L, Lp] += G[nt - 1, L2, L3] * v[L * na + L2, Lp * nb + L3]
    assert np.abs(Sx - ref).max() < 1e-14 * np.abs(ref).max()


def _single_pole_chain(n_tau=64):
    """One-band chain with a screened interaction of one bosonic pole per class R:
    W~(R, i nu) = A(R) 2 Omega / (nu^2 + Omega^2), i.e. W~(R, tau) = A(R) w(tau) with
    w(tau) = (e^{-Omega tau} + e^{-Omega (beta - tau)}) / (1 - e^{-beta Omega})."""
    ch = synth.chain_cell(n_cells_k=8, beta=20.0, n_tau=n_tau)
    ent = oracle.pair_list(ch.lattice, ch.frac, ch.kmesh, 0.0)
    N = ch.n_k
    A = np.array([0.4 / (1.0 + min(c, N - c)) for c in range(N)])  # A(R) = A(-R): A_q real
    return ch, ent, A, 0.35


def _single_pole_w(beta, Om, tau, bos):
    nu = 2 * np.pi * np.asarray(bos) / beta
    return 2 * Om / (nu ** 2 + Om ** 2), (np.exp(-Om * tau) + np.exp(-Om * (beta - tau))) / (1 - np.exp(-beta * Om))


def test_bosonic_inverse_transform_of_a_single_pole():
    """Appendix A grid, bosonic side: the least-squares inverse maps the exact Matsubara
    values w(i nu_m) = 2 Omega / (nu_m^2 + Omega^2) of the bosonic function
    w(tau) = (e^{-Omega tau} + e^{-Omega (beta - tau)}) / (1 - e^{-beta Omega}) back to w at the
    tau nodes; a grid too coarse for the pole fails."""
    beta, Om = 20.0, 0.35
    errs = {}
    for N in (12, 48, 64):
        tau = synth.tau_nodes(beta, N)
        _, bos = synth.matsubara_sets(N)
        U = oracle.inverse_matrix(oracle.fourier_matrix(beta, tau, bos, "B"))
        w_iv, w_tau = _single_pole_w(beta, Om, tau, bos)
        errs[N] = np.abs(U @ w_iv - w_tau).max() / np.abs(w_tau).max()
    assert errs[64] < 1e-10 and errs[48] < 1e-8, errs
    assert errs[12] > 1e-6, errs


def _single_pole_sigma_iw(ch, A, Om, omega_idx):
    """Sigma(k, i w_n) of the one-band G0 and the single-pole W~ by residues:
    Sigma(k, tau) = -(1/N) sum_k' G0(k', tau) W~(k - k', tau), G0(k', tau) = -e^{-xi tau}/(1 + e^{-beta xi}),
    W~(q, tau) = A_q w(tau), each exponential integrated in closed form,
    int_0^beta e^{(i w - x) tau} d tau = (1 + e^{-beta x}) / (x - i w) for fermionic w."""
    beta, N = ch.beta, ch.n_k
    xi = np.linalg.eigvalsh(ch.H_k)[:, 0] - ch.mu
    Aq = np.array([sum(A[c] * np.exp(2j * np.pi * q * c / N) for c in range(N)) for q in range(N)])
    w = (2 * np.asarray(omega_idx) + 1) * np.pi / beta
    I = lambda y: (1 + np.exp(-beta * y)) / (y - 1j * w)
    out = np.zeros((N, len(w)), complex)
    for k in range(N):
        for kp in range(N):
            x = xi[kp]
            out[k] += Aq[(k - kp) % N] / ((1 + np.exp(-beta * x)) * (1 - np.exp(-beta * Om))) * (
                I(x + Om) + np.exp(-beta * Om) * I(x - Om))
    return out / N


def test_self_energy_single_pole_closed_form():
    """Eq. S_MM on the one-band chain with a single-pole W~(i nu): the oracle's chain
    W~(R, i nu) -> W~(R, tau) (bosonic inverse) -> Sigma(R, tau) -> Sigma(R, i w) (fermionic
    forward) -> Sigma(k, i w) against the residue closed form of the Matsubara sum."""
    ch, ent, A, Om = _single_pole_chain(64)
    beta, tau = ch.beta, ch.tau
    fer, bos = synth.matsubara_sets(ch.n_tau)
    G = oracle.green0_k_tau(ch.H_k, ch.mu, beta, tau)
    GR = oracle.fourier_k_to_R(G, ent, ch.kmesh, [0, 1], [0, 1])
    w_iv, _ = _single_pole_w(beta, Om, tau, bos)
    W_iv = [(A[int(r[2])] * w_iv).astype(complex)[:, None, None] for r in ent]
    WR = oracle.transform(oracle.inverse_matrix(oracle.fourier_matrix(beta, tau, bos, "B")), W_iv)
    F = oracle.fourier_matrix(beta, tau, fer, "F")
    ref = _single_pole_sigma_iw(ch, A, Om, fer)

    def sigma_k(G_R):
        SR = oracle.self_energy_R(G_R, WR, ent, [np.ones((1, 1, 1))])
        return oracle.fourier_R_to_k(oracle.transform(F, SR), ent, ch.kmesh, [0, 1], [0, 1])[:, :, 0, 0]

    assert np.abs(sigma_k(GR) - ref).max() < 1e-9 * np.abs(ref).max()
    # the closed form fixes the pairing of Eq. S_MM: G taken at beta - tau is far off
    # (W~ is mirror symmetric in tau, G is not)
    assert np.abs(sigma_k([g[::-1] for g in GR]) - ref).max() > 1e-2 * np.abs(ref).max()


def test_self_energy_real_space_equals_kspace_route(cell0):
    c = cell0
    ent = oracle.pair_list(c.lattice, c.frac, c.kmesh, 0.0)
    G = c.green_k_tau()
    oo, po = c.orb_offsets, c.pb_offsets
    C = [c.species[s].C for s in c.species_of_atom]
    rng = np.random.default_rng(11)
    # an arbitrary W~(q, tau) with the Hermitian symmetry of a screened interaction
    Wq = rng.standard_normal((c.n_k, c.n_tau, c.n_pb_total, c.n_pb_total)) * (1 + 0j)
    Wq = Wq + 1j * rng.standard_normal(Wq.shape)
    WR = oracle.fourier_k_to_R(Wq, ent, c.kmesh, po, po)
    GR = oracle.fourier_k_to_R(G, ent, c.kmesh, oo, oo)
    SR = oracle.self_energy_R(GR, WR, ent, C)
    Sk_real = oracle.fourier_R_to_k(SR, ent, c.kmesh, oo, oo)
    Sk = oracle.self_energy_k_kspace(G, Wq, C, oo, po, c.kmesh)
    assert np.abs(Sk_real - Sk).max() < 1e-13 * np.abs(Sk).max()


def test_self_energy_hermiticity(cell0):
    c = cell0
    sysm = oracle.OracleSystem(c)
    vq, vc = c.coulomb()
    r = sysm.sweep(c.green_k_tau(), vq, vc)
    ent = sysm.entries
    key = {(int(x[0]), int(x[1]), tuple(int(y) for y in x[2:5])): e for e, x in enumerate(ent)}
    sc = max(np.abs(s).max() for s in r["Sig_R"])
    sx = max(np.abs(s).max() for s in r["Sigx_R"])
    for e, x in enumerate(ent):
        e2 = key[(int(x[1]), int(x[0]), tuple(int(y) for y in np.mod(-x[2:5], c.kmesh)))]
        assert np.abs(r["Sig_R"][e2] - r["Sig_R"][e].conj().transpose(0, 2, 1)).max() < 1e-11 * sc
        assert np.abs(r["Sigx_R"][e2] - r["Sigx_R"][e].conj().T).max() < 1e-13 * sx
    # Sigma_x(k) Hermitian and negative semidefinite for the positive v used here? Only Hermitian.
    for k in range(c.n_k):
        assert np.abs(r["Sigx_k"][k] - r["Sigx_k"][k].conj().T).max() < 1e-13 * sx


def test_self_energy_vanishes_without_screening(cell0):
    c = cell0
    sysm = oracle.OracleSystem(c)
    G = c.green_k_tau()
    GR = oracle.fourier_k_to_R(G, sysm.entries, c.kmesh, c.orb_offsets, c.orb_offsets)
    WR = [np.zeros((c.n_tau, 8, 8), complex) for _ in sysm.entries]
    SR = oracle.self_energy_R(GR, WR, sysm.entries, sysm.C_atom)
    assert max(np.abs(s).max() for s in SR) == 0.0


def test_w_solve_amplifies_errors_of_p():
    """Conditioning of the chain P -> W~ (oracle only): a relative perturbation of
    1e-7 in P(R, tau) moves W~(R, tau) by 1e-6 .. 1e-3 relative on the 8-atom cell
    (short cutoff, 2x2x2 mesh).  This fixes the tolerance of a mixed-precision chain."""
    c = synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2))
    orc = oracle.OracleSystem(c)
    G = c.green_k_tau()
    vq, _ = c.coulomb()
    GR = oracle.fourier_k_to_R(G, orc.entries, orc.kmesh, c.orb_offsets, c.orb_offsets)
    PR = oracle.polarizability_R(GR, orc.entries, orc.C_atom)
    rng = np.random.default_rng(0)
    PRn = [p * (1 + 1e-7 * rng.standard_normal(p.shape)) for p in PR]

    def w_tau(P):
        Wiw, _ = oracle.screened_W(oracle.transform(orc.B_fwd, P), orc.entries, vq, orc.kmesh, c.pb_offsets)
        return np.concatenate([x.ravel() for x in oracle.transform(orc.B_inv, Wiw)])

    a, b = w_tau(PRn), w_tau(PR)
    amp = np.linalg.norm(a - b) / np.linalg.norm(b) / 1e-7
    assert 10.0 < amp < 1e4, amp


# ----------------------------------------------------------------------------
# Reduced product basis beyond sphere B (Sec. 2, Fig. 2; worked values in Sec. 3)
# ----------------------------------------------------------------------------

def _far_cells(r_b=4.0, n_far=3):
    """cell0 twice from the same seed: with the reduced basis beyond r_b, and without."""
    full = synth.make_config(0)
    tier = synth.with_far_basis(synth.make_config(0), r_b, [n_far])
    assert np.array_equal(full.species[0].C, tier.species[0].C)
    return full, tier


def test_far_basis_storage_ratio_printed_in_sec3():
    row = [l.split() for l in open(os.path.join(GOLDEN, "far_basis_ratios.txt")) if l.strip() and not l.startswith("#")]
    r_b, r_c, shell, l_b, l_c, storage = (float(x) for x in row[0])
    assert abs((r_c ** 3 - r_b ** 3) / r_b ** 3 - shell) < 0.5
    # product functions per atom ~ (L + 1)^2: a near and a far entry of one atom pair
    ent = np.array([[0, 0, 0, 0, 0, 0, 0, 0], [0, 0, 1, 0, 0, 1, 0, 0]], np.int64)
    dims = oracle.entry_pb_dims(ent, np.array([False, True]), [int((l_b + 1) ** 2)], [int((l_c + 1) ** 2)])
    ratio = (dims[0][0] * dims[0][1]) / (dims[1][0] * dims[1][1])
    assert math.isclose(ratio, ((l_b + 1) / (l_c + 1)) ** 4, rel_tol=1e-15)
    assert abs(ratio - storage) < 0.5


def test_far_basis_tiers_by_distance():
    full, tier = _far_cells()
    orc = oracle.OracleSystem(tier)
    ent = orc.entries
    # sc a = 5 with atoms at 0 and the cube centre: onsite 0, A-B 4.33, A-A' 5 bohr
    for e, row in enumerate(ent):
        onsite = row[0] == row[1] and not row[5:8].any()
        assert orc.far[e] == (not onsite)
        assert orc.kdims[e] == ((8, 8) if onsite else (3, 3))
    assert not oracle.OracleSystem(full).far.any()


def test_far_basis_equals_masked_full_basis():
    """The reduced basis against a second route: the full-basis oracle with every
    dropped row and column of P, W~ and v set to zero (Sec. 2: the two-point functions
    of distant pairs live in the smaller basis)."""
    full, tier = _far_cells()
    of, ot = oracle.OracleSystem(full), oracle.OracleSystem(tier)
    Gk = full.green_k_tau()
    vq, vcls = full.coulomb()
    ent, po = of.entries, full.pb_offsets
    GR = oracle.fourier_k_to_R(Gk, ent, of.kmesh, full.orb_offsets, full.orb_offsets)

    def mask(blocks):
        out = []
        for e, b in enumerate(blocks):
            m = np.zeros_like(b)
            ka, kb = ot.kdims[e]
            m[..., :ka, :kb] = b[..., :ka, :kb]
            out.append(m)
        return out

    Pf = oracle.polarizability_R(GR, ent, of.C_atom, full.spin)
    Pt = oracle.polarizability_R(GR, ent, ot.C_atom, tier.spin, ot.kdims)
    for e in range(len(ent)):
        ka, kb = ot.kdims[e]
        assert Pt[e].shape[1:] == (ka, kb)
        assert np.abs(Pt[e] - Pf[e][:, :ka, :kb]).max() <= 1e-14 * np.abs(Pf[e]).max()
    Wt_iw, Wq_t = oracle.screened_W(oracle.transform(ot.B_fwd, Pt), ent, vq, ot.kmesh, po)
    Wm_iw, Wq_m = oracle.screened_W(oracle.transform(of.B_fwd, mask(Pf)), ent, vq, of.kmesh, po)
    assert np.abs(Wq_t - Wq_m).max() <= 1e-12 * np.abs(Wq_m).max()
    for e in range(len(ent)):
        ka, kb = ot.kdims[e]
        assert np.abs(Wt_iw[e] - Wm_iw[e][:, :ka, :kb]).max() <= 1e-12 * np.abs(Wm_iw[e]).max()
    WtR = oracle.transform(ot.B_inv, Wt_iw)
    WmR = mask(oracle.transform(of.B_inv, Wm_iw))
    St = oracle.self_energy_R(GR, WtR, ent, ot.C_atom)
    Sm = oracle.self_energy_R(GR, WmR, ent, of.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(St, Sm)) <= 1e-12 * max(np.abs(b).max() for b in Sm)
    Xt = oracle.exchange_R(GR, ot.v_R(vcls), ent, ot.C_atom)
    Xm = oracle.exchange_R(GR, mask(of.v_R(vcls)), ent, of.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(Xt, Xm)) <= 1e-12 * max(np.abs(b).max() for b in Xm)
    # and the reduction changes the answer (the test would be empty otherwise)
    Sf = oracle.self_energy_R(GR, oracle.transform(of.B_inv, oracle.screened_W(
        oracle.transform(of.B_fwd, Pf), ent, vq, of.kmesh, po)[0]), ent, of.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(St, Sf)) > 1e-6 * max(np.abs(b).max() for b in Sf)


def _three_level_cells(r_b=4.6, n_near=5, n_far=3):
    """cell0 twice from the same seed: with the three levels of Fig. 2 (onsite 8 functions,
    the A-B neighbour at 4.33 bohr inside sphere B keeps n_near, the A-A' image at 5 bohr
    beyond it n_far), and with the full basis everywhere."""
    full = synth.make_config(0)
    tier = synth.with_far_basis(synth.make_config(0), r_b, [n_far], n_prod_near=[n_near])
    return full, tier


def test_three_levels_by_distance():
    full, tier = _three_level_cells()
    orc = oracle.OracleSystem(tier)
    for e, row in enumerate(orc.entries):
        onsite = row[0] == row[1] and not row[5:8].any()
        near = row[0] != row[1]  # a-b: the cube centre at 4.33 bohr (every class here)
        assert orc.tier[e] == (0 if onsite else 1 if near else 2)
        assert orc.kdims[e] == ((8, 8) if onsite else (5, 5) if near else (3, 3))
    assert set(orc.tier) == {0, 1, 2}


def test_three_levels_equal_masked_full_basis():
    """Three basis sizes against the full-basis oracle with the dropped rows and columns of
    P, W~ and v set to zero, level by level."""
    full, tier = _three_level_cells()
    of, ot = oracle.OracleSystem(full), oracle.OracleSystem(tier)
    Gk = full.green_k_tau()
    vq, vcls = full.coulomb()
    ent, po = of.entries, full.pb_offsets
    GR = oracle.fourier_k_to_R(Gk, ent, of.kmesh, full.orb_offsets, full.orb_offsets)

    def mask(blocks):
        out = []
        for e, b in enumerate(blocks):
            m = np.zeros_like(b)
            ka, kb = ot.kdims[e]
            m[..., :ka, :kb] = b[..., :ka, :kb]
            out.append(m)
        return out

    Pf = oracle.polarizability_R(GR, ent, of.C_atom, full.spin)
    Pt = oracle.polarizability_R(GR, ent, ot.C_atom, tier.spin, ot.kdims)
    for e in range(len(ent)):
        ka, kb = ot.kdims[e]
        assert np.abs(Pt[e] - Pf[e][:, :ka, :kb]).max() <= 1e-14 * np.abs(Pf[e]).max()
    Wt_iw, Wq_t = oracle.screened_W(oracle.transform(ot.B_fwd, Pt), ent, vq, ot.kmesh, po)
    Wm_iw, Wq_m = oracle.screened_W(oracle.transform(of.B_fwd, mask(Pf)), ent, vq, of.kmesh, po)
    assert np.abs(Wq_t - Wq_m).max() <= 1e-12 * np.abs(Wq_m).max()
    St = oracle.self_energy_R(GR, oracle.transform(ot.B_inv, Wt_iw), ent, ot.C_atom)
    Sm = oracle.self_energy_R(GR, mask(oracle.transform(of.B_inv, Wm_iw)), ent, of.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(St, Sm)) <= 1e-12 * max(np.abs(b).max() for b in Sm)
    Xt = oracle.exchange_R(GR, ot.v_R(vcls), ent, ot.C_atom)
    Xm = oracle.exchange_R(GR, mask(of.v_R(vcls)), ent, of.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(Xt, Xm)) <= 1e-12 * max(np.abs(b).max() for b in Xm)
    # the middle level matters: the two-level reduction (near = full) gives another answer
    _, two = _far_cells(r_b=4.6, n_far=3)
    o2 = oracle.OracleSystem(two)
    P2 = oracle.polarizability_R(GR, ent, o2.C_atom, two.spin, o2.kdims)
    W2 = oracle.transform(o2.B_inv, oracle.screened_W(oracle.transform(o2.B_fwd, P2), ent, vq, o2.kmesh, po)[0])
    S2 = oracle.self_energy_R(GR, W2, ent, o2.C_atom)
    assert max(np.abs(a - b).max() for a, b in zip(St, S2)) > 1e-6 * max(np.abs(b).max() for b in S2)


def test_far_basis_beyond_every_distance_is_the_full_basis():
    full = synth.make_config(0)
    tier = synth.with_far_basis(synth.make_config(0), 1e3, [3])
    Gk = full.green_k_tau()
    vq, vcls = full.coulomb()
    rf = oracle.OracleSystem(full).sweep(Gk, vq, vcls)
    rt = oracle.OracleSystem(tier).sweep(Gk, vq, vcls)
    for key in ("P_R", "Wt_R", "Sig_R", "Sigx_R"):
        for a, b in zip(rf[key], rt[key]):
            assert a.shape == b.shape and np.array_equal(a, b)


# ----------------------------------------------------------------------------
# Eq. G_1: Dyson equation, particle number, chemical potential
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cell_dense():
    """Configuration 0 at beta = 10 with 48 nodes: the transforms are accurate to ~1e-13."""
    c = synth.make_config(0, beta=10.0, n_tau=48)
    return c, oracle.OracleSystem(c)


def _static_hermitian(rng, nk, n, scale=0.05):
    x = rng.standard_normal((nk, n, n)) + 1j * rng.standard_normal((nk, n, n))
    return scale * (x + np.conj(np.transpose(x, (0, 2, 1))))


def test_dyson_without_self_energy_is_g0(cell_dense):
    c, orc = cell_dense
    Z = np.zeros_like(c.H_k)
    G = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, Z, None, c.mu, c.beta, c.omega_idx), c.H_k, Z, c.mu,
                               c.beta, c.tau, c.omega_idx, orc.F_inv)
    G0 = oracle.green0_k_tau(c.H_k, c.mu, c.beta, c.tau)
    assert np.abs(G - G0).max() < 1e-11


def test_dyson_static_exchange_is_hartree_fock(cell_dense):
    """A static Hermitian Sigma_x and Sigma_c = 0: G is the closed-form G0 of H + Sigma_x."""
    c, orc = cell_dense
    Sx = _static_hermitian(np.random.default_rng(4), c.n_k, c.n_orb_total)
    G = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, Sx, None, c.mu, c.beta, c.omega_idx), c.H_k, Sx, c.mu,
                               c.beta, c.tau, c.omega_idx, orc.F_inv)
    GHF = oracle.green0_k_tau(c.H_k + Sx, c.mu, c.beta, c.tau)
    assert np.abs(G - GHF).max() < 1e-11


def test_dyson_inverse_equals_eq_G1_as_printed(cell0):
    """G = G0 + G0 Sigma G solved as the linear system (I - G0 Sigma) G = G0 per (k, n)."""
    c = cell0
    rng = np.random.default_rng(8)
    nk, nw, N = c.n_k, c.omega_idx.size, c.n_orb_total
    Sx = _static_hermitian(rng, nk, N)
    Sc = 0.05 * (rng.standard_normal((nk, nw, N, N)) + 1j * rng.standard_normal((nk, nw, N, N)))
    G = oracle.dyson_green_iw(c.H_k, Sx, Sc, c.mu, c.beta, c.omega_idx)
    w = (2 * c.omega_idx + 1) * np.pi / c.beta
    I = np.eye(N)
    for k in range(nk):
        for n in range(nw):
            G0 = np.linalg.inv((1j * w[n] + c.mu) * I - c.H_k[k])
            ref = np.linalg.solve(I - G0 @ (Sx[k] + Sc[k, n]), G0)
            assert np.abs(G[k, n] - ref).max() < 1e-12 * np.abs(ref).max()


def test_green_tail_terms_are_exact_matsubara_integrals(cell_dense):
    """-1/2 and (2 tau - beta)/4 are polynomials, so the forward transform of Appendix A
    maps them exactly to 1/(i w) and 1/(i w)^2: the tail added back is the tail taken out."""
    c, orc = cell_dense
    w = (2 * c.omega_idx + 1) * np.pi / c.beta
    f0 = np.full(c.n_tau, -0.5, np.complex128)
    f1 = ((2 * c.tau - c.beta) / 4).astype(np.complex128)
    assert np.abs(orc.F_fwd @ f0 - 1 / (1j * w)).max() < 1e-13
    assert np.abs(orc.F_fwd @ f1 - 1 / (1j * w) ** 2).max() < 1e-13 * c.beta


def test_chemical_potential_reproduces_fermi_filling(cell_dense):
    """Sigma = 0: the bisection on N(mu) from G(beta-) finds the mu of the Fermi sum over
    the band energies at half filling (the generator's own bisection on eigenvalues)."""
    c, orc = cell_dense
    Z = np.zeros_like(c.H_k)
    e = np.linalg.eigvalsh(c.H_k)
    mu, n = oracle.chemical_potential(c.H_k, Z, None, float(c.n_orb_total), c.beta, c.tau, c.omega_idx, orc.F_inv,
                                      c.spin, lo=float(e.min()) - 1, hi=float(e.max()) + 1, tol=1e-13)
    assert abs(n - c.n_orb_total) < 1e-9
    assert abs(mu - c.mu) < 1e-9
    # and N(mu) itself against the Fermi sum at a shifted mu
    G = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, Z, None, c.mu + 0.1, c.beta, c.omega_idx), c.H_k, Z,
                               c.mu + 0.1, c.beta, c.tau, c.omega_idx, orc.F_inv)
    ref = c.spin * synth.fermi(e - c.mu - 0.1, c.beta).sum() / c.n_k
    assert abs(oracle.particle_number(G, c.spin) - ref) < 1e-10


# ----------------------------------------------------------------------------
# Linearised quasiparticle energies
# ----------------------------------------------------------------------------

def test_qp_energies_without_correlation_are_hartree_fock(cell0):
    c = cell0
    rng = np.random.default_rng(12)
    Sx = _static_hermitian(rng, c.n_k, c.n_orb_total)
    E = oracle.qp_energies(c.H_k, Sx, None, c.mu, c.beta, c.omega_idx)
    assert np.abs(E - np.linalg.eigvalsh(c.H_k + Sx)).max() < 1e-12


def test_qp_energies_of_a_linear_self_energy_solve_the_generalised_problem(cell0):
    """Sigma_c(i w) = S0 + i w S1 exactly (Hermitian S0, negative semidefinite S1): the
    energies are the generalised eigenvalues of (H + Sigma_x + S0 - mu, I - S1) plus mu
    (SciPy's generalised Hermitian-definite solver)."""
    from scipy.linalg import eigh
    c = cell0
    rng = np.random.default_rng(13)
    nk, N = c.n_k, c.n_orb_total
    Sx = _static_hermitian(rng, nk, N)
    S0 = _static_hermitian(rng, nk, N)
    B = rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N))
    S1 = -0.1 * np.einsum("kij,klj->kil", B, B.conj())  # -B B^dagger
    w = (2 * c.omega_idx + 1) * np.pi / c.beta
    Sc = S0[:, None] + 1j * w[None, :, None, None] * S1[:, None]
    E = oracle.qp_energies(c.H_k, Sx, Sc, c.mu, c.beta, c.omega_idx)
    I = np.eye(N)
    for k in range(nk):
        ref = eigh(c.H_k[k] + Sx[k] + S0[k] - c.mu * I, I - S1[k], eigvals_only=True) + c.mu
        assert np.abs(E[k] - ref).max() < 1e-11


# ----------------------------------------------------------------------------
# Eq. sf_9: continued-fraction continuation
# ----------------------------------------------------------------------------

def test_continued_fraction_reproduces_a_pole_sum():
    """f(z) = sum_j A_j / (z - p_j) with J poles is a rational function the fraction through
    2J points represents exactly: the continuation to the real axis is f itself."""
    rng = np.random.default_rng(3)
    J = 4
    A = rng.uniform(0.1, 1.0, J)
    p = rng.uniform(-2.0, 2.0, J) - 0.05j
    f = lambda z: (A[None, :] / (np.asarray(z)[:, None] - p[None, :])).sum(axis=1)
    z = 1j * (2 * np.arange(2 * J) + 1) * np.pi / 20.0
    a = oracle.continued_fraction_coefficients(z, f(z))
    w = np.linspace(-3.0, 3.0, 41) + 0.01j
    # continuing from the imaginary axis to poles 0.05 below the real one is ill-conditioned:
    # rounding reaches ~1e-9 here, while one point too few leaves errors of order one
    assert np.abs(oracle.continued_fraction_value(a, z, w) - f(w)).max() < 1e-7 * np.abs(f(w)).max()
    a7 = oracle.continued_fraction_coefficients(z[:-1], f(z[:-1]))
    assert np.abs(oracle.continued_fraction_value(a7, z[:-1], w) - f(w)).max() > 1e-2 * np.abs(f(w)).max()


def test_continued_fraction_interpolates_its_points():
    rng = np.random.default_rng(4)
    z = 1j * (2 * np.sort(rng.choice(60, 12, replace=False)) + 1) * np.pi / 30.0
    f = rng.standard_normal((12, 3, 3)) + 1j * rng.standard_normal((12, 3, 3))
    a = oracle.continued_fraction_coefficients(z, f)
    assert np.abs(oracle.continued_fraction_value(a, z, z) - f).max() < 1e-9 * np.abs(f).max()


def test_continue_sigma_of_a_single_pole_self_energy(cell0):
    """A self-energy made of one pole per element, sampled on the stored grid of
    configuration 0: the continuation through the grid's 2 lowest non-negative
    frequencies returns it on the real axis (the rest of the grid carries the same
    rational function, so every level beyond the second vanishes)."""
    c = cell0
    idx = np.asarray(c.omega_idx)
    keep = idx[(idx >= 0)]
    keep = np.sort(keep)[:2]
    mask = np.isin(idx, keep)
    rng = np.random.default_rng(5)
    nk, N = c.n_k, c.n_orb_total
    A = rng.uniform(0.1, 1.0, (nk, N, N))
    P = rng.uniform(-1.0, 1.0, (nk, N, N)) - 0.1j
    w = (2 * idx[mask] + 1) * np.pi / c.beta
    S = A[:, None] / (1j * w[None, :, None, None] - P[:, None])
    wr = np.linspace(-1.0, 1.0, 9)
    out = oracle.continue_sigma(S, idx[mask], c.beta, wr, 0.02)
    ref = A[:, None] / ((wr + 0.02j)[None, :, None, None] - P[:, None])
    assert np.abs(out - ref).max() < 1e-10 * np.abs(ref).max()


def test_spectral_function_without_correlation_is_a_sum_of_lorentzians(cell0):
    """Sigma_c = 0: A(k, w) = sum over the levels e of H + Sigma_x of
    (delta/pi) / ((w + mu - e)^2 + delta^2), and it integrates to the number of levels."""
    c = cell0
    Sx = _static_hermitian(np.random.default_rng(14), c.n_k, c.n_orb_total)
    w = np.linspace(-3.0, 3.0, 61)
    A = oracle.spectral_function(c.H_k, Sx, None, c.mu, w, 0.05)
    e = np.linalg.eigvalsh(c.H_k + Sx)
    ref = (0.05 / np.pi / ((w[None, :, None] + c.mu - e[:, None, :]) ** 2 + 0.05 ** 2)).sum(axis=2)
    assert np.abs(A - ref).max() < 1e-12 * np.abs(ref).max()
    wd = np.linspace(-400.0, 400.0, 400001)
    Ad = oracle.spectral_function(c.H_k[:1], Sx[:1], None, c.mu, wd, 0.05)
    assert abs(np.trapezoid(Ad[0], wd) - c.n_orb_total) < 1e-3
