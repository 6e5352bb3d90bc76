"""Eq. G_1 on the device against the oracle: G(k, tau) from the Dyson solve with a static
Sigma_x and a frequency-dependent Sigma_c, the chemical potential by bisection on the
particle number, and the Dyson step fed by the device sweep's own Sigma (FP64, 1e-10)."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import TOL, dev, host, rel, system

pytestmark = pytest.mark.gpu


def _sigmas(cell, seed):
    """A static Hermitian Sigma_x(k) and a Sigma_c(k, i w) with Sigma_c(-i w) = Sigma_c(i w)^dagger."""
    rng = np.random.default_rng(seed)
    nk, N, idx = cell.n_k, cell.n_orb_total, cell.omega_idx
    x = rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N))
    Sx = 0.05 * (x + np.conj(np.transpose(x, (0, 2, 1))))
    pos = {int(n): i for i, n in enumerate(idx)}
    Sc = np.zeros((nk, len(idx), N, N), np.complex128)
    for i, n in enumerate(idx):
        if n >= 0:
            c = 0.02 * (rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N)))
            Sc[:, i] = c
            j = pos.get(-int(n) - 1)  # w_{-n-1} = -w_n
            if j is not None:
                Sc[:, j] = np.conj(np.transpose(c, (0, 2, 1)))
    return Sx, Sc


@pytest.mark.parametrize("name", ["c0", "mixed", "c1_cut5"])
def test_dyson_green_tau(name):
    s = system(name)
    c = s.cell
    Sx, Sc = _sigmas(c, 3)
    ref = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, Sx, Sc, c.mu, c.beta, c.omega_idx), c.H_k, Sx, c.mu,
                                 c.beta, c.tau, c.omega_idx, s.orc.F_inv)
    G = host(s.plan.dyson_green_tau(dev(c.H_k), c.mu, Sigx_k=dev(Sx), Sig_k_iw=dev(Sc)))
    s.plan.sync()
    assert rel(G, ref.reshape(-1)) < TOL
    # no self-energy: G0 of H through the same transform
    Z = np.zeros_like(c.H_k)
    ref0 = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, Z, None, c.mu, c.beta, c.omega_idx), c.H_k, Z, c.mu,
                                  c.beta, c.tau, c.omega_idx, s.orc.F_inv)
    G0 = host(s.plan.dyson_green_tau(dev(c.H_k), c.mu))
    s.plan.sync()
    assert rel(G0, ref0.reshape(-1)) < TOL


@pytest.mark.parametrize("name", ["c0", "mixed"])
def test_chemical_potential(name):
    s = system(name)
    c = s.cell
    Sx, Sc = _sigmas(c, 5)
    target = float(c.n_orb_total)  # half filling, s = 2
    e = np.linalg.eigvalsh(c.H_k)
    lo, hi = float(e.min()) - 1.0, float(e.max()) + 1.0
    mu_o, n_o = oracle.chemical_potential(c.H_k, Sx, Sc, target, c.beta, c.tau, c.omega_idx, s.orc.F_inv, c.spin,
                                          lo, hi, tol=1e-11)
    mu_g, n_g = s.plan.chemical_potential(dev(c.H_k), target, lo, hi, tol=1e-11, Sigx_k=dev(Sx), Sig_k_iw=dev(Sc))
    assert abs(n_o - target) < 1e-8
    assert abs(mu_g - mu_o) < 1e-9
    assert abs(n_g - n_o) < 1e-9


def test_dyson_after_the_device_sweep():
    """Sigma(k, i w) and Sigma_x(k) from the whole device sweep feed the Dyson step: the
    next iteration's G(k, tau) against the oracle's sweep and Dyson step."""
    s = system("c0")
    p, c = s.plan, s.cell
    r = s.orc.sweep(s.G_k, s.v_q, s.v_class)
    GR = p.green_k_to_R(dev(s.G_k))
    PR = p.polarizability_tau(GR)
    Wiw = p.screened_W_iw(p.transform_tau_iw("B", "tau_to_iw", "pb", PR), dev(s.v_q))
    WR = p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw)
    Sig, Sigx = p.self_energy_tau(GR, WR, v_R=p.fourier_k_to_R("pb", 1, dev(s.v_q)))
    Sk = p.fourier_R_to_k("orb", c.omega_idx.size, p.transform_tau_iw("F", "tau_to_iw", "orb", Sig))
    Sxk = p.fourier_R_to_k("orb", 1, Sigx)
    G = host(p.dyson_green_tau(dev(c.H_k), c.mu, Sigx_k=Sxk, Sig_k_iw=Sk))
    p.sync()
    ref = oracle.green_iw_to_tau(oracle.dyson_green_iw(c.H_k, r["Sigx_k"], r["Sig_k"], c.mu, c.beta, c.omega_idx),
                                 c.H_k, r["Sigx_k"], c.mu, c.beta, c.tau, c.omega_idx, s.orc.F_inv)
    assert rel(G, ref.reshape(-1)) < TOL


def _linear_sigma(cell, seed):
    """Sigma_c(i w) = S0 + i w S1 with Hermitian S0 and negative semidefinite S1, and a
    static Hermitian Sigma_x."""
    rng = np.random.default_rng(seed)
    nk, N = cell.n_k, cell.n_orb_total
    herm = lambda x: 0.5 * (x + np.conj(np.transpose(x, (0, 2, 1))))
    Sx = 0.1 * herm(rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N)))
    S0 = 0.05 * herm(rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N)))
    B = rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N))
    S1 = -0.2 / N * np.einsum("kij,klj->kil", B, B.conj())
    w = (2 * cell.omega_idx + 1) * np.pi / cell.beta
    return Sx, S0[:, None] + 1j * w[None, :, None, None] * S1[:, None]


@pytest.mark.parametrize("name", ["c0", "mixed", "c1_cut5"])
def test_qp_energies(name):
    s = system(name)
    c = s.cell
    Sx, Sc = _linear_sigma(c, 21)
    ref = oracle.qp_energies(c.H_k, Sx, Sc, c.mu, c.beta, c.omega_idx)
    E = s.plan.qp_energies(dev(c.H_k), c.mu, Sigx_k=dev(Sx), Sig_k_iw=dev(Sc))
    s.plan.sync()
    E = E.cpu().numpy().reshape(ref.shape)
    assert np.abs(E - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
    # without correlation: the Hartree-Fock levels
    E0 = s.plan.qp_energies(dev(c.H_k), c.mu, Sigx_k=dev(Sx)).cpu().numpy().reshape(ref.shape)
    assert np.abs(E0 - np.linalg.eigvalsh(c.H_k + Sx)).max() < 1e-10 * max(1.0, np.abs(E0).max())


def test_qp_energies_after_the_device_sweep():
    s = system("c0")
    p, c = s.plan, s.cell
    r = s.orc.sweep(s.G_k, s.v_q, s.v_class)
    GR = p.green_k_to_R(dev(s.G_k))
    Wiw = p.screened_W_iw(p.transform_tau_iw("B", "tau_to_iw", "pb", p.polarizability_tau(GR)), dev(s.v_q))
    Sig, Sigx = p.self_energy_tau(GR, p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw),
                                  v_R=p.fourier_k_to_R("pb", 1, dev(s.v_q)))
    Sk = p.fourier_R_to_k("orb", c.omega_idx.size, p.transform_tau_iw("F", "tau_to_iw", "orb", Sig))
    Sxk = p.fourier_R_to_k("orb", 1, Sigx)
    E = p.qp_energies(dev(c.H_k), c.mu, Sigx_k=Sxk, Sig_k_iw=Sk)
    p.sync()
    ref = oracle.qp_energies(c.H_k, r["Sigx_k"], r["Sig_k"], c.mu, c.beta, c.omega_idx)
    assert np.abs(E.cpu().numpy().reshape(ref.shape) - ref).max() < 1e-10


def _pole_sigma(cell, seed, n_poles=10):
    """Sigma(k, i w) of n_poles poles per element below the real axis, on the stored grid."""
    rng = np.random.default_rng(seed)
    nk, N = cell.n_k, cell.n_orb_total
    A = rng.uniform(0.05, 0.5, (n_poles, nk, N, N))
    P = rng.uniform(-1.5, 1.5, (n_poles, nk, N, N)) - 1j * rng.uniform(0.1, 0.5, (n_poles, nk, N, N))
    z = 1j * (2 * cell.omega_idx + 1) * np.pi / cell.beta
    return (A[:, :, None] / (z[None, None, :, None, None] - P[:, :, None])).sum(axis=0)


def _rounding_envelope(S, idx, beta, wr, delta, seeds=(0, 1, 2)):
    """How far the oracle's own continuation moves, element by element, when its input is
    perturbed at the level of FP64 rounding (1e-16 relative): continuing from the
    imaginary axis amplifies rounding, and two correct FP64 evaluations that round
    differently differ by about this much."""
    ref = oracle.continue_sigma(S, idx, beta, wr, delta)
    env = np.zeros(ref.shape)
    for sd in seeds:
        rng = np.random.default_rng(sd)
        Sp = S * (1 + 1e-16 * (rng.standard_normal(S.shape) + 1j * rng.standard_normal(S.shape)))
        env = np.maximum(env, np.abs(oracle.continue_sigma(Sp, idx, beta, wr, delta) - ref))
    return ref, env


@pytest.mark.parametrize("name", ["c0", "mixed"])
def test_continue_sigma(name):
    """Eq. sf_9 on the device against the oracle's continued fraction on the same inputs,
    element by element within the oracle's own rounding envelope (and 1e-12 of the scale)."""
    s = system(name)
    c = s.cell
    S = _pole_sigma(c, 31)
    wr = np.linspace(-1.0, 1.0, 7)
    ref, env = _rounding_envelope(S, c.omega_idx, c.beta, wr, 0.05)
    out = host(s.plan.continue_sigma(dev(S), wr, 0.05)).reshape(ref.shape)
    s.plan.sync()
    assert np.isfinite(ref).all()
    assert np.all(np.abs(out - ref) <= 100.0 * env + 1e-12 * np.abs(ref).max())
    # and most elements agree far more closely than the worst-conditioned ones
    assert np.median(np.abs(out - ref)) <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["c0", "mixed"])
def test_continue_sigma_well_conditioned(name):
    """Eq. sf_9 where the continuation is well conditioned: two poles per element at least
    0.5 Ha below the real axis (a rational function the fraction through the stored points
    reproduces exactly).  Every element, no exclusions, against the oracle and against the
    pole sum itself at a fixed 1e-9 of the scale (the oracle's own rounding envelope here
    is ~1e-13 of the scale)."""
    s = system(name)
    c = s.cell
    nk, N = c.n_k, c.n_orb_total
    rng = np.random.default_rng(41)
    A = rng.uniform(0.05, 0.5, (2, nk, N, N))
    P = rng.uniform(-1.5, 1.5, (2, nk, N, N)) - 1j * rng.uniform(0.5, 1.0, (2, nk, N, N))
    z = 1j * (2 * c.omega_idx + 1) * np.pi / c.beta
    S = (A[:, :, None] / (z[None, None, :, None, None] - P[:, :, None])).sum(axis=0)
    wr = np.linspace(-1.0, 1.0, 7)
    ref = oracle.continue_sigma(S, c.omega_idx, c.beta, wr, 0.05)
    exact = (A[:, :, None] / ((wr + 0.05j)[None, None, :, None, None] - P[:, :, None])).sum(axis=0)
    out = host(s.plan.continue_sigma(dev(S), wr, 0.05)).reshape(ref.shape)
    s.plan.sync()
    scale = np.abs(exact).max()
    assert np.isfinite(out).all()
    assert np.abs(out - ref).max() <= 1e-9 * scale
    assert np.abs(out - exact).max() <= 1e-9 * scale


def test_continue_sigma_of_the_device_sweep():
    s = system("c0")
    p, c = s.plan, s.cell
    GR = p.green_k_to_R(dev(s.G_k))
    Wiw = p.screened_W_iw(p.transform_tau_iw("B", "tau_to_iw", "pb", p.polarizability_tau(GR)), dev(s.v_q))
    Sig = p.self_energy_tau(GR, p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw))
    Sk = p.fourier_R_to_k("orb", c.omega_idx.size, p.transform_tau_iw("F", "tau_to_iw", "orb", Sig))
    wr = np.linspace(-0.5, 0.5, 5)
    out = host(p.continue_sigma(Sk, wr, 0.02))
    p.sync()
    S = host(Sk).reshape(c.n_k, c.omega_idx.size, c.n_orb_total, c.n_orb_total)
    ref, env = _rounding_envelope(S, c.omega_idx, c.beta, wr, 0.02)
    ok = np.isfinite(ref) & np.isfinite(env)
    assert ok.mean() > 0.99
    out = out.reshape(ref.shape)
    assert np.all(np.abs(out[ok] - ref[ok]) <= 100.0 * env[ok] + 1e-12 * np.abs(ref[ok]).max())


@pytest.mark.parametrize("name", ["c0", "mixed"])
def test_spectral_function(name):
    """Eqs. sf_1, sf_7 on the device: A(k, w) from a continued Sigma (the device's own,
    handed to the oracle as well) and, without correlation, the Lorentzians of H + Sigma_x."""
    s = system(name)
    c = s.cell
    nk, N = c.n_k, c.n_orb_total
    Sx, _ = _sigmas(c, 3)
    wr = np.linspace(-1.0, 1.0, 7)
    Sw = s.plan.continue_sigma(dev(_pole_sigma(c, 31)), wr, 0.05)
    A = host(s.plan.spectral_function(dev(c.H_k), wr, 0.05, c.mu, Sigx_k=dev(Sx), Sig_k_w=Sw))
    s.plan.sync()
    ref = oracle.spectral_function(c.H_k, Sx, host(Sw).reshape(nk, len(wr), N, N), c.mu, wr, 0.05)
    assert np.abs(A.reshape(ref.shape) - ref).max() <= 1e-10 * np.abs(ref).max()
    A0 = host(s.plan.spectral_function(dev(c.H_k), wr, 0.05, c.mu, Sigx_k=dev(Sx))).reshape(ref.shape)
    s.plan.sync()
    e = np.linalg.eigvalsh(c.H_k + Sx)
    ref0 = (0.05 / np.pi / ((wr[None, :, None] + c.mu - e[:, None, :]) ** 2 + 0.05 ** 2)).sum(axis=2)
    assert np.abs(A0 - ref0).max() <= 1e-10 * np.abs(ref0).max()
