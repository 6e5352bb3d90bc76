"""Mixed precision (GW_MIXED): the P and Sigma contractions in reduced precision
with FP32 accumulation against the FP64 oracle.  Bar: relative Frobenius error
<= 1e-6 on P and Sigma (the tolerance stated for the mixed path)."""
import os

import numpy as np
import pytest

import oracle
from test_gpu_parity import _random_W, dev, host, pack, rel, rel_blocks, system

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.mark.parametrize("name", ["c0", "mixed", "mixed_nonsym", "c1", "c1_cut5_far", "mixed_far", "c1_3tier"])
def test_polarizability_mixed(name):
    s = system(name)
    assert s.plan.info["mixed_queue"] == 3  # the persistent tensor-core kernels, not a fallback
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
    P = host(s.plan.polarizability_tau(dev(pack(s.G_R())), precision="mixed"))
    err = rel(P, pack(ref))
    assert err < TOL_MIXED, err
    assert rel_blocks(P, pack(ref), s.plan.off_pb, s.nt) < TOL_MIXED


@pytest.mark.parametrize("name", ["c0", "mixed", "c1", "c1_cut5_far", "mixed_far", "c1_3tier"])
def test_self_energy_mixed(name):
    s = system(name)
    WR = _random_W(s)
    ref = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    S = host(s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), precision="mixed"))
    err = rel(S, pack(ref))
    assert err < TOL_MIXED, err
    assert rel_blocks(S, pack(ref), s.plan.off_orb, s.nt) < TOL_MIXED
    # the exchange term in the same precision (W~ -> v, G(tau) -> G(beta-), opposite sign)
    vR = s.orc.v_R(s.v_class)
    refx = oracle.exchange_R(s.G_R(), vR, s.orc.entries, s.orc.C_atom)
    _, Sx = s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), v_R=dev(pack(vR)), precision="mixed")
    assert rel(host(Sx), pack(refx)) < TOL_MIXED
    assert rel_blocks(host(Sx), pack(refx), s.plan.off_orb, 1) < TOL_MIXED


def _amplification():
    """Per system, how much the oracle's own chain P -> W~ -> Sigma magnifies a relative
    perturbation of P (tests/golden/chain_amplification.txt, written by the oracle alone)."""
    out = {}
    for l in open(os.path.join(os.path.dirname(__file__), "golden", "chain_amplification.txt")):
        if l.strip() and not l.startswith("#"):
            f = l.split()
            out[f[0]] = (float(f[1]), float(f[2]))
    return out


def _chain_bound(amp, err_p):
    """What a P error of err_p can do to Sigma through the W solve (the oracle's amplification,
    x3 for the spread over directions of the error), plus the mixed Sigma contraction's own
    bound: the chain may be no worse than the error of P propagated by the problem itself."""
    return 3.0 * amp * err_p + TOL_MIXED


@pytest.mark.parametrize("name", ["c0", "c1_cut5", "c1_cut5_far"])
def test_whole_sweep_mixed(name):
    s = system(name)
    p = s.plan
    r = s.orc.sweep(s.G_k, s.v_q, s.v_class)
    GR = p.green_k_to_R(dev(s.G_k))
    PR = p.polarizability_tau(GR, precision="mixed")
    Piw = p.transform_tau_iw("B", "tau_to_iw", "pb", PR)
    Wiw = p.screened_W_iw(Piw, dev(s.v_q))
    WR = p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw)
    Sig = p.self_energy_tau(GR, WR, precision="mixed")
    Siw = p.transform_tau_iw("F", "tau_to_iw", "orb", Sig)
    Sk = p.fourier_R_to_k("orb", s.cell.omega_idx.size, Siw)
    p.sync()
    err_p = rel(host(PR), pack(r["P_R"]))
    assert err_p < TOL_MIXED
    amp_R, amp_k = _amplification()[name]
    assert rel(host(Sig), pack(r["Sig_R"])) < _chain_bound(amp_R, err_p)
    assert rel(host(Sk), r["Sig_k"].reshape(-1)) < _chain_bound(amp_k, err_p)


def _qp_chain(s, prec):
    """One whole sweep (W solve included) in the given precision, then the linearised
    quasiparticle energies from its Sigma(k, i w) and Sigma_x(k)."""
    p, c = s.plan, s.cell
    inf = p.info
    GR = p.green_k_to_R(dev(s.G_k))
    PR = p.polarizability_tau(GR, precision=prec)
    Piw = p.transform_tau_iw("B", "tau_to_iw", "pb", PR, structure="mirror" if inf["c_symmetric"] else "general")
    Wiw = p.screened_W_iw(Piw, dev(s.v_q))
    WR = p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw, structure="real" if inf["w_symmetric"] else "general")
    Sig, Sigx = p.self_energy_tau(GR, WR, v_R=p.fourier_k_to_R("pb", 1, dev(s.v_q)), precision=prec)
    Sk = p.fourier_R_to_k("orb", c.omega_idx.size, p.transform_tau_iw("F", "tau_to_iw", "orb", Sig))
    Sxk = p.fourier_R_to_k("orb", 1, Sigx)
    E = p.qp_energies(dev(c.H_k), c.mu, Sigx_k=Sxk, Sig_k_iw=Sk)
    p.sync()
    return host(PR), host(Sk), host(E)


def test_mixed_quasiparticle_energies_within_1_meV():
    """The 8-atom, 4x4x4, 48-node workload: the linearised quasiparticle energies of the mixed
    chain within 1 meV of the FP64 chain's (the FP64 device path equals the oracle to 1e-10
    row by row on this system: test_green_k_to_R, test_polarizability, test_transform,
    test_screened_W_sampled_full_size, test_self_energy_and_exchange, test_fourier_R_to_k),
    and Sigma(k, i w) within what the mixed P error does through the W solve."""
    s = system("c1")
    P64, S64, E64 = _qp_chain(s, "fp64")
    Pm, Sm, Em = _qp_chain(s, "mixed")
    err_p = rel(Pm, P64)
    assert err_p < TOL_MIXED
    assert rel(Sm, S64) < _chain_bound(_amplification()["c1"][1], err_p)
    hartree_meV = 27211.386245988
    assert np.abs(Em - E64).max() * hartree_meV < 1.0


def test_mixed_largest_blocks():
    """n = 16, K = 128 (the compiled maxima): the queue kernels with the reduction in chunks
    (n^2 = 256 columns of P's dense stage) and one thread group for Sigma's 256-wide stage."""
    import synth
    from test_gpu_parity import Sys
    lat = np.eye(3) * 6.0
    sp = [synth.Species("big", 16, 128, None)]
    cell = synth.SynthCell("big1", lat, np.zeros((1, 3)), np.zeros(1, np.int32), sp, (2, 1, 1), 20.0, 8, 0.0,
                           seed=77, gap=None, hop_cutoff=6.5).build()
    s = Sys(cell)
    assert s.plan.info["mixed_queue"] == 3
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, cell.spin)
    assert rel(host(s.plan.polarizability_tau(dev(pack(s.G_R())), precision="mixed")), pack(ref)) < TOL_MIXED
    WR = _random_W(s)
    refS = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    assert rel(host(s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), precision="mixed")),
               pack(refS)) < TOL_MIXED
