"""Mixed precision (GW_MIXED): the P and Sigma contractions in reduced precision
with FP32 accumulation against the FP64 oracle.  Bar: relative Frobenius error
<= 1e-6 on P and Sigma (the tolerance stated for the mixed path)."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import _random_W, dev, host, pack, rel, system

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.mark.parametrize("name", ["c0", "mixed", "mixed_nonsym", "c1", "c1_cut5_far", "mixed_far"])
def test_polarizability_mixed(name):
    s = system(name)
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
    P = host(s.plan.polarizability_tau(dev(pack(s.G_R())), precision="mixed"))
    err = rel(P, pack(ref))
    assert err < TOL_MIXED, err


@pytest.mark.parametrize("name", ["c0", "mixed", "c1", "c1_cut5_far", "mixed_far"])
def test_self_energy_mixed(name):
    s = system(name)
    WR = _random_W(s)
    ref = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    S = host(s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), precision="mixed"))
    err = rel(S, pack(ref))
    assert err < TOL_MIXED, err


# The W solve amplifies relative errors of P by ~10^3 on these systems (the CPU test
# test_w_solve_amplifies_errors_of_p measures it with the oracle alone), so a chain whose
# P is good to <= 1e-6 delivers W~ and Sigma to <= 1e-3.
TOL_CHAIN = 1e-3


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
    assert rel(host(PR), pack(r["P_R"])) < TOL_MIXED
    assert rel(host(Sig), pack(r["Sig_R"])) < TOL_CHAIN
    assert rel(host(Sk), r["Sig_k"].reshape(-1)) < TOL_CHAIN


def test_mixed_largest_blocks_cuda_core_path():
    """n = 16, K = 128 is outside the tensor-core tile limits: the FP32 CUDA-core form runs."""
    import synth
    from test_gpu_parity import Sys
    lat = np.eye(3) * 6.0
    sp = [synth.Species("big", 16, 128, None)]
    cell = synth.SynthCell("big1", lat, np.zeros((1, 3)), np.zeros(1, np.int32), sp, (2, 1, 1), 20.0, 8, 0.0,
                           seed=77, gap=None, hop_cutoff=6.5).build()
    s = Sys(cell)
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, cell.spin)
    assert rel(host(s.plan.polarizability_tau(dev(pack(s.G_R())), precision="mixed")), pack(ref)) < TOL_MIXED
    WR = _random_W(s)
    refS = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    assert rel(host(s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), precision="mixed")),
               pack(refS)) < TOL_MIXED
