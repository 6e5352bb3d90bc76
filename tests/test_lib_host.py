"""Host-side checks of libgw: the library loads, exports what include/gw.h
declares, and its plan tables (pair list, k-mesh rule, transform matrices)
agree with the oracle.  No GPU is needed: plans are built with host_only."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(gw_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol(gwlib):
    names = _declared_symbols()
    assert {"gw_plan_create", "gw_polarizability_tau", "gw_self_energy_tau", "gw_screened_W_iw"} <= names
    for n in sorted(names):
        assert hasattr(gwlib, n), n
    from paper_1911_05633_gb300 import gw
    assert set(gw.EXPORTED) <= names


def _plan(cell, **kw):
    from paper_1911_05633_gb300 import gw
    return gw.Plan.from_cell(cell, host_only=True, **kw)


@pytest.mark.parametrize("which", ["c0", "c1", "mixed", "c1_short_cutoff", "c2_16"])
def test_plan_tables_match_oracle(gwlib, which):
    if which == "c0":
        cell = synth.make_config(0)
    elif which == "c1":
        cell = synth.make_config(1, build=False)
        cell._draw_basis(np.random.default_rng(0))
    elif which == "mixed":
        cell = synth.mixed_species_cell()
    elif which == "c1_short_cutoff":
        cell = synth.make_config(1, build=False, cutoff=5.0)
        cell._draw_basis(np.random.default_rng(0))
    else:
        cell = synth.make_config(2, atoms=16, build=False)
        cell._draw_basis(np.random.default_rng(0))
    p = _plan(cell)
    ent = oracle.pair_list(cell.lattice, cell.frac, cell.kmesh, cell.cutoff)
    assert np.array_equal(p.entries, ent)
    if cell.cutoff > 0:
        assert tuple(p.info["kmesh_required"]) == oracle.kmesh_rule(cell.lattice, cell.cutoff)
    # offsets are the prefix sums of the block sizes
    no = [cell.n_orb_of(int(a)) * cell.n_orb_of(int(b)) for a, b in ent[:, :2]]
    npb = [cell.n_prod_of(int(a)) * cell.n_prod_of(int(b)) for a, b in ent[:, :2]]
    assert np.array_equal(p.off_orb, np.concatenate([[0], np.cumsum(no)]))
    assert np.array_equal(p.off_pb, np.concatenate([[0], np.cumsum(npb)]))
    for st, idx in (("F", cell.omega_idx), ("B", cell.nu_idx)):
        T = oracle.fourier_matrix(cell.beta, cell.tau, idx, st)
        U = oracle.inverse_matrix(T)
        Tl = p.transform_matrix(st, "tau_to_iw")
        Ul = p.transform_matrix(st, "iw_to_tau")
        n = len(cell.tau)
        assert np.abs(Tl - T).max() < 2.3e-16 * (n * n + np.pi * np.abs(idx).max() + 10) * np.abs(T).max()
        assert np.abs(Ul - U).max() < 1e-11 * np.abs(U).max()
        assert np.abs(Ul @ Tl - np.eye(n)).max() < 1e-11


def test_plan_errors(gwlib):
    from paper_1911_05633_gb300 import gw
    cell = synth.make_config(1, build=False)
    cell._draw_basis(np.random.default_rng(0))
    # strict k-mesh rule: 2x2x2 is below the rule for a 12-bohr cutoff on this cell
    with pytest.raises(gw.GwError) as ex:
        gw.Plan(
            cell.lattice, cell.frac, cell.species_of_atom, [9], [48], [cell.species[0].C], (2, 2, 2),
            cell.beta, cell.tau, cell.omega_idx, cell.nu_idx, cell.cutoff, strict_kmesh=True, host_only=True)
    assert ex.value.status == 4
    # tau grid not mirror symmetric
    tau = cell.tau.copy()
    tau[3] += 1e-3
    with pytest.raises(gw.GwError) as ex:
        gw.Plan(cell.lattice, cell.frac, cell.species_of_atom, [9], [48], [cell.species[0].C], cell.kmesh,
                cell.beta, tau, cell.omega_idx, cell.nu_idx, cell.cutoff, host_only=True)
    assert ex.value.status == 1
    # the smallest pair list: a tiny cutoff keeps only the onsite (a, a, R = 0) entries
    p = gw.Plan(cell.lattice, cell.frac, cell.species_of_atom, [9], [48], [cell.species[0].C], cell.kmesh,
                cell.beta, cell.tau, cell.omega_idx, cell.nu_idx, 1e-3, host_only=True)
    assert p.info["n_entries"] == cell.n_atoms
    assert np.array_equal(p.entries[:, 0], p.entries[:, 1]) and not p.entries[:, 2:].any()
    # too few Matsubara samples
    with pytest.raises(gw.GwError) as ex:
        gw.Plan(cell.lattice, cell.frac, cell.species_of_atom, [9], [48], [cell.species[0].C], cell.kmesh,
                cell.beta, cell.tau, cell.omega_idx[:10], cell.nu_idx, cell.cutoff, host_only=True)
    assert ex.value.status == 1
    # compiled limits
    big = np.zeros((129, 9, 9))
    with pytest.raises(gw.GwError) as ex:
        gw.Plan(cell.lattice, cell.frac, cell.species_of_atom, [9], [129], [big], cell.kmesh,
                cell.beta, cell.tau, cell.omega_idx, cell.nu_idx, cell.cutoff, host_only=True)
    assert ex.value.status == 10
    # compute calls on a host-only plan are refused
    p = gw.Plan.from_cell(cell, host_only=True)
    lib = gw.load_library()
    st = lib.gw_green_k_to_R(p._h, ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == 9
    assert lib.gw_status_string(9) == b"plan has no device state"


def test_w_solve_mode(gwlib):
    """Which momenta and frequencies the W solve runs on (host-side plan logic)."""
    from paper_1911_05633_gb300 import gw
    c0 = synth.make_config(0)
    p = gw.Plan.from_cell(c0, host_only=True)
    assert p.info["w_symmetric"] == 1 and p.info["n_q_solved"] == 8  # 2x2x2: every q is its own -q
    p = gw.Plan.from_cell(c0, host_only=True, no_symmetry=True)
    assert p.info["w_symmetric"] == 0 and p.info["n_q_solved"] == 8
    c1 = synth.make_config(1, build=False)
    c1._draw_basis(np.random.default_rng(0))
    p = gw.Plan.from_cell(c1, host_only=True)
    # 4x4x4 mesh: 8 momenta with q = -q and 28 pairs
    assert p.info["w_symmetric"] == 1 and p.info["n_q_solved"] == 36
    ns = synth.mixed_species_cell(symmetric_C=False, n_tau=10)
    p = gw.Plan.from_cell(ns, host_only=True)
    assert p.info["c_symmetric"] == 0 and p.info["w_symmetric"] == 0


def test_w_solver_choice(gwlib):
    """The tensor-core inverse is chosen for N_PB in {128, 256, 384} only (the range in
    which its FP32 level sums are exact), block Gauss-Jordan over such pivot blocks for
    larger multiples of 128 (pivot blocks of 256 or 128); FP64 Gauss-Jordan otherwise or
    when asked for."""
    from paper_1911_05633_gb300 import gw
    c1 = synth.make_config(1, build=False)
    c1._draw_basis(np.random.default_rng(0))
    assert c1.n_pb_total == 384
    assert gw.Plan.from_cell(c1, host_only=True).info["w_tensor"] == 1
    assert gw.Plan.from_cell(c1, host_only=True, w_solver="gauss_jordan").info["w_tensor"] == 0
    c2 = synth.make_config(2, atoms=8, build=False)
    c2._draw_basis(np.random.default_rng(0))
    assert c2.n_pb_total == 512
    assert gw.Plan.from_cell(c2, host_only=True).info["w_tensor"] == 0
    # beyond 384: block Gauss-Jordan over the largest pivot block of 256 or 128 dividing N_PB
    assert gw.Plan.from_cell(c2, host_only=True).info["w_block"] == 256
    assert gw.Plan.from_cell(c2, host_only=True, w_solver="gauss_jordan").info["w_block"] == 0
    assert gw.Plan.from_cell(c1, host_only=True).info["w_block"] == 0
    c72 = synth.make_config(2, build=False)
    c72._draw_basis(np.random.default_rng(0))
    assert c72.n_pb_total == 4608 and gw.Plan.from_cell(c72, host_only=True).info["w_block"] == 256
    mixed = synth.mixed_species_cell(n_tau=10)
    assert mixed.n_pb_total % 128 != 0
    assert gw.Plan.from_cell(mixed, host_only=True).info["w_tensor"] == 0
    assert gw.Plan.from_cell(mixed, host_only=True).info["w_block"] == 0


def test_sigma_stage_choice(gwlib):
    """The FP64 Sigma takes its W~ C^b stage from the tensor cores (every K_b within the
    compiled limit qualifies) unless the plan asks for FP64 arithmetic only."""
    from paper_1911_05633_gb300 import gw
    c1 = synth.make_config(1, build=False)
    c1._draw_basis(np.random.default_rng(0))
    assert gw.Plan.from_cell(c1, host_only=True).info["sigma_tensor"] == 1
    assert gw.Plan.from_cell(c1, host_only=True, fp64_products="fp64").info["sigma_tensor"] == 0


@pytest.mark.parametrize("which", ["c1_cut5", "mixed", "c2_16"])
def test_far_basis_tables_match_oracle(gwlib, which):
    """Reduced product basis beyond sphere B (Sec. 2, Fig. 2): the plan's per-entry
    product-basis blocks, tier count and offsets against the oracle's own tier rule."""
    from paper_1911_05633_gb300 import gw
    if which == "c1_cut5":
        cell = synth.make_config(1, build=False, cutoff=5.0, kmesh=(2, 2, 2))
        r_b, far = 4.0, [24]
    elif which == "mixed":
        cell = synth.mixed_species_cell()
        r_b, far = 4.4, [5, 11]   # A-B at 4.33 bohr stay full, A-A and B-B at 5 bohr reduced
    else:
        cell = synth.make_config(2, atoms=16, build=False)
        r_b, far = 7.5, [16]
    if cell.species[0].C is None:
        cell._draw_basis(np.random.default_rng(0))
    synth.with_far_basis(cell, r_b, far)
    p = gw.Plan.from_cell(cell, host_only=True)
    ent = oracle.pair_list(cell.lattice, cell.frac, cell.kmesh, cell.cutoff)
    assert np.array_equal(p.entries, ent)
    is_far = oracle.entry_far(cell.lattice, cell.frac, ent, r_b)
    assert 0 < is_far.sum() < len(ent)
    full = [cell.n_prod_of(a) for a in range(cell.n_atoms)]
    red = [cell.species[s].n_prod_far for s in cell.species_of_atom]
    dims = oracle.entry_pb_dims(ent, is_far, full, red)
    assert p.info["n_entries_far"] == int(is_far.sum())
    assert [p.block_shape(e, "pb") for e in range(len(ent))] == dims
    assert np.array_equal(p.off_pb, np.concatenate([[0], np.cumsum([ka * kb for ka, kb in dims])]))
    assert p.info["len_pb"] == sum(ka * kb for ka, kb in dims)
    # the orbital blocks are not reduced
    no = [cell.n_orb_of(int(a)) * cell.n_orb_of(int(b)) for a, b in ent[:, :2]]
    assert np.array_equal(p.off_orb, np.concatenate([[0], np.cumsum(no)]))
    # r_b beyond every kept distance: one basis for every entry
    q = gw.Plan.from_cell(cell, host_only=True, r_b=1e3, n_prod_far=far)
    assert q.info["n_entries_far"] == 0
    assert q.info["len_pb"] == sum(full[int(a)] * full[int(b)] for a, b in ent[:, :2])


def test_far_basis_rejects_bad_sizes(gwlib):
    from paper_1911_05633_gb300 import gw
    cell = synth.make_config(0)
    for bad in ([0], [9]):  # n_prod = 8
        with pytest.raises(gw.GwError):
            gw.Plan.from_cell(cell, host_only=True, r_b=4.0, n_prod_far=bad)


def test_every_compute_call_refuses_a_host_only_plan(gwlib):
    """GW_ERR_NO_DEVICE (9) from each device entry point of a host-only plan, before any
    pointer is touched (the pointers given here are not valid memory)."""
    from paper_1911_05633_gb300 import gw
    p = gw.Plan.from_cell(synth.make_config(0), host_only=True)
    lib = gw.load_library()
    h, q = p._h, ctypes.c_void_p(16)
    d = ctypes.c_double(0.0)
    w = (ctypes.c_double * 2)(0.0, 0.1)
    calls = {
        "gw_fourier_k_to_R": lambda: lib.gw_fourier_k_to_R(h, 1, 1, q, q, None),
        "gw_polarizability_tau": lambda: lib.gw_polarizability_tau(h, q, q, 0, None),
        "gw_transform_tau_iw": lambda: lib.gw_transform_tau_iw(h, 0, 0, 0, q, q, None),
        "gw_screened_W_iw": lambda: lib.gw_screened_W_iw(h, q, q, q, None),
        "gw_screened_W_iw_noalloc": lambda: lib.gw_screened_W_iw_noalloc(h, q, q, q, None),
        "gw_self_energy_tau": lambda: lib.gw_self_energy_tau(h, q, q, None, q, None, 0, None),
        "gw_fourier_R_to_k": lambda: lib.gw_fourier_R_to_k(h, 0, 1, q, q, None),
        "gw_dyson_green_tau": lambda: lib.gw_dyson_green_tau(h, q, None, None, 0.0, q, None),
        "gw_chemical_potential": lambda: lib.gw_chemical_potential(h, q, None, None, 8.0, -1.0, 1.0, 1e-9,
                                                                   ctypes.byref(d), None, None),
        "gw_qp_energies": lambda: lib.gw_qp_energies(h, q, None, None, 0.0, q, None),
        "gw_continue_sigma": lambda: lib.gw_continue_sigma(h, q, 2, w, 0.01, q, None),
        "gw_spectral_function": lambda: lib.gw_spectral_function(h, q, None, None, 2, w, 0.01, 0.0, q, None),
        "gw_sync": lambda: lib.gw_sync(h, None),
    }
    for name, call in calls.items():
        assert call() == 9, name
