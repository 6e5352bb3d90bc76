"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every row of the sweep is compared element by element with the oracle on the
same seeded inputs: the k -> R gather, the P contraction, the tau <-> i omega
transforms, the W solve, the Sigma contraction with its exchange term, and the
R -> k scatter; then the whole chain end to end.  FP64 bar: relative Frobenius
error <= 1e-10 (the tolerance stated for the plain FP64 path).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(autouse=True)
def _need_cuda():
    _torch()


def dev(x):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)).to("cuda")


def host(t):
    _torch().cuda.synchronize()
    return t.cpu().numpy()


def pack(blocks):
    return np.concatenate([np.ascontiguousarray(b).reshape(-1) for b in blocks]).astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_blocks(a, b, off, n_slices, floor=1e-6):
    """Largest relative error over the (entry, slice) blocks of an entry-layout buffer: each
    block's error against its own norm, so that a wrong block of small magnitude (a far entry,
    a distant pair, the middle of the tau grid) cannot hide under the global norm.
    floor = x: blocks smaller than x times the largest block are measured against that floor
    (stages computed block by block from exact inputs, whose rounding is relative per block);
    floor = "rms": against the root-mean-square block norm (stages downstream of the W solve,
    whose rounding is relative to the whole dense matrix of each (q, nu), not to each block)."""
    blocks = []
    for e in range(len(off) - 1):
        A = a[n_slices * off[e]: n_slices * off[e + 1]].reshape(n_slices, -1)
        B = b[n_slices * off[e]: n_slices * off[e + 1]].reshape(n_slices, -1)
        blocks.append((np.linalg.norm(A - B, axis=1), np.linalg.norm(B, axis=1)))
    nbs = np.concatenate([nb for _, nb in blocks])
    ref = float(np.sqrt(np.mean(nbs ** 2))) if floor == "rms" else floor * float(nbs.max())
    return max(float((d / np.maximum(nb, ref)).max()) for d, nb in blocks)


class Sys:
    """One synthetic system: the plan, the oracle and the seeded inputs."""

    def __init__(self, cell, **plan_kw):
        from paper_1911_05633_gb300 import gw
        self.cell = cell
        self.plan = gw.Plan.from_cell(cell, **plan_kw)
        # N_PB of 128, 256 or 384 selects the tensor-core inverse unless the plan asks for Gauss-Jordan
        n = cell.n_pb_total
        assert self.plan.info["w_tensor"] == int(n % 128 == 0 and n <= 384 and plan_kw.get("w_solver") != "gauss_jordan")
        # beyond 384: block Gauss-Jordan over the largest pivot block of 256 or 128 dividing N_PB
        bs = next((b for b in (256, 128) if n > 384 and n % b == 0), 0)
        assert self.plan.info["w_block"] == (bs if plan_kw.get("w_solver") != "gauss_jordan" else 0)
        # the FP64 Sigma takes its W~ C^b stage from the tensor cores for K <= 64 unless the plan
        # asks for FP64 only
        # FP64-accurate tensor-core products (reductions up to 384 terms) unless the plan asks
        # for FP64 arithmetic only
        on = plan_kw.get("fp64_products") != "fp64"
        kmax = max(sp.n_prod for sp in cell.species)
        nmax = max(sp.n_orb for sp in cell.species)
        assert self.plan.info["sigma_tensor"] == int(on and kmax <= 384)
        assert self.plan.info["p_tensor"] == int(on and nmax * nmax <= 384)
        nn, nh = cell.nu_idx.size, (cell.n_tau + 1) // 2
        want = int(on) * (int(nn <= 384) | (2 * int(2 * nh <= 384)))
        assert self.plan.info["transform_tensor"] == want
        self.orc = oracle.OracleSystem(cell)
        assert np.array_equal(self.plan.entries, self.orc.entries)
        # the product-basis block of every entry (reduced beyond sphere B) as the oracle has it
        assert [self.plan.block_shape(e, "pb") for e in range(len(self.orc.entries))] == self.orc.kdims
        assert self.plan.info["n_entries_far"] == int(self.orc.far.sum())
        full = [(cell.n_prod_of(int(r[0])), cell.n_prod_of(int(r[1]))) for r in self.orc.entries]
        near = sum(1 for t, kd, fk in zip(self.orc.tier, self.orc.kdims, full) if t == 1 and kd != fk)
        assert self.plan.info["n_entries_near"] == near
        self.G_k = cell.green_k_tau()
        self.v_q, self.v_class = cell.coulomb()
        self.nt = cell.n_tau

    def G_R(self):
        if not hasattr(self, "_GR"):
            c = self.cell
            self._GR = oracle.fourier_k_to_R(self.G_k, self.orc.entries, self.orc.kmesh, c.orb_offsets, c.orb_offsets)
        return self._GR


_CACHE = {}


def system(name):
    if name not in _CACHE:
        if name == "c0":
            _CACHE[name] = Sys(synth.make_config(0))
        elif name == "c0_nosym":
            _CACHE[name] = Sys(synth.make_config(0), no_symmetry=True)
        elif name == "mixed":
            _CACHE[name] = Sys(synth.mixed_species_cell())
        elif name == "mixed_nonsym":
            _CACHE[name] = Sys(synth.mixed_species_cell(symmetric_C=False, n_tau=10))
        elif name == "c1":
            _CACHE[name] = Sys(synth.make_config(1))
        elif name == "c1_cut5":
            _CACHE[name] = Sys(synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)))
        elif name == "c1_cut5_gj":
            _CACHE[name] = Sys(synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)), w_solver="gauss_jordan")
        elif name == "c0_fp64":
            _CACHE[name] = Sys(synth.make_config(0), fp64_products="fp64")
        elif name == "c1_fp64":
            _CACHE[name] = Sys(synth.make_config(1), fp64_products="fp64")
        elif name == "c1_cut5_far":  # 24 of 48 product functions beyond the nearest neighbours
            _CACHE[name] = Sys(synth.with_far_basis(synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)),
                                                    4.0, [24]))
        elif name == "mixed_far":  # every pair but the onsite ones reduced: K 8 -> 5, 19 -> 11
            _CACHE[name] = Sys(synth.with_far_basis(synth.mixed_species_cell(), 4.0, [5, 11]))
        elif name == "c0_3tier":  # the three levels of Fig. 2: onsite 8, neighbour 5, image beyond 4.6 bohr 3
            _CACHE[name] = Sys(synth.with_far_basis(synth.make_config(0), 4.6, [3], n_prod_near=[5]))
        elif name == "c1_3tier":  # 8-atom cell, cutoff 7.5: nearest neighbours 36 of 48, second ones 24
            _CACHE[name] = Sys(synth.with_far_basis(synth.make_config(1, cutoff=7.5, n_tau=12, kmesh=(2, 2, 2)),
                                                    4.6, [24], n_prod_near=[36]))
        elif name == "c2_8_blk":  # N_PB 512: two pivot blocks of 256
            _CACHE[name] = Sys(synth.make_config(2, atoms=8, cutoff=5.0, n_tau=12))
        elif name == "c2_16_blk":  # N_PB 1024: four pivot blocks of 256
            _CACHE[name] = Sys(synth.make_config(2, atoms=16, cutoff=5.0, n_tau=12))
        elif name == "c2_16_k48_blk":  # N_PB 768: three pivot blocks of 256
            _CACHE[name] = Sys(synth.make_config(2, atoms=16, cutoff=5.0, n_tau=12,
                                                 species=[synth.Species("spd", 9, 48, None)]))
        elif name == "c1_far_fp64":
            _CACHE[name] = Sys(synth.with_far_basis(synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)),
                                                    4.0, [24]), fp64_products="fp64")
        else:
            raise KeyError(name)
    return _CACHE[name]


SMALL = ["c0", "mixed", "mixed_nonsym", "c1_cut5"]
FAR = ["c1_cut5_far", "mixed_far", "c0_3tier", "c1_3tier"]  # reduced product bases (Sec. 2, Fig. 2)


@pytest.mark.parametrize("name", SMALL + ["c1"])
def test_green_k_to_R(name):
    s = system(name)
    GR = host(s.plan.green_k_to_R(dev(s.G_k)))
    assert rel(GR, pack(s.G_R())) < TOL


@pytest.mark.parametrize("name", SMALL + FAR + ["c1", "c0_fp64", "c1_fp64", "c1_far_fp64"])
def test_polarizability(name):
    s = system(name)
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
    P = host(s.plan.polarizability_tau(dev(pack(s.G_R()))))
    assert rel(P, pack(ref)) < TOL
    assert rel_blocks(P, pack(ref), s.plan.off_pb, s.nt) < TOL


@pytest.mark.parametrize("name", SMALL + FAR + ["c1"])
@pytest.mark.parametrize("st,direction,kind", [("B", "tau_to_iw", "pb"), ("B", "iw_to_tau", "pb"),
                                               ("F", "tau_to_iw", "orb"), ("F", "iw_to_tau", "orb")])
def test_transform(name, st, direction, kind):
    s = system(name)
    rng = np.random.default_rng(17)
    T = s.orc.B_fwd if st == "B" else s.orc.F_fwd
    if direction == "iw_to_tau":
        T = s.orc.B_inv if st == "B" else s.orc.F_inv
    n_in = T.shape[1]
    blocks = []
    for e, row in enumerate(s.orc.entries):
        a, b = int(row[0]), int(row[1])
        r, c = s.orc.kdims[e] if kind == "pb" else (s.cell.n_orb_of(a), s.cell.n_orb_of(b))
        blocks.append(rng.standard_normal((n_in, r, c)) + 1j * rng.standard_normal((n_in, r, c)))
    ref = oracle.transform(T, blocks)
    out = host(s.plan.transform_tau_iw(st, direction, kind, dev(pack(blocks))))
    assert rel(out, pack(ref)) < TOL


@pytest.mark.parametrize("name", ["c0", "mixed", "c1_cut5", "c1", "c0_fp64", "c1_fp64"] + FAR)
def test_transform_structured_inputs(name):
    """gw_transform_tau_iw_ex: P(R, tau) with P(beta - tau) = P(tau)* (symmetric C) through
    the mirror-paired bosonic transform, and a real W~(R, i nu) through the real-input
    inverse, against the oracle's general transform."""
    s = system(name)
    assert s.plan.info["c_symmetric"] == 1
    PR = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
    ref = oracle.transform(s.orc.B_fwd, PR)
    out = host(s.plan.transform_tau_iw("B", "tau_to_iw", "pb", dev(pack(PR)), structure="mirror"))
    assert rel(out, pack(ref)) < TOL
    assert np.all(out.imag == 0.0)
    rng = np.random.default_rng(11)
    nn = s.cell.nu_idx.size
    Wr = [rng.standard_normal((nn,) + blk.shape[1:]) + 0j for blk in PR]
    ref = oracle.transform(s.orc.B_inv, Wr)
    out = host(s.plan.transform_tau_iw("B", "iw_to_tau", "pb", dev(pack(Wr)), structure="real"))
    assert rel(out, pack(ref)) < TOL
    from paper_1911_05633_gb300 import gw
    with pytest.raises(gw.GwError):
        s.plan.transform_tau_iw("F", "tau_to_iw", "orb", dev(pack(s.G_R())), structure="mirror")
    # only the frequencies nu >= 0: those slices as the oracle's, the others untouched
    ref = [b[s.cell.nu_idx >= 0] for b in oracle.transform(s.orc.B_fwd, PR)]
    sentinel = np.full(s.plan.len("pb", nn), 7.0 - 3.0j)
    out = dev(sentinel)
    s.plan.transform_tau_iw("B", "tau_to_iw", "pb", dev(pack(PR)), out=out, structure="mirror_nonneg")
    out = host(out)
    neg = s.cell.nu_idx < 0
    got, kept = [], []
    for e, blk in enumerate(PR):
        o = out[s.plan.off_pb[e] * nn:s.plan.off_pb[e + 1] * nn].reshape((nn,) + blk.shape[1:])
        got.append(o[~neg])
        kept.append(o[neg])
    assert rel(pack(got), pack(ref)) < TOL
    assert np.all(pack(kept) == 7.0 - 3.0j)


BLOCK = ["c2_8_blk", "c2_16_blk", "c2_16_k48_blk"]  # N_PB beyond 384: the block Gauss-Jordan inverse


@pytest.mark.parametrize("name", SMALL + FAR + BLOCK + ["c0_nosym", "c1_cut5_gj"])
def test_screened_W(name):
    s = system(name)
    PR = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
    Piw = oracle.transform(s.orc.B_fwd, PR)
    ref, _ = oracle.screened_W(Piw, s.orc.entries, s.v_q, s.orc.kmesh, s.cell.pb_offsets)
    W = host(s.plan.screened_W_iw(dev(pack(Piw)), dev(s.v_q)))
    s.plan.sync()
    assert rel(W, pack(ref)) < TOL


def test_screened_W_sampled_full_size():
    """The 8-atom, 4x4x4, 48-node workload: W~ checked on three bosonic frequencies."""
    s = system("c1")
    PR = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin)
    Piw = oracle.transform(s.orc.B_fwd, PR)
    W = host(s.plan.screened_W_iw(dev(pack(Piw)), dev(s.v_q)))
    s.plan.sync()
    nn = s.cell.nu_idx.size
    sel = [0, nn // 2, nn - 1]
    ref, _ = oracle.screened_W([x[sel] for x in Piw], s.orc.entries, s.v_q, s.orc.kmesh, s.cell.pb_offsets)
    off = s.plan.off_pb
    num = den = 0.0
    for e in range(len(off) - 1):
        blk = W[nn * off[e]: nn * off[e + 1]].reshape(nn, -1)[sel]
        r = ref[e].reshape(len(sel), -1)
        num += np.linalg.norm(blk - r) ** 2
        den += np.linalg.norm(r) ** 2
    assert (num / den) ** 0.5 < TOL


def _random_W(s, seed=23):
    rng = np.random.default_rng(seed)
    out = []
    for e, row in enumerate(s.orc.entries):
        Ka, Kb = s.orc.kdims[e]
        out.append(rng.standard_normal((s.nt, Ka, Kb)) + 1j * rng.standard_normal((s.nt, Ka, Kb)))
    return out


@pytest.mark.parametrize("name", SMALL + FAR + ["c1", "c0_fp64", "c1_fp64", "c1_far_fp64"])
def test_self_energy_and_exchange(name):
    s = system(name)
    WR = _random_W(s)
    vR = s.orc.v_R(s.v_class)
    ref = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    refx = oracle.exchange_R(s.G_R(), vR, s.orc.entries, s.orc.C_atom)
    Sig, Sigx = s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)), v_R=dev(pack(vR)))
    assert rel(host(Sig), pack(ref)) < TOL
    assert rel(host(Sigx), pack(refx)) < TOL
    assert rel_blocks(host(Sig), pack(ref), s.plan.off_orb, s.nt) < TOL
    assert rel_blocks(host(Sigx), pack(refx), s.plan.off_orb, 1) < TOL


@pytest.mark.parametrize("name", SMALL + FAR + ["c1"])
def test_fourier_R_to_k(name):
    s = system(name)
    rng = np.random.default_rng(5)
    blocks = []
    for row in s.orc.entries:
        a, b = int(row[0]), int(row[1])
        na, nb = s.cell.n_orb_of(a), s.cell.n_orb_of(b)
        blocks.append(rng.standard_normal((3, na, nb)) + 1j * rng.standard_normal((3, na, nb)))
    oo = s.cell.orb_offsets
    ref = oracle.fourier_R_to_k(blocks, s.orc.entries, s.orc.kmesh, oo, oo)
    out = host(s.plan.fourier_R_to_k("orb", 3, dev(pack(blocks))))
    assert rel(out, ref.reshape(-1)) < TOL
    # product-basis blocks, one slice (the k -> R inverse on all-class systems)
    vq = host(s.plan.fourier_R_to_k("pb", 1, dev(pack(s.orc.v_R(s.v_class)))))
    po = s.cell.pb_offsets
    refv = oracle.fourier_R_to_k([x[None] for x in s.orc.v_R(s.v_class)], s.orc.entries, s.orc.kmesh, po, po)
    assert rel(vq, refv.reshape(-1)) < TOL


@pytest.mark.parametrize("name", ["c0", "c0_nosym", "mixed", "mixed_nonsym", "c1_cut5", "c1_cut5_gj"] + FAR)
def test_whole_sweep(name):
    """All rows chained on the device from G(k, tau) and v(q); every stage vs the oracle."""
    s = system(name)
    p = s.plan
    r = s.orc.sweep(s.G_k, s.v_q, s.v_class)
    GR = p.green_k_to_R(dev(s.G_k))
    PR = p.polarizability_tau(GR)
    # the structured transforms where the plan's symmetries provide them (as bench.py runs)
    inf = p.info
    Piw = p.transform_tau_iw("B", "tau_to_iw", "pb", PR, structure="mirror" if inf["c_symmetric"] else "general")
    Wiw = p.screened_W_iw(Piw, dev(s.v_q))
    WR = p.transform_tau_iw("B", "iw_to_tau", "pb", Wiw, structure="real" if inf["w_symmetric"] else "general")
    vR = p.fourier_k_to_R("pb", 1, dev(s.v_q))
    Sig, Sigx = p.self_energy_tau(GR, WR, v_R=vR)
    Siw = p.transform_tau_iw("F", "tau_to_iw", "orb", Sig)
    Sk = p.fourier_R_to_k("orb", s.cell.omega_idx.size, Siw)
    Sxk = p.fourier_R_to_k("orb", 1, Sigx)
    p.sync()
    assert rel(host(GR), pack(r["G_R"])) < TOL
    assert rel(host(PR), pack(r["P_R"])) < TOL
    assert rel(host(Piw), pack(r["P_iw"])) < TOL
    assert rel(host(Wiw), pack(r["Wt_iw"])) < TOL
    assert rel(host(WR), pack(r["Wt_R"])) < TOL
    assert rel(host(vR), pack(r["v_R"])) < TOL
    assert rel(host(Sig), pack(r["Sig_R"])) < TOL
    assert rel(host(Sigx), pack(r["Sigx_R"])) < TOL
    assert rel(host(Sk), r["Sig_k"].reshape(-1)) < TOL
    assert rel(host(Sxk), r["Sigx_k"].reshape(-1)) < TOL
    # block by block for every entry-layout stage (the far entries and the middle of the tau grid included)
    nt, nn, nw = s.nt, s.cell.nu_idx.size, s.cell.omega_idx.size
    oo, op = p.off_orb, p.off_pb
    for got, ref, off, ns, fl in ((GR, r["G_R"], oo, nt, 1e-6), (PR, r["P_R"], op, nt, 1e-6),
                                  (Piw, r["P_iw"], op, nn, "rms"), (Wiw, r["Wt_iw"], op, nn, "rms"),
                                  (WR, r["Wt_R"], op, nt, "rms"), (Sig, r["Sig_R"], oo, nt, "rms"),
                                  (Sigx, r["Sigx_R"], oo, 1, 1e-6)):
        assert rel_blocks(host(got), pack(ref), off, ns, fl) < TOL


def test_largest_blocks():
    """n = 16 orbitals and K = 128 product functions (the compiled maxima), one atom."""
    lat = np.eye(3) * 6.0
    sp = [synth.Species("big", 16, 128, None)]
    cell = synth.SynthCell("big1", lat, np.zeros((1, 3)), np.zeros(1, np.int32), sp, (2, 1, 1), 20.0, 8, 0.0,
                           seed=77, gap=None, hop_cutoff=6.5).build()
    s = Sys(cell)
    ref = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, cell.spin)
    assert rel(host(s.plan.polarizability_tau(dev(pack(s.G_R())))), pack(ref)) < TOL
    WR = _random_W(s)
    refS = oracle.self_energy_R(s.G_R(), WR, s.orc.entries, s.orc.C_atom)
    assert rel(host(s.plan.self_energy_tau(dev(pack(s.G_R())), dev(pack(WR)))), pack(refS)) < TOL


def test_full_size_72_atoms_sampled():
    """The 72-atom, 2x2x2, 64-node workload: G(R), P and Sigma on sampled entries."""
    cell = synth.make_config(2)
    from paper_1911_05633_gb300 import gw
    plan = gw.Plan.from_cell(cell)
    ent = plan.entries
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(len(ent), 12, replace=False))
    Gk = cell.green_k_tau()
    GR_dev = plan.green_k_to_R(dev(Gk))
    GR = host(GR_dev)
    oo = cell.orb_offsets
    refG = oracle.fourier_k_to_R(Gk, ent[sample], cell.kmesh, oo, oo)
    del Gk
    nt = cell.n_tau
    C_atom = [cell.species[s].C for s in cell.species_of_atom]
    P = host(plan.polarizability_tau(GR_dev))
    refP = oracle.polarizability_R(refG, ent[sample], C_atom, cell.spin)
    # W~ is zero except on the sampled entries (the full array would be 14 GB on the host)
    torch = _torch()
    W_dev = torch.zeros(plan.len("pb", nt), dtype=torch.complex128, device="cuda")
    rw = np.random.default_rng(9)
    WS = []
    for e in sample:
        w = rw.standard_normal((nt, 64, 64)) + 1j * rw.standard_normal((nt, 64, 64))
        WS.append(w)
        W_dev[nt * plan.off_pb[e]: nt * plan.off_pb[e + 1]] = dev(w)
    Sig = host(plan.self_energy_tau(GR_dev, W_dev))
    refS = oracle.self_energy_R(refG, WS, ent[sample], C_atom)
    keep = np.zeros(len(ent), bool)
    keep[sample] = True
    for e in np.nonzero(~keep)[0][:50]:
        assert not Sig[nt * plan.off_orb[e]: nt * plan.off_orb[e + 1]].any()
    for j, e in enumerate(sample):
        g = GR[nt * plan.off_orb[e]: nt * plan.off_orb[e + 1]]
        assert rel(g, refG[j].reshape(-1)) < TOL
        pe = P[nt * plan.off_pb[e]: nt * plan.off_pb[e + 1]]
        assert rel(pe, refP[j].reshape(-1)) < TOL
        se = Sig[nt * plan.off_orb[e]: nt * plan.off_orb[e + 1]]
        assert rel(se, refS[j].reshape(-1)) < TOL
