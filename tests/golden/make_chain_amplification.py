"""Writes chain_amplification.txt: how much the oracle's own chain
P(R, tau) -> P(R, i nu) -> W~ (Eq. W_1) -> W~(R, tau) -> Sigma(R, tau) (Eq. S_MM) -> Sigma(k, i w)
magnifies a relative perturbation of P, per test system.

P is multiplied element by element by 1 + 1e-7 x (seeded normal numbers); the ratio of the
relative change of Sigma(R, tau) and of Sigma(k, i w) to the relative change of P is recorded,
the largest over four seeds.  The mixed-precision chain tests hold the device's Sigma error
to a multiple of this ratio times its measured P error: the W solve of a nearly singular
1 - v P (the short-cutoff cells) magnifies any error of P, whatever its source.

Calls only oracle/ and the seeded inputs of synth/.  Usage:
    python tests/golden/make_chain_amplification.py [names...]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

CELLS = {
    "c0": lambda: synth.make_config(0),
    "c1_cut5": lambda: synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)),
    "c1_cut5_far": lambda: synth.with_far_basis(synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)), 4.0, [24]),
    "c1": lambda: synth.make_config(1),
}


def _chain(orc, c, PR, vq, GR):
    Wiw, _ = oracle.screened_W(oracle.transform(orc.B_fwd, PR), orc.entries, vq, orc.kmesh, c.pb_offsets)
    SR = oracle.self_energy_R(GR, oracle.transform(orc.B_inv, Wiw), orc.entries, orc.C_atom)
    Sk = oracle.fourier_R_to_k(oracle.transform(orc.F_fwd, SR), orc.entries, orc.kmesh, c.orb_offsets, c.orb_offsets)
    return np.concatenate([x.ravel() for x in SR]), Sk.ravel()


def amplification(c, seeds=(0, 1, 2, 3)):
    orc = oracle.OracleSystem(c)
    vq, _ = c.coulomb()
    GR = oracle.fourier_k_to_R(c.green_k_tau(), orc.entries, orc.kmesh, c.orb_offsets, c.orb_offsets)
    PR = oracle.polarizability_R(GR, orc.entries, orc.C_atom, c.spin, orc.kdims)
    P0 = np.concatenate([p.ravel() for p in PR])
    a0, b0 = _chain(orc, c, PR, vq, GR)
    amp_R = amp_k = 0.0
    for s in seeds:
        rng = np.random.default_rng(s)
        PRn = [p * (1 + 1e-7 * rng.standard_normal(p.shape)) for p in PR]
        dP = np.linalg.norm(np.concatenate([p.ravel() for p in PRn]) - P0) / np.linalg.norm(P0)
        a, b = _chain(orc, c, PRn, vq, GR)
        amp_R = max(amp_R, np.linalg.norm(a - a0) / np.linalg.norm(a0) / dP)
        amp_k = max(amp_k, np.linalg.norm(b - b0) / np.linalg.norm(b0) / dP)
    return amp_R, amp_k


def _write(path, rows):
    with open(path, "w") as f:
        f.write("# Oracle chain P -> W~ (Eq. W_1) -> Sigma (Eq. S_MM): relative change of Sigma per relative\n"
                "# change of P (largest over 4 seeded perturbations of 1e-7).  Written by\n"
                "# make_chain_amplification.py (oracle and synth only).\n"
                "# columns: system  amplification_Sigma_R_tau  amplification_Sigma_k_iw\n")
        for n in CELLS:
            if n in rows:
                f.write(f"{n} {rows[n][0]:.4g} {rows[n][1]:.4g}\n")


def main(names):
    path = os.path.join(HERE, "chain_amplification.txt")
    rows = {}
    if os.path.exists(path):
        for l in open(path):
            if l.strip() and not l.startswith("#"):
                f = l.split()
                rows[f[0]] = (float(f[1]), float(f[2]))
    for n in names:
        rows[n] = amplification(CELLS[n]())
        print(n, rows[n], flush=True)
        _write(path, rows)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CELLS))
