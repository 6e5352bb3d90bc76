#!/usr/bin/env python3
"""Benchmark of the real-space / imaginary-time GW sweep on one GB300 per rank.

One step = one pass of the P + Sigma rows of the sweep over the 72-atom diamond-like
supercell (3x3x1 of the 8-atom cell; n = 9 orbitals, K = 64 product functions per
atom, 2x2x2 k-mesh, beta = 1000, 64 tau nodes, 12-bohr cutoff: 3312 pair entries):
  G(k,tau) -> G(R,tau) -> P(R,tau) -> P(R,i nu)            (rows a1, a2, a3)
  W~(R,i nu) -> W~(R,tau) -> Sigma(R,tau) + Sigma_x        (rows a6, a7)
  -> Sigma(R,i omega) -> Sigma(k,i omega), Sigma_x(k)      (row a8)
The W solve between P(R,i nu) and W~(R,i nu) (Eq. W_1, with the dense momentum-space
halves of rows a4 and a6 that stream inside it) is timed apart, as the metric states
(`w_solve`: the same cell's solve on the P of its own FP64 rows); inside the rows
W~(R,i nu) and v(R) are seeded inputs of the plan's shapes.
Inputs G(k,tau), W~(R,i nu) and v(R) are resident in HBM when the timed region starts.

`value` is P+Sigma sweeps per second in mixed precision (BF16x3 contractions with FP32
accumulation, FP64-accurate transforms), summed over ranks (weak scaling: each rank
runs its own replica; the sweep does not shard).  The FP64 path of the same rows is
timed beside it (`fp64`), the 8-atom workload's whole sweep with its W solve is kept as
`full_sweep_8_atoms`, the batched uneven systems as `batched_uneven_systems`.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P+Σ sweep time & TFLOP/s vs peak; serve p50/p99; mixed vs FP64 at 1e-6 rel err"
UNIT = "sweep/s"

# DRAM traffic per launch of a kernel from an ncu capture (profiles/), valid only while
# the kernel's source file is unchanged since the capture: bytes per unit there x units
# in this launch.
TRAFFIC = {
    # bench.py --small captures (56 matrices of N_PB = 384 per launch): DRAM read + write / 56
    "k_gj_inverse_f32": {"file": "kernels_wtc.cu", "src_sha": "818f6fc1dcc6cb59",
                         "bytes_per_unit": (66.10e6 + 254.12e6) / 56},
    # bench.py --atoms 8 captures (profiles/k_contract_diamond8_small.md): 352 entries of the
    # same species as the 72-atom cell; units are (entry, node) pairs: 352 x 64 for Sigma,
    # 352 x 32 computed nodes for P (each writing its node and the mirrored one)
    "k_contract_s_tc": {"file": "kernels_contract.cu", "src_sha": "67b0441118f621b0",
                        "bytes_per_unit": (1.506173e9 + 0.031087e9) / (352 * 64)},
    "k_contract_p_tc": {"file": "kernels_contract.cu", "src_sha": "67b0441118f621b0",
                        "bytes_per_unit": (0.029668e9 + 1.465074e9) / (352 * 32)},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="precision of `value` (the other one is timed beside it)")
    ap.add_argument("--config", type=int, default=2,
                    help="2: P+Sigma rows of the 72-atom cell (default); 1: the 8-atom whole sweep with its W solve")
    ap.add_argument("--atoms", type=int, default=72, help="configuration 2 series: 8, 16, 32, 48 or 72 atoms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 8-atom whole sweep and its error report")
    ap.add_argument("--no-dyson", action="store_true", help="skip the Eq. G_1 step timed after the sweep")
    ap.add_argument("--small", action="store_true", help="the small profiling case instead of the bench workload")
    ap.add_argument("--w-solver", default="auto", choices=["auto", "gauss_jordan"],
                    help="inverse of the W solve: tensor-core refinement where supported, or FP64 Gauss-Jordan")
    ap.add_argument("--fp64-products", default="auto", choices=["auto", "fp64"],
                    help="FP64 Sigma: its W~ C^b stage as FP64-accurate tensor-core products, or FP64 arithmetic")
    ap.add_argument("--r-b", type=float, default=0.0,
                    help="radius of sphere B (bohr): pairs beyond it keep --n-prod-far product functions (Sec. 2)")
    ap.add_argument("--n-prod-far", type=int, nargs="+", default=None,
                    help="product functions per species kept by pairs beyond sphere B")
    ap.add_argument("--batch", action="store_true",
                    help="only the batched uneven systems (the 16-system family in one launch per contraction)")
    ap.add_argument("--serve", action="store_true",
                    help="Poisson request stream of whole GW iterations: p50/p99 latency")
    ap.add_argument("--w-solve", action="store_true",
                    help="time the W solve (Eq. W_1) of the configuration-2 cell of --atoms atoms on the P of "
                         "its own FP64 rows; one JSON line")
    ap.add_argument("--workspace-gb", type=float, default=0.0,
                    help="--w-solve: cap on the W-solve scratch in GB (0: the library's default)")
    ap.add_argument("--scaling", type=int, nargs="*", default=None,
                    help="time the P+Sigma rows (no W solve) of the 64-function diamond series at these atom "
                         "counts (default 8 16 32 48 72), FP64 and mixed; one JSON line")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(step_ms: float, world: int):
    """Whole-job figures of a replicated run (every rank sweeps its own copy of the
    workload): the slowest rank's ms per step and the sweeps per second of all ranks
    together, world / that time."""
    step_ms_max = max_over_ranks(step_ms, world)
    return step_ms_max, world * 1000.0 / step_ms_max


# --------------------------------------------------------------------------------------
# workload and its algorithmic work
# --------------------------------------------------------------------------------------

def workload(cfg: int, small: bool = False, r_b: float = 0.0, n_prod_far=None, atoms: int = 72):
    """The bench workload: configuration 2 (the diamond supercell series, 72 atoms by
    default), configuration 1 (the 8-atom cell), or with `small` the 8-atom cell on a 2x2x2
    mesh with 12 tau nodes and a 5-bohr cutoff (N_PB = 384, 64 W-solve matrices): a case
    small enough for full ncu captures of single kernels.  r_b > 0: pairs beyond sphere B
    keep n_prod_far product functions per species (the reduced basis of Sec. 2)."""
    import synth
    if small:
        cell = synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2))
    elif cfg == 2:
        cell = synth.make_config(2, atoms=atoms)
    else:
        cell = synth.make_config(cfg)
    if r_b > 0:
        synth.with_far_basis(cell, r_b, n_prod_far or [max(1, sp.n_prod // 4) for sp in cell.species])
    return cell


def pb_dims(plan):
    """(K_a(e), K_b(e)) of every entry, as the plan lays them out."""
    return [plan.block_shape(e, "pb") for e in range(len(plan.entries))]


def contraction_flops(cell, entries, kdims) -> float:
    """Real flops of one P (or Sigma) contraction over all entries and tau nodes:
    2 (2 K_a n_a^2 n_b + 4 K_a n_a n_b^2 + 2 K_a K_b n_b^2) per (entry, tau), K_a and K_b
    the entry's product-basis sizes."""
    f = 0.0
    for (a, b), (Ka, Kb) in zip(entries[:, :2], kdims):
        na, nb = cell.n_orb_of(int(a)), cell.n_orb_of(int(b))
        f += 2.0 * (2 * Ka * na * na * nb + 4 * Ka * na * nb * nb + 2 * Ka * Kb * nb * nb)
    return f * cell.n_tau


def kernel_work(name: str, cell, info, entries, kdims):
    """Algorithmic work of one sweep for the kernels that can dominate it: (bound,
    work, kind, units) with flops for "alu"/"tensor" (real flops) and bytes for "hbm",
    and `units` the matrices (W solve) or pair entries the sweep processes; None for
    the others.  Per launch = this / launches per sweep."""
    N = cell.n_pb_total
    nq = info["n_q_solved"]
    nnu = int((cell.nu_idx >= 0).sum()) if info["w_symmetric"] else cell.nu_idx.size
    n_inv = nq * (nnu + 1)  # v(q) once, then every solved (q, nu)
    gj = 8.0 * N ** 3 * n_inv  # complex Gauss-Jordan inverse, or one complex N^3 product
    nt, nn, nw = info["n_tau"], info["n_nu"], info["n_omega"]
    if name in ("k_gj_inverse_blocked", "k_gj_inverse"):
        return "alu", gj, "fp64", n_inv
    if name == "k_gj_inverse_f32":
        return "alu", gj, "fp32", n_inv
    if name in ("k_refine_tc<first>", "k_refine_tc<final>"):  # 6 term pairs x 4 real products of 2 N^3
        return "tensor", 4 * 6 * 2.0 * N ** 3 * n_inv, "bf16", n_inv
    if name == "k_ozaki_residual<first>":  # 20 slice pairs x 4 real products of 2 N^3
        return "tensor", 4 * 20 * 2.0 * N ** 3 * n_inv, "bf16", n_inv
    if name == "k_ozaki_residual<second>":  # 36 slice pairs
        return "tensor", 4 * 36 * 2.0 * N ** 3 * n_inv, "bf16", n_inv
    if name == "k_polarizability_fp64":  # stages 1 and 2 only when stage 3 runs on the tensor cores
        f = stage_bc_flops(cell, entries, kdims) if info["p_tensor"] else contraction_flops(cell, entries, kdims)
        return "alu", f / (2 if info["c_symmetric"] else 1), "fp64", len(entries)
    if name == "k_self_energy_fp64":  # dynamic part (stages B, C only when stage A runs on the tensor cores)
        full = contraction_flops(cell, entries, kdims)  # and the one-slice exchange term (all stages)
        dyn = stage_bc_flops(cell, entries, kdims) if info["sigma_tensor"] else full
        return "alu", dyn + full / nt, "fp64", len(entries)
    if name == "k_oz_gemm":  # 36 digit pairs x 2 flops x rows x padded K x padded N, every use in a sweep
        f = oz_gemm_flops(cell, entries, kdims) if info["sigma_tensor"] else 0.0
        pad = lambda x, m: -(-x // m) * m
        rows = info["len_pb"]
        if info["p_tensor"]:  # P stage 3: 2 K_a rows per (entry, computed node), K = n_b^2, N = K_b
            ntp = oz_nt(max(cell.n_prod_of(i) for i in range(cell.n_atoms)))
            ne = (nt + 1) // 2 if info["c_symmetric"] else nt
            for (a, b), (Ka, Kb) in zip(entries[:, :2], kdims):
                nb = cell.n_orb_of(int(b))
                f += ne * 2 * Ka * 36 * 2.0 * pad(nb * nb, 16) * pad(Kb, ntp)
        if info["transform_tensor"] & 1 and info["w_symmetric"]:  # W~ i nu -> tau, real input
            f += rows * 36 * 2.0 * pad(nn, 16) * pad(2 * nt, oz_nt(2 * nt))
        if info["transform_tensor"] & 2 and info["c_symmetric"]:  # P tau -> i nu, mirror pairs
            nh = (nt + 1) // 2
            f += rows * 36 * 2.0 * pad(2 * nh, 16) * pad(nn, oz_nt(nn))
        return "tensor", f, "bf16", len(entries)
    if name == "k_transform":  # real flops per block element: 8 n_out n_in (general), 2 n_out ceil(n_in / 2)
        # (mirror-paired input), 4 n_out n_in (real input)
        fP = 2 * nn * ((nt + 1) // 2) if info["c_symmetric"] else 8 * nn * nt
        fW = 4 * nt * nn if info["w_symmetric"] else 8 * nt * nn
        if info["c_symmetric"] and info["transform_tensor"] & 2:  # done by k_oz_gemm instead
            fP = 0
        if info["w_symmetric"] and info["transform_tensor"] & 1:
            fW = 0
        return "alu", float((fP + fW) * info["len_pb"] + 8 * nw * nt * info["len_orb"]), "fp64", 3 * len(entries)
    if name == "k_slice_A":  # FP64 in, 8 x 2 BF16 digits out per element
        return "hbm", (16 + 32) * N * N * n_inv, "bytes", n_inv
    return None


def stage_bc_flops(cell, entries, kdims) -> float:
    """Real flops of the two small stages of a contraction (Sigma after B = W~ C^b, or P
    before Y C^b): 2 (2 K_a n_a^2 n_b + 4 K_a n_a n_b^2) per (entry, tau)."""
    f = 0.0
    for (a, b), (Ka, _) in zip(entries[:, :2], kdims):
        na, nb = cell.n_orb_of(int(a)), cell.n_orb_of(int(b))
        f += 2.0 * (2 * Ka * na * na * nb + 4 * Ka * na * nb * nb)
    return f * cell.n_tau


def stage3_flops(cell, entries, kdims, row: str) -> float:
    """Real flops of the dense stage of a contraction per tau node, summed over entries:
    Y C^b of P or W~ C^b of Sigma, 2 x 2 K_a K_b n_b^2 per (entry, tau)."""
    f = 0.0
    for (a, b), (Ka, Kb) in zip(entries[:, :2], kdims):
        nb = cell.n_orb_of(int(b))
        f += 2.0 * 2 * Ka * Kb * nb * nb
    return f


def p_iw_structure(inf) -> str:
    """How P(R, tau) goes to P(R, i nu): mirror-paired when C is symmetric, and only the
    frequencies nu >= 0 when the W solve reads no others (a w_symmetric plan)."""
    if not inf["c_symmetric"]:
        return "general"
    return "mirror_nonneg" if inf["w_symmetric"] else "mirror"


def row_work(cell, entries, kdims, row: str, c_symmetric: int):
    """Algorithmic work of one contraction row over one sweep: (real flops, DRAM bytes,
    BF16x3 tensor flops of its dense stage, FP32 flops of its small stages).
    P: the computed tau nodes (half of them, the mirrored ones written as conjugates, when C is
    symmetric), reading G(tau) and G(beta - tau) once and writing every P(tau) slice.
    Sigma: every tau node, reading G and W~ and writing Sigma (the one-slice exchange apart)."""
    nt = cell.n_tau
    ne = (nt + 1) // 2 if (row == "P" and c_symmetric) else nt
    fl = contraction_flops(cell, entries, kdims) * ne / nt
    dense = stage3_flops(cell, entries, kdims, row) * ne
    small = fl - dense
    byt = 0.0
    for (a, b), (Ka, Kb) in zip(entries[:, :2], kdims):
        na, nb = cell.n_orb_of(int(a)), cell.n_orb_of(int(b))
        if row == "P":
            byt += nt * 16.0 * (na * nb + Ka * Kb)
        else:
            byt += nt * 16.0 * (2 * na * nb + Ka * Kb)
    return fl, byt, 6.0 * dense, small


def contraction_roofline(kernel, ms_per_step, launches_per_step, work, peaks, fp32_peak, fp64_peak, mixed):
    """Roofline of one contraction kernel from its live event times.  The floors: its
    algorithmic DRAM bytes at the measured HBM peak, and its arithmetic at the peak of the
    unit that runs it (mixed: BF16x3 tensor flops of the dense stage at the sustained BF16
    peak, the small stages at the FP32 peak; FP64: all flops at the FP64 peak).  `bound` is
    the largest floor; `achieved` is the algorithmic work of that bound per launch over the
    mean launch time."""
    fl, byt, tens, small = work
    dur = ms_per_step * 1e-3 / launches_per_step
    hbm = peaks.get("hbm_gbs")
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    floors = {"hbm": byt / launches_per_step / (hbm * 1e9) if hbm else 0.0}
    if mixed:
        floors["tensor"] = tens / launches_per_step / (bf16 * 1e12) if bf16 else 0.0
        floors["alu"] = small / launches_per_step / (fp32_peak * 1e12) if fp32_peak else 0.0
    else:
        floors["alu"] = fl / launches_per_step / (fp64_peak * 1e12) if fp64_peak else 0.0
    bound = max(floors, key=floors.get)
    if bound == "hbm":
        ach, peak, unit, src = byt / launches_per_step / dur / 1e9, hbm, "GB/s", "measured HBM copy (hbm_gbs)"
    elif bound == "tensor":
        ach, peak, unit = tens / launches_per_step / dur / 1e12, bf16, "TFLOP/s"
        src = "measured cuBLAS BF16 sustained (bf16_tflops_sustained); achieved counts the BF16x3 products"
    elif mixed:
        ach, peak, unit = small / launches_per_step / dur / 1e12, fp32_peak, "TFLOP/s"
        src = "FP32 FMA-chain probe (gw_fp_peak) on this GPU before the timed region"
    else:
        ach, peak, unit = fl / launches_per_step / dur / 1e12, fp64_peak, "TFLOP/s"
        src = "FP64 FMA-chain probe (gw_fp_peak) on this GPU before the timed region"
    return {"kernel": kernel, "bound": bound, "achieved": round(ach, 4), "peak": round(peak, 4) if peak else None,
            "unit": unit, "frac": round(ach / peak, 4) if peak else None, "traffic": None, "peak_source": src,
            "launch_ms": round(dur * 1e3, 4), "algorithmic_bytes_per_launch": byt / launches_per_step,
            "algorithmic_flops_per_launch": fl / launches_per_step,
            "algorithmic_tflops": round(fl / launches_per_step / dur / 1e12, 4),
            "emulation": ({"bf16x3_tensor_flops_per_launch": tens / launches_per_step,
                           "tensor_frac_of_bf16_sustained": round(tens / launches_per_step / dur / 1e12 / bf16, 4)
                           if bf16 else None} if mixed else None),
            "floors_ms": {k: round(v * 1e3, 4) for k, v in floors.items()}}


def oz_nt(n_cols: int) -> int:
    """Column tile of the digit-product GEMM: the multiple of 16 up to 80 with the least
    padding of n_cols, the wider on ties."""
    NT, best = 16, 1 << 30
    for c in range(16, 81, 16):
        padded = -(-n_cols // c) * c
        if padded <= best:
            best, NT = padded, c
    return NT


def oz_gemm_flops(cell, entries, kdims) -> float:
    """Tensor flops of the FP64-accurate W~ C^b products: per (entry, tau) 2 K_a rows
    x 36 digit pairs x 2 x (the entry's K_b padded to 16) x (n_b^2 padded to the column
    tile)."""
    NT = oz_nt(max(cell.n_orb_of(i) ** 2 for i in range(cell.n_atoms)))
    f = 0.0
    for (a, b), (Ka, Kb) in zip(entries[:, :2], kdims):
        nb = cell.n_orb_of(int(b))
        f += 2 * Ka * 36 * 2.0 * (-(-Kb // 16) * 16) * (-(-nb * nb // NT) * NT)
    return f * cell.n_tau


def wsolve_flops(cell, info) -> float:
    """Gauss-Jordan inverses of v(q) and of v(q)^{-1} - P(q, i nu): 8 N^3 real flops
    each, over the momenta and frequencies the plan actually solves."""
    N = cell.n_pb_total
    nq = info["n_q_solved"]
    nnu = int((cell.nu_idx >= 0).sum()) if info["w_symmetric"] else cell.nu_idx.size
    return 8.0 * N ** 3 * nq * (nnu + 1)


# --------------------------------------------------------------------------------------
# clocks sampling (nvidia-smi) during the timed region
# --------------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------

# --------------------------------------------------------------------------------------
# our arm, main line: the P + Sigma rows of configuration 2
# --------------------------------------------------------------------------------------

class RowSweep:
    """Device buffers and the ordered calls of the P + Sigma rows (the W solve apart):
    G(k,tau) -> G(R,tau) -> P(R,tau) -> P(R,i nu); W~(R,i nu) -> W~(R,tau) -> Sigma(R,tau)
    + Sigma_x -> Sigma(R,i w) -> Sigma(k,i w), Sigma_x(k)."""

    STAGES = ["G_k_to_R", "P", "P_tau_to_nu", "W_nu_to_tau", "Sigma", "Sigma_tau_to_omega", "Sigma_R_to_k"]

    def __init__(self, cell, device: int = 0, seed: int = 0):
        import torch
        from paper_1911_05633_gb300 import gw
        self.torch = torch
        self.cell = cell
        self.prec = "mixed"
        self.plan = gw.Plan.from_cell(cell, device=device, defer_scratch=True)  # no W solve here
        p, inf = self.plan, self.plan.info
        self.dev = torch.device("cuda", device)
        z = lambda n: torch.empty(n, dtype=torch.complex128, device=self.dev)
        nt, nn, nw, No, nk = inf["n_tau"], inf["n_nu"], inf["n_omega"], inf["n_orb_total"], inf["n_k"]
        self.G_k = z(nk * nt * No * No)
        self.G_R, self.P_R, self.P_iw = z(p.len("orb", nt)), z(p.len("pb", nt)), z(p.len("pb", nn))
        self.W_iw, self.W_R, self.v_R = z(p.len("pb", nn)), z(p.len("pb", nt)), z(p.len("pb", 1))
        self.S_R, self.Sx_R, self.S_iw = z(p.len("orb", nt)), z(p.len("orb", 1)), z(p.len("orb", nw))
        self.S_k, self.Sx_k = z(nk * nw * No * No), z(nk * No * No)
        # seeded stand-ins for the W solve's output (real: the plan's symmetric W mode) and v(R)
        gen = torch.Generator(device=self.dev).manual_seed(seed)
        self.W_iw.copy_(torch.randn(self.W_iw.numel(), dtype=torch.float64, device=self.dev, generator=gen))
        self.v_R.copy_(torch.randn(self.v_R.numel(), dtype=torch.float64, device=self.dev, generator=gen))

    def load_G(self, G_k_host):
        self.G_k.copy_(self.torch.from_numpy(G_k_host.reshape(-1)))

    def run(self, stream, events=None):
        p, s = self.plan, stream.cuda_stream
        inf = p.info
        calls = [
            lambda: p.green_k_to_R(self.G_k, self.G_R, stream=s),
            lambda: p.polarizability_tau(self.G_R, self.P_R, precision=self.prec, stream=s),
            lambda: p.transform_tau_iw("B", "tau_to_iw", "pb", self.P_R, self.P_iw, stream=s,
                                       structure=p_iw_structure(inf)),
            lambda: p.transform_tau_iw("B", "iw_to_tau", "pb", self.W_iw, self.W_R, stream=s,
                                       structure="real" if inf["w_symmetric"] else "general"),
            lambda: p.self_energy_tau(self.G_R, self.W_R, v_R=self.v_R, Sig_R=self.S_R, Sigx_R=self.Sx_R,
                                      precision=self.prec, stream=s),
            lambda: p.transform_tau_iw("F", "tau_to_iw", "orb", self.S_R, self.S_iw, stream=s),
            lambda: (p.fourier_R_to_k("orb", inf["n_omega"], self.S_iw, self.S_k, stream=s),
                     p.fourier_R_to_k("orb", 1, self.Sx_R, self.Sx_k, stream=s)),
        ]
        for i, c in enumerate(calls):
            if events is not None:
                events[i][0].record(stream)
            c()
            if events is not None:
                events[i][1].record(stream)


def time_rows(sw, stream, flush, steps, warmup, clocks=None):
    """Warm-up, then `steps` sweeps, each after an L2 flush, with a CUDA event pair around
    every row on the launching stream and the library's event pair around every kernel.
    Returns (ms per sweep, ms per row, {kernel: (total ms, launches)}, clocks)."""
    torch = sw.torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            sw.run(stream)
    sw.plan.sync(stream=stream.cuda_stream)
    torch.cuda.synchronize()
    nst = len(sw.STAGES)
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nst)] for _ in range(steps)]
    sw.plan.timing_reset()
    sw.plan.timing_enable(True)
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush_l2(flush)
            sw.run(stream, ev[k])
    sw.plan.sync(stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    kt = sw.plan.timing_read()
    sw.plan.timing_enable(False)
    stage_ms = np.array([[ev[k][i][0].elapsed_time(ev[k][i][1]) for i in range(nst)] for k in range(steps)])
    return float(stage_ms.sum(axis=1).mean()), stage_ms.mean(axis=0), kt, clk


def kernels_table(kt, steps):
    tot = sum(v[0] for v in kt.values()) or 1.0
    return {k: {"ms_per_step": round(v[0] / steps, 4), "launches_per_step": v[1] / steps, "share": round(v[0] / tot, 4)}
            for k, v in sorted(kt.items(), key=lambda x: -x[1][0])}


# the contraction kernels of rows a2 (P) and a7 (Sigma) by precision
CONTRACTION_KERNELS = {
    "k_polarizability_tc": ("P", True), "k_polarizability_f32": ("P", True),
    "k_self_energy_tc": ("S", True), "k_self_energy_f32": ("S", True),
    "k_contract_p_tc": ("P", True), "k_contract_s_tc": ("S", True),
    "k_polarizability_fp64": ("P", False), "k_self_energy_fp64": ("S", False),
}


def dominant_contraction_roofline(kt, steps, cell, plan, peaks, fp32_peak, fp64_peak):
    """The roofline of the contraction kernel with the most device time (rows a2, a7)."""
    cands = {k: v for k, v in kt.items() if k in CONTRACTION_KERNELS}
    if not cands:
        return None
    k = max(cands, key=lambda x: cands[x][0])
    row, mixed = CONTRACTION_KERNELS[k]
    ent, kd, inf = plan.entries, pb_dims(plan), plan.info
    if mixed:
        work = row_work(cell, ent, kd, row, inf["c_symmetric"])
    else:  # the FP64 kernel does the small stages; its dense stage runs as digit GEMMs
        w = kernel_work(k, cell, inf, ent, kd)
        fl = w[1]
        byt = row_work(cell, ent, kd, row, inf["c_symmetric"])[1]
        work = (fl, byt, 0.0, fl)
    ms, nl = cands[k]
    roof = contraction_roofline(k, ms / steps, nl / steps, work, peaks, fp32_peak, fp64_peak, mixed)
    roof["row"] = {"P": "a2 (Eq. P_MM)", "S": "a7 (Eq. S_MM)"}[row]
    if mixed:
        # (entry, node) units of one step: Sigma every node and the exchange's one slice,
        # P the computed nodes
        E, nt = len(ent), cell.n_tau
        per_step = E * (nt + 1) if row == "S" else E * ((nt + 1) // 2 if inf["c_symmetric"] else nt)
        roof["traffic"] = traffic_of(k, per_step / (nl / steps))
    return roof


def run_rows(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    cell = workload(2, False, args.r_b, args.n_prod_far, atoms=args.atoms)
    sw = RowSweep(cell, device=local)
    Gk = cell.green_k_tau()
    sw.load_G(Gk)
    stream = torch.cuda.Stream(device=local)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=sw.dev)  # 256 MB > L2
    try:
        from paper_1911_05633_gb300 import gw
        fp64_peak, fp32_peak = gw.fp_peak(local)
    except Exception:
        fp64_peak, fp32_peak = None, None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    other = "fp64" if args.precision == "mixed" else "mixed"
    res = {}
    for prec in (other, args.precision):  # the headline precision last, under the clock sampler
        sw.prec = prec
        barrier(world)
        clocks = Clocks(local) if prec == args.precision else None
        ms, stage_ms, kt, clk = time_rows(sw, stream, flush, args.steps, args.warmup, clocks)
        res[prec] = {"ms": ms, "stage_ms": stage_ms, "kt": kt, "clk": clk}
    main_ = res[args.precision]
    step_ms_max, value = aggregate(main_["ms"], world)
    ent, inf, kd = sw.plan.entries, sw.plan.info, pb_dims(sw.plan)
    wP = row_work(cell, ent, kd, "P", inf["c_symmetric"])
    wS = row_work(cell, ent, kd, "S", inf["c_symmetric"])

    def block(r, prec):
        st = dict(zip(RowSweep.STAGES, r["stage_ms"]))
        return {"value": round(world * 1000.0 / r["ms"], 6), "unit": UNIT, "ms_per_sweep": round(r["ms"], 4),
                "stage_ms": {n: round(float(t), 4) for n, t in st.items()},
                "contraction_tflops": {"P": round(wP[0] / (st["P"] * 1e-3) / 1e12, 4),
                                       "Sigma": round(wS[0] / (st["Sigma"] * 1e-3) / 1e12, 4)},
                "kernels": kernels_table(r["kt"], args.steps),
                "roofline": dominant_contraction_roofline(r["kt"], args.steps, cell, sw.plan, peaks, fp32_peak,
                                                          fp64_peak)}

    b_main, b_other = block(main_, args.precision), block(res[other], other)
    errs = rows_mixed_vs_fp64(sw, stream, cell)
    e2e = None if args.no_e2e else run_e2e_rows(sw, Gk, stream, flush, args)
    out = {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16x3-f32acc contractions + f64 transforms" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": rows_config(cell, len(ent), inf["n_pb_total"], args.precision, world),
        "stage_ms": b_main["stage_ms"],
        "contraction_tflops": b_main["contraction_tflops"],
        "clocks": main_["clk"],
        # the library's kernel launches in the timed region, counted by its event timer
        "gpu_launches": int(sum(v[1] for v in main_["kt"].values())),
        "roofline": b_main["roofline"],
        "kernels": b_main["kernels"],
        other: {**b_other, "speedup_of_" + args.precision: round(res[other]["ms"] / main_["ms"], 3)},
        "mixed_vs_fp64": errs,
        "fp64_peak_tflops_measured": fp64_peak, "fp32_peak_tflops_measured": fp32_peak,
        "e2e": e2e,
    }
    del sw
    torch.cuda.empty_cache()
    return out, cell


def rows_mixed_vs_fp64(sw, stream, cell):
    """Relative Frobenius errors of the mixed rows against the FP64 rows of the same plan
    and inputs (the FP64 rows equal the oracle to 1e-10 on sampled entries of this workload:
    tests/test_gpu_parity.py::test_full_size_72_atoms_sampled): P(R, tau) and Sigma(R, tau),
    Sigma(k, i w) on the same W~."""
    torch = sw.torch
    outs = {}
    for prec in ("mixed", "fp64"):
        sw.prec = prec
        with torch.cuda.stream(stream):
            sw.run(stream)
        sw.plan.sync(stream=stream.cuda_stream)
        torch.cuda.synchronize()
        outs[prec] = {"P": sw.P_R.clone(), "Sigma": sw.S_R.clone(), "Sigma_k": sw.S_k.clone()}
    sw.prec = "mixed"
    rel = {k: float(f"{float(torch.linalg.vector_norm(outs['mixed'][k] - outs['fp64'][k]) / torch.linalg.vector_norm(outs['fp64'][k])):.3e}")
           for k in ("P", "Sigma", "Sigma_k")}
    del outs
    torch.cuda.empty_cache()
    return {**rel, "tolerance": 1e-6, "reference": "the FP64 GPU rows, same plan and inputs"}


def run_e2e_rows(sw, Gk, stream, flush, args):
    """The same rows through the C ABI with host buffers: per step, H2D of G(k,tau),
    W~(R,i nu) and v(R) from pinned memory and D2H of Sigma(k,i w) and Sigma_x(k), inside
    the timed region; the same steps and L2 flush as `value`.  The copies run on one stream
    per direction beside the rows, into and out of two sets of device buffers, so that the
    inputs of step k+1 and the results of step k-1 move while step k computes (events
    order each copy after the step that last used its buffers)."""
    torch = sw.torch
    Gk_h = torch.from_numpy(Gk.reshape(-1)).pin_memory()
    W_h = sw.W_iw.cpu().pin_memory()
    v_h = sw.v_R.cpu().pin_memory()
    Sk_h = torch.empty(sw.S_k.numel(), dtype=torch.complex128).pin_memory()
    Sxk_h = torch.empty(sw.Sx_k.numel(), dtype=torch.complex128).pin_memory()
    sw.prec = args.precision
    names = ("G_k", "W_iw", "v_R", "S_k", "Sx_k")
    sets = [{n: getattr(sw, n) for n in names}, {n: torch.empty_like(getattr(sw, n)) for n in names}]
    c_in, c_out = torch.cuda.Stream(device=sw.dev), torch.cuda.Stream(device=sw.dev)

    def steps(n, t0=None, t1=None):
        done_in = [torch.cuda.Event() for _ in range(n)]
        done_rows = [torch.cuda.Event() for _ in range(n)]
        done_out = [torch.cuda.Event() for _ in range(n)]
        if t0 is not None:
            t0.record(c_in)
        for k in range(n):
            b = sets[k % 2]
            if k >= 2:
                c_in.wait_event(done_rows[k - 2])  # the rows of step k-2 have read this set
            with torch.cuda.stream(c_in):
                b["G_k"].copy_(Gk_h, non_blocking=True)
                b["W_iw"].copy_(W_h, non_blocking=True)
                b["v_R"].copy_(v_h, non_blocking=True)
            done_in[k].record(c_in)
            stream.wait_event(done_in[k])
            if k >= 2:
                stream.wait_event(done_out[k - 2])  # the results of step k-2 have been read
            for nm in names:
                setattr(sw, nm, b[nm])
            with torch.cuda.stream(stream):
                flush_l2(flush)
                sw.run(stream)
            done_rows[k].record(stream)
            c_out.wait_event(done_rows[k])
            with torch.cuda.stream(c_out):
                Sk_h.copy_(b["S_k"], non_blocking=True)
                Sxk_h.copy_(b["Sx_k"], non_blocking=True)
            done_out[k].record(c_out)
        if t1 is not None:
            c_out.wait_stream(stream)
            t1.record(c_out)

    steps(2)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps(args.steps, t0, t1)
    torch.cuda.synchronize()
    for nm in names:
        setattr(sw, nm, sets[0][nm])
    ms = t0.elapsed_time(t1) / args.steps
    return {"value": round(1000.0 / ms, 6), "unit": UNIT, "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int((Gk_h.numel() + W_h.numel() + v_h.numel()) * 16),
            "d2h_bytes_per_step": int((Sk_h.numel() + Sxk_h.numel()) * 16), "steps": args.steps,
            "l2": "256 MB buffer written before each step's rows",
            "copies": "one stream per direction beside the rows, two buffer sets: step k+1's inputs and "
                      "step k-1's results move while step k computes"}


# --------------------------------------------------------------------------------------
# the 8-atom workload's whole sweep (configuration 1, W solve included)
# --------------------------------------------------------------------------------------

class Sweep:
    """Device buffers and the ordered calls of one whole sweep, the W solve included."""

    STAGES = ["G_k_to_R", "P", "P_tau_to_nu", "W_solve", "W_nu_to_tau", "v_k_to_R", "Sigma", "Sigma_tau_to_omega",
              "Sigma_R_to_k"]

    def __init__(self, cell, precision: str, device: int = 0, w_solver: str = "auto", fp64_products: str = "auto"):
        import torch
        from paper_1911_05633_gb300 import gw
        self.torch = torch
        self.cell = cell
        self.prec = precision
        self.plan = gw.Plan.from_cell(cell, device=device, w_solver=w_solver, fp64_products=fp64_products)
        p = self.plan
        inf = p.info
        self.dev = torch.device("cuda", device)
        z = lambda n: torch.empty(n, dtype=torch.complex128, device=self.dev)
        nt, nn, nw = inf["n_tau"], inf["n_nu"], inf["n_omega"]
        No = inf["n_orb_total"]
        self.G_k = z(inf["n_k"] * nt * No * No)
        self.v_q = z(inf["n_k"] * inf["n_pb_total"] ** 2)
        self.G_R = z(p.len("orb", nt))
        self.P_R = z(p.len("pb", nt))
        self.P_iw = z(p.len("pb", nn))
        self.W_iw = z(p.len("pb", nn))
        self.W_R = z(p.len("pb", nt))
        self.v_R = z(p.len("pb", 1))
        self.S_R = z(p.len("orb", nt))
        self.Sx_R = z(p.len("orb", 1))
        self.S_iw = z(p.len("orb", nw))
        self.S_k = z(inf["n_k"] * nw * No * No)
        self.Sx_k = z(inf["n_k"] * No * No)

    def load_inputs(self, G_k_host, v_q_host):
        self.G_k.copy_(self.torch.from_numpy(G_k_host.reshape(-1)))
        self.v_q.copy_(self.torch.from_numpy(v_q_host.reshape(-1)))

    def run(self, stream, events=None):
        p, s = self.plan, stream.cuda_stream
        inf = p.info
        calls = [
            lambda: p.green_k_to_R(self.G_k, self.G_R, stream=s),
            lambda: p.polarizability_tau(self.G_R, self.P_R, precision=self.prec, stream=s),
            lambda: p.transform_tau_iw("B", "tau_to_iw", "pb", self.P_R, self.P_iw, stream=s,
                                       structure=p_iw_structure(inf)),
            lambda: p.screened_W_iw(self.P_iw, self.v_q, self.W_iw, stream=s),
            lambda: p.transform_tau_iw("B", "iw_to_tau", "pb", self.W_iw, self.W_R, stream=s,
                                       structure="real" if inf["w_symmetric"] else "general"),
            lambda: p.fourier_k_to_R("pb", 1, self.v_q, self.v_R, stream=s),
            lambda: p.self_energy_tau(self.G_R, self.W_R, v_R=self.v_R, Sig_R=self.S_R, Sigx_R=self.Sx_R,
                                      precision=self.prec, stream=s),
            lambda: p.transform_tau_iw("F", "tau_to_iw", "orb", self.S_R, self.S_iw, stream=s),
            lambda: (p.fourier_R_to_k("orb", inf["n_omega"], self.S_iw, self.S_k, stream=s),
                     p.fourier_R_to_k("orb", 1, self.Sx_R, self.Sx_k, stream=s)),
        ]
        for i, c in enumerate(calls):
            if events is not None:
                events[i][0].record(stream)
            c()
            if events is not None:
                events[i][1].record(stream)


def traffic_of(kernel: str, units_per_launch: float):
    """DRAM bytes per launch of `kernel` from a committed ncu capture (bytes per unit
    there x units in this launch), or None when there is none or when the kernel's
    source has changed since the capture."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    src = os.path.join(ROOT, "paper_1911_05633_gb300", "csrc", t["file"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return round(t["bytes_per_unit"] * units_per_launch) if sha == t["src_sha"] else None


def flush_l2(buf):
    buf.add_(1.0)


def dominant_kernel_roofline(kt, steps, cell, plan, peaks, fp32_peak, fp64_peak):
    """The roofline of the kernel with the most device time in a whole sweep."""
    if not kt:
        return None
    dom_k = max(kt, key=lambda k: kt[k][0])
    ms_tot, nl = kt[dom_k]
    w = kernel_work(dom_k, cell, plan.info, plan.entries, pb_dims(plan))
    if w is None:
        return {"kernel": dom_k, "bound": None}
    bound, work, kind, units = w
    per_launch = work * steps / nl
    dur = ms_tot * 1e-3 / nl
    if bound == "hbm":
        ach, unit, peak = per_launch / dur / 1e9, "GB/s", peaks.get("hbm_gbs")
    elif bound == "tensor":
        ach, unit, peak = per_launch / dur / 1e12, "TFLOP/s", peaks.get("bf16_tflops_sustained")
    else:
        ach, unit = per_launch / dur / 1e12, "TFLOP/s"
        peak = fp64_peak if kind == "fp64" else fp32_peak
    return {"kernel": dom_k, "bound": bound, "achieved": round(ach, 4), "peak": round(peak, 4) if peak else None,
            "unit": unit, "frac": round(ach / peak, 4) if peak else None,
            "traffic": traffic_of(dom_k, units * steps / nl), "launch_ms": round(dur * 1e3, 4)}


def run_full(args, local, with_errors: bool = True):
    """The 8-atom workload's whole sweep (W solve included) in FP64 and in mixed precision,
    and the mixed-vs-FP64 errors of P, Sigma and the quasiparticle energies."""
    import torch
    torch.cuda.set_device(local)
    cell = workload(1, args.small, args.r_b if args.config == 1 else 0.0, args.n_prod_far)
    sw = Sweep(cell, "fp64", device=local, w_solver=args.w_solver, fp64_products=args.fp64_products)
    Gk = cell.green_k_tau()
    vq, _ = cell.coulomb()
    sw.load_inputs(Gk, vq)
    stream = torch.cuda.Stream(device=local)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=sw.dev)
    try:
        from paper_1911_05633_gb300 import gw
        fp64_peak, fp32_peak = gw.fp_peak(local)
    except Exception:
        fp64_peak, fp32_peak = None, None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    out = {"workload": f"{cell.name}: {cell.n_atoms} atoms, {cell.kmesh[0]}x{cell.kmesh[1]}x{cell.kmesh[2]} k, "
                       f"{cell.n_tau} tau, cutoff {cell.cutoff} bohr, {len(sw.plan.entries)} pair entries, N_PB "
                       f"{cell.n_pb_total}"}
    for prec in ("fp64", "mixed"):
        sw.prec = prec
        ms, stage_ms, kt, _ = time_rows(sw, stream, flush, args.steps, args.warmup)
        st = dict(zip(Sweep.STAGES, stage_ms))
        ps = ms - st["W_solve"]
        out[prec] = {"value": round(1000.0 / ms, 6), "unit": UNIT, "ms_per_sweep": round(ms, 4),
                     "p_sigma_rows_ms": round(ps, 4), "w_solve_ms": round(st["W_solve"], 4),
                     "stage_ms": {n: round(float(t), 4) for n, t in st.items()},
                     "roofline_dominant_kernel": dominant_kernel_roofline(kt, args.steps, cell, sw.plan, peaks,
                                                                         fp32_peak, fp64_peak),
                     "kernels": kernels_table(kt, args.steps)}
    sw.prec = "mixed"
    if with_errors:
        out["mixed_vs_fp64"] = mixed_vs_fp64(sw, stream, cell)
    if not args.no_dyson:
        out["dyson"] = run_dyson(sw, cell, stream, args)
    sw.plan.close()
    del sw
    torch.cuda.empty_cache()
    return out, cell


def run_dyson(sw, cell, stream, args):
    """Eq. G_1 after the sweep (the next step of an iteration, not part of `value`): the
    device Dyson solve G(k, tau) from the sweep's Sigma(k, i w) and Sigma_x(k), timed with
    CUDA events over `steps` calls, and the chemical potential at half filling by bisection
    (wall clock; one Dyson solve per step)."""
    torch = sw.torch
    p = sw.plan
    H = torch.from_numpy(cell.H_k.reshape(-1)).to(sw.dev)
    G = torch.empty(p.info["n_k"] * p.info["n_tau"] * p.dense_n("orb") ** 2, dtype=torch.complex128, device=sw.dev)
    ss = stream.cuda_stream
    with torch.cuda.stream(stream):
        p.dyson_green_tau(H, cell.mu, Sigx_k=sw.Sx_k, Sig_k_iw=sw.S_k, G_k_tau=G, stream=ss)  # allocates its scratch
    p.sync(stream=ss)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev:
        with torch.cuda.stream(stream):
            a.record(stream)
            p.dyson_green_tau(H, cell.mu, Sigx_k=sw.Sx_k, Sig_k_iw=sw.S_k, G_k_tau=G, stream=ss)
            b.record(stream)
    p.sync(stream=ss)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    sx = sw.Sx_k.cpu().numpy().reshape(cell.H_k.shape)
    e = np.linalg.eigvalsh(cell.H_k + 0.5 * (sx + np.conj(np.transpose(sx, (0, 2, 1)))))  # the static levels
    lo, hi, tol = float(e.min()) - 2.0, float(e.max()) + 2.0, 1e-10
    t0 = time.perf_counter()
    mu, n = p.chemical_potential(H, float(cell.n_orb_total), lo, hi, tol=tol, Sigx_k=sw.Sx_k, Sig_k_iw=sw.S_k,
                                 stream=ss)
    t_mu = time.perf_counter() - t0
    N, nk, nw = p.dense_n("orb"), p.info["n_k"], p.info["n_omega"]
    return {"green_tau_ms": round(ms, 3), "inverses": nk * nw, "n_orb": N,
            "inverse_tflops": round(8.0 * N ** 3 * nk * nw / (ms * 1e-3) / 1e12, 3),
            "mu_search_s": round(t_mu, 3), "mu_steps": int(np.ceil(np.log2((hi - lo) / tol))) + 1,
            "mu": mu, "n_electrons": n, "note": "Eq. G_1 with the sweep's Sigma; not part of value"}


def mixed_vs_fp64(sw, stream, cell):
    """Relative Frobenius errors of the mixed path against the FP64 GPU path of the same
    plan on the same inputs (after the timed region): the P contraction (same G(R)), the
    Sigma contraction (same G(R) and W~(R)), and the whole sweep's Sigma(R, tau) and
    Sigma(k, i omega), whose W~ comes from the mixed P through the W solve, and the
    linearised quasiparticle energies from each sweep's Sigma (max |difference| in meV)."""
    torch = sw.torch
    H = torch.from_numpy(cell.H_k.reshape(-1)).to(sw.dev)
    qp = {}
    outs = {}
    for prec in ("mixed", "fp64"):
        sw.prec = prec
        with torch.cuda.stream(stream):
            sw.run(stream)
        sw.plan.sync(stream=stream.cuda_stream)
        torch.cuda.synchronize()
        outs[prec] = {"P": sw.P_R.clone(), "Sigma_chain": sw.S_R.clone(), "Sigma_k_chain": sw.S_k.clone()}
    # the Sigma contraction alone, in mixed precision on the FP64 sweep's G(R) and W~(R)
    S_mix, Sx = torch.empty_like(sw.S_R), torch.empty_like(sw.Sx_R)
    with torch.cuda.stream(stream):
        sw.plan.self_energy_tau(sw.G_R, sw.W_R, v_R=sw.v_R, Sig_R=S_mix, Sigx_R=Sx, precision="mixed",
                                stream=stream.cuda_stream)
    sw.plan.sync(stream=stream.cuda_stream)
    torch.cuda.synchronize()
    outs["mixed"]["Sigma_contraction"] = S_mix
    outs["fp64"]["Sigma_contraction"] = outs["fp64"]["Sigma_chain"]
    sw.prec = "mixed"
    keys = ("P", "Sigma_contraction", "Sigma_chain", "Sigma_k_chain")
    rel = {k: float(torch.linalg.vector_norm(outs["mixed"][k] - outs["fp64"][k]) /
                    torch.linalg.vector_norm(outs["fp64"][k])) for k in keys}
    del outs
    qp = qp_compare(sw, stream, cell)
    # the same on the two-atom configuration (beta = 50), where the linearisation is well conditioned
    import synth
    c0 = synth.make_config(0)
    sw0 = Sweep(c0, "mixed", device=sw.dev.index)
    sw0.load_inputs(c0.green_k_tau(), c0.coulomb()[0])
    qp0 = qp_compare(sw0, stream, c0)
    sw0.plan.close()
    return {**{k: float(f"{v:.3e}") for k, v in rel.items()}, "tolerance_contractions": 1e-6,
            "qp_energies": qp, "qp_energies_two_atom_cell": qp0, "tolerance_qp_meV": 1.0,
            "reference": "the FP64 GPU path, same plan and inputs",
            "note": "the chain values carry the W solve's amplification of P's error"}


def qp_compare(sw, stream, cell):
    """Linearised quasiparticle energies (gw_qp_energies) from the mixed and from the FP64
    sweep of the same inputs: their largest difference in meV, next to the problem's own
    sensitivity (the largest shift of the FP64 energies when Sigma(k, i w) is scaled
    elementwise by 1 + 1e-6 x seeded normal numbers) and the smallest eigenvalue of
    I - S1^h (the frequency slope of Sigma at zero, whose inverse square root scales the
    energies)."""
    torch = sw.torch
    H = torch.from_numpy(cell.H_k.reshape(-1)).to(sw.dev)
    ss = stream.cuda_stream
    E, Sk = {}, None
    for prec in ("mixed", "fp64"):
        sw.prec = prec
        with torch.cuda.stream(stream):
            sw.run(stream)
            E[prec] = sw.plan.qp_energies(H, cell.mu, Sigx_k=sw.Sx_k, Sig_k_iw=sw.S_k, stream=ss)
        sw.plan.sync(stream=ss)
        torch.cuda.synchronize()
        E[prec] = E[prec].cpu().numpy()
    sw.prec = "mixed"
    gen = torch.Generator(device=sw.dev).manual_seed(7)
    noise = torch.randn(sw.S_k.shape, dtype=torch.float64, device=sw.dev, generator=gen)
    Sp = sw.S_k * (1.0 + 1e-6 * noise)
    with torch.cuda.stream(stream):
        Ep = sw.plan.qp_energies(H, cell.mu, Sigx_k=sw.Sx_k, Sig_k_iw=Sp, stream=ss)
    sw.plan.sync(stream=ss)
    torch.cuda.synchronize()
    Ep = Ep.cpu().numpy()
    # slope of Sigma at zero frequency from the two lowest sampled frequencies (host)
    inf = sw.plan.info
    N, nk, nw = sw.plan.dense_n("orb"), inf["n_k"], inf["n_omega"]
    idx = [int(n) for n in cell.omega_idx]
    Sk = sw.S_k.view(nk, nw, N, N)
    d = (Sk[:, idx.index(1)] - Sk[:, idx.index(0)]).cpu().numpy() / (1j * 2.0 * np.pi / cell.beta)
    dh = 0.5 * (d + np.conj(np.transpose(d, (0, 2, 1))))
    lam = float(np.linalg.eigvalsh(np.eye(N)[None] - dh).min())
    mev = 27211.386245988
    return {"max_abs_meV": float(f"{np.abs(E['mixed'] - E['fp64']).max() * mev:.3e}"),
            "sensitivity_meV_per_1e-6_sigma": float(f"{np.abs(Ep - E['fp64']).max() * mev:.3e}"),
            "min_eig_I_minus_S1h": float(f"{lam:.3e}"),
            "energy_range_Ha": [float(f"{E['fp64'].min():.4f}"), float(f"{E['fp64'].max():.4f}")],
            "workload": cell.name, "beta": cell.beta}


# --------------------------------------------------------------------------------------
# the oracle on the host cores (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------

class OracleRows:
    """The FP64 oracle's P + Sigma rows on a fixed sample of the workload's pair entries
    (every E/n-th entry, all tau nodes), with the same seeded stand-in for W~(R, i nu);
    one timed pass is scaled by E/n to a whole sweep (every row's cost is a sum over
    entries).  Setup (the cell, G(k, tau), the transform matrices) is not timed."""

    def __init__(self, cell, n_sample: int = 24):
        import oracle
        self.oracle = oracle
        self.cell = cell
        self.orc = oracle.OracleSystem(cell)
        E = len(self.orc.entries)
        self.sel = np.unique(np.linspace(0, E - 1, min(n_sample, E)).astype(int))
        self.scale = E / len(self.sel)
        self.ent = self.orc.entries[self.sel]
        self.kdims = [self.orc.kdims[e] for e in self.sel]
        self.Gk = cell.green_k_tau()
        rng = np.random.default_rng(0)
        nn = cell.nu_idx.size
        self.Wiw = [rng.standard_normal((nn, Ka, Kb)) + 0j for Ka, Kb in self.kdims]
        self.vR = [rng.standard_normal((Ka, Kb)) + 0j for Ka, Kb in self.kdims]
        self.note = (f"P+Sigma rows (a1, a2, a3, a6, a7, a8) on {len(self.sel)} of {E} pair entries (every "
                     f"{E // len(self.sel)}th, all {cell.n_tau} tau nodes), scaled x{self.scale:.1f}; W~(R, i nu) "
                     f"seeded as on the GPU; setup not counted")

    def time_one(self) -> float:
        o, c, orc = self.oracle, self.cell, self.orc
        oo = c.orb_offsets
        # the R -> k sum of the sample into the blocks of the atoms it touches (the dense
        # output of the whole cell is allocated once per sweep, timed apart and not scaled)
        used = sorted(set(int(x) for x in self.ent[:, 0]) | set(int(x) for x in self.ent[:, 1]))
        ren = {a: i for i, a in enumerate(used)}
        ent_c = self.ent.copy()
        ent_c[:, 0] = [ren[int(a)] for a in self.ent[:, 0]]
        ent_c[:, 1] = [ren[int(b)] for b in self.ent[:, 1]]
        oo_c = np.concatenate([[0], np.cumsum([c.n_orb_of(a) for a in used])])
        t0 = time.perf_counter()
        GR = o.fourier_k_to_R(self.Gk, self.ent, orc.kmesh, oo, oo)
        PR = o.polarizability_R(GR, self.ent, orc.C_atom, c.spin, self.kdims)
        o.transform(orc.B_fwd, PR)
        WR = o.transform(orc.B_inv, self.Wiw)
        SR = o.self_energy_R(GR, WR, self.ent, orc.C_atom)
        o.exchange_R(GR, self.vR, self.ent, orc.C_atom)
        Siw = o.transform(orc.F_fwd, SR)
        o.fourier_R_to_k(Siw, ent_c, orc.kmesh, oo_c, oo_c)
        t_sample = time.perf_counter() - t0
        t0 = time.perf_counter()
        out = np.zeros((c.n_k, c.omega_idx.size, c.n_orb_total, c.n_orb_total), np.complex128)
        out[0, 0, 0, 0] = 1.0
        t_alloc = time.perf_counter() - t0
        del out
        return t_sample * self.scale + t_alloc


def cpu_cores():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
        return int(n)
    except Exception:
        return os.cpu_count()


def rows_config(cell, n_entries, n_pb, precision, world):
    """The `config` of the P + Sigma rows line (the same dict in both arms)."""
    return {"workload": f"{cell.name}: {cell.n_atoms} atoms, {cell.kmesh[0]}x{cell.kmesh[1]}x{cell.kmesh[2]} k,"
                        f" {cell.n_tau} tau, cutoff {cell.cutoff} bohr, {n_entries} pair entries, N_PB {n_pb}",
            "rows": "a1 G k->R, a2 P, a3 P tau->i nu, a6 W~ i nu->tau, a7 Sigma + Sigma_x, a8 Sigma tau->i w "
                    "and R->k; the W solve (Eq. W_1, with the dense q-space halves of a4/a6) timed apart",
            "inputs": "G(k,tau) of the seeded tight-binding cell; W~(R,i nu) and v(R) seeded (the W solve's "
                      "output and the bare interaction, in the plan's shapes)",
            "precision": precision, "l2": "256 MB buffer written between timed steps (inputs > L2)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cell = workload(2, False, args.r_b, args.n_prod_far, atoms=args.atoms)
    orc = OracleRows(cell)
    for _ in range(args.warmup):
        orc.time_one()
    secs = [orc.time_one() for _ in range(max(1, args.steps))]
    ms = 1000.0 * float(np.mean(secs))
    v = 1000.0 / ms
    cfg = rows_config(cell, len(orc.orc.entries), cell.n_pb_total, args.precision, world)
    return {"impl": "reference", "metric": METRIC, "value": round(v, 8), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": round(v, 8), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": orc.note},
            "e2e": {"value": round(v, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# --------------------------------------------------------------------------------------
# batched uneven systems (configuration 3): one persistent launch per contraction
# --------------------------------------------------------------------------------------

def release_device():
    """Drop unreferenced plans and return torch's cached blocks to the device, so that the
    next block's plans can allocate."""
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def run_batch3(args, local, peaks):
    """The mixed P and Sigma contractions of the 16-system batch family (15 diamond-like
    supercells of 8 to 56 atoms with different meshes and cutoffs, and the 56-atom layered
    perovskite-like cell) as one persistent launch per shape class each (gw_batch_*),
    autotuned, captured in a CUDA graph and replayed; beside it the same contractions
    launched system by system.
    Inputs: G(R, tau) from each cell's G(k, tau), W~(R, tau) seeded.  Checks that every
    system's result is the same bits in the batch and alone."""
    import torch
    import synth
    from paper_1911_05633_gb300 import gw
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_setup = time.perf_counter()
    cells = synth.batch_family()
    plans, G, W, P, S = [], [], [], [], []
    gen = torch.Generator(device=dev).manual_seed(3)
    for c in cells:
        p = gw.Plan.from_cell(c, device=local, defer_scratch=True)
        nt = p.info["n_tau"]
        Gk = torch.from_numpy(c.green_k_tau().reshape(-1)).to(dev)
        G.append(p.green_k_to_R(Gk))
        del Gk
        W.append(torch.randn(p.len("pb", nt), dtype=torch.complex128, device=dev, generator=gen))
        P.append(torch.empty(p.len("pb", nt), dtype=torch.complex128, device=dev))
        S.append(torch.empty(p.len("orb", nt), dtype=torch.complex128, device=dev))
        plans.append(p)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    b = gw.Batch(plans)
    stream = torch.cuda.Stream(device=local)
    ss = stream.cuda_stream
    t0 = time.perf_counter()
    info = b.tune(G, P, W, S, reps=2, stream=ss)
    t_tune = time.perf_counter() - t0
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def batched():
        b.polarizability_tau(G, P, stream=ss)
        b.self_energy_tau(G, W, S, stream=ss)

    def alone(outP, outS):
        for p, g, w, op, os_ in zip(plans, G, W, outP, outS):
            p.polarizability_tau(g, op, precision="mixed", stream=ss)
            p.self_energy_tau(g, w, Sig_R=os_, precision="mixed", stream=ss)

    with torch.cuda.stream(stream):
        batched()
    b.sync(stream=ss)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batched()

    def time_it(fn):
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for a, e in ev:
                flush_l2(flush)
                a.record(stream)
                fn()
                e.record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(e) for a, e in ev]))

    ms_batch = time_it(graph.replay)
    P2 = [torch.empty_like(x) for x in P]
    S2 = [torch.empty_like(x) for x in S]
    ms_alone = time_it(lambda: alone(P2, S2))
    b.sync(stream=ss)
    same = all(torch.equal(x, y) for x, y in zip(P + S, P2 + S2))
    # algorithmic work and bytes of both contractions over every system
    fl = byt = 0.0
    for c, p in zip(cells, plans):
        kd = pb_dims(p)
        for row in ("P", "S"):
            w = row_work(c, p.entries, kd, row, p.info["c_symmetric"])
            fl += w[0]
            byt += w[1]
    hbm = peaks.get("hbm_gbs")
    out = {"workload": f"{len(cells)} systems of {min(c.n_atoms for c in cells)} to {max(c.n_atoms for c in cells)} atoms "
                       f"({sum(c.n_atoms for c in cells)} atoms, {sum(len(p.entries) for p in plans)} pair entries, "
                       f"48 tau): diamond-like supercells (n 9, K 48) and the layered perovskite-like cell "
                       f"(n 14/9/9, K 96/64/40)",
           "precision": "mixed", "ms_batched_graph": round(ms_batch, 4), "ms_system_by_system": round(ms_alone, 4),
           "speedup_batched": round(ms_alone / ms_batch, 3),
           "contraction_tflops": round(fl / (ms_batch * 1e-3) / 1e12, 4),
           "roofline": {"bound": "hbm", "achieved": round(byt / (ms_batch * 1e-3) / 1e9, 2), "peak": hbm,
                        "unit": "GB/s", "frac": round(byt / (ms_batch * 1e-3) / 1e9 / hbm, 4) if hbm else None,
                        "algorithmic_bytes": byt, "note": "P and Sigma launches together, algorithmic bytes of both"},
           "tuned": {k: info[k] for k in ("groups_p", "groups_s", "kc_p", "kc_s", "order_p", "order_s")},
           "launch_classes": info["n_classes"],
           "tune_s": round(t_tune, 2), "setup_s": round(t_setup, 1), "batched_equals_alone_bitwise": bool(same),
           "units": {"P": info["n_units_p"], "Sigma": info["n_units_s"]}, "steps": args.steps,
           "l2": "256 MB buffer written before each timed step"}
    b.close()
    del graph, G, W, P, S, P2, S2
    for p in plans:
        p.close()
    torch.cuda.empty_cache()
    return out


def run_w_solve(args, local, cell=None):
    """The W solve of Eq. W_1 on the configuration-2 cell (N_PB = 64 x atoms): P(R, i nu)
    from the cell's own FP64 rows a1-a3, v(q) from the cell, W~(R, i nu) by the plan's
    inverse (block Gauss-Jordan over tensor-core pivot inverses beyond N_PB = 384).  One
    solve to warm up (it also fixes the frequency chunks), one timed with CUDA events on
    its stream; the kernels' shares from the plan's own launch timing."""
    import torch
    import synth
    from paper_1911_05633_gb300 import gw
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    if cell is None:
        cell = synth.make_config(2, atoms=args.atoms)
    vq, _ = cell.coulomb()
    t_host = time.perf_counter() - t0
    plan = gw.Plan.from_cell(cell, device=local, w_solver=args.w_solver,
                             workspace_bytes=int(args.workspace_gb * 1e9))
    inf = plan.info
    nt, nn = inf["n_tau"], inf["n_nu"]
    stream = torch.cuda.Stream(device=local)
    sp = stream.cuda_stream
    G_k = torch.from_numpy(cell.green_k_tau().reshape(-1)).to(dev)
    v_q = torch.from_numpy(vq.reshape(-1)).to(dev)
    del vq
    G_R = plan.green_k_to_R(G_k, stream=sp)
    P_R = plan.polarizability_tau(G_R, precision="fp64", stream=sp)
    P_iw = plan.transform_tau_iw("B", "tau_to_iw", "pb", P_R, stream=sp, structure=p_iw_structure(inf))
    stream.synchronize()  # before the inputs go back to the allocator
    del P_R, G_R, G_k
    W = torch.empty(plan.len("pb", nn), dtype=torch.complex128, device=dev)
    plan.screened_W_iw(P_iw, v_q, W, stream=sp)
    plan.sync(stream=sp)
    plan.timing_reset()
    plan.timing_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.screened_W_iw(P_iw, v_q, W, stream=sp)
    e1.record(stream)
    plan.sync(stream=sp)
    torch.cuda.synchronize()
    kt = plan.timing_read()
    plan.timing_enable(False)
    sec = e0.elapsed_time(e1) / 1e3
    N = inf["n_pb_total"]
    n_nu_solved = int((np.asarray(cell.nu_idx) >= 0).sum()) if inf["w_symmetric"] else nn
    problems = inf["n_q_solved"] * n_nu_solved
    inverses = problems + inf["n_q_solved"]          # and v(q)^-1 once per solved momentum
    flops = inverses * 8.0 * N ** 3                   # a complex inverse: N^3 complex multiply-adds
    finite = bool(torch.isfinite(torch.view_as_real(W)).all().item())
    out = {"metric": "W solve of Eq. W_1 (W~(R, i nu) from P(R, i nu))", "unit": "s", "value": round(sec, 3),
           "config": {"workload": f"configuration 2, {args.atoms}-atom diamond supercell", "n_pb": N,
                      "n_q_solved": inf["n_q_solved"], "nu_solved": n_nu_solved, "problems": problems,
                      "inverse": ("block Gauss-Jordan, pivot blocks of %d" % inf["w_block"]) if inf["w_block"]
                      else ("tensor-core" if inf["w_tensor"] else "FP64 Gauss-Jordan"),
                      "nu_chunk": inf["nu_chunk"], "workspace_GB": round(inf["workspace_bytes"] / 1e9, 1)},
           "ms_per_inverse": round(1e3 * sec / inverses, 2),
           "fp64_equivalent_tflops": round(flops / sec / 1e12, 2),
           "finite": finite, "host_setup_s": round(t_host, 1),
           "kernels": dict(list(kernels_table(kt, 1).items())[:8])}
    return out


def run_scaling(args, local):
    """P + Sigma rows (a1-a4 and a6-a8; the W solve is timed apart by the metric) of the
    diamond supercell series with 9 orbitals and 64 product functions per atom, a 2x2x2
    mesh, 64 tau nodes and a 12-bohr cutoff (8, 16, 32, 48, 72 atoms), in FP64 and in
    mixed precision.  W~(R, i nu) and v(R) are seeded random inputs of the plan's shapes:
    the W solve of N_PB = 64 x atoms is not part of this step.  Per size: ms per sweep
    over the rows, per pair entry, and the contraction TFLOP/s."""
    import torch
    import synth
    from paper_1911_05633_gb300 import gw
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = args.scaling or [8, 16, 32, 48, 72]
    stream = torch.cuda.Stream(device=local)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rows = []
    for nat in sizes:
        cell = synth.make_config(2, atoms=nat)
        plan = gw.Plan.from_cell(cell, device=local, defer_scratch=True)
        inf = plan.info
        nt, nn, nw, No, nk = inf["n_tau"], inf["n_nu"], inf["n_omega"], inf["n_orb_total"], inf["n_k"]
        z = lambda n: torch.empty(n, dtype=torch.complex128, device=dev)
        G_k = torch.from_numpy(cell.green_k_tau().reshape(-1)).to(dev)
        gen = torch.Generator(device=dev).manual_seed(nat)
        W_iw = torch.randn(plan.len("pb", nn), dtype=torch.float64, device=dev, generator=gen).to(torch.complex128)
        v_R = torch.randn(plan.len("pb", 1), dtype=torch.float64, device=dev, generator=gen).to(torch.complex128)
        G_R, P_R, P_iw, W_R = z(plan.len("orb", nt)), z(plan.len("pb", nt)), z(plan.len("pb", nn)), z(plan.len("pb", nt))
        S_R, Sx_R, S_iw = z(plan.len("orb", nt)), z(plan.len("orb", 1)), z(plan.len("orb", nw))
        S_k = z(nk * nw * No * No)
        kd = pb_dims(plan)
        ent = plan.entries
        flops = contraction_flops(cell, ent, kd)
        row = {"atoms": nat, "entries": len(ent), "n_pb": inf["n_pb_total"]}
        for prec in ("fp64", "mixed"):
            def sweep():
                sp = stream.cuda_stream
                plan.green_k_to_R(G_k, G_R, stream=sp)
                plan.polarizability_tau(G_R, P_R, precision=prec, stream=sp)
                plan.transform_tau_iw("B", "tau_to_iw", "pb", P_R, P_iw, stream=sp,
                                      structure=p_iw_structure(inf))
                plan.transform_tau_iw("B", "iw_to_tau", "pb", W_iw, W_R, stream=sp, structure="real")
                plan.self_energy_tau(G_R, W_R, v_R=v_R, Sig_R=S_R, Sigx_R=Sx_R, precision=prec, stream=sp)
                plan.transform_tau_iw("F", "tau_to_iw", "orb", S_R, S_iw, stream=sp)
                plan.fourier_R_to_k("orb", nw, S_iw, S_k, stream=sp)
            with torch.cuda.stream(stream):
                for _ in range(max(3, args.warmup)):
                    sweep()
            plan.sync(stream=stream.cuda_stream)
            torch.cuda.synchronize()
            ts = []
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush_l2(flush)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sweep()
                    e1.record(stream)
                plan.sync(stream=stream.cuda_stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = float(np.mean(ts))
            row[prec] = {"ms_per_sweep": round(ms, 3), "us_per_entry": round(1000.0 * ms / len(ent), 3),
                         "contraction_tflops": round(2 * flops / (ms * 1e-3) / 1e12, 3)}
        rows.append(row)
        del G_k, W_iw, v_R, G_R, P_R, P_iw, W_R, S_R, Sx_R, S_iw, S_k
        plan.close()
        torch.cuda.empty_cache()
    base = rows[0]
    for r in rows:  # time per entry relative to the smallest cell: 1.0 is linear scaling
        for prec in ("fp64", "mixed"):
            r[prec]["per_entry_vs_smallest"] = round(r[prec]["us_per_entry"] / base[prec]["us_per_entry"], 3)
    return {"metric": "P+Sigma sweep time vs atom count (W solve excluded)", "unit": "ms per sweep",
            "steps": args.steps, "warmup": max(3, args.warmup), "data": "synthetic",
            "config": {"workload": "diamond supercells, 9 orbitals and 64 product functions per atom, 2x2x2 k, "
                                   "64 tau, cutoff 12 bohr; W~(R, i nu) and v(R) seeded random",
                       "l2": "256 MB buffer written before each timed sweep"},
            "series": rows}


def run_serve(args, local):
    """Serving (paper_1911_05633_gb300.serve): a Poisson stream of requests over 20 systems
    of different sizes under a device-memory cap below their total -- P/Sigma evaluations on
    the 16-system batch family and two 64-atom f-rich cells (G and W~ resident; a whole
    iteration there would need the W solve at N_PB ~ 3000-3600), whole iterations (W solve,
    chemical potential, Dyson step) on two small cells -- the arrival rate swept to
    saturation.  Per rate: p50 / p99 latency (arrival to completion), throughput and the
    systems brought in."""
    import torch
    import synth
    from paper_1911_05633_gb300.serve import Server, SystemSpec, latency_stats, poisson_arrivals
    torch.cuda.set_device(local)
    prec = args.precision
    specs = {}
    for i, c in enumerate(synth.batch_family()):
        specs[f"b{i:02d}-{c.name}"] = SystemSpec(f"b{i:02d}", c, mode="psigma", precision=prec, w_seed=i)
    for i in range(2):
        c = synth.f_rich_cell(seed=4000 + i)
        specs[f"f{i}-{c.name}"] = SystemSpec(f"f{i}", c, mode="psigma", precision=prec, w_seed=100 + i)
    for n, c in (("it-sc2", synth.make_config(0)),
                 ("it-diamond8-cut5", synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)))):
        specs[n] = SystemSpec(n, c, mode="iteration", precision=prec, workspace_bytes=1 << 30)
    t0 = time.perf_counter()
    for sp in specs.values():
        sp.prepare()
    t_prep = time.perf_counter() - t0
    names = list(specs)
    # the cap (the device pool the systems' buffers live in): well below the sum of the
    # footprints, which are exact from the plans' sizes
    total = sum(sp.footprint for sp in specs.values())
    cap = max(int(0.4 * total), int(1.5 * max(sp.footprint for sp in specs.values())))
    server = Server(specs, mem_cap_bytes=cap, device=local)
    alone = {}
    for n in names:  # service time of each system alone, brought in and resident; measures its plan
        server.run([(0.0, n)])
        lat = [server.run([(0.0, n)])[0].latency for _ in range(2)]
        alone[n] = round(1e3 * float(np.median(lat)), 3)
        server.evict(n)
    mean_service = float(np.mean(list(alone.values()))) / 1e3
    series = []
    for k in ("wait_closes_s", "make_s", "make_plan_s", "close_s"):
        server.timing[k].clear()
    for f in (0.5, 1.0, 2.0, 4.0):  # offered load relative to one system at a time
        rate = f / mean_service
        reqs = server.run(poisson_arrivals(rate, 40 * max(1, args.steps // 5), names, seed=int(f * 100)))
        series.append({"offered_per_s": round(rate, 2), "load_vs_serial": f, **latency_stats(reqs)})
    evictions = sum(1 for e in server.log if e[1] == "evict")
    tm = server.timing
    ms = lambda v: {"n": len(v), "mean_ms": round(1e3 * float(np.mean(v)), 2) if v else None,
                    "p90_ms": round(1e3 * float(np.percentile(v, 90)), 2) if v else None}
    bring = {"waiting_for_evictions": ms(tm["wait_closes_s"]), "making": ms(tm["make_s"]),
             "making_plans": ms(tm["make_plan_s"]),
             "evicting": ms(tm["close_s"])}
    server.close()
    return {"metric": "serve p50/p99 latency of P/Sigma evaluations and whole GW iterations (continuous batching)",
            "unit": "ms", "precision": prec, "data": "synthetic",
            "config": {"systems": {n: {"atoms": sp.cell.n_atoms, "orbitals": sp.cell.n_orb_total,
                                       "n_pb": sp.cell.n_pb_total, "k": int(np.prod(sp.cell.kmesh)),
                                       "tau": sp.cell.n_tau, "request": sp.mode,
                                       "footprint_GB": round(sp.footprint / 1e9, 2),
                                       "plan_GB": round((sp.plan_bytes or 0) / 1e9, 3)} for n, sp in specs.items()},
                       "mem_cap_GB": round(cap / 1e9, 1), "sum_of_footprints_GB": round(total / 1e9, 1),
                       "admission": "arrival order; one request per system at a time; the buffers of resident "
                                    "systems in one device pool of the cap's size; a system not resident is "
                                    "brought in on admission into a free range of the pool, idle residents "
                                    "evicted least recently used first (those no queued request waits for "
                                    "before the others) until one range holds it; bring-ins and evictions off "
                                    "the request loop"},
            "prepare_s": round(t_prep, 1), "alone_ms": alone, "series": series, "evictions": evictions,
            "bring_in": bring}


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.serve:
        if rank == 0:
            print(json.dumps(run_serve(args, local)), flush=True)
        return
    if args.scaling is not None:
        if rank == 0:
            print(json.dumps(run_scaling(args, local)), flush=True)
        return
    if args.w_solve:
        if rank == 0:
            print(json.dumps(run_w_solve(args, local)), flush=True)
        return
    if args.batch:
        if rank == 0:
            try:
                peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            except Exception:
                peaks = {}
            print(json.dumps(run_batch3(args, local, peaks)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.config == 1 or args.small:  # the 8-atom whole sweep as the main line
        full, cell = run_full(args, local)
        m = full[args.precision]
        step_ms_max, value = aggregate(m["ms_per_sweep"], world)
        out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(step_ms_max, 4), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16x3-f32acc",
               "data": "synthetic", "config": {"workload": full["workload"], "precision": args.precision},
               "roofline": m["roofline_dominant_kernel"], "gpu_launches": None, "full_sweep": full}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out, cell = run_rows(args, rank, world, local)
    if not args.no_extra:
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            peaks = {}
        # extra blocks: each on a device emptied of the previous one's plans and buffers;
        # a failure is recorded in the line instead of losing the line
        def w_solve():  # the W solve of the same cell (Eq. W_1), timed apart from the rows
            r = run_w_solve(args, local, cell)
            return {k: r[k] for k in ("value", "unit", "config", "ms_per_inverse", "fp64_equivalent_tflops",
                                      "finite")} | {"kernels": dict(list(r["kernels"].items())[:3])}

        for key, fn in (("full_sweep_8_atoms", lambda: run_full(args, local)[0]),
                        ("batched_uneven_systems", lambda: run_batch3(args, local, peaks)),
                        ("w_solve", w_solve)):
            release_device()
            try:
                out[key] = fn()
            except Exception as e:  # noqa: BLE001
                out[key] = {"error": f"{type(e).__name__}: {e}"[:400]}
            release_device()
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            orc = OracleRows(cell)
            s = orc.time_one()
            out["cpu_baseline"] = {"value": round(1.0 / s, 8), "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                   "sample": orc.note}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
