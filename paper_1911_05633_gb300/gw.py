"""Python binding of libgw (include/gw.h): argument marshalling only.

Every entry point of the C ABI has a method of the same name on ``Plan``.  Device
buffers are torch tensors (complex128, contiguous, on the plan's device) used as
plain memory; all arithmetic of the sweep runs in the library's CUDA kernels.
The binding fails loudly when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgw.so")

GW_OK = 0
GW_FP64, GW_MIXED = 0, 1
GW_FERMION, GW_BOSON = 0, 1
GW_TAU_TO_IW, GW_IW_TO_TAU = 0, 1
GW_BLOCK_ORB, GW_BLOCK_PB = 0, 1

_PREC = {"fp64": GW_FP64, "mixed": GW_MIXED}
_STAT = {"F": GW_FERMION, "B": GW_BOSON, "fermion": GW_FERMION, "boson": GW_BOSON}
_DIR = {"tau_to_iw": GW_TAU_TO_IW, "iw_to_tau": GW_IW_TO_TAU}
_BLK = {"orb": GW_BLOCK_ORB, "pb": GW_BLOCK_PB}
_STRUCT = {"general": 0, "mirror": 1, "real": 2, "mirror_nonneg": 5}

EXPORTED = [
    "gw_plan_create", "gw_plan_destroy", "gw_plan_query", "gw_plan_entries", "gw_plan_offsets", "gw_plan_entry_dims",
    "gw_dyson_green_tau", "gw_chemical_potential", "gw_qp_energies", "gw_continue_sigma", "gw_spectral_function",
    "gw_plan_transform_matrix", "gw_fourier_k_to_R", "gw_green_k_to_R", "gw_polarizability_tau",
    "gw_transform_tau_iw", "gw_screened_W_iw", "gw_self_energy_tau", "gw_fourier_R_to_k", "gw_sync",
    "gw_status_string", "gw_last_error", "gw_fp_peak", "gw_screened_W_iw_noalloc",
    "gw_timing_enable", "gw_timing_read", "gw_timing_reset", "gw_transform_tau_iw_ex",
    "gw_batch_create", "gw_batch_destroy", "gw_batch_query", "gw_batch_polarizability_tau",
    "gw_batch_self_energy_tau", "gw_batch_tune", "gw_batch_sync",
]


class GwCell(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("n_atoms", C.c_int), ("frac", C.POINTER(C.c_double)),
                ("species", C.POINTER(C.c_int))]


class GwBasis(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_orb", C.POINTER(C.c_int)), ("n_prod", C.POINTER(C.c_int)),
                ("C", C.POINTER(C.POINTER(C.c_double))), ("n_prod_far", C.POINTER(C.c_int)),
                ("n_prod_near", C.POINTER(C.c_int))]


class GwGrid(C.Structure):
    _fields_ = [("beta", C.c_double), ("n_tau", C.c_int), ("tau", C.POINTER(C.c_double)),
                ("n_omega", C.c_int), ("omega_idx", C.POINTER(C.c_int)),
                ("n_nu", C.c_int), ("nu_idx", C.POINTER(C.c_int))]


class GwOptions(C.Structure):
    _fields_ = [("spin", C.c_int), ("strict_kmesh", C.c_int), ("host_only", C.c_int), ("device", C.c_int),
                ("workspace_bytes", C.c_size_t), ("no_symmetry", C.c_int), ("w_solver", C.c_int),
                ("fp64_products", C.c_int), ("r_b", C.c_double), ("defer_scratch", C.c_int)]


class GwPlanInfo(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_entries", C.c_int), ("n_k", C.c_int), ("n_tau", C.c_int),
                ("n_omega", C.c_int), ("n_nu", C.c_int), ("n_orb_total", C.c_int), ("n_pb_total", C.c_int),
                ("kmesh", C.c_int * 3), ("kmesh_required", C.c_int * 3), ("c_symmetric", C.c_int),
                ("len_orb", C.c_int64), ("len_pb", C.c_int64), ("workspace_bytes", C.c_size_t),
                ("nu_chunk", C.c_int), ("cond_fermion", C.c_double), ("cond_boson", C.c_double),
                ("w_symmetric", C.c_int), ("n_q_solved", C.c_int), ("w_tensor", C.c_int),
                ("sigma_tensor", C.c_int), ("p_tensor", C.c_int), ("transform_tensor", C.c_int),
                ("n_entries_far", C.c_int), ("n_entries_near", C.c_int), ("mixed_queue", C.c_int),
                ("w_block", C.c_int)]


class GwBatchInfo(C.Structure):
    _fields_ = [("n_plans", C.c_int), ("n_units_p", C.c_longlong), ("n_units_s", C.c_longlong),
                ("groups_p", C.c_int), ("groups_s", C.c_int), ("kc_p", C.c_int), ("kc_s", C.c_int),
                ("order_p", C.c_int), ("order_s", C.c_int), ("tuned", C.c_int), ("n_classes", C.c_int)]


class GwError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what}: {detail} (status {status})")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgw.so (built in-tree by paper_1911_05633_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgw.so not found at {path}: run `python -m paper_1911_05633_gb300.build`")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.gw_plan_create.argtypes = [C.POINTER(GwCell), C.POINTER(GwBasis), C.POINTER(C.c_int), C.POINTER(GwGrid),
                                   C.c_double, C.POINTER(GwOptions), C.POINTER(vp)]
    lib.gw_plan_destroy.argtypes = [vp]
    lib.gw_plan_query.argtypes = [vp, C.POINTER(GwPlanInfo)]
    lib.gw_plan_entries.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.gw_plan_offsets.argtypes = [vp, C.c_int, C.POINTER(C.c_int64)]
    lib.gw_plan_entry_dims.argtypes = [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.gw_dyson_green_tau.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp]
    lib.gw_qp_energies.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp]
    lib.gw_continue_sigma.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_double), C.c_double, vp, vp]
    lib.gw_spectral_function.argtypes = [vp, vp, vp, vp, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_double,
                                         vp, vp]
    lib.gw_chemical_potential.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    lib.gw_plan_transform_matrix.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double)]
    lib.gw_fourier_k_to_R.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
    lib.gw_green_k_to_R.argtypes = [vp, vp, vp, vp]
    lib.gw_polarizability_tau.argtypes = [vp, vp, vp, C.c_int, vp]
    lib.gw_transform_tau_iw.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    lib.gw_transform_tau_iw_ex.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]
    lib.gw_screened_W_iw.argtypes = [vp, vp, vp, vp, vp]
    lib.gw_screened_W_iw_noalloc.argtypes = [vp, vp, vp, vp, vp]
    lib.gw_self_energy_tau.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int, vp]
    lib.gw_fourier_R_to_k.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
    lib.gw_sync.argtypes = [vp, vp]
    lib.gw_timing_enable.argtypes = [vp, C.c_int]
    lib.gw_timing_read.argtypes = [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                   C.POINTER(C.c_longlong)]
    lib.gw_timing_reset.argtypes = [vp]
    lib.gw_fp_peak.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    vpp = C.POINTER(C.c_void_p)
    lib.gw_batch_create.argtypes = [vpp, C.c_int, C.POINTER(vp)]
    lib.gw_batch_destroy.argtypes = [vp]
    lib.gw_batch_query.argtypes = [vp, C.POINTER(GwBatchInfo)]
    lib.gw_batch_polarizability_tau.argtypes = [vp, vpp, vpp, vp]
    lib.gw_batch_self_energy_tau.argtypes = [vp, vpp, vpp, vpp, vp]
    lib.gw_batch_tune.argtypes = [vp, vpp, vpp, vpp, vpp, C.c_int, vp]
    lib.gw_batch_sync.argtypes = [vp, vp]
    lib.gw_status_string.argtypes = [C.c_int]
    lib.gw_status_string.restype = C.c_char_p
    lib.gw_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("gw_status_string", "gw_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        lib = load_library()
        raise GwError(status, what, f"{lib.gw_status_string(status).decode()}; {lib.gw_last_error().decode()}")


def _ptr(arr: np.ndarray, ctype):
    return arr.ctypes.data_as(C.POINTER(ctype))


def fp_peak(device: int = 0):
    """(FP64, FP32) dense FMA throughput in TFLOP/s measured on `device` (gw_fp_peak)."""
    lib = load_library()
    a, b = C.c_double(), C.c_double()
    _check(lib.gw_fp_peak(int(device), C.byref(a), C.byref(b)), "gw_fp_peak")
    return a.value, b.value


class Plan:
    """A gw_plan_t: pair list, phases, basis coefficients and transform matrices."""

    def __init__(self, lattice, frac, species, n_orb: Sequence[int], n_prod: Sequence[int], C_list,
                 kmesh, beta: float, tau, omega_idx, nu_idx, cutoff: float, spin: int = 2,
                 strict_kmesh: bool = False, host_only: bool = False, device: int = 0, workspace_bytes: int = 0,
                 no_symmetry: bool = False, w_solver: str = "auto", fp64_products: str = "auto",
                 n_prod_far: Sequence[int] = None, r_b: float = 0.0, n_prod_near: Sequence[int] = None,
                 defer_scratch: bool = False):
        lib = load_library()
        self._lib = lib
        self._keep = []
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
        frac = np.ascontiguousarray(np.asarray(frac, dtype=np.float64).reshape(-1, 3))
        species = np.ascontiguousarray(np.asarray(species, dtype=np.int32))
        n_orb = np.ascontiguousarray(np.asarray(n_orb, dtype=np.int32))
        n_prod = np.ascontiguousarray(np.asarray(n_prod, dtype=np.int32))
        Cs = [np.ascontiguousarray(np.asarray(c, dtype=np.float64)) for c in C_list]
        Cptr = (C.POINTER(C.c_double) * len(Cs))(*[_ptr(c, C.c_double) for c in Cs])
        tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
        om = np.ascontiguousarray(np.asarray(omega_idx, dtype=np.int32))
        nu = np.ascontiguousarray(np.asarray(nu_idx, dtype=np.int32))
        far = None if n_prod_far is None else np.ascontiguousarray(np.asarray(n_prod_far, dtype=np.int32))
        near = None if n_prod_near is None else np.ascontiguousarray(np.asarray(n_prod_near, dtype=np.int32))
        self._keep += [lat, frac, species, n_orb, n_prod, Cs, Cptr, tau, om, nu, far, near]
        cell = GwCell((C.c_double * 9)(*lat), len(frac), _ptr(frac, C.c_double), _ptr(species, C.c_int))
        basis = GwBasis(len(Cs), _ptr(n_orb, C.c_int), _ptr(n_prod, C.c_int), Cptr,
                        _ptr(far, C.c_int) if far is not None else C.POINTER(C.c_int)(),
                        _ptr(near, C.c_int) if near is not None else C.POINTER(C.c_int)())
        grid = GwGrid(float(beta), len(tau), _ptr(tau, C.c_double), len(om), _ptr(om, C.c_int),
                      len(nu), _ptr(nu, C.c_int))
        opt = GwOptions(int(spin), int(bool(strict_kmesh)), int(bool(host_only)), int(device), int(workspace_bytes),
                        int(bool(no_symmetry)), {"auto": 0, "gauss_jordan": 1}[w_solver],
                        {"auto": 0, "fp64": 1}[fp64_products], float(r_b), int(bool(defer_scratch)))
        km = (C.c_int * 3)(*[int(x) for x in kmesh])
        h = C.c_void_p()
        _check(lib.gw_plan_create(C.byref(cell), C.byref(basis), km, C.byref(grid), float(cutoff),
                                  C.byref(opt), C.byref(h)), "gw_plan_create")
        self._h = h
        self.device = int(device)
        self.host_only = bool(host_only)
        inf = GwPlanInfo()
        _check(lib.gw_plan_query(h, C.byref(inf)), "gw_plan_query")
        self.info = {f: (list(getattr(inf, f)) if f in ("kmesh", "kmesh_required") else getattr(inf, f))
                     for f, _ in GwPlanInfo._fields_}
        E = self.info["n_entries"]
        ent = np.empty((E, 8), np.int64)
        _check(lib.gw_plan_entries(h, _ptr(ent, C.c_int64)), "gw_plan_entries")
        self.entries = ent
        self.off_orb = np.empty(E + 1, np.int64)
        self.off_pb = np.empty(E + 1, np.int64)
        _check(lib.gw_plan_offsets(h, GW_BLOCK_ORB, _ptr(self.off_orb, C.c_int64)), "gw_plan_offsets")
        _check(lib.gw_plan_offsets(h, GW_BLOCK_PB, _ptr(self.off_pb, C.c_int64)), "gw_plan_offsets")
        self._dims = {}
        for kind, code in (("orb", GW_BLOCK_ORB), ("pb", GW_BLOCK_PB)):
            r, c = np.empty(E, np.int32), np.empty(E, np.int32)
            _check(lib.gw_plan_entry_dims(h, code, _ptr(r, C.c_int32), _ptr(c, C.c_int32)), "gw_plan_entry_dims")
            self._dims[kind] = (r, c)

    @classmethod
    def from_cell(cls, cell, **kw) -> "Plan":
        """Plan for a synthetic cell object (geometry, basis and grids are read from it,
        with its reduced basis beyond sphere B when it has one)."""
        if getattr(cell, "r_b", 0.0) > 0 and "r_b" not in kw:
            kw = dict(kw, r_b=cell.r_b, n_prod_far=[s.n_prod_far for s in cell.species])
            if any(getattr(s, "n_prod_near", None) for s in cell.species):
                kw["n_prod_near"] = [getattr(s, "n_prod_near", None) or s.n_prod for s in cell.species]
        return cls(cell.lattice, cell.frac, cell.species_of_atom, [s.n_orb for s in cell.species],
                   [s.n_prod for s in cell.species], [s.C for s in cell.species], cell.kmesh, cell.beta,
                   cell.tau, cell.omega_idx, cell.nu_idx, cell.cutoff, spin=cell.spin, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gw_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host queries -----------------------------------------------------------
    def offsets(self, kind: str) -> np.ndarray:
        return self.off_pb if kind == "pb" else self.off_orb

    def transform_matrix(self, stat: str, direction: str) -> np.ndarray:
        inf = self.info
        nf = inf["n_omega"] if _STAT[stat] == GW_FERMION else inf["n_nu"]
        shape = (nf, inf["n_tau"]) if _DIR[direction] == GW_TAU_TO_IW else (inf["n_tau"], nf)
        out = np.empty(shape, np.complex128)
        _check(self._lib.gw_plan_transform_matrix(self._h, _STAT[stat], _DIR[direction],
                                                  out.ctypes.data_as(C.POINTER(C.c_double))),
               "gw_plan_transform_matrix")
        return out

    def len(self, kind: str, n_slices: int) -> int:
        return int(n_slices * (self.info["len_pb"] if kind == "pb" else self.info["len_orb"]))

    def dense_n(self, kind: str) -> int:
        return int(self.info["n_pb_total"] if kind == "pb" else self.info["n_orb_total"])

    # ---- device buffers (torch as plain device memory) --------------------------
    def _torch(self):
        import torch
        return torch

    def _dev(self):
        return self._torch().device("cuda", self.device)

    def _stream(self, stream):
        if stream is not None:
            return C.c_void_p(int(stream))
        return C.c_void_p(self._torch().cuda.current_stream(self._dev()).cuda_stream)

    def _buf(self, t, n: int, name: str):
        torch = self._torch()
        if t is None:
            return torch.empty(n, dtype=torch.complex128, device=self._dev())
        if t.dtype != torch.complex128 or not t.is_contiguous() or t.device != self._dev() or t.numel() != n:
            raise ValueError(f"{name}: need a contiguous complex128 tensor of {n} elements on {self._dev()}")
        return t

    def _in(self, t, n: int, name: str):
        return C.c_void_p(self._buf(t, n, name).data_ptr())

    # ---- the sweep ------------------------------------------------------------------
    def fourier_k_to_R(self, kind: str, n_slices: int, F_k, F_R=None, stream=None):
        N = self.dense_n(kind)
        F_R = self._buf(F_R, self.len(kind, n_slices), "F_R")
        _check(self._lib.gw_fourier_k_to_R(self._h, _BLK[kind], int(n_slices),
                                           self._in(F_k, self.info["n_k"] * n_slices * N * N, "F_k"),
                                           C.c_void_p(F_R.data_ptr()), self._stream(stream)), "gw_fourier_k_to_R")
        return F_R

    def green_k_to_R(self, G_k, G_R=None, stream=None):
        nt, N = self.info["n_tau"], self.dense_n("orb")
        G_R = self._buf(G_R, self.len("orb", nt), "G_R")
        _check(self._lib.gw_green_k_to_R(self._h, self._in(G_k, self.info["n_k"] * nt * N * N, "G_k"),
                                         C.c_void_p(G_R.data_ptr()), self._stream(stream)), "gw_green_k_to_R")
        return G_R

    def polarizability_tau(self, G_R, P_R=None, precision: str = "fp64", stream=None):
        nt = self.info["n_tau"]
        P_R = self._buf(P_R, self.len("pb", nt), "P_R")
        _check(self._lib.gw_polarizability_tau(self._h, self._in(G_R, self.len("orb", nt), "G_R"),
                                               C.c_void_p(P_R.data_ptr()), _PREC[precision], self._stream(stream)),
               "gw_polarizability_tau")
        return P_R

    def transform_tau_iw(self, stat: str, direction: str, kind: str, inp, out=None, stream=None,
                         structure: str = "general"):
        """gw_transform_tau_iw, or gw_transform_tau_iw_ex when `structure` is "mirror"
        (input with F(beta - tau) = F(tau)*), "mirror_nonneg" (the same, writing only the
        slices of the frequencies nu >= 0) or "real" (input with zero imaginary parts)."""
        nt = self.info["n_tau"]
        nf = self.info["n_omega"] if _STAT[stat] == GW_FERMION else self.info["n_nu"]
        n_in, n_out = (nt, nf) if _DIR[direction] == GW_TAU_TO_IW else (nf, nt)
        out = self._buf(out, self.len(kind, n_out), "out")
        _check(self._lib.gw_transform_tau_iw_ex(self._h, _STAT[stat], _DIR[direction], _BLK[kind],
                                                _STRUCT[structure], self._in(inp, self.len(kind, n_in), "in"),
                                                C.c_void_p(out.data_ptr()), self._stream(stream)),
               "gw_transform_tau_iw_ex")
        return out

    def screened_W_iw(self, P_R_iw, v_q, Wt_R_iw=None, stream=None):
        nn, N = self.info["n_nu"], self.dense_n("pb")
        Wt_R_iw = self._buf(Wt_R_iw, self.len("pb", nn), "Wt_R_iw")
        _check(self._lib.gw_screened_W_iw(self._h, self._in(P_R_iw, self.len("pb", nn), "P_R_iw"),
                                          self._in(v_q, self.info["n_k"] * N * N, "v_q"),
                                          C.c_void_p(Wt_R_iw.data_ptr()), self._stream(stream)), "gw_screened_W_iw")
        return Wt_R_iw

    def screened_W_iw_noalloc(self, P_R_iw, v_q, Wt_R_iw, stream=None):
        """gw_screened_W_iw_noalloc: the W solve with the library's fixed 32 MiB scratch
        (for callers that cannot allocate device memory while they run); Wt_R_iw must be given."""
        nn, N = self.info["n_nu"], self.dense_n("pb")
        _check(self._lib.gw_screened_W_iw_noalloc(self._h, self._in(P_R_iw, self.len("pb", nn), "P_R_iw"),
                                                  self._in(v_q, self.info["n_k"] * N * N, "v_q"),
                                                  self._in(Wt_R_iw, self.len("pb", nn), "Wt_R_iw"),
                                                  self._stream(stream)), "gw_screened_W_iw_noalloc")
        return Wt_R_iw

    def self_energy_tau(self, G_R, Wt_R, v_R=None, Sig_R=None, Sigx_R=None, precision: str = "fp64",
                        stream=None):
        nt = self.info["n_tau"]
        Sig_R = self._buf(Sig_R, self.len("orb", nt), "Sig_R")
        vp = C.c_void_p(0)
        xp = C.c_void_p(0)
        if v_R is not None:
            vp = self._in(v_R, self.len("pb", 1), "v_R")
            Sigx_R = self._buf(Sigx_R, self.len("orb", 1), "Sigx_R")
            xp = C.c_void_p(Sigx_R.data_ptr())
        _check(self._lib.gw_self_energy_tau(self._h, self._in(G_R, self.len("orb", nt), "G_R"),
                                            self._in(Wt_R, self.len("pb", nt), "Wt_R"), vp,
                                            C.c_void_p(Sig_R.data_ptr()), xp, _PREC[precision],
                                            self._stream(stream)), "gw_self_energy_tau")
        return (Sig_R, Sigx_R) if v_R is not None else Sig_R

    def fourier_R_to_k(self, kind: str, n_slices: int, F_R, F_k=None, stream=None):
        N = self.dense_n(kind)
        F_k = self._buf(F_k, self.info["n_k"] * n_slices * N * N, "F_k")
        _check(self._lib.gw_fourier_R_to_k(self._h, _BLK[kind], int(n_slices),
                                           self._in(F_R, self.len(kind, n_slices), "F_R"),
                                           C.c_void_p(F_k.data_ptr()), self._stream(stream)), "gw_fourier_R_to_k")
        return F_k

    # ---- Eq. G_1 -------------------------------------------------------------------------
    def _dyson_inputs(self, H_k, Sigx_k, Sig_k_iw):
        nk, N, nw = self.info["n_k"], self.dense_n("orb"), self.info["n_omega"]
        h = self._in(H_k, nk * N * N, "H_k")
        x = self._in(Sigx_k, nk * N * N, "Sigx_k") if Sigx_k is not None else C.c_void_p(0)
        c = self._in(Sig_k_iw, nk * nw * N * N, "Sig_k_iw") if Sig_k_iw is not None else C.c_void_p(0)
        return h, x, c

    def dyson_green_tau(self, H_k, mu: float, Sigx_k=None, Sig_k_iw=None, G_k_tau=None, stream=None):
        """gw_dyson_green_tau: G(k, tau) [N_k][N_tau][N][N] from Eq. G_1 with Sigma_x(k) and
        Sigma_c(k, i w) (None: zero)."""
        nk, N, nt = self.info["n_k"], self.dense_n("orb"), self.info["n_tau"]
        G_k_tau = self._buf(G_k_tau, nk * nt * N * N, "G_k_tau")
        h, x, c = self._dyson_inputs(H_k, Sigx_k, Sig_k_iw)
        _check(self._lib.gw_dyson_green_tau(self._h, h, x, c, float(mu), C.c_void_p(G_k_tau.data_ptr()),
                                            self._stream(stream)), "gw_dyson_green_tau")
        return G_k_tau

    def chemical_potential(self, H_k, n_electrons: float, lo: float, hi: float, tol: float = 1e-12,
                           Sigx_k=None, Sig_k_iw=None, stream=None):
        """gw_chemical_potential: (mu, N(mu)) with N(mu) = n_electrons by bisection on [lo, hi]."""
        h, x, c = self._dyson_inputs(H_k, Sigx_k, Sig_k_iw)
        mu, n = C.c_double(), C.c_double()
        _check(self._lib.gw_chemical_potential(self._h, h, x, c, float(n_electrons), float(lo), float(hi), float(tol),
                                               C.byref(mu), C.byref(n), self._stream(stream)),
               "gw_chemical_potential")
        return mu.value, n.value

    def qp_energies(self, H_k, mu: float, Sigx_k=None, Sig_k_iw=None, E_k=None, stream=None):
        """gw_qp_energies: linearised quasiparticle energies [N_k][N] (float64, ascending)."""
        torch = self._torch()
        nk, N = self.info["n_k"], self.dense_n("orb")
        if E_k is None:
            E_k = torch.empty(nk * N, dtype=torch.float64, device=self._dev())
        elif E_k.dtype != torch.float64 or not E_k.is_contiguous() or E_k.numel() != nk * N:
            raise ValueError(f"E_k: need a contiguous float64 tensor of {nk * N} elements")
        h, x, c = self._dyson_inputs(H_k, Sigx_k, Sig_k_iw)
        _check(self._lib.gw_qp_energies(self._h, h, x, c, float(mu), C.c_void_p(E_k.data_ptr()),
                                        self._stream(stream)), "gw_qp_energies")
        return E_k

    def continue_sigma(self, Sig_k_iw, w_real, delta: float, Sig_k_w=None, stream=None):
        """gw_continue_sigma: Sigma(k, w + i delta) [N_k][len(w_real)][N][N] by the continued
        fraction of Eq. sf_9 through the non-negative sampled frequencies."""
        nk, N, nw = self.info["n_k"], self.dense_n("orb"), self.info["n_omega"]
        wr = np.ascontiguousarray(np.asarray(w_real, dtype=np.float64))
        Sig_k_w = self._buf(Sig_k_w, nk * len(wr) * N * N, "Sig_k_w")
        _check(self._lib.gw_continue_sigma(self._h, self._in(Sig_k_iw, nk * nw * N * N, "Sig_k_iw"), len(wr),
                                           _ptr(wr, C.c_double), float(delta), C.c_void_p(Sig_k_w.data_ptr()),
                                           self._stream(stream)), "gw_continue_sigma")
        return Sig_k_w

    def spectral_function(self, H_k, w_real, delta: float, mu: float, Sigx_k=None, Sig_k_w=None, stream=None):
        """gw_spectral_function: A(k, w) [N_k][len(w_real)] (float64) from the retarded G."""
        torch = self._torch()
        nk, N = self.info["n_k"], self.dense_n("orb")
        wr = np.ascontiguousarray(np.asarray(w_real, dtype=np.float64))
        A = torch.empty(nk * len(wr), dtype=torch.float64, device=self._dev())
        h = self._in(H_k, nk * N * N, "H_k")
        x = self._in(Sigx_k, nk * N * N, "Sigx_k") if Sigx_k is not None else C.c_void_p(0)
        c = self._in(Sig_k_w, nk * len(wr) * N * N, "Sig_k_w") if Sig_k_w is not None else C.c_void_p(0)
        _check(self._lib.gw_spectral_function(self._h, h, x, c, len(wr), _ptr(wr, C.c_double), float(delta), float(mu),
                                              C.c_void_p(A.data_ptr()), self._stream(stream)), "gw_spectral_function")
        return A

    def sync(self, stream=None):
        _check(self._lib.gw_sync(self._h, self._stream(stream)), "gw_sync")

    # ---- per-kernel event timing -----------------------------------------------------
    def timing_enable(self, on: bool = True):
        _check(self._lib.gw_timing_enable(self._h, 1 if on else 0), "gw_timing_enable")

    def timing_reset(self):
        _check(self._lib.gw_timing_reset(self._h), "gw_timing_reset")

    def timing_read(self) -> dict:
        """{kernel name: (total device ms, launches)} since the last reset."""
        out = {}
        name, ms, n = C.c_char_p(), C.c_double(), C.c_longlong()
        i = 0
        while self._lib.gw_timing_read(self._h, i, C.byref(name), C.byref(ms), C.byref(n)) == GW_OK:
            out[name.value.decode()] = (ms.value, n.value)
            i += 1
        return out

    # ---- ragged layout helpers (host side) ------------------------------------------
    def block_shape(self, e: int, kind: str):
        """(rows, cols) of entry e's block: (n_a, n_b) or (K_a(e), K_b(e))."""
        r, c = self._dims[kind]
        return int(r[e]), int(c[e])

    def unpack(self, flat: np.ndarray, kind: str, n_slices: int):
        """Entry-layout vector -> list of [n_slices][rows][cols] arrays."""
        off = self.offsets(kind)
        out = []
        for e in range(len(self.entries)):
            r, c = self.block_shape(e, kind)
            out.append(flat[n_slices * off[e]: n_slices * off[e + 1]].reshape(n_slices, r, c))
        return out

    def pack(self, blocks, kind: str) -> np.ndarray:
        return np.concatenate([np.ascontiguousarray(b).reshape(-1) for b in blocks]).astype(np.complex128)


class Batch:
    """A gw_batch_t: the GW_MIXED P and Sigma contractions of several plans (systems of
    uneven sizes) in one persistent launch each."""

    def __init__(self, plans: Sequence[Plan]):
        lib = load_library()
        self._lib = lib
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = C.c_void_p()
        _check(lib.gw_batch_create(arr, len(self.plans), C.byref(h)), "gw_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gw_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        inf = GwBatchInfo()
        _check(self._lib.gw_batch_query(self._h, C.byref(inf)), "gw_batch_query")
        return {f: getattr(inf, f) for f, _ in GwBatchInfo._fields_}

    def _ptrs(self, ts, kind, n_slices, name, create=False):
        out = []
        for p, t in zip(self.plans, ts if ts is not None else [None] * len(self.plans)):
            out.append(p._buf(t, p.len(kind, n_slices(p)), name) if create else p._buf(t, p.len(kind, n_slices(p)),
                                                                                       name))
        return out, (C.c_void_p * len(out))(*[t.data_ptr() for t in out])

    def _stream(self, stream):
        return self.plans[0]._stream(stream)

    def polarizability_tau(self, G_R, P_R=None, stream=None):
        nt = lambda p: p.info["n_tau"]
        G, gp = self._ptrs(G_R, "orb", nt, "G_R")
        P, pp = self._ptrs(P_R, "pb", nt, "P_R", create=True)
        _check(self._lib.gw_batch_polarizability_tau(self._h, gp, pp, self._stream(stream)),
               "gw_batch_polarizability_tau")
        return P

    def self_energy_tau(self, G_R, Wt_R, Sig_R=None, stream=None):
        nt = lambda p: p.info["n_tau"]
        G, gp = self._ptrs(G_R, "orb", nt, "G_R")
        W, wp = self._ptrs(Wt_R, "pb", nt, "Wt_R")
        S, sp = self._ptrs(Sig_R, "orb", nt, "Sig_R", create=True)
        _check(self._lib.gw_batch_self_energy_tau(self._h, gp, wp, sp, self._stream(stream)),
               "gw_batch_self_energy_tau")
        return S

    def tune(self, G_R, P_R, Wt_R, Sig_R, reps: int = 3, stream=None):
        nt = lambda p: p.info["n_tau"]
        _, gp = self._ptrs(G_R, "orb", nt, "G_R")
        _, pp = self._ptrs(P_R, "pb", nt, "P_R")
        _, wp = self._ptrs(Wt_R, "pb", nt, "Wt_R")
        _, sp = self._ptrs(Sig_R, "orb", nt, "Sig_R")
        _check(self._lib.gw_batch_tune(self._h, gp, pp, wp, sp, int(reps), self._stream(stream)), "gw_batch_tune")
        return self.info

    def sync(self, stream=None):
        _check(self._lib.gw_batch_sync(self._h, self._stream(stream)), "gw_batch_sync")
