"""The allocation-free W solve (gw_screened_W_iw_noalloc) against the plan's W solve.

Callers that cannot call cudaMalloc once they run (codes that hand all device memory
to their own pool up front, or run under an allocator that forbids growth) use this
entry point: its scratch is a fixed 32 MiB device array inside the library.  This
test calls it through the C ABI twice in a row on the same inputs and compares each
result with gw_screened_W_iw's, at the tolerance of the FP64 parity tests (1e-10).
It lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _setup(cell):
    import torch
    from paper_1911_05633_gb300 import gw
    lib = gw.load_library()
    fn = lib.gw_screened_W_iw_noalloc
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    # the plan's W solve with the same FP64 Gauss-Jordan inverse as the fixed-scratch variant
    plan = gw.Plan.from_cell(cell, w_solver="gauss_jordan")
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to("cuda")
    Gk = cell.green_k_tau()
    vq, _ = cell.coulomb()
    GR = plan.green_k_to_R(d(Gk))
    PR = plan.polarizability_tau(GR)
    Piw = plan.transform_tau_iw("B", "tau_to_iw", "pb", PR)
    v = d(vq)
    return torch, plan, fn, Piw, v


@pytest.mark.parametrize("which", ["sc2", "diamond8_short"])
def test_noalloc_w_matches_plan_path(which):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if which == "sc2":
        cell = synth.make_config(0)
    else:
        cell = synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2))
    torch, plan, fn, Piw, v = _setup(cell)
    ref = plan.screened_W_iw(Piw, v)
    plan.sync()
    ref_h = ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(ref, complex(np.nan, np.nan))
        st = fn(plan._h, ctypes.c_void_p(Piw.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, plan._lib.gw_last_error().decode()
        plan.sync()
        got = out.cpu().numpy()
        err = float(np.linalg.norm(got - ref_h) / np.linalg.norm(ref_h))
        assert err < TOL, (call, err)


def test_noalloc_w_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_05633_gb300 import gw
    # 9 atoms x 128 product functions: N_PB = 1152, two matrices exceed 32 MiB
    lat = np.eye(3) * 30.0
    frac = np.array([[i / 9.0, 0.0, 0.0] for i in range(9)])
    sp = [synth.Species("big", 1, 128, np.ones((128, 1, 1)))]
    cell = synth.SynthCell("nine", lat, frac, np.zeros(9, np.int32), sp, (1, 1, 1), 10.0, 8, 0.0, seed=5)
    plan = gw.Plan(cell.lattice, cell.frac, cell.species_of_atom, [1], [128], [sp[0].C], (1, 1, 1), cell.beta,
                   cell.tau, cell.omega_idx, cell.nu_idx, 0.0)
    lib = gw.load_library()
    fn = lib.gw_screened_W_iw_noalloc
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    buf = torch.zeros(16, dtype=torch.complex128, device="cuda")
    st = fn(plan._h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
            ctypes.c_void_p(buf.data_ptr()), None)
    assert st == 10  # GW_ERR_UNSUPPORTED, nothing launched
    assert b"32 MiB" in lib.gw_last_error()
