"""Per-kernel event timing of the C ABI (gw_timing_enable / read / reset) on the GPU:
every launch of an entry point is counted under its kernel name with a positive time,
and timing changes no result."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_timing_counts_launches_and_changes_nothing():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_05633_gb300 import gw
    cell = synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2))
    plan = gw.Plan.from_cell(cell)
    assert plan.info["w_tensor"] == 1
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to("cuda")
    Gk = d(cell.green_k_tau())
    vq = d(cell.coulomb()[0])

    def sweep():
        GR = plan.green_k_to_R(Gk)
        PR = plan.polarizability_tau(GR)
        Piw = plan.transform_tau_iw("B", "tau_to_iw", "pb", PR)
        W = plan.screened_W_iw(Piw, vq)
        plan.sync()
        return W.cpu().numpy()

    ref = sweep()
    plan.timing_reset()
    assert plan.timing_read() == {}
    plan.timing_enable(True)
    out = sweep()
    plan.timing_enable(False)
    t = plan.timing_read()
    assert np.array_equal(out, ref)
    # the general bosonic tau -> i nu transform runs as fused digit products on the tensor cores
    assert t["k_gather_k_to_R"][1] >= 1 and t["k_polarizability_fp64"][1] == 1 and t["k_oz_transform"][1] == 1
    # two batched tensor-core inverses (v(q), then v^-1 - P): each kernel of the inverse twice
    for k in ("k_gj_inverse_f32", "k_ozaki_residual<first>", "k_ozaki_residual<second>", "k_slice_A"):
        assert t[k][1] == 2, (k, t[k])
    assert all(ms > 0.0 for ms, _ in t.values())
    # disabled: nothing more is recorded
    sweep()
    assert plan.timing_read() == t
    plan.timing_reset()
    assert plan.timing_read() == {}
