"""The request loop on the device (paper_1911_05633_gb300.serve): residency under a
memory cap below the systems' total (bring in on admission, eviction of idle systems with
their state kept on the host), a system's result the same alone and in the mix, the state
advancing per iteration with the chemical potential updated, every buffer in the
server's device pool, and the device memory measured by the driver staying within the
pool and the plans' tables."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def specs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_05633_gb300.serve import SystemSpec
    cells = {"c0": (synth.make_config(0), "iteration"), "mixed": (synth.mixed_species_cell(), "iteration"),
             "c1_cut5": (synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2)), "iteration"),
             "d16": (synth.make_config(2, atoms=16, n_tau=16), "psigma")}
    return {n: SystemSpec(n, c, mode=m, w_seed=7, workspace_bytes=1 << 30) for n, (c, m) in cells.items()}


def _rel(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _fresh(specs):
    for s in specs.values():
        s.state = None


def test_result_alone_equals_result_in_the_mix(specs):
    from paper_1911_05633_gb300.serve import Server
    _fresh(specs)
    srv = Server(specs, mem_cap_bytes=sum(s.footprint for s in specs.values()) * 2)
    alone = {n: srv.run([(0.0, n)], keep_sigma=True)[0].sigma_k for n in ("c1_cut5", "d16")}
    srv.close()
    _fresh(specs)
    srv = Server(specs, mem_cap_bytes=sum(s.footprint for s in specs.values()) * 2)
    mix = srv.run([(0.0, "c0"), (0.0, "mixed"), (0.0, "c1_cut5"), (0.0, "d16"), (0.001, "c0"), (0.001, "mixed"),
                   (0.002, "c1_cut5")], keep_sigma=True)
    for n in ("c1_cut5", "d16"):
        first = [r for r in mix if r.system == n][0]
        assert _rel(first.sigma_k, alone[n]) <= 1e-14
    # the second iteration starts from the first one's G and chemical potential: it differs
    seconds = [r for r in mix if r.system == "c1_cut5"]
    assert _rel(seconds[1].sigma_k, alone["c1_cut5"]) > 1e-8
    spans = sorted((r.admitted, r.done) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))  # requests overlapped
    srv.close()


def test_memory_cap_binds_on_real_allocations(specs):
    """A cap below the sum of the footprints: systems are evicted and brought back, the
    state survives (the same Sigma as an uninterrupted run), and the driver's count of
    device memory in use stays within the cap of the baseline."""
    import torch
    from paper_1911_05633_gb300.serve import Server
    _fresh(specs)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    baseline = total - free
    # references (and each plan's bytes, measured) from one pass with room for everything
    srv = Server(specs, mem_cap_bytes=sum(s.footprint for s in specs.values()) * 2)
    ref = {n: [r.sigma_k for r in srv.run([(0.0, n), (0.0, n)], keep_sigma=True)] for n in specs}
    srv.close()
    fp = {n: s.footprint for n, s in specs.items()}
    cap = max(fp.values()) + sorted(fp.values())[-2] // 2   # the two largest never resident together
    assert cap < sum(fp.values())
    _fresh(specs)
    srv = Server(specs, mem_cap_bytes=cap)
    order = ["d16", "c1_cut5", "mixed", "c0", "c1_cut5", "d16", "mixed", "c0"]
    reqs = srv.run([(0.002 * i, n) for i, n in enumerate(order)], keep_sigma=True)
    assert any(e[1] == "evict" for e in srv.log)
    # outside the pool the device holds only the plans' tables (measured per system when it
    # was first brought in; at most all of them at once)
    plans = sum(s.plan_bytes for s in specs.values())
    for t, ev, name, resident, used in srv.log:
        assert resident <= cap
        assert used - baseline <= cap + plans + (64 << 20)  # the driver's own count, 64 MiB of slack
    # every buffer of a resident system lies in its range of the pool
    base = srv._dpool.buf.data_ptr()
    for n, sysm in srv.resident.items():
        off, nb = srv.ranges[n]
        for k in ("G_k", "G_R", "P_R", "P_iw", "W_iw", "W_R", "S_R", "Sx_R", "S_iw", "S_k", "Sx_k", "v_R"):
            t = getattr(sysm, k)
            lo = t.data_ptr() - base
            assert off <= lo and lo + t.numel() * t.element_size() <= off + nb, (n, k)
    for n in specs:
        got = [r.sigma_k for r in reqs if r.system == n]
        for a, b in zip(got, ref[n]):
            assert _rel(a, b) <= 1e-14
    srv.close()


def test_chemical_potential_updates_between_iterations(specs):
    from paper_1911_05633_gb300.serve import Server, System
    spec = specs["c0"]
    s = System("c0", spec.cell, mode="iteration")
    mu0 = s.mu
    s.run_request()
    s.finish()
    assert s.mu != mu0
    # the new mu gives the cell's electron count with the new Sigma
    n = s.plan.chemical_potential(s.H_k, float(spec.cell.n_orb_total), s.mu - 1e-6, s.mu + 1e-6, tol=1e-12,
                                  Sigx_k=s.Sx_k, Sig_k_iw=s.S_k)[1]
    assert abs(n - spec.cell.n_orb_total) < 1e-6
    s.close()
