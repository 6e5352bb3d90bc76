"""The request loop (paper_1911_05633_gb300.serve): a system's result is the same alone
and in a mix with other systems running concurrently, the state advances per
iteration, and the memory cap bounds what runs at once."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def systems():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_05633_gb300.serve import System
    cells = {"c0": synth.make_config(0), "mixed": synth.mixed_species_cell(),
             "c1_cut5": synth.make_config(1, cutoff=5.0, n_tau=12, kmesh=(2, 2, 2))}
    out = {n: System(n, c) for n, c in cells.items()}
    yield out
    for s in out.values():
        s.close()


def _rel(a, b):
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_result_alone_equals_result_in_the_mix(systems):
    from paper_1911_05633_gb300.serve import Server
    server = Server(systems, mem_cap_bytes=sum(s.footprint for s in systems.values()))
    for s in systems.values():
        s.reset()
    alone = server.run([(0.0, "c1_cut5")], keep_sigma=True)[0].sigma_k
    for s in systems.values():
        s.reset()
    mix = server.run([(0.0, "c0"), (0.0, "mixed"), (0.0, "c1_cut5"), (0.0, "c0"), (0.001, "mixed"),
                      (0.002, "c1_cut5")], keep_sigma=True)
    firsts = [r for r in mix if r.system == "c1_cut5"]
    assert _rel(firsts[0].sigma_k, alone) <= 1e-14
    # the second iteration of the same system starts from the first one's G: it differs
    assert _rel(firsts[1].sigma_k, alone) > 1e-8
    # requests of different systems overlapped on the device
    spans = sorted((r.admitted, r.done) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    assert all(r.done is not None and r.done >= r.admitted >= r.arrival - 1e-9 for r in mix)


def test_memory_cap_bounds_what_runs_at_once(systems):
    """A cap equal to the largest system's footprint: that system never runs beside
    another, and the footprints of the requests running at any moment fit the cap."""
    from paper_1911_05633_gb300.serve import Server
    cap = max(s.footprint for s in systems.values())
    big = max(systems, key=lambda n: systems[n].footprint)
    server = Server(systems, mem_cap_bytes=cap)
    for s in systems.values():
        s.reset()
    reqs = server.run([(0.0, n) for n in ("c0", "mixed", "c1_cut5", "c0", "mixed", "c1_cut5")])
    # footprint only grows at admissions: at each one, what runs then fits the cap
    for r in reqs:
        t = r.admitted
        running = [q for q in reqs if q.admitted <= t < q.done]
        assert sum(systems[q.system].footprint for q in running) <= cap
        if r.system == big:
            assert not [q for q in reqs if q is not r and q.admitted < r.done and r.admitted < q.done]
