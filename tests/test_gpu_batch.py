"""Batched systems of uneven sizes (gw_batch_*): the GW_MIXED P and Sigma contractions of
several plans in one persistent launch each.  Each system's result is bit for bit the
same alone and in the batch (the per-unit arithmetic does not depend on the batch), within
1e-6 of the FP64 oracle, unchanged after the autotuner picks its launch configuration, and
unchanged when the launches are replayed from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
from test_gpu_parity import _random_W, dev, host, pack, rel, system

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6
NAMES = ["c0", "mixed", "c1_cut5_far", "mixed_far", "mixed_nonsym"]


def _batch(names):
    from paper_1911_05633_gb300 import gw
    ss = [system(n) for n in names]
    return ss, gw.Batch([s.plan for s in ss])


def _inputs(ss):
    G = [dev(pack(s.G_R())) for s in ss]
    W = [dev(pack(_random_W(s))) for s in ss]
    return G, W


def test_batch_equals_alone_and_oracle():
    ss, b = _batch(NAMES)
    G, W = _inputs(ss)
    P = b.polarizability_tau(G)
    S = b.self_energy_tau(G, W)
    b.sync()
    for s, g, w, p, sg in zip(ss, G, W, P, S):
        p_alone = s.plan.polarizability_tau(g, precision="mixed")
        s_alone = s.plan.self_energy_tau(g, w, precision="mixed")
        s.plan.sync()
        assert np.array_equal(host(p), host(p_alone))
        assert np.array_equal(host(sg), host(s_alone))
        refP = oracle.polarizability_R(s.G_R(), s.orc.entries, s.orc.C_atom, s.cell.spin, s.orc.kdims)
        assert rel(host(p), pack(refP)) < TOL_MIXED
        refS = oracle.self_energy_R(s.G_R(), _random_W(s), s.orc.entries, s.orc.C_atom)
        assert rel(host(sg), pack(refS)) < TOL_MIXED
    b.close()


def test_batch_autotuner_and_graph_replay():
    import torch
    ss, b = _batch(NAMES)
    G, W = _inputs(ss)
    P0 = [t.clone() for t in b.polarizability_tau(G)]
    S0 = [t.clone() for t in b.self_energy_tau(G, W)]
    b.sync()
    P = [torch.empty_like(t) for t in P0]
    S = [torch.empty_like(t) for t in S0]
    info = b.tune(G, P, W, S, reps=2)
    assert info["tuned"] == 1 and info["groups_p"] in (1, 2) and info["order_p"] in (0, 1)
    assert 1 <= info["n_classes"] <= len(NAMES)
    for x in P + S:
        x.zero_()
    stream = torch.cuda.Stream()
    b.polarizability_tau(G, P, stream=stream.cuda_stream)  # warm-up on the capture stream
    b.self_energy_tau(G, W, S, stream=stream.cuda_stream)
    b.sync(stream=stream.cuda_stream)
    for x in P + S:
        x.zero_()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.polarizability_tau(G, P, stream=stream.cuda_stream)
        b.self_energy_tau(G, W, S, stream=stream.cuda_stream)
    graph.replay()
    torch.cuda.synchronize()
    b.sync()
    for a, c in zip(P + S, P0 + S0):
        assert torch.equal(a, c)
    b.close()
