"""adscl_evolve as a CUDA graph: replaying the cached graph (updated in place as t_end changes)
gives the same bits as direct launches, in batched and one-per-launch mode; with device outputs
the call can be captured into the caller's own graph."""
import numpy as np
import pytest

from paper_1706_07413_b300 import workloads as W

pytestmark = pytest.mark.gpu

NS = [4097, 2049, 8193, 1025, 129, 4097, 8193, 513]


@pytest.fixture(scope="module")
def ad():
    from paper_1706_07413_b300 import adscl
    adscl.load()
    return adscl


def _fields(Ns, seed=11):
    f = [W.smooth_random(n, seed=seed + i, amp=2.0) for i, n in enumerate(Ns)]
    return W.packed([x[0] for x in f]), W.packed([x[1] for x in f])


def _run(ad, Ns, t_ends, **kw):
    Phi, Pi = _fields(Ns)
    s = ad.Solver(Ns, chunk_steps=5, **kw)
    s.set_initial(Phi, Pi)
    outs = [s.evolve(t) for t in t_ends]
    states = [s.get_state(b) for b in range(len(Ns))]
    s.close()
    return outs, states


def _same(r1, r2):
    for o1, o2 in zip(r1[0], r2[0]):
        for x, y in zip(o1, o2):
            assert np.array_equal(x, y)
    for s1, s2 in zip(r1[1], r2[1]):
        for x, y in zip(s1, s2):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("one_per_launch", [False, True])
def test_graph_replay_equals_direct_launches(ad, one_per_launch):
    t_ends = (0.004, 0.011, 0.011, 0.03)   # t_end changes between calls: in-place graph update
    g = _run(ad, NS, t_ends, one_per_launch=one_per_launch)
    d = _run(ad, NS, t_ends, one_per_launch=one_per_launch, direct_launch=True)
    _same(g, d)


def test_graph_increments_equal_one_call(ad):
    g = _run(ad, NS, (0.004, 0.011, 0.02, 0.03))
    one = _run(ad, NS, (0.03,))
    _same(([g[0][-1]], g[1]), one)


def test_evolve_captured_into_caller_graph(ad):
    import torch
    B = len(NS)
    Phi, Pi = _fields(NS)
    st = torch.cuda.Stream()
    s = ad.Solver(NS, chunk_steps=5, stream=st.cuda_stream)
    s.set_initial(Phi, Pi)
    dev = torch.device("cuda", 0)
    outs = (torch.empty(B, dtype=torch.float64, device=dev), torch.empty(B, dtype=torch.float64, device=dev),
            torch.empty(B, dtype=torch.float64, device=dev), torch.empty(B, dtype=torch.int32, device=dev))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        s.evolve(0.03, out=outs)
    clk = s.clock()[1]
    assert (clk == 0).all()          # capture records the work without running it
    g.replay()
    torch.cuda.synchronize()
    ref = _run(ad, NS, (0.03,))
    for x, y in zip(outs, ref[0][0]):
        assert np.array_equal(x.cpu().numpy(), y)
    for b in range(B):
        for x, y in zip(s.get_state(b), ref[1][b]):
            assert np.array_equal(x, y)
    g.replay()                       # the same t_end again: nothing left to do
    torch.cuda.synchronize()
    for x, y in zip(outs, ref[0][0]):
        assert np.array_equal(x.cpu().numpy(), y)
    del g
    s.close()
