"""The persistent batched launch (grmhd_batch_step_persistent): nsteps steps of every
problem of a batch in one cooperative launch, with grid-wide barriers between the
phases, over the same work lists and per-item bodies as the per-kind batched kernels.
For uneven 1-D/2-D/3-D problems including FIXED boundaries and a metric, in FP64 and
mixed precision:
- a problem's state is bitwise the same alone and in the mix, and whether its steps
  run in one launch or one launch each, and the launch is deterministic;
- against grmhd_batch_step it agrees to round-off (the compiler contracts the item
  bodies inlined into the one kernel differently from the per-kind kernels: measured
  <= 1e-14 relative; bound here 1e-12 relative L1);
- a member matches the oracle (1e-10 relative L1).

The barrier waits are bounded: with a wait limit of zero, a block that has to wait
gives up at once, sets the batch's error flag and every block leaves the kernel, which
the call reports as GRMHD_ERR_TIMEOUT -- a wait that runs out by design, with no
fault.  The batch stays usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


def mix_of_problems():
    # uneven sizes, 1-D/2-D/3-D, periodic / outflow / FIXED (charged vortex), flat and
    # metric (random box, star)
    return [P.orszag_tang(48, phase=(0.3, 1.1)), P.random_box(4, 3, [11, 9, 8], bc="outflow", metric=True),
            P.shock_tube(67), P.charged_vortex(24), P.star(n=16), P.orszag_tang(37, eta=1e-2),
            P.random_box(2, 2, [29, 23], bc="periodic")]


def states(S):
    return [t.clone() for t in S.q + S.bf]


def make(G, probs, precision):
    solvers = [G.Solver.from_problem(pr, precision=precision) for pr in probs]
    B = G.Batch(solvers)
    B.set_dt([s.compute_dt() for s in solvers])
    return solvers, B


def rel_l1(a, b):
    return float((a - b).abs().sum() / max(float(b.abs().sum()), 1e-3 * b.numel()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_alone_equals_mix_and_matches_batch_step(G, precision):
    probs = mix_of_problems()
    s1, B1 = make(G, probs, precision)    # per-kind batched step
    s2, B2 = make(G, probs, precision)    # persistent, 3 steps in one launch
    s3, B3 = make(G, probs, precision)    # persistent, one launch per step
    s4, B4 = make(G, probs, precision)    # persistent again (determinism)
    alone = [make(G, [pr], precision) for pr in probs]
    for _ in range(3):
        B1.step()
        B3.step_persistent(1)
    B2.step_persistent(3)
    B4.step_persistent(3)
    for s, B in alone:
        B.step_persistent(3)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        a = alone[i][0][0]
        for w, x, y, z, v in zip(states(a), states(s2[i]), states(s3[i]), states(s4[i]), states(s1[i])):
            assert torch.equal(w, x), (precision, probs[i].name, "alone vs in the mix")
            assert torch.equal(x, y), (precision, probs[i].name, "3 steps in one launch vs one each")
            assert torch.equal(x, z), (precision, probs[i].name, "deterministic")
            assert rel_l1(x, v) <= 1e-12, (precision, probs[i].name, "vs grmhd_batch_step")
        assert s2[i].diagnostics()[2] == 0


def test_persistent_member_matches_oracle(G):
    pr = P.orszag_tang(40)
    other = P.random_box(9, 3, [8, 8, 8], bc="periodic", metric=True)
    st = oracle.from_problem(pr)
    S = G.Solver.from_problem(pr)
    O = G.Solver.from_problem(other)
    B = G.Batch([S, O])
    dt = oracle.cfl_dt(st.grid, pr.cfl)
    B.set_dt([dt, O.compute_dt()])
    for _ in range(3):
        st.step(dt)
    B.step_persistent(3)
    torch.cuda.synchronize()
    I = st.grid.interior()
    for v in range(8):
        a, b = S.q[v].cpu().numpy()[I], st.q[v][I]
        assert np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-3 * b.size) <= 1e-10
    for d in range(3):
        a, b = S.bf[d].cpu().numpy()[I], st.bf[d][I]
        assert np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-3 * b.size) <= 1e-10


def test_persistent_wait_limit_runs_out(G):
    """A zero wait limit makes the first block to reach a barrier give up: the launch
    ends with the error flag set, the call reports GRMHD_ERR_TIMEOUT, and the batch and
    its contexts stay usable (after restoring the state the next steps run and agree
    with an untouched batch)."""
    probs = [P.orszag_tang(64), P.random_box(3, 3, [12, 10, 9], bc="outflow"), P.shock_tube(200)]
    s1, B1 = make(G, probs, "fp64")
    s2, B2 = make(G, probs, "fp64")
    saved = [S.checkpoint() for S in s2]
    B2.set_wait_limit(0.0)
    timed_out = False
    for _ in range(3):   # the first block at a barrier always has to wait (>= 2 blocks)
        st = G.lib().grmhd_batch_step_persistent(B2.b, 2, 1, G._stream(None))
        if st == G.GRMHD_ERR_TIMEOUT:
            timed_out = True
            break
        assert st == 0
    assert timed_out
    assert B2.persistent_status() == G.GRMHD_ERR_TIMEOUT
    assert b"ran out" in G.lib().grmhd_last_error()
    torch.cuda.synchronize()   # no CUDA error: the context is intact
    for S, ck in zip(s2, saved):
        S.restore(ck)
    B2.set_wait_limit(1.0)
    B2.step_persistent(2)
    assert B2.persistent_status() == 0
    B1.step_persistent(2)
    torch.cuda.synchronize()
    for a, b in zip(s1, s2):
        for x, y in zip(states(a), states(b)):
            assert torch.equal(x, y)
    with pytest.raises(G.GrmhdError):
        B2.set_wait_limit(-1.0)


def test_persistent_launch_in_a_cuda_graph(G):
    """The persistent step without synchronisation (a memset and a cooperative launch)
    captured in a CUDA graph and replayed gives the same state as direct launches."""
    probs = [P.orszag_tang(32, phase=(0.1 * i, 0.2 * i)) for i in range(5)] + [P.shock_tube(50)]
    d1, B1 = make(G, probs, "mixed")
    d2, B2 = make(G, probs, "mixed")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            B2.step_persistent(2, synchronize=False, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        B1.step_persistent(2)
        graph.replay()
    torch.cuda.synchronize()
    assert B2.persistent_status() == 0
    for a, b in zip(d1, d2):
        for x, y in zip(states(a), states(b)):
            assert torch.equal(x, y)
