"""Checkpoint / resume: a run stopped after some steps, saved (state, face fields and
the context's Newton start blob) and resumed in a fresh context continues bitwise as
the uninterrupted run, for FP64, mixed precision and GLM.  Without the start blob the
resumed run still agrees to the Newton tolerance (the roots do not depend on the start),
but not bitwise."""
import pytest

from paper_2110_03732_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


def fields(S):
    out = [t.clone() for t in S.q + S.bf]
    if S.phi is not None:
        out.append(S.phi.clone())
    return out


@pytest.mark.parametrize("kw", [{}, {"precision": "mixed"}, {"divb": "glm"}], ids=["fp64", "mixed", "glm"])
def test_resume_is_bitwise(G, kw):
    pr = P.orszag_tang(64, kappa=1.0) if kw.get("divb") == "glm" else P.orszag_tang(64)
    A = G.Solver.from_problem(pr, **kw)
    dt = A.compute_dt()
    for _ in range(5):
        A.step(dt)
    ck = A.checkpoint()
    for _ in range(5):
        A.step(dt)
    torch.cuda.synchronize()
    want = fields(A)
    B = G.Solver.from_problem(pr, **kw)
    B.restore(ck)
    for _ in range(5):
        B.step(dt)
    torch.cuda.synchronize()
    for x, y in zip(fields(B), want):
        assert torch.equal(x, y)


def test_resume_without_start_agrees_to_tolerance(G):
    pr = P.orszag_tang(64)
    A = G.Solver.from_problem(pr)
    dt = A.compute_dt()
    for _ in range(5):
        A.step(dt)
    ck = A.checkpoint()
    for _ in range(3):
        A.step(dt)
    B = G.Solver.from_problem(pr)
    for t, s in zip(B.q, ck["q"]):
        t.copy_(s)
    for t, s in zip(B.bf, ck["bf"]):
        t.copy_(s)
    for _ in range(3):
        B.step(dt)
    torch.cuda.synchronize()
    for x, y in zip(fields(B), fields(A)):
        den = max(float(y.abs().sum()), 1e-30)
        assert float((x - y).abs().sum()) / den <= 1e-10


def test_start_blob_of_another_grid_is_refused(G):
    A = G.Solver.from_problem(P.orszag_tang(32))
    B = G.Solver.from_problem(P.orszag_tang(48))
    ck = A.checkpoint()
    with pytest.raises(G.GrmhdError):
        B.restore(ck)
