"""The Python binding has no CPU fallback: with libgrmhd.so absent, loading the
library and building a solver raise GrmhdError rather than computing anything."""
import pytest


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2110_03732_gb300 import build as _build
    from paper_2110_03732_gb300 import grmhd
    from paper_2110_03732_gb300 import problems as P
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libgrmhd.so"))
    monkeypatch.setattr(grmhd, "_lib", None)
    with pytest.raises(grmhd.GrmhdError):
        grmhd.lib()
    with pytest.raises(grmhd.GrmhdError):
        grmhd.Solver.from_problem(P.orszag_tang(16), device="cpu")


def test_binding_imports_no_oracle():
    """The product package never imports the oracle (test infrastructure only)."""
    import os
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2110_03732_gb300")
    for dirpath, _, files in os.walk(root):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


class _FakeLib:
    """Stands in for libgrmhd.so: records the pointers each call receives."""

    def __init__(self):
        import ctypes as C
        self.C = C
        self.calls = {}

    def __getattr__(self, name):
        if not name.startswith("grmhd_"):
            raise AttributeError(name)

        def call(*args):
            self.calls.setdefault(name, []).append(args)
            if name == "grmhd_scratch_bytes":
                args[2]._obj.value = 256
            elif name == "grmhd_create":
                args[3]._obj.value = 1
            elif name == "grmhd_last_error":
                return b""
            return 0
        return call


def _addr(p, i):
    v = p[i]
    return 0 if v is None else int(v)


def test_binding_passes_arrays_through_unchanged(monkeypatch):
    """The binding only marshals: on a GLM problem with a metric every array that
    reaches the library is the problem's own data, bitwise, at the address the call
    receives.  In particular the primitive Phi goes in as prim[8] and is not
    densitised in Python (the library forms q_Phi = psi^6 Phi)."""
    import numpy as np
    import torch
    from paper_2110_03732_gb300 import grmhd
    from paper_2110_03732_gb300 import problems as P
    import contextlib
    import ctypes as C
    fake = _FakeLib()
    monkeypatch.setattr(grmhd, "_lib", fake)
    # no CUDA device here: the device context and the stream handle are placeholders
    monkeypatch.setattr(grmhd.torch.cuda, "device", lambda dev: contextlib.nullcontext())
    monkeypatch.setattr(grmhd, "_stream", lambda stream: C.c_void_p(None))
    pr = P.random_box(4, 2, [10, 8], bc="outflow", metric=True, glm=True)
    assert pr.phi is not None and pr.psi is not None and np.abs(pr.psi - 1).max() > 1e-3
    S = grmhd.Solver.from_problem(pr, device="cpu", divb="glm")
    tensors = {}
    for t in list(S._keep[0]) + list(S._keep[1] or []) + [S.alpha, S.psi, S.eta] + list(S.bf) + list(S.q):
        if t is not None:
            tensors[t.data_ptr()] = t
    (ctx, pp, pa, stream), = fake.calls["grmhd_init_from_prims"]
    want = list(pr.prim) + [pr.phi]
    for v in range(9):
        t = tensors[_addr(pp, v)]
        assert torch.equal(t, torch.as_tensor(want[v])), v
    assert pr.A_cell is None and pa is None   # the cell fields are given directly
    for d in range(3):
        assert torch.equal(S.bf[d], torch.as_tensor(pr.bcell[d]))
    (ctx, a, p), = fake.calls["grmhd_set_metric"]
    assert torch.equal(tensors[a.value], torch.as_tensor(pr.alpha))
    assert torch.equal(tensors[p.value], torch.as_tensor(pr.psi))
    (ctx, pq, pb, scratch, nbytes), = fake.calls["grmhd_bind"]
    for v in range(8):
        assert _addr(pq, v) == S.q[v].data_ptr()
    for d in range(3):
        assert _addr(pb, d) == S.bf[d].data_ptr()
    (ctx, qphi), = fake.calls["grmhd_bind_phi"]
    assert qphi.value == S.phi.data_ptr()
