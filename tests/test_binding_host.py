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
