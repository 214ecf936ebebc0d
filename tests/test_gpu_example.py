"""The usage example of the package docstring runs as written."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_package_docstring_example_runs(capsys):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2312_02968_gb300 as pkg

    doc = pkg.__doc__
    start = doc.index("::\n") + 3
    end = doc.index("\nModules:")
    lines = [ln[4:] if ln.startswith("    ") else ln for ln in doc[start:end].splitlines()]
    exec(compile("\n".join(lines), "package-docstring-example", "exec"), {})
    out = capsys.readouterr().out.split()
    e_kin = float(out[0])
    assert 0.3 < e_kin < 0.37  # sqrt(G M a0)/3 for the isothermal sphere (Sect. 4.3)
