"""The oracle and the CUDA path share nothing: no module of either imports the other, the
oracle never loads the library, and the product package neither imports nor runs anything
under oracle/ (the seeded input generators live in their own module, synth.py, which holds
none of the method's arithmetic).  Static checks of the sources; no GPU."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            out.add(node.module.split(".")[0])
    return out


def test_oracle_imports_nothing_of_the_package():
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        imps = _imports(p)
        assert "paper_2010_06697_gb300" not in imps, p
        assert not ({"ctypes", "torch"} & imps), p
        assert "librve" not in open(p).read(), p


def test_package_never_touches_the_oracle():
    for p in glob.glob(os.path.join(ROOT, "paper_2010_06697_gb300", "*.py")):
        assert "oracle" not in _imports(p), p
        src = open(p).read()
        # no dynamic import or path into the oracle either
        assert not re.search(r"import_module\(\s*['\"]oracle|['\"]oracle[/'\"]", src), p
    for p in glob.glob(os.path.join(ROOT, "paper_2010_06697_gb300", "csrc", "*")):
        src = open(p, errors="replace").read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), p
        assert not re.search(r"\"[^\"\n]*oracle/", src), p


def test_input_generators_hold_no_solver_arithmetic():
    """synth.py draws seeded numbers and builds geometries; it must not import the
    oracle, the library binding or an FFT."""
    p = os.path.join(ROOT, "paper_2010_06697_gb300", "synth.py")
    imps = _imports(p)
    assert imps <= {"numpy", "__future__"}, imps
    # the one FFT use is the periodic Gaussian smoothing of the director field (its recipe)
    tree = ast.parse(open(p).read())
    for fn in [n for n in tree.body if isinstance(n, ast.FunctionDef)]:
        uses_fft = any(isinstance(n, ast.Attribute) and n.attr == "fft" for n in ast.walk(fn))
        assert not uses_fft or fn.name == "director_grf", fn.name
