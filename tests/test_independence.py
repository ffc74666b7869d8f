"""The oracle and the CUDA path share no code, and only the permitted places run the oracle.

Static checks over the sources (CPU): nothing under ``oracle/`` imports the package or reads its
CUDA sources; nothing in the package (Python or CUDA) refers to ``oracle``; the seeded input
generators (``workloads/``) import neither side; ``bench.py`` imports the oracle only inside its
CPU-baseline function; ``__graft_entry__`` only inside ``smoke()``."""
import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    """(module, enclosing top-level function or None) for every import in a Python file."""
    tree = ast.parse(open(path).read())
    out = []
    for top in tree.body:
        fn = top.name if isinstance(top, (ast.FunctionDef, ast.AsyncFunctionDef)) else None
        for node in ast.walk(top):
            if isinstance(node, ast.Import):
                out += [(a.name, fn) for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mod = ("." * node.level) + (node.module or "")
                out.append((mod, fn))
    return out


def _roots(mods):
    return {m.lstrip(".").split(".")[0] for m, _ in mods if m}


def test_oracle_does_not_touch_the_cuda_path():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_2405_16076_gb300" not in _roots(_imports(f)), f
        assert "csrc" not in open(f).read(), f


def test_package_does_not_use_the_oracle():
    for f in glob.glob(os.path.join(ROOT, "paper_2405_16076_gb300", "*.py")):
        assert "oracle" not in _roots(_imports(f)), f
    for f in glob.glob(os.path.join(ROOT, "paper_2405_16076_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read().lower(), f
    for f in glob.glob(os.path.join(ROOT, "include", "*.h")):
        assert "oracle" not in open(f).read().lower(), f


def test_input_generators_import_neither_side():
    for f in glob.glob(os.path.join(ROOT, "workloads", "*.py")):
        assert not ({"oracle", "paper_2405_16076_gb300"} & _roots(_imports(f))), f


def test_oracle_runs_only_in_the_permitted_places():
    bench = [(m, fn) for m, fn in _imports(os.path.join(ROOT, "bench.py")) if m.split(".")[0] == "oracle"]
    assert bench and all(fn == "cpu_baseline" for _, fn in bench), bench
    entry = [(m, fn) for m, fn in _imports(os.path.join(ROOT, "__graft_entry__.py")) if m.split(".")[0] == "oracle"]
    assert entry and all(fn == "smoke" for _, fn in entry), entry
