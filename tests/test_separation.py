"""The oracle and the CUDA path share no code, and the product never calls the
oracle: only the tests, smoke() and bench.py's CPU-baseline and reference
legs import it."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1908_00587_gb300"


def _imports(path):
    """(module, enclosing function name or None) for every import in a file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = ch.name if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(ch, ast.Import):
                out.extend((a.name, fn) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom):
                out.append(((ch.module or "") if ch.level == 0 else "." + (ch.module or ""), fn))
            visit(ch, f)

    visit(tree, None)
    return out


def _py_files(d):
    for dp, _, fs in os.walk(os.path.join(ROOT, d)):
        for f in fs:
            if f.endswith(".py"):
                yield os.path.join(dp, f)


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_oracle_imports_nothing_of_the_package():
    for path in _py_files("oracle"):
        for mod, _ in _imports(path):
            assert PKG not in mod and not mod.startswith("inputs"), (path, mod)
        src = open(path).read()
        assert "libtc" not in src and "csrc" not in src, path


def test_cuda_sources_do_not_reach_the_oracle():
    csrc = os.path.join(ROOT, PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f)).read()
        assert "oracle" not in src.lower(), f


def test_entry_points_call_the_oracle_only_where_allowed():
    allowed = {"bench.py": {"oracle_throughput"}, "__graft_entry__.py": {"smoke"}}
    for name, fns in allowed.items():
        for mod, fn in _imports(os.path.join(ROOT, name)):
            if mod.split(".")[0] == "oracle":
                assert fn in fns, (name, fn)


def test_input_generators_hold_no_method_arithmetic():
    """The seeded inputs module serves both sides; it imports neither."""
    for path in _py_files("inputs"):
        for mod, _ in _imports(path):
            root = mod.split(".")[0]
            assert root not in ("oracle", PKG), (path, mod)
