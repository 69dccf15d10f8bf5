"""The oracle and the CUDA path share no code (the parity tests compare two
independent implementations):

* nothing in the package (Python or CUDA/C++ sources) imports, includes or
  names the oracle, and nothing in the oracle imports the package;
* outside ``tests/``, only ``bench.py`` (its CPU-baseline / reference leg,
  ``oracle_solves_per_s``) and ``__graft_entry__.smoke()`` import the oracle,
  inside those functions, so importing either module does not load it;
* the product path imports no CPU fallback: loading the binding loads the
  compiled library and no oracle module;
* no Python source names an absolute path other than the CUDA toolkit's."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2604_15796_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _imports(path):
    """(module, enclosing top-level function or None) for every import."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = fn
            if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None:
                f = ch.name
            if isinstance(ch, ast.Import):
                out.extend((a.name, f) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom) and ch.level == 0 and ch.module:
                out.append((ch.module, f))
            visit(ch, f)
    visit(tree, None)
    return out


def _top(mod):
    return mod.split(".")[0]


def test_package_does_not_use_the_oracle():
    for p in _files(PKG, (".py",)):
        for mod, _ in _imports(p):
            assert _top(mod) != "oracle", (p, mod)
    for p in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        text = open(p).read()
        assert "oracle" not in text.lower(), p


def test_oracle_does_not_use_the_package():
    for p in _files(ORACLE, (".py",)):
        for mod, _ in _imports(p):
            assert _top(mod) not in ("paper_2604_15796_gb300", "torch", "bench"), (p, mod)


def test_only_the_sanctioned_entry_points_import_the_oracle():
    allowed = {"bench.py": {"oracle_solves_per_s"}, "__graft_entry__.py": {"smoke"}}
    for name in os.listdir(ROOT):
        if not name.endswith(".py"):
            continue
        for mod, fn in _imports(os.path.join(ROOT, name)):
            if _top(mod) == "oracle":
                assert fn in allowed.get(name, set()), (name, mod, fn)


def test_importing_the_binding_bench_and_entry_loads_no_oracle():
    code = ("import sys; import paper_2604_15796_gb300.libfwi, bench, __graft_entry__; "
            "print(sorted(m for m in sys.modules if m.split('.')[0] == 'oracle'))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         check=True).stdout.strip().splitlines()[-1]
    assert out == "[]", out


def test_no_absolute_paths_but_the_toolkit():
    """Every absolute path a Python source names is the CUDA toolkit's: the
    tests, the bench and the library read their inputs from the repository
    (and the autotune cache from the user's cache directory)."""
    roots = [PKG, ORACLE, os.path.join(ROOT, "tests")]
    files = [p for r in roots for p in _files(r, (".py",))]
    files += [os.path.join(ROOT, n) for n in ("bench.py", "__graft_entry__.py")]
    allowed = ("/usr/local/cuda",)
    for p in files:
        for node in ast.walk(ast.parse(open(p).read(), p)):
            v = getattr(node, "value", None)
            if isinstance(node, ast.Constant) and isinstance(v, str) and v.startswith("/") \
                    and len(v) > 1 and " " not in v and "\n" not in v:
                assert v.startswith(allowed), (p, v)
