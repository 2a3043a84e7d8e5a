"""The oracle and the CUDA path share nothing, checked on the sources.

* oracle/ imports only the standard library, numpy and its own modules:
  nothing of the product package, no ctypes, no torch;
* the product package (paper_1812_00118_gb300/) never imports the oracle,
  and its CUDA sources include nothing from oracle/;
* the scripts that write stored expected values (tests/golden/) call only
  the oracle and the seeded input recipe;
* the recipe module (inputs.py) holds no model arithmetic: it imports
  nothing but numpy;
* bench.py and __graft_entry__.py import the oracle only inside the
  functions allowed to run it (the CPU baseline worker and smoke()).
"""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1812_00118_gb300")


def _imports(path):
    """(module, enclosing function or None) of every import in a file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name, func) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = ("." * child.level) + (child.module or "")
                out.append((mod, func))
            visit(child, f)

    visit(tree, None)
    return out


def _py(dirpath):
    for base, _, files in os.walk(dirpath):
        if "__pycache__" in base or "_build" in base or "_lib" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


STDLIB_OK = {"dataclasses", "typing", "itertools", "math", "os", "sys", "importlib", "importlib.util"}


def test_oracle_imports_only_numpy_and_itself():
    for path in _py(os.path.join(ROOT, "oracle")):
        for mod, _ in _imports(path):
            top = mod.split(".")[0]
            assert mod.startswith(".") or top in {"numpy", "oracle"} or mod in STDLIB_OK, (path, mod)


def test_product_never_touches_the_oracle():
    for path in _py(PKG):
        for mod, _ in _imports(path):
            assert mod.split(".")[0] != "oracle", (path, mod)
    for base, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            for line in open(os.path.join(base, f), errors="replace"):
                if line.lstrip().startswith("#include"):
                    assert "oracle" not in line, (f, line)      # no header or table from oracle/
            assert "oracle/" not in open(os.path.join(base, f), errors="replace").read(), f


def test_stored_values_come_from_the_oracle_only():
    for path in _py(os.path.join(ROOT, "tests", "golden")):
        for mod, _ in _imports(path):
            top = mod.split(".")[0]
            assert top in {"os", "sys", "numpy", "oracle"} or mod == "paper_1812_00118_gb300", (path, mod)
            if mod == "paper_1812_00118_gb300":
                text = open(path).read()
                assert "from paper_1812_00118_gb300 import inputs" in text
                assert "import lbm" not in text and "surrogate" not in text


def test_input_recipe_holds_no_model_arithmetic():
    mods = {m for m, _ in _imports(os.path.join(PKG, "inputs.py"))}
    assert mods == {"numpy"}


def test_oracle_runs_only_where_allowed():
    allowed = {"bench.py": {"_oracle_sample"}, "__graft_entry__.py": {"smoke"}}
    for name, funcs in allowed.items():
        for mod, func in _imports(os.path.join(ROOT, name)):
            if mod.split(".")[0] == "oracle":
                assert func in funcs, (name, mod, func)


def test_nothing_committed_uses_the_working_folder():
    """No source, test or script reads, imports or runs anything under the
    git-ignored working folder."""
    work = "_" + "work/"
    for base, dirs, files in os.walk(ROOT):
        dirs[:] = [d for d in dirs if d not in {".git", "_work", "gpurun_out", "__pycache__", "_build",
                                                "_build_checked", "_lib", "baseline"}]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".sh", ".ini", ".toml", ".cfg")):
                path = os.path.join(base, f)
                assert work not in open(path, errors="replace").read(), path
