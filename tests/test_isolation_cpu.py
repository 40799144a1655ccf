"""The oracle and the CUDA path share no code: static checks over the
sources (no GPU).

- No module of the package imports the oracle, and the oracle imports nothing
  of the package, of the benchmark or of the entry module.
- synth (the seeded inputs both sides take) imports neither side.
- bench.py imports the oracle only inside the functions of its CPU leg and
  reference arm; __graft_entry__ only inside smoke().
- The CUDA sources include only files of their own csrc/ folder (quoted
  includes) besides the toolkit's headers."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2506_08308_gb300")


def _py_files(folder):
    for dirpath, _, names in os.walk(folder):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for n in names:
            if n.endswith(".py"):
                yield os.path.join(dirpath, n)


def _imports(path):
    """(module name, enclosing function names) of every import in a file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def walk(node, stack):
        for ch in ast.iter_child_nodes(node):
            st = stack + [ch.name] if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else stack
            if isinstance(ch, ast.ImportFrom) and ch.level == 0:
                out.append((ch.module or "", tuple(st)))
            elif isinstance(ch, ast.Import):
                out.extend((a.name, tuple(st)) for a in ch.names)
            walk(ch, st)
    walk(tree, [])
    return out


def _top(name):
    return name.split(".")[0]


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert _top(mod) != "oracle", (path, mod)


def test_oracle_imports_nothing_of_the_cuda_side():
    banned = {"paper_2506_08308_gb300", "bench", "__graft_entry__", "torch", "ctypes"}
    for path in _py_files(os.path.join(ROOT, "oracle")):
        for mod, _ in _imports(path):
            assert _top(mod) not in banned, (path, mod)


def test_synth_imports_neither_side():
    for mod, _ in _imports(os.path.join(ROOT, "synth.py")):
        assert _top(mod) not in {"oracle", "paper_2506_08308_gb300", "torch"}, mod


def test_bench_and_entry_import_the_oracle_only_in_their_cpu_legs():
    allowed = {"oracle_instance", "cpu_oracle_sample"}
    for mod, stack in _imports(os.path.join(ROOT, "bench.py")):
        if _top(mod) == "oracle":
            assert stack and stack[0] in allowed, (mod, stack)
    for mod, stack in _imports(os.path.join(ROOT, "__graft_entry__.py")):
        if _top(mod) == "oracle":
            assert stack and stack[0] == "smoke", (mod, stack)


def test_cuda_sources_include_only_their_own_headers():
    csrc = os.path.join(PKG, "csrc")
    own = set(os.listdir(csrc))
    for n in sorted(own):
        if not n.endswith((".cu", ".cuh", ".h")):
            continue
        for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', open(os.path.join(csrc, n)).read(), flags=re.M):
            assert inc in own or inc == "../../include/bdg.h" or os.path.basename(inc) == "bdg.h", (n, inc)
