"""The oracle and the CUDA path share no code: the package (Python, CUDA,
C++) never imports, includes or loads anything under oracle/, the oracle
never reaches into the package, the one shared module (the seeded input
descriptions) imports neither, and bench.py touches the oracle only in its
CPU-baseline and reference legs."""
import ast
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
PKG = ROOT / "paper_1606_01805_gb300"
ORACLE = ROOT / "oracle"


def _sources(base, exts):
    return [p for p in base.rglob("*") if p.suffix in exts and "_build" not in p.parts
            and "__pycache__" not in p.parts]


def _imports(path):
    tree = ast.parse(path.read_text())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            out.append(("." * node.level) + (node.module or ""))
    return out


def test_package_never_reaches_the_oracle():
    for p in _sources(PKG, {".py"}):
        assert not any(m.split(".")[0] == "oracle" for m in _imports(p)), p
        assert "lbib_oracle" not in p.read_text(), p
    oracle_api = set(re.findall(r"\b(ob_\w+)\s*\(", (ORACLE / "lbib_oracle.h").read_text()))
    assert oracle_api
    for p in _sources(PKG / "csrc", {".cu", ".cuh", ".h", ".cpp"}):
        txt = p.read_text()
        assert not re.search(r'#include\s+"[^"]*oracle', txt), p
        assert "lbib_oracle" not in txt, p
        assert not oracle_api & set(re.findall(r"\bob_\w+", txt)), p


def test_oracle_never_reaches_the_package():
    for p in _sources(ORACLE, {".py"}):
        assert not any(m.split(".")[0] == "paper_1606_01805_gb300" for m in _imports(p)), p
    for p in _sources(ORACLE, {".c", ".h"}):
        txt = p.read_text()
        for inc in re.findall(r'#include\s+"([^"]+)"', txt):
            assert (ORACLE / inc).exists(), (p, inc)  # only its own headers
        assert "csrc" not in txt and "lbib.h" not in txt.replace("lbib_oracle.h", ""), p


def test_shared_input_module_imports_neither_side():
    mods = _imports(PKG / "workloads.py")
    assert not any(m.split(".")[0] in ("oracle", "paper_1606_01805_gb300") or m.startswith(".")
                   for m in mods), mods


def test_bench_uses_the_oracle_only_in_its_baseline_and_reference_legs():
    tree = ast.parse((ROOT / "bench.py").read_text())
    allowed = {"cpu_oracle_rates", "main", "main_screening"}
    parents = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    for node in ast.walk(tree):
        if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
            fn, up = None, node
            while up in parents:
                up = parents[up]
                if isinstance(up, ast.FunctionDef):
                    fn = up
                    break
            assert fn is not None and fn.name in allowed, ast.dump(node)
            if fn.name != "cpu_oracle_rates":
                # inside main / main_screening: only under `if args.impl == "reference"`
                up, guarded = node, False
                while up in parents and up is not fn:
                    up = parents[up]
                    if isinstance(up, ast.If) and "reference" in ast.unparse(up.test):
                        guarded = True
                assert guarded, f"oracle import in {fn.name} outside the reference leg"
