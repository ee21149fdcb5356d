"""The oracle is test infrastructure: the library package never imports or
links it, and bench.py runs it only in its CPU-baseline leg and its reference
arm (``--impl reference``); ``__graft_entry__`` builds it and uses it in the
smoke check only."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1210_2536_gb300")


def _functions_using_oracle(path):
    """Names of the top-level functions whose bodies mention `oracle`, and
    whether it is mentioned at module level."""
    tree = ast.parse(open(path).read())
    users, top = set(), False
    for node in tree.body:
        hit = any((isinstance(n, ast.Name) and n.id == "oracle") or
                  (isinstance(n, ast.alias) and n.name.split(".")[0] == "oracle") or
                  (isinstance(n, ast.ImportFrom) and (n.module or "").split(".")[0] == "oracle")
                  for n in ast.walk(node))
        if hit and isinstance(node, ast.FunctionDef):
            users.add(node.name)
        elif hit:
            top = True
    return users, top


def test_package_never_imports_or_links_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                users, top = _functions_using_oracle(path)
                assert not users and not top, (path, users)
            if f.endswith((".cu", ".cuh", ".h", ".c")) or f == "_build.py":
                src = open(path, errors="replace").read()
                assert "liboracle" not in src and "oracle.h" not in src and "oracle_" not in src, path


def _callers(path, name):
    """Top-level functions whose bodies call `name`."""
    tree = ast.parse(open(path).read())
    return {node.name for node in tree.body if isinstance(node, ast.FunctionDef)
            and any(isinstance(n, ast.Call) and isinstance(n.func, ast.Name) and n.func.id == name
                    for n in ast.walk(node))}


def test_bench_runs_the_oracle_only_in_its_baseline_and_reference_arms():
    path = os.path.join(ROOT, "bench.py")
    users, top = _functions_using_oracle(path)
    assert not top
    assert users <= {"cpu_baseline", "run_reference", "reference_specs"}, users
    # the reference arm's input builder serves the reference arm alone
    assert _callers(path, "reference_specs") <= {"run_reference"}


def test_graft_entry_uses_the_oracle_only_to_build_it_and_in_smoke():
    users, top = _functions_using_oracle(os.path.join(ROOT, "__graft_entry__.py"))
    assert not top and users <= {"build", "smoke"}, users
