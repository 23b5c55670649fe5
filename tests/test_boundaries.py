"""Static checks of the separation between the product path and the oracle (no GPU): the
package never imports the oracle, and the benchmark loads it in one function only, the one
behind its CPU-baseline leg and reference arm."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _oracle_imports(path):
    """Names of the functions (or '<module>') that import the oracle in a Python file."""
    tree = ast.parse(open(path).read())
    found = []

    def visit(node, where):
        for child in ast.iter_child_nodes(node):
            scope = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else where
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append(where)
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append(where)
            visit(child, scope)
    visit(tree, "<module>")
    return found


def test_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_04070_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                assert _oracle_imports(os.path.join(dirpath, f)) == [], f


def test_benchmark_loads_the_oracle_only_for_the_cpu_baseline():
    assert set(_oracle_imports(os.path.join(ROOT, "bench.py"))) == {"cpu_oracle_sample"}


def test_entry_points_load_the_oracle_only_to_build_and_smoke_check():
    assert set(_oracle_imports(os.path.join(ROOT, "__graft_entry__.py"))) <= {"build", "smoke"}
