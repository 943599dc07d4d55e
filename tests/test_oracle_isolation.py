"""The oracle is test infrastructure: nothing in the library package imports
it, bench.py imports it only in its CPU-baseline sampler, __graft_entry__ only
in smoke(); and the oracle imports nothing from the library."""

import ast
import glob
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    """(module name, enclosing function or None) of every import in a file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append(((child.module or "") if child.level == 0 else "." * child.level + (child.module or ""), f))
            visit(child, f)

    visit(tree, None)
    return out


def test_library_never_imports_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "paper_1202_2462_gb300", "**", "*.py"), recursive=True):
        for mod, _ in _imports(path):
            assert not mod.startswith("oracle"), (path, mod)


def test_bench_and_entry_import_the_oracle_only_where_allowed():
    allowed = {"bench.py": {"_oracle_worker", "_oracle_kernel_worker", "oracle_study"}, "__graft_entry__.py": {"smoke"}}
    for name, funcs in allowed.items():
        for mod, func in _imports(os.path.join(ROOT, name)):
            if mod.startswith("oracle"):
                assert func in funcs, (name, mod, func)


def test_oracle_does_not_import_the_library():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for mod, _ in _imports(path):
            assert "paper_1202_2462_gb300" not in mod and "torch" not in mod, (path, mod)
