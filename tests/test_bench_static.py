"""bench.py is only executed in full on a GPU; this catches names it uses before defining them."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _undefined(fn, module_names):
    known = set(dir(builtins)) | module_names
    known.update(a.arg for a in fn.args.args + fn.args.kwonlyargs)
    for node in ast.walk(fn):
        if isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
            known.add(node.id)
        elif isinstance(node, (ast.FunctionDef, ast.Lambda)):
            if isinstance(node, ast.FunctionDef):
                known.add(node.name)
            known.update(a.arg for a in node.args.args + node.args.kwonlyargs)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            known.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            known.add(node.name)
    used = {n.id for n in ast.walk(fn) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    return sorted(used - known)


def test_bench_functions_use_only_defined_names():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    module_names = set()
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            module_names.add(node.name)
        elif isinstance(node, ast.Assign):
            module_names.update(t.id for t in node.targets if isinstance(t, ast.Name))
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            module_names.update((a.asname or a.name).split(".")[0] for a in node.names)
    bad = {fn.name: _undefined(fn, module_names) for fn in tree.body if isinstance(fn, ast.FunctionDef)}
    bad = {k: v for k, v in bad.items() if v}
    assert not bad, bad
