"""Static check of the Python sources (CPU): every module compiles, and every
name a module reads is bound somewhere in it (an assignment, argument,
import, definition or builtin).  It catches a renamed variable left behind on
a path no CPU test executes, such as the GPU-only experiment drivers."""
import ast
import builtins
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources():
    out = [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    for d in ("paper_2509_25044_gb300", "oracle", "tests"):
        for f in sorted(os.listdir(os.path.join(ROOT, d))):
            if f.endswith(".py"):
                out.append(os.path.join(ROOT, d, f))
    return out


def _bound(tree):
    names = set(dir(builtins)) | {"__file__", "__name__"}
    for n in ast.walk(tree):
        if isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            names.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            names.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            names.add(n.id)
        elif isinstance(n, ast.arg):
            names.add(n.arg)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            names.update(n.names)
        elif isinstance(n, ast.ExceptHandler) and n.name:
            names.add(n.name)
        elif isinstance(n, ast.MatchAs) and n.name:
            names.add(n.name)
    return names


@pytest.mark.parametrize("path", _sources(), ids=lambda p: os.path.relpath(p, ROOT))
def test_every_read_name_is_bound(path):
    src = open(path).read()
    tree = ast.parse(src, filename=path)
    compile(tree, path, "exec")
    bound = _bound(tree)
    unbound = sorted({(n.id, n.lineno) for n in ast.walk(tree)
                      if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in bound})
    assert not unbound, f"names read but never bound: {unbound}"


def _module_aliases(tree):
    """alias -> module name, for imports of this project's own modules."""
    own = ("paper_2509_25044_gb300", "oracle")
    out = {}
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            for a in n.names:
                if a.name.split(".")[0] in own and a.asname:
                    out[a.asname] = a.name
        elif isinstance(n, ast.ImportFrom) and n.module and n.level == 0 and n.module.split(".")[0] in own:
            for a in n.names:
                out[a.asname or a.name] = f"{n.module}.{a.name}"
        elif isinstance(n, ast.ImportFrom) and n.level == 1:  # from . import x (inside the package)
            for a in n.names:
                out[a.asname or a.name] = f"paper_2509_25044_gb300.{a.name}" if n.module is None else None
    return {k: v for k, v in out.items() if v}


@pytest.mark.parametrize("path", _sources(), ids=lambda p: os.path.relpath(p, ROOT))
def test_attributes_of_own_modules_exist(path):
    """capi.reg_x, synth.make, O.warp ...: every attribute read from one of the
    project's modules exists in it."""
    import importlib
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    tree = ast.parse(open(path).read(), filename=path)
    missing = []
    for alias, mod in _module_aliases(tree).items():
        try:
            m = importlib.import_module(mod)
        except ImportError:
            continue  # a name imported from a module, not a module
        for n in ast.walk(tree):
            if (isinstance(n, ast.Attribute) and isinstance(n.value, ast.Name) and n.value.id == alias
                    and isinstance(n.ctx, ast.Load) and not hasattr(m, n.attr)):
                missing.append((alias, n.attr, n.lineno))
    assert not missing, f"attributes that do not exist: {sorted(set(missing))}"


def _resolve(mod: str):
    import importlib
    try:
        return importlib.import_module(mod)
    except ImportError:
        parent, _, name = mod.rpartition(".")
        return getattr(importlib.import_module(parent), name, None)


@pytest.mark.parametrize("path", _sources(), ids=lambda p: os.path.relpath(p, ROOT))
def test_calls_of_own_functions_fit_their_signatures(path):
    """Every call of one of the project's Python functions or classes
    (capi.reg_loss(...), Registration(...)) passes no unknown keyword and no
    more positional arguments than the signature takes."""
    import inspect
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    tree = ast.parse(open(path).read(), filename=path)
    objs = {alias: _resolve(mod) for alias, mod in _module_aliases(tree).items()}
    bad = []
    for n in ast.walk(tree):
        if not isinstance(n, ast.Call):
            continue
        f = n.func
        target = None
        if isinstance(f, ast.Attribute) and isinstance(f.value, ast.Name) and inspect.ismodule(objs.get(f.value.id)):
            target = getattr(objs[f.value.id], f.attr, None)
        elif isinstance(f, ast.Name) and f.id in objs and not inspect.ismodule(objs[f.id]):
            target = objs[f.id]
        if not (inspect.isfunction(target) or inspect.isclass(target)):
            continue
        if any(isinstance(a, ast.Starred) for a in n.args) or any(k.arg is None for k in n.keywords):
            continue
        try:
            sig = inspect.signature(target)
        except (TypeError, ValueError):
            continue
        try:
            sig.bind_partial(*[None] * len(n.args), **{k.arg: None for k in n.keywords})
        except TypeError as e:
            bad.append((ast.unparse(f), n.lineno, str(e)))
    assert not bad, f"calls that do not fit: {bad}"
