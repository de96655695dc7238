"""Static checks of bench.py that need no GPU: it parses, and no function
assigns a local name that shadows a module-level import (such a name is
local in the whole function, so using the module before the assignment
fails at run time)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_has_no_local_names_shadowing_imports():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    imported = {a.asname or a.name.split(".")[0] for node in tree.body if isinstance(node, (ast.Import, ast.ImportFrom))
                for a in node.names}
    bad = {}
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        assigned = set()
        for node in ast.walk(fn):
            targets = node.targets if isinstance(node, ast.Assign) else (
                [node.target] if isinstance(node, (ast.AugAssign, ast.AnnAssign, ast.For)) else [])
            for t in targets:
                for x in ast.walk(t):
                    if isinstance(x, ast.Name):
                        assigned.add(x.id)
        clash = assigned & imported
        if clash:
            bad[fn.name] = sorted(clash)
    assert not bad, bad


def test_bench_json_keys_are_present_in_every_arm():
    src = open(os.path.join(ROOT, "bench.py")).read()
    for key in ('"metric"', '"value"', '"unit"', '"n_gpus"', '"steps"', '"warmup"', '"ms_per_step"',
                '"higher_is_better"', '"scaling"', '"vs_baseline"', '"dtype"', '"data"', '"config"', '"roofline"',
                '"cpu_baseline"', '"e2e"', '"clocks"', '"gpu_launches"'):
        # the learned arm, the batching arm and the fixed-ratio arm each print one line
        assert src.count(key) >= 3, key
