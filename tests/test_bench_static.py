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


def test_committed_traffic_needs_the_same_source_and_operating_point(tmp_path, monkeypatch):
    # a DRAM-traffic record counts only for the kernel source it was taken on
    # and, for the learned arm, the label setup and margins it was taken at
    import json
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2411_14754_gb300 import learn as L
    setup = bench.learned_setup(L, "full", (0.75, 0.75))
    assert setup["alpha_grid"] == list(L.ALPHA_GRID) and setup["margin"] == [0.75, 0.75]
    rec = {"5-learned": {"kernel_source_hash": bench.kernel_source_hash(), "dram_bytes_per_launch": 123.0,
                         "operating_point": setup},
           "5": {"kernel_source_hash": "0" * 16, "dram_bytes_per_launch": 7.0}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["5-learned"]["kernel_source_hash"])
    assert bench.committed_traffic("5-learned", setup) == 123.0
    assert bench.committed_traffic("5-learned", bench.learned_setup(L, "full", (0.5, 0.75))) is None
    assert bench.committed_traffic("5-learned", bench.learned_setup(L, "lagrange", (0.75, 0.75))) is None
    assert bench.committed_traffic("5") is None          # taken on another source
    assert bench.committed_traffic("missing") is None
