"""The CS_DEBUG build (device index checks that record CS_ERR_BOUNDS and skip
the access, no trap) runs the parity cases clean: every check holds on the
tiny scene in the cost mode, a conservatism sweep with groups, the persistent
tile shapes, the four-CTA quad shapes, the flags mode with groups, the adjoint and ellipsoids, and the results still match the FP64
oracle.  It runs in a child process that loads libcs_b300_debug.so through
CS_B300_LIBRARY.  Also: the autotuner's JSON log."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import cs_synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import numpy as np, torch
import cs_synth as S, oracle
from _parity import compare, to_np
import paper_2609_35619_b300 as cs
assert "CS_DEBUG" in cs.abi.cs_version(), cs.abi.cs_version()
sc = S.tiny_scene(); q = S.tiny_queries(q=1000)
scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
P = oracle.Params()
out = to_np(scene.query(torch.as_tensor(q), 1.0, want_count=True, params=cs.QueryParams(group_size=32)))
scene.sync()
compare(out, oracle.query(sc, q, 0, 1.0, P), 0, P, "debug cost")
sw = to_np(scene.query(torch.as_tensor(q), 0.0, want_count=True,
                       params=cs.QueryParams(group_size=64, sweep=(0.0, 1.0, 2.0), tile_config=27)))
scene.sync()
for b, ns in enumerate((0.0, 1.0, 2.0)):
    blk = {{k: v[b * 1000:(b + 1) * 1000] for k, v in sw.items() if v.shape[0] == 3000}}
    compare(blk, oracle.query(sc, q, 0, ns, P), 0, P, f"debug sweep ns={{ns}}")
for t in (28, 29, 30):
    pe = to_np(scene.query(torch.as_tensor(q), 1.0, want_count=True, params=cs.QueryParams(group_size=32, tile_config=t)))
    scene.sync()
    compare(pe, oracle.query(sc, q, 0, 1.0, P), 0, P, f"debug shape {{t}}")
sw = to_np(scene.query(torch.as_tensor(q), 0.0, want_count=True,
                       params=cs.QueryParams(group_size=64, sweep=(0.0, 1.0, 2.0, 0.5), tile_config=30)))
scene.sync()
for b, ns in enumerate((0.0, 1.0, 2.0, 0.5)):
    blk = {{k: v[b * 1000:(b + 1) * 1000] for k, v in sw.items() if v.shape[0] == 4000}}
    compare(blk, oracle.query(sc, q, 0, ns, P), 0, P, f"debug persistent sweep ns={{ns}}")
fl = to_np(scene.query(torch.as_tensor(q), 1.0, params=cs.QueryParams(group_size=16, mode=cs.CS_METRIC_FLAGS)))
scene.sync()
g = scene.query_grad(torch.as_tensor(q), 1.0, params=cs.QueryParams(group_size=32))
scene.sync()
go = oracle.grad(sc, q, 0, 1.0)
assert np.isfinite(g.cpu().numpy()).all() and np.abs(go).max() > 0
rng = np.random.default_rng(3)
e = S.ellipsoid_queries(4, rng.uniform(0, 2, (500, 3)), 0.03, 0.2)
eo = to_np(scene.query(torch.as_tensor(e), 1.0, prim_type=1, want_count=True))
scene.sync()
print("debug build clean")
"""


def test_debug_build_runs_parity_cases_clean(cuda_device):
    from paper_2609_35619_b300 import abi, build
    lib = abi.DEBUG_LIB_PATH
    if not os.path.exists(lib):
        build.build(debug=True)
    env = dict(os.environ, CS_B300_LIBRARY=lib)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    proc = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=900)
    assert proc.returncode == 0, proc.stdout[-3000:] + proc.stderr[-3000:]
    assert "debug build clean" in proc.stdout


def test_autotune_log_lines(cuda_device, tmp_path):
    import paper_2609_35619_b300 as cs
    sc = S.tiny_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    q = torch.as_tensor(S.tiny_queries(q=3000), device=cuda_device)
    log = tmp_path / "tune.jsonl"
    assert cs.abi.cs_autotune_log(str(log)) == cs.abi.CS_OK
    try:
        best, ms = scene.autotune(q, 1.0, reps=1)
        best2, _ = scene.autotune(q, 0.0, params=cs.QueryParams(sweep=(0.0, 2.0)), reps=1)
    finally:
        cs.abi.cs_autotune_log(None)
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert len(lines) == 2
    a, b = lines
    assert a["best"] == best and a["rows"] == 3000 and a["sweep"] == 1 and a["launch_rows"] == 3000
    assert set(int(k) for k in a["ms"]) == set(ms)
    assert a["ms"][str(a["best"])] == min(a["ms"].values())
    assert b["best"] == best2 and b["sweep"] == 2 and b["launch_rows"] == 6000
    assert a["n_gaussians"] == scene.info()["n_kept"]
    # logging stopped: a further call appends nothing
    scene.autotune(q, 1.0, reps=1)
    assert len(log.read_text().splitlines()) == 2
