"""Launch-shape autotuner of the persistent stencil kernels.

The shape (CTAs per SM, time-chunk length of the marching kernel) decides
only how work units are shared among CTAs and the order in which per-CTA dot
partials are summed, so:

* every recorded choice is the fastest of its measured candidates, and the
  candidates are the shapes the launch allows;
* a solve with measured shapes and one with the default shapes give the same
  posterior mean to the solver's tolerance (and both the oracle's);
* launches recorded into a CUDA graph (the device-driven solve) queue their
  measurement and the graph is captured again with the measured shapes;
* GMRF_AUTOTUNE_FILE carries the choices to a new process, which then
  measures nothing;
* GMRF_AUTOTUNE=0 records nothing.

Each case runs in a fresh process so that the process-wide table starts empty.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
from paper_2503_08343_gb300 import gmrf
from paper_2503_08343_gb300 import workloads as W
kind = sys.argv[1]
if kind == "matern":
    pr, ob = W.c2_matern(n=256, m=3000, seed=4)
else:
    pr, ob = W.c5_st2d(n=64, nt=64, m=2000, seed=5)
post = gmrf.Posterior(gmrf.Prior(pr), ob)
mu, info = post.solve_mean()
_, _, isamp = post.sample(16, 7)
print(json.dumps({"log": gmrf.autotune_log(), "mode": gmrf.autotune_mode(), "mu": mu.tolist(),
                  "converged": int(info["converged"]) and int(isamp["converged"])}))
"""


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2503_08343_gb300 import build
    build.build()


def _child(kind, **env):
    e = dict(os.environ)
    e.pop("GMRF_AUTOTUNE", None)
    e.pop("GMRF_AUTOTUNE_FILE", None)
    e.update(env)
    r = subprocess.run([sys.executable, "-c", CHILD, kind], cwd=ROOT, env=e, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def _check_choices(log):
    assert log, "no launch shape was measured"
    for ent in log:
        ms = ent["ms"]
        assert ms, ent
        chosen = f"{ent['ctas_per_sm']}x{ent['aux']}"
        assert chosen in ms and ms[chosen] == min(ms.values()), ent
        assert all(v > 0 for v in ms.values()), ent
        for lab in ms:
            k, aux = (int(v) for v in lab.split("x"))
            assert k >= 1
            assert aux in ((0,) if "|stencil<" in ent["key"] else (1, 2, 4)), ent


@pytest.mark.parametrize("kind", ["matern", "st2d"])
def test_measured_shapes_are_the_fastest_candidates_and_keep_the_result(kind):
    on = _child(kind)
    off = _child(kind, GMRF_AUTOTUNE="0")
    assert on["mode"] == 1 and off["mode"] == 0
    assert on["converged"] and off["converged"]
    _check_choices(on["log"])
    assert off["log"] == []
    kinds = {ent["key"].split("|")[1].split("<")[0] for ent in on["log"]}
    assert ("stencil" if kind == "matern" else "march") in kinds, kinds
    a, b = np.array(on["mu"]), np.array(off["mu"])
    assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))


def test_choices_persist_through_the_file(tmp_path):
    f = tmp_path / "shapes.jsonl"
    first = _child("matern", GMRF_AUTOTUNE_FILE=str(f))
    lines = [json.loads(x) for x in f.read_text().splitlines()]
    assert sorted(x["key"] for x in lines) == sorted(x["key"] for x in first["log"])
    second = _child("matern", GMRF_AUTOTUNE_FILE=str(f))
    # loaded, not measured again: no new lines, no timings in this process
    assert len(f.read_text().splitlines()) == len(lines)
    assert {x["key"]: x["ctas_per_sm"] for x in second["log"]} == {x["key"]: x["ctas_per_sm"] for x in lines}
    assert all(x["ms"] is None for x in second["log"])
    a, b = np.array(first["mu"]), np.array(second["mu"])
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_in_process_mode_switch():
    from paper_2503_08343_gb300 import gmrf
    prev = gmrf.autotune_mode(0)
    try:
        assert gmrf.autotune_mode() == 0
    finally:
        gmrf.autotune_mode(prev)
    assert gmrf.autotune_mode() == prev
