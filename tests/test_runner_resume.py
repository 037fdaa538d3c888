"""Checkpoint / resume of batched sweeps (paper_2606_05581_b300.runner), on
the host: a sweep killed between meshes resumes where it stopped and its files
equal an uninterrupted sweep's; incomplete writes are never taken for
results; a resume with other settings is refused.  The chunk estimate here is
the CPU oracle on small meshes (tests/_runner_fake.py); the GPU test of the
same runner uses the library's batched estimate."""
import os
import signal
import subprocess
import sys
import time

import numpy as np
import pytest

from paper_2606_05581_b300 import runner

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SETTINGS = {"workload": "oracle icospheres", "walks": 8}

CHILD = """
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {here!r})
import _runner_fake
from paper_2606_05581_b300 import runner
runner.run_sweep(range(10), {out!r}, _runner_fake.estimate, {settings!r}, chunk=2)
"""


def _same(dir_a, dir_b, ids):
    for i in ids:
        a, ma = runner.read_mesh(dir_a, i)
        b, mb = runner.read_mesh(dir_b, i)
        assert sorted(a) == sorted(b)
        for k in a:
            assert a[k].dtype == b[k].dtype and np.array_equal(a[k], b[k]), (i, k)
        assert ma == mb


def test_sweep_killed_between_meshes_resumes_bit_identically(tmp_path):
    import _runner_fake  # noqa: F401  (tests/ is on sys.path through conftest's rootdir)
    clean = str(tmp_path / "clean")
    runner.run_sweep(range(10), clean, lambda ids: _runner_fake.estimate(ids, sleep=0.0), SETTINGS, chunk=3)
    out = str(tmp_path / "killed")
    child = subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT, here=HERE, out=out, settings=SETTINGS)])
    try:
        deadline = time.time() + 120
        while len(runner.done_ids(out)) < 3 and time.time() < deadline and child.poll() is None:
            time.sleep(0.05)
    finally:
        if child.poll() is None:
            os.kill(child.pid, signal.SIGKILL)
        child.wait()
    have = runner.done_ids(out)
    assert 3 <= len(have) < 10, have
    r = runner.run_sweep(range(10), out, lambda ids: _runner_fake.estimate(ids, sleep=0.0), SETTINGS, chunk=4)
    assert r["skipped"] == len(have) and r["written"] == 10 - len(have)
    assert runner.done_ids(out) == set(range(10))
    assert not [n for n in os.listdir(out) if n.endswith(".tmp")]
    _same(clean, out, range(10))


def test_incomplete_writes_are_not_results(tmp_path):
    import _runner_fake
    out = str(tmp_path / "s")
    runner.run_sweep(range(2), out, lambda ids: _runner_fake.estimate(ids, sleep=0.0), SETTINGS)
    # a write cut off before its rename leaves only a temporary file
    with open(os.path.join(out, ".mesh_0000005.npz.999.tmp"), "wb") as fh:
        fh.write(b"partial")
    assert runner.done_ids(out) == {0, 1}
    r = runner.run_sweep(range(6), out, lambda ids: _runner_fake.estimate(ids, sleep=0.0), SETTINGS)
    assert r == {"requested": 6, "skipped": 2, "written": 4}
    assert not [n for n in os.listdir(out) if n.endswith(".tmp")]


def test_resume_with_other_settings_is_refused(tmp_path):
    import _runner_fake
    out = str(tmp_path / "s")
    runner.run_sweep(range(1), out, lambda ids: _runner_fake.estimate(ids, sleep=0.0), SETTINGS)
    with pytest.raises(ValueError):
        runner.run_sweep(range(2), out, lambda ids: _runner_fake.estimate(ids, sleep=0.0), dict(SETTINGS, walks=16))
