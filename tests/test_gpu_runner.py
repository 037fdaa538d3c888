"""Checkpointed sweeps on the GPU: a sweep over in-the-wild meshes that fails
on the host after its third mesh file (a raising callback, between meshes)
resumes with other chunk boundaries and ends with files bit-identical to an
uninterrupted one-chunk sweep: histograms, row weights, killing hits, Lambda
and rows.  Per-mesh results do not depend on which meshes share a batch."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402
from paper_2606_05581_b300 import runner  # noqa: E402


def _mesh(i):
    return meshgen.wild_union(3 + i % 3, 3000 + 700 * i, seed=200 + i)


class Stop(Exception):
    pass


def test_interrupted_sweep_resumes_bit_identically(tmp_path):
    p = mcs.default_params(walks_per_row=64, killing_walks=2048)
    est = runner.gpu_estimate(_mesh, 256, p, keep_lambda=True)
    settings = {"rows": 256, "walks": 64, "killing_walks": 2048}
    ids = list(range(7))
    clean = str(tmp_path / "clean")
    runner.run_sweep(ids, clean, est, settings, chunk=7)
    out = str(tmp_path / "resumed")
    seen = []

    def fail_after_three(mid):
        seen.append(mid)
        if len(seen) == 3:
            raise Stop()

    with pytest.raises(Stop):
        runner.run_sweep(ids, out, est, settings, chunk=2, on_written=fail_after_three)
    assert runner.done_ids(out) == set(seen)
    r = runner.run_sweep(ids, out, est, settings, chunk=3)
    assert r["skipped"] == 3 and r["written"] == 4
    for i in ids:
        a, ma = runner.read_mesh(clean, i)
        b, mb = runner.read_mesh(out, i)
        assert sorted(a) == sorted(b)
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)
        assert ma == mb
    assert any(runner.read_mesh(out, i)[0]["H0"].sum() > 0 for i in ids if i % 2)
