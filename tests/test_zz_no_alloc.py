"""The allocation-free estimate (mcs_estimate_dtn_noalloc) against the regular one.

Some callers cannot allocate device memory when they need an estimate (they
run inside a pool or arena they do not own, or under an allocator that
forbids cudaMalloc at that point); the no-alloc entry point serves them from
a fixed scratch array reserved by the library.  This file is collected last
so that a run stopping at its first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _outputs(R, W):
    cap = min(W, R)
    return dict(hist_bin=torch.empty(R * cap, dtype=torch.int32, device="cuda"),
                hist_cnt=torch.empty(R * cap, dtype=torch.int32, device="cuda"),
                hist_nnz=torch.empty(R, dtype=torch.int32, device="cuda"),
                Lambda=torch.empty((R, R), dtype=torch.float64, device="cuda"),
                omega=torch.empty(R, dtype=torch.float64, device="cuda"),
                H0=torch.empty(R, dtype=torch.int32, device="cuda"), exit_tri=None)


@pytest.mark.parametrize("exterior", [False, True])
def test_noalloc_matches_regular_estimate_twice(exterior):
    """Two calls in a row give the regular estimate's hit counts, Lambda, H0
    and step count, and neither changes the device's free memory."""
    m = meshgen.two_spheres(2, 0.5, 1.5) if exterior else meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    W = 128
    p = mcs.default_params(walks_per_row=W, prec=32, seed=7, domain=int(exterior),
                           killing_walks=1024 if exterior else 0)
    ref = mcs.estimate_dtn(mesh, rows, p)
    torch.cuda.synchronize()
    R = m.nv
    Href = mcs.dense_hist(ref, R).cpu().numpy()
    Lref = ref["Lambda"].cpu().numpy()
    for _ in range(2):  # the fixed scratch keeps the previous call's contents
        o = _outputs(R, W)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = mcs.estimate_dtn_noalloc(mesh, rows, p, o)
        torch.cuda.synchronize()
        # the call reserved no device memory (its code and scratch were loaded with the mesh)
        assert torch.cuda.mem_get_info()[0] == free0
        o["cap"] = min(W, R)
        H = mcs.dense_hist(o, R).cpu().numpy()
        assert np.array_equal(H, Href)
        L = o["Lambda"].cpu().numpy()
        assert np.abs(L - Lref).max() <= 1e-12 * np.abs(Lref).max()
        if exterior:
            assert np.array_equal(o["H0"].cpu().numpy(), ref["H0"].cpu().numpy())
        assert st["steps"] == ref["stats"]["steps"]


def test_noalloc_rejects_an_estimate_beyond_its_scratch():
    m = meshgen.icosphere(4)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    cap = mcs.lib().mcs_estimate_dtn_noalloc_capacity()
    W = 2 * (cap // (4 * m.nv) // 2 + 2)  # exit bins alone exceed the scratch
    with pytest.raises(mcs.MCSError) as e:
        mcs.estimate_dtn_noalloc(mesh, rows, mcs.default_params(walks_per_row=W), _outputs(m.nv, 2))
    assert e.value.status == -1 and "scratch" in str(e.value)
