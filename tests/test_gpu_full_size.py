"""Full-size launches checked on sampled outputs against the oracle.

The ~2.0M-face union (10,000 farthest-point sample rows, 4096 walks per
row, interior) and full-size meshes of the 512-mesh batch (1024 sample rows
x 512 walks, one persistent launch over several meshes, exterior for odd
mesh ids) run on the GPU exactly as the benchmark launches them.  The
oracle, brute force over every triangle, computes its own sample rows (the
whole farthest-point selection, orientation of the rows it checks) and then
the first walks of a few rows, with the walk counters of the full launch;
rows, exit triangles and tangent-ball data are compared bit for bit in FP32
and FP64."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _check_rows(oracle, m, g, o, checked):
    """Selections, owners, areas and positions bit for bit; normals of the
    rows the oracle oriented equal, or flipped only where the oracle's FP64
    winding-number gap is a near tie (both sides orient by its sign).
    Returns the mask of checked rows whose normals are equal."""
    assert np.array_equal(g["sel"].cpu().numpy(), o["sel"])
    assert np.array_equal(g["tri2bin"].cpu().numpy(), o["tri2bin"])
    assert np.array_equal(g["area"].cpu().numpy(), o["area"])
    assert np.array_equal(g["pos"].cpu().numpy(), o["pos"])
    gn = g["nrm"].cpu().numpy()[checked]
    on = o["nrm"][checked]
    same = np.all(gn == on, axis=1)
    assert np.all(same | np.all(gn == -on, axis=1))
    for i in np.asarray(checked)[~same]:
        f = o["sel"][i]
        a, b, c = m.V[m.F[f]]
        delta = 0.25 * np.sqrt(0.5 * np.linalg.norm(np.cross(b - a, c - a)))
        gi = oracle.gwn(m.V, m.F, o["pos"][i] - delta * o["nrm"][i], skip=f)
        go = oracle.gwn(m.V, m.F, o["pos"][i] + delta * o["nrm"][i], skip=f)
        assert abs(gi - go) < 1e-3, (i, gi, go)
    assert same.mean() > 0.9
    return same


def _rows_np(o):
    return dict(pos=o["pos"], nrm=o["nrm"], area=o["area"], tri2bin=o["tri2bin"])


def _walk_parity(oracle, m, rows_np, res, rl, W, nwalk, prec, exterior, origin, seed, min_walked=8):
    est = oracle.estimate(m.V, m.F, rows_np, W, 1e-3, exterior=exterior, origin=origin, seed=seed, prec=prec,
                          row_list=rl, record_exits=True, params=dict(walk_limit=nwalk))
    gt = res["exit_tri"].cpu().numpy()[rl, :nwalk]
    ot = est["exit_tri"][:, :nwalk]
    assert np.array_equal(gt, ot), f"{np.sum(gt != ot)} of {gt.size} exit triangles differ"
    om = res["omega"].cpu().numpy()[rl]
    assert np.array_equal(om, oracle.row_weights(est, rows_np))
    assert np.all(ot[est["discarded"] == 0] >= 0)  # discarded rows (ball below 4 eps) have no walks
    assert np.sum(est["discarded"] == 0) >= min_walked
    return est


@pytest.fixture(scope="module")
def wild_2m():
    return meshgen.wild_union(300, 2_000_000, seed=0)


@pytest.mark.parametrize("prec", [32, 64])
def test_wild_2m_full_size_sampled_rows(oracle, wild_2m, prec):
    """The 2.0M-face union at full size: all 10,000 rows x 4096 walks on the GPU;
    16 rows x 32 walks recomputed by the oracle."""
    m = wild_2m
    R, W = 10_000, 4096
    rng = np.random.default_rng(prec)
    rl = np.sort(rng.choice(R, 16, replace=False)).astype(np.int32)
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, R, orient=True)
    o = oracle.fps_rows(m.V, m.F, R, orient=True, orient_rows=rl)
    same = _check_rows(oracle, m, g, o, rl)
    rows_np = _rows_np(o)
    rl = rl[same]  # rows whose orientation was a near tie start different walks
    rows_g = {k: g[k] for k in ("pos", "nrm", "area", "tri2bin")}
    p = mcs.default_params(walks_per_row=W, prec=prec, seed=1, domain=0)
    res = mcs.estimate_dtn(mesh, rows_g, p, assemble=False, record_exits=True)
    torch.cuda.synchronize()
    assert res["stats"]["capped"] == 0 or prec == 64
    _walk_parity(oracle, m, rows_np, res, rl, W, 32, prec, False, None, 1)


@pytest.mark.parametrize("prec", [32, 64])
def test_batch_full_size_meshes_sampled_rows(oracle, prec):
    """Full-size batch meshes in one persistent launch (mesh ids 0 and 1, the
    largest interior mesh 74 and the largest exterior mesh 231 of the 512-mesh
    batch; seed = mesh id, killing walks 64 W): 128 rows x 16 walks of meshes
    74 and 231 recomputed by the oracle, with its own inversion centre (most
    rows of these meshes lie on tiny primitives and are discarded: tangent
    ball below 4 eps; the discards must agree too)."""
    ids = [0, 1, 74, 231]
    hosts = [meshgen.batch_mesh(i) for i in ids]
    W, R = 512, 1024
    meshes = [mcs.Mesh(h.V, h.F) for h in hosts]
    rows = mcs.sample_rows_batched(meshes, R, orient=True)
    items = [dict(mesh=mesh, rows={k: r[k] for k in ("pos", "nrm", "area", "tri2bin")}, domain=i % 2, seed=i)
             for i, mesh, r in zip(ids, meshes, rows)]
    b = mcs.Batch(items, mcs.default_params(walks_per_row=W, prec=prec, killing_walks=64 * W), assemble=True,
                  record_exits=True)
    _, tot, per = b.run()
    torch.cuda.synchronize()
    for k in (2, 3):
        m, i = hosts[k], ids[k]
        rng = np.random.default_rng(i + prec)
        rl = np.sort(rng.choice(R, 128, replace=False)).astype(np.int32)
        ext = bool(i % 2)
        st = oracle.origin_stride(R)
        orient = np.union1d(rl, np.arange(0, R, st)).astype(np.int32) if ext else rl
        o = oracle.fps_rows(m.V, m.F, R, orient=True, orient_rows=orient)
        same = _check_rows(oracle, m, rows[k], o, orient)
        rows_np = _rows_np(o)
        rl = np.intersect1d(rl, orient[same]).astype(np.int32)
        origin = oracle.interior_origin(m.V, m.F, rows_np) if ext else None
        if ext:
            assert np.array_equal(np.array(per[k]["origin"]), origin)
        _walk_parity(oracle, m, rows_np, b.result(k), rl, W, 16, prec, ext, origin, i, min_walked=8)
