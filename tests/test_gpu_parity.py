"""CUDA path vs the CPU oracle, through the C ABI.

Hit counts, closest points, rows and Philox words are compared bit for bit
(both sides follow the same written arithmetic, in the precision the kernel
decides in); Lambda within 1e-12 of its largest entry (the FP64 row sums are
accumulated in a different order).
"""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _rows_to_torch(rows):
    out = dict(pos=torch.from_numpy(rows["pos"]).cuda(), nrm=torch.from_numpy(rows["nrm"]).cuda(),
               area=torch.from_numpy(rows["area"]).cuda(), tri2bin=None)
    if rows.get("tri2bin") is not None:
        out["tri2bin"] = torch.from_numpy(rows["tri2bin"].astype(np.int32)).cuda()
    return out


def test_philox_words_match(oracle):
    n = 1 << 20
    g = mcs.philox_words(5, n, 3, 7, 0x0123456789ABCDEF).cpu().numpy().view(np.uint32)
    c = oracle.philox(5, n, 3, 7, 0x0123456789ABCDEF)
    assert np.array_equal(g, c)


@pytest.mark.parametrize("layout", [2, 4])
@pytest.mark.parametrize("which", ["ico2", "two3", "wild"])
@pytest.mark.parametrize("prec", [64, 32])
def test_closest_points_bit_exact(oracle, which, prec, layout):
    m = {"ico2": lambda: meshgen.icosphere(2), "two3": lambda: meshgen.two_spheres(3, 0.5, 1.5),
         "wild": lambda: meshgen.wild_union(6, 6000, seed=4)}[which]()
    rng = np.random.default_rng(7)
    lo, hi = m.V.min(0), m.V.max(0)
    P = rng.uniform(lo - 0.3, hi + 0.3, size=(4000, 3))
    P[:50] = m.V[:50]                         # on vertices: exact ties between faces
    P[50:100] = m.V[m.F[:50]].mean(1)         # on faces
    mesh = mcs.Mesh(m.V, m.F)
    if layout == 4:
        mesh.build_wide()
    d2g, fg, bg = (t.cpu().numpy() for t in mcs.closest_points(mesh, torch.from_numpy(P), prec, layout))
    d2c, fc, bc = oracle.closest_points(m.V, m.F, P, prec)
    assert np.array_equal(fg, fc)
    assert np.array_equal(d2g, d2c)
    assert np.array_equal(bg, bc)


def test_vertex_rows_bit_exact(oracle):
    m = meshgen.wild_union(5, 4000, seed=1)
    mesh = mcs.Mesh(m.V, m.F)
    r = mcs.vertex_rows(mesh)
    o = oracle.vertex_rows(m.V, m.F)
    for k in ("pos", "nrm", "area"):
        assert np.array_equal(r[k].cpu().numpy(), o[k]), k


def _compare(oracle, m, rows_np, W, eps, prec, exterior=False, killing=0, seed=0, row_list=None, check_L=True,
             origin=None):
    mesh = mcs.Mesh(m.V, m.F)
    rows = _rows_to_torch(rows_np)
    kw = dict(walks_per_row=W, eps=eps, prec=prec, seed=seed, domain=1 if exterior else 0, killing_walks=killing)
    if origin is not None:
        kw["origin"] = origin
    p = mcs.default_params(**kw)
    res = mcs.estimate_dtn(mesh, rows, p, assemble=check_L, record_exits=True)
    torch.cuda.synchronize()
    R = rows["pos"].shape[0]
    H = mcs.dense_hist(res, R).cpu().numpy()
    st = res["stats"]
    o = np.array(st["origin"]) if exterior else None
    est = oracle.estimate(m.V, m.F, rows_np, W, eps, exterior=exterior, origin=o, seed=seed, prec=prec,
                          row_list=row_list, killing_walks=killing, record_exits=True)
    rl = est["row_list"]
    assert np.array_equal(H[rl], est["H"]), f"hit counts differ in {np.sum(H[rl] != est['H'])} entries"
    assert np.array_equal(res["exit_tri"].cpu().numpy()[rl], est["exit_tri"])
    if killing:
        assert np.array_equal(res["H0"].cpu().numpy(), est["H0"])
    if row_list is None:
        assert st["lost"] == est["lost"].sum() + est["kill_stats"][2]
    om = res["omega"].cpu().numpy()[rl]
    assert np.array_equal(om, oracle.row_weights(est, rows_np))
    if check_L and row_list is None:
        L = res["Lambda"].cpu().numpy()
        Lo = oracle.assemble(est, rows_np, exterior=exterior, origin=o, killing=killing > 0)
        assert np.array_equal(L, L.T)
        assert np.abs(L - Lo).max() <= 1e-12 * np.abs(Lo).max()
    return res, est


@pytest.mark.parametrize("prec", [64, 32])
def test_interior_icosphere_bit_exact(oracle, prec):
    """The small sphere workload: icosphere s2, 128 walks per vertex, eps 1e-3, seed 0."""
    m = meshgen.icosphere(2)
    rows = oracle.vertex_rows(m.V, m.F)
    res, est = _compare(oracle, m, rows, 128, 1e-3, prec)
    assert res["stats"]["steps"] == est["steps"].sum()
    assert np.all(res["hist_nnz"].cpu().numpy() <= 128)


@pytest.mark.parametrize("prec", [64, 32])
def test_exterior_two_spheres_bit_exact(oracle, prec):
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = oracle.interior_origin(m.V, m.F, rows)
    res, est = _compare(oracle, m, rows, 64, 1e-3, prec, exterior=True, killing=2048, seed=3)
    assert np.array_equal(np.array(res["stats"]["origin"]), o)


@pytest.mark.parametrize("prec", [64, 32])
def test_sample_rows_wild_bit_exact(oracle, prec):
    """FPS sample rows on a small in-the-wild union (flips, noise, slivers), tri2bin columns."""
    m = meshgen.wild_union(6, 5000, seed=9)
    rows = oracle.fps_rows(m.V, m.F, 300, orient=True)
    _compare(oracle, m, rows, 64, 1e-3, prec)


def test_two_spheres_full_size_sampled_rows(oracle):
    """Two s4 spheres, exterior, FP32, 1024 walks per vertex: the full-size launch,
    checked on sampled rows (the oracle recomputes each row's walks alone)."""
    m = meshgen.two_spheres(4, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    rl = np.array([0, 1, 777, 2561, 2562, 4000, 5123], np.int32)
    _compare(oracle, m, rows, 1024, 1e-3, 32, exterior=True, row_list=rl, check_L=False,
             origin=oracle.interior_origin(m.V, m.F, rows))


def test_ragged_and_degenerate_rows(oracle):
    """Odd row counts, a zero-normal row and a row whose tangent ball is too small."""
    m = meshgen.icosphere(2)
    rows = oracle.vertex_rows(m.V, m.F)
    rows = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rows.items()}
    rows["nrm"][3] = 0.0
    res, est = _compare(oracle, m, rows, 6, 1e-3, 64)
    assert res["hist_nnz"].cpu().numpy()[3] == 0
    assert res["stats"]["discarded_rows"] == 1


def test_lambda_invariants_icosphere():
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32), fp32_copy=True)
    L = res["Lambda"].cpu().numpy()
    assert np.array_equal(res["Lambda32"].cpu().numpy(), L.astype(np.float32))
    assert np.array_equal(L, L.T)
    assert np.abs(L.sum(1)).max() < 1e-12 * np.abs(L).max()
    assert np.linalg.eigvalsh(L).min() > -1e-10 * np.abs(L).max()
    nnz = res["hist_nnz"].cpu().numpy()
    cnt = res["hist_cnt"].cpu().numpy().reshape(m.nv, -1)
    assert all(cnt[v, :nnz[v]].sum() == 256 for v in range(m.nv))


def test_invalid_arguments_are_rejected():
    m = meshgen.icosphere(1)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    with pytest.raises(mcs.MCSError):
        mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=7))
    with pytest.raises(mcs.MCSError):
        mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=8, eps=-1.0))
    bad = m.V.copy()
    bad[0, 0] = np.nan
    with pytest.raises(mcs.MCSError):
        mcs.Mesh(bad, m.F)
    with pytest.raises(mcs.MCSError):
        mcs.Mesh(m.V, m.F + 1000)


def test_sample_rows_match_oracle(oracle):
    """FPS selections, owners (tri2bin), Voronoi areas and positions bit for bit; the
    orientation sign agrees wherever the oracle's winding-number gap is not a near tie."""
    m = meshgen.wild_union(8, 12000, seed=11)
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, 500, orient=True)
    o = oracle.fps_rows(m.V, m.F, 500, orient=True)
    assert np.array_equal(g["sel"].cpu().numpy(), o["sel"])
    assert np.array_equal(g["tri2bin"].cpu().numpy(), o["tri2bin"])
    assert np.array_equal(g["area"].cpu().numpy(), o["area"])
    assert np.array_equal(g["pos"].cpu().numpy(), o["pos"])
    gn, on = g["nrm"].cpu().numpy(), o["nrm"]
    same = np.all(gn == on, axis=1)
    flipped = np.all(gn == -on, axis=1)
    assert np.all(same | flipped)
    for i in np.flatnonzero(flipped):
        f = o["sel"][i]
        a, b, c = m.V[m.F[f]]
        delta = 0.25 * np.sqrt(0.5 * np.linalg.norm(np.cross(b - a, c - a)))
        gi = oracle.gwn(m.V, m.F, o["pos"][i] - delta * on[i], skip=f)
        go = oracle.gwn(m.V, m.F, o["pos"][i] + delta * on[i], skip=f)
        assert abs(gi - go) < 1e-3, (i, gi, go)
    assert flipped.mean() < 0.01


def test_hierarchical_orientation_equals_brute_force(oracle):
    """Sample-row orientation by the BVH sums with certified far-field bounds
    (orient 3) against brute force on every row (orient 2) and the oracle's
    FP64 winding numbers: the same sampling, the same normal wherever the gap
    is not a near tie, gaps within the far-field tolerance."""
    m = meshgen.wild_union(10, 40000, seed=17)
    mesh = mcs.Mesh(m.V, m.F)
    h = mcs.sample_rows(mesh, 1500, orient=3)
    b = mcs.sample_rows(mesh, 1500, orient=2)
    for k in ("sel", "tri2bin", "area", "pos"):
        assert torch.equal(h[k], b[k]), k
    gh, gb = h["gap"].cpu().numpy().astype(np.float64), b["gap"].cpu().numpy().astype(np.float64)
    hn, bn = h["nrm"].cpu().numpy(), b["nrm"].cpu().numpy()
    same = np.all(hn == bn, axis=1)
    assert np.all(same | np.all(hn == -bn, axis=1))
    assert np.all(same | (np.abs(gb) < 1e-4)), np.abs(gb[~same]).max()
    assert np.abs(gh - gb).max() < 0.02, np.abs(gh - gb).max()
    # against the FP64 oracle on a sample of rows
    o = oracle.fps_rows(m.V, m.F, 1500, orient=False)
    assert np.array_equal(o["sel"], h["sel"].cpu().numpy())
    for i in range(0, 1500, 97):
        f = o["sel"][i]
        a_, b_, c_ = m.V[m.F[f]]
        delta = 0.25 * np.sqrt(0.5 * np.linalg.norm(np.cross(b_ - a_, c_ - a_)))
        nrm = o["nrm"][i]
        gi = oracle.gwn(m.V, m.F, o["pos"][i] - delta * nrm, skip=f)
        go = oracle.gwn(m.V, m.F, o["pos"][i] + delta * nrm, skip=f)
        g = gi - go
        # both gaps refer to the unoriented face normal; the GPU keeps it when its gap is positive
        kept = np.all(hn[i] == nrm)
        if abs(g) > 1e-3:
            assert (g > 0) == kept, (i, g)
        assert abs(gh[i] - g) < 0.02, (i, gh[i], g)


def test_sample_rows_large_mesh_match_oracle(oracle):
    """Above 2^18 faces the farthest-point sampling runs on a thread-block
    cluster (sub-range culling, candidates exchanged through distributed
    shared memory): selections, owners, areas and positions bit for bit."""
    m = meshgen.wild_union(24, 320000, seed=23)
    assert m.nf > 1 << 18
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, 1200, orient=0)
    o = oracle.fps_rows(m.V, m.F, 1200, orient=False)
    assert np.array_equal(g["sel"].cpu().numpy(), o["sel"])
    assert np.array_equal(g["tri2bin"].cpu().numpy(), o["tri2bin"])
    assert np.array_equal(g["area"].cpu().numpy(), o["area"])
    assert np.array_equal(g["pos"].cpu().numpy(), o["pos"])
    assert np.array_equal(g["nrm"].cpu().numpy(), o["nrm"])


def test_brute_force_orientation_of_a_few_rows():
    """A handful of rows: the brute-force pass splits the faces into many
    chunks to fill the grid, with the same normals as the hierarchical pass."""
    m = meshgen.wild_union(6, 20000, seed=5)
    mesh = mcs.Mesh(m.V, m.F)
    h = mcs.sample_rows(mesh, 5, orient=3)
    b = mcs.sample_rows(mesh, 5, orient=2)
    gb = b["gap"].cpu().numpy()
    for i in range(5):
        if abs(gb[i]) > 1e-4:
            assert torch.equal(h["nrm"][i], b["nrm"][i]), i


@pytest.mark.parametrize("prec", [64, 32])
def test_sample_rows_estimate_bit_exact(oracle, prec):
    """The estimate on GPU sample rows equals the oracle's on the same rows."""
    m = meshgen.wild_union(6, 5000, seed=9)
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, 300, orient=True)
    rows_np = dict(pos=g["pos"].cpu().numpy(), nrm=g["nrm"].cpu().numpy(), area=g["area"].cpu().numpy(),
                   tri2bin=g["tri2bin"].cpu().numpy())
    _compare(oracle, m, rows_np, 64, 1e-3, prec)


@pytest.mark.parametrize("prec", [64, 32])
def test_exterior_escapes_bit_exact(oracle, prec):
    """Exterior of nested spheres with the inversion centre in the gap: walks of
    the inner sphere's rows that wander towards the centre are retired without a
    hit, on the GPU exactly as in the oracle (reading R17)."""
    A = meshgen.icosphere(3, 1.0)
    B = meshgen.icosphere(3, 0.3)
    m = meshgen.Mesh(np.concatenate([A.V, B.V]), np.concatenate([A.F, B.F + A.nv]), "nested spheres")
    rows = oracle.vertex_rows(m.V, m.F)
    res, est = _compare(oracle, m, rows, 16, 1e-3, prec, exterior=True, killing=256, seed=5,
                        origin=np.array([0.65, 0.0, 0.0]))
    assert res["stats"]["lost"] > 0 and res["stats"]["capped"] == 0
    assert res["status"] == 3


@pytest.mark.parametrize("prec", [64, 32])
def test_interior_walks_retired_in_the_unbounded_component(oracle, prec):
    """An inside-out sphere: interior walks start outside; the ones that wander
    off are retired without a hit on the GPU exactly as in the oracle (R18)."""
    m = meshgen.icosphere(3, 1.0)
    m = meshgen.Mesh(m.V, m.F[:, ::-1].copy(), "inside-out sphere")
    rows = oracle.vertex_rows(m.V, m.F)
    res, est = _compare(oracle, m, rows, 16, 1e-3, prec, seed=3)
    assert res["stats"]["lost"] > 0 and res["stats"]["capped"] == 0
    assert res["status"] == 3


def test_wild_exterior_rows_bit_exact(oracle):
    """Sample rows of an overlapping union, exterior, FP32: pockets, escapes and all."""
    m = meshgen.wild_union(6, 5000, seed=9)
    rows = oracle.fps_rows(m.V, m.F, 200, orient=True)
    _compare(oracle, m, rows, 32, 1e-3, 32, exterior=True, killing=512, seed=2)


@pytest.mark.parametrize("prec", [32, 64])
def test_group_traversal_bit_exact(oracle, prec):
    """Four lanes per walk on the 4-wide BVH: the same hit counts as the oracle."""
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    mesh = mcs.Mesh(m.V, m.F).build_wide()
    r = _rows_to_torch(rows)
    p = mcs.default_params(walks_per_row=64, prec=prec, seed=3, domain=1, killing_walks=1024, bvh_layout=4,
                           lanes_per_query=4)
    res = mcs.estimate_dtn(mesh, r, p, assemble=False, record_exits=True)
    st = res["stats"]
    est = oracle.estimate(m.V, m.F, rows, 64, 1e-3, exterior=True, origin=np.array(st["origin"]), seed=3, prec=prec,
                          killing_walks=1024, record_exits=True)
    assert np.array_equal(mcs.dense_hist(res, m.nv).cpu().numpy(), est["H"])
    assert np.array_equal(res["exit_tri"].cpu().numpy(), est["exit_tri"])
    assert np.array_equal(res["H0"].cpu().numpy(), est["H0"])
    assert st["steps"] == est["steps"].sum()



def _csr_row(res, v):
    cap = res["cap"]
    n = int(res["hist_nnz"][v])
    return (res["hist_bin"][v * cap: v * cap + n].cpu().numpy(), res["hist_cnt"][v * cap: v * cap + n].cpu().numpy())


def test_more_rows_than_the_shared_histogram_holds(oracle):
    """60,000 sample rows (beyond the 51,200 of the shared-memory histogram):
    each row's exits are sorted within its block and run-length counted.  The
    rows equal the oracle's own sampling, sampled rows' (bin, count) pairs
    equal the oracle's histograms, and every row's counts sum to W less its
    walks retired without a hit."""
    m = meshgen.wild_union(10, 70000, seed=31)
    R, W = 60000, 64
    assert m.nf > R
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, R, orient=True)
    rl = np.array([0, 1, 12345, 51199, 51200, 51201, 59998, 59999], np.int32)
    o = oracle.fps_rows(m.V, m.F, R, orient=True, orient_rows=rl)
    assert np.array_equal(g["sel"].cpu().numpy(), o["sel"])
    assert np.array_equal(g["tri2bin"].cpu().numpy(), o["tri2bin"])
    assert np.array_equal(g["pos"].cpu().numpy(), o["pos"])
    rows = {k: g[k] for k in ("pos", "nrm", "area", "tri2bin")}
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=W, seed=4), assemble=False)
    torch.cuda.synchronize()
    nnz = res["hist_nnz"].cpu().numpy()
    cnt = res["hist_cnt"].view(R, res["cap"]).cpu().numpy()
    bins = res["hist_bin"].view(R, res["cap"]).cpu().numpy()
    sums = np.array([cnt[v, :nnz[v]].sum() for v in range(R)])
    disc = res["omega"].cpu().numpy() == 0.0
    # walks retired without a hit (reading R18, stats.lost) leave their row short
    assert np.all(sums[~disc] <= W) and np.all(nnz[disc] == 0)
    assert int((W - sums[~disc]).sum()) == res["stats"]["lost"]
    assert all(np.all(np.diff(bins[v, :nnz[v]]) > 0) for v in range(0, R, 97))  # ascending, distinct
    same = np.all(g["nrm"].cpu().numpy()[rl] == o["nrm"][rl], axis=1)
    rl = rl[same]
    rows_np = dict(pos=o["pos"], nrm=o["nrm"], area=o["area"], tri2bin=o["tri2bin"])
    est = oracle.estimate(m.V, m.F, rows_np, W, 1e-3, seed=4, prec=32, row_list=rl)
    for li, v in enumerate(rl):
        b, c = _csr_row(res, int(v))
        ob = np.flatnonzero(est["H"][li])
        assert np.array_equal(b, ob) and np.array_equal(c, est["H"][li][ob]), int(v)


def test_lambda_beyond_the_shared_histogram():
    """Lambda assembled from the sorted histograms at 52,000 rows (a 21.6 GB
    matrix): symmetric and with zero row sums on sampled rows, as everywhere."""
    m = meshgen.wild_union(8, 60000, seed=37)
    R, W = 52000, 32
    mesh = mcs.Mesh(m.V, m.F)
    g = mcs.sample_rows(mesh, R, orient=True)
    rows = {k: g[k] for k in ("pos", "nrm", "area", "tri2bin")}
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=W, seed=5))
    torch.cuda.synchronize()
    L = res["Lambda"]
    scale = float(L.diagonal().abs().max())
    for v in (0, 7, 25000, 51199, 51200, 51999):
        assert torch.equal(L[v], L[:, v])
        assert abs(float(L[v].sum())) <= 1e-12 * scale * 50
    del L, res
    torch.cuda.empty_cache()
