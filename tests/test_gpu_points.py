"""Point-based Galerkin basis (Sec. 4.4 "Point-based Galerkin basis";
appendix "Point-based k-NN Interpolator") on the GPU against the oracle: the
k-nearest-point query (bit-exact indices and squared distances), the
bilateral weights, the point-cloud Laplacian, the point-basis Galerkin
matrix, its projection, and the sphere's spectrum through the whole chain."""
import math

import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _fib(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    ph = i * math.pi * (3 - math.sqrt(5))
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)


def _point_sets():
    rng = np.random.default_rng(3)
    S = _fib(800)
    yield "fibonacci", S, S.copy()
    m = meshgen.icosphere(3)          # 642 symmetric vertices: many exact distance ties
    yield "icosphere", m.V.astype(np.float64), m.V / np.linalg.norm(m.V, axis=1, keepdims=True)
    g = 20
    xy = np.stack(np.meshgrid(np.arange(g), np.arange(g), indexing="ij"), -1).reshape(-1, 2) * 0.05
    xy = xy + rng.uniform(-0.01, 0.01, xy.shape)
    P = np.concatenate([xy, np.zeros((len(xy), 1))], 1)  # flat: one grid layer
    yield "plane", P, np.tile([0, 0, 1.0], (len(P), 1))
    w = meshgen.wild_union(6, 5000, seed=9)
    rows = mcs.sample_rows(mcs.Mesh(w.V, w.F), 1500, orient=True)
    yield "wild", rows["pos"].cpu().numpy(), rows["nrm"].cpu().numpy()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k", [1, 8, 32])
def test_knn_bit_exact(oracle, k):
    rng = np.random.default_rng(k)
    for name, P, N in _point_sets():
        lo, hi = P.min(0), P.max(0)
        # queries inside, on the points themselves, and well outside the box
        Q = np.concatenate([rng.uniform(lo - 0.1, hi + 0.1, (500, 3)), P[::7], [[5.0, -3.0, 2.0]]])
        NQ = rng.standard_normal(Q.shape)
        NQ /= np.linalg.norm(NQ, axis=1, keepdims=True)
        idx, w, d2 = mcs.point_knn(_t(P), _t(N), _t(Q), _t(NQ), k=k, sigma=0.1, tau_n=0.8)
        ri, rd = oracle.knn(P, Q, k)
        assert np.array_equal(idx.cpu().numpy(), ri), name
        assert np.array_equal(d2.cpu().numpy(), rd), name
        if k > 1:
            _, rw = oracle.knn_bilateral(P, N, Q, NQ, k, 0.1, 0.8)
            wq = w.cpu().numpy()
            far = np.isfinite(rw).all(1)        # the oracle's plain form underflows far from the points
            assert np.abs(wq[far] - rw[far]).max() <= 1e-13, name
            assert np.abs(wq.sum(1) - 1).max() <= 1e-14 * k
        ei, _, ed = mcs.point_knn(_t(P), None, _t(P), None, k=k, exclude_self=True, weights=False)
        ri, rd = oracle.knn(P, P, k, exclude=np.arange(len(P)))
        assert np.array_equal(ei.cpu().numpy(), ri) and np.array_equal(ed.cpu().numpy(), rd), name


def test_knn_edge_cases(oracle):
    P = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [1.0, 1.0, 1.0]])
    Q = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0]])
    idx, _, d2 = mcs.point_knn(_t(P), None, _t(Q), None, k=5, weights=False)   # k = all points
    ri, rd = oracle.knn(P, Q, 5)
    assert np.array_equal(idx.cpu().numpy(), ri) and np.array_equal(d2.cpu().numpy(), rd)
    one = np.array([[0.3, 0.2, 0.1]])
    idx, w, _ = mcs.point_knn(_t(one), _t([[0, 0, 1.0]]), _t(Q), _t([[0, 0, 1.0]] * 2), k=1)
    assert idx.cpu().numpy().tolist() == [[0], [0]] and np.all(w.cpu().numpy() == 1.0)
    idx, _, _ = mcs.point_knn(_t(P), None, _t(np.zeros((0, 3))), None, k=3, weights=False)
    assert idx.shape == (0, 3)
    with pytest.raises(mcs.MCSError):
        mcs.point_knn(_t(P), None, _t(Q), None, k=6, weights=False)        # more than the points
    with pytest.raises(mcs.MCSError):
        mcs.point_knn(_t(P), None, _t(P), None, k=5, exclude_self=True, weights=False)
    with pytest.raises(mcs.MCSError):
        mcs.point_knn(_t(P), None, _t(Q), None, k=33, weights=False)


def test_point_laplacian_matches_oracle(oracle):
    for name, P, N in _point_sets():
        L, area, nbr, nbw = mcs.point_laplacian(_t(P), _t(N), 16)
        Lr, ar, ir, wr = oracle.point_laplacian(P, N, 16)
        assert np.array_equal(nbr.cpu().numpy(), ir), name
        sc = np.abs(wr).max()
        assert np.abs(nbw.cpu().numpy() - wr).max() <= 1e-11 * sc, name
        assert np.abs(area.cpu().numpy() - ar).max() <= 1e-11 * np.abs(ar).max(), name
        Lg = L.cpu().numpy()
        assert np.array_equal(Lg, Lg.T), name
        assert np.abs(Lg - Lr).max() <= 1e-11 * np.abs(Lr).max(), name


def _sample_case(kind):
    if kind == "sphere":
        m = meshgen.icosphere(2)
        return m, m.nf, 0, 0.1
    if kind == "sphere_ext":
        m = meshgen.icosphere(2)
        return m, m.nf, 1, 0.1
    return meshgen.wild_union(6, 5000, seed=9), 300, 0, 0.025


@pytest.mark.parametrize("kind", ["sphere", "sphere_ext", "wild"])
def test_point_galerkin_lambda_matches_oracle(oracle, kind):
    m, n, dom, sigma = _sample_case(kind)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.sample_rows(mesh, n, orient=kind == "wild")
    rows_np = dict(pos=rows["pos"].cpu().numpy(), nrm=rows["nrm"].cpu().numpy(),
                   area=rows["area"].cpu().numpy(), tri2bin=rows["tri2bin"].cpu().numpy())
    W, kill = 64, 4096 if dom else 0
    o = np.zeros(3)
    p = mcs.default_params(walks_per_row=W, prec=32, domain=dom, seed=5, killing_walks=kill)
    if dom:
        p.origin_auto = 0
        for i in range(3):
            p.origin[i] = 0.0
    res = mcs.estimate_dtn(mesh, rows, p, record_exits=True, record_bary=True)
    est = oracle.estimate(m.V, m.F, rows_np, W, 1e-3, exterior=bool(dom), origin=o, seed=5, prec=32,
                          record_exits=True, killing_walks=kill)
    assert np.array_equal(res["exit_tri"].cpu().numpy(), est["exit_tri"])
    Lp = mcs.point_galerkin_lambda(mesh, rows, res, exterior=bool(dom), killing_walks=kill, sigma=sigma)
    Lr = oracle.point_galerkin_lambda(m.V, m.F, est, rows_np, rows_np["pos"], rows_np["nrm"], exterior=bool(dom),
                                      origin=o, killing=bool(kill), sigma=sigma)
    Lg = Lp.cpu().numpy()
    assert np.abs(Lg - Lr).max() <= 1e-12 * np.abs(Lr).max()
    # projection onto a random M-orthonormal basis through the tensor-core product
    K = 32
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, K)))
    S = mcs.galerkin_project(Lp, _t(q)).cpu().numpy()
    Sref = q.T @ Lr @ q
    scale = np.abs(q).T @ np.abs(Lr) @ np.abs(q)
    assert np.all(np.abs(S - Sref) <= 2e-5 * scale)


def test_point_basis_sphere_spectrum():
    """Unit icosphere s3, 1280 face sample rows as the points, sigma at the
    point spacing: the point Laplacian's modes as the basis and the
    point-basis Galerkin eigenvalues come in multiplets 1, 3, 5 with the l = 1
    triple near the cap-corrected l/R (0.978 at 2.5 degrees)."""
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.sample_rows(mesh, m.nf, orient=False)
    Phi, lev, st = mcs.point_basis(rows, 48)
    assert st["status"] == 0
    lev = lev.cpu().numpy()
    # the constant mode: zero to the eigensolver's stated accuracy (residual
    # <= tol x upper bound, tol = 1e-5), whichever product it took
    assert abs(lev[0]) <= 1e-5 * st["upper_bound"], (lev[0], st["upper_bound"], st["product"])
    assert np.abs(lev[1:4] - 2).max() < 0.1 and np.abs(lev[4:9] - 6).max() < 0.3
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32, seed=1), record_exits=True,
                           record_bary=True)
    spacing = math.sqrt(4 * math.pi / m.nf)
    Lp = mcs.point_galerkin_lambda(mesh, rows, res, sigma=spacing)
    S = mcs.galerkin_project(Lp, Phi)
    ev, _, _ = mcs.galerkin_modes(S, 9)
    ev = ev.cpu().numpy()
    assert abs(ev[0]) < 1e-5 * abs(ev).max()
    assert ev[1:4].max() < ev[4:9].min()
    assert np.abs(ev[1:4] - 0.978).max() < 0.08


def test_point_basis_agrees_with_cotan_basis_exterior():
    """Two spheres (s3, radius 0.5, centres 1.5 apart), exterior with killing
    walks, vertex rows: the point basis (vertex rows as the points, sigma =
    the mean spacing) and the cotangent-Laplacian basis are two independent
    function spaces over the same walks; their lowest Galerkin eigenvalues
    agree to a few percent (the two bases discretise the same operator)."""
    m = meshgen.two_spheres(3, 0.5, 1.5)
    mesh = mcs.Mesh(m.V, m.F)
    vrows = mcs.vertex_rows(mesh)
    kill = 64 * 256
    p = mcs.default_params(walks_per_row=256, prec=32, domain=1, seed=3, killing_walks=kill)
    res = mcs.estimate_dtn(mesh, vrows, p, record_exits=True, record_bary=True)
    K = 48
    _, Phi, st = mcs.steklov_modes(mcs.cotan_laplacian(mesh), vrows["area"], K)
    assert st["status"] == 0
    ev_c, _, _ = mcs.galerkin_modes(mcs.galerkin_dtn(mesh, vrows, res, Phi, exterior=True, killing_walks=kill), 8)
    PhiP, _, pst = mcs.point_basis(vrows, K)
    assert pst["status"] == 0
    sigma = float(torch.sqrt(vrows["area"].sum() / vrows["area"].numel()))
    Lp = mcs.point_galerkin_lambda(mesh, vrows, res, exterior=True, killing_walks=kill, sigma=sigma)
    ev_p, _, _ = mcs.galerkin_modes(mcs.galerkin_project(Lp, PhiP), 8)
    ev_c, ev_p = ev_c.cpu().numpy()[:8], ev_p.cpu().numpy()[:8]
    assert np.all(ev_c > 0) and np.all(ev_p > 0)
    assert np.abs(ev_p - ev_c).max() < 0.05 * ev_c.max()
