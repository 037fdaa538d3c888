"""Steklov eigensolve (tensor-core Chebyshev subspace iteration) vs LAPACK (numpy eigh) and
the tensor-core split product vs an FP64 matmul."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


@pytest.mark.parametrize("n,m", [(300, 32), (1000, 96), (777, 160)])
def test_tc_split_product_matches_fp64(n, m):
    g = torch.Generator().manual_seed(n + m)
    A = torch.randn(n, n, generator=g, dtype=torch.float64)
    A = 0.5 * (A + A.T)
    Xt = torch.randn(m, n, generator=g, dtype=torch.float64)
    Z = mcs.tc_symm_product(A.cuda(), Xt.cuda()).cpu()
    ref = (A @ Xt.T).T
    # tf32 high/low split: ~2^-20 relative per product, FP32 accumulation over n terms
    scale = (A.abs() @ Xt.abs().T).T
    err = ((Z - ref).abs() / scale).max().item()
    assert err < 2e-5, err


def _oracle_lambda(oracle, subdiv=3, W=128):
    m = meshgen.icosphere(subdiv)
    rows = oracle.vertex_rows(m.V, m.F)
    est = oracle.estimate(m.V, m.F, rows, W, 1e-3, seed=0)
    return oracle.assemble(est, rows), rows["area"]


@pytest.mark.parametrize("k", [16, 64])
def test_steklov_modes_match_lapack(oracle, k):
    L, mass = _oracle_lambda(oracle)
    ref, Xr = oracle.steklov(L, mass, k)
    ev, X, st = mcs.steklov_modes(torch.from_numpy(L).cuda(), torch.from_numpy(mass).cuda(), k)
    assert st["status"] == 0, st
    ev = ev.cpu().numpy()
    lmax = np.linalg.eigvalsh(L / np.sqrt(np.outer(mass, mass))).max()
    assert np.abs(ev - ref).max() <= 1e-4 * lmax + 1e-6, (np.abs(ev - ref).max(), lmax)
    # M-orthonormal eigenvectors spanning the same space (compare projectors, not vectors)
    X = X.cpu().numpy()
    G = X.T @ (mass[:, None] * X)
    assert np.abs(G - np.eye(k)).max() < 1e-6
    sq = np.sqrt(mass)[:, None]
    # clusters can be cut at k: compare the well-separated leading part only
    gaps = np.flatnonzero(np.diff(ref) > 1e-3 * lmax)
    kk = gaps[gaps < k - 1].max() + 1 if len(gaps[gaps < k - 1]) else 1
    P1 = (sq * X[:, :kk]) @ (sq * X[:, :kk]).T
    P2 = (sq * Xr[:, :kk]) @ (sq * Xr[:, :kk]).T
    assert np.abs(P1 - P2).max() < 1e-3


def test_steklov_on_gpu_estimate_end_to_end():
    """GPU estimate -> GPU eigensolve; the sphere's spectrum comes in multiplets 1, 3, 5."""
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32))
    ev, X, st = mcs.steklov_modes(res["Lambda"], rows["area"], 9)
    ev = ev.cpu().numpy()
    # the constant mode: zero up to the solver's stated accuracy, tol x upper
    # bound (tol = 1e-5), which the residual test below establishes
    assert abs(ev[0]) <= 1e-5 * st["upper_bound"]
    assert ev[1:4].max() < ev[4:9].min()


def test_steklov_solver_meets_its_stated_accuracy():
    """Converged pairs have residuals |A x - theta x| <= tol * upper bound
    (A = M^-1/2 Lambda M^-1/2, x = M^1/2 psi, tol = 1e-5), recomputed here in
    FP64; for a symmetric A each Ritz value lies within its residual of an
    eigenvalue, so the constant mode of a Laplacian-form Lambda (exactly 0)
    comes out within its residual, about tol * upper bound, of 0."""
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32, seed=5))
    k = 24
    ev, X, st = mcs.steklov_modes(res["Lambda"], rows["area"], k)
    assert st["status"] == 0, st
    L = res["Lambda"].cpu().numpy()
    mass = rows["area"].cpu().numpy()
    sq = np.sqrt(mass)
    A = L / np.outer(sq, sq)
    x = sq[:, None] * X.cpu().numpy()
    x /= np.linalg.norm(x, axis=0)
    th = ev.cpu().numpy()
    r = np.linalg.norm(A @ x - x * th[None, :], axis=0)
    # the solver takes its residuals on the tensor-core split product (error
    # ~1e-6 of the upper bound) before a final FP64 re-orthonormalisation, so
    # the FP64 residual of the returned pairs may exceed tol by that much
    tol = 1e-5 * st["upper_bound"]
    assert r.max() <= 1.5 * tol, (r.max(), tol)
    assert st["max_residual"] <= tol
    assert st["upper_bound"] >= np.linalg.eigvalsh(A).max() * (1 - 1e-12)
    assert abs(th[0]) <= r[0] + 1e-12 * st["upper_bound"]


def test_two_sphere_exterior_capacitance_and_symmetry(two_sphere_capacitance):
    """Exterior of two spheres (R = 0.5, icosphere s3, centres 1.5 apart) with
    killing walks, on the GPU at full rate:
    - the killing mass is 4 pi C (C: the pair's capacitance by the method of
      images), split evenly between the spheres;
    - the unsymmetrised jump mass from one sphere to the other equals that
      back (J(s, t) = J(t, s)), although only one sphere holds the inversion
      centre;
    - the lowest eigenvalue lies below the constant's Rayleigh quotient
      4 pi C / |boundary| and above zero, and Lambda is symmetric."""
    R, D = 0.5, 1.5
    m = meshgen.two_spheres(3, R, D)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    W, N = 2048, 1 << 20
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=W, prec=32, domain=1,
                                                          killing_walks=N, seed=4))
    st = res["stats"]
    assert res["status"] == 0 and st["discarded_rows"] == 0
    o = np.asarray(st["origin"])
    pos = rows["pos"].cpu().numpy()
    area = rows["area"].cpu().numpy()
    cf = np.linalg.norm(pos - o, axis=1)
    a = (pos - 0.5 * (pos.max(0) + pos.min(0))) @ (o - 0.5 * (pos.max(0) + pos.min(0))) > 0
    assert a.sum() == m.nv // 2
    k = 4 * np.pi * cf * res["H0"].cpu().numpy() / N
    C = two_sphere_capacitance(R, D)
    assert abs(k.sum() / (4 * np.pi * C) - 1) < 0.01, k.sum() / (4 * np.pi * C)
    assert abs(k[a].sum() / k.sum() - 0.5) < 0.01
    H = mcs.dense_hist(res, m.nv).cpu().numpy().astype(np.float64)
    Wm = res["omega"].cpu().numpy()[:, None] * H / W * cf[None, :]
    ab, ba = Wm[np.ix_(a, ~a)].sum(), Wm[np.ix_(~a, a)].sum()
    assert 0.8 < ab / ba < 1.25, (ab, ba)
    L = res["Lambda"]
    assert torch.equal(L, L.T)
    ev, _, sst = mcs.steklov_modes(L, rows["area"], 16, vectors=False)
    assert sst["status"] == 0
    ev = ev.cpu().numpy()
    rq = k.sum() / area.sum()
    # the solver resolves eigenvalues to ~1e-6 of the spectral upper bound
    assert 0 < ev[0] <= rq + 1e-5 * sst["upper_bound"], (ev[0], rq)
    assert ev[0] > 0.9 * rq


@pytest.mark.parametrize("domain,k,c,nt", [(0, 64, 1, 5), (0, 100, 37, 20), (1, 48, 16, 17)])
def test_steklov_heat_and_hks_match_oracle(oracle, domain, k, c, nt):
    """Steklov heat (Eq. spectralSteklovHeat) and heat kernel signatures from
    GPU eigenpairs, against the oracle's plain sums on the same pairs: FP64 in
    another summation order.  Sizes cross the kernels' row, channel, time and
    eigenvector tiles with ragged ends."""
    m = meshgen.icosphere(3) if domain == 0 else meshgen.two_spheres(2, 0.5, 1.5)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32, domain=domain,
                                                          killing_walks=4096 if domain else 0))
    ev, X, st = mcs.steklov_modes(res["Lambda"], rows["area"], k)
    assert st["status"] == 0
    n = m.nv
    g = torch.Generator().manual_seed(k + c)
    u0 = torch.randn(n, c, generator=g, dtype=torch.float64).cuda()
    times = np.geomspace(1e-3, 5.0, nt)
    u = mcs.steklov_heat(ev, X, rows["area"], u0, times).cpu().numpy()
    h = mcs.hks(ev, X, times).cpu().numpy()
    evh, Xh, mh = ev.cpu().numpy(), X.cpu().numpy(), rows["area"].cpu().numpy()
    ur = oracle.steklov_heat(evh, Xh, mh, u0.cpu().numpy(), times)
    hr = oracle.hks(evh, Xh, times)
    assert u.shape == ur.shape and h.shape == hr.shape
    assert np.abs(u - ur).max() <= 1e-12 * np.abs(ur).max()
    assert np.abs(h - hr).max() <= 1e-12 * np.abs(hr).max()
    # fixed summation order: a second call is bitwise identical
    assert torch.equal(mcs.steklov_heat(ev, X, rows["area"], u0, times), torch.from_numpy(u).cuda())


def test_interior_steklov_heat_conserves_total_heat():
    """The interior spectrum's first mode is the constant (lambda ~ 0): total
    heat sum_x m_x u_t(x) of a unit impulse stays m_x0, up to the computed
    lambda_0 (zero to the solver's accuracy, ~1e-5 of the spectral bound) and
    the constant mode's own accuracy."""
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    rows = mcs.vertex_rows(mesh)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32))
    ev, X, st = mcs.steklov_modes(res["Lambda"], rows["area"], 16)
    u0 = torch.zeros(m.nv, dtype=torch.float64, device="cuda")
    u0[11] = 1.0
    times = np.array([0.01, 0.5, 5.0])
    u = mcs.steklov_heat(ev, X, rows["area"], u0, times)
    tot = (u * rows["area"][None, :]).sum(1).cpu().numpy()
    m0 = float(rows["area"][11])
    lam0 = abs(float(ev[0]))
    assert lam0 < 1e-5 * st["upper_bound"]
    assert np.all(np.abs(tot - m0) <= m0 * (lam0 * times + 1e-3)), (tot, m0, lam0)


def _knn_laplacian(n, nb=8, seed=0):
    """A sparse Laplacian-form matrix (zero row sums, symmetric, positive
    semidefinite): Gaussian weights of a symmetrised nb-nearest-neighbour graph
    of random points on the unit sphere, with random positive masses."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    d, idx = cKDTree(P).query(P, nb + 1)
    h2 = np.mean(d[:, 1:] ** 2)
    Wg = np.zeros((n, n))
    for i in range(n):
        Wg[i, idx[i, 1:]] = np.exp(-d[i, 1:] ** 2 / h2)
    Wg = np.maximum(Wg, Wg.T)
    L = np.diag(Wg.sum(1)) - Wg
    mass = rng.uniform(0.5, 1.5, n) * (4 * np.pi / n)
    return L, mass


def _float_nonzeros(L, mass):
    s = 1.0 / np.sqrt(mass)
    return int(np.count_nonzero((L * (s[:, None] * s[None, :])).astype(np.float32)))


@pytest.mark.parametrize("n,k,product", [(3000, 64, 0), (1000, 128, 2), (700, 16, 2), (3000, 64, 1)])
def test_sparse_and_dense_products_match_lapack(n, k, product):
    """The eigensolver on a sparse Laplacian-form matrix with the CSR product
    (chosen automatically at 0.3 % density, or forced) and with the dense
    tensor-core product: eigenvalues against LAPACK to the dense test's bound,
    M-orthonormal vectors, the zero mode, and the reported nonzero count and
    operator (the rule: sparse when at most one entry in 32 is nonzero).
    Blocks of 48, 96 and 160 vectors take the sparse kernel's 2-, 3- and
    5-word lane layouts."""
    L, mass = _knn_laplacian(n, seed=n + k)
    sq = np.sqrt(mass)
    A = L / np.outer(sq, sq)
    ref = np.linalg.eigvalsh(A)
    lmax = ref.max()
    p = mcs.default_eig_params(product=product)
    ev, X, st = mcs.steklov_modes(torch.from_numpy(L).cuda(), torch.from_numpy(mass).cuda(), k, params=p)
    assert st["status"] == 0, st
    nnz = _float_nonzeros(L, mass)
    assert st["nnz"] == nnz
    want = product if product else (2 if nnz * 32 <= n * n else 1)
    assert st["product"] == want
    ev = ev.cpu().numpy()
    assert np.abs(ev - ref[:k]).max() <= 1e-4 * lmax + 1e-6, (np.abs(ev - ref[:k]).max(), lmax)
    assert abs(ev[0]) <= 1e-5 * st["upper_bound"]
    X = X.cpu().numpy()
    G = X.T @ (mass[:, None] * X)
    assert np.abs(G - np.eye(k)).max() < 1e-6


def test_sparse_product_on_an_estimated_lambda(oracle):
    """The oracle's Lambda of the icosphere (vertex rows, W = 128) through the
    forced sparse product gives LAPACK's spectrum like the dense product does;
    the automatic choice follows the density rule."""
    L, mass = _oracle_lambda(oracle)
    ref, _ = oracle.steklov(L, mass, 32)
    lmax = np.linalg.eigvalsh(L / np.sqrt(np.outer(mass, mass))).max()
    Ld, md = torch.from_numpy(L).cuda(), torch.from_numpy(mass).cuda()
    ev2, _, st2 = mcs.steklov_modes(Ld, md, 32, params=mcs.default_eig_params(product=2))
    ev0, _, st0 = mcs.steklov_modes(Ld, md, 32)
    assert st2["status"] == 0 and st0["status"] == 0
    assert st2["product"] == 2
    nnz = _float_nonzeros(L, mass)
    assert st0["nnz"] == st2["nnz"] == nnz
    assert st0["product"] == (2 if nnz * 32 <= L.shape[0] ** 2 else 1)
    for ev in (ev2, ev0):
        assert np.abs(ev.cpu().numpy() - ref).max() <= 1e-4 * lmax + 1e-6
