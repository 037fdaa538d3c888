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
    # the constant mode: zero up to the solver's accuracy (~1e-6 of the spectral upper bound)
    assert abs(ev[0]) < 1e-5 * st["upper_bound"]
    assert ev[1:4].max() < ev[4:9].min()


def test_two_spheres_tend_to_the_single_sphere_limit(oracle):
    """Exterior of two spheres (R = 0.5, icosphere s3) with killing walks: as the
    separation grows, the spectrum tends to two copies of the single-sphere
    exterior spectrum, lambda_l(theta0) + 1/R with multiplicity 2(2l+1) (the
    cap-corrected jump form plus the killing term; (l+1)/R as theta0 -> 0).
    The limit is approached up to the lumping/faceting bias of the s3 mesh."""
    R = 0.5
    lam = oracle.sphere_eigs_cap(2, 2.5, R) + 1.0 / R
    limit = np.sort(np.concatenate([np.repeat(lam[l], 2 * (2 * l + 1)) for l in range(3)]))[:16]
    errs = {}
    for D in (1.5, 20.0):
        m = meshgen.two_spheres(3, R, D)
        mesh = mcs.Mesh(m.V, m.F)
        rows = mcs.vertex_rows(mesh)
        res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=2048, prec=32, domain=1,
                                                              killing_walks=64 * 2048, seed=4))
        L = res["Lambda"]
        assert torch.equal(L, L.T)
        ev, _, st = mcs.steklov_modes(L, rows["area"], 16, vectors=False)
        assert st["status"] == 0
        errs[D] = np.abs(ev.cpu().numpy() - limit) / limit
    assert errs[20.0].max() < 0.08, errs[20.0]
    assert errs[20.0].mean() < errs[1.5].mean()
