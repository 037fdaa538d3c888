"""Galerkin estimator (Sec. 4.4, mesh-based Galerkin basis with barycentric
evaluation) on the GPU against the oracle: recorded exit barycentrics, the
cotangent Laplacian, the hat-basis matrix Lambda_bary, its projection
S = Phi^T Lambda_bary Phi onto the cotangent-Laplacian basis, and the K x K
eigenpairs."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _case(kind):
    if kind == "sphere":
        m = meshgen.icosphere(2)
        return m, "vertex", 0
    if kind == "two_spheres":
        return meshgen.two_spheres(2, 0.5, 1.5), "vertex", 1
    return meshgen.wild_union(6, 5000, seed=9), "sample", 0


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["sphere", "two_spheres", "wild"])
def test_exit_barycentrics_bit_exact(oracle, kind, prec):
    m, rk, dom = _case(kind)
    mesh = mcs.Mesh(m.V, m.F)
    if rk == "vertex":
        rows_np = oracle.vertex_rows(m.V, m.F)
        rows = mcs.vertex_rows(mesh)
    else:
        rows = mcs.sample_rows(mesh, 200, orient=True)
        rows_np = dict(pos=rows["pos"].cpu().numpy(), nrm=rows["nrm"].cpu().numpy(),
                       area=rows["area"].cpu().numpy(), tri2bin=rows["tri2bin"].cpu().numpy())
    o = oracle.interior_origin(m.V, m.F, rows_np) if dom else None
    est = oracle.estimate(m.V, m.F, rows_np, 32, 1e-3, exterior=bool(dom), origin=o, seed=7, prec=prec,
                          record_exits=True)
    p = mcs.default_params(walks_per_row=32, prec=prec, domain=dom, seed=7)
    if dom:
        p.origin_auto = 0
        for i in range(3):
            p.origin[i] = float(o[i])
    res = mcs.estimate_dtn(mesh, rows, p, record_exits=True, record_bary=True)
    tri = res["exit_tri"].cpu().numpy()
    assert np.array_equal(tri, est["exit_tri"])
    ok = tri >= 0
    assert ok.mean() > 0.9
    assert np.array_equal(res["exit_bary"].cpu().numpy()[ok], est["exit_bary"][ok])


def test_cotan_laplacian_matches_oracle(oracle):
    m = meshgen.wild_union(4, 3000, seed=3)
    L = mcs.cotan_laplacian(mcs.Mesh(m.V, m.F)).cpu().numpy()
    ref = oracle.cotan_laplacian(m.V, m.F)
    assert np.array_equal(L, L.T)
    assert np.abs(L - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["sphere", "two_spheres", "wild"])
def test_galerkin_matrix_projection_and_modes(oracle, kind):
    m, rk, dom = _case(kind)
    mesh = mcs.Mesh(m.V, m.F)
    vrows = mcs.vertex_rows(mesh)
    if rk == "vertex":
        rows = vrows
        rows_np = oracle.vertex_rows(m.V, m.F)
        rf = None
    else:
        rows = mcs.sample_rows(mesh, 200, orient=True)
        rows_np = dict(pos=rows["pos"].cpu().numpy(), nrm=rows["nrm"].cpu().numpy(),
                       area=rows["area"].cpu().numpy(), tri2bin=rows["tri2bin"].cpu().numpy())
        rf = rows["sel"].cpu().numpy()
    W, kill = 64, 4096 if dom else 0
    o = oracle.interior_origin(m.V, m.F, rows_np) if dom else np.zeros(3)
    p = mcs.default_params(walks_per_row=W, prec=32, domain=dom, seed=5, killing_walks=kill)
    if dom:
        p.origin_auto = 0
        for i in range(3):
            p.origin[i] = float(o[i])
    res = mcs.estimate_dtn(mesh, rows, p, record_exits=True, record_bary=True)
    est = oracle.estimate(m.V, m.F, rows_np, W, 1e-3, exterior=bool(dom), origin=o, seed=5, prec=32,
                          record_exits=True, killing_walks=kill)
    # the basis: the cotangent Laplacian's lowest modes, M-orthonormal in the
    # vertex areas; on the in-the-wild union (slivers, flipped faces) any basis
    # serves the parity checks: a random orthonormal one
    K = 32
    if kind == "wild":
        q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((m.nv, K)))
        Phi = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    else:
        _, Phi, st = mcs.steklov_modes(mcs.cotan_laplacian(mesh), vrows["area"], K)
        assert st["status"] == 0
    S, Lb = mcs.galerkin_dtn(mesh, rows, res, Phi, exterior=bool(dom), killing_walks=kill, want_lambda=True)
    Lref = oracle.galerkin_lambda(m.V, m.F, est, rows_np, exterior=bool(dom), origin=o, row_face=rf,
                                  killing=bool(kill))
    Lb = Lb.cpu().numpy()
    assert np.abs(Lb - Lref).max() <= 1e-12 * np.abs(Lref).max()
    P = Phi.cpu().numpy()
    Sref = P.T @ Lref @ P
    scale = np.abs(P).T @ np.abs(Lref) @ np.abs(P)
    assert np.all(np.abs(S.cpu().numpy() - Sref) <= 2e-5 * scale)
    ev, Cm, psi = mcs.galerkin_modes(S, 16, Phi)
    evr = np.linalg.eigvalsh(S.cpu().numpy())
    assert np.abs(ev.cpu().numpy() - evr).max() <= 1e-10 * np.abs(evr).max()
    Cn = Cm.cpu().numpy()
    assert np.abs(Cn.T @ Cn - np.eye(K)).max() < 1e-10
    Sn = S.cpu().numpy()
    assert np.abs(Sn @ Cn - Cn * ev.cpu().numpy()[None, :]).max() <= 1e-9 * np.abs(evr).max()
    assert np.abs(psi.cpu().numpy() - P @ Cn[:, :16]).max() <= 1e-12 * np.abs(P).max() * K


def test_galerkin_sphere_spectrum():
    """Unit icosphere s3, interior, face sample rows at every face, W = 256:
    the Galerkin eigenvalues come in multiplets 1, 3, 5 with the l = 1 triple
    near the cap-corrected l/R (0.978 at 2.5 degrees)."""
    m = meshgen.icosphere(3)
    mesh = mcs.Mesh(m.V, m.F)
    vrows = mcs.vertex_rows(mesh)
    rows = mcs.sample_rows(mesh, m.nf, orient=False)
    res = mcs.estimate_dtn(mesh, rows, mcs.default_params(walks_per_row=256, prec=32, seed=1), record_exits=True,
                           record_bary=True)
    _, Phi, st = mcs.steklov_modes(mcs.cotan_laplacian(mesh), vrows["area"], 48)
    S = mcs.galerkin_dtn(mesh, rows, res, Phi)
    ev, _, _ = mcs.galerkin_modes(S, 9)
    ev = ev.cpu().numpy()
    # the constant mode: zero up to the split tensor-core product (~2^-20 of the
    # scale) and the basis' own accuracy (its constant to ~1e-5 of its bound)
    assert abs(ev[0]) < 1e-5 * abs(ev).max()
    assert ev[1:4].max() < ev[4:9].min()
    assert np.abs(ev[1:4] - 0.978).max() < 0.06
