"""Vertex rows of the unit icosphere under refinement, on the GPU.

The small sphere workload (icosphere s2 vertex rows) overestimates the
cap-corrected closed form lambda_l(theta0) of the sphere (Sec. 4.2 boxed
estimator; the cap of Sec. 5): a vertex of a convex polyhedron stands a
depth r - rho above its empty ball, and the excess tracks the jump mass
times that depth, which falls like h^2.  The oracle pins the trend at
subdivisions 2-4 (CPU); here the same estimator (bit-exact with the oracle
elsewhere) continues it to subdivisions 5 and 6: Rayleigh quotients of the
l = 1, 2 harmonics from the hit histograms (linear in Lambda, so unbiased in
the walk count), and at subdivision 5 the l = 1 and l = 2 eigenvalue
multiplets within 5% of the closed form."""
import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_05581_b300 as mcs  # noqa: E402


def _rayleigh_excess(res, rows, V, W, lam):
    """Mean relative excess of f' Lambda f / f' M f over lambda_l for f = z, x
    (l = 1) and x^2 - y^2, xy (l = 2), from the padded CSR: f' Lambda f =
    1/2 sum_v (omega_v / W) sum_u H_vu (f_v - f_u)^2."""
    R, cap = V.shape[0], res["cap"]
    nnz = res["hist_nnz"].long()
    mask = torch.arange(cap, device=nnz.device)[None, :] < nnz[:, None]
    # slots beyond hist_nnz are not written: index with bin 0 there (count 0)
    bins = torch.where(mask, res["hist_bin"].view(R, cap).long(), torch.zeros((), dtype=torch.long, device=nnz.device))
    assert int(bins.min()) >= 0 and int(bins.max()) < R
    cnt = res["hist_cnt"].view(R, cap).double() * mask
    om = res["omega"].double()
    P = torch.from_numpy(V).cuda()
    area = rows["area"]
    out = []
    for l, f in ((1, P[:, 2]), (1, P[:, 0]), (2, P[:, 0] ** 2 - P[:, 1] ** 2), (2, P[:, 0] * P[:, 1])):
        d = f[:, None] - f[bins]
        num = 0.5 * torch.sum(om[:, None] / W * cnt * d * d)
        out.append(float(num / torch.sum(area * f * f)) / lam[l] - 1.0)
    return float(np.mean(out)), out


def test_vertex_rows_converge_to_the_cap_corrected_spectrum(oracle):
    lam = oracle.sphere_eigs_cap(2, 2.5)
    W = 256
    gaps = {}
    for s in (4, 5, 6):
        m = meshgen.icosphere(s)
        mesh = mcs.Mesh(m.V, m.F)
        rows = mcs.vertex_rows(mesh)
        p = mcs.default_params(walks_per_row=W, prec=32, seed=0)
        res = mcs.estimate_dtn(mesh, rows, p, assemble=(s == 5))
        torch.cuda.synchronize()
        gaps[s], each = _rayleigh_excess(res, rows, m.V, W, lam)
        if s == 5:
            # the CSR form equals the quadratic form of the assembled Lambda
            f = torch.from_numpy(m.V[:, 2]).cuda()
            L = res["Lambda"]
            q = float(f @ (L @ f) / torch.sum(rows["area"] * f * f))
            assert abs(q / lam[1] - 1.0 - each[0]) < 1e-9
            ev, _, st = mcs.steklov_modes(L, rows["area"], 9, vectors=False)
            ev = ev.cpu().numpy()
            assert abs(ev[0]) <= 1e-5 * st["upper_bound"]  # the solver's stated accuracy
            rel1 = ev[1:4] / lam[1] - 1.0
            rel2 = ev[4:9] / lam[2] - 1.0
            assert np.all(np.abs(rel1) < 0.05) and np.all(np.abs(rel2) < 0.05), (rel1, rel2)
    assert gaps[4] > gaps[5] > gaps[6] > 0, gaps
    assert gaps[5] < 0.5 * gaps[4] and gaps[5] < 0.05 and gaps[6] < 0.02, gaps
