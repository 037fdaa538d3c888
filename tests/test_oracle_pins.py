"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form (ball Poisson / jump kernel, harmonic functions, the sphere's
DtN spectrum, the Kelvin-transformed point-charge potential), an independent
definition (projection optimality, greedy farthest-point order, the rank-1
update form of Alg. 2), or a distributional property (Philox uniformity,
Marsaglia directions, the jump-kernel importance density).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import meshgen


# --------------------------------------------------------------------------- philox / uniforms
def test_philox_uniform_bytes_and_bits(oracle):
    w = oracle.philox(0, 1 << 16, 7, 3, 0x123456789ABCDEF)
    b = w.view(np.uint8).ravel()
    hist = np.bincount(b, minlength=256)
    chi2 = ((hist - b.size / 256) ** 2 / (b.size / 256)).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 8)
    freq = bits.mean(0)
    assert np.all(np.abs(freq - 0.5) < 6 * 0.5 / math.sqrt(bits.shape[0]))
    x = w[:, 0].astype(np.float64)
    r = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(r) < 6 / math.sqrt(x.size)


def test_philox_counter_and_key_sensitivity(oracle):
    a = oracle.philox(100, 64, 0, 0, 1)
    b = oracle.philox(100, 64, 0, 1, 1)
    c = oracle.philox(100, 64, 0, 0, 2)
    assert len({tuple(r) for r in np.concatenate([a, b, c])}) == 192
    assert np.array_equal(a, oracle.philox(100, 64, 0, 0, 1))


# --------------------------------------------------------------------------- samplers
@pytest.mark.parametrize("prec", [64, 32])
def test_marsaglia_directions_are_uniform(oracle, prec):
    U = np.concatenate([oracle.directions(9, g, 64, prec) for g in range(400)])
    tol = 1e-15 if prec == 64 else 3e-7
    assert np.abs(np.linalg.norm(U, axis=1) - 1).max() < tol
    n = U.shape[0]
    assert np.all(np.abs(U.mean(0)) < 5 / math.sqrt(3 * n))
    Cm = U.T @ U / n
    assert np.abs(Cm - np.eye(3) / 3).max() < 5 * math.sqrt(4 / 45 / n)
    # Archimedes: each coordinate of a uniform direction is uniform on [-1, 1]
    for k in range(3):
        assert stats.kstest(U[:, k], "uniform", args=(-1, 2)).pvalue > 1e-4


@pytest.mark.parametrize("prec", [64, 32])
def test_jump_importance_sampler(oracle, prec):
    cap = 2.5
    c = np.array([0.1, -0.2, 0.3]); rho = 0.7; nrm = np.array([0.0, 0.6, 0.8])
    Z = oracle.start_points(11, cap, c, rho, nrm, 20000, prec)
    tol = 2e-15 if prec == 64 else 5e-7
    assert np.abs(np.linalg.norm(Z - c, axis=1) - rho).max() < tol
    p = c + rho * nrm
    cth = (Z - c) @ nrm / rho
    theta = np.arccos(np.clip(cth, -1, 1))
    assert theta.min() >= math.radians(cap) * (1 - 1e-5)
    # w = sin(theta/2) has density ~ 1/w^2 on [w0, 1]
    w = np.sqrt(np.clip((1 - cth) / 2, 0, 1))
    w0 = math.sin(math.radians(cap) / 2)
    cdf = lambda x: (1 / w0 - 1 / np.clip(x, w0, 1)) / (1 / w0 - 1)
    assert stats.kstest(w[::2], cdf).pvalue > 1e-4
    # antithetic partners: same |p - z|, azimuths opposite about the axis
    d = np.linalg.norm(Z - p, axis=1)
    assert np.abs(d[0::2] - d[1::2]).max() < 10 * tol
    perp = (Z - c) - np.outer((Z - c) @ nrm, nrm)
    assert np.abs(perp[0::2] + perp[1::2]).max() < 10 * tol
    # importance weight: M * E[g(z)] reproduces int_{theta>theta0} J^B(p,z) g(z) dz
    M = oracle.jump_mass(rho, cap)
    g = lambda th: np.cos(th) ** 2 + 0.5
    Jg = lambda th: g(th) * 2 * math.pi * rho ** 2 * math.sin(th) / (2 * math.pi * (2 * rho * math.sin(th / 2)) ** 3)
    exact = integrate.quad(Jg, math.radians(cap), math.pi, limit=200)[0]
    pairs = (M * g(theta)).reshape(-1, 2).mean(1)
    assert abs(pairs.mean() - exact) < 4 * pairs.std() / math.sqrt(pairs.size)


def test_jump_mass_matches_quadrature(oracle):
    """M_v returned by the C estimator equals int over the ball sphere outside the cap of
    J^B(p, z) = 1/(2 pi |p - z|^3) (Eq. ball-jump-kernel)."""
    m = meshgen.icosphere(2)
    rows = oracle.vertex_rows(m.V, m.F)
    est = oracle.estimate(m.V, m.F, rows, 2, 1e-3, row_list=[0, 5])
    assert est["discarded"].sum() == 0
    for li in range(2):
        rho = est["rho"][li]
        f = lambda th: 2 * math.pi * rho ** 2 * math.sin(th) / (2 * math.pi * (2 * rho * math.sin(th / 2)) ** 3)
        q = integrate.quad(f, math.radians(2.5), math.pi, limit=200)[0]
        assert abs(est["M"][li] - q) < 1e-9 * q


def test_ball_kernels_closed_forms(oracle):
    """The ball jump kernel is the inward normal derivative of the ball Poisson kernel
    (App. B.2): finite differences of P^B at s - h n reproduce 1/(2 pi |s - z|^3)."""
    c = np.array([0.3, -0.1, 0.2]); r = 0.8
    s = c + r * np.array([0, 0, 1.0]); n = np.array([0, 0, 1.0])
    z = c + r * np.array([math.sin(1.1), 0, math.cos(1.1)])
    for h in (1e-4, 1e-5):
        fd = oracle.ball_poisson(s - h * n, z, c, r) / h
        assert abs(fd - oracle.ball_jump(s, z)) < 5 * h * oracle.ball_jump(s, z) / r
    x = c + np.array([0.2, 0.1, -0.3])
    f = lambda th, ph: oracle.ball_poisson(x, c + r * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]), c, r) * r * r * math.sin(th)
    tot = integrate.dblquad(lambda ph, th: f(th, ph), 0, math.pi, 0, 2 * math.pi, epsabs=1e-9)[0]
    assert abs(tot - 1) < 1e-6


# --------------------------------------------------------------------------- closest point
def _rand_tris(rng, n):
    T = rng.normal(size=(n, 3, 3))
    k = n // 8
    T[:k, 2] = T[:k, 0] + 0.37 * (T[:k, 1] - T[:k, 0])      # collinear up to rounding
    T[k:2 * k, 1] = T[k:2 * k, 0]                            # repeated vertex
    T[2 * k:3 * k, 2] = T[2 * k:3 * k, 0] + 1e-7 * rng.normal(size=(k, 3)) + 0.5 * (T[2 * k:3 * k, 1] - T[2 * k:3 * k, 0])
    T[3 * k:3 * k + 8] = T[3 * k:3 * k + 8, :1]              # a point
    return T


@pytest.mark.parametrize("prec", [64, 32])
def test_closest_point_is_the_projection(oracle, prec):
    """q is the Euclidean projection of p onto the convex triangle T iff q in T and
    (p - q).(y - q) <= 0 for every y in T (enough: the three vertices)."""
    rng = np.random.default_rng(5)
    T = _rand_tris(rng, 400)
    P = rng.normal(size=(400, 3)) * 1.5
    tolr = 1e-9 if prec == 64 else 2e-3
    for i in range(400):
        V = T[i]; F = np.array([[0, 1, 2]], np.int32)
        d2, f, b = oracle.closest_points(V, F, P[i:i + 1], prec)
        assert f[0] == 0 and np.isfinite(d2[0])
        bb = b[0]
        assert bb.min() >= -1e-9 and abs(bb.sum() - 1) < 1e-6
        q = bb @ V
        scale = 1 + np.abs(V).max() + np.abs(P[i]).max()
        assert abs(d2[0] - np.sum((P[i] - q) ** 2)) < tolr * scale ** 2
        assert ((P[i] - q) @ (V - q).T).max() < tolr * scale ** 2
        assert d2[0] <= np.min(np.sum((V - P[i]) ** 2, 1)) * (1 + 1e-6) + 1e-12


def test_brute_force_argmin_lexicographic(oracle):
    m = meshgen.icosphere(2)
    rng = np.random.default_rng(3)
    P = rng.normal(size=(200, 3)) * 0.8
    P[:20] = 0.0  # the centre: many near-ties
    d2, f, _ = oracle.closest_points(m.V, m.F, P)
    one = np.array([[0, 1, 2]], np.int32)
    for i in range(0, 200, 7):
        per = np.array([oracle.closest_points(m.V[m.F[t]], one, P[i:i + 1])[0][0] for t in range(m.nf)])
        best = per.min()
        assert d2[i] == best
        assert f[i] == int(np.flatnonzero(per == best)[0])


# --------------------------------------------------------------------------- rows
def test_vertex_rows_areas_and_normals(oracle):
    m = meshgen.icosphere(3)
    rows = oracle.vertex_rows(m.V, m.F)
    a, b, c = (m.V[m.F[:, k]] for k in range(3))
    tri_area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    assert abs(rows["area"].sum() - tri_area.sum()) < 1e-12 * tri_area.sum()
    assert np.abs(np.linalg.norm(rows["nrm"], axis=1) - 1).max() < 1e-15
    assert np.min(np.einsum("ij,ij->i", rows["nrm"], m.V)) > 0.999


def test_fps_rows_are_greedy_farthest_points(oracle):
    m = meshgen.wild_union(4, 3000, seed=2, min_faces=200)
    r = oracle.fps_rows(m.V, m.F, 64, orient=False)
    cen = m.V[m.F].mean(1)
    sel = r["sel"]
    assert sel[0] == 0 and len(set(sel.tolist())) == 64
    # each choice is the farthest face up to single-precision rounding of the
    # squared distances (the sampling runs in float)
    for i in range(1, 64):
        dmin = np.min(np.sum((cen[:, None, :] - cen[sel[:i]][None]) ** 2, -1), 1)
        assert dmin[sel[i]] >= dmin.max() * (1 - 1e-5)
    owner = np.argmin(np.sum((cen[:, None, :] - cen[sel][None]) ** 2, -1), 1)
    assert np.mean(owner == r["tri2bin"]) > 0.999
    a, b, c = (m.V[m.F[:, k]] for k in range(3))
    tri_area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    assert abs(r["area"].sum() - tri_area.sum()) < 1e-10 * tri_area.sum()


def test_gwn_and_normal_repair(oracle):
    """Winding number 1 inside, 0 outside a closed outward surface (Jacobson et al. 2013);
    sample normals on faces flipped in the input are repaired outward (App. A item 1)."""
    m = meshgen.icosphere(2)
    assert abs(oracle.gwn(m.V, m.F, np.zeros(3)) - 1) < 1e-9
    assert abs(oracle.gwn(m.V, m.F, np.array([2.0, 0.3, 0.1]))) < 1e-9
    flipped = m.F.copy()
    flipped[::20, 1], flipped[::20, 2] = m.F[::20, 2], m.F[::20, 1]
    r = oracle.fps_rows(m.V, flipped, m.nf, orient=True)
    assert np.min(np.einsum("ij,ij->i", r["nrm"], r["pos"])) > 0.9
    r0 = oracle.fps_rows(m.V, flipped, m.nf, orient=False)
    assert np.sum(np.einsum("ij,ij->i", r0["nrm"], r0["pos"]) < 0) == len(range(0, m.nf, 20))


def _cube():
    V = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float64)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for a, b, c, d in quads:
        F += [(a, b, c), (a, c, d)]
    F = np.array(F, np.int32)
    cen = V[F].mean(1)
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return V, F


@pytest.mark.parametrize("kappa", [0.05, 1e-6])
def test_tangent_ball_bisection_on_a_cube(oracle, kappa):
    """Cube [-1,1]^3: rmax = 1 (half the shortest AABB side).  At the top-face centre the
    inscribed ball r = rho = 1; at (0.5, 0.5, 1) the distance from s - r n to the surface is
    min(0.5, r, 2 - r), so bisection accepts r <= 0.5/(1-kappa)."""
    V, F = _cube()
    rows = dict(pos=np.array([[0, 0, 1.0], [0.5, 0.5, 1.0]]), nrm=np.array([[0, 0, 1.0], [0, 0, 1.0]]))
    r, c, rho = oracle.tangent_balls(V, F, rows, params=dict(kappa=kappa))
    assert r[0] == 1.0 and rho[0] == 1.0
    lo, hi = 0.0, 1.0
    for _ in range(10):
        mid = 0.5 * (lo + hi)
        if min(0.5, mid, 2 - mid) >= (1 - kappa) * mid:
            lo = mid
        else:
            hi = mid
    assert r[1] == lo
    assert abs(rho[1] - min(0.5, lo)) < 1e-15


# --------------------------------------------------------------------------- walk-on-spheres
def test_wos_interior_harmonic_polynomials(oracle):
    """u(x) = E[g(B_tau)] (Eq. poisson-kernel-probabilistic): harmonic g is reproduced."""
    m = meshgen.icosphere(3)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(6, 3))
    X = X / np.linalg.norm(X, axis=1, keepdims=True) * rng.uniform(0.2, 0.8, (6, 1))
    P, tri, steps, capped = oracle.walk_from_points(m.V, m.F, X, 1200, 1e-4, seed=3)
    assert capped == 0
    for g in (lambda p: p[..., 0], lambda p: p[..., 0] ** 2 - p[..., 1] ** 2, lambda p: p[..., 0] * p[..., 1] + p[..., 2]):
        v = g(P)
        z = (v.mean(1) - g(X)) / (v.std(1) / math.sqrt(v.shape[1]))
        assert np.all(np.abs(z) < 4.0), z


def test_wos_exterior_point_charge(oracle):
    """Exterior Dirichlet data g(t) = 1/|t - o'| with o' inside Omega has the decaying
    solution u(x) = 1/|x - o'|.  Through the Kelvin transform (Eq. poisson-kernel-kelvin)
    u(x) = |x~| E[|t| g(t)], with t sampled by walks in the inverted domain."""
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = oracle.interior_origin(m.V, m.F, rows)
    X = np.array([[0.75, 0.3, 0.1], [-1.0, 0.2, 0.0], [1.5, 0.9, 0.0], [3.0, 1.0, 2.0]])
    op = np.array([1.6, 0.05, -0.1])
    P, tri, steps, capped = oracle.walk_from_points(m.V, m.F, X, 1500, 1e-4, exterior=True, origin=o, seed=5)
    assert capped == 0
    vals = np.linalg.norm(P - o, axis=-1) / np.linalg.norm(P - op, axis=-1)
    xt = np.linalg.norm(X - o, axis=-1)
    est = vals.mean(1) / xt
    se = vals.std(1) / math.sqrt(vals.shape[1]) / xt
    exact = 1 / np.linalg.norm(X - op, axis=-1)
    # faceting of the s2 spheres moves the boundary by O(h^2); allow 1%
    assert np.all(np.abs(est - exact) < 4 * se + 0.01 * exact), (est, exact, se)


# --------------------------------------------------------------------------- the estimator
def _quadform(rows, est, P, f, tn=None):
    d = f(rows["pos"])[:, None] - f(P)
    fac = rows["area"] * est["M"] * est["kfac"]
    vals = fac[:, None] * 0.5 * d ** 2 * (1.0 if tn is None else tn)
    pairs = vals.reshape(vals.shape[0], -1, 2).mean(-1).sum(0)  # one sample per antithetic pair index
    return pairs.mean(), pairs.std(ddof=1) / math.sqrt(pairs.size)


def test_interior_estimator_matches_sphere_closed_form(oracle):
    """With exact tangent balls (face-point rows, tiny slack), the estimator's quadratic
    form of Y_lm, evaluated at the walks' exit points, is the DtN jump form with the cap
    theta < theta0 removed: lambda_l(theta0) = int (1 - P_l) J 2 pi R^2 sin t dt."""
    m = meshgen.icosphere(3)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    est = oracle.estimate(m.V, m.F, rows, 48, 1e-4, seed=0, record_exits=True)
    P = oracle.exit_points(m.V, m.F, est["exit_tri"], est["exit_bary"])
    lam = oracle.sphere_eigs_cap(2, 2.5)
    assert abs(lam[1] - 0.9782) < 1e-3
    for f, nrm2, l in ((lambda p: p[..., 2], 4 * math.pi / 3, 1),
                       (lambda p: p[..., 0] ** 2 - p[..., 1] ** 2, 16 * math.pi / 15, 2)):
        E, se = _quadform(rows, est, P, f)
        assert abs(E / nrm2 - lam[l]) < 4 * se / nrm2 + 0.02 * lam[l], (E / nrm2, se / nrm2, lam[l])


def test_slack_on_face_rows_biases_the_estimator(oracle):
    """With a slack of 0.05 on face rows the pole p = c + rho n sinks a depth r - rho into
    the domain and the walks' self-jumps inflate the form by ~M (r - rho): the reason the
    strict test is used on face-interior rows."""
    m = meshgen.icosphere(2)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    est = oracle.estimate(m.V, m.F, rows, 32, 1e-4, seed=0, record_exits=True, params=dict(kappa=0.05))
    P = oracle.exit_points(m.V, m.F, est["exit_tri"], est["exit_bary"])
    E, se = _quadform(rows, est, P, lambda p: p[..., 2])
    assert E / (4 * math.pi / 3) > 1.3 * oracle.sphere_eigs_cap(1, 2.5)[1]


def test_sphere_cap_spectrum_limits(oracle):
    lam0 = oracle.sphere_eigs_cap(6, 1e-6)
    assert np.allclose(lam0, np.arange(7), atol=2e-5)
    lam = oracle.sphere_eigs_cap(6, 2.5)
    l = np.arange(7)
    approx = l - l * (l + 1) * math.radians(2.5) / 4
    assert np.allclose(lam, approx, atol=5e-3)


def test_exterior_estimator_sphere_jump_and_killing(oracle):
    """Exterior of a sphere of radius R centred at the inversion centre: the jump kernel
    is 1/(2 pi |s-t|^3) (Eq. exterior-jump-kernel-final) so the jump form gives the
    interior values l/R (cap-corrected), and the killing measure K = 1/R (escape
    probability 1 - R/|x|) adds 1/R: (l + 1)/R.  Total killing mass 4 pi R."""
    R = 0.5
    m = meshgen.icosphere(3, R)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    est = oracle.estimate(m.V, m.F, rows, 48, 1e-4, exterior=True, origin=(0, 0, 0), seed=1,
                          record_exits=True, killing_walks=20000)
    P = oracle.exit_points(m.V, m.F, est["exit_tri"], est["exit_bary"])
    tn = np.linalg.norm(P, axis=-1)
    lam = oracle.sphere_eigs_cap(2, 2.5, R)
    for f, nrm2, l in ((lambda p: p[..., 2] / R, 4 * math.pi / 3 * R * R, 1),
                       (lambda p: (p[..., 0] ** 2 - p[..., 1] ** 2) / R ** 2, 16 * math.pi / 15 * R * R, 2)):
        E, se = _quadform(rows, est, P, f, tn)
        # s3 faceting at R = 0.5 is visible in the exterior (it converges at s4); 10%
        assert abs(E / nrm2 - lam[l]) < 4 * se / nrm2 + 0.10 * lam[l], (E / nrm2, se / nrm2, lam[l])
    cf = np.linalg.norm(rows["pos"], axis=1)
    k = 4 * math.pi * cf * est["H0"] / est["killing_walks"]
    assert abs(k.sum() - 4 * math.pi * R) < 0.01 * 4 * math.pi * R
    f = rows["pos"][:, 2] / R
    assert abs((k * f * f).sum() / (4 * math.pi / 3 * R * R) - 1 / R) < 0.05 / R


def test_estimator_invariants_and_assembly(oracle):
    """Sum_u H_vu = W (every walk lands once); Lambda = L(Wsym) equals the paper's sum of
    rank-1 updates (A_v M_v / 2W) d d^T, d = e_v - e_u (Alg. 2 last line); symmetric,
    Lambda 1 = 0, PSD (Sec. 4.2 'Guaranteeing a PSD estimate'); the sphere's spectrum comes
    in multiplets 1, 3, 5."""
    m = meshgen.icosphere(2)
    rows = oracle.vertex_rows(m.V, m.F)
    est = oracle.estimate(m.V, m.F, rows, 128, 1e-3, seed=0)
    H = est["H"]
    assert np.all(H.sum(1) == 128) and est["discarded"].sum() == 0
    L = oracle.assemble(est, rows)
    n = L.shape[0]
    S = np.zeros((n, n))
    w = rows["area"] * est["M"] / 128
    for v in range(n):
        for u in np.flatnonzero(H[v]):
            d = np.zeros(n); d[v] += 1; d[u] -= 1
            S += 0.5 * w[v] * H[v, u] * np.outer(d, d)
    assert np.abs(L - S).max() < 1e-12 * np.abs(S).max()
    assert np.array_equal(L, L.T)
    assert np.abs(L @ np.ones(n)).max() < 1e-12 * np.abs(L).max()
    ev = np.linalg.eigvalsh(L)
    assert ev.min() > -1e-12 * np.abs(L).max()
    lam, _ = oracle.steklov(L, rows["area"], 9)
    assert abs(lam[0]) < 1e-10
    g1, g2 = lam[1:4], lam[4:9]
    assert g1.max() < g2.min()
    assert (g1.max() - g1.min()) < 0.2 * g1.mean() and (g2.max() - g2.min()) < 0.2 * g2.mean()


def test_steklov_solver_against_generalized_eigh(oracle):
    from scipy.linalg import eigh
    rng = np.random.default_rng(0)
    A = rng.random((40, 40)); Ws = 0.5 * (A + A.T); np.fill_diagonal(Ws, 0)
    L = np.diag(Ws.sum(1)) - Ws
    M = rng.uniform(0.5, 2, 40)
    lam, X = oracle.steklov(L, M, 6)
    ref = eigh(L, np.diag(M), eigvals_only=True)[:6]
    assert np.allclose(lam, ref, rtol=1e-10, atol=1e-12)
    assert np.allclose(L @ X, (M[:, None] * X) * lam[None, :], atol=1e-9)


def test_fp32_mode_agrees_statistically_with_fp64(oracle):
    """Common random numbers: FP32 walks follow the FP64 walks' draws, so the spectra of
    the two estimates agree closely."""
    m = meshgen.icosphere(2)
    rows = oracle.vertex_rows(m.V, m.F)
    e64 = oracle.estimate(m.V, m.F, rows, 64, 1e-3, seed=4, prec=64)
    e32 = oracle.estimate(m.V, m.F, rows, 64, 1e-3, seed=4, prec=32)
    assert np.all(e32["H"].sum(1) == 64)
    l64, _ = oracle.steklov(oracle.assemble(e64, rows), rows["area"], 16)
    l32, _ = oracle.steklov(oracle.assemble(e32, rows), rows["area"], 16)
    assert np.allclose(l32, l64, rtol=0.05, atol=1e-9)
    assert np.mean(e32["H"] == e64["H"]) > 0.9


@pytest.mark.parametrize("prec", [64, 32])
def test_exterior_walks_stay_in_the_exterior(oracle, prec):
    """Every exterior walk ends on the surface within the step cap: the inverted tangent
    balls stay inside the Kelvin image of the exterior, so no walk starts in (or leaks
    into) the image of the interior, where inverted walks drift off to infinity."""
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = oracle.interior_origin(m.V, m.F, rows)
    est = oracle.estimate(m.V, m.F, rows, 16, 1e-3, exterior=True, origin=o, seed=3, prec=prec,
                          record_exits=True, killing_walks=512)
    assert est["capped"].sum() == 0 and est["kill_stats"][1] == 0
    assert np.all(est["exit_tri"][est["discarded"] == 0] >= 0)
    # the inverted balls exclude the inversion centre: |c~| > rho~
    ok = est["discarded"] == 0
    assert np.all(np.linalg.norm(est["center"][ok], axis=1) > est["rho"][ok])


@pytest.mark.parametrize("prec", [64, 32])
def test_exterior_walks_in_the_origin_component_escape(oracle, prec):
    """Reading R17.  Nested spheres A (R = 1) and B (R = 0.3), both outward,
    inversion centre in the gap between them.  Exterior walks of A's rows live
    in the true exterior: none is retired.  B's rows face the gap, a bounded
    component that contains the centre: its Kelvin image is unbounded, and
    walks that wander towards the centre are retired as escaped instead of
    running to the step cap (FP64) or overflowing (FP32).  Every walk ends:
    with a hit or escaped, none capped."""
    A = meshgen.icosphere(3, 1.0)
    B = meshgen.icosphere(3, 0.3)
    V = np.concatenate([A.V, B.V])
    F = np.concatenate([A.F, B.F + A.nv])
    rows = oracle.vertex_rows(V, F)
    W = 16
    est = oracle.estimate(V, F, rows, W, 1e-3, exterior=True, origin=np.array([0.65, 0.0, 0.0]), seed=5,
                          prec=prec)
    nA = A.nv
    lost, capped, disc = est["lost"], est["capped"], est["discarded"].astype(bool)
    assert capped.sum() == 0
    assert lost[:nA].sum() == 0
    assert lost[nA:].sum() > 0
    kept = ~disc
    assert np.array_equal(est["H"].sum(1)[kept] + lost[kept], np.full(kept.sum(), W))


@pytest.mark.parametrize("prec", [64, 32])
def test_interior_walks_in_the_unbounded_component_are_retired(oracle, prec):
    """Reading R18.  An inside-out sphere: every row's inward normal points out,
    so the interior walks start in the unbounded component.  3-D Brownian
    motion is transient; the walks that wander off are retired once they are
    farther from the box centre than the box diagonal, instead of running to
    the step cap (FP64) or overflowing (FP32).  Every walk ends: hit or
    retired, none capped; a right-side-out sphere retires none."""
    m = meshgen.icosphere(3, 1.0)
    flipped = m.F[:, ::-1].copy()
    W = 16
    for F, inside_out in ((flipped, True), (m.F, False)):
        rows = oracle.vertex_rows(m.V, F)
        est = oracle.estimate(m.V, F, rows, W, 1e-3, seed=3, prec=prec)
        lost, capped = est["lost"], est["capped"]
        assert capped.sum() == 0
        assert (lost.sum() > 0) == inside_out
        kept = ~est["discarded"].astype(bool)
        assert np.array_equal(est["H"].sum(1)[kept] + lost[kept], np.full(kept.sum(), W))


def test_exterior_start_balls_touch_their_rows(oracle):
    """The tangent-ball decomposition (Sec. 4.2, applied in the inverted domain
    by Sec. 4.3) needs a ball tangent to the inverted surface at s~.  With the
    slack kappa the accepted start ball B(c~, rho~) is empty, has rho~ >=
    (1 - kappa) r and passes within kappa r of s~ (r: the bisected inverted
    radius).  Two spheres, one holding the inversion centre: the rows of the
    near sphere that face the other one are where a slack on the primal
    image radius let the ball reach across the gap."""
    kappa = 0.05
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = np.zeros(3)
    est = oracle.estimate(m.V, m.F, rows, 2, 1e-3, exterior=True, origin=o, seed=1,
                          params=dict(kappa=kappa))
    assert est["discarded"].sum() == 0
    sp = rows["pos"] - o
    st = sp / np.einsum("ij,ij->i", sp, sp)[:, None]
    r, rho = est["r_t"], est["rho"]
    gap = np.linalg.norm(st - est["center"], axis=1) - rho
    assert np.all(r > 0)
    assert np.all(gap >= -1e-9 * r)
    assert np.all(gap <= kappa * r * (1 + 1e-9))
    assert np.all(rho >= (1 - kappa) * r * (1 - 1e-9))


def test_exterior_jump_mass_between_components_is_symmetric(oracle):
    """J(s, t) = J(t, s) (Eq. exterior-jump-kernel-final), so the jump mass from
    sphere A to sphere B equals that from B to A.  Two spheres (R = 0.5,
    centres 1.5 apart), inversion centre at A's centre; the 2.5 degree cap
    reaches neither sphere from the other at this gap, so both sums estimate
    the same integral.  A vertex-row bias of order 20% remains at s2; the
    tolerance allows it and the noise of ~200 cross hits."""
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = np.zeros(3)
    W = 256
    est = oracle.estimate(m.V, m.F, rows, W, 1e-3, exterior=True, origin=o, seed=1)
    a = rows["pos"][:, 0] < 0.75
    Wm = (oracle.row_weights(est, rows)[:, None] * est["H"] / W
          * oracle.column_factor(rows, True, o)[None, :])
    ab, ba = Wm[np.ix_(a, ~a)].sum(), Wm[np.ix_(~a, a)].sum()
    assert est["H"][np.ix_(a, ~a)].sum() > 100
    assert 2 / 3 < ab / ba < 1.5, (ab, ba)


def test_exterior_killing_mass_of_two_spheres_is_their_capacitance(oracle, two_sphere_capacitance):
    """The killing measure is the normal derivative of the escape probability
    (Eq. killing-measure-normal-derivative), so its total is the flux of the
    equilibrium potential: 4 pi C, with C the capacitance of the surface
    (4 pi R for one sphere).  Two spheres of radius 0.5, centres 1.5 apart,
    inversion centre at one of them: C by the method of images; by symmetry
    each sphere carries half of it, although only one holds the centre
    (Eq. killing-measure-poisson-kernel)."""
    m = meshgen.two_spheres(2, 0.5, 1.5)
    rows = oracle.vertex_rows(m.V, m.F)
    o = np.zeros(3)
    N = 20000
    est = oracle.estimate(m.V, m.F, rows, 2, 1e-3, exterior=True, origin=o, seed=1, killing_walks=N)
    assert est["kill_stats"][1] == 0 and est["kill_stats"][2] == 0
    k = 4 * math.pi * oracle.column_factor(rows, True, o) * est["H0"] / N
    ref = 4 * math.pi * two_sphere_capacitance(0.5, 1.5)
    assert abs(k.sum() / ref - 1) < 0.03, k.sum() / ref
    a = rows["pos"][:, 0] < 0.75
    assert abs(k[a].sum() / k.sum() - 0.5) < 0.03


def _dtn_like(n, seed):
    """A symmetric Lambda with zero row sums and non-negative off-diagonal
    weights (the assembled form), positive lumped masses."""
    rng = np.random.default_rng(seed)
    W = rng.random((n, n)) * (rng.random((n, n)) < 0.3)
    W = 0.5 * (W + W.T)
    np.fill_diagonal(W, 0.0)
    L = np.diag(W.sum(1)) - W
    mass = 0.5 + rng.random(n)
    return L, mass


def test_steklov_heat_equals_the_matrix_exponential(oracle):
    """Eq. steklovHeat, du/dt = -Lambda u in the M inner product: with the
    full generalized eigenbasis the spectral sum of Eq. spectralSteklovHeat
    equals expm(-t M^-1 Lambda) u0 (scipy's Pade exponential)."""
    from scipy.linalg import eigh, expm
    n = 40
    L, mass = _dtn_like(n, 3)
    ev, psi = eigh(L, np.diag(mass))
    u0 = np.random.default_rng(4).standard_normal((n, 3))
    times = [0.0, 0.05, 0.7, 3.0]
    got = oracle.steklov_heat(ev, psi, mass, u0, times)
    for i, t in enumerate(times):
        ref = expm(-t * (L / mass[:, None])) @ u0
        assert np.abs(got[i] - ref).max() < 1e-10 * max(1.0, np.abs(ref).max()), t


def test_steklov_heat_conserves_total_heat_with_the_constant_mode(oracle):
    """Interior Lambda annihilates constants, so the constant is the lambda = 0
    mode; every other mode is M-orthogonal to it, so sum_x m_x u_t(x) stays
    sum_x m_x u0(x) for any truncation that keeps the constant mode."""
    from scipy.linalg import eigh
    n = 50
    L, mass = _dtn_like(n, 5)
    ev, psi = eigh(L, np.diag(mass))
    u0 = np.zeros(n)
    u0[7] = 1.0  # a unit impulse at one node
    for k in (1, 5, 20):
        u = oracle.steklov_heat(ev[:k], psi[:, :k], mass, u0, [0.1, 1.0, 10.0])
        assert np.allclose(u @ mass, mass[7], rtol=1e-12, atol=0), k


def test_hks_diagonal_and_trace(oracle):
    """With the complete M-orthonormal basis, sum_j psi_j(x)^2 = 1/m_x (the
    diagonal of M^-1), so HKS(x, 0) = 1/m_x; and sum_x m_x HKS(x, t) is the heat
    trace sum_j exp(-lambda_j t)."""
    from scipy.linalg import eigh
    n = 30
    L, mass = _dtn_like(n, 6)
    ev, psi = eigh(L, np.diag(mass))
    h = oracle.hks(ev, psi, [0.0, 0.3, 2.0])
    assert np.allclose(h[0], 1.0 / mass, rtol=1e-10)
    for i, t in enumerate([0.0, 0.3, 2.0]):
        assert np.isclose(h[i] @ mass, np.exp(-ev * t).sum(), rtol=1e-10)


def test_cotan_laplacian_properties(oracle):
    """The cotangent Laplacian is symmetric with zero row sums; it is exact on
    linear functions at interior vertices of a planar mesh (linear
    precision); on the unit icosphere its smallest generalized eigenvalues
    with lumped vertex areas approach l(l+1) = 0, 2 (x3), 6 (x5)."""
    from scipy.linalg import eigh
    # planar: a jittered 9 x 9 grid of the unit square, two triangles per cell
    rng = np.random.default_rng(2)
    g = 9
    xs, ys = np.meshgrid(np.linspace(0, 1, g), np.linspace(0, 1, g), indexing="ij")
    P = np.stack([xs.ravel(), ys.ravel(), np.zeros(g * g)], 1)
    inner = (xs.ravel() > 0) & (xs.ravel() < 1) & (ys.ravel() > 0) & (ys.ravel() < 1)
    P[inner, :2] += 0.02 * rng.standard_normal((inner.sum(), 2))
    idx = np.arange(g * g).reshape(g, g)
    F = []
    for i in range(g - 1):
        for j in range(g - 1):
            a, b, c, d = idx[i, j], idx[i + 1, j], idx[i + 1, j + 1], idx[i, j + 1]
            F += [[a, b, c], [a, c, d]]
    L = oracle.cotan_laplacian(P, np.array(F))
    assert np.allclose(L, L.T, atol=1e-14) and np.allclose(L.sum(1), 0, atol=1e-12)
    for f in (P[:, 0], P[:, 1], 2 * P[:, 0] - 3 * P[:, 1] + 0.5):
        assert np.abs((L @ f)[inner]).max() < 1e-12
    m = meshgen.icosphere(3)
    rows = oracle.vertex_rows(m.V, m.F)
    mu = eigh(oracle.cotan_laplacian(m.V, m.F), np.diag(rows["area"]), eigvals_only=True)[:9]
    ref = np.array([0, 2, 2, 2, 6, 6, 6, 6, 6.0])
    assert abs(mu[0]) < 1e-10 and np.abs(mu[1:] - ref[1:]).max() < 0.03 * 6


def test_galerkin_quadratic_form_of_linear_functions(oracle):
    """Barycentric interpolation reproduces linear functions exactly, so for a
    linear f the hat-basis Galerkin form f^T Lambda_bary f equals the jump
    form sum_walks w (f(s) - f(t))^2 summed over the exit points t in space
    (Sec. 4.4 with the boxed estimators), for vertex and sample rows, interior
    and exterior; on the unit sphere it approaches the cap-corrected l = 1
    value (Funk-Hecke) for f = z.  With one-hot barycentrics at the bin
    vertex the Galerkin matrix is exactly the nodal Lambda (symmetrised
    histogram assembly)."""
    R = 1.0
    m = meshgen.icosphere(2, R)
    lam = oracle.sphere_eigs_cap(1, 2.5, R)
    for kind in ("vertex", "sample"):
        rows = oracle.vertex_rows(m.V, m.F) if kind == "vertex" else oracle.fps_rows(m.V, m.F, m.nf, orient=False)
        rf = None if kind == "vertex" else rows["sel"]
        for ext in (False, True):
            o = np.zeros(3)
            est = oracle.estimate(m.V, m.F, rows, 64, 1e-3, exterior=ext, origin=o, seed=2, record_exits=True)
            L = oracle.galerkin_lambda(m.V, m.F, est, rows, exterior=ext, origin=o, row_face=rf)
            W = est["walks"]
            omega = oracle.row_weights(est, rows)
            P = oracle.exit_points(m.V, m.F, est["exit_tri"], est["exit_bary"])
            ok = est["exit_tri"] >= 0
            for f3 in (np.array([0, 0, 1.0]), np.array([0.3, -1.0, 0.2])):
                f = m.V @ f3
                fs = rows["pos"] @ f3
                ft = P @ f3
                w = np.where(ok, 0.5 * omega[:, None] / W, 0.0)
                if ext:
                    w = w * np.linalg.norm(P - o, axis=-1)
                E = float(np.sum(w * (fs[:, None] - ft) ** 2))
                assert abs(f @ L @ f - E) <= 1e-10 * E, (kind, ext)
            if kind == "vertex":
                est1 = dict(est)
                eb = np.zeros_like(est["exit_bary"])
                tri = np.maximum(est["exit_tri"], 0)
                vb = m.F[tri]                                   # R x W x 3
                # the bin is the vertex with the largest barycentric (ties -> lower vertex id)
                best = est["exit_bary"].max(-1, keepdims=True)
                cand = np.where(est["exit_bary"] == best, vb, np.iinfo(np.int32).max)
                binv = cand.min(-1)
                eb[vb == binv[..., None]] = 1.0
                est1["exit_bary"] = eb
                L1 = oracle.galerkin_lambda(m.V, m.F, est1, rows, exterior=ext, origin=o)
                Ln = oracle.assemble(est, rows, exterior=ext, origin=o)
                assert np.abs(L1 - Ln).max() <= 1e-12 * np.abs(Ln).max(), (kind, ext)
            if not ext and kind == "sample":
                f = m.V[:, 2]
                Mf = np.sum(rows["area"] * rows["pos"][:, 2] ** 2)
                assert abs((f @ L @ f) / Mf - lam[1]) < 0.12 * lam[1]


def test_uniform_ball_weights_have_mean_one(oracle):
    """Start mode 1 samples cos(theta) uniformly outside the cap and weights
    each walk by q = |dB outside the cap| J^B(p, z) / M, whose mean is exactly
    1 (so the weighted estimator has the importance sampler's expectation);
    Var(q) = (1 - w0^2)(w0^-4 - 1) / (8 (1/w0 - 1)^2) - 1 sets the tolerance."""
    m = meshgen.icosphere(3)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    est = oracle.estimate(m.V, m.F, rows, 64, 1e-3, seed=4, record_exits=True, params=dict(start_mode=1))
    q = est["walk_w"][est["exit_tri"] >= 0]
    w0 = math.sin(math.radians(2.5) / 2)
    var = (1 - w0 ** 2) * (w0 ** -4 - 1) / (8 * (1 / w0 - 1) ** 2) - 1
    assert abs(q.mean() - 1) < 5 * math.sqrt(var / q.size), (q.mean(), q.size)
    assert q.min() > 0 and q.max() <= (1 - w0 ** 2) / (2 * w0 ** 3 * (1 / w0 - 1)) * (1 + 1e-9)
    est0 = oracle.estimate(m.V, m.F, rows, 8, 1e-3, seed=4, record_exits=True)
    assert np.all(est0["walk_w"] == 1.0)


def test_naive_estimator_is_unbiased_for_linear_functions(oracle):
    """Alg. 1 on the hat basis: a linear f is its own harmonic extension, so
    E f(t) = f(s - h n_s) exactly and the naive form's expectation is
    sum_s A_s f(s) (f(s) - f(s - h n_s)) / h, computed here directly (equal
    to int f df/dn up to the quadrature).  The estimate agrees within its
    Monte Carlo error."""
    m = meshgen.icosphere(3)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    h = 0.02
    W = 64
    est = oracle.estimate(m.V, m.F, rows, W, 1e-4, seed=6, record_exits=True,
                          params=dict(start_mode=2, inset=h))
    assert est["discarded"].sum() == 0
    assert np.allclose(est["M"], 1.0 / h)
    L = oracle.galerkin_lambda(m.V, m.F, est, rows, row_face=rows["sel"], form="naive")
    P = oracle.exit_points(m.V, m.F, est["exit_tri"], est["exit_bary"])
    for f3 in (np.array([0, 0, 1.0]), np.array([0.4, 0.5, -0.2])):
        f = m.V @ f3
        fs = rows["pos"] @ f3
        ref = float(np.sum(rows["area"] * fs * (fs - (rows["pos"] - h * rows["nrm"]) @ f3) / h))
        got = float(f @ L @ f)
        # per-walk terms A_s f(s) (f(s) - f(t)) / (W h); their spread sets the error
        terms = rows["area"][:, None] * fs[:, None] * (fs[:, None] - P @ f3) / (W * h)
        se = math.sqrt(terms.shape[0] * W * terms.var())
        assert abs(got - ref) < 5 * se + 1e-3 * abs(ref), (got, ref, se)


# ---------------------------------------------------------------------------
# point-based Galerkin basis (Sec. 4.4; appendix "Point-based k-NN Interpolator")
# ---------------------------------------------------------------------------

def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    ph = i * math.pi * (3 - math.sqrt(5))
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)


def test_knn_matches_kdtree(oracle):
    """Brute-force k nearest points = scipy's k-d tree (distinct distances),
    and the self-exclusion drops exactly the query's own point."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(0)
    P = rng.standard_normal((700, 3))
    Q = rng.standard_normal((300, 3))
    idx, d2 = oracle.knn(P, Q, 8)
    dd, jj = cKDTree(P).query(Q, 8)
    assert np.array_equal(idx, jj)
    assert np.abs(np.sqrt(d2) - dd).max() <= 1e-14
    idx, _ = oracle.knn(P, P, 5, exclude=np.arange(700))
    _, jj = cKDTree(P).query(P, 6)
    assert np.array_equal(idx, jj[:, 1:])
    # equal distances: the smaller index first
    G = np.array([[1.0, 0, 0], [0, 1.0, 0], [-1.0, 0, 0], [0, -1.0, 0], [3.0, 0, 0]])
    idx, _ = oracle.knn(G[::-1].copy(), np.zeros((1, 3)), 4)
    assert list(idx[0]) == [1, 2, 3, 4]


def test_bilateral_weights_special_cases(oracle):
    """The interpolator's weights sum to one; they are uniform when both
    falloffs are switched off and when the neighbours are equidistant with one
    normal; a point at distance sigma weighs e^(-1/2) against one at the query,
    and an opposite normal e^(-2/tau_n) against an aligned one (the scales of
    the two factors); with a tiny sigma the query's own point takes it all."""
    rng = np.random.default_rng(1)
    P = rng.standard_normal((200, 3))
    NP = rng.standard_normal((200, 3))
    NP /= np.linalg.norm(NP, axis=1, keepdims=True)
    Q = rng.standard_normal((50, 3))
    NQ = NP[:50]
    idx, w = oracle.knn_bilateral(P, NP, Q, NQ, 8, 0.5, 0.8)
    assert np.abs(w.sum(1) - 1).max() <= 1e-15 * 8
    _, w = oracle.knn_bilateral(P, NP, Q, NQ, 8, 1e8, 1e16)
    assert np.abs(w - 1 / 8).max() <= 1e-12
    ang = 2 * math.pi * np.arange(6) / 6
    ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], 1)
    up = np.tile([0, 0, 1.0], (6, 1))
    _, w = oracle.knn_bilateral(ring, up, np.zeros((1, 3)), up[:1], 6, 0.3, 0.8)
    assert np.abs(w - 1 / 6).max() <= 1e-15
    sig = 0.2
    two = np.array([[0, 0, 0], [sig, 0, 0]], float)
    _, w = oracle.knn_bilateral(two, up[:2], np.zeros((1, 3)), up[:1], 2, sig, 0.8)
    assert abs(w[0, 1] / w[0, 0] - math.exp(-0.5)) <= 1e-15
    sym = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    nrm = np.array([[0, 0, 1.0], [0, 0, -1.0]])
    _, w = oracle.knn_bilateral(sym, nrm, np.zeros((1, 3)), nrm[:1], 2, 1.0, 0.8)
    assert abs(w[0, 1] / w[0, 0] - math.exp(-2 / 0.8)) <= 1e-15
    idx, w = oracle.knn_bilateral(P, NP, P[:20], NP[:20], 8, 1e-3, 0.8)
    assert np.array_equal(idx[:, 0], np.arange(20)) and np.abs(w[:, 0] - 1).max() <= 1e-15


def test_point_laplacian_is_the_planar_voronoi_dual(oracle):
    """On a jittered planar grid (one normal) every inner point's local cell is
    its Voronoi cell: the areas and the weights |Voronoi edge| / |x_i - x_j|
    equal scipy's Voronoi diagram, and L reproduces linear functions."""
    from scipy.spatial import ConvexHull, Voronoi
    rng = np.random.default_rng(0)
    g = 14
    xy = np.stack(np.meshgrid(np.arange(g), np.arange(g), indexing="ij"), -1).reshape(-1, 2) * 0.1
    xy = xy + rng.uniform(-0.03, 0.03, xy.shape)
    P = np.concatenate([xy, np.zeros((len(xy), 1))], 1)
    L, area, _, _ = oracle.point_laplacian(P, np.tile([0, 0, 1.0], (len(P), 1)), 16)
    vor = Voronoi(xy)
    inner = {i for i in range(len(xy)) if 3 <= i // g < g - 3 and 3 <= i % g < g - 3}
    nchk = 0
    for i in inner:
        A = ConvexHull(vor.vertices[vor.regions[vor.point_region[i]]]).volume
        assert abs(A - area[i]) <= 1e-12 * A
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if a in inner and b in inner and -1 not in rv:
            ratio = np.linalg.norm(vor.vertices[rv[0]] - vor.vertices[rv[1]]) / np.linalg.norm(xy[a] - xy[b])
            assert abs(-L[a, b] - ratio) <= 1e-12 * max(ratio, 1.0)
            nchk += 1
    assert nchk > 150
    assert np.array_equal(L, L.T)
    ii = sorted(inner)
    for f in (P[:, 0], P[:, 1], 0.3 * P[:, 0] - 2.0 * P[:, 1]):
        assert np.abs((L @ f)[ii]).max() <= 1e-12 * np.abs(L).max()
    assert np.abs(L.sum(1)).max() <= 1e-12 * np.abs(L).max()


def test_point_laplacian_sphere_spectrum(oracle):
    """800 Fibonacci points on the unit sphere, normals = positions, mass
    4 pi / n: the generalised eigenvalues approach l (l + 1) with
    multiplicities 1, 3, 5, 7 (to 2%: the O(h^2) discretisation error at
    h^2 ~ 4 pi / n)."""
    import scipy.linalg as sl
    n = 800
    S = _fibonacci_sphere(n)
    L, area, _, _ = oracle.point_laplacian(S, S, 16)
    assert abs(area.sum() - 4 * math.pi) < 0.01 * 4 * math.pi
    ev = sl.eigh(L, np.diag(np.full(n, 4 * math.pi / n)), eigvals_only=True)[:16]
    assert abs(ev[0]) < 1e-10
    for lo, hi, l in ((1, 4, 1), (4, 9, 2), (9, 16, 3)):
        assert np.abs(ev[lo:hi] - l * (l + 1)).max() < 0.02 * l * (l + 1)


def test_point_galerkin_lambda_properties(oracle):
    """Point-basis Galerkin matrix on the unit icosphere (face sample rows as
    the point set, W = 64): symmetric positive semidefinite, constants in its
    null space (both interpolators are partitions of unity), and the Rayleigh
    quotient of z near the cap-corrected l = 1 value (Funk-Hecke); exterior
    walks (origin at the centre, with killing walks) keep the same
    structure."""
    m = meshgen.icosphere(2)
    rows = oracle.fps_rows(m.V, m.F, m.nf, orient=False)
    lam = oracle.sphere_eigs_cap(1, 2.5, 1.0)
    est = oracle.estimate(m.V, m.F, rows, 64, 1e-3, seed=2, record_exits=True)
    L = oracle.point_galerkin_lambda(m.V, m.F, est, rows, rows["pos"], rows["nrm"], sigma=0.1)
    sc = np.abs(L).max()
    assert np.abs(L - L.T).max() <= 1e-14 * sc
    assert np.abs(L.sum(1)).max() <= 1e-13 * sc
    assert np.linalg.eigvalsh(L).min() >= -1e-13 * sc
    z = rows["pos"][:, 2]
    assert abs((z @ L @ z) / np.sum(rows["area"] * z * z) - lam[1]) < 0.12 * lam[1]
    est = oracle.estimate(m.V, m.F, rows, 64, 1e-3, exterior=True, origin=np.zeros(3), seed=2, record_exits=True,
                          killing_walks=4096)
    Le = oracle.point_galerkin_lambda(m.V, m.F, est, rows, rows["pos"], rows["nrm"], exterior=True,
                                      origin=np.zeros(3), killing=True, sigma=0.1)
    assert np.abs(Le - Le.T).max() <= 1e-14 * np.abs(Le).max()
    assert np.linalg.eigvalsh(Le).min() >= -1e-13 * np.abs(Le).max()
    # exterior of the unit sphere: the constant is not in the null space (the
    # killing walks carry it: l = 0 exterior eigenvalue 1)
    one = np.ones(len(z))
    assert (one @ Le @ one) / rows["area"].sum() > 0.5


# --------------------------------------------------------------------------- inversion centre (Sec. 4.3)
def _gwn_numpy(V, F, q):
    """Generalized winding number (Jacobson et al. 2013) at q: the signed solid
    angles of the triangles (van Oosterom and Strackee 1983) over 4 pi."""
    a, b, c = (V[F[:, k]] - q for k in range(3))
    la, lb, lc = (np.linalg.norm(x, axis=1) for x in (a, b, c))
    det = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = (la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", b, c) * la
           + np.einsum("ij,ij->i", c, a) * lb)
    return float(np.sum(2.0 * np.arctan2(det, den)) / (4.0 * math.pi))


@pytest.mark.parametrize("which", ["two_spheres", "wild"])
def test_interior_origin_lies_inside_the_shape(oracle, which):
    """The Kelvin transform needs its centre inside Omega (Sec. 4.3: 0 in Omega by
    translation).  The chosen centre (reading R14: the centre of the largest interior
    tangent ball of a strided row subset) has winding number >= 1 (inside at least one
    component of a union), a positive empty radius, and that radius is its distance to
    the surface.  On two spheres (vertex rows) it lies inside one of them; on a union
    of thin and overlapping primitives the rows are farthest-point sample rows, the
    row kind of the exterior batch meshes (vertex rows, with their relative slack,
    can reach through a feature thinner than kappa r_max: reading R1)."""
    if which == "two_spheres":
        m = meshgen.two_spheres(3, 0.5, 1.5)
        rows = oracle.vertex_rows(m.V, m.F)
    else:
        m = meshgen.wild_union(8, 8000, seed=3, flip_frac=0.0)
        rows = oracle.fps_rows(m.V, m.F, 1024, orient=True)
    o = oracle.interior_origin(m.V, m.F, rows)
    st = oracle.origin_stride(len(rows["pos"]))
    sub = dict(pos=np.ascontiguousarray(rows["pos"][::st]), nrm=np.ascontiguousarray(rows["nrm"][::st]),
               tri2bin=rows.get("tri2bin"))
    _, c, rho = oracle.tangent_balls(m.V, m.F, sub)
    assert rho.max() > 0
    d2, _, _ = oracle.closest_points(m.V, m.F, o[None], 64)
    assert abs(math.sqrt(d2[0]) - rho.max()) <= 1e-12 * rho.max()
    assert _gwn_numpy(m.V, m.F, o) > 0.99
    if which == "two_spheres":
        assert min(np.linalg.norm(o), np.linalg.norm(o - np.array([1.5, 0, 0]))) < 0.5 - rho.max() * 0.5


# --------------------------------------------------------------------------- sample rows (reading R16)
def test_fps_float_selection_equals_fp64_selection_until_a_near_tie(oracle):
    """Farthest-point sampling in FP64 (numpy, the greedy definition) picks the same
    faces as the oracle's single-precision sampling up to the first step whose two best
    FP64 candidates lie within single-precision rounding of each other; on this mesh
    that step comes late or never."""
    m = meshgen.wild_union(6, 5000, seed=9)
    n = 300
    r = oracle.fps_rows(m.V, m.F, n, orient=False)
    cen = ((m.V[m.F[:, 0]] + m.V[m.F[:, 1]]) + m.V[m.F[:, 2]]) / 3.0
    mind = np.full(m.nf, np.inf)
    sel = [0]
    agree = n
    for i in range(n - 1):
        mind = np.minimum(mind, np.sum((cen - cen[sel[-1]]) ** 2, 1))
        top2 = np.partition(mind, -2)[-2:]
        nxt = int(np.argmax(mind))
        if nxt != r["sel"][i + 1]:
            # a disagreement is allowed only at a near tie of the FP64 distances
            assert top2[1] - top2[0] <= 1e-5 * top2[1], (i + 1, top2)
            agree = i + 1
            break
        sel.append(nxt)
    assert agree >= 100


# --------------------------------------------------------------------------- vertex rows under refinement (reading R1)
def test_vertex_row_rayleigh_quotients_converge_under_refinement(oracle):
    """Vertex rows of the unit icosphere (the small sphere workload at subdivision 2,
    then 3 and 4): the Rayleigh quotients f' Lambda f / f' M f of the l = 1 and l = 2
    harmonics (linear in Lambda, so unbiased in the walk count) approach the
    cap-corrected closed form lambda_l(theta0).  The excess tracks the jump mass times
    the depth r - rho of the vertex above its empty ball, which falls like h^2: it must
    shrink by more than half per subdivision and be below 12% at subdivision 4."""
    lam = oracle.sphere_eigs_cap(2, 2.5)
    gaps = []
    for s in (2, 3, 4):
        m = meshgen.icosphere(s)
        rows = oracle.vertex_rows(m.V, m.F)
        est = oracle.estimate(m.V, m.F, rows, 32, 1e-3, seed=0)
        L = oracle.assemble(est, rows)
        P = m.V
        g = []
        for l, f in ((1, P[:, 2]), (1, P[:, 0]), (2, P[:, 0] ** 2 - P[:, 1] ** 2), (2, P[:, 0] * P[:, 1])):
            g.append((f @ L @ f) / (f @ (rows["area"] * f)) / lam[l] - 1.0)
        gaps.append(float(np.mean(g)))
    assert gaps[0] > 0 and gaps[1] > 0 and gaps[2] > 0
    assert gaps[1] < 0.5 * gaps[0] and gaps[2] < 0.5 * gaps[1], gaps
    assert gaps[2] < 0.12, gaps
