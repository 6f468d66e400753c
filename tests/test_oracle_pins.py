"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each checks it against a closed form,
an identity, a physical definition, a brute force or a claim the paper prints.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import tsr_oracle as O
from paper_2203_12339_gb300 import scene

MATERIALS = [
    (0.0021, 2.19, 1.3), (0.0041, 2.62, 1.3), (0.0071, 3.00, 1.3),   # marble RGB (Section 5 style)
    (0.5, 0.4, 1.2), (0.02, 7.0, 1.5), (1.0, 0.37, 1.0), (0.001, 1.0, 1.8),
]


# ---------------------------------------------------------------- Section 2.1
def _internal_diffuse_fresnel(eta):
    """Diffuse Fresnel reflectance seen from inside a medium of relative index eta (exact Fresnel, TIR included)."""
    def r(mu):
        st = eta * math.sqrt(max(0.0, 1.0 - mu * mu))
        if st >= 1.0:
            return 1.0
        ct = math.sqrt(1.0 - st * st)
        rs = (eta * mu - ct) / (eta * mu + ct)
        rp = (eta * ct - mu) / (eta * ct + mu)
        return 0.5 * (rs * rs + rp * rp)
    crit = math.sqrt(max(0.0, 1.0 - 1.0 / eta ** 2))
    v, _ = quad(lambda mu: 2.0 * mu * r(mu), 0.0, 1.0, points=[crit], limit=200)
    return v


@pytest.mark.parametrize("eta", [1.1, 1.2, 1.3, 1.4, 1.5, 1.8])
def test_fresnel_fit_matches_physical_diffuse_reflectance(eta):
    # The polynomial of Section 2.1 is a fit of the hemispherical diffuse Fresnel
    # reflectance; it agrees with the exact integral to ~1e-3 on [1.1, 1.8].
    assert abs(O.fresnel_dr(eta) - _internal_diffuse_fresnel(eta)) < 2e-3


def test_fresnel_matched_index_is_nearly_zero():
    assert abs(O.fresnel_dr(1.0)) < 2e-3
    assert abs(O.boundary_a(1.0) - 1.0) < 5e-3


def _plane_total_closed_form(sa, ss, eta):
    # int_0^inf 2 pi r R_d dr = alpha'/2 (1 + e^{-4/3 A sqrt(3(1-alpha'))}) e^{-sqrt(3(1-alpha'))}
    alpha = ss / (sa + ss)
    F = -1.440 / eta ** 2 + 0.710 / eta + 0.668 + 0.0636 * eta
    A = (1 + F) / (1 - F)
    q = math.sqrt(3 * (1 - alpha))
    return alpha / 2 * (1 + math.exp(-4.0 / 3.0 * A * q)) * math.exp(-q)


@pytest.mark.parametrize("sa,ss,eta", MATERIALS)
def test_dipole_plane_integral_closed_form(sa, ss, eta):
    # Every dipole term integrates in closed form over the plane; a dropped term,
    # a wrong sign, 1/d in place of 1/d_v or a wrong z_v breaks this identity.
    num, _ = quad(lambda r: 2 * math.pi * r * O.dipole_rd(r, sa, ss, eta), 0, np.inf,
                  limit=800, epsabs=0, epsrel=1e-13)
    assert num == pytest.approx(_plane_total_closed_form(sa, ss, eta), rel=1e-9)


def test_dipole_plane_integral_marble_values():
    # Total diffuse reflectance of the RGB marble at eta = 1.3 (closed form above).
    got = [_plane_total_closed_form(a, s, 1.3) for a, s in zip(scene.MARBLE_SIGMA_A, scene.MARBLE_SIGMA_S)]
    assert got == pytest.approx([0.866540583, 0.833804102, 0.800993416], abs=2e-9)


@pytest.mark.parametrize("sa,ss,eta", MATERIALS[:4])
@pytest.mark.parametrize("R", [0.5, 5.0, 40.0])
def test_dipole_truncated_integral(sa, ss, eta, R):
    # int_0^R 2 pi r R_d dr = alpha'/2 sum_z (e^{-s_tr z} - z e^{-s_tr D_z}/D_z), D_z = sqrt(R^2+z^2)
    st = sa + ss
    s_tr = math.sqrt(3 * sa * st)
    F = -1.440 / eta ** 2 + 0.710 / eta + 0.668 + 0.0636 * eta
    A = (1 + F) / (1 - F)
    zr = 1 / st
    zv = zr * (1 + 4 * A / 3)
    ref = ss / st / 2 * sum(math.exp(-s_tr * z) - z * math.exp(-s_tr * math.hypot(R, z)) / math.hypot(R, z)
                            for z in (zr, zv))
    num, _ = quad(lambda r: 2 * math.pi * r * O.dipole_rd(r, sa, ss, eta), 0, R, limit=800, epsabs=0, epsrel=1e-13)
    assert num == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("sa,ss,eta", MATERIALS)
def test_dipole_partials_match_complex_step(sa, ss, eta):
    r = np.linspace(0.0, 40.0, 257)
    h = 1e-30
    cs = [O.dipole_rd(r, sa + 1j * h, ss, eta).imag / h,
          O.dipole_rd(r, sa, ss + 1j * h, eta).imag / h,
          O.dipole_rd(r, sa, ss, eta + 1j * h).imag / h]
    hand = O.dipole_rd_partials(r, sa, ss, eta)
    for a, b in zip(hand, cs):
        scale = np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= 1e-11 * scale


def test_dipole_partials_integrate_to_closed_form_derivative():
    # d/dsigma_a of the plane total (complex step of the closed form) = plane integral of dR/dsigma_a.
    sa, ss, eta = 0.05, 1.2, 1.4
    h = 1e-30

    def closed(sa_, ss_):
        alpha = ss_ / (sa_ + ss_)
        F = -1.440 / eta ** 2 + 0.710 / eta + 0.668 + 0.0636 * eta
        A = (1 + F) / (1 - F)
        q = np.sqrt(3 * (1 - alpha))
        return alpha / 2 * (1 + np.exp(-4.0 / 3.0 * A * q)) * np.exp(-q)

    want = closed(sa + 1j * h, ss).imag / h
    got, _ = quad(lambda r: 2 * math.pi * r * O.dipole_rd_partials(r, sa, ss, eta)[0], 0, np.inf,
                  limit=800, epsabs=0, epsrel=1e-12)
    assert got == pytest.approx(want, rel=1e-8)


# ---------------------------------------------------------------- Section 2.2
def test_pca_basis_orthonormal(pca_basis_k16):
    f, _ = pca_basis_k16
    assert np.max(np.abs(f @ f.T - np.eye(f.shape[0]))) < 1e-12


def test_pca_sign_convention(pca_basis_k16):
    f, _ = pca_basis_k16
    for k in range(f.shape[0]):
        m = int(np.argmax(np.abs(f[k])))
        assert f[k, m] > 0


def test_pca_eckart_young_and_monotone(pca_basis_k16):
    f, s = pca_basis_k16
    sa, ss = scene.pca_materials(256, seed=0)
    R = O.sample_matrix(sa, ss, 1.3)
    prev = np.inf
    for K in (1, 2, 4, 8, 12, 16):
        fk = f[:K]
        resid = np.linalg.norm(R - (R @ fk.T) @ fk) ** 2
        assert resid == pytest.approx(np.sum(s[K:] ** 2), rel=1e-6, abs=1e-22 * np.sum(s ** 2))
        assert resid < prev
        prev = resid


def test_pca_leading_vectors_by_power_iteration(pca_basis_k16):
    # f_0, f_1 are the dominant eigenvectors of R^T R: found independently by
    # power iteration with deflation (no SVD).
    f, s = pca_basis_k16
    sa, ss = scene.pca_materials(256, seed=0)
    R = O.sample_matrix(sa, ss, 1.3)
    G = R.T @ R
    rng = np.random.default_rng(1)
    found = []
    for k in range(2):
        v = rng.standard_normal(G.shape[0])
        for _ in range(3000):
            for u in found:
                v -= (u @ v) * u
            v = G @ v
            v /= np.linalg.norm(v)
        found.append(v)
        assert abs(abs(v @ f[k]) - 1.0) < 1e-9
        assert math.sqrt(v @ G @ v) == pytest.approx(s[k], rel=1e-9)


def test_pca_spectrum_matches_paper_claims(pca_basis_k16):
    # Section 2.2: eigenvalues after the tenth are close to zero; 15 basis
    # functions give an L2 error below 1e-4.
    _, s = pca_basis_k16
    eig = s ** 2
    assert np.all(eig[10:] / eig[0] < 1e-8)
    rel_err_15 = math.sqrt(np.sum(s[15:] ** 2) / np.sum(s ** 2))
    assert rel_err_15 < 1e-4


def test_projection_reconstructs_sample_rows_at_full_rank():
    # A sampled material lies in the row space of R, so with every right singular
    # vector kept, sum_k g_k f_k reproduces its R_d samples exactly.
    sa, ss = scene.pca_materials(32, seed=3)
    f, s = O.fit_pca_basis(sa, ss, 1.3, 1024, 40.0, 32)
    g = O.project_material(f, np.stack([sa] * 3, 1), np.stack([ss] * 3, 1), np.full(32, 1.3))
    R = O.sample_matrix(sa, ss, 1.3)
    rec = g[:, 0, :] @ f
    assert np.max(np.abs(rec - R)) < 1e-10 * np.max(np.abs(R))


def test_projection_residual_of_new_material(pca_basis_k16):
    f, s = pca_basis_k16
    sa, ss, eta = scene.edit_materials(8, seed=11)
    eta = np.full(8, 1.3)
    g = O.project_material(f, sa, ss, eta)
    R = O.dipole_rd(O.radius_grid()[None, None, :], sa[..., None], ss[..., None], eta[:, None, None])
    rec = g @ f
    rel = np.linalg.norm(rec - R) / np.linalg.norm(R)
    assert rel < 1e-3


def test_projection_vjp_matches_complex_step(pca_basis_k16):
    f, _ = pca_basis_k16
    sa, ss, eta = scene.edit_materials(3, seed=5)
    rng = np.random.default_rng(2)
    dg = rng.standard_normal((3, 3, f.shape[0]))
    d_sa, d_ss, d_eta = O.project_material_vjp(f, sa, ss, eta, dg)
    h = 1e-30
    for e in range(3):
        for c in range(3):
            sa_c = sa.astype(complex)
            sa_c[e, c] += 1j * h
            want = (O.project_material(f, sa_c, ss, eta).imag / h * dg).sum()
            assert d_sa[e, c] == pytest.approx(want, rel=1e-10, abs=1e-14)
            ss_c = ss.astype(complex)
            ss_c[e, c] += 1j * h
            want = (O.project_material(f, sa, ss_c, eta).imag / h * dg).sum()
            assert d_ss[e, c] == pytest.approx(want, rel=1e-10, abs=1e-14)
        et = eta.astype(complex)
        et[e] += 1j * h
        want = (O.project_material(f, sa, ss, et).imag / h * dg).sum()
        assert d_eta[e] == pytest.approx(want, rel=1e-10, abs=1e-14)


# ---------------------------------------------------------------- f_k(r)
def test_basis_eval_is_linear_interpolation(pca_basis_k16):
    f, _ = pca_basis_k16
    grid = O.radius_grid()
    r = np.random.default_rng(0).uniform(0, 40, 5000)
    got = O.basis_eval(f, r)
    for k in (0, 5, 15):
        assert np.max(np.abs(got[k] - np.interp(r, grid, f[k]))) < 1e-14
    assert np.allclose(O.basis_eval(f, grid), f, atol=1e-15, rtol=0)
    assert np.all(O.basis_eval(f, np.array([40.0001, 45.0])) == 0.0)


def test_cutoff_decided_on_fp32_r2():
    xo = np.array([[0.0, 0.0, 20.0]], dtype=np.float32)
    xi = np.array([[0.0, 0.0, -20.0], [0.0, 0.0, -20.00002]], dtype=np.float32)
    r2 = O.pair_r2_fp32(xo, xi)
    assert r2.dtype == np.float32
    assert r2[0] == np.float32(1600.0)
    assert r2[1] > np.float32(1600.0)


# ---------------------------------------------------------------- Eq. 6-7 transfer
def _brute_transfer(f, pos, area, T):
    """Pure-Python double loop over (o, i) with scalar interpolation (tiny meshes only)."""
    K, n_r = f.shape
    dr = 40.0 / (n_r - 1)
    N = pos.shape[0]
    J = T.shape[0]
    M = np.zeros((K, J, N))
    p = pos.astype(np.float64)
    for o in range(N):
        for i in range(N):
            r = math.dist(p[o], p[i])
            d32 = [np.float32(pos[o][a]) - np.float32(pos[i][a]) for a in range(3)]
            r2 = np.float32(np.float32(np.float32(d32[0] * d32[0]) + np.float32(d32[1] * d32[1])) + np.float32(d32[2] * d32[2]))
            if r2 > np.float32(1600.0):
                continue
            x = r / dr
            m = min(int(math.floor(x)), n_r - 2)
            t = x - m
            for k in range(K):
                fk = f[k, m] * (1 - t) + f[k, m + 1] * t
                for j in range(J):
                    M[k, j, o] += area[i] * fk * T[j, i]
    return M


@pytest.mark.parametrize("nu", [1, 2])
def test_transfer_matches_double_loop(pca_basis_k16, nu):
    f, _ = pca_basis_k16
    sc = scene.make_scene(nu, K=4, J=4, amp=0.1 if nu == 2 else 0.0, seed=3)
    pos = sc.mesh.pos.astype(np.float32)
    area = sc.mesh.area.astype(np.float32)
    T = sc.T.astype(np.float32)
    got = O.transfer_full(f[:4], pos, area, T)
    want = _brute_transfer(f[:4], pos, area.astype(np.float64), T.astype(np.float64))
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_transfer_k1_j1_is_weighted_sum():
    sc = scene.make_scene(4, K=1, J=1, amp=0.1, seed=4)
    pos = sc.mesh.pos.astype(np.float32)
    area = sc.mesh.area
    f = np.ones((1, 1024))
    M = O.transfer_full(f, pos, area, np.ones((1, pos.shape[0])))
    # f = 1 inside r_max: M[o] = sum of areas of the vertices within 40 mm (all of them here but the far side)
    p = pos.astype(np.float64)
    for o in (0, 17, 100):
        inside = O.pair_r2_fp32(pos[o][None, :], pos) <= np.float32(1600.0)
        assert M[0, 0, o] == pytest.approx(area[inside].sum(), rel=1e-13)


def test_transfer_linear_in_T(pca_basis_k16):
    f, _ = pca_basis_k16
    sc = scene.make_scene(4, K=3, J=4, amp=0.1, seed=5)
    pos = sc.mesh.pos.astype(np.float32)
    rng = np.random.default_rng(0)
    T1, T2 = rng.standard_normal((2, 4, pos.shape[0]))
    rows = np.array([0, 5, 77])
    a = O.transfer_rows(f[:3], pos, sc.mesh.area, 2.0 * T1 - 3.0 * T2, rows)
    b = 2.0 * O.transfer_rows(f[:3], pos, sc.mesh.area, T1, rows) - 3.0 * O.transfer_rows(f[:3], pos, sc.mesh.area, T2, rows)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_transfer_sphere_identity_converges():
    # On a sphere of radius rho, dA = 2 pi r dr in chord length r, so with T = 1 and
    # the radial kernel R_d, sum_i A_i R_d(r_oi) -> int_0^{2 rho} 2 pi r R_d dr (O(h^2)).
    sa, ss, eta = 0.01, 0.4, 1.3
    n_r = 40001
    table = O.dipole_rd(O.radius_grid(n_r), sa, ss, eta)[None, :]
    st = sa + ss
    s_tr = math.sqrt(3 * sa * st)
    F = O.fresnel_dr(eta)
    A = (1 + F) / (1 - F)
    zr = 1 / st
    zv = zr * (1 + 4 * A / 3)
    R = 40.0
    want = ss / st / 2 * sum(math.exp(-s_tr * z) - z * math.exp(-s_tr * math.hypot(R, z)) / math.hypot(R, z) for z in (zr, zv))
    errs = []
    for nu in (8, 16, 32):
        m = scene.icosphere(nu)
        pos = m.pos.astype(np.float32)
        rows = np.array([0, 10 * nu * nu // 3, 10 * nu * nu + 1])
        M = O.transfer_rows(table, pos, m.area, np.ones((1, m.n)), rows)
        errs.append(np.max(np.abs(M[0, 0] - want)) / want)
    assert errs[2] < 3e-3
    assert errs[1] < errs[0] / 2.5 and errs[2] < errs[1] / 2.5


# ---------------------------------------------------------------- Eq. 9-10 Haar
def test_haar_explicit_matrix_n4():
    H = np.array([[0.5, 0.5, 0.5, 0.5],
                  [0.5, 0.5, -0.5, -0.5],
                  [1 / math.sqrt(2), -1 / math.sqrt(2), 0, 0],
                  [0, 0, 1 / math.sqrt(2), -1 / math.sqrt(2)]])
    got = np.stack([O.haar_forward_1d(e) for e in np.eye(4)], axis=1)
    assert np.allclose(got, H, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 8, 64, 1024])
def test_haar_round_trip_parseval_constant(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n))
    c = O.haar_forward_1d(x)
    assert np.allclose(O.haar_inverse_1d(c), x, atol=1e-13)
    assert np.allclose((c ** 2).sum(-1), (x ** 2).sum(-1), rtol=1e-13)
    cc = O.haar_forward_1d(np.full(n, 2.5))
    assert cc[0] == pytest.approx(2.5 * math.sqrt(n))
    assert np.allclose(cc[1:], 0.0, atol=1e-13)


def test_haar_delta_column():
    n = 16
    x = np.zeros(n)
    x[5] = 1.0
    c = O.haar_forward_1d(x)
    # delta at 5 touches the scaling function and one detail per level
    assert np.count_nonzero(np.abs(c) > 1e-15) == 1 + 4
    assert c[0] == pytest.approx(1 / 4)
    assert c[8 + 2] == pytest.approx(-1 / math.sqrt(2))   # finest level pair (4,5), 5 is the odd member


def test_morton_known_values_and_bijection():
    assert [int(O.morton_index(r, c, 4)) for r, c in [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0), (3, 3)]] == \
        [0, 1, 2, 3, 4, 8, 15]
    P = 8
    rr, cc = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    m = O.morton_index(rr, cc, P).reshape(-1)
    assert sorted(m.tolist()) == list(range(P * P))


@pytest.mark.parametrize("nu", [2, 3, 4, 5])
def test_chart_wavelet_round_trip_and_energy(nu):
    rng = np.random.default_rng(nu)
    N = 10 * nu * nu + 2
    X = rng.standard_normal((2, N))
    C = O.chart_to_wavelet(X, nu)
    assert np.allclose(O.wavelet_to_chart(C, nu), X, atol=1e-13)
    assert np.allclose((C ** 2).sum(-1), (X ** 2).sum(-1), rtol=1e-13)
    # discarded energy equals the squared reconstruction error (orthonormality)
    mask = np.abs(C) > 0.8
    mask[:, -2:] = True
    rec = O.wavelet_to_chart(np.where(mask, C, 0.0), nu)
    if nu & (nu - 1) == 0:
        assert np.sum((rec - X) ** 2) == pytest.approx(np.sum(np.where(mask, 0.0, C) ** 2), rel=1e-12)
    else:
        assert np.sum((rec - X) ** 2) <= np.sum(np.where(mask, 0.0, C) ** 2) * (1 + 1e-12)


# ---------------------------------------------------------------- Step 2 selection
def test_keep_count():
    assert O.keep_count(0.10, 40960) == 4096
    assert O.keep_count(0.05, 163840) == 8192
    assert O.keep_count(0.0, 10) == 1
    assert O.keep_count(1.0, 10) == 10


def test_select_top_brute_force_with_ties():
    nu = 2
    n_coef = 40
    rng = np.random.default_rng(0)
    vals = rng.integers(-5, 6, size=(2, 3, n_coef + 2)).astype(np.float32)   # many ties
    mask = O.select_top(vals, nu, 0.3)
    nk = O.keep_count(0.3, n_coef)
    for k in range(2):
        for j in range(3):
            ranked = sorted(range(n_coef), key=lambda w: (-abs(float(vals[k, j, w])), w))
            want = set(ranked[:nk])
            assert set(np.nonzero(mask[k, j, :n_coef])[0].tolist()) == want
            assert mask[k, j, n_coef:].all()


def _min_subset_size_reaching(vals, target):
    """Brute force: the size of the smallest subset of vals whose squares sum to >= target
    (exact rational arithmetic on the integer-valued inputs)."""
    from itertools import combinations
    sq = [int(v) * int(v) for v in vals]
    for n in range(1, len(vals) + 1):
        if any(sum(c) >= target for c in combinations(sq, n)):
            return n
    return len(vals)


def test_energy_keep_count_is_the_smallest_subset_by_brute_force():
    """Greedy-by-magnitude is optimal: for integer coefficients (exact squares and sums) the
    count equals the smallest subset of any kind that reaches the energy fraction."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    for trial in range(40):
        n = int(rng.integers(3, 11))
        vals = rng.integers(-6, 7, size=n)
        if not vals.any():
            continue
        e = [0.5, 0.8, 0.9, 0.95, 0.98, 1.0][trial % 6]
        total = sum(int(v) * int(v) for v in vals)
        target = Fraction(e).limit_denominator(1000) * total
        want = _min_subset_size_reaching(vals, target)
        assert O.energy_keep_count(vals.astype(np.float32), e) == want, (vals, e)


def test_energy_keep_count_properties():
    rng = np.random.default_rng(4)
    c = rng.standard_normal(5000) * np.exp(rng.uniform(-6, 0, 5000))
    en = np.sort(c ** 2)[::-1]
    prev = 0
    for e in (0.5, 0.9, 0.95, 0.98, 0.999):
        n = O.energy_keep_count(c, e)
        assert n >= prev                                             # monotone in e
        assert en[:n].sum() >= e * en.sum() * (1 - 1e-14)            # reaches the threshold ...
        assert n == 1 or en[:n - 1].sum() < e * en.sum() * (1 + 1e-14)   # ... and no fewer would
        prev = n
    z = np.zeros(9)
    assert O.energy_keep_count(z, 0.95) == 1                         # all zero: keep one
    z[[2, 5, 7]] = [1.0, -2.0, 0.5]
    assert O.energy_keep_count(z, 1.0) == 3                          # e = 1: every nonzero value
    nu = 1   # P = 1: 10 chart coefficients + 2 poles
    row = np.array([3.0, -3.0, 1.0, 0.0, 3.0, 2.0, 0.0, 1.0, -1.0, 0.0, 5.0, 6.0])
    mask = O.select_energy(row[None, None, :], nu, 0.6)
    # energies 9, 9, 9, 4, 1, 1, 1 (total 34): 0.6 * 34 = 20.4 needs three 9s; ties by index: 0, 1, 4
    assert np.nonzero(mask[0, 0, :10])[0].tolist() == [0, 1, 4]
    assert mask[0, 0, 10:].all()


# ---------------------------------------------------------------- Fresnel factors (readings R34, R35)
@pytest.mark.parametrize("eta", [1.2, 1.3, 1.5])
def test_fresnel_transmittance_limits(eta):
    mu = np.linspace(1e-6, 1.0, 2001)
    Ft = O.fresnel_transmittance(eta, mu)
    assert np.all(np.diff(Ft) > 0)                                                    # rises towards the normal
    assert Ft[-1] == pytest.approx(1 - ((eta - 1) / (eta + 1)) ** 2, rel=1e-14)      # normal incidence
    assert O.fresnel_transmittance(eta, 1e-9) < 1e-7                                 # grazing: everything reflected
    assert O.fresnel_transmittance(eta, -0.3) == 0.0 and O.fresnel_transmittance(eta, 0.0) == 0.0
    assert np.allclose(O.fresnel_transmittance(1.0, mu), 1.0, atol=1e-15)            # matched index


def test_fresnel_transmittance_derivative_by_complex_step():
    mu = np.array([0.05, 0.3, 0.7, 1.0])
    for eta in (1.15, 1.3, 1.6):
        h = 1e-30
        cs = np.imag(O.fresnel_transmittance(eta + 1j * h, mu.astype(complex))) / h
        assert np.allclose(O.fresnel_transmittance_deta(eta, mu), cs, rtol=1e-11, atol=1e-14)


def test_fresnel_output_vjp_matches_finite_differences():
    rng = np.random.default_rng(12)
    E, N = 2, 7
    B = rng.standard_normal((E, 3, N))
    eta = np.array([1.25, 1.45])
    cos_o = np.array([0.9, 0.4, -0.2, 0.05, 1.0, 0.7, 0.0])
    W = rng.standard_normal((E, 3, N))
    L = lambda B_, e_: float(np.sum(W * O.fresnel_output(B_, e_, cos_o)))
    dB, deta = O.fresnel_output_vjp(B, eta, cos_o, W)
    h = 1e-6
    for e in range(E):
        ep, em = eta.copy(), eta.copy()
        ep[e] += h
        em[e] -= h
        assert deta[e] == pytest.approx((L(B, ep) - L(B, em)) / (2 * h), rel=1e-7)
    Bp = B.copy()
    Bp[1, 2, 3] += 1.0
    assert dB[1, 2, 3] == pytest.approx(L(Bp, eta) - L(B, eta), rel=1e-12)


def test_oracle_sh_closed_forms_addition_theorem_and_orthonormality():
    """The oracle's real SH (reading R19: no Condon-Shortley phase, j = l^2 + l + m) against the
    textbook Cartesian forms for l <= 2, the addition theorem sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi)
    P_l(a.b), and orthonormality by a product Gauss quadrature on the sphere."""
    rng = np.random.default_rng(21)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x, y, z = d.T
    Y = O.sh_real_oracle(3, d)
    c0, c1 = 0.5 / math.sqrt(math.pi), math.sqrt(3 / (4 * math.pi))
    want = [np.full(50, c0), c1 * y, c1 * z, c1 * x,
            0.5 * math.sqrt(15 / math.pi) * x * y, 0.5 * math.sqrt(15 / math.pi) * y * z,
            0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1), 0.5 * math.sqrt(15 / math.pi) * x * z,
            0.25 * math.sqrt(15 / math.pi) * (x * x - y * y)]
    for j in range(9):
        assert np.allclose(Y[j], want[j], atol=1e-13), j
    Ya = O.sh_real_oracle(6, d[:25])
    Yb = O.sh_real_oracle(6, d[25:])
    cosg = np.sum(d[:25] * d[25:], axis=1)
    for l in range(6):
        lhs = np.sum(Ya[l * l:(l + 1) ** 2] * Yb[l * l:(l + 1) ** 2], axis=0)
        Pl = np.polynomial.legendre.Legendre.basis(l)(cosg)
        assert np.allclose(lhs, (2 * l + 1) / (4 * math.pi) * Pl, atol=1e-13), l
    xg, wg = np.polynomial.legendre.leggauss(16)
    ph = (np.arange(32) + 0.5) * (2 * math.pi / 32)
    Z, PH = np.meshgrid(xg, ph, indexing="ij")
    st = np.sqrt(1 - Z ** 2)
    dirs = np.stack([st * np.cos(PH), st * np.sin(PH), Z], axis=-1).reshape(-1, 3)
    w = np.outer(wg, np.full(32, 2 * math.pi / 32)).reshape(-1)
    Yq = O.sh_real_oracle(5, dirs)
    assert np.allclose((Yq * w) @ Yq.T, np.eye(25), atol=1e-12)


def test_sh_zonal_fresnel_reduces_to_the_clamped_cosine():
    A = O.sh_zonal_fresnel(1.0, 5)
    assert np.allclose(A, [math.pi, 2 * math.pi / 3, math.pi / 4, 0.0, -math.pi / 24], atol=1e-12)
    normals = scene.icosphere(2, 0.0, 3, 0).normal
    assert np.allclose(O.sh_transfer_fresnel(normals, 16, 1.0), scene.sh_transfer(normals, 16), atol=1e-12)


def test_sh_transfer_fresnel_by_direct_integration():
    """T_j(n) = int Y_j(w) F_t(eta, n.w) max(n.w, 0) dw integrated over the hemisphere around n
    (Gauss-Legendre in n.w, uniform in azimuth), against A_l(eta) Y_j(n) (Funk-Hecke)."""
    eta, order = 1.4, 5
    x, wq = np.polynomial.legendre.leggauss(96)
    mu = 0.5 * (x + 1.0)
    wmu = 0.5 * wq
    phi = np.arange(128) * (2 * math.pi / 128)
    rng = np.random.default_rng(5)
    for _ in range(3):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        t1 = np.cross(n, [0.3, 0.5, 0.8])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(n, t1)
        M, F = np.meshgrid(mu, phi, indexing="ij")
        st = np.sqrt(1 - M ** 2)
        dirs = (M[..., None] * n + (st * np.cos(F))[..., None] * t1 + (st * np.sin(F))[..., None] * t2).reshape(-1, 3)
        Y = scene.sh_real(order, dirs)                                        # (25, n_dirs)
        weight = (np.outer(wmu, np.full(phi.size, 2 * math.pi / phi.size)) * O.fresnel_transmittance(eta, M) * M).reshape(-1)
        direct = Y @ weight
        want = O.sh_transfer_fresnel(n[None, :], order * order, eta)[:, 0]
        assert np.allclose(direct, want, atol=1e-9)


# ---------------------------------------------------------------- visibility transfer (reading R36)
def test_onb_is_orthonormal_and_right_handed():
    rng = np.random.default_rng(13)
    n = rng.standard_normal((200, 3))
    n = np.concatenate([n, [[0, 0, 1.0], [0, 0, -1.0], [1e-9, 0, -1.0], [1.0, 0, 0]]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t1, t2 = O.onb_from_normal(n)
    for a, b in ((t1, t2), (t1, n), (t2, n)):
        assert np.abs(np.sum(a * b, axis=1)).max() < 1e-12
    for a in (t1, t2):
        assert np.abs(np.linalg.norm(a, axis=1) - 1).max() < 1e-12
    assert np.abs(np.cross(t1, t2) - n).max() < 1e-12


def test_hemisphere_samples_integrate_the_cosine_lobe():
    """(pi/S) sum_s Y_j(w_s) over cosine-weighted directions estimates A_l Y_j(z): exact for l = 0,
    within the quasi-Monte Carlo error for the rest."""
    loc = O.hemisphere_samples(1024)
    assert np.abs(np.linalg.norm(loc, axis=1) - 1).max() < 1e-12 and loc[:, 2].min() > 0
    est = (math.pi / 1024) * scene.sh_real(5, loc).sum(axis=1)
    exact = scene.sh_transfer(np.array([[0.0, 0.0, 1.0]]), 25)[:, 0]
    assert est[0] == pytest.approx(exact[0], rel=1e-13)
    assert np.abs(est - exact).max() < 3e-3


def test_ray_hits_match_an_independent_solver():
    """The FP32 Moller-Trumbore decision against solving o + t d = v0 + u e1 + v e2 in FP64, away
    from the decision boundaries (where FP32 rounding may legitimately differ)."""
    rng = np.random.default_rng(14)
    R, F = 300, 40
    orig = rng.uniform(-1, 1, (R, 3))
    dirs = rng.standard_normal((R, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    v0, v1, v2 = (rng.uniform(-2, 2, (F, 3)) for _ in range(3))
    got = O.ray_hits_any(orig, dirs, v0, v1, v2)
    clear = np.ones(R, dtype=bool)
    want = np.zeros(R, dtype=bool)
    for r in range(R):
        for f in range(F):
            A = np.stack([-dirs[r], v1[f] - v0[f], v2[f] - v0[f]], axis=1)
            t, u, v = np.linalg.solve(A, orig[r] - v0[f])
            margin = min(abs(u), abs(v), abs(1 - u - v), abs(t - 1e-4))
            if margin < 1e-4:
                clear[r] = False
            if u >= 0 and v >= 0 and u + v <= 1 and t > 1e-4:
                want[r] = True
    assert clear.sum() > 200
    assert np.array_equal(got[clear], want[clear])


def test_visibility_transfer_convex_and_covered():
    """On the undisplaced (convex) sphere no ray is blocked, so T is the plain quadrature of the clamped
    cosine; under a roof that covers the hemisphere every ray is blocked."""
    m = scene.icosphere(3, 0.0, 3, 0)
    T = O.visibility_transfer(m.pos, m.tris, m.normal, 16, 1024)
    assert np.abs(T - scene.sh_transfer(m.normal, 16)).max() < 3e-3
    roof = np.array([[-1e4, -1e4, 1.0], [1e4, -1e4, 1.0], [0.0, 1e4, 1.0]])   # a point under a huge triangle
    loc = O.hemisphere_samples(256)
    hits = O.ray_hits_any(np.repeat([[0.0, 0.0, 1e-3]], 256, axis=0), loc, roof[[0]], roof[[1]], roof[[2]])
    assert hits.all()


# ---------------------------------------------------------------- CDF 9/7 (reading R33)
# Analysis filters of the CDF 9/7 pair as published (the JPEG 2000 irreversible
# filter bank): lowpass normalised to sum 1, highpass to centre value 1.115...
CDF97_LOW_PUBLISHED = [0.026748757411, -0.016864118443, -0.078223266529, 0.266864118443, 0.602949018236,
                       0.266864118443, -0.078223266529, -0.016864118443, 0.026748757411]
CDF97_HIGH_PUBLISHED = [0.091271763114, -0.057543526229, -0.591271763114, 1.115087052457,
                        -0.591271763114, -0.057543526229, 0.091271763114]


def test_cdf97_lifting_reproduces_the_published_filters():
    """The lifting steps (alpha..delta, zeta) compose to the published 9-tap / 7-tap analysis
    filters, scaled by sqrt2 and 1/sqrt2 (DC gain sqrt2 of the low band, as for the Haar)."""
    n = 32
    low = np.array([O._lift_1d(np.eye(n)[p])[8] for p in range(n)])          # s_8: taps at x[12..20]
    high = np.array([O._lift_1d(np.eye(n)[p])[16 + 8] for p in range(n)])    # d_8: taps at x[14..20]
    assert np.allclose(low[12:21], np.sqrt(2) * np.array(CDF97_LOW_PUBLISHED), atol=1e-11)
    assert np.abs(np.delete(low, range(12, 21))).max() < 1e-15
    assert np.allclose(high[14:21], np.array(CDF97_HIGH_PUBLISHED) / np.sqrt(2), atol=1e-11)
    assert np.abs(np.delete(high, range(14, 21))).max() < 1e-15


def test_cdf97_moments_boundaries_and_reconstruction():
    rng = np.random.default_rng(9)
    i = np.arange(64, dtype=np.float64)
    cubic = 0.3 - 0.02 * i + 1e-3 * i ** 2 - 2e-5 * i ** 3
    y = O._lift_1d(cubic)
    assert np.abs(y[32 + 3:64 - 3]).max() < 1e-12 * np.abs(cubic).max()   # 4 vanishing moments (interior)
    const = O._lift_1d(np.full(16, 2.5))                                     # symmetric ends: exact at the borders
    assert np.allclose(const[:8], 2.5 * np.sqrt(2), atol=1e-14) and np.abs(const[8:]).max() < 1e-14
    x = rng.standard_normal((4, 16))
    assert np.abs(O._unlift_1d(O._lift_1d(x)) - x).max() < 1e-14
    img = rng.standard_normal((2, 32, 32))
    assert np.abs(O.cdf97_inverse_2d(O.cdf97_forward_2d(img)) - img).max() < 1e-13
    for nu in (1, 3, 4, 6):
        X = rng.standard_normal((2, 10 * nu * nu + 2))
        C = O.chart_to_cdf97(X, nu)
        assert np.abs(O.cdf97_to_chart(C, nu) - X).max() < 1e-13
        S = O.cdf97_synthesis_matrix(nu)
        assert np.abs(C @ S.T - X).max() < 1e-13                            # B = S b^w as a matrix


def test_cdf97_pyramid_matches_separable_filtering():
    """One 2D level equals filtering rows then columns with the 1D analysis (an independent restatement
    through the published taps with mirrored ends)."""
    rng = np.random.default_rng(10)
    img = rng.standard_normal((8, 8))
    lo = np.sqrt(2) * np.array(CDF97_LOW_PUBLISHED)
    hi = np.array(CDF97_HIGH_PUBLISHED) / np.sqrt(2)

    def analyse(v):
        n = v.size
        ext = lambda q: v[abs(q) if q < n else 2 * (n - 1) - q]
        low = [sum(lo[t] * ext(2 * i + t - 4) for t in range(9)) for i in range(n // 2)]
        high = [sum(hi[t] * ext(2 * i + 1 + t - 3) for t in range(7)) for i in range(n // 2)]
        return np.array(low + high)

    rows = np.array([analyse(r) for r in img])
    both = np.array([analyse(c) for c in rows.T]).T
    level = O.cdf97_forward_2d(img)
    # the first level touches everything; the pyramid then continues on the 4 x 4 low-low band
    assert np.allclose(level[4:, :], both[4:, :], atol=1e-10) and np.allclose(level[:4, 4:], both[:4, 4:], atol=1e-10)
    assert np.allclose(level[:4, :4], O.cdf97_forward_2d(both[:4, :4]), atol=1e-10)


# ---------------------------------------------------------------- Steps 3-5 relight
def test_relight_uncompressed_equals_direct_eq6(pca_basis_k16):
    f, _ = pca_basis_k16
    sc = scene.make_scene(4, K=6, J=9, amp=0.1, seed=6)
    pos = sc.mesh.pos.astype(np.float32)
    M = O.transfer_full(f[:6], pos, sc.mesh.area, sc.T)
    Cw = O.chart_to_wavelet(M, 4)
    sa, ss, eta = scene.edit_materials(2, seed=9)
    g = O.project_material(f[:6], sa, ss, eta)
    B = O.relight(Cw, 4, g, sc.light)
    rows = np.arange(0, sc.n, 7)
    want = O.relight_direct(f[:6], pos, sc.mesh.area, sc.T, g, sc.light, rows=rows)
    assert np.allclose(B[:, :, rows], want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_relight_vjp_matches_finite_differences():
    nu = 3
    rng = np.random.default_rng(4)
    K, J, E = 3, 4, 2
    P = O.chart_side(nu)
    Cw = rng.standard_normal((K, J, 10 * P * P + 2))
    Cw[np.abs(Cw) < 0.5] = 0.0
    g = rng.standard_normal((E, 3, K))
    light = rng.standard_normal(J)
    target = rng.standard_normal((E, 3, 10 * nu * nu + 2))

    def loss(g_, l_):
        return np.sum((O.relight(Cw, nu, g_, l_) - target) ** 2)

    B = O.relight(Cw, nu, g, light)
    dg, dl = O.relight_vjp(Cw, nu, g, light, 2.0 * (B - target))
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 2), (0, 1, 1)]:
        gp = g.copy(); gp[idx] += h
        gm = g.copy(); gm[idx] -= h
        assert dg[idx] == pytest.approx((loss(gp, light) - loss(gm, light)) / (2 * h), rel=1e-6)
    for j in range(J):
        lp = light.copy(); lp[j] += h
        lm = light.copy(); lm[j] -= h
        assert dl[j] == pytest.approx((loss(g, lp) - loss(g, lm)) / (2 * h), rel=1e-6)
