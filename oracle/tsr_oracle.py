"""FP64 CPU oracle of the translucent-transfer hot path.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
definition that the CUDA path is checked against.  Only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
product path never does.  It shares no code with the CUDA library.

Everything is numpy float64 (complex128 where a complex step is taken).  Each
function names the part of the paper it restates:

  * Section 2.1, Eq. 4: Jensen's dipole diffuse reflectance R_d and the
    polynomial Fresnel fit F_dr.
  * Section 2.2, Eq. 5: the PCA factorisation R_d(r, sigma) ~ sum_k s_k(sigma) b_k(r)
    from an SVD M = U S V of sampled R_d; b_k are columns of V.  Here b_k is
    called f_k and s_k is called g_k.
  * Section 3, Eq. 6-7: the transfer M[k,j,o] = sum_i A_i f_k(|x_o - x_i|) T[j,i].
  * Section 3.2, Eq. 9-10 and precompute Step 2: spatial wavelet transform of
    the transfer and truncation of its coefficients.
  * Section 4, rendering Steps 3-5: project the material, weight the wavelet
    transfer by s_k, inverse wavelet transform.

Readings where the paper is silent or garbled (each is also listed with the
design notes):
  R1  sigma_t' = sigma_a + sigma_s' (printed "sigma_s + sigma_s'").
  R2  sigma_tr = sqrt(3 sigma_a sigma_t') (printed "sqrt(3 sigma_s sigma_t')").
  R3  the second dipole term uses 1/d_v (printed "1/d").
  R4  z_v = z_r (1 + 4A/3); both dipole terms are added, as printed.
  R7  the radial basis is the right singular vectors of the (material x radius)
      sample matrix R[s, m] = R_d(r_m; sigma_s): R = U S V^T, f_k = V[:, k].
  R8  the SVD is uncentred (the approximation has no mean term).
  R9  sign: each f_k is flipped so its largest-magnitude entry is positive
      (ties: lowest index).
  R11 radius grid r_m = r_max * m / (n_r - 1), m = 0..n_r-1.
  R12 f_k(r) is piecewise linear on that grid and zero for r > r_max; the
      cutoff is decided on the FP32 squared distance (see ``pair_r2_fp32``).
  R13 g_k = sum_m f_k(r_m) R_d(r_m) (plain discrete inner product).
  R15 the self pair i = o is included.
  R21 the spatial domain of chart d is its nu x nu grid in Morton order,
      zero-padded to P x P, P = 2^ceil(log2 nu); poles pass through.
  R22 the spatial wavelet is the orthonormal Haar.
  R23 keep rule: per (k, j), the round(p * 10 P^2) largest |coefficients| of the
      charts (ties: lower index); the two pole values are always kept.
  R34 F_t(eta, omega) = 1 - exact unpolarised Fresnel reflectance (relative index
      eta, outside cosine mu), 0 for mu <= 0; the output factor (1/pi) F_t(eta, omega_o)
      of Eq. 6 uses the caller's per-vertex cosine n_o . omega_o.
  R35 the incident F_t(eta, omega_i) is folded into the SH transfer T through the
      zonal coefficients A_l(eta) (Funk-Hecke) at the precompute's eta.
  R36 visibility in T (E11-E14): T[j, i] = (pi/S) sum_s Y_j(w_s) V(x_i, w_s), w_s the
      S cosine-weighted Hammersley directions in the Duff et al. frame of n_i, rays
      from x_i + eps n_i, V by an FP32 Moller-Trumbore any-hit over the mesh.
  R33 the paper's Step-2 wavelet "Daubechies 9/7": the biorthogonal CDF 9/7 pair
      by lifting (symmetric extension, low band DC gain sqrt 2), separable 2D
      Mallat pyramid of each chart's P x P image down to 1 x 1.
  R32 energy keep rule: per (k, j), the fewest largest |coefficients| of the charts
      (ties: lower index) whose squares sum to at least the fraction e of the
      row's energy ("exceeds" read as >=; energies in FP64); at least one; the
      poles always kept and not counted.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# Section 2.1, Eq. 4: dipole diffuse reflectance
# ----------------------------------------------------------------------------


def fresnel_dr(eta):
    """Polynomial diffuse Fresnel reflectance F_dr(eta) of Section 2.1 (text after Eq. 4)."""
    return -1.440 / (eta * eta) + 0.710 / eta + 0.668 + 0.0636 * eta


def boundary_a(eta):
    """A = (1 + F_dr) / (1 - F_dr) (Section 2.1)."""
    F = fresnel_dr(eta)
    return (1.0 + F) / (1.0 - F)


def dipole_rd(r, sigma_a, sigma_s, eta):
    """Eq. 4: R_d(r; sigma_a, sigma_s', eta), readings R1-R4.  Broadcasts; accepts complex."""
    st = sigma_a + sigma_s                      # sigma_t'
    alpha = sigma_s / st                        # alpha'
    s_tr = np.sqrt(3.0 * sigma_a * st)          # sigma_tr
    zr = 1.0 / st
    zv = zr * (1.0 + 4.0 * boundary_a(eta) / 3.0)
    dr = np.sqrt(r * r + zr * zr)
    dv = np.sqrt(r * r + zv * zv)
    real_term = zr * (s_tr + 1.0 / dr) * np.exp(-s_tr * dr) / (dr * dr)
    virt_term = zv * (s_tr + 1.0 / dv) * np.exp(-s_tr * dv) / (dv * dv)
    return alpha / (4.0 * math.pi) * (real_term + virt_term)


def dipole_rd_partials(r, sigma_a, sigma_s, eta):
    """Hand-derived partial derivatives of Eq. 4: (dR/dsigma_a, dR/dsigma_s', dR/deta).

    With h(z) = z (s_tr + 1/d) e^{-s_tr d} / d^2, d = sqrt(r^2 + z^2):
      dh/ds_tr = -s_tr z e^{-s_tr d} / d
      dh/dz    = (s_tr + 1/d) e^{-s_tr d}/d^2 - (z^2/d) e^{-s_tr d} (s_tr^2/d^2 + 3 s_tr/d^3 + 3/d^4)
    and R_d = alpha'/(4 pi) (h(z_r) + h(z_v)).
    """
    st = sigma_a + sigma_s
    alpha = sigma_s / st
    s_tr = np.sqrt(3.0 * sigma_a * st)
    zr = 1.0 / st
    F = fresnel_dr(eta)
    A = (1.0 + F) / (1.0 - F)
    c_v = 1.0 + 4.0 * A / 3.0
    zv = zr * c_v

    def h_parts(z):
        d = np.sqrt(r * r + z * z)
        e = np.exp(-s_tr * d)
        h = z * (s_tr + 1.0 / d) * e / (d * d)
        dh_ds = -s_tr * z * e / d
        dh_dz = (s_tr + 1.0 / d) * e / (d * d) - (z * z / d) * e * (
            s_tr * s_tr / (d * d) + 3.0 * s_tr / d ** 3 + 3.0 / d ** 4)
        return h, dh_ds, dh_dz

    hr, hr_s, hr_z = h_parts(zr)
    hv, hv_s, hv_z = h_parts(zv)
    pref = 1.0 / (4.0 * math.pi)
    dalpha_da = -sigma_s / (st * st)
    dalpha_ds = sigma_a / (st * st)
    dstr_da = 3.0 * (st + sigma_a) / (2.0 * s_tr)
    dstr_ds = 3.0 * sigma_a / (2.0 * s_tr)
    dzr = -1.0 / (st * st)            # same for sigma_a and sigma_s'
    dzv = c_v * dzr
    dF = 2.0 * 1.440 / eta ** 3 - 0.710 / (eta * eta) + 0.0636
    dA = 2.0 * dF / ((1.0 - F) ** 2)
    dzv_deta = zr * 4.0 * dA / 3.0
    hs = hr + hv
    d_a = pref * (dalpha_da * hs + alpha * ((hr_s + hv_s) * dstr_da + hr_z * dzr + hv_z * dzv))
    d_s = pref * (dalpha_ds * hs + alpha * ((hr_s + hv_s) * dstr_ds + hr_z * dzr + hv_z * dzv))
    d_e = pref * alpha * hv_z * dzv_deta
    return d_a, d_s, d_e


# ----------------------------------------------------------------------------
# Section 2.2, Eq. 5: PCA of sampled R_d
# ----------------------------------------------------------------------------


def radius_grid(n_r: int = 1024, r_max: float = 40.0) -> np.ndarray:
    """Reading R11: r_m = r_max * m / (n_r - 1)."""
    return r_max * np.arange(n_r, dtype=np.float64) / (n_r - 1)


def sample_matrix(sigma_a, sigma_s, eta, n_r=1024, r_max=40.0):
    """R[s, m] = R_d(r_m; sigma_a[s], sigma_s'[s], eta): the matrix factorised in Eq. 5."""
    r = radius_grid(n_r, r_max)
    sa = np.asarray(sigma_a, dtype=np.float64)[:, None]
    ss = np.asarray(sigma_s, dtype=np.float64)[:, None]
    return dipole_rd(r[None, :], sa, ss, eta)


def fit_pca_basis(sigma_a, sigma_s, eta=1.3, n_r=1024, r_max=40.0, K=12):
    """Eq. 5 and Section 2.2: radial basis f_k = k-th right singular vector of R (R7-R9).

    Returns (f [K][n_r], singular values [min(S, n_r)]).  The SVD is a library
    primitive (LAPACK via numpy).
    """
    R = sample_matrix(sigma_a, sigma_s, eta, n_r, r_max)
    _, s, vt = np.linalg.svd(R, full_matrices=False)
    f = vt[:K].copy()
    for k in range(K):
        m = int(np.argmax(np.abs(f[k])))
        if f[k, m] < 0:
            f[k] = -f[k]
    return f, s


def project_material(f, sigma_a, sigma_s, eta, r_max=40.0):
    """Section 2.2 (coefficients by projection) and rendering Step 3: g_k = sum_m f_k(r_m) R_d(r_m).

    sigma_a, sigma_s: (n, 3) per RGB channel; eta: (n,).  Returns g (n, 3, K).
    """
    K, n_r = f.shape
    r = radius_grid(n_r, r_max)
    sa = np.asarray(sigma_a)
    ss = np.asarray(sigma_s)
    eta = np.asarray(eta)
    R = dipole_rd(r[None, None, :], sa[..., None], ss[..., None], eta[:, None, None])  # (n,3,n_r)
    return R @ f.T


def project_material_vjp(f, sigma_a, sigma_s, eta, dg, r_max=40.0):
    """Reverse mode of ``project_material``: given dL/dg (n,3,K) return dL/dsigma_a (n,3), dL/dsigma_s' (n,3), dL/deta (n,)."""
    K, n_r = f.shape
    r = radius_grid(n_r, r_max)
    sa = np.asarray(sigma_a)[..., None]
    ss = np.asarray(sigma_s)[..., None]
    et = np.asarray(eta)[:, None, None]
    d_a, d_s, d_e = dipole_rd_partials(r[None, None, :], sa, ss, et)   # (n,3,n_r)
    w = dg @ f                                                         # (n,3,n_r): sum_k dg_k f_k(r_m)
    return (w * d_a).sum(-1), (w * d_s).sum(-1), (w * d_e).sum(-1).sum(-1)


# ----------------------------------------------------------------------------
# Section 3, Eq. 6-7: the transfer
# ----------------------------------------------------------------------------


def pair_r2_fp32(xo, xi):
    """FP32 squared distance used only for the r > r_max cutoff decision (reading R12).

    dx = fl(x_o - x_i) per axis, r2 = fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)), all
    IEEE binary32 round-to-nearest, so the cutoff is taken in the same
    precision on the CPU and the GPU.
    """
    d = (np.asarray(xo, dtype=np.float32)[..., :] - np.asarray(xi, dtype=np.float32)).astype(np.float32)
    sq = (d * d).astype(np.float32)
    return ((sq[..., 0] + sq[..., 1]).astype(np.float32) + sq[..., 2]).astype(np.float32)


def basis_eval(f, r, r_max=40.0, r2_fp32=None):
    """Reading R12: f_k(r) piecewise linear on the grid of R11, zero beyond r_max.

    f: (K, n_r); r: any shape (float64).  If ``r2_fp32`` is given, the cutoff
    is ``r2_fp32 > fl32(r_max^2)``; otherwise ``r > r_max``.
    Returns (K,) + r.shape.
    """
    K, n_r = f.shape
    dr = r_max / (n_r - 1)
    x = np.asarray(r, dtype=np.float64) / dr
    m = np.minimum(np.floor(x).astype(np.int64), n_r - 2)
    m = np.maximum(m, 0)
    t = x - m
    val = f[:, m] * (1.0 - t) + f[:, m + 1] * t
    if r2_fp32 is not None:
        outside = r2_fp32 > np.float32(r_max * r_max)
    else:
        outside = np.asarray(r) > r_max
    return np.where(outside, 0.0, val)


def transfer_rows(f, pos, area, T, rows, r_max=40.0):
    """Eq. 6-7 by brute force: M[k, j, o] = sum_i A_i f_k(|x_o - x_i|) T[j, i] for o in ``rows``.

    pos: (N, 3) float32 positions (mm); area: (N,); T: (J, N).  The double sum
    is taken one output row at a time, over every i (the self pair included).
    Returns (K, J, len(rows)).
    """
    pos32 = np.asarray(pos, dtype=np.float32)
    p64 = pos32.astype(np.float64)
    Tw = np.asarray(T, dtype=np.float64) * np.asarray(area, dtype=np.float64)[None, :]   # T'[j,i] = A_i T[j,i]
    K = f.shape[0]
    out = np.empty((K, Tw.shape[0], len(rows)))
    for q, o in enumerate(rows):
        r = np.sqrt(((p64[o][None, :] - p64) ** 2).sum(axis=1))
        F = basis_eval(f, r, r_max, r2_fp32=pair_r2_fp32(pos32[o][None, :], pos32))   # (K, N)
        out[:, :, q] = F @ Tw.T
    return out


def transfer_full(f, pos, area, T, r_max=40.0):
    """All rows of ``transfer_rows``."""
    return transfer_rows(f, pos, area, T, np.arange(np.asarray(pos).shape[0]), r_max)


# ----------------------------------------------------------------------------
# Section 3.2, Eq. 9-10: spatial Haar over the rhombic charts
# ----------------------------------------------------------------------------


def chart_side(nu: int) -> int:
    """P = 2^ceil(log2 nu): padded chart side (reading R21)."""
    P = 1
    while P < nu:
        P *= 2
    return P


def morton_index(row, col, P):
    """Morton (Z-order) index of (row, col) in a P x P chart: col bits even, row bits odd."""
    row = np.asarray(row, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    m = np.zeros(np.broadcast(row, col).shape, dtype=np.int64)
    b = 0
    while (1 << b) < P:
        m |= ((col >> b) & 1) << (2 * b)
        m |= ((row >> b) & 1) << (2 * b + 1)
        b += 1
    return m


def haar_forward_1d(x):
    """Orthonormal Haar analysis by its recursive definition (pairwise (a+b)/sqrt2, (a-b)/sqrt2).

    Output order: [scaling, coarsest detail, ..., finest details (len/2)].  len(x) = 2^L.
    """
    x = np.asarray(x)
    if x.shape[-1] == 1:
        return x.copy()
    a = (x[..., 0::2] + x[..., 1::2]) / math.sqrt(2.0)
    d = (x[..., 0::2] - x[..., 1::2]) / math.sqrt(2.0)
    return np.concatenate([haar_forward_1d(a), d], axis=-1)


def haar_inverse_1d(c):
    """Inverse of ``haar_forward_1d``."""
    c = np.asarray(c)
    n = c.shape[-1]
    if n == 1:
        return c.copy()
    a = haar_inverse_1d(c[..., : n // 2])
    d = c[..., n // 2:]
    x = np.empty(c.shape, dtype=np.result_type(c, np.float64))
    x[..., 0::2] = (a + d) / math.sqrt(2.0)
    x[..., 1::2] = (a - d) / math.sqrt(2.0)
    return x


def chart_to_wavelet(X, nu):
    """Spatial wavelet transform w_1 of Eq. 9 applied to per-vertex data X[..., N].

    Chart d's nu x nu values go to Morton positions of a zero-padded P x P
    domain and are Haar-analysed; the result has layout [..., 10 P^2 + 2] with
    chart d at [d P^2, (d+1) P^2) and the two poles last.
    """
    X = np.asarray(X, dtype=np.float64)
    P = chart_side(nu)
    rr, cc = np.meshgrid(np.arange(nu), np.arange(nu), indexing="ij")
    mort = morton_index(rr, cc, P).reshape(-1)
    lead = X.shape[:-1]
    out = np.zeros(lead + (10 * P * P + 2,))
    for d in range(10):
        dom = np.zeros(lead + (P * P,))
        dom[..., mort] = X[..., d * nu * nu:(d + 1) * nu * nu]
        out[..., d * P * P:(d + 1) * P * P] = haar_forward_1d(dom)
    out[..., 10 * P * P:] = X[..., 10 * nu * nu:]
    return out


def wavelet_to_chart(C, nu):
    """Inverse spatial transform w_1^{-1} (Eq. 10, rendering Step 5); drops the padding."""
    C = np.asarray(C, dtype=np.float64)
    P = chart_side(nu)
    rr, cc = np.meshgrid(np.arange(nu), np.arange(nu), indexing="ij")
    mort = morton_index(rr, cc, P).reshape(-1)
    lead = C.shape[:-1]
    out = np.zeros(lead + (10 * nu * nu + 2,))
    for d in range(10):
        dom = haar_inverse_1d(C[..., d * P * P:(d + 1) * P * P])
        out[..., d * nu * nu:(d + 1) * nu * nu] = dom[..., mort]
    out[..., 10 * nu * nu:] = C[..., 10 * P * P:]
    return out


# ---------------------------------------------------------------- Fresnel transmittance
def fresnel_transmittance(eta, mu):
    """F_t(eta, omega) of Eq. 3 and Eq. 6 under reading R34: one minus the exact unpolarised
    Fresnel reflectance of a dielectric boundary of relative index eta, for a direction outside at
    cosine mu to the normal (by reciprocity the same for light leaving towards omega); 0 for mu <= 0."""
    mu = np.asarray(mu)
    eta = np.asarray(eta)
    mpos = np.where(np.real(mu) > 0, mu, 1.0)
    ct = np.sqrt(1.0 - (1.0 - mpos * mpos) / (eta * eta))          # cosine of the refracted ray
    rs = (mpos - eta * ct) / (mpos + eta * ct)
    rp = (eta * mpos - ct) / (eta * mpos + ct)
    Ft = 1.0 - 0.5 * (rs * rs + rp * rp)
    return np.where(np.real(mu) > 0, Ft, 0.0)


def fresnel_transmittance_deta(eta, mu):
    """Hand derivative dF_t/deta of fresnel_transmittance (0 for mu <= 0)."""
    mu = np.asarray(mu, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    mpos = np.where(mu > 0, mu, 1.0)
    q = 1.0 - mpos * mpos
    ct = np.sqrt(1.0 - q / (eta * eta))
    dct = q / (eta ** 3 * ct)
    a, da = eta * ct, ct + eta * dct
    rs = (mpos - a) / (mpos + a)
    drs = -2.0 * mpos * da / (mpos + a) ** 2
    u, w = eta * mpos - ct, eta * mpos + ct
    rp = u / w
    drp = ((mpos - dct) * w - u * (mpos + dct)) / (w * w)
    return np.where(mu > 0, -(rs * drs + rp * drp), 0.0)


def fresnel_output(B, eta, cos_o):
    """Eq. 6's view-dependent factor (1/pi) F_t(eta, omega_o) applied to B (E, 3, N), per edit eta (E,)
    and per output vertex cos_o (N,) = n_o . omega_o."""
    fac = fresnel_transmittance(np.asarray(eta, dtype=np.float64)[:, None], np.asarray(cos_o, dtype=np.float64)[None, :])
    return np.asarray(B, dtype=np.float64) * (fac / math.pi)[:, None, :]


def fresnel_output_vjp(B, eta, cos_o, dBout):
    """Reverse mode of fresnel_output: (dL/dB (E,3,N), dL/deta (E,))."""
    eta = np.asarray(eta, dtype=np.float64)[:, None]
    cos_o = np.asarray(cos_o, dtype=np.float64)[None, :]
    fac = fresnel_transmittance(eta, cos_o) / math.pi
    dfac = fresnel_transmittance_deta(eta, cos_o) / math.pi
    dBout = np.asarray(dBout, dtype=np.float64)
    dB = dBout * fac[:, None, :]
    deta = np.einsum("eco,eco,eo->e", dBout, np.asarray(B, dtype=np.float64), dfac)
    return dB, deta


def sh_real_oracle(order: int, dirs) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_j(w), j = l^2 + l + m, l < order (reading R19):
    Y_l0 = N_l0 P_l(z), Y_lm = sqrt(2) N_lm P_l^m(z) cos(m phi), Y_l,-m = sqrt(2) N_lm P_l^m(z) sin(m phi),
    N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), with P_l^m the associated Legendre function WITHOUT the
    Condon-Shortley phase (scipy's lpmv carries (-1)^m, which is removed here).  Returns (order^2, R)."""
    from scipy.special import lpmv
    d = np.asarray(dirs, dtype=np.float64)
    z = np.clip(d[:, 2], -1.0, 1.0)
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.empty((order * order, d.shape[0]))
    for l in range(order):
        for m in range(0, l + 1):
            Nlm = math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            Plm = (-1.0) ** m * lpmv(m, l, z)
            if m == 0:
                out[l * l + l] = Nlm * Plm
            else:
                out[l * l + l + m] = math.sqrt(2.0) * Nlm * Plm * np.cos(m * phi)
                out[l * l + l - m] = math.sqrt(2.0) * Nlm * Plm * np.sin(m * phi)
    return out


def sh_zonal_fresnel(eta, order):
    """Zonal coefficients of h(mu) = F_t(eta, mu) max(mu, 0) (reading R35):
    A_l = 2 pi int_0^1 F_t(eta, mu) mu P_l(mu) dmu, l < order, so that by the Funk-Hecke theorem
    int Y_lm(w) h(n . w) dw = A_l Y_lm(n).  eta = 1 gives the clamped cosine."""
    from scipy.integrate import quad
    from numpy.polynomial import legendre
    out = np.empty(order)
    for l in range(order):
        Pl = legendre.Legendre.basis(l)
        val, _ = quad(lambda m: float(fresnel_transmittance(eta, m)) * m * Pl(m), 0.0, 1.0,
                      limit=400, epsabs=1e-13, epsrel=1e-13)
        out[l] = 2.0 * math.pi * val
    return out


def sh_transfer_fresnel(normals, J, eta):
    """T[j, i] = A_l(eta) Y_lm(n_i): the unshadowed irradiance transfer with the incident Fresnel
    transmittance folded in (Eq. 6 with F_t(eta, omega_i) inside E; readings R18, R19, R35)."""
    order = int(round(math.sqrt(J)))
    Y = sh_real_oracle(order, np.asarray(normals, dtype=np.float64))
    A = sh_zonal_fresnel(eta, order)
    for l in range(order):
        Y[l * l:(l + 1) * (l + 1)] *= A[l]
    return Y


# ---------------------------------------------------------------- ray-cast visibility (reading R36)
def onb_from_normal(n):
    """Orthonormal tangents (t1, t2) of unit normals n (..., 3) by the branchless construction of
    Duff et al. (2017, "Building an orthonormal basis, revisited")."""
    n = np.asarray(n, dtype=np.float64)
    sign = np.where(n[..., 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sign + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t1 = np.stack([1.0 + sign * n[..., 0] ** 2 * a, sign * b, -sign * n[..., 0]], axis=-1)
    t2 = np.stack([b, sign + n[..., 1] ** 2 * a, -n[..., 1]], axis=-1)
    return t1, t2


def hemisphere_samples(S: int):
    """Cosine-weighted directions in the local frame (z = normal) from the Hammersley set:
    u1 = (s + 1/2) / S, u2 = bit-reversed s; r = sqrt(u1), phi = 2 pi u2, z = sqrt(1 - u1)."""
    s = np.arange(S)
    u1 = (s + 0.5) / S
    u2 = np.zeros(S)
    f, v = 0.5, s.copy()
    while np.any(v):
        u2 += f * (v & 1)
        v >>= 1
        f *= 0.5
    r = np.sqrt(u1)
    return np.stack([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2), np.sqrt(1.0 - u1)], axis=-1)


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def ray_hits_any(orig, dirs, v0, v1, v2, t_min=1e-4):
    """Any-hit of rays (R, 3) against triangles (F, 3 each) by the Moller-Trumbore test, in FP32
    with a fixed operation order (no fused multiply-add) so that the decision is reproducible:
    dot(a, b) = (a.x b.x + a.y b.y) + a.z b.z, cross by components, inv = 1/det, a hit needs
    |det| >= 1e-12, u, v >= 0, u + v <= 1 and t > t_min.  Returns a bool (R,) array."""
    o, d = _f32(orig)[:, None, :], _f32(dirs)[:, None, :]
    a, b, c = _f32(v0)[None], _f32(v1)[None], _f32(v2)[None]

    def cross(x, y):
        return np.stack([x[..., 1] * y[..., 2] - x[..., 2] * y[..., 1],
                         x[..., 2] * y[..., 0] - x[..., 0] * y[..., 2],
                         x[..., 0] * y[..., 1] - x[..., 1] * y[..., 0]], axis=-1)

    def dot(x, y):
        return (x[..., 0] * y[..., 0] + x[..., 1] * y[..., 1]) + x[..., 2] * y[..., 2]

    e1, e2 = b - a, c - a
    p = cross(d, e2)
    det = dot(e1, p)
    ok = np.abs(det) >= np.float32(1e-12)
    inv = np.float32(1.0) / np.where(ok, det, np.float32(1.0))
    tv = o - a
    u = dot(tv, p) * inv
    q = cross(tv, e1)
    v = dot(d, q) * inv
    t = dot(e2, q) * inv
    hit = ok & (u >= 0) & (v >= 0) & (u + v <= np.float32(1.0)) & (t > np.float32(t_min))
    return hit.any(axis=1)


def visibility_transfer(pos, tris, normals, J, S, eps=1e-3, eta=None):
    """Self-shadowed SH irradiance transfer T[j, i] = (pi / S) sum_s Y_j(w_s) V(x_i, w_s) [F_t(eta, mu_s)]
    (Eq. 6's E with visibility; reading R36): w_s the cosine-weighted Hammersley directions in the frame
    of n_i, rays from x_i + eps n_i (FP32), V = 0 when the ray hits any triangle of the mesh."""
    pos32, n32 = _f32(pos), _f32(normals)
    t1, t2 = onb_from_normal(n32.astype(np.float64))
    loc = hemisphere_samples(S)
    order = int(round(math.sqrt(J)))
    N = pos32.shape[0]
    v0, v1, v2 = pos32[tris[:, 0]], pos32[tris[:, 1]], pos32[tris[:, 2]]
    T = np.zeros((J, N))
    for i in range(N):
        dirs = _f32(loc[:, :1] * t1[i] + loc[:, 1:2] * t2[i] + loc[:, 2:3] * n32[i].astype(np.float64))
        orig = np.repeat((pos32[i] + np.float32(eps) * n32[i])[None, :], S, axis=0)
        vis = ~ray_hits_any(orig, dirs, v0, v1, v2)
        w = (math.pi / S) * vis.astype(np.float64)
        if eta is not None:
            w = w * fresnel_transmittance(eta, loc[:, 2])
        T[:, i] = sh_real_oracle(order, dirs.astype(np.float64)) @ w
    return T


# ---------------------------------------------------------------- CDF 9/7 spatial wavelet
# The paper's Step-2 wavelet ("Daubechies 9/7", Section 5), reading R33: the
# biorthogonal Cohen-Daubechies-Feauveau 9/7 pair in the lifting factorisation of
# Daubechies and Sweldens (the one JPEG 2000 uses), whole-sample symmetric
# extension at the ends, scaled so that the low band has DC gain sqrt(2) (the
# normalisation of the orthonormal Haar); on each chart the separable 2D Mallat
# pyramid of the P x P image (row-major, chart pixel (r, c) = vertex d nu^2 + r nu + c,
# zero padding), every level transforming rows then columns of the low-low band,
# down to 1 x 1.
CDF97_ALPHA = -1.586134342059924
CDF97_BETA = -0.052980118572961
CDF97_GAMMA = 0.882911075530934
CDF97_DELTA = 0.443506852043971
CDF97_ZETA = 1.149604398860241


def _lift_1d(x):
    """One analysis level on the last axis (even length n): returns [low (n/2) | high (n/2)]."""
    x = np.asarray(x, dtype=np.float64)
    s = x[..., 0::2].copy()
    d = x[..., 1::2].copy()
    for c, target in ((CDF97_ALPHA, "d"), (CDF97_BETA, "s"), (CDF97_GAMMA, "d"), (CDF97_DELTA, "s")):
        if target == "d":    # d_i += c (s_i + s_{i+1}), s beyond the end mirrored: s_m = s_{m-1}
            s_next = np.concatenate([s[..., 1:], s[..., -1:]], axis=-1)
            d = d + c * (s + s_next)
        else:                # s_i += c (d_{i-1} + d_i), d_{-1} = d_0
            d_prev = np.concatenate([d[..., :1], d[..., :-1]], axis=-1)
            s = s + c * (d_prev + d)
    return np.concatenate([s * CDF97_ZETA, d / CDF97_ZETA], axis=-1)


def _unlift_1d(y):
    """Inverse of _lift_1d on the last axis."""
    y = np.asarray(y, dtype=np.float64)
    m = y.shape[-1] // 2
    s = y[..., :m] / CDF97_ZETA
    d = y[..., m:] * CDF97_ZETA
    for c, target in ((CDF97_DELTA, "s"), (CDF97_GAMMA, "d"), (CDF97_BETA, "s"), (CDF97_ALPHA, "d")):
        if target == "d":
            s_next = np.concatenate([s[..., 1:], s[..., -1:]], axis=-1)
            d = d - c * (s + s_next)
        else:
            d_prev = np.concatenate([d[..., :1], d[..., :-1]], axis=-1)
            s = s - c * (d_prev + d)
    x = np.empty(y.shape)
    x[..., 0::2] = s
    x[..., 1::2] = d
    return x


def cdf97_forward_2d(img):
    """Mallat pyramid of (..., P, P) images: per level rows then columns of the low-low band."""
    a = np.array(img, dtype=np.float64)
    n = a.shape[-1]
    while n >= 2:
        a[..., :n, :n] = _lift_1d(a[..., :n, :n])
        a[..., :n, :n] = np.swapaxes(_lift_1d(np.swapaxes(a[..., :n, :n], -1, -2)), -1, -2)
        n //= 2
    return a


def cdf97_inverse_2d(coef):
    a = np.array(coef, dtype=np.float64)
    P = a.shape[-1]
    n = 2
    while n <= P:
        a[..., :n, :n] = np.swapaxes(_unlift_1d(np.swapaxes(a[..., :n, :n], -1, -2)), -1, -2)
        a[..., :n, :n] = _unlift_1d(a[..., :n, :n])
        n *= 2
    return a


def chart_to_cdf97(X, nu):
    """Spatial CDF 9/7 transform of per-vertex data X[..., N] (reading R33): chart d's image
    at [d P^2, (d+1) P^2) of the result (row-major pyramid), the two poles last."""
    X = np.asarray(X, dtype=np.float64)
    P = chart_side(nu)
    lead = X.shape[:-1]
    out = np.zeros(lead + (10 * P * P + 2,))
    for d in range(10):
        img = np.zeros(lead + (P, P))
        img[..., :nu, :nu] = X[..., d * nu * nu:(d + 1) * nu * nu].reshape(lead + (nu, nu))
        out[..., d * P * P:(d + 1) * P * P] = cdf97_forward_2d(img).reshape(lead + (P * P,))
    out[..., 10 * P * P:] = X[..., 10 * nu * nu:]
    return out


def cdf97_to_chart(C, nu):
    """Inverse of chart_to_cdf97 (synthesis; drops the padding)."""
    C = np.asarray(C, dtype=np.float64)
    P = chart_side(nu)
    lead = C.shape[:-1]
    out = np.zeros(lead + (10 * nu * nu + 2,))
    for d in range(10):
        img = cdf97_inverse_2d(C[..., d * P * P:(d + 1) * P * P].reshape(lead + (P, P)))
        out[..., d * nu * nu:(d + 1) * nu * nu] = img[..., :nu, :nu].reshape(lead + (nu * nu,))
    out[..., 10 * nu * nu:] = C[..., 10 * P * P:]
    return out


def cdf97_synthesis_matrix(nu):
    """The explicit matrix S (N x (10 P^2 + 2)) of cdf97_to_chart, column by column (small nu only)."""
    P = chart_side(nu)
    NW = 10 * P * P + 2
    return cdf97_to_chart(np.eye(NW), nu).T


def keep_count(p: float, n_coef: int) -> int:
    """Reading R23: n_keep = floor(p * n_coef + 0.5), clamped to [1, n_coef]."""
    return int(min(n_coef, max(1, math.floor(p * n_coef + 0.5))))


def energy_keep_count(coef, e: float) -> int:
    """Precompute Step 2 (Section 3, "a threshold energy is pre-determined ... so that the
    reserved energy exceeds the threshold") under reading R32: the smallest n >= 1 such that
    the n largest |c| (ties: lower index) hold at least the fraction e of the row's energy
    sum c^2.  Energies in FP64, accumulated in that order (the total is the full sum)."""
    c = np.asarray(coef, dtype=np.float64).reshape(-1)
    order = np.lexsort((np.arange(c.size), -np.abs(c)))
    cum = np.cumsum(c[order] ** 2)
    total = cum[-1]
    if total == 0.0:
        return 1
    n = int(np.searchsorted(cum, e * total, side="left")) + 1   # first n with cum[n-1] >= e * total
    return min(max(n, 1), c.size)


def select_energy(Cw, nu, e):
    """Keep mask of the energy rule (reading R32) for wavelet coefficients Cw (K, J, 10 P^2 + 2):
    per (k, j) the energy_keep_count largest chart magnitudes (ties: lower index) plus the poles."""
    P = chart_side(nu)
    n_coef = 10 * P * P
    K, J, _ = Cw.shape
    mask = np.zeros(Cw.shape, dtype=bool)
    idx = np.arange(n_coef)
    for k in range(K):
        for j in range(J):
            row = Cw[k, j, :n_coef]
            nk = energy_keep_count(row, e)
            order = np.lexsort((idx, -np.abs(row).astype(np.float64)))
            mask[k, j, order[:nk]] = True
    mask[:, :, n_coef:] = True
    return mask


def select_top(Cw, nu, p):
    """Precompute Step 2 (Section 3.2) with the top-p keep rule of reading R23.

    Cw: (K, J, 10 P^2 + 2) wavelet coefficients (any float dtype; the ranking is
    taken on |value| in that dtype).  Returns a boolean keep mask of the same
    shape: per (k, j) the n_keep largest chart magnitudes (ties: lower index)
    plus the two poles.
    """
    P = chart_side(nu)
    n_coef = 10 * P * P
    nk = keep_count(p, n_coef)
    K, J, _ = Cw.shape
    mask = np.zeros(Cw.shape, dtype=bool)
    idx = np.arange(n_coef)
    for k in range(K):
        for j in range(J):
            mag = np.abs(Cw[k, j, :n_coef])
            order = np.lexsort((idx, -mag.astype(np.float64)))   # by -|c|, then index
            mask[k, j, order[:nk]] = True
    mask[:, :, n_coef:] = True
    return mask


# ----------------------------------------------------------------------------
# Section 4, rendering Steps 3-5: relight and its adjoint
# ----------------------------------------------------------------------------


def relight(Cw_kept, nu, g, light, wavelet="haar"):
    """Rendering Steps 3-5: B[e, ch, o] = w^{-1}( sum_{k,j} g[e,ch,k] l_j Cw[k, j, :] ).

    Cw_kept: (K, J, 10 P^2 + 2) kept wavelet coefficients (zeros where
    discarded); g: (E, 3, K); light: (J,).  Returns (E, 3, N).  wavelet: "haar"
    (R22) or "cdf97" (R33), the transform the coefficients are in.
    """
    c = np.asarray(g, dtype=np.float64)[..., :, None] * np.asarray(light, dtype=np.float64)[None, None, None, :]
    bw = np.einsum("eckj,kjw->ecw", c, np.asarray(Cw_kept, dtype=np.float64))
    return wavelet_to_chart(bw, nu) if wavelet == "haar" else cdf97_to_chart(bw, nu)


def relight_direct(f, pos, area, T, g, light, r_max=40.0, rows=None):
    """Uncompressed relight straight from Eq. 6: B[e,ch,o] = sum_i A_i (sum_k g_k f_k(r_oi)) E_i, E_i = sum_j l_j T[j,i]."""
    pos32 = np.asarray(pos, dtype=np.float32)
    p64 = pos32.astype(np.float64)
    N = p64.shape[0]
    rows = np.arange(N) if rows is None else rows
    E = np.asarray(light, dtype=np.float64) @ np.asarray(T, dtype=np.float64)          # (N,)
    AE = np.asarray(area, dtype=np.float64) * E
    g = np.asarray(g, dtype=np.float64)
    out = np.empty(g.shape[:2] + (len(rows),))
    for q, o in enumerate(rows):
        r = np.sqrt(((p64[o][None, :] - p64) ** 2).sum(axis=1))
        F = basis_eval(f, r, r_max, r2_fp32=pair_r2_fp32(pos32[o][None, :], pos32))   # (K, N)
        out[:, :, q] = g @ (F @ AE)
    return out


def relight_vjp(Cw_kept, nu, g, light, dB, wavelet="haar"):
    """Reverse mode of ``relight``: given dL/dB (E,3,N) return (dL/dg (E,3,K), dL/dl (J,)).

    dL/db^w = S^T dL/dB with S the synthesis (for the orthonormal Haar S^T is the
    analysis w_1; for CDF 9/7 the explicit transpose of the synthesis matrix),
    dL/dc[e,ch,k,j] = sum_w Cw[k,j,w] dL/db^w[e,ch,w],
    dL/dg_k = sum_j l_j dL/dc_kj, dL/dl_j = sum_{e,ch,k} g_k dL/dc_kj.
    """
    if wavelet == "haar":
        rw = chart_to_wavelet(dB, nu)
    else:
        rw = np.asarray(dB, dtype=np.float64) @ cdf97_synthesis_matrix(nu)
    dc = np.einsum("kjw,ecw->eckj", np.asarray(Cw_kept, dtype=np.float64), rw)
    light = np.asarray(light, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    dg = dc @ light
    dl = np.einsum("eck,eckj->j", g, dc)
    return dg, dl
