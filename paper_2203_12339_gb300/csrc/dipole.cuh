// Dipole diffuse reflectance R_d (Section 2.1, Eq. 4) and its analytic partial
// derivatives, in FP64 on the device.
//
// Readings of the printed formula: sigma_t' = sigma_a + sigma_s',
// sigma_tr = sqrt(3 sigma_a sigma_t'), the virtual-source term uses 1/d_v,
// z_r = 1/sigma_t', z_v = z_r (1 + 4A/3), A = (1 + F_dr)/(1 - F_dr) with the
// polynomial F_dr(eta) of Section 2.1; both source terms are added.
#pragma once

namespace tsr {

struct DipoleMaterial {
  double alpha;   // alpha' = sigma_s' / sigma_t'
  double s_tr;    // sigma_tr
  double zr, zv;  // source depths
  // partials of the intermediates (used only for gradients)
  double dalpha_da, dalpha_ds, dstr_da, dstr_ds, dzr, dzv, dzv_deta;
};

__device__ __forceinline__ DipoleMaterial dipole_material(double sa, double ss, double eta) {
  DipoleMaterial m;
  const double st = sa + ss;
  m.alpha = ss / st;
  m.s_tr = sqrt(3.0 * sa * st);
  m.zr = 1.0 / st;
  const double F = -1.440 / (eta * eta) + 0.710 / eta + 0.668 + 0.0636 * eta;
  const double A = (1.0 + F) / (1.0 - F);
  const double cv = 1.0 + 4.0 * A / 3.0;
  m.zv = m.zr * cv;
  m.dalpha_da = -ss / (st * st);
  m.dalpha_ds = sa / (st * st);
  m.dstr_da = 3.0 * (st + sa) / (2.0 * m.s_tr);
  m.dstr_ds = 3.0 * sa / (2.0 * m.s_tr);
  m.dzr = -1.0 / (st * st);
  m.dzv = cv * m.dzr;
  const double dF = 2.0 * 1.440 / (eta * eta * eta) - 0.710 / (eta * eta) + 0.0636;
  const double dA = 2.0 * dF / ((1.0 - F) * (1.0 - F));
  m.dzv_deta = m.zr * 4.0 * dA / 3.0;
  return m;
}

// One source term h(z) = z (s_tr + 1/d) e^{-s_tr d} / d^2, d = sqrt(r^2 + z^2).
__device__ __forceinline__ double dipole_term(double r, double z, double s_tr) {
  const double d = sqrt(r * r + z * z);
  return z * (s_tr + 1.0 / d) * exp(-s_tr * d) / (d * d);
}

__device__ __forceinline__ double dipole_rd(double r, const DipoleMaterial &m) {
  return m.alpha * (0.25 / 3.14159265358979323846) *
         (dipole_term(r, m.zr, m.s_tr) + dipole_term(r, m.zv, m.s_tr));
}

// R_d and (dR/dsigma_a, dR/dsigma_s', dR/deta).  With h as above:
//   dh/ds_tr = -s_tr z e^{-s_tr d} / d
//   dh/dz    = (s_tr + 1/d) e^{-s_tr d}/d^2 - (z^2/d) e^{-s_tr d} (s_tr^2/d^2 + 3 s_tr/d^3 + 3/d^4)
__device__ __forceinline__ void dipole_rd_grad(double r, const DipoleMaterial &m, double &R,
                                               double &dRa, double &dRs, double &dRe) {
  double h[2], hs[2], hz[2];
  const double z2[2] = {m.zr, m.zv};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double z = z2[q];
    const double d = sqrt(r * r + z * z);
    const double id = 1.0 / d;
    const double e = exp(-m.s_tr * d);
    h[q] = z * (m.s_tr + id) * e * id * id;
    hs[q] = -m.s_tr * z * e * id;
    hz[q] = (m.s_tr + id) * e * id * id -
            z * z * id * e * (m.s_tr * m.s_tr * id * id + 3.0 * m.s_tr * id * id * id + 3.0 * id * id * id * id);
  }
  const double pref = 0.25 / 3.14159265358979323846;
  const double hsum = h[0] + h[1];
  R = pref * m.alpha * hsum;
  const double dstr_term = hs[0] + hs[1];
  dRa = pref * (m.dalpha_da * hsum + m.alpha * (dstr_term * m.dstr_da + hz[0] * m.dzr + hz[1] * m.dzv));
  dRs = pref * (m.dalpha_ds * hsum + m.alpha * (dstr_term * m.dstr_ds + hz[0] * m.dzr + hz[1] * m.dzv));
  dRe = pref * m.alpha * hz[1] * m.dzv_deta;
}

}  // namespace tsr
