// Host-side geometry of one shell: grid spacings, FP64 metric tables and the
// Schwarz exchange tables (Sec. 2 Yin/Yang maps, Sec. 4 MAC placement and
// interpolated boundary data).
#include "geometry.h"

#include <cmath>
#include <vector>

namespace ys {

static const double kPi = 3.14159265358979323846;

double GridGeo::rhalf(int m) const {
  const int lo = -kGhostHalf, hi = 2 * Nr + kGhostHalf;
  if (m < lo) return rh[0] - (lo - m) * (rh[1] - rh[0]);
  if (m > hi) return rh.back() + (m - hi) * (rh.back() - rh[rh.size() - 2]);
  return rh[m + kGhostHalf];
}
double GridGeo::rc(int i) const { return rh.empty() ? R1 + (i + 0.5) * hr : rhalf(2 * i + 1); }
double GridGeo::rf(int i) const { return rh.empty() ? R1 + i * hr : rhalf(2 * i); }
double GridGeo::hc(int i) const { return rh.empty() ? hr : rf(i + 1) - rf(i); }
double GridGeo::hf(int i) const { return rh.empty() ? hr : rc(i) - rc(i - 1); }

int make_grid(const GridSpec &g, GridGeo &out) {
  if (!(g.R1 > 0.0) || !(g.R2 > g.R1)) return 1;
  if (g.overlap < 1 || g.Nth <= 2 * g.overlap + 4) return 1;
  out.hr = (g.R2 - g.R1) / g.Nr;
  out.R1 = g.R1;
  out.Nr = g.Nr;
  out.rh.clear();
  if (g.r_half) {
    // 2 Nr + 1 strictly increasing radii from R1 to R2; ghosts mirrored about the walls
    const int n = 2 * g.Nr + 1;
    const double tol = 1e-12 * (g.R2 - g.R1);
    for (int m = 0; m < n; ++m)
      if (!std::isfinite(g.r_half[m]) || (m > 0 && !(g.r_half[m] > g.r_half[m - 1]))) return 1;
    if (std::fabs(g.r_half[0] - g.R1) > tol || std::fabs(g.r_half[n - 1] - g.R2) > tol) return 1;
    out.rh.assign(n + 2 * kGhostHalf, 0.0);
    for (int m = 0; m < n; ++m) out.rh[m + kGhostHalf] = g.r_half[m];
    out.rh[kGhostHalf] = g.R1;
    out.rh[kGhostHalf + n - 1] = g.R2;
    for (int k = 1; k <= kGhostHalf; ++k) {
      out.rh[kGhostHalf - k] = 2.0 * g.R1 - out.rh[kGhostHalf + k];
      out.rh[kGhostHalf + n - 1 + k] = 2.0 * g.R2 - out.rh[kGhostHalf + n - 1 - k];
    }
  }
  out.ht = (kPi / 2) / (g.Nth - 2 * g.overlap);
  out.delta = g.overlap * out.ht;
  out.hp = (1.5 * kPi + 2 * out.delta) / g.Nph;
  out.th0 = kPi / 4 - out.delta;
  out.ph0 = -0.75 * kPi - out.delta;
  if (!(out.th0 > 0.0)) return 1;
  return 0;
}

void make_metric(const GridSpec &g, const GridGeo &G, std::vector<double> &tab, int &pad, int &len) {
  // kMetricTables tables (rc, rf, sc, sf, cc, cf and the reciprocals of rc,
  // rf, sc, sf), each indexed by logical index with `pad` slots below 0
  pad = 2;
  int n = (g.Nr > g.Nth ? g.Nr : g.Nth) + 2 * pad + 2;
  len = n;
  tab.assign(kMetricTables * (size_t)n, 0.0);
  auto inv = [](double v) { return v != 0.0 ? 1.0 / v : 0.0; };
  for (int t = 0; t < n; ++t) {
    int i = t - pad;
    double rc = G.rc(i), rf = G.rf(i);
    double thc = G.th0 + (i + 0.5) * G.ht, thf = G.th0 + i * G.ht;
    tab[0 * n + t] = rc;
    tab[1 * n + t] = rf;
    tab[2 * n + t] = std::sin(thc);
    tab[3 * n + t] = std::sin(thf);
    tab[4 * n + t] = std::cos(thc);
    tab[5 * n + t] = std::cos(thf);
    tab[6 * n + t] = inv(rc);
    tab[7 * n + t] = inv(rf);
    tab[8 * n + t] = inv(std::sin(thc));
    tab[9 * n + t] = inv(std::sin(thf));
    // radial spacing of cell i, its reciprocal, and the radial norm factors
    // r sqrt(h / h_r) of centres and faces (r on a uniform grid)
    tab[10 * n + t] = G.hc(i);
    tab[11 * n + t] = inv(G.hc(i));
    tab[12 * n + t] = rc * std::sqrt(G.hc(i) / G.hr);
    tab[13 * n + t] = rf * std::sqrt(G.hf(i) / G.hr);
  }
}

void make_rowcoef(const GridSpec &g, const GridGeo &G, const std::vector<double> &met, int pad, int len,
                  const RowPhys &ph, std::vector<double> tab[kRowTables]) {
  // metric lookups by logical index (tables of make_metric)
  auto T = [&](int t, int i) { return met[(size_t)t * len + i + pad]; };
  auto rc = [&](int i) { return T(0, i); };
  auto rf = [&](int i) { return T(1, i); };
  auto sc = [&](int j) { return T(2, j); };
  auto sf = [&](int j) { return T(3, j); };
  auto cc = [&](int j) { return T(4, j); };
  auto cf = [&](int j) { return T(5, j); };
  auto irc = [&](int i) { return T(6, i); };
  auto irf = [&](int i) { return T(7, i); };
  auto isc = [&](int j) { return T(8, j); };
  auto isf = [&](int j) { return T(9, j); };
  const double iht = 1.0 / G.ht, ihp = 1.0 / G.hp;
  // reciprocal radial spacings: of cell i (centre), and between the centres
  // on either side of face i (both 1/h_r on a uniform radial grid)
  auto ihc = [&](int i) { return 1.0 / G.hc(i); };
  auto ihf = [&](int i) { return 1.0 / G.hf(i); };
  const double dt = ph.dt, nu = ph.nu, ka = ph.kappa, i2chi = ph.i2chi;
  const int NJ = g.Nth + 2;
  const size_t rows = (size_t)(g.Nr + 2) * NJ;
  for (int t = 0; t < kRowTables; ++t) tab[t].assign(rows * row_m(t), 0.0);
  auto rec = [&](int t, int i, int j) { return &tab[t][((size_t)(i + 1) * NJ + (j + 1)) * row_m(t)]; };

  // temperature at cell centres (i, j): kappa Laplacian, advection by the
  // 2-point face averages of the advecting velocity (the kernel forms their
  // sums), and the deviation-form source
  for (int i = 0; i < g.Nr; ++i)
    for (int j = 0; j < g.Nth; ++j) {
      double *c = rec(RT_T, i, j);
      const double ir = irc(i), is = isc(j), ir2 = ir * ir;
      c[T_RP] = 0.5 * dt * ka * rf(i + 1) * rf(i + 1) * ir2 * ihc(i) * ihf(i + 1);
      c[T_RM] = 0.5 * dt * ka * rf(i) * rf(i) * ir2 * ihc(i) * ihf(i);
      c[T_TP] = 0.5 * dt * ka * sf(j + 1) * ir2 * is * iht * iht;
      c[T_TM] = 0.5 * dt * ka * sf(j) * ir2 * is * iht * iht;
      c[T_PP] = 0.5 * dt * ka * ir2 * is * is * ihp * ihp;
      c[T_AR] = 0.125 * dt * ihc(i);
      c[T_AT] = 0.125 * dt * ir * iht;
      c[T_AP] = 0.125 * dt * ir * is * ihp;
      c[T_G0] = ph.Tc_lap ? dt * ka * ph.Tc_lap[i] : 0.0;
      c[T_G1] = ph.Tc_dr ? 0.5 * dt * ph.Tc_dr[i] : 0.0;
    }

  // u_r at r-face i (1 .. Nr-1), cell row j
  for (int i = 1; i < g.Nr; ++i)
    for (int j = 0; j < g.Nth; ++j) {
      double *c = rec(RT_UR, i, j);
      const double ir = irf(i), is = isc(j), ir2 = ir * ir;
      const double rfp = rf(i + 1), rf0 = rf(i), rfm = rf(i - 1);
      const double icc = irc(i), icm = irc(i - 1);   // the two cells sharing face i
      c[UR_RP] = 0.5 * dt * nu * rc(i) * rc(i) * ir2 * ihf(i) * ihc(i);
      c[UR_RM] = 0.5 * dt * nu * rc(i - 1) * rc(i - 1) * ir2 * ihf(i) * ihc(i - 1);
      c[UR_TP] = 0.5 * dt * nu * sf(j + 1) * ir2 * is * iht * iht;
      c[UR_TM] = 0.5 * dt * nu * sf(j) * ir2 * is * iht * iht;
      c[UR_PP] = 0.5 * dt * nu * ir2 * is * is * ihp * ihp;
      // own values outside the Laplacian: the curvature term of the vector
      // Laplacian and the r-part of grad(div) across the two cells
      const double G = 0.5 * dt * ihf(i) * i2chi;
      c[UR_O1] = 0.5 * dt * nu * ir2 * ir * ihf(i) * rfp * rfp + G * rfp * rfp * icc * icc * ihc(i);
      c[UR_O0] = -dt * nu * ir2 - G * rf0 * rf0 * (icc * icc * ihc(i) + icm * icm * ihc(i - 1));
      c[UR_OM] = -0.5 * dt * nu * ir2 * ir * ihf(i) * rfm * rfm + G * rfm * rfm * icm * icm * ihc(i - 1);
      // u_theta at (q + P, q, q - SI + P, q - SI): theta-part of grad(div)
      c[UR_GT1] = G * sf(j + 1) * icc * is * iht;
      c[UR_GT0] = -G * sf(j) * icc * is * iht;
      c[UR_GTM1] = -G * sf(j + 1) * icm * is * iht;
      c[UR_GTM0] = G * sf(j) * icm * is * iht;
      // u_phi differences (q + 1) - q and (q - SI + 1) - (q - SI)
      c[UR_GP1] = G * icc * is * ihp;
      c[UR_GPM1] = -G * icm * is * ihp;
      c[UR_AR] = 0.25 * dt * ihf(i);
      c[UR_AT] = 0.0625 * dt * ir * iht;
      c[UR_AP] = 0.0625 * dt * ir * is * ihp;
      c[UR_CV] = dt * ir / 32.0;
      c[UR_GPR] = dt * ihf(i);
      c[UR_BY] = 0.25 * dt * ph.PrRa;
    }

  // u_theta at cell row i, theta-face j (1 .. Nth-1)
  for (int i = 0; i < g.Nr; ++i)
    for (int j = 1; j < g.Nth; ++j) {
      double *c = rec(RT_UT, i, j);
      const double ir = irc(i), is = isf(j), cs = cf(j), ir2 = ir * ir;
      const double rfp = rf(i + 1), rf0 = rf(i);
      const double isj = isc(j), ism = isc(j - 1);   // the two cells sharing face j
      c[UT_RP] = 0.5 * dt * nu * rfp * rfp * ir2 * ihc(i) * ihf(i + 1);
      c[UT_RM] = 0.5 * dt * nu * rf0 * rf0 * ir2 * ihc(i) * ihf(i);
      c[UT_TP] = 0.5 * dt * nu * sc(j) * ir2 * is * iht * iht;
      c[UT_TM] = 0.5 * dt * nu * sc(j - 1) * ir2 * is * iht * iht;
      c[UT_PP] = 0.5 * dt * nu * ir2 * is * is * ihp * ihp;
      const double G = 0.5 * dt * i2chi * ir * iht;
      const double E = 0.5 * dt * nu * cs * ir2 * is * is * iht;
      c[UT_OTP] = E * sf(j + 1) + G * sf(j + 1) * ir * isj * iht;
      c[UT_O0] = -0.5 * dt * nu * ir2 * is * is - G * sf(j) * ir * (isj + ism) * iht;
      c[UT_OTM] = -E * sf(j - 1) + G * sf(j - 1) * ir * ism * iht;
      // u_r at (q + SI, q, q + SI - P, q - P): vector-Laplacian coupling and
      // r-part of grad(div)
      const double a = 0.5 * dt * nu * ir2 * iht, b = 0.5 * dt * nu * cs * ir2 * ir * is * ihc(i);
      c[UT_W1] = a + b * rfp * rfp + G * rfp * rfp * ir * ir * ihc(i);
      c[UT_W0] = a - b * rf0 * rf0 - G * rf0 * rf0 * ir * ir * ihc(i);
      c[UT_WM1] = -a + b * rfp * rfp - G * rfp * rfp * ir * ir * ihc(i);
      c[UT_WM0] = -a - b * rf0 * rf0 + G * rf0 * rf0 * ir * ir * ihc(i);
      c[UT_GP1] = G * ir * isj * ihp;
      c[UT_GPM1] = -G * ir * ism * ihp;
      c[UT_AR] = 0.0625 * dt * ihc(i);
      c[UT_AT] = 0.25 * dt * ir * iht;
      c[UT_AP] = 0.0625 * dt * ir * is * ihp;
      c[UT_CW] = 0.125 * dt * ir;
      c[UT_CP] = dt * ir * cs * is / 32.0;
      c[UT_GPR] = dt * irc(i) * iht;
    }

  // u_phi at cell row (i, j), phi-faces
  for (int i = 0; i < g.Nr; ++i)
    for (int j = 0; j < g.Nth; ++j) {
      double *c = rec(RT_UP, i, j);
      const double ir = irc(i), is = isc(j), cs = cc(j), ir2 = ir * ir;
      const double rfp = rf(i + 1), rf0 = rf(i);
      c[UP_RP] = 0.5 * dt * nu * rfp * rfp * ir2 * ihc(i) * ihf(i + 1);
      c[UP_RM] = 0.5 * dt * nu * rf0 * rf0 * ir2 * ihc(i) * ihf(i);
      c[UP_TP] = 0.5 * dt * nu * sf(j + 1) * ir2 * is * iht * iht;
      c[UP_TM] = 0.5 * dt * nu * sf(j) * ir2 * is * iht * iht;
      // the phi-part of grad(div) has the stencil of the phi-diffusion
      c[UP_PP] = 0.5 * dt * (nu + i2chi) * ir2 * is * is * ihp * ihp;
      c[UP_E0] = -0.5 * dt * nu * ir2 * is * is;
      const double G = 0.5 * dt * i2chi * ir * is * ihp;
      const double a = 0.5 * dt * nu * ir2 * is * ihp, b = 0.5 * dt * nu * cs * ir2 * is * is * ihp;
      // u_r at (q + SI, q, q - 1 + SI, q - 1)
      c[UP_W1] = a + G * rfp * rfp * ir2 * ihc(i);
      c[UP_W0] = a - G * rf0 * rf0 * ir2 * ihc(i);
      c[UP_WM1] = -a - G * rfp * rfp * ir2 * ihc(i);
      c[UP_WM0] = -a + G * rf0 * rf0 * ir2 * ihc(i);
      // u_theta at (q + P, q, q - 1 + P, q - 1)
      c[UP_Y1] = b + G * sf(j + 1) * ir * is * iht;
      c[UP_Y0] = b - G * sf(j) * ir * is * iht;
      c[UP_YM1] = -b - G * sf(j + 1) * ir * is * iht;
      c[UP_YM0] = -b + G * sf(j) * ir * is * iht;
      c[UP_AR] = 0.0625 * dt * ihc(i);
      c[UP_AT] = 0.0625 * dt * ir * iht;
      c[UP_AP] = 0.25 * dt * ir * is * ihp;
      c[UP_CW] = 0.125 * dt * ir;
      c[UP_CY] = 0.125 * dt * ir * cs * is;
      c[UP_GPR] = dt * ir * is * ihp;
    }

  // divergence of the half-level velocity times 1/chi at cell (i, j), and the
  // weight r^2 sin(theta) of the pressure-increment norm
  for (int i = 0; i < g.Nr; ++i)
    for (int j = 0; j < g.Nth; ++j) {
      double *c = rec(RT_DIV, i, j);
      const double ir = irc(i), is = isc(j);
      c[DV_R1] = i2chi * rf(i + 1) * rf(i + 1) * ir * ir * ihc(i);
      c[DV_R0] = i2chi * rf(i) * rf(i) * ir * ir * ihc(i);
      c[DV_T1] = i2chi * sf(j + 1) * ir * is * iht;
      c[DV_T0] = i2chi * sf(j) * ir * is * iht;
      c[DV_P] = i2chi * ir * is * ihp;
      c[DV_W] = rc(i) * rc(i) * sc(j) * (G.hc(i) / G.hr);   // r^2 sin(theta) h / h_r
    }
}

void make_faccoef(const GridSpec &g, const GridGeo &G, const std::vector<double> &met, int pad, int len,
                  const FacPhys &ph, std::vector<double> &tab) {
  auto T = [&](int t, int i) { return met[(size_t)t * len + i + pad]; };
  auto rc = [&](int i) { return T(0, i); };
  auto rf = [&](int i) { return T(1, i); };
  auto sc = [&](int j) { return T(2, j); };
  auto sf = [&](int j) { return T(3, j); };
  auto cf = [&](int j) { return T(5, j); };
  auto irc = [&](int i) { return T(6, i); };
  auto irf = [&](int i) { return T(7, i); };
  auto isc = [&](int j) { return T(8, j); };
  auto isf = [&](int j) { return T(9, j); };
  const double iht = 1.0 / G.ht, ihp = 1.0 / G.hp;
  auto ihc = [&](int i) { return 1.0 / G.hc(i); };   // as in make_rowcoef
  auto ihf = [&](int i) { return 1.0 / G.hf(i); };
  const int NJ = g.Nth + 2;
  const size_t rows = (size_t)(g.Nr + 2) * NJ;
  tab.assign((size_t)kFacTables * rows * FC_M, 0.0);
  for (int loc = LC; loc <= LP; ++loc)
    for (int dir = DR; dir <= DP; ++dir)
      for (int i = (loc == LR) ? 1 : 0; i < g.Nr; ++i)
        for (int j = (loc == LT) ? 1 : 0; j < g.Nth; ++j) {
          // (I - dt/2 Ahat_dir): the diffusion along dir (modified operators
          // with R1 and theta_1 for theta and phi), the own-direction extras
          // of the vector Laplacian and of grad(div)/(2 chi), and the
          // advection a d/dx_dir whose coefficient is ka
          const double nu = (loc == LC) ? ph.kappa : ph.nu;
          const double ir = (loc == LR) ? irf(i) : irc(i);
          const double is = (loc == LT) ? isf(j) : isc(j);
          const double ir2 = ir * ir;
          double cm, c0, cp, ka;
          if (dir == DR) {
            // h of the row's point and of the half points on either side
            const double ih = (loc == LR) ? ihf(i) : ihc(i);
            const double ihp_ = (loc == LR) ? ihc(i) : ihf(i + 1), ihm_ = (loc == LR) ? ihc(i - 1) : ihf(i);
            const double cp_d = (loc == LR) ? rc(i) * rc(i) * (ir2 * ih * ihp_) : rf(i + 1) * rf(i + 1) * (ir2 * ih * ihp_);
            const double cm_d = (loc == LR) ? rc(i - 1) * rc(i - 1) * (ir2 * ih * ihm_) : rf(i) * rf(i) * (ir2 * ih * ihm_);
            cm = nu * cm_d;
            c0 = -nu * (cp_d + cm_d);
            cp = nu * cp_d;
            ka = 0.5 * ih;
            if (loc == LR) {
              const double rfm = rf(i - 1), rf0 = rf(i), rfp = rf(i + 1), irm = irc(i - 1), ic = irc(i);
              cm -= nu * rfm * rfm * (ir2 * ir * ih);
              cp += nu * rfp * rfp * (ir2 * ir * ih);
              c0 -= nu * 2.0 * ir2;
              cm += ph.i2chi * rfm * rfm * (irm * irm * ihm_ * ih);
              c0 -= ph.i2chi * (rf0 * rf0 * (ic * ic * ihp_ * ih) + rf0 * rf0 * (irm * irm * ihm_ * ih));
              cp += ph.i2chi * rfp * rfp * (ic * ic * ihp_ * ih);
            }
          } else if (dir == DT) {
            const double cp_d = (loc == LT) ? sc(j) * (ph.iR1sq * is * iht * iht) : sf(j + 1) * (ph.iR1sq * is * iht * iht);
            const double cm_d = (loc == LT) ? sc(j - 1) * (ph.iR1sq * is * iht * iht) : sf(j) * (ph.iR1sq * is * iht * iht);
            cm = nu * cm_d;
            c0 = -nu * (cp_d + cm_d);
            cp = nu * cp_d;
            ka = 0.5 * ir * iht;
            if (loc == LT) {
              const double qq = cf(j) * ir2 * is * is * iht;
              cm -= nu * qq * sf(j - 1);
              cp += nu * qq * sf(j + 1);
              c0 -= nu * ir2 * is * is;
              const double isc0 = isc(j), iscm = isc(j - 1);
              cp += ph.i2chi * sf(j + 1) * (ir2 * isc0 * iht * iht);
              c0 -= ph.i2chi * (sf(j) * (ir2 * isc0 * iht * iht) + sf(j) * (ir2 * iscm * iht * iht));
              cm += ph.i2chi * sf(j - 1) * (ir2 * iscm * iht * iht);
            }
          } else {
            cm = nu * ph.cphi;
            c0 = -2.0 * nu * ph.cphi;
            cp = nu * ph.cphi;
            ka = 0.5 * ir * is * ihp;
            if (loc == LP) {
              c0 -= nu * ir2 * is * is;
              const double qq = ph.i2chi * ir2 * is * is * ihp * ihp;
              cm += qq;
              c0 -= 2.0 * qq;
              cp += qq;
            }
          }
          double *c = &tab[((size_t)(3 * loc + dir) * rows + (size_t)(i + 1) * NJ + (j + 1)) * FC_M];
          c[FC_L0] = -0.5 * ph.dt * cm;
          c[FC_D0] = 1.0 - 0.5 * ph.dt * c0;
          c[FC_U0] = -0.5 * ph.dt * cp;
          c[FC_LA] = -0.5 * ph.dt * ka;
        }
  (void)rc;
  (void)sc;
}

namespace {

struct V3 {
  double x, y, z;
};
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// M(x, y, z) = (-x, z, y): Yin <-> Yang local Cartesian coordinates
inline V3 Mmap(V3 a) { return V3{-a.x, a.z, a.y}; }
inline V3 unit(double th, double ph) {
  return V3{std::sin(th) * std::cos(ph), std::sin(th) * std::sin(ph), std::cos(th)};
}
inline V3 e_th(double th, double ph) {
  return V3{std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph), -std::sin(th)};
}
inline V3 e_ph(double, double ph) { return V3{-std::sin(ph), std::cos(ph), 0.0}; }

// bilinear stencil of a donor quantity staggered (face_t, face_p) at donor
// angles; checks that the 2x2 stencil lies within [jlo, jhi] x [klo, khi]
bool stencil(const GridSpec &g, const GridGeo &G, bool face_t, bool face_p, double th, double ph, int shrink,
             int &j0, int &k0, double &wj, double &wk) {
  double jf = (th - G.th0) / G.ht - (face_t ? 0.0 : 0.5);
  double kf = (ph - G.ph0) / G.hp - (face_p ? 0.0 : 0.5);
  j0 = (int)std::floor(jf);
  k0 = (int)std::floor(kf);
  wj = jf - j0;
  wk = kf - k0;
  int jlo = face_t ? 1 : 0, jhi = face_t ? g.Nth - 1 : g.Nth - 1;
  int klo = face_p ? 1 : 0, khi = face_p ? g.Nph - 1 : g.Nph - 1;
  jlo += shrink;
  jhi -= shrink;
  klo += shrink;
  khi -= shrink;
  return j0 >= jlo && j0 + 1 <= jhi && k0 >= klo && k0 + 1 <= khi;
}

}  // namespace

int make_exchange(const GridSpec &g, const GridGeo &G, std::vector<XEntry> tabs[XNUM]) {
  const int Nt = g.Nth, Np = g.Nph;
  for (int kind = 0; kind < XNUM; ++kind) {
    std::vector<XEntry> &T = tabs[kind];
    T.clear();
    std::vector<std::pair<int, int>> pts;
    if (kind == XT || kind == XUR) {
      for (int j : {-1, Nt})
        for (int k = 0; k < Np; ++k) pts.push_back({j, k});
      for (int k : {-1, Np})
        for (int j = 0; j < Nt; ++j) pts.push_back({j, k});
    } else if (kind == XUT) {
      for (int j : {0, Nt})
        for (int k = 0; k < Np; ++k) pts.push_back({j, k});
      for (int k : {-1, Np})
        for (int j = 1; j < Nt; ++j) pts.push_back({j, k});
    } else if (kind == XUP) {
      for (int k : {0, Np})
        for (int j = 0; j < Nt; ++j) pts.push_back({j, k});
      for (int j : {-1, Nt})
        for (int k = 1; k < Np; ++k) pts.push_back({j, k});
    } else {  // pressure ring: outermost interior cells
      for (int j = 0; j < Nt; ++j)
        for (int k = 0; k < Np; ++k)
          if (j == 0 || j == Nt - 1 || k == 0 || k == Np - 1) pts.push_back({j, k});
    }
    for (auto &pt : pts) {
      XEntry e{};
      e.tj = pt.first;
      e.tk = pt.second;
      double th = G.th0 + (pt.first + (kind == XUT ? 0.0 : 0.5)) * G.ht;
      double ph = G.ph0 + (pt.second + (kind == XUP ? 0.0 : 0.5)) * G.hp;
      V3 xd = Mmap(unit(th, ph));
      double thd = std::acos(xd.z < -1 ? -1 : (xd.z > 1 ? 1 : xd.z));
      double phd = std::atan2(xd.y, xd.x);
      if (kind == XT || kind == XUR || kind == XP) {
        if (!stencil(g, G, false, false, thd, phd, kind == XP ? 1 : 0, e.j0a, e.k0a, e.wja, e.wka)) return 1;
        e.ra = 1.0;
        e.rb = 0.0;
      } else {
        if (!stencil(g, G, true, false, thd, phd, 0, e.j0a, e.k0a, e.wja, e.wka)) return 1;
        if (!stencil(g, G, false, true, thd, phd, 0, e.j0b, e.k0b, e.wjb, e.wkb)) return 1;
        V3 et = (kind == XUT) ? e_th(th, ph) : e_ph(th, ph);
        e.ra = dot(et, Mmap(e_th(thd, phd)));
        e.rb = dot(et, Mmap(e_ph(thd, phd)));
      }
      T.push_back(e);
    }
  }
  return 0;
}

}  // namespace ys
