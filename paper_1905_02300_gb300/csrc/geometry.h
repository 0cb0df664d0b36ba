// Host-side geometry of one shell (see geometry.cpp).
#pragma once
#include <vector>

#include "ys_internal.cuh"

namespace ys {

struct GridSpec {
  double R1, R2;
  int Nr, Nth, Nph, overlap;
  const double *r_half;   // 2 Nr + 1 radial half-point radii (faces even, centres odd), or null (uniform)
};

// Grid spacings and the radial positions.  hr is the uniform grid's radial
// spacing (R2 - R1) / Nr, the reference of the norms' cell volume.  A
// non-uniform radial grid keeps its half points in rh with kGhostHalf ghost
// half points on either side, mirrored about the walls; positions beyond
// them (used only by table padding) are extended linearly.
constexpr int kGhostHalf = 4;
struct GridGeo {
  double hr, ht, hp, delta, th0, ph0;
  double R1 = 0.0;
  int Nr = 0;
  std::vector<double> rh;   // empty: uniform
  double rhalf(int m) const;
  double rc(int i) const;   // centre of radial cell i
  double rf(int i) const;   // radial face i
  double hc(int i) const;   // width of radial cell i, rf(i + 1) - rf(i)
  double hf(int i) const;   // distance of the centres on either side of face i, rc(i) - rc(i - 1)
};

// 0 on success, 1 if the parameters do not define a valid patch
int make_grid(const GridSpec &g, GridGeo &out);
// kMetricTables FP64 tables rc, rf, sc, sf, cc, cf, 1/rc, 1/rf, 1/sc, 1/sf of
// length `len`, logical index i at slot i + pad
void make_metric(const GridSpec &g, const GridGeo &G, std::vector<double> &tab, int &pad, int &len);
// physical constants entering the residual row coefficients
struct RowPhys {
  double dt, nu, kappa, i2chi, PrRa;
  const double *Tc_lap, *Tc_dr;   // deviation-form temperature sources per cell row i, or null
};
// row-coefficient tables (RowTable) of length (Nr + 2) (Nth + 2) row_m(t),
// from the FP64 metric tables `met` (layout of make_metric)
void make_rowcoef(const GridSpec &g, const GridGeo &G, const std::vector<double> &met, int pad, int len,
                  const RowPhys &ph, std::vector<double> tab[kRowTables]);
// static line-operator coefficient tables (FacCoef), [kFacTables][(Nr + 2)(Nth + 2)][FC_M]
struct FacPhys {
  double dt, nu, kappa, i2chi, iR1sq, cphi;
};
void make_faccoef(const GridSpec &g, const GridGeo &G, const std::vector<double> &met, int pad, int len,
                  const FacPhys &ph, std::vector<double> &tab);
// exchange tables for every kind; 1 if a donor stencil leaves the donor's
// unknowns (grid too coarse)
int make_exchange(const GridSpec &g, const GridGeo &G, std::vector<XEntry> tabs[XNUM]);

}  // namespace ys
