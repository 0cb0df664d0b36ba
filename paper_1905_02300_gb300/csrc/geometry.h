// Host-side geometry of one shell (see geometry.cpp).
#pragma once
#include <vector>

#include "ys_internal.cuh"

namespace ys {

struct GridSpec {
  double R1, R2;
  int Nr, Nth, Nph, overlap;
};

struct GridGeo {
  double hr, ht, hp, delta, th0, ph0;
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
