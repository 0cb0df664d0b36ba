// Internal definitions shared by the CUDA translation units of the solver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ys {

// Location types of the MAC grid (Sec. 4): cell centre, r-face, theta-face, phi-face.
enum Loc { LC = 0, LR = 1, LT = 2, LP = 3 };
enum Dir { DR = 0, DT = 1, DP = 2 };

// Device layout of one field of one shell: both patches, each a box of logical
// indices i in [-1, Nr], j in [-1, Nth], k in [-1, Nph] (faces use their face
// index, which fits the same box).  Rows along phi have pitch P (a multiple of
// 8 elements) and start 8 elements into the allocation, so k = 0 of every row
// is 64-byte aligned for FP64 and k = -1 lives in the previous row's padding.
struct Layout {
  int Nr, Nt, Np;   // cells per patch
  int NJ;           // Nt + 2 rows per r-plane
  int P;            // row pitch in elements
  long SI;          // r-plane stride = NJ * P
  long PS;          // patch stride
  long total;       // elements per field (both patches)
};

__host__ __device__ inline long lidx(const Layout &L, int p, int i, int j, int k) {
  return p * L.PS + ((long)(i + 1) * L.NJ + (j + 1)) * (long)L.P + k + 8;
}

struct Shell;

// Number of FP64 metric tables (rc, rf, sc, sf, cc, cf, irc, irf, isc, isf).
constexpr int kMetricTables = 10;
enum MetricTable { MT_RC = 0, MT_RF, MT_SC, MT_SF, MT_CC, MT_CF, MT_IRC, MT_IRF, MT_ISC, MT_ISF };
// scalar constants mirrored in both arithmetic types
enum ShellConst { CS_IHR = 0, CS_IHT, CS_IHP, CS_I2CHI, CS_IR1SQ, CS_CPHI, CS_DT, CS_NU, CS_KAPPA, CS_PRRA, CS_NUM };

// Everything a kernel needs about one shell (passed by value).
struct Shell {
  Layout L;
  double hr, ht, hp;        // spacings
  double R1, sin_theta1;    // modified operators (Sec. 3.2)
  double dt, nu, kappa, chi, PrRa;
  // metric tables in FP64, indexed by logical index (pointers offset so that
  // index -2 .. N+2 is valid)
  const double *rc, *rf;    // r at centres / faces
  const double *sc, *sf;    // sin(theta) at centres / faces
  const double *cc, *cf;    // cos(theta) at centres / faces
  const double *irc, *irf;  // 1/r at centres / faces
  const double *isc, *isf;  // 1/sin(theta) at centres / faces
  double ihr, iht, ihp;     // 1/h_r, 1/h_theta, 1/h_phi
  double i2chi;             // 1/(2 chi)
  double iR1sq;             // 1/R1^2 (modified theta operator)
  double cphi;              // 1/(R1^2 sin^2(theta_1) h_phi^2) (modified phi operator)
  // the same metric tables and constants indexed by MetricTable / ShellConst,
  // in FP64 and rounded to FP32 (computed in FP64 on the host), so that FP32
  // stencils need no per-use conversions
  const double *dtab[kMetricTables];
  const float *ftab[kMetricTables];
  double dcs[CS_NUM];
  float fcs[CS_NUM];
  double T_in, T_out;       // wall temperatures (of the stored temperature)
  // deviation form (mixed precision): the stored temperature is T - T_c with
  // T_c the discrete conductive profile; its rate gets the FP64 source
  // Tc_lap[i] - a_r Tc_dr[i] (null in the FP64 form)
  const double *Tc_lap, *Tc_dr;
  int step7;
};


// Exchange table entry: one target point in the (theta, phi) plane of a patch,
// with one or two bilinear donor stencils on the other patch and, for
// tangential vector components, the 2x2 rotation row.
struct XEntry {
  int tj, tk;           // target logical (j, k)
  int j0a, k0a;         // donor stencil A base (logical)
  double wja, wka;      // donor stencil A weights along theta, phi
  int j0b, k0b;         // donor stencil B base (vectors: u_phi donor)
  double wjb, wkb;
  double ra, rb;        // target = ra * A + rb * B (vectors); ra = 1, rb = 0 for scalars
};

// Table kinds.
enum XKind { XT = 0, XUR = 1, XUT = 2, XUP = 3, XP = 4, XNUM = 5 };

}  // namespace ys

namespace ys {

// metric table / constant in the arithmetic type V
template <typename V>
__host__ __device__ inline const V *mt(const Shell &S, int t);
template <>
__host__ __device__ inline const double *mt<double>(const Shell &S, int t) {
  return S.dtab[t];
}
template <>
__host__ __device__ inline const float *mt<float>(const Shell &S, int t) {
  return S.ftab[t];
}
template <typename V>
__host__ __device__ inline V cs(const Shell &S, int c);
template <>
__host__ __device__ inline double cs<double>(const Shell &S, int c) {
  return S.dcs[c];
}
template <>
__host__ __device__ inline float cs<float>(const Shell &S, int c) {
  return S.fcs[c];
}

// fill dtab / dcs from the named FP64 fields (ftab / fcs are filled by the owner)
inline void shell_fill_fp64(Shell &S) {
  const double *t[kMetricTables] = {S.rc, S.rf, S.sc, S.sf, S.cc, S.cf, S.irc, S.irf, S.isc, S.isf};
  for (int k = 0; k < kMetricTables; ++k) S.dtab[k] = t[k];
  const double c[CS_NUM] = {S.ihr, S.iht, S.ihp, S.i2chi, S.iR1sq, S.cphi, S.dt, S.nu, S.kappa, S.PrRa};
  for (int k = 0; k < CS_NUM; ++k) {
    S.dcs[k] = c[k];
    S.fcs[k] = (float)c[k];
  }
}

}  // namespace ys
