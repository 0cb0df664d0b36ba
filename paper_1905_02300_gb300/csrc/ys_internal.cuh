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

// Number of FP64 metric tables (rc, rf, sc, sf, cc, cf, irc, irf, isc, isf;
// then the radial cell width hc, its reciprocal, and the radial norm factors
// nrc = rc sqrt(hc / h_r), nrf = rf sqrt(hf / h_r) of centres and faces, which
// equal rc, rf on a uniform radial grid).
constexpr int kMetricTables = 14;
// Divergence watch of the Schwarz iteration (failure detection; the paper
// has none): the largest squared increment norm of the previous iteration of
// the step in progress, and a sticky flag, kept beside the norm accumulators.
// An iteration whose increment norms are not finite sets it, and so does,
// from a step's third iteration on, a largest increment norm above
// kWatchGrowth times the previous iteration's that is also above the step's
// first increment: a working defect correction contracts from its second
// iteration on (the first may jump, e.g. where the buoyancy of the first
// temperature increment starts the velocity), so growth by three orders of
// magnitude in one iteration past the first increment is divergence.  (An
// iteration that has converged to the rounding level of its arithmetic can
// grow by that much from a still smaller second increment, but stays far
// below the first.)
constexpr int kWatchPrev = 24, kWatchFlag = 25, kWatchFirst = 26;   // indices in the per-context norm buffer (32 doubles)
constexpr double kWatchGrowth = 1e3;
enum MetricTable {
  MT_RC = 0, MT_RF, MT_SC, MT_SF, MT_CC, MT_CF, MT_IRC, MT_IRF, MT_ISC, MT_ISF, MT_HC, MT_IHC, MT_NRC, MT_NRF
};
// scalar constants mirrored in both arithmetic types
// (CS_VOL = h_r h_theta h_phi, the coordinate cell volume of the midpoint-rule
// norms on a uniform radial grid; a non-uniform one carries the ratio h / h_r
// of each point in its norm factors nrc, nrf)
enum ShellConst { CS_IHR = 0, CS_IHT, CS_IHP, CS_I2CHI, CS_IR1SQ, CS_CPHI, CS_DT, CS_NU, CS_KAPPA, CS_PRRA, CS_VOL, CS_NUM };

// Row-coefficient tables of the explicit residuals.  On the MAC grid every
// metric factor of the residual stencils depends on the row (i, j) only, so
// the products of metric factors, spacings, dt, nu, kappa and 1/(2 chi) that
// multiply each stencil value are formed once per row on the host in FP64
// (geometry.cpp) and kept in FP64 and FP32.  The stencils take sums
// S = psi + psi^n of the two time levels (the half-level value is S / 2; the
// 1/2 is folded into the coefficients).  One record of *_M values per row,
// record index (i + 1) * (Nth + 2) + (j + 1).
enum RowTable { RT_T = 0, RT_UR, RT_UT, RT_UP, RT_DIV, kRowTables };
// temperature (cell centres)
enum RowT { T_RP = 0, T_RM, T_TP, T_TM, T_PP, T_AR, T_AT, T_AP, T_G0, T_G1, T_M };
// u_r (r-faces)
enum RowUR { UR_RP = 0, UR_RM, UR_TP, UR_TM, UR_PP, UR_O1, UR_O0, UR_OM, UR_GT1, UR_GT0, UR_GTM1, UR_GTM0,
             UR_GP1, UR_GPM1, UR_AR, UR_AT, UR_AP, UR_CV, UR_GPR, UR_BY, UR_M };
// u_theta (theta-faces)
enum RowUT { UT_RP = 0, UT_RM, UT_TP, UT_TM, UT_PP, UT_OTP, UT_O0, UT_OTM, UT_W1, UT_W0, UT_WM1, UT_WM0,
             UT_GP1, UT_GPM1, UT_AR, UT_AT, UT_AP, UT_CW, UT_CP, UT_GPR, UT_M };
// u_phi (phi-faces)
enum RowUP { UP_RP = 0, UP_RM, UP_TP, UP_TM, UP_PP, UP_E0, UP_W1, UP_W0, UP_WM1, UP_WM0, UP_Y1, UP_Y0,
             UP_YM1, UP_YM0, UP_AR, UP_AT, UP_AP, UP_CW, UP_CY, UP_GPR, UP_M };
// divergence times 1/chi for the pressure update, and the norm weight r^2 sin(theta)
enum RowDiv { DV_R1 = 0, DV_R0, DV_T1, DV_T0, DV_P, DV_W, DV_M };
// values per record of table t
__host__ __device__ constexpr int row_m(int t) {
  return t == RT_T ? T_M : t == RT_UR ? UR_M : t == RT_UT ? UT_M : t == RT_UP ? UP_M : DV_M;
}

// Static parts of the line-operator coefficients: the rows of
// (I - dt/2 Ahat_dir) at a point of location loc are lo = L0 + a La,
// di = D0, up = U0 - a La, with a the advecting velocity along dir at the
// point; L0, D0, U0, La depend on the row (i, j) only.  Table
// t = 3 loc + dir, record index (i + 1) (Nth + 2) + (j + 1).
enum FacCoef { FC_L0 = 0, FC_D0, FC_U0, FC_LA, FC_M };
constexpr int kFacTables = 12;

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
  const double *hc, *ihc;   // radial cell width and its reciprocal per cell
  const double *nrc, *nrf;  // radial norm factors r sqrt(h / h_r) of centres / faces
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
  // FP32 remainders x - (double)ftab[x] of the tables and constants: with
  // ftab / fcs they carry each FP64 value as a double-float pair
  const float *ltab[kMetricTables];
  float lcs[CS_NUM];
  // row-coefficient tables (RowTable), FP64 and the same values rounded to FP32
  const double *rowd[kRowTables];
  const float *rowf[kRowTables];
  // line-operator coefficient tables (FacCoef), [kFacTables][rows][FC_M]
  const double *facd;
  const float *facf;
  double T_in, T_out;       // wall temperatures (of the stored temperature)
  // temperature ghost beyond wall w: gamma[w] T_0 + delta[w] T_wall (the wall
  // condition a T + b dT/dn = T_wall; Dirichlet: -1, 2)
  double Tgam[2], Tdel[2];
  // deviation form (mixed precision): the stored temperature is T - T_c with
  // T_c the discrete conductive profile; its rate gets the FP64 source
  // Tc_lap[i] - a_r Tc_dr[i] (null in the FP64 form)
  const double *Tc_lap, *Tc_dr;
  // Dirichlet wall velocity (FP64, user layout [wall][patch][j][k] per
  // component, as ys_set_wall_velocity); null = no-slip
  const double *wall_ur, *wall_ut, *wall_up;
  int step7;
};

// Time-dependent wall data tau(t) W (ys_set_wall_data), passed to the wall
// kernel beside the shell: wall temperature [wall][patch][j][k] at the
// cell-centre angles, added to T_in / T_out, and wall velocity in the layouts
// of Shell::wall_*, added to the steady one; tau at the time of the state
// whose boundary values the launch fills.  Null pointers: no such part.
struct WallData {
  const double *T, *ur, *ut, *up;
  double tau;
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
// row-coefficient record of row (i, j) in table t, in the arithmetic type V
template <typename V>
__host__ __device__ inline const V *rowc(const Shell &S, int t, int i, int j);
template <>
__host__ __device__ inline const double *rowc<double>(const Shell &S, int t, int i, int j) {
  return S.rowd[t] + ((long)(i + 1) * (S.L.Nt + 2) + (j + 1)) * row_m(t);
}
template <>
__host__ __device__ inline const float *rowc<float>(const Shell &S, int t, int i, int j) {
  return S.rowf[t] + ((long)(i + 1) * (S.L.Nt + 2) + (j + 1)) * row_m(t);
}
// static line-operator coefficients of row (i, j) for (loc, dir), in the arithmetic type V
template <typename V>
__host__ __device__ inline const V *facc(const Shell &S, int loc, int dir, int i, int j);
template <>
__host__ __device__ inline const double *facc<double>(const Shell &S, int loc, int dir, int i, int j) {
  const long rows = (long)(S.L.Nr + 2) * (S.L.Nt + 2);
  return S.facd + ((3 * loc + dir) * rows + (long)(i + 1) * (S.L.Nt + 2) + (j + 1)) * FC_M;
}
template <>
__host__ __device__ inline const float *facc<float>(const Shell &S, int loc, int dir, int i, int j) {
  const long rows = (long)(S.L.Nr + 2) * (S.L.Nt + 2);
  return S.facf + ((3 * loc + dir) * rows + (long)(i + 1) * (S.L.Nt + 2) + (j + 1)) * FC_M;
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

// Ghost of the temperature wall condition a T + b dT/dn = T_w (inner: w = 0,
// outer: w = 1) with T = (T_g + T_0)/2 and dT/dn = (T_g - T_0)/h on the wall,
// h the distance of the ghost centre from the first one (h_in, h_out):
// T_g = Tgam[w] T_0 + Tdel[w] T_w.  a = 1, b = 0 is the Dirichlet reflection
// T_g = 2 T_w - T_0.
inline void shell_set_T_walls(Shell &S, const double a[2], const double b[2], double h_in, double h_out) {
  const double h[2] = {h_in, h_out};
  for (int w = 0; w < 2; ++w) {
    const double den = 0.5 * a[w] + b[w] / h[w];
    S.Tgam[w] = -(0.5 * a[w] - b[w] / h[w]) / den;
    S.Tdel[w] = 1.0 / den;
  }
}

// fill dtab / dcs / fcs / lcs from the named FP64 fields (ftab / ltab are filled by the owner)
inline void shell_fill_fp64(Shell &S) {
  const double *t[kMetricTables] = {S.rc, S.rf, S.sc, S.sf, S.cc, S.cf, S.irc, S.irf, S.isc, S.isf,
                                    S.hc, S.ihc, S.nrc, S.nrf};
  for (int k = 0; k < kMetricTables; ++k) S.dtab[k] = t[k];
  const double c[CS_NUM] = {S.ihr, S.iht, S.ihp, S.i2chi, S.iR1sq, S.cphi, S.dt, S.nu, S.kappa, S.PrRa,
                            S.hr * S.ht * S.hp};
  for (int k = 0; k < CS_NUM; ++k) {
    S.dcs[k] = c[k];
    S.fcs[k] = (float)c[k];
    S.lcs[k] = (float)(c[k] - (double)S.fcs[k]);
  }
}

}  // namespace ys
