// Explicit MAC-stencil kernels: extrapolation, residuals of the defect
// correction (-F = dt Rate(psi^{1/2}) - (psi - psi^n), Sec. 4 Eq. er), pressure
// updates (Eq. nst_Mass1 and Eq. ac2), and host-layout packing.
//
// Every rate is the discrete operator of Sec. 3.2 / Sec. 3.3 on the MAC grid:
// conservative 3-point diffusion with the metric at half points, centred
// first derivatives (2-point across a half-cell offset, 2h otherwise),
// off-location values as arithmetic means of the 2 or 4 nearest stored
// values, metric factors evaluated exactly at the row's point.
#include "kernels.cuh"

namespace ys {

namespace {

constexpr int TPB = 128;

template <typename R>
__device__ __forceinline__ double H(const R *a, const R *b, long q) {
  return 0.5 * ((double)a[q] + (double)b[q]);
}

template <typename R>
__device__ __forceinline__ double avg4(const R *a, long q1, long q2, long q3, long q4) {
  return (((double)a[q1] + (double)a[q2]) + (double)a[q3] + (double)a[q4]) * 0.25;
}

// half-level average of 4 points of a pair of arrays
template <typename R>
__device__ __forceinline__ double havg4(const R *a, const R *b, long q1, long q2, long q3, long q4) {
  return ((H(a, b, q1) + H(a, b, q2)) + H(a, b, q3) + H(a, b, q4)) * 0.25;
}

// region of unknowns of a location type, logical half-open ranges
__device__ __forceinline__ void region(const Layout &L, int loc, int &i0, int &i1, int &j0, int &j1, int &k0,
                                       int &k1) {
  i0 = (loc == LR) ? 1 : 0;
  i1 = L.Nr;
  j0 = (loc == LT) ? 1 : 0;
  j1 = L.Nt;
  k0 = (loc == LP) ? 1 : 0;
  k1 = L.Np;
}

// Point decode for the residual grids: blockIdx.y enumerates (p, i, j) rows
// of the region, threads run along k.
__device__ __forceinline__ bool decode_point(const Layout &L, int loc, int patch_mask, int &p, int &i, int &j,
                                             int &k) {
  int i0, i1, j0, j1, k0, k1;
  region(L, loc, i0, i1, j0, j1, k0, k1);
  int nj = j1 - j0, ni = i1 - i0;
  int row = blockIdx.y;
  j = j0 + row % nj;
  row /= nj;
  i = i0 + row % ni;
  p = row / ni;
  k = k0 + blockIdx.x * blockDim.x + threadIdx.x;
  return k < k1 && ((patch_mask >> p) & 1);
}

// discrete divergence of the half-level velocity at cell (p, i, j, k)
template <typename R>
__device__ __forceinline__ double divh(const Shell &S, const R *ri, const R *rn, const R *ti, const R *tn,
                                       const R *pi, const R *pn, int i, int j, long q) {
  const Layout &L = S.L;
  double ir = S.irc[i], is = S.isc[j];
  double d_r = (S.rf[i + 1] * S.rf[i + 1] * H(ri, rn, q + L.SI) - S.rf[i] * S.rf[i] * H(ri, rn, q)) *
               (ir * ir * S.ihr);
  double d_t = (S.sf[j + 1] * H(ti, tn, q + L.P) - S.sf[j] * H(ti, tn, q)) * (ir * is * S.iht);
  double d_p = (H(pi, pn, q + 1) - H(pi, pn, q)) * (ir * is * S.ihp);
  return d_r + d_t + d_p;
}

// ----------------------------------------------------------------- extrapolate
template <typename R>
__global__ void k_extrapolate(long total, State<R> it, State<R> n, State<R> nm1, R *A0, R *A1, R *A2) {
  long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long stride = (long)gridDim.x * blockDim.x;
  for (; q < total; q += stride) {
#pragma unroll
    for (int f = 0; f < NF; ++f) it.f[f][q] = (R)(2.0 * (double)n.f[f][q] - (double)nm1.f[f][q]);
    A0[q] = (R)(1.5 * (double)n.f[F_U2R][q] - 0.5 * (double)nm1.f[F_U2R][q]);
    A1[q] = (R)(1.5 * (double)n.f[F_U2T][q] - 0.5 * (double)nm1.f[F_U2T][q]);
    A2[q] = (R)(1.5 * (double)n.f[F_U2P][q] - 0.5 * (double)nm1.f[F_U2P][q]);
  }
}

template <typename R>
__global__ void k_combine(long total, Modes<R> M, R *o0, R *o1, R *o2, R *o3) {
  long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long stride = (long)gridDim.x * blockDim.x;
  R *out[4] = {o0, o1, o2, o3};
  for (; q < total; q += stride) {
    for (int c = 0; c < 4; ++c) {
      double acc = 0.0;
      for (int m = 0; m < M.n; ++m) acc = acc + M.tau[m] * (double)M.F[m][c][q];
      out[c][q] = (R)acc;
    }
  }
}

// ----------------------------------------------------------------- residual T
template <typename R>
__global__ void k_resid_T(Shell S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LC, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  const R *a = it.f[F_T], *b = n.f[F_T];
  const double ir = S.irc[i], is = S.isc[j], ir2 = ir * ir;
  const double ihr = S.ihr, iht = S.iht, ihp = S.ihp;
  double X0 = H(a, b, q);
  double Xrp = H(a, b, q + L.SI), Xrm = H(a, b, q - L.SI);
  double Xtp = H(a, b, q + L.P), Xtm = H(a, b, q - L.P);
  double Xpp = H(a, b, q + 1), Xpm = H(a, b, q - 1);
  double Drr = (S.rf[i + 1] * S.rf[i + 1] * (Xrp - X0) - S.rf[i] * S.rf[i] * (X0 - Xrm)) * (ir2 * ihr * ihr);
  double Dtt = (S.sf[j + 1] * (Xtp - X0) - S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  double Dpp = (Xpp - 2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  double ar = ((double)ax.A[0][q] + (double)ax.A[0][q + L.SI]) * 0.5;
  double at = ((double)ax.A[1][q] + (double)ax.A[1][q + L.P]) * 0.5;
  double ap = ((double)ax.A[2][q] + (double)ax.A[2][q + 1]) * 0.5;
  double adv = ar * (Xrp - Xrm) * (0.5 * ihr) + at * (Xtp - Xtm) * (0.5 * ir * iht) +
               ap * (Xpp - Xpm) * (0.5 * ir * is * ihp);
  double f = ax.fT ? (double)ax.fT[q] : 0.0;
  double rate = S.kappa * (Drr + Dtt + Dpp) - adv + f;
  B[q] = (R)(S.dt * rate - ((double)a[q] - (double)b[q]));
}

// ----------------------------------------------------------------- residual u
template <typename R>
__device__ __forceinline__ double pres(const State<R> &it, const State<R> &n, int sys, long q) {
  if (sys == 1) return (double)n.f[F_P1][q];
  return (double)n.f[F_P2][q] + 0.5 * ((double)it.f[F_P1][q] - (double)n.f[F_P1][q]);
}

template <typename R>
__global__ void k_resid_ur(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LR, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *xi = it.f[F_U1R + o], *xn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const double ir = S.irf[i], is = S.isc[j], ir2 = ir * ir;
  const double ihr = S.ihr, iht = S.iht, ihp = S.ihp;
  const long SI = L.SI, P = L.P;
  double X0 = H(xi, xn, q);
  double Xrp = H(xi, xn, q + SI), Xrm = H(xi, xn, q - SI);
  double Xtp = H(xi, xn, q + P), Xtm = H(xi, xn, q - P);
  double Xpp = H(xi, xn, q + 1), Xpm = H(xi, xn, q - 1);
  double Drr = (S.rc[i] * S.rc[i] * (Xrp - X0) - S.rc[i - 1] * S.rc[i - 1] * (X0 - Xrm)) * (ir2 * ihr * ihr);
  double Dtt = (S.sf[j + 1] * (Xtp - X0) - S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  double Dpp = (Xpp - 2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  double extra = -2.0 * X0 * ir2 +
                 2.0 * ir2 * ir * (S.rf[i + 1] * S.rf[i + 1] * Xrp - S.rf[i - 1] * S.rf[i - 1] * Xrm) * (0.5 * ihr);
  double ar = (double)ax.A[0][q];
  double at = avg4(ax.A[1], q - SI, q - SI + P, q, q + P);
  double ap = avg4(ax.A[2], q - SI, q - SI + 1, q, q + 1);
  double bt = havg4(yi, yn, q - SI, q - SI + P, q, q + P);
  double bp = havg4(zi, zn, q - SI, q - SI + 1, q, q + 1);
  double adv = ar * (Xrp - Xrm) * (0.5 * ihr) + at * (Xtp - Xtm) * (0.5 * ir * iht) +
               ap * (Xpp - Xpm) * (0.5 * ir * is * ihp) - (at * bt + ap * bp) * ir;
  double gradP = (pres(it, n, sys, q) - pres(it, n, sys, q - SI)) * ihr;
  double Dc = divh(S, xi, xn, yi, yn, zi, zn, i, j, q);
  double Dm = divh(S, xi, xn, yi, yn, zi, zn, i - 1, j, q - SI);
  double gdiv = (Dc - Dm) * ihr;
  double buoy = S.PrRa * 0.5 * (H(it.f[F_T], n.f[F_T], q - SI) + H(it.f[F_T], n.f[F_T], q));
  double f = ax.fr ? (double)ax.fr[q] : 0.0;
  double rate = S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * S.i2chi + buoy + f;
  B[q] = (R)(S.dt * rate - ((double)xi[q] - (double)xn[q]));
}

template <typename R>
__global__ void k_resid_ut(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LT, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *xi = it.f[F_U1T + o], *xn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const double ir = S.irc[i], is = S.isf[j], c = S.cf[j], ir2 = ir * ir;
  const double ihr = S.ihr, iht = S.iht, ihp = S.ihp;
  const long SI = L.SI, P = L.P;
  double X0 = H(xi, xn, q);
  double Xrp = H(xi, xn, q + SI), Xrm = H(xi, xn, q - SI);
  double Xtp = H(xi, xn, q + P), Xtm = H(xi, xn, q - P);
  double Xpp = H(xi, xn, q + 1), Xpm = H(xi, xn, q - 1);
  double Drr = (S.rf[i + 1] * S.rf[i + 1] * (Xrp - X0) - S.rf[i] * S.rf[i] * (X0 - Xrm)) * (ir2 * ihr * ihr);
  double Dtt = (S.sc[j] * (Xtp - X0) - S.sc[j - 1] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  double Dpp = (Xpp - 2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  double W_j = 0.5 * (H(wi, wn, q) + H(wi, wn, q + SI));
  double W_jm = 0.5 * (H(wi, wn, q - P) + H(wi, wn, q - P + SI));
  double dW = (W_j - W_jm) * iht;
  double qj = (S.rf[i + 1] * S.rf[i + 1] * H(wi, wn, q + SI) - S.rf[i] * S.rf[i] * H(wi, wn, q)) * ihr;
  double qjm = (S.rf[i + 1] * S.rf[i + 1] * H(wi, wn, q + SI - P) - S.rf[i] * S.rf[i] * H(wi, wn, q - P)) * ihr;
  double drr2W = 0.5 * (qj + qjm);
  double extra = -X0 * ir2 * is * is +
                 2.0 * c * ir2 * is * is * (S.sf[j + 1] * Xtp - S.sf[j - 1] * Xtm) * (0.5 * iht) +
                 2.0 * ir2 * dW + 2.0 * c * ir2 * ir * is * drr2W;
  double ar = avg4(ax.A[0], q - P, q - P + SI, q, q + SI);
  double at = (double)ax.A[1][q];
  double ap = avg4(ax.A[2], q - P, q - P + 1, q, q + 1);
  double br = havg4(wi, wn, q - P, q - P + SI, q, q + SI);
  double bp = havg4(zi, zn, q - P, q - P + 1, q, q + 1);
  double adv = ar * (Xrp - Xrm) * (0.5 * ihr) + at * (Xtp - Xtm) * (0.5 * ir * iht) +
               ap * (Xpp - Xpm) * (0.5 * ir * is * ihp) + (at * br - ap * bp * c * is) * ir;
  double gradP = (pres(it, n, sys, q) - pres(it, n, sys, q - P)) * (ir * iht);
  double Dc = divh(S, wi, wn, xi, xn, zi, zn, i, j, q);
  double Dm = divh(S, wi, wn, xi, xn, zi, zn, i, j - 1, q - P);
  double gdiv = (Dc - Dm) * (ir * iht);
  double f = ax.ft ? (double)ax.ft[q] : 0.0;
  double rate = S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * S.i2chi + f;
  B[q] = (R)(S.dt * rate - ((double)xi[q] - (double)xn[q]));
}

template <typename R>
__global__ void k_resid_up(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LP, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *xi = it.f[F_U1P + o], *xn = n.f[F_U1P + o];
  const double ir = S.irc[i], is = S.isc[j], c = S.cc[j], ir2 = ir * ir;
  const double ihr = S.ihr, iht = S.iht, ihp = S.ihp;
  const long SI = L.SI, P = L.P;
  double X0 = H(xi, xn, q);
  double Xrp = H(xi, xn, q + SI), Xrm = H(xi, xn, q - SI);
  double Xtp = H(xi, xn, q + P), Xtm = H(xi, xn, q - P);
  double Xpp = H(xi, xn, q + 1), Xpm = H(xi, xn, q - 1);
  double Drr = (S.rf[i + 1] * S.rf[i + 1] * (Xrp - X0) - S.rf[i] * S.rf[i] * (X0 - Xrm)) * (ir2 * ihr * ihr);
  double Dtt = (S.sf[j + 1] * (Xtp - X0) - S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  double Dpp = (Xpp - 2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  double W_k = 0.5 * (H(wi, wn, q) + H(wi, wn, q + SI));
  double W_km = 0.5 * (H(wi, wn, q - 1) + H(wi, wn, q - 1 + SI));
  double Y_k = 0.5 * (H(yi, yn, q) + H(yi, yn, q + P));
  double Y_km = 0.5 * (H(yi, yn, q - 1) + H(yi, yn, q - 1 + P));
  double extra = -X0 * ir2 * is * is + 2.0 * ir2 * is * (W_k - W_km) * ihp +
                 2.0 * c * ir2 * is * is * (Y_k - Y_km) * ihp;
  double ar = avg4(ax.A[0], q - 1, q - 1 + SI, q, q + SI);
  double at = avg4(ax.A[1], q - 1, q - 1 + P, q, q + P);
  double ap = (double)ax.A[2][q];
  double br = havg4(wi, wn, q - 1, q - 1 + SI, q, q + SI);
  double bt = havg4(yi, yn, q - 1, q - 1 + P, q, q + P);
  double adv = ar * (Xrp - Xrm) * (0.5 * ihr) + at * (Xtp - Xtm) * (0.5 * ir * iht) +
               ap * (Xpp - Xpm) * (0.5 * ir * is * ihp) + (ap * br + ap * bt * c * is) * ir;
  double gradP = (pres(it, n, sys, q) - pres(it, n, sys, q - 1)) * (ir * is * ihp);
  double Dc = divh(S, wi, wn, yi, yn, xi, xn, i, j, q);
  double Dm = divh(S, wi, wn, yi, yn, xi, xn, i, j, q - 1);
  double gdiv = (Dc - Dm) * (ir * is * ihp);
  double f = ax.fp ? (double)ax.fp[q] : 0.0;
  double rate = S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * S.i2chi + f;
  B[q] = (R)(S.dt * rate - ((double)xi[q] - (double)xn[q]));
}

// ----------------------------------------------------------------- pressure
template <typename R>
__global__ void k_pressure(Shell S, int sys, State<R> it, State<R> n, double *norm, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  bool ok = decode_point(L, LC, patch_mask, p, i, j, k);
  double contrib = 0.0;
  if (ok) {
    long q = lidx(L, p, i, j, k);
    int o = (sys == 1) ? 0 : 4;
    double D = divh(S, it.f[F_U1R + o], n.f[F_U1R + o], it.f[F_U1T + o], n.f[F_U1T + o], it.f[F_U1P + o],
                    n.f[F_U1P + o], i, j, q);
    double pnew;
    R *dst;
    if (sys == 1) {
      pnew = (double)n.f[F_P1][q] - D * (2.0 * S.i2chi);
      dst = it.f[F_P1];
    } else {
      pnew = (double)n.f[F_P2][q] + ((double)it.f[F_P1][q] - (double)n.f[F_P1][q]) - D * (2.0 * S.i2chi);
      dst = it.f[F_P2];
    }
    double c = pnew - (double)dst[q];
    dst[q] = (R)pnew;
    bool ringcell = (j == 0 || j == L.Nt - 1 || k == 0 || k == L.Np - 1);
    if (!(S.step7 && ringcell)) {
      double r = S.rc[i];
      double w = r * r * S.sc[j] * S.hr * S.ht * S.hp;
      contrib = w * c * c;
    }
  }
  // warp reduction, one atomic per warp
  for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
  if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(&norm[sys == 1 ? 4 : 8], contrib);
}

// ----------------------------------------------------------------- packing
__device__ __forceinline__ void user_extent(const Layout &L, int loc, int &ni, int &nj, int &nk) {
  ni = L.Nr + (loc == LR ? 1 : 0);
  nj = L.Nt + (loc == LT ? 1 : 0);
  nk = L.Np + (loc == LP ? 1 : 0);
}

template <typename R>
__global__ void k_unpack(Layout L, int loc, const double *src, R *dst) {
  int ni, nj, nk;
  user_extent(L, loc, ni, nj, nk);
  long n = 2L * ni * nj * nk;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
    int k = (int)(u % nk);
    long t = u / nk;
    int j = (int)(t % nj);
    t /= nj;
    int i = (int)(t % ni);
    int p = (int)(t / ni);
    dst[lidx(L, p, i, j, k)] = (R)src[u];
  }
}

template <typename R>
__global__ void k_pack(Layout L, int loc, const R *src, double *dst) {
  int ni, nj, nk;
  user_extent(L, loc, ni, nj, nk);
  long n = 2L * ni * nj * nk;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
    int k = (int)(u % nk);
    long t = u / nk;
    int j = (int)(t % nj);
    t /= nj;
    int i = (int)(t % ni);
    int p = (int)(t / ni);
    dst[u] = (double)src[lidx(L, p, i, j, k)];
  }
}

dim3 point_grid(const Layout &L, int loc) {
  int ni = L.Nr - (loc == LR ? 1 : 0);
  int nj = L.Nt - (loc == LT ? 1 : 0);
  int nk = L.Np - (loc == LP ? 1 : 0);
  return dim3((nk + TPB - 1) / TPB, 2 * ni * nj);
}

int flat_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 152L * 16 ? b : 152L * 16);
}

}  // namespace

template <typename R>
void Launch<R>::extrapolate(const Layout &L, State<R> it, State<R> n, State<R> nm1, R *A[3], cudaStream_t st) {
  k_extrapolate<R><<<flat_blocks(L.total), 256, 0, st>>>(L.total, it, n, nm1, A[0], A[1], A[2]);
}

template <typename R>
void Launch<R>::combine_forcing(long total, Modes<R> modes, R *out[4], cudaStream_t st) {
  k_combine<R><<<flat_blocks(total), 256, 0, st>>>(total, modes, out[0], out[1], out[2], out[3]);
}

template <typename R>
void Launch<R>::resid_T(const Shell &S, State<R> it, State<R> n, StepAux<R> ax, R *B, int pm, cudaStream_t st) {
  k_resid_T<R><<<point_grid(S.L, LC), TPB, 0, st>>>(S, it, n, ax, B, pm);
}

template <typename R>
void Launch<R>::resid_u(const Shell &S, int sys, int comp, State<R> it, State<R> n, StepAux<R> ax, R *B, int pm,
                        cudaStream_t st) {
  if (comp == 0)
    k_resid_ur<R><<<point_grid(S.L, LR), TPB, 0, st>>>(S, sys, it, n, ax, B, pm);
  else if (comp == 1)
    k_resid_ut<R><<<point_grid(S.L, LT), TPB, 0, st>>>(S, sys, it, n, ax, B, pm);
  else
    k_resid_up<R><<<point_grid(S.L, LP), TPB, 0, st>>>(S, sys, it, n, ax, B, pm);
}

template <typename R>
void Launch<R>::pressure(const Shell &S, int sys, State<R> it, State<R> n, double *norm, int pm, cudaStream_t st) {
  k_pressure<R><<<point_grid(S.L, LC), TPB, 0, st>>>(S, sys, it, n, norm, pm);
}

template <typename R>
void Launch<R>::unpack(const Layout &L, int loc, const double *src, R *dst, cudaStream_t st) {
  long n = 2L * (L.Nr + 1) * (L.Nt + 1) * (L.Np + 1);
  k_unpack<R><<<flat_blocks(n), 256, 0, st>>>(L, loc, src, dst);
}

template <typename R>
void Launch<R>::pack(const Layout &L, int loc, const R *src, double *dst, cudaStream_t st) {
  long n = 2L * (L.Nr + 1) * (L.Nt + 1) * (L.Np + 1);
  k_pack<R><<<flat_blocks(n), 256, 0, st>>>(L, loc, src, dst);
}

template struct StepAux<double>;
template void Launch<double>::extrapolate(const Layout &, State<double>, State<double>, State<double>, double *[3],
                                          cudaStream_t);
template void Launch<double>::combine_forcing(long, Modes<double>, double *[4], cudaStream_t);
template void Launch<double>::resid_T(const Shell &, State<double>, State<double>, StepAux<double>, double *, int,
                                      cudaStream_t);
template void Launch<double>::resid_u(const Shell &, int, int, State<double>, State<double>, StepAux<double>,
                                      double *, int, cudaStream_t);
template void Launch<double>::pressure(const Shell &, int, State<double>, State<double>, double *, int,
                                       cudaStream_t);
template void Launch<double>::unpack(const Layout &, int, const double *, double *, cudaStream_t);
template void Launch<double>::pack(const Layout &, int, const double *, double *, cudaStream_t);

}  // namespace ys
