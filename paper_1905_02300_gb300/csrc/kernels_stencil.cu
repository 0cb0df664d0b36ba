// Explicit MAC-stencil kernels: extrapolation, residuals of the defect
// correction (-F = dt Rate(psi^{1/2}) - (psi - psi^n), Sec. 4 Eq. er), pressure
// updates (Eq. nst_Mass1 and Eq. ac2), and host-layout packing.
//
// Every rate is the discrete operator of Sec. 3.2 / Sec. 3.3 on the MAC grid:
// conservative 3-point diffusion with the metric at half points, centred
// first derivatives (2-point across a half-cell offset, 2h otherwise),
// off-location values as arithmetic means of the 2 or 4 nearest stored
// values, metric factors evaluated exactly at the row's point (FP64 tables of
// r, sin(theta), cos(theta) and their reciprocals).  Bulk arithmetic runs in
// the storage type (FP64, or FP32 in the mixed form); pressures and the
// divergence that updates them are FP64 in both forms.
#include "kernels.cuh"

namespace ys {

namespace {

constexpr int TPB = 128;

template <typename V, typename R>
__device__ __forceinline__ V H(const R *a, const R *b, long q) {
  return (V)0.5 * ((V)a[q] + (V)b[q]);
}

template <typename V, typename R>
__device__ __forceinline__ V avg4(const R *a, long q1, long q2, long q3, long q4) {
  return (((V)a[q1] + (V)a[q2]) + (V)a[q3] + (V)a[q4]) * (V)0.25;
}

// half-level average of 4 points of a pair of arrays
template <typename V, typename R>
__device__ __forceinline__ V havg4(const R *a, const R *b, long q1, long q2, long q3, long q4) {
  return ((H<V>(a, b, q1) + H<V>(a, b, q2)) + H<V>(a, b, q3) + H<V>(a, b, q4)) * (V)0.25;
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
template <typename V, typename R>
__device__ __forceinline__ V divh(const Shell &S, const R *ri, const R *rn, const R *ti, const R *tn, const R *pi,
                                  const R *pn, int i, int j, long q) {
  const Layout &L = S.L;
  const V ir = (V)S.irc[i], is = (V)S.isc[j];
  const V rfp = (V)S.rf[i + 1], rf0 = (V)S.rf[i];
  V d_r = (rfp * rfp * H<V>(ri, rn, q + L.SI) - rf0 * rf0 * H<V>(ri, rn, q)) * (ir * ir * (V)S.ihr);
  V d_t = ((V)S.sf[j + 1] * H<V>(ti, tn, q + L.P) - (V)S.sf[j] * H<V>(ti, tn, q)) * (ir * is * (V)S.iht);
  V d_p = (H<V>(pi, pn, q + 1) - H<V>(pi, pn, q)) * (ir * is * (V)S.ihp);
  return d_r + d_t + d_p;
}

// ----------------------------------------------------------------- extrapolate
template <typename R>
__global__ void k_extrapolate(long total, State<R> it, State<R> n, State<R> nm1, R *A0, R *A1, R *A2) {
  using V = typename Cmp<R>::type;
  long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long stride = (long)gridDim.x * blockDim.x;
  const int bulk[7] = {F_T, F_U1R, F_U1T, F_U1P, F_U2R, F_U2T, F_U2P};
  for (; q < total; q += stride) {
#pragma unroll
    for (int b = 0; b < 7; ++b) {
      int f = bulk[b];
      it.f[f][q] = (R)((V)2.0 * (V)n.f[f][q] - (V)nm1.f[f][q]);
    }
    it.p[0][q] = 2.0 * n.p[0][q] - nm1.p[0][q];
    it.p[1][q] = 2.0 * n.p[1][q] - nm1.p[1][q];
    A0[q] = (R)((V)1.5 * (V)n.f[F_U2R][q] - (V)0.5 * (V)nm1.f[F_U2R][q]);
    A1[q] = (R)((V)1.5 * (V)n.f[F_U2T][q] - (V)0.5 * (V)nm1.f[F_U2T][q]);
    A2[q] = (R)((V)1.5 * (V)n.f[F_U2P][q] - (V)0.5 * (V)nm1.f[F_U2P][q]);
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
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LC, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  const R *a = it.f[F_T], *b = n.f[F_T];
  const V ir = (V)S.irc[i], is = (V)S.isc[j], ir2 = ir * ir;
  const V ihr = (V)S.ihr, iht = (V)S.iht, ihp = (V)S.ihp;
  const V rfp = (V)S.rf[i + 1], rf0 = (V)S.rf[i];
  V X0 = H<V>(a, b, q);
  V Xrp = H<V>(a, b, q + L.SI), Xrm = H<V>(a, b, q - L.SI);
  V Xtp = H<V>(a, b, q + L.P), Xtm = H<V>(a, b, q - L.P);
  V Xpp = H<V>(a, b, q + 1), Xpm = H<V>(a, b, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = ((V)S.sf[j + 1] * (Xtp - X0) - (V)S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V ar = ((V)ax.A[0][q] + (V)ax.A[0][q + L.SI]) * (V)0.5;
  V at = ((V)ax.A[1][q] + (V)ax.A[1][q + L.P]) * (V)0.5;
  V ap = ((V)ax.A[2][q] + (V)ax.A[2][q + 1]) * (V)0.5;
  V adv = ar * (Xrp - Xrm) * ((V)0.5 * ihr) + at * (Xtp - Xtm) * ((V)0.5 * ir * iht) +
          ap * (Xpp - Xpm) * ((V)0.5 * ir * is * ihp);
  V f = ax.fT ? (V)ax.fT[q] : (V)0.0;
  V rate = (V)S.kappa * (Drr + Dtt + Dpp) - adv + f;
  if (S.Tc_lap) rate += (V)(S.kappa * S.Tc_lap[i]) - ar * (V)S.Tc_dr[i];
  B[q] = (R)((V)S.dt * rate - ((V)a[q] - (V)b[q]));
}

// ----------------------------------------------------------------- residual u
// pressure entering the momentum rows: P_1 = p_1^n, P_2 = p_2^n + (p_1 - p_1^n)/2
template <typename R>
__device__ __forceinline__ double pres(const State<R> &it, const State<R> &n, int sys, long q) {
  if (sys == 1) return n.p[0][q];
  return n.p[1][q] + 0.5 * (it.p[0][q] - n.p[0][q]);
}

template <typename R>
__global__ void k_resid_ur(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LR, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *xi = it.f[F_U1R + o], *xn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const V ir = (V)S.irf[i], is = (V)S.isc[j], ir2 = ir * ir;
  const V ihr = (V)S.ihr, iht = (V)S.iht, ihp = (V)S.ihp;
  const V rc0 = (V)S.rc[i], rcm = (V)S.rc[i - 1], rfp = (V)S.rf[i + 1], rfm = (V)S.rf[i - 1];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rc0 * rc0 * (Xrp - X0) - rcm * rcm * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = ((V)S.sf[j + 1] * (Xtp - X0) - (V)S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V extra = (V)-2.0 * X0 * ir2 + (V)2.0 * ir2 * ir * (rfp * rfp * Xrp - rfm * rfm * Xrm) * ((V)0.5 * ihr);
  V ar = (V)ax.A[0][q];
  V at = avg4<V>(ax.A[1], q - SI, q - SI + P, q, q + P);
  V ap = avg4<V>(ax.A[2], q - SI, q - SI + 1, q, q + 1);
  V bt = havg4<V>(yi, yn, q - SI, q - SI + P, q, q + P);
  V bp = havg4<V>(zi, zn, q - SI, q - SI + 1, q, q + 1);
  V adv = ar * (Xrp - Xrm) * ((V)0.5 * ihr) + at * (Xtp - Xtm) * ((V)0.5 * ir * iht) +
          ap * (Xpp - Xpm) * ((V)0.5 * ir * is * ihp) - (at * bt + ap * bp) * ir;
  V gradP = (V)((pres(it, n, sys, q) - pres(it, n, sys, q - SI)) * S.ihr);
  V Dc = divh<V>(S, xi, xn, yi, yn, zi, zn, i, j, q);
  V Dm = divh<V>(S, xi, xn, yi, yn, zi, zn, i - 1, j, q - SI);
  V gdiv = (Dc - Dm) * ihr;
  V buoy = (V)S.PrRa * (V)0.5 * (H<V>(it.f[F_T], n.f[F_T], q - SI) + H<V>(it.f[F_T], n.f[F_T], q));
  V f = ax.fr ? (V)ax.fr[q] : (V)0.0;
  V rate = (V)S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * (V)S.i2chi + buoy + f;
  B[q] = (R)((V)S.dt * rate - ((V)xi[q] - (V)xn[q]));
}

template <typename R>
__global__ void k_resid_ut(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LT, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *xi = it.f[F_U1T + o], *xn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const V ir = (V)S.irc[i], is = (V)S.isf[j], c = (V)S.cf[j], ir2 = ir * ir;
  const V ihr = (V)S.ihr, iht = (V)S.iht, ihp = (V)S.ihp;
  const V rfp = (V)S.rf[i + 1], rf0 = (V)S.rf[i];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = ((V)S.sc[j] * (Xtp - X0) - (V)S.sc[j - 1] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V W_j = (V)0.5 * (H<V>(wi, wn, q) + H<V>(wi, wn, q + SI));
  V W_jm = (V)0.5 * (H<V>(wi, wn, q - P) + H<V>(wi, wn, q - P + SI));
  V dW = (W_j - W_jm) * iht;
  V qj = (rfp * rfp * H<V>(wi, wn, q + SI) - rf0 * rf0 * H<V>(wi, wn, q)) * ihr;
  V qjm = (rfp * rfp * H<V>(wi, wn, q + SI - P) - rf0 * rf0 * H<V>(wi, wn, q - P)) * ihr;
  V drr2W = (V)0.5 * (qj + qjm);
  V extra = -X0 * ir2 * is * is +
            (V)2.0 * c * ir2 * is * is * ((V)S.sf[j + 1] * Xtp - (V)S.sf[j - 1] * Xtm) * ((V)0.5 * iht) +
            (V)2.0 * ir2 * dW + (V)2.0 * c * ir2 * ir * is * drr2W;
  V ar = avg4<V>(ax.A[0], q - P, q - P + SI, q, q + SI);
  V at = (V)ax.A[1][q];
  V ap = avg4<V>(ax.A[2], q - P, q - P + 1, q, q + 1);
  V br = havg4<V>(wi, wn, q - P, q - P + SI, q, q + SI);
  V bp = havg4<V>(zi, zn, q - P, q - P + 1, q, q + 1);
  V adv = ar * (Xrp - Xrm) * ((V)0.5 * ihr) + at * (Xtp - Xtm) * ((V)0.5 * ir * iht) +
          ap * (Xpp - Xpm) * ((V)0.5 * ir * is * ihp) + (at * br - ap * bp * c * is) * ir;
  V gradP = (V)((pres(it, n, sys, q) - pres(it, n, sys, q - P)) * (S.irc[i] * S.iht));
  V Dc = divh<V>(S, wi, wn, xi, xn, zi, zn, i, j, q);
  V Dm = divh<V>(S, wi, wn, xi, xn, zi, zn, i, j - 1, q - P);
  V gdiv = (Dc - Dm) * (ir * iht);
  V f = ax.ft ? (V)ax.ft[q] : (V)0.0;
  V rate = (V)S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * (V)S.i2chi + f;
  B[q] = (R)((V)S.dt * rate - ((V)xi[q] - (V)xn[q]));
}

template <typename R>
__global__ void k_resid_up(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LP, patch_mask, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *xi = it.f[F_U1P + o], *xn = n.f[F_U1P + o];
  const V ir = (V)S.irc[i], is = (V)S.isc[j], c = (V)S.cc[j], ir2 = ir * ir;
  const V ihr = (V)S.ihr, iht = (V)S.iht, ihp = (V)S.ihp;
  const V rfp = (V)S.rf[i + 1], rf0 = (V)S.rf[i];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = ((V)S.sf[j + 1] * (Xtp - X0) - (V)S.sf[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V W_k = (V)0.5 * (H<V>(wi, wn, q) + H<V>(wi, wn, q + SI));
  V W_km = (V)0.5 * (H<V>(wi, wn, q - 1) + H<V>(wi, wn, q - 1 + SI));
  V Y_k = (V)0.5 * (H<V>(yi, yn, q) + H<V>(yi, yn, q + P));
  V Y_km = (V)0.5 * (H<V>(yi, yn, q - 1) + H<V>(yi, yn, q - 1 + P));
  V extra = -X0 * ir2 * is * is + (V)2.0 * ir2 * is * (W_k - W_km) * ihp +
            (V)2.0 * c * ir2 * is * is * (Y_k - Y_km) * ihp;
  V ar = avg4<V>(ax.A[0], q - 1, q - 1 + SI, q, q + SI);
  V at = avg4<V>(ax.A[1], q - 1, q - 1 + P, q, q + P);
  V ap = (V)ax.A[2][q];
  V br = havg4<V>(wi, wn, q - 1, q - 1 + SI, q, q + SI);
  V bt = havg4<V>(yi, yn, q - 1, q - 1 + P, q, q + P);
  V adv = ar * (Xrp - Xrm) * ((V)0.5 * ihr) + at * (Xtp - Xtm) * ((V)0.5 * ir * iht) +
          ap * (Xpp - Xpm) * ((V)0.5 * ir * is * ihp) + (ap * br + ap * bt * c * is) * ir;
  V gradP = (V)((pres(it, n, sys, q) - pres(it, n, sys, q - 1)) * (S.irc[i] * S.isc[j] * S.ihp));
  V Dc = divh<V>(S, wi, wn, yi, yn, xi, xn, i, j, q);
  V Dm = divh<V>(S, wi, wn, yi, yn, xi, xn, i, j, q - 1);
  V gdiv = (Dc - Dm) * (ir * is * ihp);
  V f = ax.fp ? (V)ax.fp[q] : (V)0.0;
  V rate = (V)S.nu * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * (V)S.i2chi + f;
  B[q] = (R)((V)S.dt * rate - ((V)xi[q] - (V)xn[q]));
}

// ----------------------------------------------------------------- pressure
// FP64 divergence and FP64 pressure accumulation in both forms.
template <typename R>
__global__ void k_pressure(Shell S, int sys, State<R> it, State<R> n, double *norm, int patch_mask) {
  const Layout &L = S.L;
  int p, i, j, k;
  bool ok = decode_point(L, LC, patch_mask, p, i, j, k);
  double contrib = 0.0;
  if (ok) {
    long q = lidx(L, p, i, j, k);
    int o = (sys == 1) ? 0 : 4;
    double D = divh<double>(S, it.f[F_U1R + o], n.f[F_U1R + o], it.f[F_U1T + o], n.f[F_U1T + o],
                            it.f[F_U1P + o], n.f[F_U1P + o], i, j, q);
    double pnew;
    double *dst;
    if (sys == 1) {
      pnew = n.p[0][q] - D * (2.0 * S.i2chi);
      dst = it.p[0];
    } else {
      pnew = n.p[1][q] + (it.p[0][q] - n.p[0][q]) - D * (2.0 * S.i2chi);
      dst = it.p[1];
    }
    double c = pnew - dst[q];
    dst[q] = pnew;
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
__global__ void k_unpack(Layout L, int loc, const double *src, R *dst, const double *bg) {
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
    double v = src[u];
    if (bg) v -= bg[i];
    dst[lidx(L, p, i, j, k)] = (R)v;
  }
}

template <typename R>
__global__ void k_pack(Layout L, int loc, const R *src, double *dst, const double *bg) {
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
    double v = (double)src[lidx(L, p, i, j, k)];
    if (bg) v += bg[i];
    dst[u] = v;
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

long user_max(const Layout &L) { return 2L * (L.Nr + 1) * (L.Nt + 1) * (L.Np + 1); }

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
void Launch<R>::unpack(const Layout &L, int loc, const double *src, R *dst, const double *bg, cudaStream_t st) {
  k_unpack<R><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, loc, src, dst, bg);
}

template <typename R>
void Launch<R>::pack(const Layout &L, int loc, const R *src, double *dst, const double *bg, cudaStream_t st) {
  k_pack<R><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, loc, src, dst, bg);
}

void unpack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st) {
  k_unpack<double><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, LC, src, dst, bg);
}

void pack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st) {
  k_pack<double><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, LC, src, dst, bg);
}

#define YS_INST_STENCIL(R)                                                                                         \
  template void Launch<R>::extrapolate(const Layout &, State<R>, State<R>, State<R>, R *[3], cudaStream_t);       \
  template void Launch<R>::combine_forcing(long, Modes<R>, R *[4], cudaStream_t);                                  \
  template void Launch<R>::resid_T(const Shell &, State<R>, State<R>, StepAux<R>, R *, int, cudaStream_t);        \
  template void Launch<R>::resid_u(const Shell &, int, int, State<R>, State<R>, StepAux<R>, R *, int,             \
                                   cudaStream_t);                                                                  \
  template void Launch<R>::pressure(const Shell &, int, State<R>, State<R>, double *, int, cudaStream_t);         \
  template void Launch<R>::unpack(const Layout &, int, const double *, R *, const double *, cudaStream_t);        \
  template void Launch<R>::pack(const Layout &, int, const R *, double *, const double *, cudaStream_t);
YS_INST_STENCIL(double)
YS_INST_STENCIL(float)

}  // namespace ys
