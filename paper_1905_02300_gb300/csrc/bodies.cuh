// Device bodies of the solver's kernels, shared by the single-shell kernels
// and the batched persistent kernels.  Each body takes its block coordinates
// (bx, by) explicitly instead of reading blockIdx, so one CTA of a batched
// launch can execute the work of any shell's block.
#pragma once
#include "kernels.cuh"

namespace ys {
namespace bd {


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

// Point decode for the residual grids: block row `by` enumerates (p, i, j)
// rows of the region, block column `bx` and the threads run along k.
__device__ __forceinline__ bool decode_point(const Layout &L, int loc, int patch_mask, int bx, int by, int &p,
                                             int &i, int &j, int &k) {
  int i0, i1, j0, j1, k0, k1;
  region(L, loc, i0, i1, j0, j1, k0, k1);
  int nj = j1 - j0, ni = i1 - i0;
  int row = by;
  j = j0 + row % nj;
  row /= nj;
  i = i0 + row % ni;
  p = row / ni;
  k = k0 + bx * blockDim.x + threadIdx.x;
  return k < k1 && ((patch_mask >> p) & 1);
}

// discrete divergence of the half-level velocity at cell (p, i, j, k)
template <typename V, typename R>
__device__ __forceinline__ V divh(const Shell &S, const R *ri, const R *rn, const R *ti, const R *tn, const R *pi,
                                  const R *pn, int i, int j, long q) {
  const Layout &L = S.L;
  const V ir = mt<V>(S, MT_IRC)[i], is = mt<V>(S, MT_ISC)[j];
  const V rfp = mt<V>(S, MT_RF)[i + 1], rf0 = mt<V>(S, MT_RF)[i];
  V d_r = (rfp * rfp * H<V>(ri, rn, q + L.SI) - rf0 * rf0 * H<V>(ri, rn, q)) * (ir * ir * cs<V>(S, CS_IHR));
  V d_t = (mt<V>(S, MT_SF)[j + 1] * H<V>(ti, tn, q + L.P) - mt<V>(S, MT_SF)[j] * H<V>(ti, tn, q)) * (ir * is * cs<V>(S, CS_IHT));
  V d_p = (H<V>(pi, pn, q + 1) - H<V>(pi, pn, q)) * (ir * is * cs<V>(S, CS_IHP));
  return d_r + d_t + d_p;
}


template <typename R>
__device__ __forceinline__ void body_resid_T(Shell S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LC, patch_mask, bx, by, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  const R *a = it.f[F_T], *b = n.f[F_T];
  const V ir = mt<V>(S, MT_IRC)[i], is = mt<V>(S, MT_ISC)[j], ir2 = ir * ir;
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V rfp = mt<V>(S, MT_RF)[i + 1], rf0 = mt<V>(S, MT_RF)[i];
  V X0 = H<V>(a, b, q);
  V Xrp = H<V>(a, b, q + L.SI), Xrm = H<V>(a, b, q - L.SI);
  V Xtp = H<V>(a, b, q + L.P), Xtm = H<V>(a, b, q - L.P);
  V Xpp = H<V>(a, b, q + 1), Xpm = H<V>(a, b, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = (mt<V>(S, MT_SF)[j + 1] * (Xtp - X0) - mt<V>(S, MT_SF)[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V ar = ((V)ax.A[0][q] + (V)ax.A[0][q + L.SI]) * (V)0.5;
  V at = ((V)ax.A[1][q] + (V)ax.A[1][q + L.P]) * (V)0.5;
  V ap = ((V)ax.A[2][q] + (V)ax.A[2][q + 1]) * (V)0.5;
  V adv = ar * (Xrp - Xrm) * ((V)0.5 * ihr) + at * (Xtp - Xtm) * ((V)0.5 * ir * iht) +
          ap * (Xpp - Xpm) * ((V)0.5 * ir * is * ihp);
  V f = ax.fT ? (V)ax.fT[q] : (V)0.0;
  V rate = cs<V>(S, CS_KAPPA) * (Drr + Dtt + Dpp) - adv + f;
  if (S.Tc_lap) rate += (V)(S.kappa * S.Tc_lap[i]) - ar * (V)S.Tc_dr[i];
  B[q] = (R)(cs<V>(S, CS_DT) * rate - ((V)a[q] - (V)b[q]));
}

// pressure entering the momentum rows: P_1 = p_1^n, P_2 = p_2^n + (p_1 - p_1^n)/2
template <typename R>
__device__ __forceinline__ double pres(const State<R> &it, const State<R> &n, int sys, long q) {
  if (sys == 1) return n.p[0][q];
  return n.p[1][q] + 0.5 * (it.p[0][q] - n.p[0][q]);
}


template <typename R>
__device__ __forceinline__ void body_resid_ur(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LR, patch_mask, bx, by, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *xi = it.f[F_U1R + o], *xn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const V ir = mt<V>(S, MT_IRF)[i], is = mt<V>(S, MT_ISC)[j], ir2 = ir * ir;
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V rc0 = mt<V>(S, MT_RC)[i], rcm = mt<V>(S, MT_RC)[i - 1], rfp = mt<V>(S, MT_RF)[i + 1], rfm = mt<V>(S, MT_RF)[i - 1];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rc0 * rc0 * (Xrp - X0) - rcm * rcm * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = (mt<V>(S, MT_SF)[j + 1] * (Xtp - X0) - mt<V>(S, MT_SF)[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
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
  V buoy = cs<V>(S, CS_PRRA) * (V)0.5 * (H<V>(it.f[F_T], n.f[F_T], q - SI) + H<V>(it.f[F_T], n.f[F_T], q));
  V f = ax.fr ? (V)ax.fr[q] : (V)0.0;
  V rate = cs<V>(S, CS_NU) * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * cs<V>(S, CS_I2CHI) + buoy + f;
  B[q] = (R)(cs<V>(S, CS_DT) * rate - ((V)xi[q] - (V)xn[q]));
}

template <typename R>
__device__ __forceinline__ void body_resid_ut(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LT, patch_mask, bx, by, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *xi = it.f[F_U1T + o], *xn = n.f[F_U1T + o];
  const R *zi = it.f[F_U1P + o], *zn = n.f[F_U1P + o];
  const V ir = mt<V>(S, MT_IRC)[i], is = mt<V>(S, MT_ISF)[j], c = mt<V>(S, MT_CF)[j], ir2 = ir * ir;
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V rfp = mt<V>(S, MT_RF)[i + 1], rf0 = mt<V>(S, MT_RF)[i];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = (mt<V>(S, MT_SC)[j] * (Xtp - X0) - mt<V>(S, MT_SC)[j - 1] * (X0 - Xtm)) * (ir2 * is * iht * iht);
  V Dpp = (Xpp - (V)2.0 * X0 + Xpm) * (ir2 * is * is * ihp * ihp);
  V W_j = (V)0.5 * (H<V>(wi, wn, q) + H<V>(wi, wn, q + SI));
  V W_jm = (V)0.5 * (H<V>(wi, wn, q - P) + H<V>(wi, wn, q - P + SI));
  V dW = (W_j - W_jm) * iht;
  V qj = (rfp * rfp * H<V>(wi, wn, q + SI) - rf0 * rf0 * H<V>(wi, wn, q)) * ihr;
  V qjm = (rfp * rfp * H<V>(wi, wn, q + SI - P) - rf0 * rf0 * H<V>(wi, wn, q - P)) * ihr;
  V drr2W = (V)0.5 * (qj + qjm);
  V extra = -X0 * ir2 * is * is +
            (V)2.0 * c * ir2 * is * is * (mt<V>(S, MT_SF)[j + 1] * Xtp - mt<V>(S, MT_SF)[j - 1] * Xtm) * ((V)0.5 * iht) +
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
  V rate = cs<V>(S, CS_NU) * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * cs<V>(S, CS_I2CHI) + f;
  B[q] = (R)(cs<V>(S, CS_DT) * rate - ((V)xi[q] - (V)xn[q]));
}

template <typename R>
__device__ __forceinline__ void body_resid_up(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LP, patch_mask, bx, by, p, i, j, k)) return;
  long q = lidx(L, p, i, j, k);
  int o = (sys == 1) ? 0 : 4;
  const R *wi = it.f[F_U1R + o], *wn = n.f[F_U1R + o];
  const R *yi = it.f[F_U1T + o], *yn = n.f[F_U1T + o];
  const R *xi = it.f[F_U1P + o], *xn = n.f[F_U1P + o];
  const V ir = mt<V>(S, MT_IRC)[i], is = mt<V>(S, MT_ISC)[j], c = mt<V>(S, MT_CC)[j], ir2 = ir * ir;
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V rfp = mt<V>(S, MT_RF)[i + 1], rf0 = mt<V>(S, MT_RF)[i];
  const long SI = L.SI, P = L.P;
  V X0 = H<V>(xi, xn, q);
  V Xrp = H<V>(xi, xn, q + SI), Xrm = H<V>(xi, xn, q - SI);
  V Xtp = H<V>(xi, xn, q + P), Xtm = H<V>(xi, xn, q - P);
  V Xpp = H<V>(xi, xn, q + 1), Xpm = H<V>(xi, xn, q - 1);
  V Drr = (rfp * rfp * (Xrp - X0) - rf0 * rf0 * (X0 - Xrm)) * (ir2 * ihr * ihr);
  V Dtt = (mt<V>(S, MT_SF)[j + 1] * (Xtp - X0) - mt<V>(S, MT_SF)[j] * (X0 - Xtm)) * (ir2 * is * iht * iht);
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
  V rate = cs<V>(S, CS_NU) * (Drr + Dtt + Dpp + extra) - adv - gradP + gdiv * cs<V>(S, CS_I2CHI) + f;
  B[q] = (R)(cs<V>(S, CS_DT) * rate - ((V)xi[q] - (V)xn[q]));
}

template <typename R>
__device__ __forceinline__ void body_pressure(Shell S, int sys, State<R> it, State<R> n, double *norm, int patch_mask, int bx, int by) {
  const Layout &L = S.L;
  int p, i, j, k;
  bool ok = decode_point(L, LC, patch_mask, bx, by, p, i, j, k);
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

// elements [q0, q1) of every field, threads striding by blockDim.x
template <typename R>
__device__ __forceinline__ void body_extrapolate(long q0, long q1, State<R> it, State<R> n, State<R> nm1, R *A0,
                                                 R *A1, R *A2) {
  using V = typename Cmp<R>::type;
  const int bulk[7] = {F_T, F_U1R, F_U1T, F_U1P, F_U2R, F_U2T, F_U2P};
  for (long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
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
__device__ __forceinline__ double bilin(const R *a, const Layout &L, int p, int i, int j0, int k0, double wj,
                                        double wk) {
  long q = lidx(L, p, i, j0, k0);
  return (1 - wj) * (1 - wk) * (double)a[q] + (1 - wj) * wk * (double)a[q + 1] + wj * (1 - wk) * (double)a[q + L.P] +
         wj * wk * (double)a[q + L.P + 1];
}


template <typename R>
__device__ __forceinline__ void body_exchange(Shell S, const XEntry *__restrict__ e, int n, int kind, State<R> s, int patch_mask, int bx, int by) {
  const Layout &L = S.L;
  int p = by;
  if (!((patch_mask >> p) & 1)) return;
  int d = 1 - p;
  int ni = (kind == XUR) ? L.Nr - 1 : L.Nr;
  int i0 = (kind == XUR) ? 1 : 0;
  long t = bx * (long)blockDim.x + threadIdx.x;
  if (t >= (long)n * ni) return;
  int ent = (int)(t % n);
  int i = i0 + (int)(t / n);
  const XEntry E = e[ent];
  long qt = lidx(L, p, i, E.tj, E.tk);
  if (kind == XT) {
    s.f[F_T][qt] = (R)bilin(s.f[F_T], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else if (kind == XUR) {
    s.f[F_U1R][qt] = (R)bilin(s.f[F_U1R], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
    s.f[F_U2R][qt] = (R)bilin(s.f[F_U2R], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else if (kind == XP) {
    s.p[0][qt] = bilin(s.p[0], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
    s.p[1][qt] = bilin(s.p[1], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else {
    int slot = (kind == XUT) ? F_U1T : F_U1P;
    for (int o = 0; o <= 4; o += 4) {
      double vt = bilin(s.f[F_U1T + o], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
      double vp = bilin(s.f[F_U1P + o], L, d, i, E.j0b, E.k0b, E.wjb, E.wkb);
      s.f[slot + o][qt] = (R)(E.ra * vt + E.rb * vp);
    }
  }
}

template <typename R>
__device__ __forceinline__ void body_walls(Shell S, State<R> s, int patch_mask, int bx, int by) {
  const Layout &L = S.L;
  int p = by;
  if (!((patch_mask >> p) & 1)) return;
  long t = bx * (long)blockDim.x + threadIdx.x;
  long plane = (long)(L.Nt + 2) * (L.Np + 2);
  if (t >= plane) return;
  int j = (int)(t / (L.Np + 2)) - 1;
  int k = (int)(t % (L.Np + 2)) - 1;
  const int Nr = L.Nr, Nt = L.Nt, Np = L.Np;
  long lo = lidx(L, p, -1, j, k), l0 = lidx(L, p, 0, j, k);
  long hi = lidx(L, p, Nr, j, k), h0 = lidx(L, p, Nr - 1, j, k);
  // u_r on the wall faces i = 0 and i = Nr, the whole plane
  s.f[F_U1R][l0] = (R)0.0;
  s.f[F_U2R][l0] = (R)0.0;
  s.f[F_U1R][hi] = (R)0.0;
  s.f[F_U2R][hi] = (R)0.0;
  if (j >= 0 && j < Nt && k >= 0 && k < Np) {
    s.f[F_T][lo] = (R)(2.0 * S.T_in - (double)s.f[F_T][l0]);
    s.f[F_T][hi] = (R)(2.0 * S.T_out - (double)s.f[F_T][h0]);
  }
  if (j >= 1 && j < Nt && k >= 0 && k < Np) {
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1T + o];
      u[lo] = (R)(-(double)u[l0]);
      u[hi] = (R)(-(double)u[h0]);
    }
  }
  if (j >= 0 && j < Nt && k >= 1 && k < Np) {
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1P + o];
      u[lo] = (R)(-(double)u[l0]);
      u[hi] = (R)(-(double)u[h0]);
    }
  }
}

// Advecting velocity (a_r, a_th, a_ph) at a point of location `loc`: own
// component as stored, others averaged from their nearest stored values.
template <typename R>
__device__ __forceinline__ void advecting(const Shell &S, const StepAux<R> &ax, int loc, long q, double &ar,
                                          double &at, double &ap) {
  const long SI = S.L.SI, P = S.L.P;
  const R *A0 = ax.A[0], *A1 = ax.A[1], *A2 = ax.A[2];
  switch (loc) {
    case LC:
      ar = ((double)A0[q] + (double)A0[q + SI]) * 0.5;
      at = ((double)A1[q] + (double)A1[q + P]) * 0.5;
      ap = ((double)A2[q] + (double)A2[q + 1]) * 0.5;
      break;
    case LR:
      ar = (double)A0[q];
      at = avg4<double>(A1, q - SI, q - SI + P, q, q + P);
      ap = avg4<double>(A2, q - SI, q - SI + 1, q, q + 1);
      break;
    case LT:
      ar = avg4<double>(A0, q - P, q - P + SI, q, q + SI);
      at = (double)A1[q];
      ap = avg4<double>(A2, q - P, q - P + 1, q, q + 1);
      break;
    default:
      ar = avg4<double>(A0, q - 1, q - 1 + SI, q, q + SI);
      at = avg4<double>(A1, q - 1, q - 1 + P, q, q + P);
      ap = (double)A2[q];
      break;
  }
}

// Coefficients (lo, di, up) of (I - dt/2 Ahat_dir) at point (i, j, k) of `loc`
// (divisions replaced by FP64 reciprocal metric tables).
template <typename V, typename R>
__device__ __forceinline__ void coef(const Shell &S, const StepAux<R> &ax, int loc, int dir, int i, int j, long q,
                                     V &lo, V &di, V &up) {
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V nu = (loc == LC) ? cs<V>(S, CS_KAPPA) : cs<V>(S, CS_NU);
  double ar_d, at_d, ap_d;
  advecting(S, ax, loc, q, ar_d, at_d, ap_d);
  const V ar = (V)ar_d, at = (V)at_d, ap = (V)ap_d;
  const V ir = (loc == LR) ? mt<V>(S, MT_IRF)[i] : mt<V>(S, MT_IRC)[i];
  const V is = (loc == LT) ? mt<V>(S, MT_ISF)[j] : mt<V>(S, MT_ISC)[j];
  const V ir2 = ir * ir;
  const V rc0 = mt<V>(S, MT_RC)[i], rcm = mt<V>(S, MT_RC)[i - 1], rf0 = mt<V>(S, MT_RF)[i], rfp = mt<V>(S, MT_RF)[i + 1], rfm = mt<V>(S, MT_RF)[i - 1];
  const V sc0 = mt<V>(S, MT_SC)[j], scm = mt<V>(S, MT_SC)[j - 1], sf0 = mt<V>(S, MT_SF)[j], sfp = mt<V>(S, MT_SF)[j + 1], sfm = mt<V>(S, MT_SF)[j - 1];
  V cm, c0, cp;
  if (dir == DR) {
    V cp_d, cm_d;
    if (loc == LR) {
      cp_d = rc0 * rc0 * (ir2 * ihr * ihr);
      cm_d = rcm * rcm * (ir2 * ihr * ihr);
    } else {
      cp_d = rfp * rfp * (ir2 * ihr * ihr);
      cm_d = rf0 * rf0 * (ir2 * ihr * ihr);
    }
    cm = nu * cm_d + ar * ((V)0.5 * ihr);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - ar * ((V)0.5 * ihr);
    if (loc == LR) {
      cm = cm - nu * rfm * rfm * (ir2 * ir * ihr);
      cp = cp + nu * rfp * rfp * (ir2 * ir * ihr);
      c0 = c0 - nu * (V)2.0 * ir2;
      const V k = cs<V>(S, CS_I2CHI), irm = mt<V>(S, MT_IRC)[i - 1], irc = mt<V>(S, MT_IRC)[i];
      cm = cm + k * rfm * rfm * (irm * irm * ihr * ihr);
      c0 = c0 - k * (rf0 * rf0 * (irc * irc * ihr * ihr) + rf0 * rf0 * (irm * irm * ihr * ihr));
      cp = cp + k * rfp * rfp * (irc * irc * ihr * ihr);
    }
  } else if (dir == DT) {
    V cp_d, cm_d;
    const V iR1sq = cs<V>(S, CS_IR1SQ);
    if (loc == LT) {
      cp_d = sc0 * (iR1sq * is * iht * iht);
      cm_d = scm * (iR1sq * is * iht * iht);
    } else {
      cp_d = sfp * (iR1sq * is * iht * iht);
      cm_d = sf0 * (iR1sq * is * iht * iht);
    }
    cm = nu * cm_d + at * ((V)0.5 * ir * iht);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - at * ((V)0.5 * ir * iht);
    if (loc == LT) {
      const V c = mt<V>(S, MT_CF)[j], s = sf0;
      const V qq = c * ir2 * is * is * iht;
      cm = cm - nu * qq * sfm;
      cp = cp + nu * qq * sfp;
      c0 = c0 - nu * ir2 * is * is;
      const V k = cs<V>(S, CS_I2CHI), isc0 = mt<V>(S, MT_ISC)[j], iscm = mt<V>(S, MT_ISC)[j - 1];
      cp = cp + k * sfp * (ir2 * isc0 * iht * iht);
      c0 = c0 - k * (s * (ir2 * isc0 * iht * iht) + s * (ir2 * iscm * iht * iht));
      cm = cm + k * sfm * (ir2 * iscm * iht * iht);
    }
  } else {
    const V cpm = cs<V>(S, CS_CPHI);
    cm = nu * cpm + ap * ((V)0.5 * ir * is * ihp);
    c0 = (V)-2.0 * nu * cpm;
    cp = nu * cpm - ap * ((V)0.5 * ir * is * ihp);
    if (loc == LP) {
      c0 = c0 - nu * ir2 * is * is;
      const V qq = cs<V>(S, CS_I2CHI) * ir2 * is * is * ihp * ihp;
      cm = cm + qq;
      c0 = c0 - (V)2.0 * qq;
      cp = cp + qq;
    }
  }
  lo = (V)-0.5 * cs<V>(S, CS_DT) * cm;
  di = (V)1.0 - (V)0.5 * cs<V>(S, CS_DT) * c0;
  up = (V)-0.5 * cs<V>(S, CS_DT) * cp;
}

// Line of a (loc, dir) sweep: thread (lane, row) -> patch p, first point
// (i, j, k), row range [m0, m1) and element stride along the line.  Lanes run
// along phi for r- and theta-sweeps (coalesced) and along theta for
// phi-sweeps.
struct Line {
  int p, i, j, k, m0, m1;
  long step;
  bool valid;
};

__device__ __forceinline__ Line decode_line(const Layout &L, int loc, int dir, int lane, int row) {
  const int i0 = (loc == LR) ? 1 : 0, i1 = L.Nr;
  const int j0 = (loc == LT) ? 1 : 0, j1 = L.Nt;
  const int k0 = (loc == LP) ? 1 : 0, k1 = L.Np;
  Line ln;
  if (dir == DR) {
    int nj = j1 - j0;
    ln.k = k0 + lane;
    ln.j = j0 + row % nj;
    ln.p = row / nj;
    ln.i = i0;
    ln.valid = ln.k < k1;
    ln.m0 = i0;
    ln.m1 = i1;
    ln.step = L.SI;
  } else if (dir == DT) {
    int ni = i1 - i0;
    ln.k = k0 + lane;
    ln.i = i0 + row % ni;
    ln.p = row / ni;
    ln.j = j0;
    ln.valid = ln.k < k1;
    ln.m0 = j0;
    ln.m1 = j1;
    ln.step = L.P;
  } else {
    int ni = i1 - i0;
    ln.j = j0 + lane;
    ln.i = i0 + row % ni;
    ln.p = row / ni;
    ln.k = k0;
    ln.valid = ln.j < j1;
    ln.m0 = k0;
    ln.m1 = k1;
    ln.step = 1;
  }
  return ln;
}


template <typename R>
__device__ __forceinline__ void body_factorize(Shell S, int loc, int dir, StepAux<R> ax, R *__restrict__ Lo,
                                               R *__restrict__ Iv, R *__restrict__ Cp, int patch_mask, int bx,
                                               int by) {
  using V = typename Cmp<R>::type;
  constexpr int U = 4;   // rows whose coefficients are formed before the recurrence consumes them
  const Layout &L = S.L;
  const Line ln = decode_line(L, loc, dir, bx * blockDim.x + threadIdx.x, by);
  if (!ln.valid || !((patch_mask >> ln.p) & 1)) return;
  const bool reflect = (dir == DR) && (loc != LR);
  const long step = ln.step;
  V cprev = (V)0.0;
  long q = lidx(L, ln.p, ln.i, ln.j, ln.k);
  for (int m = ln.m0; m < ln.m1; m += U, q += U * step) {
    V lo[U], di[U], up[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int mm = m + u;
      if (mm < ln.m1) {
        int ii = (dir == DR) ? mm : ln.i, jj = (dir == DT) ? mm : ln.j;
        coef<V>(S, ax, loc, dir, ii, jj, q + u * step, lo[u], di[u], up[u]);
        if (mm == ln.m0) {
          if (reflect) di[u] -= lo[u];
          lo[u] = (V)0.0;
        }
        if (mm == ln.m1 - 1) {
          if (reflect) di[u] -= up[u];
          up[u] = (V)0.0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (m + u < ln.m1) {
        V inv = (V)1.0 / (di[u] - lo[u] * cprev);
        V c = up[u] * inv;
        Lo[q + u * step] = (R)lo[u];
        Iv[q + u * step] = (R)inv;
        Cp[q + u * step] = (R)c;
        cprev = c;
      }
    }
  }
}

// Thomas solve with a stored factorisation: forward d'_m = (b_m - lo_m d'_{m-1})
// / pivot_m into the scratch W, back x_m = d'_m - c'_m x_{m+1}.  Rows are
// handled in register chunks of U: the loads of a chunk are independent of
// the recurrence and of every store (separate arrays), so they are in flight
// together.  Non-final factors write x to B (the next factor's right-hand
// side); the final factor of an unknown adds x to the iterate and accumulates
// the FP64 midpoint-rule norm of the increment (Sec. 5.1).
template <typename R>
__device__ __forceinline__ void body_solve(Shell S, int loc, int dir, int final, const R *__restrict__ Lo,
                                           const R *__restrict__ Iv, const R *__restrict__ Cp, R *__restrict__ B,
                                           R *__restrict__ W, R *__restrict__ dst, double *norm, int slot,
                                           int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  constexpr int U = 8;
  const Layout &L = S.L;
  const Line ln = decode_line(L, loc, dir, bx * blockDim.x + threadIdx.x, by);
  double contrib = 0.0;
  if (ln.valid && ((patch_mask >> ln.p) & 1)) {
    const long step = ln.step;
    const long q0 = lidx(L, ln.p, ln.i, ln.j, ln.k);
    const int n = ln.m1 - ln.m0;
    // forward elimination: B -> W
    V d = (V)0.0;
    for (int m = 0; m < n; m += U) {
      V b[U], lo[U], iv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        long qq = q0 + (long)(m + u) * step;
        if (m + u < n) {
          b[u] = (V)B[qq];
          lo[u] = (V)Lo[qq];
          iv[u] = (V)Iv[qq];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (m + u < n) {
          d = (b[u] - lo[u] * d) * iv[u];
          W[q0 + (long)(m + u) * step] = (R)d;
        }
      }
    }
    // back substitution: W -> B or the iterate, last row first
    V x = d;
    for (int m = n - 1; m >= 0; m -= U) {
      V w[U], c[U], o[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        long qq = q0 + (long)(m - u) * step;
        if (m - u >= 0) {
          w[u] = (V)W[qq];
          c[u] = (V)Cp[qq];
          o[u] = final ? (V)dst[qq] : (V)0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int mm = m - u;
        if (mm >= 0) {
          long qq = q0 + (long)mm * step;
          if (mm < n - 1) x = w[u] - c[u] * x;
          if (final) {
            dst[qq] = (R)(o[u] + x);
            int row = ln.m0 + mm;
            int ii = (dir == DR) ? row : ln.i, jj = (dir == DT) ? row : ln.j;
            double r = (loc == LR) ? S.rf[ii] : S.rc[ii];
            double s = (loc == LT) ? S.sf[jj] : S.sc[jj];
            contrib += r * r * s * S.hr * S.ht * S.hp * (double)x * (double)x;
          } else {
            B[qq] = (R)x;
          }
        }
      }
    }
  }
  if (final) {
    for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
    if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(&norm[slot], contrib);
  }
}

// Line solve along phi (the contiguous index) through shared memory.  Each
// warp owns 32 adjacent lines (consecutive theta rows at one radius) and
// walks them in chunks of 32 rows: the chunk's right-hand side and factors
// are loaded as a [32 lines][32 rows] tile with coalesced row reads, the 32
// recurrences run from shared memory (rows padded to 33: no bank conflicts),
// and results leave the same way.  Same arithmetic as body_solve.
constexpr int kPhiWarps = 4;   // warps (tiles of 32 lines) per CTA
template <typename R>
constexpr int phi_smem_bytes() {
  return kPhiWarps * 3 * 32 * 33 * (int)sizeof(R);
}

template <typename R>
__device__ __forceinline__ void body_solve_phi(Shell S, int loc, int final, const R *__restrict__ Lo,
                                               const R *__restrict__ Iv, const R *__restrict__ Cp,
                                               R *__restrict__ B, R *__restrict__ W, R *__restrict__ dst,
                                               double *norm, int slot, int patch_mask, int bx, R *smem) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = (loc == LR) ? 1 : 0, j0 = (loc == LT) ? 1 : 0, k0 = (loc == LP) ? 1 : 0;
  const int ni = L.Nr - i0, nj = L.Nt - j0, nk = L.Np - k0;
  const int jt = (nj + 31) / 32;
  const long tile = (long)bx * kPhiWarps + warp;
  double contrib = 0.0;
  if (tile < 2L * ni * jt) {
    const int jb = (int)(tile % jt) * 32;
    const long rest = tile / jt;
    const int i = i0 + (int)(rest % ni), p = (int)(rest / ni);
    if ((patch_mask >> p) & 1) {
      R *t0 = smem + warp * 3 * 32 * 33, *t1 = t0 + 32 * 33, *t2 = t1 + 32 * 33;
      const bool lv = jb + lane < nj;
      const long rowbase = lidx(L, p, i, j0 + jb, k0);   // line jb, first row
      const long lstride = L.P;                          // between adjacent lines
      const int nch = (nk + 31) / 32;
      V d = (V)0.0;
      for (int c = 0; c < nch; ++c) {
        const int kc = c * 32;
        const bool kv = kc + lane < nk;
        for (int r0 = 0; r0 < 32; r0 += 8) {   // 8 rows of loads in flight, then to shared memory
          R a0[8], a1[8], a2[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int rr = r0 + u;
            if (jb + rr < nj && kv) {
              long q = rowbase + rr * lstride + kc + lane;
              a0[u] = B[q];
              a1[u] = Lo[q];
              a2[u] = Iv[q];
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int rr = r0 + u;
            if (jb + rr < nj && kv) {
              t0[rr * 33 + lane] = a0[u];
              t1[rr * 33 + lane] = a1[u];
              t2[rr * 33 + lane] = a2[u];
            }
          }
        }
        __syncwarp();
        if (lv) {
          const int kmax = (nk - kc < 32) ? nk - kc : 32;
          for (int u = 0; u < kmax; ++u) {
            d = ((V)t0[lane * 33 + u] - (V)t1[lane * 33 + u] * d) * (V)t2[lane * 33 + u];
            t0[lane * 33 + u] = (R)d;
          }
        }
        __syncwarp();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr)
          if (jb + rr < nj && kv) W[rowbase + rr * lstride + kc + lane] = t0[rr * 33 + lane];
        __syncwarp();
      }
      double wline = 0.0;
      if (final && lv) {
        int jj = j0 + jb + lane;
        double r = (loc == LR) ? S.rf[i] : S.rc[i];
        double sn = (loc == LT) ? S.sf[jj] : S.sc[jj];
        wline = r * r * sn * S.hr * S.ht * S.hp;
      }
      V x = d;
      for (int c = nch - 1; c >= 0; --c) {
        const int kc = c * 32;
        const bool kv = kc + lane < nk;
        for (int r0 = 0; r0 < 32; r0 += 8) {
          R a0[8], a1[8], a2[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int rr = r0 + u;
            if (jb + rr < nj && kv) {
              long q = rowbase + rr * lstride + kc + lane;
              a0[u] = W[q];
              a1[u] = Cp[q];
              if (final) a2[u] = dst[q];
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int rr = r0 + u;
            if (jb + rr < nj && kv) {
              t0[rr * 33 + lane] = a0[u];
              t1[rr * 33 + lane] = a1[u];
              if (final) t2[rr * 33 + lane] = a2[u];
            }
          }
        }
        __syncwarp();
        if (lv) {
          const int kmax = (nk - kc < 32) ? nk - kc : 32;
          for (int u = kmax - 1; u >= 0; --u) {
            if (kc + u < nk - 1) x = (V)t0[lane * 33 + u] - (V)t1[lane * 33 + u] * x;
            if (final) {
              t2[lane * 33 + u] = (R)((V)t2[lane * 33 + u] + x);
              contrib += wline * (double)x * (double)x;
            } else {
              t0[lane * 33 + u] = (R)x;
            }
          }
        }
        __syncwarp();
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) {
          if (jb + rr < nj && kv) {
            long q = rowbase + rr * lstride + kc + lane;
            if (final)
              dst[q] = t2[rr * 33 + lane];
            else
              B[q] = t0[rr * 33 + lane];
          }
        }
        __syncwarp();
      }
    }
  }
  if (final) {
    for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
    if (lane == 0 && contrib != 0.0) atomicAdd(&norm[slot], contrib);
  }
}

// CTAs of kPhiWarps warps needed by body_solve_phi for one shell
inline int phi_ctas(const Layout &L, int loc) {
  int ni = L.Nr - (loc == LR ? 1 : 0), nj = L.Nt - (loc == LT ? 1 : 0);
  long tiles = 2L * ni * ((nj + 31) / 32);
  return (int)((tiles + kPhiWarps - 1) / kPhiWarps);
}

// Per-step factorisation of the phi factor through shared memory (same warp
// tiles as body_solve_phi): coefficients of a [32 lines][32 rows] tile are
// formed with lanes along phi (coalesced reads of the advecting velocity),
// the 32 line recurrences run from shared memory, and the factors leave with
// coalesced row writes.  Same arithmetic as body_factorize.
template <typename R>
__device__ __forceinline__ void body_factorize_phi(Shell S, int loc, StepAux<R> ax, R *__restrict__ Lo,
                                                   R *__restrict__ Iv, R *__restrict__ Cp, int patch_mask, int bx,
                                                   R *smem) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = (loc == LR) ? 1 : 0, j0 = (loc == LT) ? 1 : 0, k0 = (loc == LP) ? 1 : 0;
  const int ni = L.Nr - i0, nj = L.Nt - j0, nk = L.Np - k0;
  const int jt = (nj + 31) / 32;
  const long tile = (long)bx * kPhiWarps + warp;
  if (tile >= 2L * ni * jt) return;
  const int jb = (int)(tile % jt) * 32;
  const long rest = tile / jt;
  const int i = i0 + (int)(rest % ni), p = (int)(rest / ni);
  if (!((patch_mask >> p) & 1)) return;
  R *t0 = smem + warp * 3 * 32 * 33, *t1 = t0 + 32 * 33, *t2 = t1 + 32 * 33;
  const long rowbase = lidx(L, p, i, j0 + jb, k0);
  const long lstride = L.P;
  const int nch = (nk + 31) / 32;
  V cprev = (V)0.0;
  for (int c = 0; c < nch; ++c) {
    const int kc = c * 32;
    const int kk = kc + lane;
    if (kk < nk) {
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        if (jb + rr < nj) {
          V lo, di, up;
          coef<V>(S, ax, loc, DP, i, j0 + jb + rr, rowbase + rr * lstride + kk, lo, di, up);
          if (kk == 0) lo = (V)0.0;
          if (kk == nk - 1) up = (V)0.0;
          t0[rr * 33 + lane] = (R)lo;
          t1[rr * 33 + lane] = (R)di;
          t2[rr * 33 + lane] = (R)up;
        }
      }
    }
    __syncwarp();
    if (jb + lane < nj) {
      const int kmax = (nk - kc < 32) ? nk - kc : 32;
      for (int u = 0; u < kmax; ++u) {
        V lo = (V)t0[lane * 33 + u];
        V inv = (V)1.0 / ((V)t1[lane * 33 + u] - lo * cprev);
        V cc = (V)t2[lane * 33 + u] * inv;
        t1[lane * 33 + u] = (R)inv;
        t2[lane * 33 + u] = (R)cc;
        cprev = cc;
      }
    }
    __syncwarp();
    if (kk < nk) {
#pragma unroll 8
      for (int rr = 0; rr < 32; ++rr) {
        if (jb + rr < nj) {
          long q = rowbase + rr * lstride + kk;
          Lo[q] = t0[rr * 33 + lane];
          Iv[q] = t1[rr * 33 + lane];
          Cp[q] = t2[rr * 33 + lane];
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace bd
}  // namespace ys
