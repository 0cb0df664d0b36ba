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

// Double-float arithmetic: a value carried as the unevaluated sum hi + lo of
// two FP32 numbers (about 48 significant bits), built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the FMA form of
// Dekker's TwoProduct (Dekker 1971), each result renormalised by FastTwoSum.
// On this GPU FP64 instructions (conversions included) issue at 1/64 of the
// FP32 rate, so FP64-accurate sums of FP32 data are cheaper this way.  The
// explicit _rn intrinsics keep the compiler from contracting the error terms.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = two_sum(x.hi, y.hi);
  return ff_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ FF ff_sub(FF x, FF y) { return ff_add(x, FF{-y.hi, -y.lo}); }

__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ff_fast(p, e);
}

__device__ __forceinline__ double ff_double(FF x) { return (double)x.hi + (double)x.lo; }

// metric table entry / shell constant as a double-float pair
__device__ __forceinline__ FF ff_mt(const Shell &S, int t, int i) { return {S.ftab[t][i], S.ltab[t][i]}; }
__device__ __forceinline__ FF ff_cs(const Shell &S, int c) { return {S.fcs[c], S.lcs[c]}; }

// exact half-level average 0.5 (a + b) of two FP32 values
__device__ __forceinline__ FF ff_H(const float *a, const float *b, long q) {
  const FF s = two_sum(a[q], b[q]);
  return {0.5f * s.hi, 0.5f * s.lo};
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

// velocity component c (0 r, 1 theta, 2 phi) of system sys, chosen by selects
// (an index computed at run time would move the State structs to local memory)
template <typename R>
__device__ __forceinline__ R *velf(const State<R> &s, int sys, int c) {
  if (c == 0) return sys == 1 ? s.f[F_U1R] : s.f[F_U2R];
  if (c == 1) return sys == 1 ? s.f[F_U1T] : s.f[F_U2T];
  return sys == 1 ? s.f[F_U1P] : s.f[F_U2P];
}

// Discrete divergence of the half-level FP32 velocity at cell (p, i, j, k)
// (Sec. 3.3: conservative face differences with the metric at the faces), in
// double-float arithmetic: FP64-accurate terms at FP32 instruction cost.
__device__ __forceinline__ FF divh_ff(const Shell &S, const float *ri, const float *rn, const float *ti,
                                      const float *tn, const float *pi, const float *pn, int i, int j, long q) {
  const Layout &L = S.L;
  const FF ir = ff_mt(S, MT_IRC, i), is = ff_mt(S, MT_ISC, j);
  const FF rfp = ff_mt(S, MT_RF, i + 1), rf0 = ff_mt(S, MT_RF, i);
  FF d_r = ff_sub(ff_mul(ff_mul(rfp, rfp), ff_H(ri, rn, q + L.SI)), ff_mul(ff_mul(rf0, rf0), ff_H(ri, rn, q)));
  d_r = ff_mul(d_r, ff_mul(ff_mul(ir, ir), ff_mt(S, MT_IHC, i)));
  const FF irs = ff_mul(ir, is);
  FF d_t = ff_sub(ff_mul(ff_mt(S, MT_SF, j + 1), ff_H(ti, tn, q + L.P)), ff_mul(ff_mt(S, MT_SF, j), ff_H(ti, tn, q)));
  d_t = ff_mul(d_t, ff_mul(irs, ff_cs(S, CS_IHT)));
  FF d_p = ff_sub(ff_H(pi, pn, q + 1), ff_H(pi, pn, q));
  d_p = ff_mul(d_p, ff_mul(irs, ff_cs(S, CS_IHP)));
  return ff_add(ff_add(d_r, d_t), d_p);
}


// sum S = a + b of the two time levels at q (twice the half-level value)
template <typename V, typename R>
__device__ __forceinline__ V Sm(const R *a, const R *b, long q) {
  return (V)a[q] + (V)b[q];
}

// Residuals -F = dt Rate(psi^{1/2}) - (psi - psi^n) of the defect correction
// (Sec. 4, Eq. er) on the MAC grid (Sec. 3.2, 3.3).  Each is the discrete
// operator written as a linear form in the two-level sums S of the stencil
// values, with the per-row coefficient records of RowTable (all metric
// factors, spacings, dt and the physical constants folded in), plus the
// products of the extrapolated advecting velocity with differences of S.
// The diffusion parts keep the differenced form (S_+ - S_0) - (S_0 - S_-)
// of the conservative three-point operator.

// Lane vectors: a residual thread computes NV consecutive points along phi.
// NV = 1 is one point per thread (any k); NV > 1 (FP32 storage, NV = 4)
// starts at a k that is a multiple of NV, so that every row's group is one
// 16-byte vector (rows start 32-byte aligned: k = 0 sits 8 elements into a
// row whose pitch is a multiple of 8), and masks the lanes outside the
// region.  Lanes outside the region still load: a group never reaches more
// than NV + 3 elements past the last point of a row, which stays inside the
// row's padding, the next row's leading pad, or the patch box's tail slack.
//
// kFlat (the batched launches): bx is a flat block index over the shell's
// groups, rows one after another (ceil(Np / NV) groups a row), so that short
// rows do not leave most of a CTA idle; by is unused.
template <int NV, bool kFlat = false>
__device__ __forceinline__ int decode_group(const Layout &L, int loc, int patch_mask, int bx, int by, int &p, int &i,
                                            int &j, int &k) {
  int i0, i1, j0, j1, k0, k1;
  region(L, loc, i0, i1, j0, j1, k0, k1);
  int nj = j1 - j0, ni = i1 - i0;
  int row = by;
  int grp = bx * blockDim.x + threadIdx.x;
  if constexpr (kFlat) {
    const int gpr = (L.Np + NV - 1) / NV;
    row = grp / gpr;
    grp -= row * gpr;
    if (row >= 2 * ni * nj) return 0;
  }
  j = j0 + row % nj;
  row /= nj;
  i = i0 + row % ni;
  p = row / ni;
  if (!((patch_mask >> p) & 1)) return 0;
  if constexpr (NV == 1) {
    k = k0 + grp;
    return k < k1 ? 1 : 0;
  } else {
    k = NV * grp;
    int m = 0;
#pragma unroll
    for (int l = 0; l < NV; ++l)
      if (k + l >= k0 && k + l < k1) m |= 1 << l;
    return m;
  }
}

// o[l] = p[l]: one scalar (NV = 1) or 16-byte vector loads
template <int NV, typename R, typename V>
__device__ __forceinline__ void vld(const R *__restrict__ p, V (&o)[NV]) {
  if constexpr (NV == 1) {
    o[0] = (V)p[0];
  } else if constexpr (sizeof(R) == 4 && NV == 2) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    o[0] = (V)t.x;
    o[1] = (V)t.y;
  } else if constexpr (sizeof(R) == 4) {
    static_assert(NV % 4 == 0, "FP32 lane vectors are float2 or whole float4");
#pragma unroll
    for (int v = 0; v < NV / 4; ++v) {
      const float4 t = *reinterpret_cast<const float4 *>(p + 4 * v);
      o[4 * v] = (V)t.x;
      o[4 * v + 1] = (V)t.y;
      o[4 * v + 2] = (V)t.z;
      o[4 * v + 3] = (V)t.w;
    }
  } else {
    static_assert(NV % 2 == 0, "FP64 lane vectors are whole double2");
#pragma unroll
    for (int v = 0; v < NV / 2; ++v) {
      const double2 t = *reinterpret_cast<const double2 *>(p + 2 * v);
      o[2 * v] = (V)t.x;
      o[2 * v + 1] = (V)t.y;
    }
  }
}

// o[l] = a[q + l] + b[q + l]: the two-level sums S of the stencil
template <int NV, typename R, typename V>
__device__ __forceinline__ void vsm(const R *__restrict__ a, const R *__restrict__ b, long q, V (&o)[NV]) {
  V x[NV], y[NV];
  vld<NV>(a + q, x);
  vld<NV>(b + q, y);
#pragma unroll
  for (int l = 0; l < NV; ++l) o[l] = x[l] + y[l];
}

// values one position up (o[l] = value at l + 1) from the group c and the
// value e at position NV
template <int NV, typename V>
__device__ __forceinline__ void vup(const V (&c)[NV], V e, V (&o)[NV]) {
#pragma unroll
  for (int l = 0; l + 1 < NV; ++l) o[l] = c[l + 1];
  o[NV - 1] = e;
}

// values one position down (o[l] = value at l - 1) from the group c and the
// value e at position -1
template <int NV, typename V>
__device__ __forceinline__ void vdn(const V (&c)[NV], V e, V (&o)[NV]) {
#pragma unroll
  for (int l = NV - 1; l > 0; --l) o[l] = c[l - 1];
  o[0] = e;
}

// o = ((a + b) + c) + d: a 4-point sum of the advecting velocity, in the
// order the tables of StepAux::As use
template <int NV, typename V>
__device__ __forceinline__ void vsum4(const V (&a)[NV], const V (&b)[NV], const V (&c)[NV], const V (&d)[NV],
                                      V (&o)[NV]) {
#pragma unroll
  for (int l = 0; l < NV; ++l) o[l] = ((a[l] + b[l]) + c[l]) + d[l];
}

// store the lanes set in `lanes` (one vector store when all are)
template <int NV, typename R, typename V>
__device__ __forceinline__ void vst(R *__restrict__ p, const V (&v)[NV], int lanes) {
  if constexpr (NV == 1) {
    p[0] = (R)v[0];
  } else {
    static_assert(sizeof(R) == 4 && (NV == 2 || NV == 4), "vector stores are FP32 float2 or float4");
    if (lanes == (1 << NV) - 1) {
      if constexpr (NV == 2)
        *reinterpret_cast<float2 *>(p) = make_float2((float)v[0], (float)v[1]);
      else
        *reinterpret_cast<float4 *>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    } else {
#pragma unroll
      for (int l = 0; l < NV; ++l)
        if ((lanes >> l) & 1) p[l] = (R)v[l];
    }
  }
}

// kTab (the single-shell launches): the sums of the advecting velocity come
// from the per-step tables StepAux::As; otherwise (batched shells) the body
// forms them.  Both add the same values in the same order.

// temperature at cell centres: kappa Laplacian, advection, forcing, and in
// the deviation form the conductive-profile source
template <typename R, bool kTab = false, bool kSum = false>
__device__ __forceinline__ void body_resid_T(Shell S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by,
                                             const R *ST = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LC, patch_mask, bx, by, p, i, j, k)) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_T, i, j);
  const R *a = it.f[F_T], *b = n.f[F_T];
  // two-level sums: precomputed (kSum) or added here
  auto sT = [&](long qq) -> V {
    if constexpr (kSum) return (V)ST[qq];
    else return Sm<V>(a, b, qq);
  };
  const V S0 = sT(q);
  const V Srp = sT(q + SI), Srm = sT(q - SI);
  const V Stp = sT(q + P), Stm = sT(q - P);
  const V Spp = sT(q + 1), Spm = sT(q - 1);
  const V diff = c[T_RP] * (Srp - S0) - c[T_RM] * (S0 - Srm) + c[T_TP] * (Stp - S0) - c[T_TM] * (S0 - Stm) +
                 c[T_PP] * (Spp - (V)2.0 * S0 + Spm);
  const V sAr = kTab ? (V)ax.As[LC][DR][q] : (V)ax.A[0][q] + (V)ax.A[0][q + SI];
  const V sAt = kTab ? (V)ax.As[LC][DT][q] : (V)ax.A[1][q] + (V)ax.A[1][q + P];
  const V sAp = kTab ? (V)ax.As[LC][DP][q] : (V)ax.A[2][q] + (V)ax.A[2][q + 1];
  const V adv = c[T_AR] * sAr * (Srp - Srm) + c[T_AT] * sAt * (Stp - Stm) + c[T_AP] * sAp * (Spp - Spm);
  V out = diff - adv;
  if (ax.fT) out += cs<V>(S, CS_DT) * (V)ax.fT[q];
  if (S.Tc_lap) out += c[T_G0] - sAr * c[T_G1];
  B[q] = (R)(out - ((V)a[q] - (V)b[q]));
}

// pressure entering the momentum rows: P_1 = p_1^n, P_2 = p_2^n + (p_1 - p_1^n)/2
template <typename R>
__device__ __forceinline__ double pres(const State<R> &it, const State<R> &n, int sys, long q) {
  if (sys == 1) return n.p[0][q];
  return n.p[1][q] + 0.5 * (it.p[0][q] - n.p[0][q]);
}

// u_r at r-faces: nu (vector Laplacian), -advection (with the curvature
// terms), -grad P, grad(div)/(2 chi), buoyancy, forcing.
// kSum (the single-shell FP64 launches): the two-level sums S = psi + psi^n
// of the system's three velocity components and of T are read from
// Sv[0..3] (LevelSums), fields formed by k_sum_levels with the same addition,
// instead of being added here at every stencil point (17 FP64 additions and
// 17 loads fewer a point), and the momentum pressure from Sv[4].
template <typename R, bool kTab = false, bool kSum = false>
__device__ __forceinline__ void body_resid_ur(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by,
                                               const R *const *Sv = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LR, patch_mask, bx, by, p, i, j, k)) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UR, i, j);
  const R *xi = velf(it, sys, 0), *xn = velf(n, sys, 0);
  const R *yi = velf(it, sys, 1), *yn = velf(n, sys, 1);
  const R *zi = velf(it, sys, 2), *zn = velf(n, sys, 2);
  auto sx = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[0][qq];
    else return Sm<V>(xi, xn, qq);
  };
  auto sy = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[1][qq];
    else return Sm<V>(yi, yn, qq);
  };
  auto sz = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[2][qq];
    else return Sm<V>(zi, zn, qq);
  };
  const V S0 = sx(q);
  const V Srp = sx(q + SI), Srm = sx(q - SI);
  const V Stp = sx(q + P), Stm = sx(q - P);
  const V Spp = sx(q + 1), Spm = sx(q - 1);
  // u_theta and u_phi around the face: the two cells sharing it
  const V y1 = sy(q + P), y0 = sy(q), ym1 = sy(q - SI + P), ym0 = sy(q - SI);
  const V z1 = sz(q + 1), z0 = sz(q), zm1 = sz(q - SI + 1), zm0 = sz(q - SI);
  const R *A1 = ax.A[1], *A2 = ax.A[2];
  const V ar = (V)ax.A[0][q];
  const V sAt = kTab ? (V)ax.As[LR][DT][q] : ((V)A1[q - SI] + (V)A1[q - SI + P]) + (V)A1[q] + (V)A1[q + P];
  const V sAp = kTab ? (V)ax.As[LR][DP][q] : ((V)A2[q - SI] + (V)A2[q - SI + 1]) + (V)A2[q] + (V)A2[q + 1];
  // every term multiply-added into one accumulator (diffusion, own-component
  // couplings, grad-div couplings, -advection, curvature, -grad P, buoyancy)
  V out = c[UR_RP] * (Srp - S0);
  out -= c[UR_RM] * (S0 - Srm);
  out += c[UR_TP] * (Stp - S0);
  out -= c[UR_TM] * (S0 - Stm);
  out += c[UR_PP] * (Spp - (V)2.0 * S0 + Spm);
  out += c[UR_O1] * Srp;
  out += c[UR_O0] * S0;
  out += c[UR_OM] * Srm;
  out += c[UR_GT1] * y1;
  out += c[UR_GT0] * y0;
  out += c[UR_GTM1] * ym1;
  out += c[UR_GTM0] * ym0;
  out += c[UR_GP1] * (z1 - z0);
  out += c[UR_GPM1] * (zm1 - zm0);
  out -= (c[UR_AR] * ar) * (Srp - Srm);
  // advection along theta / phi and the curvature term of the same advecting component
  out += sAt * (c[UR_CV] * (((ym0 + ym1) + y0) + y1) - c[UR_AT] * (Stp - Stm));
  out += sAp * (c[UR_CV] * (((zm0 + zm1) + z0) + z1) - c[UR_AP] * (Spp - Spm));
  if constexpr (kSum)
    out -= c[UR_GPR] * (V)((double)Sv[4][q] - (double)Sv[4][q - SI]);
  else
    out -= c[UR_GPR] * (V)(pres(it, n, sys, q) - pres(it, n, sys, q - SI));
  if constexpr (kSum)
    out += c[UR_BY] * ((V)Sv[3][q - SI] + (V)Sv[3][q]);
  else
    out += c[UR_BY] * (Sm<V>(it.f[F_T], n.f[F_T], q - SI) + Sm<V>(it.f[F_T], n.f[F_T], q));
  if (ax.fr) out += cs<V>(S, CS_DT) * (V)ax.fr[q];
  B[q] = (R)(out - ((V)xi[q] - (V)xn[q]));
}

// u_theta at theta-faces
template <typename R, bool kTab = false, bool kSum = false>
__device__ __forceinline__ void body_resid_ut(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by,
                                               const R *const *Sv = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LT, patch_mask, bx, by, p, i, j, k)) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UT, i, j);
  const R *wi = velf(it, sys, 0), *wn = velf(n, sys, 0);
  const R *xi = velf(it, sys, 1), *xn = velf(n, sys, 1);
  const R *zi = velf(it, sys, 2), *zn = velf(n, sys, 2);
  auto sw = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[0][qq];
    else return Sm<V>(wi, wn, qq);
  };
  auto sx = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[1][qq];
    else return Sm<V>(xi, xn, qq);
  };
  auto sz = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[2][qq];
    else return Sm<V>(zi, zn, qq);
  };
  const V S0 = sx(q);
  const V Srp = sx(q + SI), Srm = sx(q - SI);
  const V Stp = sx(q + P), Stm = sx(q - P);
  const V Spp = sx(q + 1), Spm = sx(q - 1);
  // u_r and u_phi around the face: the two cells sharing it
  const V w1 = sw(q + SI), w0 = sw(q), wm1 = sw(q + SI - P), wm0 = sw(q - P);
  const V z1 = sz(q + 1), z0 = sz(q), zm1 = sz(q - P + 1), zm0 = sz(q - P);
  const R *A0 = ax.A[0], *A2 = ax.A[2];
  const V sAr = kTab ? (V)ax.As[LT][DR][q] : ((V)A0[q - P] + (V)A0[q - P + SI]) + (V)A0[q] + (V)A0[q + SI];
  const V at = (V)ax.A[1][q];
  const V sAp = kTab ? (V)ax.As[LT][DP][q] : ((V)A2[q - P] + (V)A2[q - P + 1]) + (V)A2[q] + (V)A2[q + 1];
  // every term multiply-added into one accumulator
  V out = c[UT_RP] * (Srp - S0);
  out -= c[UT_RM] * (S0 - Srm);
  out += c[UT_TP] * (Stp - S0);
  out -= c[UT_TM] * (S0 - Stm);
  out += c[UT_PP] * (Spp - (V)2.0 * S0 + Spm);
  out += c[UT_OTP] * Stp;
  out += c[UT_O0] * S0;
  out += c[UT_OTM] * Stm;
  out += c[UT_W1] * w1;
  out += c[UT_W0] * w0;
  out += c[UT_WM1] * wm1;
  out += c[UT_WM0] * wm0;
  out += c[UT_GP1] * (z1 - z0);
  out += c[UT_GPM1] * (zm1 - zm0);
  out -= (c[UT_AR] * sAr) * (Srp - Srm);
  // advection along theta / phi and the curvature term of the same advecting component
  out -= at * (c[UT_AT] * (Stp - Stm) + c[UT_CW] * (((wm0 + wm1) + w0) + w1));
  out += sAp * (c[UT_CP] * (((zm0 + zm1) + z0) + z1) - c[UT_AP] * (Spp - Spm));
  if constexpr (kSum)
    out -= c[UT_GPR] * (V)((double)Sv[4][q] - (double)Sv[4][q - P]);
  else
    out -= c[UT_GPR] * (V)(pres(it, n, sys, q) - pres(it, n, sys, q - P));
  if (ax.ft) out += cs<V>(S, CS_DT) * (V)ax.ft[q];
  B[q] = (R)(out - ((V)xi[q] - (V)xn[q]));
}

// u_phi at phi-faces
template <typename R, bool kTab = false, bool kSum = false>
__device__ __forceinline__ void body_resid_up(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, int bx, int by,
                                               const R *const *Sv = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  if (!decode_point(L, LP, patch_mask, bx, by, p, i, j, k)) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UP, i, j);
  const R *wi = velf(it, sys, 0), *wn = velf(n, sys, 0);
  const R *yi = velf(it, sys, 1), *yn = velf(n, sys, 1);
  const R *xi = velf(it, sys, 2), *xn = velf(n, sys, 2);
  auto sw = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[0][qq];
    else return Sm<V>(wi, wn, qq);
  };
  auto sy = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[1][qq];
    else return Sm<V>(yi, yn, qq);
  };
  auto sx = [&](long qq) -> V {
    if constexpr (kSum) return (V)Sv[2][qq];
    else return Sm<V>(xi, xn, qq);
  };
  const V S0 = sx(q);
  const V Srp = sx(q + SI), Srm = sx(q - SI);
  const V Stp = sx(q + P), Stm = sx(q - P);
  const V Spp = sx(q + 1), Spm = sx(q - 1);
  // u_r and u_theta around the face: the two cells sharing it
  const V w1 = sw(q + SI), w0 = sw(q), wm1 = sw(q - 1 + SI), wm0 = sw(q - 1);
  const V y1 = sy(q + P), y0 = sy(q), ym1 = sy(q - 1 + P), ym0 = sy(q - 1);
  const R *A0 = ax.A[0], *A1 = ax.A[1];
  const V sAr = kTab ? (V)ax.As[LP][DR][q] : ((V)A0[q - 1] + (V)A0[q - 1 + SI]) + (V)A0[q] + (V)A0[q + SI];
  const V sAt = kTab ? (V)ax.As[LP][DT][q] : ((V)A1[q - 1] + (V)A1[q - 1 + P]) + (V)A1[q] + (V)A1[q + P];
  const V ap = (V)ax.A[2][q];
  // every term multiply-added into one accumulator
  V out = c[UP_RP] * (Srp - S0);
  out -= c[UP_RM] * (S0 - Srm);
  out += c[UP_TP] * (Stp - S0);
  out -= c[UP_TM] * (S0 - Stm);
  out += c[UP_PP] * (Spp - (V)2.0 * S0 + Spm);
  out += c[UP_E0] * S0;
  out += c[UP_W1] * w1;
  out += c[UP_W0] * w0;
  out += c[UP_WM1] * wm1;
  out += c[UP_WM0] * wm0;
  out += c[UP_Y1] * y1;
  out += c[UP_Y0] * y0;
  out += c[UP_YM1] * ym1;
  out += c[UP_YM0] * ym0;
  out -= (c[UP_AR] * sAr) * (Srp - Srm);
  out -= (c[UP_AT] * sAt) * (Stp - Stm);
  // advection along phi and the curvature terms, all with the advecting a_phi
  out -= ap * (c[UP_AP] * (Spp - Spm) + c[UP_CW] * (((wm0 + wm1) + w0) + w1) +
               c[UP_CY] * (((ym0 + ym1) + y0) + y1));
  if constexpr (kSum)
    out -= c[UP_GPR] * (V)((double)Sv[4][q] - (double)Sv[4][q - 1]);
  else
    out -= c[UP_GPR] * (V)(pres(it, n, sys, q) - pres(it, n, sys, q - 1));
  if (ax.fp) out += cs<V>(S, CS_DT) * (V)ax.fp[q];
  B[q] = (R)(out - ((V)xi[q] - (V)xn[q]));
}

// The same residuals with NV consecutive points along phi per thread (FP32
// storage): identical arithmetic per point, the stencil values gathered with
// vector loads of the aligned group plus one scalar at each end where a
// stencil reaches past it.  kTab (the single-shell launches): the sums of the
// advecting velocity come from the per-step tables StepAux::As; otherwise
// (the batched launches) they are formed here, in the tables' order.

// temperature (body_resid_T)
template <typename R, int NV, bool kTab = true, bool kFlat = false>
__device__ __forceinline__ void body_resid_T_vec(Shell S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask,
                                             int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  const int lanes = decode_group<NV, kFlat>(L, LC, patch_mask, bx, by, p, i, j, k);
  if (!lanes) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_T, i, j);
  const R *a = it.f[F_T], *b = n.f[F_T];
  V ta[NV], tb[NV], S0[NV], Srp[NV], Srm[NV], Stp[NV], Stm[NV], Spp[NV], Spm[NV];
  vld<NV>(a + q, ta);
  vld<NV>(b + q, tb);
#pragma unroll
  for (int l = 0; l < NV; ++l) S0[l] = ta[l] + tb[l];
  vsm<NV>(a, b, q + SI, Srp);
  vsm<NV>(a, b, q - SI, Srm);
  vsm<NV>(a, b, q + P, Stp);
  vsm<NV>(a, b, q - P, Stm);
  vup<NV>(S0, Sm<V>(a, b, q + NV), Spp);
  vdn<NV>(S0, Sm<V>(a, b, q - 1), Spm);
  V sAr[NV], sAt[NV], sAp[NV], f[NV];
  if constexpr (kTab) {
    vld<NV>(ax.As[LC][DR] + q, sAr);
    vld<NV>(ax.As[LC][DT] + q, sAt);
    vld<NV>(ax.As[LC][DP] + q, sAp);
  } else {
    V a[NV], b[NV];
    vld<NV>(ax.A[0] + q, a);
    vld<NV>(ax.A[0] + q + SI, b);
#pragma unroll
    for (int l = 0; l < NV; ++l) sAr[l] = a[l] + b[l];
    vld<NV>(ax.A[1] + q, a);
    vld<NV>(ax.A[1] + q + P, b);
#pragma unroll
    for (int l = 0; l < NV; ++l) sAt[l] = a[l] + b[l];
    vld<NV>(ax.A[2] + q, a);
    vup<NV>(a, (V)ax.A[2][q + NV], b);
#pragma unroll
    for (int l = 0; l < NV; ++l) sAp[l] = a[l] + b[l];
  }
  if (ax.fT) vld<NV>(ax.fT + q, f);
  V o[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) {
    const V diff = c[T_RP] * (Srp[l] - S0[l]) - c[T_RM] * (S0[l] - Srm[l]) + c[T_TP] * (Stp[l] - S0[l]) -
                   c[T_TM] * (S0[l] - Stm[l]) + c[T_PP] * (Spp[l] - (V)2.0 * S0[l] + Spm[l]);
    const V adv = c[T_AR] * sAr[l] * (Srp[l] - Srm[l]) + c[T_AT] * sAt[l] * (Stp[l] - Stm[l]) +
                  c[T_AP] * sAp[l] * (Spp[l] - Spm[l]);
    V out = diff - adv;
    if (ax.fT) out += cs<V>(S, CS_DT) * f[l];
    if (S.Tc_lap) out += c[T_G0] - sAr[l] * c[T_G1];
    o[l] = out - (ta[l] - tb[l]);
  }
  vst<NV>(B + q, o, lanes);
}

// the same for the NV points of a group
template <int NV, typename R>
__device__ __forceinline__ void vpres(const State<R> &it, const State<R> &n, int sys, long q, double (&o)[NV]) {
  if (sys == 1) {
    vld<NV>(n.p[0] + q, o);
    return;
  }
  double a[NV], b[NV], c[NV];
  vld<NV>(n.p[1] + q, a);
  vld<NV>(it.p[0] + q, b);
  vld<NV>(n.p[0] + q, c);
#pragma unroll
  for (int l = 0; l < NV; ++l) o[l] = a[l] + 0.5 * (b[l] - c[l]);
}

// u_r (body_resid_ur)
template <typename R, int NV, bool kTab = true, bool kFlat = false>
__device__ __forceinline__ void body_resid_ur_vec(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B,
                                              int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  const int lanes = decode_group<NV, kFlat>(L, LR, patch_mask, bx, by, p, i, j, k);
  if (!lanes) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UR, i, j);
  const R *xi = velf(it, sys, 0), *xn = velf(n, sys, 0);
  const R *yi = velf(it, sys, 1), *yn = velf(n, sys, 1);
  const R *zi = velf(it, sys, 2), *zn = velf(n, sys, 2);
  V xa[NV], xb[NV], S0[NV], Srp[NV], Srm[NV], Stp[NV], Stm[NV], Spp[NV], Spm[NV];
  vld<NV>(xi + q, xa);
  vld<NV>(xn + q, xb);
#pragma unroll
  for (int l = 0; l < NV; ++l) S0[l] = xa[l] + xb[l];
  vsm<NV>(xi, xn, q + SI, Srp);
  vsm<NV>(xi, xn, q - SI, Srm);
  vsm<NV>(xi, xn, q + P, Stp);
  vsm<NV>(xi, xn, q - P, Stm);
  vup<NV>(S0, Sm<V>(xi, xn, q + NV), Spp);
  vdn<NV>(S0, Sm<V>(xi, xn, q - 1), Spm);
  // u_theta and u_phi around the face: the two cells sharing it
  V y1[NV], y0[NV], ym1[NV], ym0[NV], z1[NV], z0[NV], zm1[NV], zm0[NV];
  vsm<NV>(yi, yn, q + P, y1);
  vsm<NV>(yi, yn, q, y0);
  vsm<NV>(yi, yn, q - SI + P, ym1);
  vsm<NV>(yi, yn, q - SI, ym0);
  vsm<NV>(zi, zn, q, z0);
  vup<NV>(z0, Sm<V>(zi, zn, q + NV), z1);
  vsm<NV>(zi, zn, q - SI, zm0);
  vup<NV>(zm0, Sm<V>(zi, zn, q - SI + NV), zm1);
  V ar[NV], sAt[NV], sAp[NV];
  vld<NV>(ax.A[0] + q, ar);
  if constexpr (kTab) {
    vld<NV>(ax.As[LR][DT] + q, sAt);
    vld<NV>(ax.As[LR][DP] + q, sAp);
  } else {
    const R *A1 = ax.A[1], *A2 = ax.A[2];
    V a[NV], b[NV], c2[NV], d[NV];
    vld<NV>(A1 + q - SI, a);
    vld<NV>(A1 + q - SI + P, b);
    vld<NV>(A1 + q, c2);
    vld<NV>(A1 + q + P, d);
    vsum4<NV>(a, b, c2, d, sAt);
    vld<NV>(A2 + q - SI, a);
    vup<NV>(a, (V)A2[q - SI + NV], b);
    vld<NV>(A2 + q, c2);
    vup<NV>(c2, (V)A2[q + NV], d);
    vsum4<NV>(a, b, c2, d, sAp);
  }
  double P0[NV], Pm[NV];
  vpres<NV>(it, n, sys, q, P0);
  vpres<NV>(it, n, sys, q - SI, Pm);
  V tm[NV], t0[NV], f[NV];
  vsm<NV>(it.f[F_T], n.f[F_T], q - SI, tm);
  vsm<NV>(it.f[F_T], n.f[F_T], q, t0);
  if (ax.fr) vld<NV>(ax.fr + q, f);
  V o[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) {
    V out = c[UR_RP] * (Srp[l] - S0[l]);
    out -= c[UR_RM] * (S0[l] - Srm[l]);
    out += c[UR_TP] * (Stp[l] - S0[l]);
    out -= c[UR_TM] * (S0[l] - Stm[l]);
    out += c[UR_PP] * (Spp[l] - (V)2.0 * S0[l] + Spm[l]);
    out += c[UR_O1] * Srp[l];
    out += c[UR_O0] * S0[l];
    out += c[UR_OM] * Srm[l];
    out += c[UR_GT1] * y1[l];
    out += c[UR_GT0] * y0[l];
    out += c[UR_GTM1] * ym1[l];
    out += c[UR_GTM0] * ym0[l];
    out += c[UR_GP1] * (z1[l] - z0[l]);
    out += c[UR_GPM1] * (zm1[l] - zm0[l]);
    out -= (c[UR_AR] * ar[l]) * (Srp[l] - Srm[l]);
    out += sAt[l] * (c[UR_CV] * (((ym0[l] + ym1[l]) + y0[l]) + y1[l]) - c[UR_AT] * (Stp[l] - Stm[l]));
    out += sAp[l] * (c[UR_CV] * (((zm0[l] + zm1[l]) + z0[l]) + z1[l]) - c[UR_AP] * (Spp[l] - Spm[l]));
    out -= c[UR_GPR] * (V)(P0[l] - Pm[l]);
    out += c[UR_BY] * (tm[l] + t0[l]);
    if (ax.fr) out += cs<V>(S, CS_DT) * f[l];
    o[l] = out - (xa[l] - xb[l]);
  }
  vst<NV>(B + q, o, lanes);
}

// u_theta (body_resid_ut)
template <typename R, int NV, bool kTab = true, bool kFlat = false>
__device__ __forceinline__ void body_resid_ut_vec(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B,
                                              int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  const int lanes = decode_group<NV, kFlat>(L, LT, patch_mask, bx, by, p, i, j, k);
  if (!lanes) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UT, i, j);
  const R *wi = velf(it, sys, 0), *wn = velf(n, sys, 0);
  const R *xi = velf(it, sys, 1), *xn = velf(n, sys, 1);
  const R *zi = velf(it, sys, 2), *zn = velf(n, sys, 2);
  V xa[NV], xb[NV], S0[NV], Srp[NV], Srm[NV], Stp[NV], Stm[NV], Spp[NV], Spm[NV];
  vld<NV>(xi + q, xa);
  vld<NV>(xn + q, xb);
#pragma unroll
  for (int l = 0; l < NV; ++l) S0[l] = xa[l] + xb[l];
  vsm<NV>(xi, xn, q + SI, Srp);
  vsm<NV>(xi, xn, q - SI, Srm);
  vsm<NV>(xi, xn, q + P, Stp);
  vsm<NV>(xi, xn, q - P, Stm);
  vup<NV>(S0, Sm<V>(xi, xn, q + NV), Spp);
  vdn<NV>(S0, Sm<V>(xi, xn, q - 1), Spm);
  // u_r and u_phi around the face: the two cells sharing it
  V w1[NV], w0[NV], wm1[NV], wm0[NV], z1[NV], z0[NV], zm1[NV], zm0[NV];
  vsm<NV>(wi, wn, q + SI, w1);
  vsm<NV>(wi, wn, q, w0);
  vsm<NV>(wi, wn, q + SI - P, wm1);
  vsm<NV>(wi, wn, q - P, wm0);
  vsm<NV>(zi, zn, q, z0);
  vup<NV>(z0, Sm<V>(zi, zn, q + NV), z1);
  vsm<NV>(zi, zn, q - P, zm0);
  vup<NV>(zm0, Sm<V>(zi, zn, q - P + NV), zm1);
  V sAr[NV], at[NV], sAp[NV];
  vld<NV>(ax.A[1] + q, at);
  if constexpr (kTab) {
    vld<NV>(ax.As[LT][DR] + q, sAr);
    vld<NV>(ax.As[LT][DP] + q, sAp);
  } else {
    const R *A0 = ax.A[0], *A2 = ax.A[2];
    V a[NV], b[NV], c2[NV], d[NV];
    vld<NV>(A0 + q - P, a);
    vld<NV>(A0 + q - P + SI, b);
    vld<NV>(A0 + q, c2);
    vld<NV>(A0 + q + SI, d);
    vsum4<NV>(a, b, c2, d, sAr);
    vld<NV>(A2 + q - P, a);
    vup<NV>(a, (V)A2[q - P + NV], b);
    vld<NV>(A2 + q, c2);
    vup<NV>(c2, (V)A2[q + NV], d);
    vsum4<NV>(a, b, c2, d, sAp);
  }
  double P0[NV], Pm[NV];
  vpres<NV>(it, n, sys, q, P0);
  vpres<NV>(it, n, sys, q - P, Pm);
  V f[NV];
  if (ax.ft) vld<NV>(ax.ft + q, f);
  V o[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) {
    V out = c[UT_RP] * (Srp[l] - S0[l]);
    out -= c[UT_RM] * (S0[l] - Srm[l]);
    out += c[UT_TP] * (Stp[l] - S0[l]);
    out -= c[UT_TM] * (S0[l] - Stm[l]);
    out += c[UT_PP] * (Spp[l] - (V)2.0 * S0[l] + Spm[l]);
    out += c[UT_OTP] * Stp[l];
    out += c[UT_O0] * S0[l];
    out += c[UT_OTM] * Stm[l];
    out += c[UT_W1] * w1[l];
    out += c[UT_W0] * w0[l];
    out += c[UT_WM1] * wm1[l];
    out += c[UT_WM0] * wm0[l];
    out += c[UT_GP1] * (z1[l] - z0[l]);
    out += c[UT_GPM1] * (zm1[l] - zm0[l]);
    out -= (c[UT_AR] * sAr[l]) * (Srp[l] - Srm[l]);
    out -= at[l] * (c[UT_AT] * (Stp[l] - Stm[l]) + c[UT_CW] * (((wm0[l] + wm1[l]) + w0[l]) + w1[l]));
    out += sAp[l] * (c[UT_CP] * (((zm0[l] + zm1[l]) + z0[l]) + z1[l]) - c[UT_AP] * (Spp[l] - Spm[l]));
    out -= c[UT_GPR] * (V)(P0[l] - Pm[l]);
    if (ax.ft) out += cs<V>(S, CS_DT) * f[l];
    o[l] = out - (xa[l] - xb[l]);
  }
  vst<NV>(B + q, o, lanes);
}

// u_phi (body_resid_up)
template <typename R, int NV, bool kTab = true, bool kFlat = false>
__device__ __forceinline__ void body_resid_up_vec(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B,
                                              int patch_mask, int bx, int by) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  int p, i, j, k;
  const int lanes = decode_group<NV, kFlat>(L, LP, patch_mask, bx, by, p, i, j, k);
  if (!lanes) return;
  const long q = lidx(L, p, i, j, k), SI = L.SI, P = L.P;
  const V *c = rowc<V>(S, RT_UP, i, j);
  const R *wi = velf(it, sys, 0), *wn = velf(n, sys, 0);
  const R *yi = velf(it, sys, 1), *yn = velf(n, sys, 1);
  const R *xi = velf(it, sys, 2), *xn = velf(n, sys, 2);
  V xa[NV], xb[NV], S0[NV], Srp[NV], Srm[NV], Stp[NV], Stm[NV], Spp[NV], Spm[NV];
  vld<NV>(xi + q, xa);
  vld<NV>(xn + q, xb);
#pragma unroll
  for (int l = 0; l < NV; ++l) S0[l] = xa[l] + xb[l];
  vsm<NV>(xi, xn, q + SI, Srp);
  vsm<NV>(xi, xn, q - SI, Srm);
  vsm<NV>(xi, xn, q + P, Stp);
  vsm<NV>(xi, xn, q - P, Stm);
  vup<NV>(S0, Sm<V>(xi, xn, q + NV), Spp);
  vdn<NV>(S0, Sm<V>(xi, xn, q - 1), Spm);
  // u_r and u_theta around the face: the two cells sharing it
  V w1[NV], w0[NV], wm1[NV], wm0[NV], y1[NV], y0[NV], ym1[NV], ym0[NV];
  vsm<NV>(wi, wn, q + SI, w1);
  vsm<NV>(wi, wn, q, w0);
  vdn<NV>(w1, Sm<V>(wi, wn, q - 1 + SI), wm1);
  vdn<NV>(w0, Sm<V>(wi, wn, q - 1), wm0);
  vsm<NV>(yi, yn, q + P, y1);
  vsm<NV>(yi, yn, q, y0);
  vdn<NV>(y1, Sm<V>(yi, yn, q - 1 + P), ym1);
  vdn<NV>(y0, Sm<V>(yi, yn, q - 1), ym0);
  V sAr[NV], sAt[NV], ap[NV];
  vld<NV>(ax.A[2] + q, ap);
  if constexpr (kTab) {
    vld<NV>(ax.As[LP][DR] + q, sAr);
    vld<NV>(ax.As[LP][DT] + q, sAt);
  } else {
    const R *A0 = ax.A[0], *A1 = ax.A[1];
    V a[NV], b[NV], c2[NV], d[NV];
    vld<NV>(A0 + q, c2);
    vld<NV>(A0 + q + SI, d);
    vdn<NV>(c2, (V)A0[q - 1], a);
    vdn<NV>(d, (V)A0[q - 1 + SI], b);
    vsum4<NV>(a, b, c2, d, sAr);
    vld<NV>(A1 + q, c2);
    vld<NV>(A1 + q + P, d);
    vdn<NV>(c2, (V)A1[q - 1], a);
    vdn<NV>(d, (V)A1[q - 1 + P], b);
    vsum4<NV>(a, b, c2, d, sAt);
  }
  double P0[NV], Pm[NV];
  vpres<NV>(it, n, sys, q, P0);
  vdn<NV>(P0, pres(it, n, sys, q - 1), Pm);
  V f[NV];
  if (ax.fp) vld<NV>(ax.fp + q, f);
  V o[NV];
#pragma unroll
  for (int l = 0; l < NV; ++l) {
    V out = c[UP_RP] * (Srp[l] - S0[l]);
    out -= c[UP_RM] * (S0[l] - Srm[l]);
    out += c[UP_TP] * (Stp[l] - S0[l]);
    out -= c[UP_TM] * (S0[l] - Stm[l]);
    out += c[UP_PP] * (Spp[l] - (V)2.0 * S0[l] + Spm[l]);
    out += c[UP_E0] * S0[l];
    out += c[UP_W1] * w1[l];
    out += c[UP_W0] * w0[l];
    out += c[UP_WM1] * wm1[l];
    out += c[UP_WM0] * wm0[l];
    out += c[UP_Y1] * y1[l];
    out += c[UP_Y0] * y0[l];
    out += c[UP_YM1] * ym1[l];
    out += c[UP_YM0] * ym0[l];
    out -= (c[UP_AR] * sAr[l]) * (Srp[l] - Srm[l]);
    out -= (c[UP_AT] * sAt[l]) * (Stp[l] - Stm[l]);
    out -= ap[l] * (c[UP_AP] * (Spp[l] - Spm[l]) + c[UP_CW] * (((wm0[l] + wm1[l]) + w0[l]) + w1[l]) +
                    c[UP_CY] * (((ym0[l] + ym1[l]) + y0[l]) + y1[l]));
    out -= c[UP_GPR] * (V)(P0[l] - Pm[l]);
    if (ax.fp) out += cs<V>(S, CS_DT) * f[l];
    o[l] = out - (xa[l] - xb[l]);
  }
  vst<NV>(B + q, o, lanes);
}

// Pressure update of one cell (Eq. nst_Mass1 for system 1, Eq. ac2 for system
// 2).  Returns the cell's share r^2 sin(theta) (p_new - p_old)^2 of the
// midpoint-rule norm of the pressure increment without the constant cell
// volume (norm_flush applies it); step-7 ring cells contribute nothing.  The
// caller accumulates shares over many cells, so that one atomic serves many
// thousands of cells.
template <typename R, bool kSum = false>
__device__ __forceinline__ typename Cmp<R>::type body_pressure_at(Shell S, int sys, State<R> it, State<R> n,
                                                                  int p, int i, int j, int k,
                                                                  const R *const *Sv = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  const long q = lidx(L, p, i, j, k);
  double D;
  if constexpr (sizeof(R) == sizeof(float)) {
    // FP32 storage: double-float divergence (FP64-accurate, FP32 instructions)
    // (divergence / chi) with the factor 2 (2 chi)^-1 applied in double-float
    const FF kc = ff_mul(ff_cs(S, CS_I2CHI), FF{2.0f, 0.0f});
    D = ff_double(ff_mul(kc, divh_ff(S, velf(it, sys, 0), velf(n, sys, 0), velf(it, sys, 1), velf(n, sys, 1),
                                     velf(it, sys, 2), velf(n, sys, 2), i, j, q)));
  } else {
    // divergence of the half-level velocity times 1/chi from the row record
    const double *c = rowc<double>(S, RT_DIV, i, j);
    const R *ri = velf(it, sys, 0), *rn = velf(n, sys, 0), *ti = velf(it, sys, 1), *tn = velf(n, sys, 1);
    const R *pi = velf(it, sys, 2), *pn = velf(n, sys, 2);
    if constexpr (kSum)   // precomputed two-level sums (LevelSums)
      D = (c[DV_R1] * (double)Sv[0][q + L.SI] - c[DV_R0] * (double)Sv[0][q]) +
          (c[DV_T1] * (double)Sv[1][q + L.P] - c[DV_T0] * (double)Sv[1][q]) +
          c[DV_P] * ((double)Sv[2][q + 1] - (double)Sv[2][q]);
    else
      D = (c[DV_R1] * Sm<double>(ri, rn, q + L.SI) - c[DV_R0] * Sm<double>(ri, rn, q)) +
          (c[DV_T1] * Sm<double>(ti, tn, q + L.P) - c[DV_T0] * Sm<double>(ti, tn, q)) +
          c[DV_P] * (Sm<double>(pi, pn, q + 1) - Sm<double>(pi, pn, q));
  }
  double pnew;
  double *dst;
  if (sys == 1) {
    pnew = n.p[0][q] - D;
    dst = it.p[0];
  } else {
    pnew = n.p[1][q] + (it.p[0][q] - n.p[0][q]) - D;
    dst = it.p[1];
  }
  const V c = (V)(pnew - dst[q]);
  dst[q] = pnew;
  const bool ringcell = (j == 0 || j == L.Nt - 1 || k == 0 || k == L.Np - 1);
  if (S.step7 && ringcell) return (V)0.0;
  return rowc<V>(S, RT_DIV, i, j)[DV_W] * c * c;
}

// the pressure update of the cell of (bx, by) in a row-per-block grid
template <typename R, bool kSum = false>
__device__ __forceinline__ typename Cmp<R>::type body_pressure(Shell S, int sys, State<R> it, State<R> n,
                                                               int patch_mask, int bx, int by,
                                                               const R *const *Sv = nullptr) {
  int p, i, j, k;
  if (!decode_point(S.L, LC, patch_mask, bx, by, p, i, j, k)) return (typename Cmp<R>::type)0.0;
  return body_pressure_at<R, kSum>(S, sys, it, n, p, i, j, k, Sv);
}

// Warp sum of per-thread norm shares, scaled once and added to *dst by lane 0.
// Every lane of the warp must call it.
template <typename V>
__device__ __forceinline__ void norm_flush(V part, double scale, double *dst) {
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0 && part != (V)0.0) atomicAdd(dst, (double)part * scale);
}

// elements [q0, q1) of every field, threads striding by blockDim.x
template <typename R>
__device__ __forceinline__ void body_extrapolate(long q0, long q1, State<R> it, State<R> n, State<R> nm1, R *A0,
                                                 R *A1, R *A2) {
  using V = typename Cmp<R>::type;
  const int bulk[7] = {F_T, F_U1R, F_U1T, F_U1P, F_U2R, F_U2T, F_U2P};
  for (long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    // every load first: the stores below may alias the inputs as far as the
    // compiler knows, so loads placed after a store would wait for it
    V a[7], b[7];
    double pa[2], pb[2];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      a[k] = (V)n.f[bulk[k]][q];
      b[k] = (V)nm1.f[bulk[k]][q];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      pa[k] = n.p[k][q];
      pb[k] = nm1.p[k][q];
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) it.f[bulk[k]][q] = (R)((V)2.0 * a[k] - b[k]);
    it.p[0][q] = 2.0 * pa[0] - pb[0];
    it.p[1][q] = 2.0 * pa[1] - pb[1];
    A0[q] = (R)((V)1.5 * a[4] - (V)0.5 * b[4]);
    A1[q] = (R)((V)1.5 * a[5] - (V)0.5 * b[5]);
    A2[q] = (R)((V)1.5 * a[6] - (V)0.5 * b[6]);
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
__device__ __forceinline__ void body_walls(Shell S, WallData wt, State<R> s, int patch_mask, int bx, int by) {
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
  // u_r on the wall faces i = 0 and i = Nr: the wall velocity on the unknown
  // columns (0 = no-slip unless wall data is set), 0 on the ghost columns
  const bool cc = (j >= 0 && j < Nt && k >= 0 && k < Np);
  double g0 = 0.0, g1 = 0.0;
  const long qc0 = ((long)(0 * 2 + p) * Nt + j) * Np + k, qc1 = ((long)(1 * 2 + p) * Nt + j) * Np + k;
  if (S.wall_ur && cc) {
    g0 = S.wall_ur[qc0];
    g1 = S.wall_ur[qc1];
  }
  if (wt.ur && cc) {
    g0 += wt.tau * wt.ur[qc0];
    g1 += wt.tau * wt.ur[qc1];
  }
  s.f[F_U1R][l0] = (R)g0;
  s.f[F_U2R][l0] = (R)g0;
  s.f[F_U1R][hi] = (R)g1;
  s.f[F_U2R][hi] = (R)g1;
  if (cc) {
    double T0 = S.T_in, T1 = S.T_out;
    if (wt.T) {
      T0 += wt.tau * wt.T[qc0];
      T1 += wt.tau * wt.T[qc1];
    }
    s.f[F_T][lo] = (R)(S.Tgam[0] * (double)s.f[F_T][l0] + S.Tdel[0] * T0);
    s.f[F_T][hi] = (R)(S.Tgam[1] * (double)s.f[F_T][h0] + S.Tdel[1] * T1);
  }
  // u_theta, u_phi: reflection ghosts 2 g - x_0 about the wall velocity g
  if (j >= 1 && j < Nt && k >= 0 && k < Np) {
    g0 = g1 = 0.0;
    const long q0 = ((long)(0 * 2 + p) * (Nt + 1) + j) * Np + k, q1 = ((long)(1 * 2 + p) * (Nt + 1) + j) * Np + k;
    if (S.wall_ut) {
      g0 = S.wall_ut[q0];
      g1 = S.wall_ut[q1];
    }
    if (wt.ut) {
      g0 += wt.tau * wt.ut[q0];
      g1 += wt.tau * wt.ut[q1];
    }
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1T + o];
      u[lo] = (R)(2.0 * g0 - (double)u[l0]);
      u[hi] = (R)(2.0 * g1 - (double)u[h0]);
    }
  }
  if (j >= 0 && j < Nt && k >= 1 && k < Np) {
    g0 = g1 = 0.0;
    const long q0 = ((long)(0 * 2 + p) * Nt + j) * (Np + 1) + k, q1 = ((long)(1 * 2 + p) * Nt + j) * (Np + 1) + k;
    if (S.wall_up) {
      g0 = S.wall_up[q0];
      g1 = S.wall_up[q1];
    }
    if (wt.up) {
      g0 += wt.tau * wt.up[q0];
      g1 += wt.tau * wt.up[q1];
    }
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1P + o];
      u[lo] = (R)(2.0 * g0 - (double)u[l0]);
      u[hi] = (R)(2.0 * g1 - (double)u[h0]);
    }
  }
}

// Component along `dir` of the advecting velocity at a point of location
// `loc`: the own component as stored, the others averaged from their nearest
// stored values (in the arithmetic type V).
// kTab: the other components come from the per-step sums StepAux::As (the
// same values added in the same order, times 1/2 or 1/4); without it (the
// batched launches, whose StepAux is built at run time, where indexing its
// table array would put it in local memory) they are averaged here.
template <typename V, bool kTab = false, typename R>
__device__ __forceinline__ V advecting(const Shell &S, const StepAux<R> &ax, int loc, int dir, long q) {
  if constexpr (kTab) {
    if (loc != dir + 1) return (V)ax.As[loc][dir][q] * ((loc == LC) ? (V)0.5 : (V)0.25);
  }
  const long SI = S.L.SI, P = S.L.P;
  if (dir == DR) {
    const R *A0 = ax.A[0];
    if (loc == LC) return ((V)A0[q] + (V)A0[q + SI]) * (V)0.5;
    if (loc == LR) return (V)A0[q];
    if (loc == LT) return avg4<V>(A0, q - P, q - P + SI, q, q + SI);
    return avg4<V>(A0, q - 1, q - 1 + SI, q, q + SI);
  }
  if (dir == DT) {
    const R *A1 = ax.A[1];
    if (loc == LC) return ((V)A1[q] + (V)A1[q + P]) * (V)0.5;
    if (loc == LR) return avg4<V>(A1, q - SI, q - SI + P, q, q + P);
    if (loc == LT) return (V)A1[q];
    return avg4<V>(A1, q - 1, q - 1 + P, q, q + P);
  }
  const R *A2 = ax.A[2];
  if (loc == LC) return ((V)A2[q] + (V)A2[q + 1]) * (V)0.5;
  if (loc == LR) return avg4<V>(A2, q - SI, q - SI + 1, q, q + 1);
  if (loc == LT) return avg4<V>(A2, q - P, q - P + 1, q, q + 1);
  return (V)A2[q];
}

// Coefficients (lo, di, up) of (I - dt/2 Ahat_dir) at point (i, j, k) of
// `loc`: the row's static parts (FacCoef table, formed on the host in FP64)
// and the advecting velocity at the point.
template <typename V, bool kTab = false, typename R>
__device__ __forceinline__ void coef(const Shell &S, const StepAux<R> &ax, int loc, int dir, int i, int j, long q,
                                     V &lo, V &di, V &up) {
  const V *c = facc<V>(S, loc, dir, i, j);
  const V a = advecting<V, kTab>(S, ax, loc, dir, q);
  lo = c[FC_L0] + a * c[FC_LA];
  di = c[FC_D0];
  up = c[FC_U0] - a * c[FC_LA];
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


// Coefficients (lo, di, up) of the rows [m, m + U) of a line, with the wall
// rows closed (reflection ghosts folded into the diagonal, the outside
// coupling zeroed).
template <int U, bool kTab, typename V, typename R>
__device__ __forceinline__ void factor_coefs(const Shell &S, const StepAux<R> &ax, const Line &ln, int loc, int dir,
                                             bool reflect, V gam0, V gam1, long step, int m, long qm, V (&lo)[U],
                                             V (&di)[U], V (&up)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int mm = m + u;
    if (mm < ln.m1) {
      const int ii = (dir == DR) ? mm : ln.i, jj = (dir == DT) ? mm : ln.j;
      coef<V, kTab>(S, ax, loc, dir, ii, jj, qm + u * step, lo[u], di[u], up[u]);
      if (mm == ln.m0) {
        if (reflect) di[u] += gam0 * lo[u];
        lo[u] = (V)0.0;
      }
      if (mm == ln.m1 - 1) {
        if (reflect) di[u] += gam1 * up[u];
        up[u] = (V)0.0;
      }
    }
  }
}

// kTab (the single-shell launches): the advecting velocity comes from the
// per-step sums; the batched launches average it themselves.  (Forming the
// next chunk's coefficients before the current chunk's recurrence, as the
// solves prefetch, made the factorisations slower: 42 -> 48 ms FP64,
// 12 -> 19 ms mixed per 10 steps at 128x128x384.)
template <typename R, bool kTab = false>
__device__ __forceinline__ void body_factorize(Shell S, int loc, int dir, StepAux<R> ax, R *__restrict__ Lo,
                                               R *__restrict__ Iv, R *__restrict__ Cp, int patch_mask, int bx,
                                               int by) {
  using V = typename Cmp<R>::type;
  // rows whose coefficients are formed (loads in flight) before the recurrence consumes them
  constexpr int U = sizeof(R) == sizeof(float) ? 8 : 4;
  const Layout &L = S.L;
  const Line ln = decode_line(L, loc, dir, bx * blockDim.x + threadIdx.x, by);
  if (!ln.valid || !((patch_mask >> ln.p) & 1)) return;
  // cell-centred quantities in r: correction ghost = gamma x (reflection -1;
  // the temperature's wall condition gives its own gamma)
  const bool reflect = (dir == DR) && (loc != LR);
  const V gam0 = (loc == LC) ? (V)S.Tgam[0] : (V)-1.0, gam1 = (loc == LC) ? (V)S.Tgam[1] : (V)-1.0;
  const long step = ln.step;
  V cprev = (V)0.0;
  long q = lidx(L, ln.p, ln.i, ln.j, ln.k);
  for (int m = ln.m0; m < ln.m1; m += U, q += U * step) {
    V lo[U], di[U], up[U];
    factor_coefs<U, kTab>(S, ax, ln, loc, dir, reflect, gam0, gam1, step, m, q, lo, di, up);
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

// Loads of one chunk of a line solve: forward rows [m, m + U) of b, lo and
// 1/pivot; backward rows m, m - 1, ..., m - U + 1 of d', c' and (final
// factor) the iterate.  Issued for the next chunk before the current one is
// processed.
template <int U, typename R, typename V>
__device__ __forceinline__ void solve_load_fwd(const R *__restrict__ B, const R *__restrict__ Lo,
                                               const R *__restrict__ Iv, long q0, long step, int n, int m,
                                               V (&b)[U], V (&lo)[U], V (&iv)[U]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long qq = q0 + (long)(m + u) * step;
    if (m + u < n) {
      b[u] = (V)B[qq];
      lo[u] = (V)Lo[qq];
      iv[u] = (V)Iv[qq];
    }
  }
}
template <int U, bool kSum = false, typename R, typename V>
__device__ __forceinline__ void solve_load_bwd(const R *__restrict__ W, const R *__restrict__ Cp,
                                               const R *__restrict__ dst, int final, long q0, long step, int m,
                                               V (&w)[U], V (&c)[U], V (&o)[U], const R *__restrict__ Pn = nullptr,
                                               V *pn = nullptr) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long qq = q0 + (long)(m - u) * step;
    if (m - u >= 0) {
      w[u] = (V)W[qq];
      c[u] = (V)Cp[qq];
      o[u] = final ? (V)dst[qq] : (V)0.0;
      if constexpr (kSum) pn[u] = (V)Pn[qq];
    }
  }
}

// Thomas solve with a stored factorisation: forward d'_m = (b_m - lo_m d'_{m-1})
// / pivot_m into the scratch W, back x_m = d'_m - c'_m x_{m+1}.  Rows are
// handled in register chunks of U: the loads of a chunk are independent of
// the recurrence and of every store (separate arrays), so they are in flight
// together.  Non-final factors write x to B (the next factor's right-hand
// side); the final factor of an unknown adds x to the iterate and accumulates
// the FP64 midpoint-rule norm of the increment (Sec. 5.1).  kSum (final
// factors of the FP64 single-shell launches): also Sout = new value + Pn, the
// two-level sum the next residuals read (LevelSums), with their addition.
template <typename R, bool kPf = false, bool kSum = false>
__device__ __forceinline__ void body_solve(Shell S, int loc, int dir, int final, const R *__restrict__ Lo,
                                           const R *__restrict__ Iv, const R *__restrict__ Cp, R *__restrict__ B,
                                           R *__restrict__ W, R *__restrict__ dst, double *norm, int slot,
                                           int patch_mask, int bx, int by, const R *__restrict__ Pn = nullptr,
                                           R *__restrict__ Sout = nullptr) {
  using V = typename Cmp<R>::type;
  // rows per register chunk: 8 in FP32; 4 in FP64, where 8 rows and the next
  // chunk's prefetch took 128 registers, too many for all lines of a
  // 128x128x384 sweep to be resident at once (80 with 4 rows: 20% faster)
  constexpr int U = sizeof(R) == sizeof(double) ? 4 : 8;
  const Layout &L = S.L;
  const Line ln = decode_line(L, loc, dir, bx * blockDim.x + threadIdx.x, by);
  double contrib = 0.0;
  if (ln.valid && ((patch_mask >> ln.p) & 1)) {
    const long step = ln.step;
    const long q0 = lidx(L, ln.p, ln.i, ln.j, ln.k);
    const int n = ln.m1 - ln.m0;
    // forward elimination: B -> W; with kPf the loads of the next chunk are
    // issued before the current chunk is eliminated, so that they are in
    // flight during its dependent arithmetic and stores (the single-shell
    // launches; the batched ones, short of registers, load chunk by chunk)
    V d = (V)0.0;
    V b[U], lo[U], iv[U];
    if constexpr (kPf) solve_load_fwd<U>(B, Lo, Iv, q0, step, n, 0, b, lo, iv);
    for (int m = 0; m < n; m += U) {
      V nb[U], nlo[U], niv[U];
      if constexpr (kPf) {
        if (m + U < n) solve_load_fwd<U>(B, Lo, Iv, q0, step, n, m + U, nb, nlo, niv);
      } else {
        solve_load_fwd<U>(B, Lo, Iv, q0, step, n, m, b, lo, iv);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (m + u < n) {
          d = (b[u] - lo[u] * d) * iv[u];
          W[q0 + (long)(m + u) * step] = (R)d;
        }
      }
      if constexpr (kPf) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          b[u] = nb[u];
          lo[u] = nlo[u];
          iv[u] = niv[u];
        }
      }
    }
    // back substitution: W -> B or the iterate, last row first; the final
    // factor sums w x^2 along the line in V, w the metric factor that varies
    // along it (r^2, sin(theta) or 1), and scales once by the constant rest
    V x = d;
    V acc = (V)0.0;
    V w[U], c[U], o[U], pn[kSum ? U : 1];
    if constexpr (kPf) solve_load_bwd<U, kSum>(W, Cp, dst, final, q0, step, n - 1, w, c, o, Pn, pn);
    for (int m = n - 1; m >= 0; m -= U) {
      V nw[U], nc[U], no[U], npn[kSum ? U : 1];
      if constexpr (kPf) {
        if (m - U >= 0) solve_load_bwd<U, kSum>(W, Cp, dst, final, q0, step, m - U, nw, nc, no, Pn, npn);
      } else {
        solve_load_bwd<U, kSum>(W, Cp, dst, final, q0, step, m, w, c, o, Pn, pn);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int mm = m - u;
        if (mm >= 0) {
          long qq = q0 + (long)mm * step;
          if (mm < n - 1) x = w[u] - c[u] * x;
          if (final) {
            const R nv = (R)(o[u] + x);
            dst[qq] = nv;
            if constexpr (kSum) Sout[qq] = (R)((V)nv + pn[u]);
            const int row = ln.m0 + mm;
            if (dir == DR) {
              const V t = ((loc == LR) ? mt<V>(S, MT_NRF) : mt<V>(S, MT_NRC))[row] * x;
              acc += t * t;
            } else if (dir == DT) {
              acc += ((loc == LT) ? mt<V>(S, MT_SF) : mt<V>(S, MT_SC))[row] * x * x;
            } else {
              acc += x * x;
            }
          } else {
            B[qq] = (R)x;
          }
        }
      }
      if constexpr (kPf) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          w[u] = nw[u];
          c[u] = nc[u];
          o[u] = no[u];
          if constexpr (kSum) pn[u] = npn[u];
        }
      }
    }
    if (final) {
      // r sqrt(h / h_r): the radial part of the point's midpoint-rule weight
      const double r = (loc == LR) ? S.nrf[ln.i] : S.nrc[ln.i];
      const double sn = (loc == LT) ? S.sf[ln.j] : S.sc[ln.j];
      const double w = (dir == DR) ? sn : (dir == DT) ? r * r : r * r * sn;
      contrib = (double)acc * (w * S.dcs[CS_VOL]);
    }
  }
  if (final) {
    for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
    if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(&norm[slot], contrib);
  }
}

// Line solve along phi as a warp scan: one warp per line (the line's values
// are contiguous in memory).  Lane t owns the segment of EC consecutive
// positions [c0 + t EC, c0 + (t + 1) EC) of a chunk of 32 EC positions, read
// and written with 16-byte vector accesses.  The forward recurrence
// d_m = iv_m (b_m - lo_m d_{m-1}) is the affine map d -> a_m d + f_m
// (a_m = -iv_m lo_m, f_m = iv_m b_m); each lane composes the maps of its
// segment, an inclusive Kogge-Stone scan over the lanes (5 shuffle steps)
// composes the segments, and each lane then replays its segment from its
// incoming value.  The back substitution x_m = d_m - c'_m x_{m+1} is the
// same with the scan running downwards.  The forward results d stay in a
// per-warp shared-memory buffer when the line fits (`wsm`), else in W.
// Positions outside [k0, Np) map to 0 (the chain restarts at k0 anyway) and
// are never written.
// The factorisation scan carries several times the arithmetic of the
// sequential elimination (2x2 matrix products): it pays off where memory
// latency is the bound (FP32 storage), not where the FP64 pipe is (measured:
// FP64 phi factorisation 59.9 ms per 10 steps as a scan, 50.0 sequential;
// the solve scan stays ahead in both forms, 54.1 vs 69.9 ms in FP64).
template <typename R>
__host__ __device__ constexpr bool use_phi_scan() {
  return sizeof(R) == sizeof(float);
}
constexpr int kScanWarps = 4;           // lines (warps) per CTA
constexpr int kScanSmemMax = 96 * 1024;   // shared memory a CTA may take for the forward results

template <int EC, typename R, typename V>
__device__ __forceinline__ void seg_load(const R *__restrict__ p, bool full, int k, int k0, int k1, V *out) {
  if (full) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int v = 0; v < EC / 4; ++v) {
        const float4 t = *reinterpret_cast<const float4 *>(p + 4 * v);
        out[4 * v] = (V)t.x;
        out[4 * v + 1] = (V)t.y;
        out[4 * v + 2] = (V)t.z;
        out[4 * v + 3] = (V)t.w;
      }
    } else {
#pragma unroll
      for (int v = 0; v < EC / 2; ++v) {
        const double2 t = *reinterpret_cast<const double2 *>(p + 2 * v);
        out[2 * v] = (V)t.x;
        out[2 * v + 1] = (V)t.y;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < EC; ++e) out[e] = (k + e >= k0 && k + e < k1) ? (V)p[e] : (V)0.0;
  }
}

template <int EC, typename R, typename V>
__device__ __forceinline__ void seg_store(R *__restrict__ p, bool full, int k, int k0, int k1, const V *in) {
  if (full) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int v = 0; v < EC / 4; ++v)
        *reinterpret_cast<float4 *>(p + 4 * v) =
            make_float4((float)in[4 * v], (float)in[4 * v + 1], (float)in[4 * v + 2], (float)in[4 * v + 3]);
    } else {
#pragma unroll
      for (int v = 0; v < EC / 2; ++v)
        *reinterpret_cast<double2 *>(p + 2 * v) = make_double2((double)in[2 * v], (double)in[2 * v + 1]);
    }
  } else {
#pragma unroll
    for (int e = 0; e < EC; ++e)
      if (k + e >= k0 && k + e < k1) p[e] = (R)in[e];
  }
}

template <int EC, bool kSum = false, bool kSeg = false, typename R>
__device__ __forceinline__ void solve_line_scan(int k0, int k1, int final, const R *__restrict__ Lo,
                                                const R *__restrict__ Iv, const R *__restrict__ Cp,
                                                R *__restrict__ B, R *__restrict__ wbuf, R *__restrict__ dst,
                                                typename Cmp<R>::type &acc, const R *__restrict__ Pn = nullptr,
                                                R *__restrict__ Sout = nullptr, const R *__restrict__ Aseg = nullptr,
                                                const R *__restrict__ Gseg = nullptr) {
  using V = typename Cmp<R>::type;
  const int lane = threadIdx.x & 31;
  constexpr int CH = 32 * EC;
  const int nch = (k1 + CH - 1) / CH;
  // forward elimination into wbuf
  V dcarry = (V)0.0;
  for (int c = 0; c < nch; ++c) {
    const int k = c * CH + lane * EC;
    const bool full = (k >= k0 && k + EC <= k1);
    V a[EC], f[EC];
    {
      V b[EC], lo[EC], iv[EC];
      seg_load<EC>(B + k, full, k, k0, k1, b);
      seg_load<EC>(Lo + k, full, k, k0, k1, lo);
      seg_load<EC>(Iv + k, full, k, k0, k1, iv);
#pragma unroll
      for (int e = 0; e < EC; ++e) {
        // kSeg: Lo holds a = -iv lo already (phi_segments)
        a[e] = kSeg ? lo[e] : -iv[e] * lo[e];
        f[e] = iv[e] * b[e];
      }
    }
    V A = (V)1.0, F = (V)0.0;
    if constexpr (kSeg) {
      A = (V)Aseg[c * 32 + lane];
#pragma unroll
      for (int e = 0; e < EC; ++e) F = a[e] * F + f[e];
    } else {
#pragma unroll
      for (int e = 0; e < EC; ++e) {
        A = a[e] * A;
        F = a[e] * F + f[e];
      }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const V Ao = __shfl_up_sync(0xffffffffu, A, off), Fo = __shfl_up_sync(0xffffffffu, F, off);
      if (lane >= off) {
        F = A * Fo + F;
        A = A * Ao;
      }
    }
    V Ae = __shfl_up_sync(0xffffffffu, A, 1), Fe = __shfl_up_sync(0xffffffffu, F, 1);
    if (lane == 0) {
      Ae = (V)1.0;
      Fe = (V)0.0;
    }
    V d = Ae * dcarry + Fe;
    V out[EC];
#pragma unroll
    for (int e = 0; e < EC; ++e) {
      d = a[e] * d + f[e];
      out[e] = d;
    }
    seg_store<EC>(wbuf + k, full, k, k0, k1, out);
    dcarry = __shfl_sync(0xffffffffu, A * dcarry + F, 31);
  }
  __syncwarp();
  // back substitution from the last chunk down
  V xcarry = (V)0.0;
  for (int c = nch - 1; c >= 0; --c) {
    const int k = c * CH + lane * EC;
    const bool full = (k >= k0 && k + EC <= k1);
    V g[EC], w[EC];
    {
      V cp[EC];
      seg_load<EC>(Cp + k, full, k, k0, k1, cp);
      seg_load<EC>(wbuf + k, full, k, k0, k1, w);
#pragma unroll
      for (int e = 0; e < EC; ++e) g[e] = -cp[e];
    }
    V G = (V)1.0, X = (V)0.0;
    if constexpr (kSeg) {
      G = (V)Gseg[c * 32 + lane];
#pragma unroll
      for (int e = EC - 1; e >= 0; --e) X = g[e] * X + w[e];
    } else {
#pragma unroll
      for (int e = EC - 1; e >= 0; --e) {
        G = g[e] * G;
        X = g[e] * X + w[e];
      }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const V Go = __shfl_down_sync(0xffffffffu, G, off), Xo = __shfl_down_sync(0xffffffffu, X, off);
      if (lane + off < 32) {
        X = G * Xo + X;
        G = G * Go;
      }
    }
    V Ge = __shfl_down_sync(0xffffffffu, G, 1), Xe = __shfl_down_sync(0xffffffffu, X, 1);
    if (lane == 31) {
      Ge = (V)1.0;
      Xe = (V)0.0;
    }
    V x = Ge * xcarry + Xe;
    V out[EC];
#pragma unroll
    for (int e = EC - 1; e >= 0; --e) {
      x = g[e] * x + w[e];
      out[e] = x;
    }
    if (final) {
      V o[EC];
      seg_load<EC>(dst + k, full, k, k0, k1, o);
#pragma unroll
      for (int e = 0; e < EC; ++e) {
        if (k + e >= k0 && k + e < k1) acc += out[e] * out[e];
        o[e] = o[e] + out[e];
      }
      seg_store<EC>(dst + k, full, k, k0, k1, o);
      if constexpr (kSum) {
        // the two-level sum of the stored new value (R = V here: FP64)
        V pn[EC];
        seg_load<EC>(Pn + k, full, k, k0, k1, pn);
#pragma unroll
        for (int e = 0; e < EC; ++e) pn[e] = o[e] + pn[e];
        seg_store<EC>(Sout + k, full, k, k0, k1, pn);
      }
    } else {
      seg_store<EC>(B + k, full, k, k0, k1, out);
    }
    xcarry = __shfl_sync(0xffffffffu, G * xcarry + X, 0);
  }
}

// positions per lane of a phi line of Np positions (one chunk up to 384,
// longer lines in chunks of 384)
inline __host__ __device__ int scan_ec(int Np) {
  const int e = (Np + 31) / 32;
  return e <= 4 ? 4 : e <= 8 ? 8 : 12;
}
// shared-memory positions per warp for the forward results of a line
inline __host__ __device__ int scan_pad(int Np) {
  const int ch = 32 * scan_ec(Np);
  return (Np + ch - 1) / ch * ch;
}
// lane segments of one phi line (32 per chunk) and the length of the FP64
// lane-segment product arrays of one unknown (2 Nr Nt lines at most)
inline __host__ __device__ int scan_segs(int Np) { return 32 * (scan_pad(Np) / (32 * scan_ec(Np))); }
inline __host__ __device__ long phi_seg_elems(const Layout &L) { return 2L * L.Nr * L.Nt * scan_segs(L.Np); }
// lines of a location type and the CTAs of body_solve_phi_scan for one shell
inline int phi_scan_ctas(const Layout &L, int loc) {
  const long lines = 2L * (L.Nr - (loc == LR ? 1 : 0)) * (L.Nt - (loc == LT ? 1 : 0));
  return (int)((lines + kScanWarps - 1) / kScanWarps);
}

// Per-step lane-segment products of a phi factorisation (FP64 single-shell
// solves, kSeg): for every chunk c and lane t of a line, the products over
// the lane's segment of a_m = -iv_m lo_m (in the order the forward scan
// multiplies them) and of g_m = -c'_m (in the backward order), which depend
// on the factors only, so that each of the step's solves along phi reads them
// instead of forming them; Lo is overwritten with a.  The arithmetic and the
// masks are those of solve_line_scan, so the solves give the same results.
template <int EC, typename R>
__device__ __forceinline__ void segment_line(int k0, int k1, R *__restrict__ Lo, const R *__restrict__ Iv,
                                             const R *__restrict__ Cp, R *__restrict__ Aseg,
                                             R *__restrict__ Gseg) {
  using V = typename Cmp<R>::type;
  const int lane = threadIdx.x & 31;
  constexpr int CH = 32 * EC;
  const int nch = (k1 + CH - 1) / CH;
  for (int c = 0; c < nch; ++c) {
    const int k = c * CH + lane * EC;
    const bool full = (k >= k0 && k + EC <= k1);
    V lo[EC], iv[EC], cp[EC], a[EC];
    seg_load<EC>(Lo + k, full, k, k0, k1, lo);
    seg_load<EC>(Iv + k, full, k, k0, k1, iv);
    seg_load<EC>(Cp + k, full, k, k0, k1, cp);
    V A = (V)1.0, G = (V)1.0;
#pragma unroll
    for (int e = 0; e < EC; ++e) {
      a[e] = -iv[e] * lo[e];
      A = a[e] * A;
    }
#pragma unroll
    for (int e = EC - 1; e >= 0; --e) G = -cp[e] * G;
    Aseg[c * 32 + lane] = (R)A;
    Gseg[c * 32 + lane] = (R)G;
    seg_store<EC>(Lo + k, full, k, k0, k1, a);
  }
}

template <typename R>
__device__ __forceinline__ void body_phi_segments(Shell S, int loc, R *__restrict__ Lo, const R *__restrict__ Iv,
                                                  const R *__restrict__ Cp, R *__restrict__ Aseg,
                                                  R *__restrict__ Gseg, int patch_mask, int bx) {
  const Layout &L = S.L;
  const int warp = threadIdx.x >> 5;
  const int i0 = (loc == LR) ? 1 : 0, j0 = (loc == LT) ? 1 : 0, k0 = (loc == LP) ? 1 : 0;
  const int ni = L.Nr - i0, nj = L.Nt - j0;
  const int line = bx * kScanWarps + warp;
  if (line >= 2 * ni * nj) return;
  const int j = j0 + line % nj;
  const int rest = line / nj;
  const int i = i0 + rest % ni, p = rest / ni;
  if (!((patch_mask >> p) & 1)) return;
  const long q = lidx(L, p, i, j, 0);
  const long so = (long)line * scan_segs(L.Np);
  switch (scan_ec(L.Np)) {
    case 4:
      segment_line<4>(k0, L.Np, Lo + q, Iv + q, Cp + q, Aseg + so, Gseg + so);
      break;
    case 8:
      segment_line<8>(k0, L.Np, Lo + q, Iv + q, Cp + q, Aseg + so, Gseg + so);
      break;
    default:
      segment_line<12>(k0, L.Np, Lo + q, Iv + q, Cp + q, Aseg + so, Gseg + so);
      break;
  }
}

// one phi line per warp; `smem_per_warp` positions of shared memory per warp
// (0 or too few: the forward results go through W)
template <typename R, bool kSum = false, bool kSeg = false>
__device__ __forceinline__ void body_solve_phi_scan(Shell S, int loc, int final, const R *__restrict__ Lo,
                                                    const R *__restrict__ Iv, const R *__restrict__ Cp,
                                                    R *__restrict__ B, R *__restrict__ W, R *__restrict__ dst,
                                                    double *norm, int slot, int patch_mask, int bx, R *smem,
                                                    int smem_per_warp, const R *__restrict__ Pn = nullptr,
                                                    R *__restrict__ Sout = nullptr,
                                                    const R *__restrict__ const *seg = nullptr) {
  using V = typename Cmp<R>::type;
  const Layout &L = S.L;
  const int warp = threadIdx.x >> 5;
  const int i0 = (loc == LR) ? 1 : 0, j0 = (loc == LT) ? 1 : 0, k0 = (loc == LP) ? 1 : 0;
  const int ni = L.Nr - i0, nj = L.Nt - j0;
  // 32-bit index arithmetic: a shell's lines number far below 2^31
  const int line = bx * kScanWarps + warp;
  V acc = (V)0.0;
  double scale = 0.0;
  if (line < 2 * ni * nj) {
    const int j = j0 + line % nj;
    const int rest = line / nj;
    const int i = i0 + rest % ni, p = rest / ni;
    if ((patch_mask >> p) & 1) {
      const long q = lidx(L, p, i, j, 0);
      R *wbuf = (scan_pad(L.Np) <= smem_per_warp) ? smem + (long)warp * smem_per_warp : W + q;
      const long so = (long)line * scan_segs(L.Np);   // this line's lane-segment products (kSeg)
      switch (scan_ec(L.Np)) {
        case 4:
          solve_line_scan<4, kSum, kSeg>(k0, L.Np, final, Lo + q, Iv + q, Cp + q, B + q, wbuf, dst + q, acc,
                                                kSum ? Pn + q : nullptr, kSum ? Sout + q : nullptr,
                                                kSeg ? seg[0] + so : nullptr, kSeg ? seg[1] + so : nullptr);
          break;
        case 8:
          solve_line_scan<8, kSum, kSeg>(k0, L.Np, final, Lo + q, Iv + q, Cp + q, B + q, wbuf, dst + q, acc,
                                                kSum ? Pn + q : nullptr, kSum ? Sout + q : nullptr,
                                                kSeg ? seg[0] + so : nullptr, kSeg ? seg[1] + so : nullptr);
          break;
        default:
          solve_line_scan<12, kSum, kSeg>(k0, L.Np, final, Lo + q, Iv + q, Cp + q, B + q, wbuf, dst + q, acc,
                                                kSum ? Pn + q : nullptr, kSum ? Sout + q : nullptr,
                                                kSeg ? seg[0] + so : nullptr, kSeg ? seg[1] + so : nullptr);
          break;
      }
      if (final) {
        const double r = (loc == LR) ? S.nrf[i] : S.nrc[i];   // r sqrt(h / h_r)
        const double sn = (loc == LT) ? S.sf[j] : S.sc[j];
        scale = r * r * sn * S.dcs[CS_VOL];
      }
    }
  }
  if (final) norm_flush(acc, scale, &norm[slot]);
}



// Per-step factorisation of a phi line operator as a warp scan (one warp per
// line, lane t owning the same EC-position segment as in body_solve_phi_scan).
// The pivot recurrence c'_m = up_m / (di_m - lo_m c'_{m-1}) is the Moebius
// map of the matrix M_m = [[0, up_m], [-lo_m, di_m]] acting on (N, D) with
// c' = N / D, so segments compose as 2x2 matrix products; each lane composes
// its segment, an inclusive Kogge-Stone scan over the lanes composes the
// segments (matrices rescaled by exact powers of two to stay in range), and
// each lane replays its segment from the incoming c' with the exact divisions
// of the sequential elimination.  lo = 0 at the first unknown restarts the
// chain.  Outputs as body_factorize: Lo, Iv = 1 / pivot, Cp = c'.
template <typename V>
__device__ __forceinline__ V pow2_recip(V s);
template <>
__device__ __forceinline__ float pow2_recip<float>(float s) {
  int e = (__float_as_int(s) >> 23) & 0xff;
  e = e < 253 ? e : 253;
  return __int_as_float((254 - e) << 23);   // 2^(127 - e) ~ 1 / s, exact scaling
}
template <>
__device__ __forceinline__ double pow2_recip<double>(double s) {
  int e = (__double2hiint(s) >> 20) & 0x7ff;
  e = e < 2045 ? e : 2045;
  return __hiloint2double((2046 - e) << 20, 0);   // 2^(1023 - e)
}

template <typename V>
__device__ __forceinline__ void mat_rescale(V &a, V &b, V &c, V &d) {
  const V m = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(c), fabs(d)));
  if (m > (V)0.0) {
    const V f = pow2_recip(m);
    a *= f;
    b *= f;
    c *= f;
    d *= f;
  }
}

template <int EC, bool kTab, typename R>
__device__ __forceinline__ void factor_line_scan(const Shell &S, const StepAux<R> &ax, int loc, int i, int j,
                                                 long q, int k0, int k1, R *__restrict__ Lo, R *__restrict__ Iv,
                                                 R *__restrict__ Cp) {
  using V = typename Cmp<R>::type;
  const int lane = threadIdx.x & 31;
  constexpr int CH = 32 * EC;
  const int nch = (k1 + CH - 1) / CH;
  const V *fc = facc<V>(S, loc, DP, i, j);
  const V L0 = fc[FC_L0], D0 = fc[FC_D0], U0 = fc[FC_U0], LA = fc[FC_LA];
  V ccarry = (V)0.0;
  for (int c = 0; c < nch; ++c) {
    const int k = c * CH + lane * EC;
    const bool full = (k >= k0 && k + EC <= k1);
    // the row (i, j) is fixed along a phi line: lo = L0 + a La, di = D0,
    // up = U0 - a La (as coef), only the advecting velocity a varies
    V a[EC];
#pragma unroll
    for (int e = 0; e < EC; ++e) {
      const int kk = k + e;
      a[e] = (kk >= k0 && kk < k1) ? advecting<V, kTab>(S, ax, loc, DP, q + kk) : (V)0.0;
    }
    auto lo_of = [&](int e) -> V {
      const int kk = k + e;
      return (kk > k0 && kk < k1) ? L0 + a[e] * LA : (V)0.0;
    };
    auto up_of = [&](int e) -> V {
      const int kk = k + e;
      return (kk >= k0 && kk < k1 - 1) ? U0 - a[e] * LA : (V)0.0;
    };
    auto di_of = [&](int e) -> V {
      const int kk = k + e;
      return (kk >= k0 && kk < k1) ? D0 : (V)1.0;
    };
    // segment composite M_last ... M_first
    V A = (V)1.0, B = (V)0.0, C = (V)0.0, D = (V)1.0;
#pragma unroll
    for (int e = 0; e < EC; ++e) {
      const V lo = lo_of(e), di = di_of(e), up = up_of(e);
      const V nA = up * C, nB = up * D;
      const V nC = di * C - lo * A, nD = di * D - lo * B;
      A = nA;
      B = nB;
      C = nC;
      D = nD;
      if ((e & 3) == 3) mat_rescale(A, B, C, D);
    }
    mat_rescale(A, B, C, D);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const V Ao = __shfl_up_sync(0xffffffffu, A, off), Bo = __shfl_up_sync(0xffffffffu, B, off);
      const V Co = __shfl_up_sync(0xffffffffu, C, off), Do = __shfl_up_sync(0xffffffffu, D, off);
      if (lane >= off) {
        const V nA = A * Ao + B * Co, nB = A * Bo + B * Do;
        const V nC = C * Ao + D * Co, nD = C * Bo + D * Do;
        A = nA;
        B = nB;
        C = nC;
        D = nD;
        mat_rescale(A, B, C, D);
      }
    }
    V Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
    V Ce = __shfl_up_sync(0xffffffffu, C, 1), De = __shfl_up_sync(0xffffffffu, D, 1);
    if (lane == 0) {
      Ae = (V)1.0;
      Be = (V)0.0;
      Ce = (V)0.0;
      De = (V)1.0;
    }
    V cc = (Ae * ccarry + Be) / (Ce * ccarry + De);
    V oi[EC], oc[EC];
#pragma unroll
    for (int e = 0; e < EC; ++e) {
      const V inv = (V)1.0 / (di_of(e) - lo_of(e) * cc);
      cc = up_of(e) * inv;
      oi[e] = inv;
      oc[e] = cc;
    }
#pragma unroll
    for (int e = 0; e < EC; ++e) a[e] = lo_of(e);
    seg_store<EC>(Lo + q + k, full, k, k0, k1, a);
    seg_store<EC>(Iv + q + k, full, k, k0, k1, oi);
    seg_store<EC>(Cp + q + k, full, k, k0, k1, oc);
    ccarry = __shfl_sync(0xffffffffu, cc, 31);
  }
}

template <typename R, bool kTab = false>
__device__ __forceinline__ void body_factorize_phi_scan(Shell S, int loc, StepAux<R> ax, R *__restrict__ Lo,
                                                        R *__restrict__ Iv, R *__restrict__ Cp, int patch_mask,
                                                        int bx) {
  const Layout &L = S.L;
  const int warp = threadIdx.x >> 5;
  const int i0 = (loc == LR) ? 1 : 0, j0 = (loc == LT) ? 1 : 0, k0 = (loc == LP) ? 1 : 0;
  const int ni = L.Nr - i0, nj = L.Nt - j0;
  const int line = bx * kScanWarps + warp;
  if (line >= 2 * ni * nj) return;
  const int j = j0 + line % nj;
  const int rest = line / nj;
  const int i = i0 + rest % ni, p = rest / ni;
  if (!((patch_mask >> p) & 1)) return;
  const long q = lidx(L, p, i, j, 0);
  switch (scan_ec(L.Np)) {
    case 4:
      factor_line_scan<4, kTab>(S, ax, loc, i, j, q, k0, L.Np, Lo, Iv, Cp);
      break;
    case 8:
      factor_line_scan<8, kTab>(S, ax, loc, i, j, q, k0, L.Np, Lo, Iv, Cp);
      break;
    default:
      factor_line_scan<12, kTab>(S, ax, loc, i, j, q, k0, L.Np, Lo, Iv, Cp);
      break;
  }
}

}  // namespace bd
}  // namespace ys
