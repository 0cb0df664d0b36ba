// Batched tridiagonal line solves of the direction-split factors
// (I - dt/2 Ahat_d) (Sec. 3.2 modified operators, Eq. Convect_Douglas,
// Eq. r_comp / theta_comp / phi_comp; Thomas algorithm, Sec. 4).
//
// One thread owns one grid line.  For sweeps along r and theta the lines of a
// warp are neighbours along phi (the fastest index), so every load and store
// of the recurrence is coalesced.  The forward elimination keeps the modified
// super-diagonal c' in a scratch field Cs and overwrites the right-hand side
// with d'; back substitution overwrites d' with the solution, or, for the last
// factor of an unknown, adds it to the iterate and accumulates the FP64
// midpoint-rule norm of the increment (Sec. 5.1).
#include "kernels.cuh"

namespace ys {

namespace {

constexpr int TPB = 128;

template <typename R>
__device__ __forceinline__ double avg4(const R *a, long q1, long q2, long q3, long q4) {
  return (((double)a[q1] + (double)a[q2]) + (double)a[q3] + (double)a[q4]) / 4.0;
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
      ar = ((double)A0[q] + (double)A0[q + SI]) / 2.0;
      at = ((double)A1[q] + (double)A1[q + P]) / 2.0;
      ap = ((double)A2[q] + (double)A2[q + 1]) / 2.0;
      break;
    case LR:
      ar = (double)A0[q];
      at = avg4(A1, q - SI, q - SI + P, q, q + P);
      ap = avg4(A2, q - SI, q - SI + 1, q, q + 1);
      break;
    case LT:
      ar = avg4(A0, q - P, q - P + SI, q, q + SI);
      at = (double)A1[q];
      ap = avg4(A2, q - P, q - P + 1, q, q + 1);
      break;
    default:
      ar = avg4(A0, q - 1, q - 1 + SI, q, q + SI);
      at = avg4(A1, q - 1, q - 1 + P, q, q + P);
      ap = (double)A2[q];
      break;
  }
}

// Coefficients (lo, di, up) of (I - dt/2 Ahat_dir) at point (i, j, k) of `loc`.
template <typename R>
__device__ __forceinline__ void coef(const Shell &S, const StepAux<R> &ax, int loc, int dir, int i, int j, long q,
                                     double &lo, double &di, double &up) {
  const double hr = S.hr, ht = S.ht, hp = S.hp, R1 = S.R1;
  const double nu = (loc == LC) ? S.kappa : S.nu;
  double ar, at, ap;
  advecting(S, ax, loc, q, ar, at, ap);
  const double r = (loc == LR) ? S.rf[i] : S.rc[i];
  const double s = (loc == LT) ? S.sf[j] : S.sc[j];
  double cm, c0, cp;
  if (dir == DR) {
    double cp_d, cm_d;
    if (loc == LR) {
      cp_d = S.rc[i] * S.rc[i] / (r * r * hr * hr);
      cm_d = S.rc[i - 1] * S.rc[i - 1] / (r * r * hr * hr);
    } else {
      cp_d = S.rf[i + 1] * S.rf[i + 1] / (r * r * hr * hr);
      cm_d = S.rf[i] * S.rf[i] / (r * r * hr * hr);
    }
    cm = nu * cm_d + ar / (2 * hr);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - ar / (2 * hr);
    if (loc == LR) {
      cm = cm - nu * 2.0 * S.rf[i - 1] * S.rf[i - 1] / (r * r * r * 2 * hr);
      cp = cp + nu * 2.0 * S.rf[i + 1] * S.rf[i + 1] / (r * r * r * 2 * hr);
      c0 = c0 - nu * 2.0 / (r * r);
      const double k = 1.0 / (2 * S.chi);
      cm = cm + k * S.rf[i - 1] * S.rf[i - 1] / (S.rc[i - 1] * S.rc[i - 1] * hr * hr);
      c0 = c0 - k * (S.rf[i] * S.rf[i] / (S.rc[i] * S.rc[i] * hr * hr) +
                     S.rf[i] * S.rf[i] / (S.rc[i - 1] * S.rc[i - 1] * hr * hr));
      cp = cp + k * S.rf[i + 1] * S.rf[i + 1] / (S.rc[i] * S.rc[i] * hr * hr);
    }
  } else if (dir == DT) {
    double cp_d, cm_d;
    if (loc == LT) {
      cp_d = S.sc[j] / (R1 * R1 * s * ht * ht);
      cm_d = S.sc[j - 1] / (R1 * R1 * s * ht * ht);
    } else {
      cp_d = S.sf[j + 1] / (R1 * R1 * s * ht * ht);
      cm_d = S.sf[j] / (R1 * R1 * s * ht * ht);
    }
    cm = nu * cm_d + at / (2 * r * ht);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - at / (2 * r * ht);
    if (loc == LT) {
      const double c = S.cf[j];
      const double qq = 2.0 * c / (r * r * s * s) / (2 * ht);
      cm = cm - nu * qq * S.sf[j - 1];
      cp = cp + nu * qq * S.sf[j + 1];
      c0 = c0 - nu / (r * r * s * s);
      const double k = 1.0 / (2 * S.chi);
      cp = cp + k * S.sf[j + 1] / (r * r * S.sc[j] * ht * ht);
      c0 = c0 - k * (s / (r * r * S.sc[j] * ht * ht) + s / (r * r * S.sc[j - 1] * ht * ht));
      cm = cm + k * S.sf[j - 1] / (r * r * S.sc[j - 1] * ht * ht);
    }
  } else {
    const double s1 = S.sin_theta1;
    const double cpm = 1.0 / (R1 * R1 * s1 * s1 * hp * hp);
    cm = nu * cpm + ap / (2 * r * s * hp);
    c0 = -2.0 * nu * cpm;
    cp = nu * cpm - ap / (2 * r * s * hp);
    if (loc == LP) {
      c0 = c0 - nu / (r * r * s * s);
      const double k = 1.0 / (2 * S.chi);
      const double qq = k / (r * r * s * s * hp * hp);
      cm = cm + qq;
      c0 = c0 - 2.0 * qq;
      cp = cp + qq;
    }
  }
  lo = -0.5 * S.dt * cm;
  di = 1.0 - 0.5 * S.dt * c0;
  up = -0.5 * S.dt * cp;
}

template <typename R>
__global__ void k_sweep(Shell S, int loc, int dir, int final, StepAux<R> ax, R *B, R *Cs, R *dst, double *norm,
                        int slot, int patch_mask) {
  const Layout &L = S.L;
  // unknown ranges of loc
  const int i0 = (loc == LR) ? 1 : 0, i1 = L.Nr;
  const int j0 = (loc == LT) ? 1 : 0, j1 = L.Nt;
  const int k0 = (loc == LP) ? 1 : 0, k1 = L.Np;
  // line decode: x runs along the fastest index that is not the sweep direction
  int p, i = 0, j = 0, k = 0;
  int m0, m1;
  long step;
  int lane = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  bool valid;
  if (dir == DR) {
    k = k0 + lane;
    int nj = j1 - j0;
    j = j0 + row % nj;
    p = row / nj;
    valid = k < k1;
    m0 = i0;
    m1 = i1;
    step = L.SI;
    i = i0;
  } else if (dir == DT) {
    k = k0 + lane;
    int ni = i1 - i0;
    i = i0 + row % ni;
    p = row / ni;
    valid = k < k1;
    m0 = j0;
    m1 = j1;
    step = L.P;
    j = j0;
  } else {
    j = j0 + lane;
    int ni = i1 - i0;
    i = i0 + row % ni;
    p = row / ni;
    valid = j < j1;
    m0 = k0;
    m1 = k1;
    step = 1;
    k = k0;
  }
  double contrib = 0.0;
  if (valid && ((patch_mask >> p) & 1)) {
    const bool reflect = (dir == DR) && (loc != LR);
    const long qa = lidx(L, p, i, j, k);
    // forward elimination
    double cprev = 0.0, dprev = 0.0;
    long q = qa;
    for (int m = m0; m < m1; ++m, q += step) {
      int ii = (dir == DR) ? m : i, jj = (dir == DT) ? m : j;
      double lo, di, up;
      coef(S, ax, loc, dir, ii, jj, q, lo, di, up);
      if (m == m0) {
        if (reflect) di -= lo;
        lo = 0.0;
      }
      if (m == m1 - 1) {
        if (reflect) di -= up;
        up = 0.0;
      }
      double den = di - lo * cprev;
      double c = up / den;
      double d = ((double)B[q] - lo * dprev) / den;
      Cs[q] = (R)c;
      B[q] = (R)d;
      cprev = c;
      dprev = d;
    }
    // back substitution
    q -= step;
    double x = (double)B[q];
    for (int m = m1 - 1;; --m) {
      if (final) {
        dst[q] = (R)((double)dst[q] + x);
        int ii = (dir == DR) ? m : i, jj = (dir == DT) ? m : j;
        double r = (loc == LR) ? S.rf[ii] : S.rc[ii];
        double s = (loc == LT) ? S.sf[jj] : S.sc[jj];
        contrib += r * r * s * S.hr * S.ht * S.hp * x * x;
      } else {
        B[q] = (R)x;
      }
      if (m == m0) break;
      q -= step;
      x = (double)B[q] - (double)Cs[q] * x;
    }
  }
  if (final) {
    for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
    if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(&norm[slot], contrib);
  }
}

}  // namespace

template <typename R>
void Launch<R>::sweep(const Shell &S, int loc, int dir, bool final, StepAux<R> ax, R *B, R *Cs, R *dst,
                      double *norm, int slot, int patch_mask, cudaStream_t st) {
  const Layout &L = S.L;
  int ni = L.Nr - (loc == LR ? 1 : 0);
  int nj = L.Nt - (loc == LT ? 1 : 0);
  int nk = L.Np - (loc == LP ? 1 : 0);
  dim3 grid;
  if (dir == DR)
    grid = dim3((nk + TPB - 1) / TPB, 2 * nj);
  else if (dir == DT)
    grid = dim3((nk + TPB - 1) / TPB, 2 * ni);
  else
    grid = dim3((nj + TPB - 1) / TPB, 2 * ni);
  k_sweep<R><<<grid, TPB, 0, st>>>(S, loc, dir, final ? 1 : 0, ax, B, Cs, dst, norm, slot, patch_mask);
}

template void Launch<double>::sweep(const Shell &, int, int, bool, StepAux<double>, double *, double *, double *,
                                    double *, int, int, cudaStream_t);

}  // namespace ys
