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
#include <cmath>
#include <mutex>

#include "../../include/ys.h"
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

// ---------------------------------------------------------------------------
// Allocation-free factored solve: ys_factor_solve_static (include/ys.h).
//
// For callers that cannot allocate device memory.  All scratch (padded working
// copies of the inputs, the Thomas coefficients c' and the metric tables)
// lives in one file-scope __device__ array, g_static_scratch, sized for
// grids of at most kStaticFieldElems padded elements per field.  Every GPU
// that loads the library holds it until the process exits.
namespace {

constexpr long kStaticFieldElems = 1L << 18;  // padded elements of one field (both patches)
constexpr int kStaticMaxN = 256;              // cells along any direction
constexpr int kStaticMetricLen = kStaticMaxN + 8;
constexpr long kStaticElems = 5 * kStaticFieldElems + 6L * kStaticMetricLen;
constexpr int kMaxDevices = 64;

// [A_r | A_th | A_ph | B (rhs, then solution) | Cs (c')] padded fields, then the metric
__device__ __align__(256) double g_static_scratch[kStaticElems];

std::mutex g_static_mu;
double *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  The host-side
// name of the array is only a stand-in, so the address is looked up once per
// device with that device current and cached.
int static_scratch(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return YS_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return YS_ECUDA;
    }
    g_static_addr[dev] = (double *)ptr;
  }
  *out = g_static_addr[dev];
  return YS_OK;
}

__device__ __forceinline__ void static_extent(const Layout &L, int loc, int &ni, int &nj, int &nk) {
  ni = L.Nr + (loc == LR ? 1 : 0);
  nj = L.Nt + (loc == LT ? 1 : 0);
  nk = L.Np + (loc == LP ? 1 : 0);
}

// user layout (device) -> padded layout (static scratch)
__global__ void k_static_unpack(Layout L, int loc, const double *src, double *dst) {
  int ni, nj, nk;
  static_extent(L, loc, ni, nj, nk);
  long n = 2L * ni * nj * nk;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
    int k = (int)(u % nk);
    long t = u / nk;
    int j = (int)(t % nj);
    t /= nj;
    int i = (int)(t % ni);
    int p = (int)(t / ni);
    dst[lidx(L, p, i, j, k)] = src[u];
  }
}

// solution at the unknowns -> user layout (device); boundary entries get 0
__global__ void k_static_pack(Layout L, int loc, const double *src, double *dst) {
  int ni, nj, nk;
  static_extent(L, loc, ni, nj, nk);
  long n = 2L * ni * nj * nk;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
    int k = (int)(u % nk);
    long t = u / nk;
    int j = (int)(t % nj);
    t /= nj;
    int i = (int)(t % ni);
    int p = (int)(t / ni);
    bool boundary = (loc == LR && (i == 0 || i == L.Nr)) || (loc == LT && (j == 0 || j == L.Nt)) ||
                    (loc == LP && (k == 0 || k == L.Np));
    dst[u] = boundary ? 0.0 : src[lidx(L, p, i, j, k)];
  }
}

}  // namespace

}  // namespace ys

extern "C" int ys_factor_solve_static(const ys_params *prm, int loc, const double *A_r, const double *A_th,
                                      const double *A_ph, const double *rhs, double *x, void *stream) {
  using namespace ys;
  if (!prm || loc < LC || loc > LP || !A_r || !A_th || !A_ph || !rhs || !x) return YS_EINVAL;
  if (!(prm->R1 > 0.0) || !(prm->R2 > prm->R1) || !(prm->dt > 0.0) || !(prm->chi > 0.0) || !(prm->Pr > 0.0))
    return YS_EINVAL;
  if (prm->Nr < 8 || prm->Nth < 8 || prm->Nph < 8 || prm->overlap < 1) return YS_EINVAL;
  if (prm->Nr > kStaticMaxN || prm->Nth > kStaticMaxN || prm->Nph > kStaticMaxN) return YS_EINVAL;
  if (prm->Nth <= 2 * prm->overlap + 4) return YS_EINVAL;
  Layout L;
  L.Nr = prm->Nr;
  L.Nt = prm->Nth;
  L.Np = prm->Nph;
  L.NJ = prm->Nth + 2;
  L.P = ((prm->Nph + 2) + 7) / 8 * 8;
  L.SI = (long)L.NJ * L.P;
  long box = (long)(prm->Nr + 2) * L.SI + 16;
  L.PS = (box + 31) / 32 * 32;
  L.total = 2 * L.PS;
  if (L.total > kStaticFieldElems) return YS_EINVAL;  // larger than the static scratch
  const double pi = 3.14159265358979323846;
  const double hr = (prm->R2 - prm->R1) / prm->Nr;
  const double ht = (pi / 2) / (prm->Nth - 2 * prm->overlap);
  const double th0 = pi / 4 - prm->overlap * ht;
  const double hp = (1.5 * pi + 2 * prm->overlap * ht) / prm->Nph;
  if (!(th0 > 0.0)) return YS_EINVAL;

  double *base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double *Af[3] = {base, base + kStaticFieldElems, base + 2 * kStaticFieldElems};
  double *B = base + 3 * kStaticFieldElems;
  double *Cs = base + 4 * kStaticFieldElems;
  double *met = base + 5 * kStaticFieldElems;

  // metric tables r_c, r_f, sin/cos at theta centres and faces (pad 2), on the stack
  const int pad = 2;
  double mh[6 * kStaticMetricLen];
  for (int t = 0; t < kStaticMetricLen; ++t) {
    int i = t - pad;
    mh[0 * kStaticMetricLen + t] = prm->R1 + (i + 0.5) * hr;
    mh[1 * kStaticMetricLen + t] = prm->R1 + i * hr;
    mh[2 * kStaticMetricLen + t] = std::sin(th0 + (i + 0.5) * ht);
    mh[3 * kStaticMetricLen + t] = std::sin(th0 + i * ht);
    mh[4 * kStaticMetricLen + t] = std::cos(th0 + (i + 0.5) * ht);
    mh[5 * kStaticMetricLen + t] = std::cos(th0 + i * ht);
  }
  // every call shares the scratch: clear the working fields left by the last call
  if (cudaMemsetAsync(base, 0, 4 * kStaticFieldElems * sizeof(double), st) != cudaSuccess) return YS_ECUDA;
  if (cudaMemcpyAsync(met, mh, sizeof(mh), cudaMemcpyHostToDevice, st) != cudaSuccess) return YS_ECUDA;
  const double *Ain[3] = {A_r, A_th, A_ph};
  for (int a = 0; a < 3; ++a) k_static_unpack<<<256, 256, 0, st>>>(L, LR + a, Ain[a], Af[a]);
  k_static_unpack<<<256, 256, 0, st>>>(L, loc, rhs, B);

  Shell S{};
  S.L = L;
  S.hr = hr;
  S.ht = ht;
  S.hp = hp;
  S.R1 = prm->R1;
  S.sin_theta1 = std::sin(th0);
  S.dt = prm->dt;
  S.nu = prm->Pr;
  S.kappa = 1.0;
  S.chi = prm->chi;
  S.rc = met + 0 * kStaticMetricLen + pad;
  S.rf = met + 1 * kStaticMetricLen + pad;
  S.sc = met + 2 * kStaticMetricLen + pad;
  S.sf = met + 3 * kStaticMetricLen + pad;
  S.cc = met + 4 * kStaticMetricLen + pad;
  S.cf = met + 5 * kStaticMetricLen + pad;
  StepAux<double> ax{};
  for (int a = 0; a < 3; ++a) ax.A[a] = Af[a];
  // factor order, first solved first: T r,theta,phi; u_r theta,phi,r;
  // u_theta phi,r,theta; u_phi r,theta,phi
  const int order[4][3] = {{DR, DT, DP}, {DT, DP, DR}, {DP, DR, DT}, {DR, DT, DP}};
  for (int s = 0; s < 3; ++s)
    Launch<double>::sweep(S, loc, order[loc][s], false, ax, B, Cs, nullptr, nullptr, 0, 3, st);
  k_static_pack<<<256, 256, 0, st>>>(L, loc, B, x);
  return cudaGetLastError() == cudaSuccess ? YS_OK : YS_ECUDA;
}


