// Batched tridiagonal line solves of the direction-split factors
// (I - dt/2 Ahat_d) (Sec. 3.2 modified operators, Eq. Convect_Douglas,
// Eq. r_comp / theta_comp / phi_comp; Thomas algorithm, Sec. 4).
//
// Every step first factorises each line operator once (lower diagonal,
// reciprocal pivots, modified super-diagonal c'), and every Schwarz iteration
// then solves with the stored factors.  Lines along r and theta: one thread
// per line, the lines of a warp neighbours along phi (the fastest index), so
// every load and store of the recurrences is coalesced.  Lines along phi
// (contiguous in memory): solves as warp scans (one warp per line, see
// body_solve_phi_scan); factorisation as a warp scan with FP32 storage
// (body_factorize_phi_scan) and, in FP64, where the FP64 pipe is the bound,
// one thread per line as along r and theta (lanes along theta).  The
// last factor of an unknown adds its solution to the iterate and accumulates
// the midpoint-rule norm of the increment (Sec. 5.1).
//
// k_sweep is the allocation-free variant (ys_factor_solve_static): one pass
// that forms the coefficients, eliminates and substitutes without stored
// factors.
#include <cmath>
#include <mutex>

#include "../../include/ys.h"
#include "bodies.cuh"

namespace ys {

namespace {

constexpr int TPB = 128;

// Coefficients (lo, di, up) of (I - dt/2 Ahat_dir) at point (i, j, k) of `loc`
// formed from the metric tables alone: the allocation-free entry point keeps
// no precomputed line-operator tables.  Same operator as the host tables of
// make_faccoef (diffusion with the modified theta / phi operators, the
// own-direction extras of the vector Laplacian and grad(div)/(2 chi), and the
// advection along dir).
template <typename V, typename R>
__device__ __forceinline__ void coef_metric(const Shell &S, const StepAux<R> &ax, int loc, int dir, int i, int j, long q,
                                     V &lo, V &di, V &up) {
  const V ihr = cs<V>(S, CS_IHR), iht = cs<V>(S, CS_IHT), ihp = cs<V>(S, CS_IHP);
  const V nu = (loc == LC) ? cs<V>(S, CS_KAPPA) : cs<V>(S, CS_NU);
  const V adv = bd::advecting<V>(S, ax, loc, dir, q);
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
    cm = nu * cm_d + adv * ((V)0.5 * ihr);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - adv * ((V)0.5 * ihr);
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
    cm = nu * cm_d + adv * ((V)0.5 * ir * iht);
    c0 = -nu * (cp_d + cm_d);
    cp = nu * cp_d - adv * ((V)0.5 * ir * iht);
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
    cm = nu * cpm + adv * ((V)0.5 * ir * is * ihp);
    c0 = (V)-2.0 * nu * cpm;
    cp = nu * cpm - adv * ((V)0.5 * ir * is * ihp);
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

template <typename R>
__global__ void k_sweep(Shell S, int loc, int dir, int final, StepAux<R> ax, R *B, R *Cs, R *dst, double *norm,
                        int slot, int patch_mask) {
  const Layout &L = S.L;
  const bd::Line ln = bd::decode_line(L, loc, dir, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
  const int m0 = ln.m0, m1 = ln.m1, i = ln.i, j = ln.j;
  const long step = ln.step;
  double contrib = 0.0;
  if (ln.valid && ((patch_mask >> ln.p) & 1)) {
    const bool reflect = (dir == DR) && (loc != LR);
    // forward elimination
    double cprev = 0.0, dprev = 0.0;
    long q = lidx(L, ln.p, ln.i, ln.j, ln.k);
    for (int m = m0; m < m1; ++m, q += step) {
      int ii = (dir == DR) ? m : i, jj = (dir == DT) ? m : j;
      double lo, di, up;
      coef_metric<double>(S, ax, loc, dir, ii, jj, q, lo, di, up);
      if (m == m0) {
        if (reflect) di += ((loc == LC) ? S.Tgam[0] : -1.0) * lo;
        lo = 0.0;
      }
      if (m == m1 - 1) {
        if (reflect) di += ((loc == LC) ? S.Tgam[1] : -1.0) * up;
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

// Per-step LU factorisation of one factor (I - dt/2 Ahat_dir) of `loc` on
// every line, in the storage type's arithmetic from the FP64 metric tables: the line matrices depend only on the advecting velocity, fixed
// for the whole step, so both AC systems and every Schwarz iteration reuse
// them.  Row m stores the sub-diagonal lo_m, the reciprocal pivot
// 1/(di_m - lo_m c'_{m-1}) and c'_m = up_m / pivot_m.
template <typename R>
__global__ void k_factorize(Shell S, int loc, int dir, StepAux<R> ax, R *Lo, R *Iv, R *Cp, int patch_mask) {
  bd::body_factorize<R, true>(S, loc, dir, ax, Lo, Iv, Cp, patch_mask, blockIdx.x, blockIdx.y);
}

// Thomas solve with a stored factorisation: forward d'_m = (b_m - lo_m d'_{m-1})
// / pivot_m, back x_m = d'_m - c'_m x_{m+1}.  Non-final factors leave x in B;
// the final factor of an unknown adds x to the iterate and accumulates the
// FP64 midpoint-rule norm of the increment (Sec. 5.1).
template <typename R>
__global__ void k_solve(Shell S, int loc, int dir, int final, const R *__restrict__ Lo, const R *__restrict__ Iv,
                        const R *__restrict__ Cp, R *B, R *W, R *dst, double *norm, int slot, int patch_mask) {
  bd::body_solve<R, true>(S, loc, dir, final, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, blockIdx.x, blockIdx.y);
}

// final factor of the FP64 form, also writing the two-level sum Sout = dst + Pn
__global__ void k_solve_sum(Shell S, int loc, int dir, const double *__restrict__ Lo,
                            const double *__restrict__ Iv, const double *__restrict__ Cp, double *B, double *W,
                            double *dst, double *norm, int slot, int patch_mask, const double *__restrict__ Pn,
                            double *__restrict__ Sout) {
  bd::body_solve<double, true, true>(S, loc, dir, 1, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, blockIdx.x,
                                     blockIdx.y, Pn, Sout);
}

dim3 line_grid(const Layout &L, int loc, int dir) {
  int ni = L.Nr - (loc == LR ? 1 : 0);
  int nj = L.Nt - (loc == LT ? 1 : 0);
  int nk = L.Np - (loc == LP ? 1 : 0);
  if (dir == DR) return dim3((nk + TPB - 1) / TPB, 2 * nj);
  if (dir == DT) return dim3((nk + TPB - 1) / TPB, 2 * ni);
  return dim3((nj + TPB - 1) / TPB, 2 * ni);
}

}  // namespace

template <typename R>
__global__ void k_factorize_phi(Shell S, int loc, StepAux<R> ax, R *Lo, R *Iv, R *Cp, int patch_mask) {
  bd::body_factorize_phi_scan<R, true>(S, loc, ax, Lo, Iv, Cp, patch_mask, blockIdx.x);
}

template <typename R>
__global__ void k_solve_phi(Shell S, int loc, int final, const R *__restrict__ Lo, const R *__restrict__ Iv,
                            const R *__restrict__ Cp, R *B, R *W, R *dst, double *norm, int slot, int patch_mask,
                            int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char phi_smem[];
  bd::body_solve_phi_scan(S, loc, final, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, blockIdx.x, (R *)phi_smem,
                          smem_per_warp);
}

// FP64 phi solves reading the per-step lane-segment products (k_phi_segments);
// the final ones also write the two-level sum Sout = dst + Pn
struct PhiSegs {
  const double *S[2];   // products of a (forward) and of g (backward)
};
__global__ void k_solve_phi_seg(Shell S, int loc, const double *__restrict__ Lo, const double *__restrict__ Iv,
                                const double *__restrict__ Cp, double *B, double *W, double *dst, double *norm,
                                int slot, int patch_mask, int smem_per_warp, PhiSegs sg) {
  extern __shared__ __align__(16) unsigned char phi_smem[];
  bd::body_solve_phi_scan<double, false, true>(S, loc, 0, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask,
                                               blockIdx.x, (double *)phi_smem, smem_per_warp, nullptr, nullptr,
                                               sg.S);
}

__global__ void k_solve_phi_sum(Shell S, int loc, const double *__restrict__ Lo, const double *__restrict__ Iv,
                                const double *__restrict__ Cp, double *B, double *W, double *dst, double *norm,
                                int slot, int patch_mask, int smem_per_warp, const double *__restrict__ Pn,
                                double *__restrict__ Sout, PhiSegs sg) {
  extern __shared__ __align__(16) unsigned char phi_smem[];
  bd::body_solve_phi_scan<double, true, true>(S, loc, 1, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, blockIdx.x,
                                              (double *)phi_smem, smem_per_warp, Pn, Sout, sg.S);
}

// the lane-segment products of the FP64 phi factor of `loc` (after k_factorize)
__global__ void k_phi_segments(Shell S, int loc, double *Lo, const double *Iv, const double *Cp, double *Aseg,
                               double *Gseg, int patch_mask) {
  bd::body_phi_segments<double>(S, loc, Lo, Iv, Cp, Aseg, Gseg, patch_mask, blockIdx.x);
}

template <typename R>
void Launch<R>::sweep(const Shell &S, int loc, int dir, bool final, StepAux<R> ax, R *B, R *Cs, R *dst,
                      double *norm, int slot, int patch_mask, cudaStream_t st) {
  k_sweep<R><<<line_grid(S.L, loc, dir), TPB, 0, st>>>(S, loc, dir, final ? 1 : 0, ax, B, Cs, dst, norm, slot,
                                                        patch_mask);
}

template <typename R>
void Launch<R>::factorize(const Shell &S, int loc, int dir, StepAux<R> ax, R *Lo, R *Iv, R *Cp, int patch_mask,
                          cudaStream_t st, R *const *seg) {
  if (dir == DP && bd::use_phi_scan<R>()) {
    k_factorize_phi<R><<<bd::phi_scan_ctas(S.L, loc), 32 * bd::kScanWarps, 0, st>>>(S, loc, ax, Lo, Iv, Cp,
                                                                                   patch_mask);
    return;
  }
  k_factorize<R><<<line_grid(S.L, loc, dir), TPB, 0, st>>>(S, loc, dir, ax, Lo, Iv, Cp, patch_mask);
  if constexpr (sizeof(R) == sizeof(double)) {
    if (dir == DP && seg)
      k_phi_segments<<<bd::phi_scan_ctas(S.L, loc), 32 * bd::kScanWarps, 0, st>>>(S, loc, Lo, Iv, Cp, seg[0], seg[1],
                                                                                  patch_mask);
  }
}

template <typename R>
void Launch<R>::solve(const Shell &S, int loc, int dir, bool final, const R *Lo, const R *Iv, const R *Cp, R *B,
                      R *W, R *dst, double *norm, int slot, int patch_mask, cudaStream_t st, const R *Pn,
                      R *Sout, R *const *seg) {
  // FP64 final factors given a sum field: the launches that also write it
  constexpr bool k64 = sizeof(R) == sizeof(double);
  const bool with_sum = k64 && final && Sout != nullptr;
  if (dir == DP) {
    // forward results of each warp's line in shared memory when they fit
    static std::atomic<unsigned long long> attr_done{0}, attr_sum_done{0}, attr_seg_done{0};
    smem_attr_once(attr_done, k_solve_phi<R>, bd::kScanSmemMax);
    const int pad = bd::scan_pad(S.L.Np);
    const size_t bytes = (size_t)bd::kScanWarps * pad * sizeof(R);
    const bool fits = bytes <= (size_t)bd::kScanSmemMax;
    if constexpr (k64) {
      // FP64 phi factors with lane-segment products (factorize given seg):
      // Lo holds a = -iv lo, so these factors take the segment solves only
      if (seg) {
        const PhiSegs sg{{seg[0], seg[1]}};
        if (with_sum) {
          smem_attr_once(attr_sum_done, k_solve_phi_sum, bd::kScanSmemMax);
          k_solve_phi_sum<<<bd::phi_scan_ctas(S.L, loc), 32 * bd::kScanWarps, fits ? bytes : 0, st>>>(
              S, loc, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, fits ? pad : 0, Pn, Sout, sg);
        } else {
          smem_attr_once(attr_seg_done, k_solve_phi_seg, bd::kScanSmemMax);
          k_solve_phi_seg<<<bd::phi_scan_ctas(S.L, loc), 32 * bd::kScanWarps, fits ? bytes : 0, st>>>(
              S, loc, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, fits ? pad : 0, sg);
        }
        return;
      }
    }
    k_solve_phi<R><<<bd::phi_scan_ctas(S.L, loc), 32 * bd::kScanWarps, fits ? bytes : 0, st>>>(
        S, loc, final ? 1 : 0, Lo, Iv, Cp, B, W, dst, norm, slot, patch_mask, fits ? pad : 0);
    return;
  }
  if constexpr (k64) {
    if (with_sum) {
      k_solve_sum<<<line_grid(S.L, loc, dir), TPB, 0, st>>>(S, loc, dir, Lo, Iv, Cp, B, W, dst, norm, slot,
                                                            patch_mask, Pn, Sout);
      return;
    }
  }
  k_solve<R><<<line_grid(S.L, loc, dir), TPB, 0, st>>>(S, loc, dir, final ? 1 : 0, Lo, Iv, Cp, B, W, dst, norm,
                                                        slot, patch_mask);
}

long phi_seg_elems(const Layout &L) { return bd::phi_seg_elems(L); }

#define YS_INST_SWEEP(R)                                                                                          \
  template void Launch<R>::factorize(const Shell &, int, int, StepAux<R>, R *, R *, R *, int, cudaStream_t,         \
                                     R *const *);                                                                  \
  template void Launch<R>::solve(const Shell &, int, int, bool, const R *, const R *, const R *, R *, R *, R *,       \
                                 double *, int, int, cudaStream_t, const R *, R *, R *const *);
YS_INST_SWEEP(double)
YS_INST_SWEEP(float)
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
constexpr long kStaticElems = 5 * kStaticFieldElems + (long)kMetricTables * kStaticMetricLen;
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

// The 14 metric tables of a uniform radial grid (r and 1/r at centres and
// faces, sin, cos and 1/sin at theta centres and faces, the radial cell
// width and its reciprocal, the norm factors r), each kStaticMetricLen long
// with `pad` entries before index 0, formed on the device so that a call
// queues no host-to-device copy.
__global__ void k_static_metric(double *met, double R1, double hr, double th0, double ht, int pad) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kStaticMetricLen; t += gridDim.x * blockDim.x) {
    const int i = t - pad;
    const double rc = R1 + (i + 0.5) * hr, rf = R1 + i * hr;
    const double sc = sin(th0 + (i + 0.5) * ht), sf = sin(th0 + i * ht);
    const double v[kMetricTables] = {rc,
                                     rf,
                                     sc,
                                     sf,
                                     cos(th0 + (i + 0.5) * ht),
                                     cos(th0 + i * ht),
                                     rc != 0.0 ? 1.0 / rc : 0.0,
                                     rf != 0.0 ? 1.0 / rf : 0.0,
                                     sc != 0.0 ? 1.0 / sc : 0.0,
                                     sf != 0.0 ? 1.0 / sf : 0.0,
                                     hr,
                                     1.0 / hr,
                                     rc,
                                     rf};
#pragma unroll
    for (int k = 0; k < kMetricTables; ++k) met[k * kStaticMetricLen + t] = v[k];
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
  if (prm->r_half) return YS_EINVAL;  // uniform radial grids only
  const double tb[4] = {prm->Tbc_inner_a, prm->Tbc_inner_b, prm->Tbc_outer_a, prm->Tbc_outer_b};
  for (int w = 0; w < 2; ++w)
    if (!(tb[2 * w] >= 0.0) || !(tb[2 * w + 1] >= 0.0) || !(tb[2 * w] + tb[2 * w + 1] > 0.0)) return YS_EINVAL;
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

  // Every call shares the scratch.  The padded copies of the advecting
  // velocity and of the right-hand side are cleared over this grid's extent
  // (the unpacks write the unknowns only; the rest of the box must read 0,
  // not the last call's values); c' is written before it is read.  The
  // metric tables are formed on the device: the call queues memsets and
  // kernels only, no copy from host memory.
  const int pad = 2;
  for (int f = 0; f < 4; ++f)
    if (cudaMemsetAsync(base + f * kStaticFieldElems, 0, L.total * sizeof(double), st) != cudaSuccess)
      return YS_ECUDA;
  k_static_metric<<<2, 256, 0, st>>>(met, prm->R1, hr, th0, ht, pad);
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
  S.irc = met + 6 * kStaticMetricLen + pad;
  S.irf = met + 7 * kStaticMetricLen + pad;
  S.isc = met + 8 * kStaticMetricLen + pad;
  S.isf = met + 9 * kStaticMetricLen + pad;
  S.hc = met + 10 * kStaticMetricLen + pad;
  S.ihc = met + 11 * kStaticMetricLen + pad;
  S.nrc = met + 12 * kStaticMetricLen + pad;
  S.nrf = met + 13 * kStaticMetricLen + pad;
  S.ihr = 1.0 / hr;
  S.iht = 1.0 / ht;
  S.ihp = 1.0 / hp;
  S.i2chi = 1.0 / (2.0 * prm->chi);
  S.iR1sq = 1.0 / (prm->R1 * prm->R1);
  S.cphi = 1.0 / (prm->R1 * prm->R1 * S.sin_theta1 * S.sin_theta1 * hp * hp);
  {
    // the temperature factor's wall rows follow the wall condition in prm
    const double a[2] = {prm->Tbc_inner_a, prm->Tbc_outer_a}, b[2] = {prm->Tbc_inner_b, prm->Tbc_outer_b};
    shell_set_T_walls(S, a, b, hr, hr);
  }
  shell_fill_fp64(S);
  StepAux<double> ax{};
  for (int a = 0; a < 3; ++a) ax.A[a] = Af[a];
  // factor order, first solved first: T r,theta,phi; u_r theta,phi,r;
  // u_theta phi,r,theta; u_phi r,theta,phi
  const int order[4][3] = {{DR, DT, DP}, {DT, DP, DR}, {DP, DR, DT}, {DR, DT, DP}};
  for (int s = 0; s < 3; ++s)
    Launch<double>::sweep(S, loc, order[loc][s], false, ax, B, Cs, nullptr, nullptr, 0, 3, st);
  k_static_pack<<<256, 256, 0, st>>>(L, loc, B, x);
  // a launch error of this call, or an error that earlier work left pending
  // in the caller's CUDA context, is returned as YS_ECUDA (and cleared)
  return cudaGetLastError() == cudaSuccess ? YS_OK : YS_ECUDA;
}
