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
#include <type_traits>
#include "bodies.cuh"

namespace ys {

namespace {

constexpr int TPB = 128;

// ----------------------------------------------------------------- extrapolate
template <typename R>
__global__ void k_extrapolate(long total, State<R> it, State<R> n, State<R> nm1, R *A0, R *A1, R *A2) {
  const long chunk = 4096;
  for (long c = blockIdx.x; c * chunk < total; c += gridDim.x)
    bd::body_extrapolate(c * chunk, (c + 1) * chunk < total ? (c + 1) * chunk : total, it, n, nm1, A0, A1, A2);
}

// Per-step sums of the advecting velocity around every point location
// (StepAux::As): at cell centres the two faces of each component, at a face
// the four nearest stored values of each other component, added in the
// order the stencils and the line factors use, so that the tables hold the
// same values those kernels formed themselves.  Every element q in
// [SI, total - SI) is written (the regions of all locations lie inside it).
template <typename R>
__global__ void k_adv_sums(long lo, long hi, long SI, long P, const R *__restrict__ A0, const R *__restrict__ A1,
                           const R *__restrict__ A2, R *cr, R *ct, R *cp, R *rt, R *rp, R *tr, R *tp, R *pr, R *pt) {
  using V = typename Cmp<R>::type;
  for (long q = lo + blockIdx.x * (long)blockDim.x + threadIdx.x; q < hi; q += (long)gridDim.x * blockDim.x) {
    // every load before the first store (the outputs may alias the inputs as
    // far as the compiler knows)
    const V a0 = (V)A0[q], a1 = (V)A1[q], a2 = (V)A2[q];
    const V a0r = (V)A0[q + SI], a1t = (V)A1[q + P], a2p = (V)A2[q + 1];
    const V a1m = (V)A1[q - SI], a1mt = (V)A1[q - SI + P], a2m = (V)A2[q - SI], a2mp = (V)A2[q - SI + 1];
    const V a0t = (V)A0[q - P], a0tr = (V)A0[q - P + SI], a2t = (V)A2[q - P], a2tp = (V)A2[q - P + 1];
    const V a0p = (V)A0[q - 1], a0pr = (V)A0[q - 1 + SI], a1p = (V)A1[q - 1], a1pt = (V)A1[q - 1 + P];
    cr[q] = (R)(a0 + a0r);
    ct[q] = (R)(a1 + a1t);
    cp[q] = (R)(a2 + a2p);
    rt[q] = (R)(((a1m + a1mt) + a1) + a1t);
    rp[q] = (R)(((a2m + a2mp) + a2) + a2p);
    tr[q] = (R)(((a0t + a0tr) + a0) + a0r);
    tp[q] = (R)(((a2t + a2tp) + a2) + a2p);
    pr[q] = (R)(((a0p + a0pr) + a0) + a0r);
    pt[q] = (R)(((a1p + a1pt) + a1) + a1t);
  }
}

// sum over modes of tau_m(t) F_m, accumulated in the arithmetic type
template <typename R>
__global__ void k_combine(long total, Modes<R> M, R *o0, R *o1, R *o2, R *o3) {
  using V = typename Cmp<R>::type;
  long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long stride = (long)gridDim.x * blockDim.x;
  R *out[4] = {o0, o1, o2, o3};
  V tau[kMaxModes];
#pragma unroll
  for (int m = 0; m < kMaxModes; ++m) tau[m] = (m < M.n) ? (V)M.tau[m] : (V)0.0;
  for (; q < total; q += stride) {
    // every load before the first store (the outputs may alias the modes as
    // far as the compiler knows)
    V f[kMaxModes][4];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m)
#pragma unroll
      for (int c = 0; c < 4; ++c) f[m][c] = (m < M.n) ? (V)M.F[m][c][q] : (V)0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      V acc = (V)0.0;
#pragma unroll
      for (int m = 0; m < kMaxModes; ++m)
        if (m < M.n) acc = acc + tau[m] * f[m][c];
      out[c][q] = (R)acc;
    }
  }
}

// ----------------------------------------------------------------- residuals

// Points per thread along phi of a residual launch.  FP32 storage is bound by
// memory latency: several points per thread (the *_vec bodies, vector loads)
// put more bytes in flight per thread.  FP64 storage is bound by the FP64
// pipe and computes one point per thread with 10 CTAs of 128 threads per SM
// for the velocity rows (the register budget they take without a bound).
template <typename R>
__host__ __device__ constexpr int resid_nv() {
  return sizeof(R) == sizeof(float) ? 4 : 1;
}
constexpr int kResidVecTpb = 256;  // most threads per CTA of a vector launch
template <typename R>
struct ResidOcc {
  static constexpr int kTpb = resid_nv<R>() == 1 ? TPB : kResidVecTpb;
  static constexpr int kMinCtas = resid_nv<R>() == 1 ? 10 : 2;  // vector: at most 128 registers
  static constexpr int kTpbT = resid_nv<R>() == 1 ? 1024 : kResidVecTpb;  // 1024: no tighter bound than the default
};

template <typename R>
__global__ void __launch_bounds__(ResidOcc<R>::kTpbT)
    k_resid_T(Shell S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask, LevelSums<R> ls) {
  if constexpr (resid_nv<R>() == 1)
    bd::body_resid_T<R, true, true>(S, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y, ls.S[3]);
  else
    bd::body_resid_T_vec<R, resid_nv<R>()>(S, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------- residual u
template <typename R>
__global__ void __launch_bounds__(ResidOcc<R>::kTpb, ResidOcc<R>::kMinCtas)
    k_resid_ur(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask,
               LevelSums<R> ls) {
  if constexpr (resid_nv<R>() == 1)
    bd::body_resid_ur<R, true, true>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y, ls.S);
  else
    bd::body_resid_ur_vec<R, resid_nv<R>()>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(ResidOcc<R>::kTpb, ResidOcc<R>::kMinCtas)
    k_resid_ut(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask,
               LevelSums<R> ls) {
  if constexpr (resid_nv<R>() == 1)
    bd::body_resid_ut<R, true, true>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y, ls.S);
  else
    bd::body_resid_ut_vec<R, resid_nv<R>()>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(ResidOcc<R>::kTpb, ResidOcc<R>::kMinCtas)
    k_resid_up(Shell S, int sys, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask,
               LevelSums<R> ls) {
  if constexpr (resid_nv<R>() == 1)
    bd::body_resid_up<R, true, true>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y, ls.S);
  else
    bd::body_resid_up_vec<R, resid_nv<R>()>(S, sys, it, n, ax, B, patch_mask, blockIdx.x, blockIdx.y);
}

// ----------------------------------------------------------------- pressure
// FP64-accurate divergence and FP64 pressure accumulation in both forms.  One
// CTA per pres_rows<R>() consecutive cell rows: with FP32 storage the kernel
// is latency-bound and takes one row per CTA (the most CTAs in flight); in
// FP64 it is bound by the FP64 pipe and four rows per CTA amortise the norm
// reduction.  Each thread sums its cells' norm shares, the CTA reduces them
// once and writes part[block] without atomics, and k_sum_parts adds the
// shares up.
template <typename R>
__host__ __device__ constexpr int pres_rows() {
  return sizeof(R) == sizeof(float) ? 1 : 4;
}
template <typename R, bool kSum>
__device__ __forceinline__ void pressure_cta(const Shell &S, int sys, const State<R> &it, const State<R> &n,
                                             double *part, int rows, int patch_mask, const R *const *Sv) {
  using V = typename Cmp<R>::type;
  __shared__ V ws[TPB];
  V v = (V)0.0;
  for (int t = 0; t < pres_rows<R>(); ++t) {
    const int by = blockIdx.y * pres_rows<R>() + t;
    if (by < rows) v += bd::body_pressure<R, kSum>(S, sys, it, n, patch_mask, blockIdx.x, by, Sv);
  }
  ws[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    V w = ws[threadIdx.x];
    for (int u = threadIdx.x + 32; u < TPB; u += 32) w += ws[u];
    for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
    if (threadIdx.x == 0) part[(long)blockIdx.y * gridDim.x + blockIdx.x] = (double)w;
  }
}

template <typename R>
__global__ void k_pressure(Shell S, int sys, State<R> it, State<R> n, double *part, int rows, int patch_mask) {
  pressure_cta<R, false>(S, sys, it, n, part, rows, patch_mask, nullptr);
}

// the FP64 form, reading the two-level sums of the velocity (LevelSums)
__global__ void k_pressure_sum(Shell S, int sys, State<double> it, State<double> n, double *part, int rows,
                               int patch_mask, LevelSums<double> ls) {
  pressure_cta<double, true>(S, sys, it, n, part, rows, patch_mask, ls.S);
}

// dst += scale * sum(part[0, n)): CTAs take interleaved slices, one atomic each
constexpr int kSumCtas = 64;
__global__ void k_sum_parts(const double *part, long n, double scale, double *dst) {
  __shared__ double ws[8];
  double t = 0.0;
  for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) t += part[u];
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    if (s != 0.0) atomicAdd(dst, s * scale);
  }
}

// ----------------------------------------------------------------- packing
__device__ __forceinline__ void user_extent(const Layout &L, int loc, int &ni, int &nj, int &nk) {
  ni = L.Nr + (loc == LR ? 1 : 0);
  nj = L.Nt + (loc == LT ? 1 : 0);
  nk = L.Np + (loc == LP ? 1 : 0);
}

// user layout -> padded field(s); src may be device memory or mapped pinned
// host memory (read once, written to dst and, when given, dst2)
template <typename R>
__global__ void k_unpack(Layout L, int loc, const double *src, R *dst, const double *bg, R *dst2) {
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
    const long q = lidx(L, p, i, j, k);
    dst[q] = (R)v;
    if (dst2) dst2[q] = (R)v;
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

// grid and CTA size of a residual launch over the points of `loc`, nv points
// per thread: one CTA row per (patch, i, j) row, groups of nv along k from
// k = 0 (aligned) covering [k0, Np)
struct ResidLaunch {
  dim3 grid;
  int tpb;
};
ResidLaunch resid_launch(const Layout &L, int loc, int nv) {
  if (nv == 1) return {point_grid(L, loc), TPB};
  const int ni = L.Nr - (loc == LR ? 1 : 0);
  const int nj = L.Nt - (loc == LT ? 1 : 0);
  const int groups = (L.Np + nv - 1) / nv;
  int tpb = (groups + 31) / 32 * 32;
  if (tpb > kResidVecTpb) tpb = kResidVecTpb;
  return {dim3((groups + tpb - 1) / tpb, 2 * ni * nj), tpb};
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
void Launch<R>::adv_sums(const Layout &L, R *const A[3], R *const As[4][3], cudaStream_t st) {
  k_adv_sums<R><<<flat_blocks(L.total), 256, 0, st>>>(L.SI, L.total - L.SI, L.SI, L.P, A[0], A[1], A[2], As[LC][DR],
                                                       As[LC][DT], As[LC][DP], As[LR][DT], As[LR][DP], As[LT][DR],
                                                       As[LT][DP], As[LP][DR], As[LP][DT]);
}

template <typename R>
void Launch<R>::combine_forcing(long total, Modes<R> modes, R *out[4], cudaStream_t st) {
  k_combine<R><<<flat_blocks(total), 256, 0, st>>>(total, modes, out[0], out[1], out[2], out[3]);
}

template <typename R>
void Launch<R>::resid_T(const Shell &S, State<R> it, State<R> n, StepAux<R> ax, R *B, int pm, cudaStream_t st,
                        LevelSums<R> ls) {
  const ResidLaunch g = resid_launch(S.L, LC, resid_nv<R>());
  k_resid_T<R><<<g.grid, g.tpb, 0, st>>>(S, it, n, ax, B, pm, ls);
}

template <typename R>
void Launch<R>::resid_u(const Shell &S, int sys, int comp, State<R> it, State<R> n, StepAux<R> ax, R *B, int pm,
                        cudaStream_t st, LevelSums<R> ls) {
  const ResidLaunch g = resid_launch(S.L, LR + comp, resid_nv<R>());
  if (comp == 0)
    k_resid_ur<R><<<g.grid, g.tpb, 0, st>>>(S, sys, it, n, ax, B, pm, ls);
  else if (comp == 1)
    k_resid_ut<R><<<g.grid, g.tpb, 0, st>>>(S, sys, it, n, ax, B, pm, ls);
  else
    k_resid_up<R><<<g.grid, g.tpb, 0, st>>>(S, sys, it, n, ax, B, pm, ls);
}

// s[f] = a[f] + b[f] elementwise over whole fields (16-byte accesses; a
// field's length is a multiple of 32 elements and its start 256-byte aligned)
template <typename R>
__global__ void k_sum_levels(long total, SumJob<R> job) {
  constexpr int W = 16 / sizeof(R);
  using Vec = typename std::conditional<sizeof(R) == 8, double2, float4>::type;
  const long nv = total / W;
  for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!job.s[f]) continue;
      const Vec x = reinterpret_cast<const Vec *>(job.a[f])[v], y = reinterpret_cast<const Vec *>(job.b[f])[v];
      Vec z;
      if constexpr (sizeof(R) == 8) {
        z.x = x.x + y.x;
        z.y = x.y + y.y;
      } else {
        z.x = x.x + y.x;
        z.y = x.y + y.y;
        z.z = x.z + y.z;
        z.w = x.w + y.w;
      }
      reinterpret_cast<Vec *>(job.s[f])[v] = z;
    }
  }
}

template <typename R>
void Launch<R>::sum_levels(const Layout &L, SumJob<R> job, cudaStream_t st) {
  k_sum_levels<R><<<152 * 8, 256, 0, st>>>(L.total, job);
}

// P2 = p2n + (p1 - p1n) / 2, the expression of the momentum rows' pressure
__global__ void k_bootstrap_pressure(long total, const double *p2n, const double *p1, const double *p1n,
                                     double *P2) {
  const long nv = total / 2;
  for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long)gridDim.x * blockDim.x) {
    const double2 a = reinterpret_cast<const double2 *>(p2n)[v], b = reinterpret_cast<const double2 *>(p1)[v],
                  c = reinterpret_cast<const double2 *>(p1n)[v];
    double2 o;
    o.x = a.x + 0.5 * (b.x - c.x);
    o.y = a.y + 0.5 * (b.y - c.y);
    reinterpret_cast<double2 *>(P2)[v] = o;
  }
}

template <typename R>
void Launch<R>::bootstrap_pressure(const Layout &L, const double *p2n, const double *p1, const double *p1n,
                                   double *P2, cudaStream_t st) {
  k_bootstrap_pressure<<<152 * 8, 256, 0, st>>>(L.total, p2n, p1, p1n, P2);
}

template <typename R>
void Launch<R>::pressure(const Shell &S, int sys, State<R> it, State<R> n, double *norm, double *part, int pm,
                         cudaStream_t st, LevelSums<R> ls) {
  const dim3 g = point_grid(S.L, LC);
  const dim3 gp(g.x, (g.y + pres_rows<R>() - 1) / pres_rows<R>());
  if constexpr (sizeof(R) == sizeof(double))
    k_pressure_sum<<<gp, TPB, 0, st>>>(S, sys, it, n, part, (int)g.y, pm, ls);
  else
    k_pressure<R><<<gp, TPB, 0, st>>>(S, sys, it, n, part, (int)g.y, pm);
  k_sum_parts<<<kSumCtas, 256, 0, st>>>(part, (long)gp.x * gp.y, S.dcs[CS_VOL], &norm[sys == 1 ? 4 : 8]);
}

template <typename R>
void Launch<R>::unpack(const Layout &L, int loc, const double *src, R *dst, const double *bg, cudaStream_t st,
                       R *dst2) {
  k_unpack<R><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, loc, src, dst, bg, dst2);
}

template <typename R>
void Launch<R>::pack(const Layout &L, int loc, const R *src, double *dst, const double *bg, cudaStream_t st) {
  k_pack<R><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, loc, src, dst, bg);
}

void unpack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st, double *dst2) {
  k_unpack<double><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, LC, src, dst, bg, dst2);
}

void pack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st) {
  k_pack<double><<<flat_blocks(user_max(L)), 256, 0, st>>>(L, LC, src, dst, bg);
}

// One iteration's divergence test (one thread): norm[0..NF) hold the squared
// increment norms of iteration k (1-based) of the step just finished
// (non-negative sums); `prev` holds the largest of iteration k - 1, `flag`
// the sticky flag.
__global__ void k_norm_watch(const double *norm, double *prev, double *first, double *flag, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double cur = 0.0;
  bool bad = false;
  for (int f = 0; f < NF; ++f) {
    const double v = norm[f];
    if (!(v <= 1.79e308)) bad = true;   // NaN or +Inf
    else cur = fmax(cur, v);
  }
  if (k == 1) *first = cur;
  if (k >= 3 && cur > kWatchGrowth * kWatchGrowth * *prev && cur > *first) bad = true;
  if (bad) *flag = 1.0;
  *prev = cur;
}

void norm_watch(double *norm, int k, cudaStream_t st) {
  k_norm_watch<<<1, 32, 0, st>>>(norm, norm + kWatchPrev, norm + kWatchFirst, norm + kWatchFlag, k);
}

#define YS_INST_STENCIL(R)                                                                                         \
  template void Launch<R>::extrapolate(const Layout &, State<R>, State<R>, State<R>, R *[3], cudaStream_t);       \
  template void Launch<R>::combine_forcing(long, Modes<R>, R *[4], cudaStream_t);                                  \
  template void Launch<R>::adv_sums(const Layout &, R *const[3], R *const[4][3], cudaStream_t);                   \
  template void Launch<R>::resid_T(const Shell &, State<R>, State<R>, StepAux<R>, R *, int, cudaStream_t,         \
                                   LevelSums<R>);                                                                  \
  template void Launch<R>::resid_u(const Shell &, int, int, State<R>, State<R>, StepAux<R>, R *, int,             \
                                   cudaStream_t, LevelSums<R>);                                                    \
  template void Launch<R>::sum_levels(const Layout &, SumJob<R>, cudaStream_t);                                   \
  template void Launch<R>::bootstrap_pressure(const Layout &, const double *, const double *, const double *,       \
                                              double *, cudaStream_t);                                             \
  template void Launch<R>::pressure(const Shell &, int, State<R>, State<R>, double *, double *, int, cudaStream_t,  \
                                    LevelSums<R>);                                                                 \
  template void Launch<R>::unpack(const Layout &, int, const double *, R *, const double *, cudaStream_t, R *);   \
  template void Launch<R>::pack(const Layout &, int, const R *, double *, const double *, cudaStream_t);
YS_INST_STENCIL(double)
YS_INST_STENCIL(float)

}  // namespace ys
