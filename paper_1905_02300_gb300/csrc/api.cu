// C ABI of the solver: context lifetime, field I/O and the AC time step
// (Sec. 3.3 artificial compressibility with bootstrapping, Sec. 4 Schwarz
// iteration with splitting-error reduction, Eq. er).
//
// Two storage forms share one code path, templated on the bulk type R:
//   YS_FP64  : every field FP64;
//   YS_MIXED : T, u1, u2 FP32 (stencils and sweeps in FP32), pressures FP64,
//              line coefficients factored in FP64, norms FP64.  The mixed form
//              stores the deviations T - T_c and p - p_c from the discrete
//              conductive profile T_c (walls T_inner, T_outer) and its discrete
//              hydrostatic pressure p_c, so that FP32 only carries the
//              perturbation; T_c's discrete Laplacian and radial derivative
//              enter the temperature rate as FP64 tables.  This is an exact
//              rewrite of the same discrete equations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ys.h"
#include "ctx.h"

using namespace ys;

namespace {

const char *kClassNames[K_NUM] = {"extrapolate", "forcing",  "exchange", "walls",   "ring",     "resid_T",
                                  "resid_u",     "sweep_r",  "sweep_t",  "sweep_p", "pressure", "pack",
                                  "factorize",   "watch",    "sums"};

}  // namespace

namespace {

template <typename R>
Fields<R> &F(ys_ctx *c);
template <>
Fields<double> &F<double>(ys_ctx *c) {
  return *c->f64;
}
template <>
Fields<float> &F<float>(ys_ctx *c) {
  return *c->f32;
}

inline int cuda_ok(cudaError_t e) { return e == cudaSuccess ? YS_OK : YS_ECUDA; }

void prof_begin(ys_ctx *c, int cls) {
  if (!c->prof_on) return;
  if (c->prof_used == c->prof.size()) {
    ProfRec r{cls, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    c->prof.push_back(r);
  }
  ProfRec &r = c->prof[c->prof_used];
  r.cls = cls;
  cudaEventRecord(r.a, c->stream);
}

void prof_end(ys_ctx *c, int nk) {
  c->launches += nk;
  if (!c->prof_on) return;
  cudaEventRecord(c->prof[c->prof_used].b, c->stream);
  c->prof_used++;
}

#define LAUNCH(ctx, cls, nk, expr) \
  do {                             \
    prof_begin(ctx, cls);          \
    expr;                          \
    prof_end(ctx, nk);             \
  } while (0)

// FP64 rate probe (ys_measure_fp64_rate): kRateChains independent FMA
// chains per thread, so that each warp always has a ready FP64 instruction;
// the conditional store keeps the chains live.
constexpr int kRateChains = 8, kRateThreads = 256, kRateBlocksPerSM = 8;
__global__ void __launch_bounds__(kRateThreads) k_fp64_rate(double *sink, double seed, int iters) {
  double a[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double b = 0.999999999, d = 1e-9;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += a[c];
  if (s == -1.0) *sink = s;
}

int validate(const ys_params *p) {
  if (!p) return YS_EINVAL;
  if (!(p->R1 > 0.0) || !(p->R2 > p->R1) || !(p->dt > 0.0)) return YS_EINVAL;
  if (p->Nr < 8 || p->Nth < 8 || p->Nph < 8 || p->Nph < p->Nth) return YS_EINVAL;
  if (!(p->chi > 0.0) || p->overlap < 1) return YS_EINVAL;
  if (p->precision != YS_FP64 && p->precision != YS_MIXED) return YS_EINVAL;
  if (p->schwarz_mode != YS_ADDITIVE && p->schwarz_mode != YS_MULTIPLICATIVE) return YS_EINVAL;
  if (!(p->Pr > 0.0) || !(p->Ra >= 0.0) || !(p->schwarz_tol >= 0.0)) return YS_EINVAL;
  if (p->step4 && (!(p->step4_eps > 0.0) || !(p->step4_tol >= 0.0))) return YS_EINVAL;
  const double tb[4] = {p->Tbc_inner_a, p->Tbc_inner_b, p->Tbc_outer_a, p->Tbc_outer_b};
  for (int w = 0; w < 2; ++w)
    if (!(tb[2 * w] >= 0.0) || !(tb[2 * w + 1] >= 0.0) || !(tb[2 * w] + tb[2 * w + 1] > 0.0)) return YS_EINVAL;
  return YS_OK;
}

size_t user_elems(const Layout &L, int loc) {
  return 2ul * (L.Nr + (loc == LR)) * (L.Nt + (loc == LT)) * (L.Np + (loc == LP));
}

// Device address of a user host buffer that kernels may access directly:
// page-locked (pinned or registered) host memory mapped into the device's
// address space; null for pageable memory (which goes through the staging
// buffer).  Over the CPU-GPU link such a buffer is read or written by the
// (un)pack kernel itself, in one pass instead of a copy plus a kernel.
const void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

// source of an unpack: device memory as is, mapped host memory directly, else
// a host-to-device copy into the staging buffer
int unpack_source(ys_ctx *c, const double *src, size_t n, bool device_src, const double **from) {
  if (device_src) {
    *from = src;
    return YS_OK;
  }
  if (const void *m = mapped_host(src)) {
    *from = (const double *)m;
    return YS_OK;
  }
  if (cudaMemcpyAsync(c->stage, src, n * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return YS_ECUDA;
  *from = c->stage;
  return YS_OK;
}

// user array -> padded field(s), unpacked into dst and, when dst2 is given,
// into dst2 from the same read (the two velocity systems and the two
// pressures start from the same values)
template <typename R>
int copy_in(ys_ctx *c, int loc, const double *src, R *dst, const double *bg, bool device_src, R *dst2 = nullptr) {
  const double *from = nullptr;
  if (int rc = unpack_source(c, src, user_elems(c->L, loc), device_src, &from)) return rc;
  LAUNCH(c, K_PACK, 1, Launch<R>::unpack(c->L, loc, from, dst, bg, c->stream, dst2));
  return YS_OK;
}

int copy_in_p(ys_ctx *c, const double *src, double *dst, bool device_src, double *dst2 = nullptr) {
  const double *from = nullptr;
  if (int rc = unpack_source(c, src, user_elems(c->L, LC), device_src, &from)) return rc;
  LAUNCH(c, K_PACK, 1, unpack_p(c->L, from, dst, c->p_bg, c->stream, dst2));
  return YS_OK;
}

// padded field -> user array: packed straight into mapped host memory, else
// through the staging buffer and a device-to-host copy; queued on the
// context's stream (the staging buffer is reused in stream order), the caller
// synchronises once after the last field
template <typename R>
int copy_out(ys_ctx *c, int loc, const R *src, double *dst, const double *bg) {
  size_t n = user_elems(c->L, loc);
  if (void *m = const_cast<void *>(mapped_host(dst))) {
    LAUNCH(c, K_PACK, 1, Launch<R>::pack(c->L, loc, src, (double *)m, bg, c->stream));
    return YS_OK;
  }
  LAUNCH(c, K_PACK, 1, Launch<R>::pack(c->L, loc, src, c->stage, bg, c->stream));
  cudaError_t e = cudaMemcpyAsync(dst, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  return e == cudaSuccess ? YS_OK : YS_ECUDA;
}

int copy_out_p(ys_ctx *c, const double *src, double *dst) {
  size_t n = user_elems(c->L, LC);
  if (void *m = const_cast<void *>(mapped_host(dst))) {
    LAUNCH(c, K_PACK, 1, pack_p(c->L, src, (double *)m, c->p_bg, c->stream));
    return YS_OK;
  }
  LAUNCH(c, K_PACK, 1, pack_p(c->L, src, c->stage, c->p_bg, c->stream));
  cudaError_t e = cudaMemcpyAsync(dst, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  return e == cudaSuccess ? YS_OK : YS_ECUDA;
}

// time function id of separable forcing and wall modes
double time_fn(int id, double t) {
  switch (id) {
    case 0: return 1.0;
    case 1: return std::cos(t);
    case 2: return std::sin(t);
    case 3: return std::cos(t) * std::cos(t);
    case 4: return std::sin(t) * std::cos(t);
  }
  return 0.0;
}

// exchange + walls (+ pressure ring) of a whole state: boundary values as
// functions of the interior; t: the time of the state (time-dependent wall data)
template <typename R>
void exchange_walls(ys_ctx *c, State<R> s, int mask, double t) {
  WallData wt = c->wall_t;
  wt.tau = time_fn(c->wall_tfn, t);
  LAUNCH(c, K_EXCH, 4, Launch<R>::exchange(c->S, c->X, s, mask, c->stream));
  LAUNCH(c, K_WALLS, 1, Launch<R>::walls(c->S, wt, s, mask, c->stream));
  if (c->prm.step4)
    LAUNCH(c, K_EXCH, 2,
           Launch<R>::mass_flux(c->S, s, mask, c->norm + 16, c->s4_alpha, c->s4_wsq,
                                c->s4_cwall[0] + wt.tau * c->s4_cwall_t[0],
                                c->s4_cwall[1] + wt.tau * c->s4_cwall_t[1], c->prm.step4_tol, c->stream));
}

template <typename R>
void refresh(ys_ctx *c, State<R> s, int mask, double t) {
  exchange_walls<R>(c, s, mask, t);
  if (c->prm.step7) LAUNCH(c, K_RING, 1, Launch<R>::ring(c->S, c->X, s, mask, c->stream));
}

const int kOrder[4][3] = {
    {DR, DT, DP},  // T (LC): r, theta, phi
    {DT, DP, DR},  // u_r: theta, phi, r
    {DP, DR, DT},  // u_theta: phi, r, theta
    {DR, DT, DP},  // u_phi: r, theta, phi
};
const int kSweepClass[3] = {K_SWEEP_R, K_SWEEP_T, K_SWEEP_P};

template <typename R>
void solve_unknown(ys_ctx *c, int loc, int slot, int mask) {
  Fields<R> &D = F<R>(c);
  State<R> &it = D.lev[2], &n = D.lev[0];
  // FP64: the final factor also refreshes the unknown's two-level sum
  // (LevelSums: velocity component loc - LR, or T)
  R *sum = D.Sv[0] ? D.Sv[loc == LC ? 3 : loc - LR] : nullptr;
  for (int s = 0; s < 3; ++s) {
    int dir = kOrder[loc][s];
    bool fin = (s == 2);
    R *const *Fc = D.fac[loc][dir];
    R *const *sg = (dir == DP && D.seg[loc][0]) ? D.seg[loc] : nullptr;
    LAUNCH(c, kSweepClass[dir], 1,
           Launch<R>::solve(c->S, loc, dir, fin, Fc[0], Fc[1], Fc[2], D.B, D.Cs, it.f[slot], c->norm, slot, mask,
                            c->stream, fin ? n.f[slot] : nullptr, fin ? sum : nullptr, sg));
  }
}

// LU factors of every line operator for this step (they depend only on a)
template <typename R>
void factorize_all(ys_ctx *c, StepAux<R> ax) {
  Fields<R> &D = F<R>(c);
  for (int loc = LC; loc <= LP; ++loc)
    for (int dir = DR; dir <= DP; ++dir) {
      R *const *Fc = D.fac[loc][dir];
      // FP64 phi factors also get their lane-segment products (D.seg)
      R *const *sg = (dir == DP && D.seg[loc][0]) ? D.seg[loc] : nullptr;
      LAUNCH(c, K_FACTOR, sg ? 2 : 1, Launch<R>::factorize(c->S, loc, dir, ax, Fc[0], Fc[1], Fc[2], 3, c->stream, sg));
    }
}

// boundary values of both stored levels from their interiors
template <typename R>
void refresh_levels(ys_ctx *c) {
  Fields<R> &D = F<R>(c);
  refresh<R>(c, D.lev[0], 3, c->t);
  refresh<R>(c, D.lev[1], 3, c->t - c->prm.dt);
}

// one defect-correction pass over T, u1, p1, u2, p2 on the masked patches
template <typename R>
void iterate(ys_ctx *c, StepAux<R> ax, int mask) {
  Fields<R> &D = F<R>(c);
  State<R> &it = D.lev[2], &n = D.lev[0];
  // FP64: residuals and pressure updates read two-level sums S = psi + psi^n
  // (LevelSums), formed by whole-field passes (T's after the exchange, a
  // velocity system's three components before its first residual) and
  // refreshed by the final solve of each unknown, which changes it
  const bool sums = D.Sv[0] != nullptr;
  // S[4]: the momentum pressure, p1^n itself for system 1, the field P2
  // (formed after the first pressure update) for system 2
  const LevelSums<R> lsys[2] = {{{D.Sv[0], D.Sv[1], D.Sv[2], D.Sv[3], (const R *)n.p[0]}},
                                {{D.Sv[0], D.Sv[1], D.Sv[2], D.Sv[3], D.Sv[4]}}};
  const LevelSums<R> &ls = lsys[0];
  auto sum = [&](int sys, int comp_mask, bool with_T) {
    SumJob<R> job{};
    const int o = (sys == 1) ? F_U1R : F_U2R;
    for (int f = 0; f < 3; ++f)
      if ((comp_mask >> f) & 1) {
        job.a[f] = it.f[o + f];
        job.b[f] = n.f[o + f];
        job.s[f] = D.Sv[f];
      }
    if (with_T) {
      job.a[3] = it.f[F_T];
      job.b[3] = n.f[F_T];
      job.s[3] = D.Sv[3];
    }
    LAUNCH(c, K_SUMS, 1, Launch<R>::sum_levels(c->L, job, c->stream));
  };
  if (sums) sum(1, 0, true);
  LAUNCH(c, K_RES_T, 1, Launch<R>::resid_T(c->S, it, n, ax, D.B, mask, c->stream, ls));
  solve_unknown<R>(c, LC, F_T, mask);
  for (int sys = 1; sys <= 2; ++sys) {
    int o = (sys == 1) ? 0 : 4;
    if (sums) sum(sys, 7, false);
    for (int comp = 0; comp < 3; ++comp) {
      LAUNCH(c, K_RES_U, 1, Launch<R>::resid_u(c->S, sys, comp, it, n, ax, D.B, mask, c->stream, lsys[sys - 1]));
      solve_unknown<R>(c, LR + comp, F_U1R + comp + o, mask);
    }
    LAUNCH(c, K_PRES, 2, Launch<R>::pressure(c->S, sys, it, n, c->norm, c->stage, mask, c->stream, ls));
    if (sums && sys == 1)
      LAUNCH(c, K_SUMS, 1,
             Launch<R>::bootstrap_pressure(c->L, n.p[1], it.p[0], n.p[0], (double *)D.Sv[4], c->stream));
  }
}


template <typename R>
int step_t(ys_ctx *c, int n_steps, int n_schwarz) {
  const ys_params &prm = c->prm;
  Fields<R> &D = F<R>(c);
  // the divergence watch reports on this call's iterations only
  cudaMemsetAsync(c->norm + kWatchFlag, 0, sizeof(double), c->stream);
  for (int st = 0; st < n_steps; ++st) {
    State<R> n = D.lev[0], nm1 = D.lev[1], it = D.lev[2];
    LAUNCH(c, K_EXTRAP, 1, Launch<R>::extrapolate(c->L, it, n, nm1, D.A, c->stream));
    LAUNCH(c, K_EXTRAP, 1, Launch<R>::adv_sums(c->L, D.A, D.As, c->stream));
    StepAux<R> ax{};
    for (int a = 0; a < 3; ++a) ax.A[a] = D.A[a];
    for (int loc = 0; loc < 4; ++loc)
      for (int dir = 0; dir < 3; ++dir) ax.As[loc][dir] = D.As[loc][dir];
    ax.fT = ax.fr = ax.ft = ax.fp = nullptr;
    if (c->nmodes_set > 0) {
      // pointers and time weights of the modes at t_n + dt/2, passed by value
      Modes<R> md{};
      for (int m = 0; m < c->nmodes_set; ++m) {
        if (!c->mode_set[m]) continue;
        for (int a = 0; a < 4; ++a) md.F[md.n][a] = D.modes[m][a];
        md.tau[md.n] = time_fn(c->mode_fn[m], c->t + 0.5 * prm.dt);
        ++md.n;
      }
      LAUNCH(c, K_FORCE, 1, Launch<R>::combine_forcing(c->L.total, md, D.fcomb, c->stream));
      ax.fT = D.fcomb[0];
      ax.fr = D.fcomb[1];
      ax.ft = D.fcomb[2];
      ax.fp = D.fcomb[3];
    }
    factorize_all<R>(c, ax);
    c->iters_last = 0;
    for (int k = 1; k <= n_schwarz; ++k) {
      cudaMemsetAsync(c->norm, 0, YS_NFIELDS * sizeof(double), c->stream);
      if (prm.schwarz_mode == YS_ADDITIVE) {
        exchange_walls<R>(c, it, 3, c->t + prm.dt);
        iterate<R>(c, ax, 3);
        if (prm.step7) LAUNCH(c, K_RING, 1, Launch<R>::ring(c->S, c->X, it, 3, c->stream));
      } else {
        for (int p = 0; p < 2; ++p) {
          int m = 1 << p;
          exchange_walls<R>(c, it, m, c->t + prm.dt);
          iterate<R>(c, ax, m);
          if (prm.step7) LAUNCH(c, K_RING, 1, Launch<R>::ring(c->S, c->X, it, m, c->stream));
        }
      }
      c->iters_last = k;
      LAUNCH(c, K_WATCH, 1, norm_watch(c->norm, k, c->stream));
      if (prm.schwarz_tol > 0.0) {
        double h[YS_NFIELDS];
        if (cudaMemcpyAsync(h, c->norm, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
          return YS_ECUDA;
        double mx = 0.0;
        for (int f = 0; f < YS_NFIELDS; ++f) mx = std::fmax(mx, std::sqrt(h[f]));
        if (mx < prm.schwarz_tol) break;
      }
    }
    refresh<R>(c, it, 3, c->t + prm.dt);
    // rotate time levels: n-1 <- n, n <- iterate, iterate <- old n-1
    D.lev[0] = it;
    D.lev[1] = n;
    D.lev[2] = nm1;
    c->t += prm.dt;
    c->steps_done++;
  }
  if (cudaGetLastError() != cudaSuccess) return YS_ECUDA;
  if (n_steps > 0) {
    double h[kWatchFlag + 1];
    if (cudaMemcpyAsync(h, c->norm, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return YS_ECUDA;
    bool bad = h[kWatchFlag] != 0.0;
    for (int f = 0; f < YS_NFIELDS; ++f) {
      c->norms_host[f] = std::sqrt(h[f]);
      if (!std::isfinite(c->norms_host[f])) bad = true;
    }
    if (bad) return YS_EDIVERGED;
  }
  return YS_OK;
}

template <typename R>
int set_fields_t(ys_ctx *c, int level, const double *T, const double *ur, const double *uth, const double *uph,
                 const double *p, const double *aux, bool dev) {
  Fields<R> &D = F<R>(c);
  State<R> &s = D.lev[level];
  const Layout &L = c->L;
  int rc = 0;
  rc |= copy_in<R>(c, LC, T, s.f[F_T], c->T_bg, dev);
  const double *u[3] = {ur, uth, uph};
  for (int m = 0; m < 3; ++m)
    rc |= copy_in<R>(c, LR + m, u[m], s.f[F_U2R + m], nullptr, dev, aux ? nullptr : s.f[F_U1R + m]);
  rc |= copy_in_p(c, p, s.p[1], dev, aux ? nullptr : s.p[0]);
  if (aux) {
    size_t o = 0;
    for (int m = 0; m < 3; ++m) {
      rc |= copy_in<R>(c, LR + m, aux + o, s.f[F_U1R + m], nullptr, dev);
      o += user_elems(L, LR + m);
    }
    rc |= copy_in_p(c, aux + o, s.p[0], dev);
  }
  if (rc) return YS_ECUDA;
  refresh<R>(c, s, 3, c->t - level * c->prm.dt);
  if (level == 0 && !c->level1_set) {
    const int bulk[7] = {F_T, F_U1R, F_U1T, F_U1P, F_U2R, F_U2T, F_U2P};
    for (int b = 0; b < 7; ++b)
      cudaMemcpyAsync(D.lev[1].f[bulk[b]], s.f[bulk[b]], L.total * sizeof(R), cudaMemcpyDeviceToDevice, c->stream);
    for (int q = 0; q < 2; ++q)
      cudaMemcpyAsync(D.lev[1].p[q], s.p[q], L.total * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  }
  if (level == 1) c->level1_set = 1;
  return cuda_ok(cudaStreamSynchronize(c->stream));
}

template <typename R>
int get_fields_t(ys_ctx *c, int level, double *T, double *ur, double *uth, double *uph, double *p, double *aux) {
  Fields<R> &D = F<R>(c);
  State<R> &s = D.lev[level];
  int rc = 0;
  if (T) rc |= copy_out<R>(c, LC, s.f[F_T], T, c->T_bg);
  if (ur) rc |= copy_out<R>(c, LR, s.f[F_U2R], ur, nullptr);
  if (uth) rc |= copy_out<R>(c, LT, s.f[F_U2T], uth, nullptr);
  if (uph) rc |= copy_out<R>(c, LP, s.f[F_U2P], uph, nullptr);
  if (p) rc |= copy_out_p(c, s.p[1], p);
  if (aux) {
    size_t o = 0;
    for (int m = 0; m < 3; ++m) {
      rc |= copy_out<R>(c, LR + m, s.f[F_U1R + m], aux + o, nullptr);
      o += user_elems(c->L, LR + m);
    }
    rc |= copy_out_p(c, s.p[0], aux + o);
  }
  if (rc) return YS_ECUDA;
  return cuda_ok(cudaStreamSynchronize(c->stream));
}

template <typename R>
int set_forcing_t(ys_ctx *c, int mode, const double *f_T, const double *f_r, const double *f_th,
                  const double *f_ph) {
  Fields<R> &D = F<R>(c);
  if (!c->modes_mem[mode]) {
    size_t bytes = 4 * (size_t)c->L.total * sizeof(R);
    if (cudaMalloc(&c->modes_mem[mode], bytes) != cudaSuccess) {
      cudaGetLastError();
      c->modes_mem[mode] = nullptr;
      return YS_ENOMEM;
    }
    cudaMemsetAsync(c->modes_mem[mode], 0, bytes, c->stream);
    for (int a = 0; a < 4; ++a) D.modes[mode][a] = (R *)c->modes_mem[mode] + a * c->L.total;
    c->dbytes += bytes;
  }
  int rc = 0;
  rc |= copy_in<R>(c, LC, f_T, D.modes[mode][0], nullptr, false);
  rc |= copy_in<R>(c, LR, f_r, D.modes[mode][1], nullptr, false);
  rc |= copy_in<R>(c, LT, f_th, D.modes[mode][2], nullptr, false);
  rc |= copy_in<R>(c, LP, f_ph, D.modes[mode][3], nullptr, false);
  if (rc) return YS_ECUDA;
  return cuda_ok(cudaStreamSynchronize(c->stream));
}

// FP64 fields: p1, p2 of the three levels
constexpr size_t kPresFields = 6;

// carve the typed state out of one device allocation starting at `base`
template <typename R>
char *carve(ys_ctx *c, Fields<R> &D, char *base) {
  const long T = c->L.total;
  R *f = (R *)base;
  size_t fi = 0;
  const int bulk[7] = {F_T, F_U1R, F_U1T, F_U1P, F_U2R, F_U2T, F_U2P};
  for (int l = 0; l < 3; ++l) {
    for (int b = 0; b < NF; ++b) D.lev[l].f[b] = nullptr;
    for (int b = 0; b < 7; ++b) D.lev[l].f[bulk[b]] = f + (fi++) * T;
  }
  for (int a = 0; a < 3; ++a) D.A[a] = f + (fi++) * T;
  for (int a = 0; a < 4; ++a) D.fcomb[a] = f + (fi++) * T;
  D.B = f + (fi++) * T;
  D.Cs = f + (fi++) * T;
  for (int loc = 0; loc < 4; ++loc)
    for (int dir = 0; dir < 3; ++dir)
      for (int a = 0; a < 3; ++a) D.fac[loc][dir][a] = f + (fi++) * T;
  for (int loc = 0; loc < 4; ++loc)
    for (int dir = 0; dir < 3; ++dir) D.As[loc][dir] = (loc == dir + 1) ? nullptr : f + (fi++) * T;
  for (int a = 0; a < kLevelSums; ++a) D.Sv[a] = (sizeof(R) == sizeof(double)) ? f + (fi++) * T : nullptr;
  for (int m = 0; m < kMaxModes; ++m)
    for (int a = 0; a < 4; ++a) D.modes[m][a] = nullptr;
  char *next = base + ((fi * T * sizeof(R) + 255) / 256) * 256;
  double *pp = (double *)next;
  for (int l = 0; l < 3; ++l)
    for (int q = 0; q < 2; ++q) D.lev[l].p[q] = pp + (2 * l + q) * T;
  next += ((kPresFields * T * sizeof(double) + 255) / 256) * 256;
  // FP64: the phi factors' lane-segment products, 8 arrays of phi_seg_elems
  const long ns = phi_seg_elems(c->L);
  for (int loc = 0; loc < 4; ++loc)
    for (int a = 0; a < 2; ++a) D.seg[loc][a] = (sizeof(R) == sizeof(double)) ? (R *)next + (2 * loc + a) * ns : nullptr;
  if (sizeof(R) == sizeof(double)) next += ((8 * ns * sizeof(double) + 255) / 256) * 256;
  return next;
}

// number of bulk fields of one shell (3 x 7 levels, 3 a, 4 forcing, B, Cs, 36 factors, 9 sums of a),
// and the FP64 form's 5 LevelSums fields (velocity of the system being iterated, T, P2)
constexpr size_t kBulkFields = 3 * 7 + 3 + 4 + 2 + 36 + 9;
constexpr size_t kSumFields64 = kLevelSums;
static_assert(sizeof(Fields<double>::Sv) == kSumFields64 * sizeof(double *), "one pointer per LevelSums field");

// padded field layout of a shell (both patches)
void set_layout(const ys_params *p, Layout &L) {
  L.Nr = p->Nr;
  L.Nt = p->Nth;
  L.Np = p->Nph;
  L.NJ = p->Nth + 2;
  L.P = ((p->Nph + 2) + 7) / 8 * 8;
  L.SI = (long)L.NJ * L.P;
  long box = (long)(p->Nr + 2) * L.SI + 16;
  L.PS = (box + 31) / 32 * 32;
  L.total = 2 * L.PS;
}

// Byte offsets of the parts of a shell's one device allocation, in order: bulk
// fields, FP64 pressures, metric tables (FP64, FP32 pairs), row tables (FP64,
// FP32; the line-operator tables follow the residual tables), exchange
// entries, the deviation profiles, norms, staging.  ys_create_ex allocates
// `total` bytes; the serving queue admits shells by the same figure.
struct ShellPlan {
  size_t row_off[kRowTables], fac_off, row_elems;
  size_t off_metric, off_fmet, off_rowd, off_rowf, off_x, off_dev, off_norm, off_stage, total;
};

ShellPlan plan_shell(const Layout &L, bool mixed, size_t met_n, const size_t (&row_n)[kRowTables], size_t fact_n,
                     size_t xcount) {
  ShellPlan s{};
  const size_t Rsz = mixed ? sizeof(float) : sizeof(double);
  const size_t nbulk = kBulkFields + (mixed ? 0 : kSumFields64);
  const size_t bulk_bytes = ((nbulk * L.total * Rsz + 255) / 256) * 256;
  const size_t p_bytes = ((kPresFields * L.total * sizeof(double) + 255) / 256) * 256 +
                         (mixed ? 0 : ((8 * (size_t)phi_seg_elems(L) * sizeof(double) + 255) / 256) * 256);
  size_t stage_elems = user_elems(L, LR);
  if (user_elems(L, LT) > stage_elems) stage_elems = user_elems(L, LT);
  if (user_elems(L, LP) > stage_elems) stage_elems = user_elems(L, LP);
  s.row_elems = 0;
  for (int t = 0; t < kRowTables; ++t) {
    s.row_off[t] = s.row_elems;
    s.row_elems += (row_n[t] + 31) / 32 * 32;
  }
  s.fac_off = s.row_elems;
  s.row_elems += (fact_n + 31) / 32 * 32;
  s.off_metric = bulk_bytes + p_bytes;
  s.off_fmet = s.off_metric + ((met_n * sizeof(double) + 255) / 256) * 256;
  s.off_rowd = s.off_fmet + ((2 * met_n * sizeof(float) + 255) / 256) * 256;
  s.off_rowf = s.off_rowd + ((s.row_elems * sizeof(double) + 255) / 256) * 256;
  s.off_x = s.off_rowf + ((s.row_elems * sizeof(float) + 255) / 256) * 256;
  s.off_dev = s.off_x + ((xcount * sizeof(XEntry) + 255) / 256) * 256;
  const size_t dev_bytes = ((4 * (size_t)(L.Nr + 2) * sizeof(double) + 255) / 256) * 256;
  s.off_norm = s.off_dev + dev_bytes;
  s.off_stage = s.off_norm + 256;
  s.total = s.off_stage + stage_elems * sizeof(double);
  return s;
}

}  // namespace

extern "C" {

void ys_default_params(ys_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->chi = 1.0;
  p->overlap = 2;
  p->precision = YS_FP64;
  p->schwarz_mode = YS_ADDITIVE;
  p->schwarz_tol = 0.0;
  p->step7 = 1;
  p->step4 = 0;
  p->step4_eps = 1e-8;
  p->step4_tol = 1e-13;
  p->Tbc_inner_a = 1.0;
  p->Tbc_inner_b = 0.0;
  p->Tbc_outer_a = 1.0;
  p->Tbc_outer_b = 0.0;
}

const char *ys_strerror(int code) {
  switch (code) {
    case YS_OK: return "ok";
    case YS_EINVAL: return "invalid argument";
    case YS_ENOMEM: return "out of memory";
    case YS_ECUDA: return "CUDA error";
    case YS_EDIVERGED: return "diverged (NaN/Inf or Schwarz blow-up)";
    case YS_ETIMEOUT: return "deadline passed";
    case YS_EAGAIN: return "not ready";
    case YS_EBUSY: return "busy";
    case YS_ECANCELED: return "cancelled";
  }
  return "unknown error";
}

int ys_create(double R1, double R2, double Pr, double Ra, int Nr, int Nth, int Nph, double dt, ys_ctx **out) {
  ys_params p;
  ys_default_params(&p);
  p.R1 = R1;
  p.R2 = R2;
  p.Pr = Pr;
  p.Ra = Ra;
  p.Nr = Nr;
  p.Nth = Nth;
  p.Nph = Nph;
  p.dt = dt;
  return ys_create_ex(&p, out);
}

int ys_destroy(ys_ctx *c) {
  if (!c) return YS_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto &r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (int m = 0; m < kMaxModes; ++m)
    if (c->modes_mem[m]) cudaFree(c->modes_mem[m]);
  if (c->dmem) cudaFree(c->dmem);
  if (c->dwall) cudaFree(c->dwall);
  if (c->dwall_t) cudaFree(c->dwall_t);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c->f64;
  delete c->f32;
  delete c;
  return YS_OK;
}

int ys_line_coefficients(const ys_params *p, double *out, size_t cap, size_t *count) {
  if (!count) return YS_EINVAL;
  int rc = validate(p);
  if (rc) return rc;
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap, p->r_half};
  GridGeo G;
  if (make_grid(gs, G)) return YS_EINVAL;
  const size_t n = (size_t)kFacTables * (p->Nr + 2) * (p->Nth + 2) * FC_M;
  *count = n;
  if (!out) return YS_OK;
  if (cap < n) return YS_EINVAL;
  std::vector<double> met, fact;
  int pad, len;
  make_metric(gs, G, met, pad, len);
  const double s1 = std::sin(G.th0);
  FacPhys fp{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), 1.0 / (p->R1 * p->R1),
             1.0 / (p->R1 * p->R1 * s1 * s1 * G.hp * G.hp)};
  make_faccoef(gs, G, met, pad, len, fp, fact);
  std::memcpy(out, fact.data(), n * sizeof(double));
  return YS_OK;
}

int ys_residual_coefficients(const ys_params *p, int table, double *out, size_t cap, size_t *count, int *record) {
  if (!count || !record || table < 0 || table >= kRowTables) return YS_EINVAL;
  int rc = validate(p);
  if (rc) return rc;
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap, p->r_half};
  GridGeo G;
  if (make_grid(gs, G)) return YS_EINVAL;
  *record = row_m(table);
  const size_t n = (size_t)(p->Nr + 2) * (p->Nth + 2) * row_m(table);
  *count = n;
  if (!out) return YS_OK;
  if (cap < n) return YS_EINVAL;
  std::vector<double> met, rowt[kRowTables];
  int pad, len;
  make_metric(gs, G, met, pad, len);
  RowPhys ph{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), p->Pr * p->Ra, nullptr, nullptr};
  make_rowcoef(gs, G, met, pad, len, ph, rowt);
  std::memcpy(out, rowt[table].data(), n * sizeof(double));
  return YS_OK;
}

int ys_exchange_table(const ys_params *p, int kind, double *out, size_t cap, size_t *count) {
  if (!count || kind < 0 || kind >= XNUM) return YS_EINVAL;
  int rc = validate(p);
  if (rc) return rc;
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap, p->r_half};
  GridGeo G;
  if (make_grid(gs, G)) return YS_EINVAL;
  std::vector<XEntry> xt[XNUM];
  if (make_exchange(gs, G, xt)) return YS_EINVAL;
  const std::vector<XEntry> &T = xt[kind];
  const size_t n = T.size() * 12;
  *count = n;
  if (!out) return YS_OK;
  if (cap < n) return YS_EINVAL;
  for (size_t e = 0; e < T.size(); ++e) {
    const XEntry &x = T[e];
    const double rec[12] = {(double)x.tj, (double)x.tk, (double)x.j0a, (double)x.k0a, x.wja, x.wka,
                            (double)x.j0b, (double)x.k0b, x.wjb, x.wkb, x.ra, x.rb};
    std::memcpy(out + 12 * e, rec, sizeof rec);
  }
  return YS_OK;
}

size_t ys_shell_device_bytes(const ys_params *p) {
  if (validate(p)) return 0;
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap, p->r_half};
  GridGeo G;
  if (make_grid(gs, G)) return 0;
  std::vector<XEntry> xt[XNUM];
  if (make_exchange(gs, G, xt)) return 0;
  size_t xcount = 0;
  for (int k = 0; k < XNUM; ++k) xcount += xt[k].size();
  std::vector<double> met, rowt[kRowTables], fact;
  int pad, len;
  make_metric(gs, G, met, pad, len);
  RowPhys ph{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), p->Pr * p->Ra, nullptr, nullptr};
  make_rowcoef(gs, G, met, pad, len, ph, rowt);
  const double s1 = std::sin(G.th0);
  FacPhys fp{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), 1.0 / (p->R1 * p->R1),
             1.0 / (p->R1 * p->R1 * s1 * s1 * G.hp * G.hp)};
  make_faccoef(gs, G, met, pad, len, fp, fact);
  size_t row_n[kRowTables];
  for (int t = 0; t < kRowTables; ++t) row_n[t] = rowt[t].size();
  Layout L;
  set_layout(p, L);
  return plan_shell(L, p->precision == YS_MIXED, met.size(), row_n, fact.size(), xcount).total;
}

int ys_create_ex(const ys_params *p, ys_ctx **out) {
  if (!out) return YS_EINVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap, p->r_half};
  GridGeo G;
  if (make_grid(gs, G)) return YS_EINVAL;
  std::vector<XEntry> xt[XNUM];
  if (make_exchange(gs, G, xt)) return YS_EINVAL;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return YS_ECUDA;

  ys_ctx *c = new (std::nothrow) ys_ctx();
  if (!c) return YS_ENOMEM;
  c->prm = *p;
  c->geo = G;
  // the context owns its radial half points (the caller's array may go away)
  c->prm.r_half = c->geo.rh.empty() ? nullptr : c->geo.rh.data() + kGhostHalf;
  const bool mixed = (p->precision == YS_MIXED);
  Layout &L = c->L;
  set_layout(p, L);

  std::vector<double> met;
  int pad, len;
  make_metric(gs, G, met, pad, len);
  // deviation backgrounds of the mixed form (per radial index)
  std::vector<double> Tc(p->Nr + 2), Tlap(p->Nr, 0.0), Tdr(p->Nr, 0.0), pc(p->Nr, 0.0);
  const bool dirichlet_T = (p->Tbc_inner_b == 0.0 && p->Tbc_outer_b == 0.0);
  const bool deviation = mixed && dirichlet_T && (p->T_inner != 0.0 || p->T_outer != 0.0);
  if (deviation) {
    double Ac = (p->T_inner - p->T_outer) / (1.0 / p->R1 - 1.0 / p->R2);
    double Bc = p->T_inner - Ac / p->R1;
    for (int i = 0; i < p->Nr; ++i) Tc[i + 1] = Ac / G.rc(i) + Bc;
    Tc[0] = 2.0 * p->T_inner - Tc[1];             // reflection ghosts, as for T
    Tc[p->Nr + 1] = 2.0 * p->T_outer - Tc[p->Nr];
    // the discrete operators of the residuals applied to T_c (local radial
    // spacings), and the hydrostatic pressure of its buoyancy
    for (int i = 0; i < p->Nr; ++i) {
      double rc = G.rc(i), rfp = G.rf(i + 1), rf0 = G.rf(i);
      Tlap[i] = (rfp * rfp * (Tc[i + 2] - Tc[i + 1]) / G.hf(i + 1) - rf0 * rf0 * (Tc[i + 1] - Tc[i]) / G.hf(i)) /
                (rc * rc * G.hc(i));
      Tdr[i] = (Tc[i + 2] - Tc[i]) / (2.0 * G.hc(i));
      if (i > 0) pc[i] = pc[i - 1] + G.hf(i) * p->Pr * p->Ra * 0.5 * (Tc[i] + Tc[i + 1]);
    }
  }
  size_t xcount = 0;
  for (int k = 0; k < XNUM; ++k) xcount += xt[k].size();
  // residual row-coefficient tables (FP64 and FP32 copies)
  std::vector<double> rowt[kRowTables];
  RowPhys ph{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), p->Pr * p->Ra, deviation ? Tlap.data() : nullptr,
             deviation ? Tdr.data() : nullptr};
  make_rowcoef(gs, G, met, pad, len, ph, rowt);
  std::vector<double> fact;
  {
    const double s1 = std::sin(G.th0);
    FacPhys fp{p->dt, p->Pr, 1.0, 1.0 / (2.0 * p->chi), 1.0 / (p->R1 * p->R1),
               1.0 / (p->R1 * p->R1 * s1 * s1 * G.hp * G.hp)};
    make_faccoef(gs, G, met, pad, len, fp, fact);
  }
  size_t row_n[kRowTables];
  for (int t = 0; t < kRowTables; ++t) row_n[t] = rowt[t].size();
  const ShellPlan plan = plan_shell(L, mixed, met.size(), row_n, fact.size(), xcount);
  const size_t *row_off = plan.row_off;
  const size_t fac_off = plan.fac_off, row_elems = plan.row_elems;
  const size_t off_metric = plan.off_metric, off_fmet = plan.off_fmet, off_rowd = plan.off_rowd;
  const size_t off_rowf = plan.off_rowf, off_x = plan.off_x, off_dev = plan.off_dev;
  const size_t off_norm = plan.off_norm, off_stage = plan.off_stage, total = plan.total;

  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ys_destroy(c);
    return YS_ECUDA;
  }
  c->stream = c->own_stream;
  if (cudaMalloc(&c->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    ys_destroy(c);
    return YS_ENOMEM;
  }
  c->dbytes = total;
  char *base = (char *)c->dmem;
  if (cudaMemsetAsync(base, 0, off_metric, c->stream) != cudaSuccess) {
    ys_destroy(c);
    return YS_ECUDA;
  }
  if (mixed) {
    c->f32 = new (std::nothrow) Fields<float>();
    if (!c->f32) {
      ys_destroy(c);
      return YS_ENOMEM;
    }
    carve<float>(c, *c->f32, base);
  } else {
    c->f64 = new (std::nothrow) Fields<double>();
    if (!c->f64) {
      ys_destroy(c);
      return YS_ENOMEM;
    }
    carve<double>(c, *c->f64, base);
  }
  double *metric = (double *)(base + off_metric);
  float *fmetric = (float *)(base + off_fmet);
  // FP64 tables rounded once to FP32, then the FP32 remainders (double-float pairs)
  std::vector<float> fmet(2 * met.size());
  for (size_t u = 0; u < met.size(); ++u) {
    fmet[u] = (float)met[u];
    fmet[met.size() + u] = (float)(met[u] - (double)fmet[u]);
  }
  cudaMemcpyAsync(fmetric, fmet.data(), fmet.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  double *rowd = (double *)(base + off_rowd);
  float *rowf = (float *)(base + off_rowf);
  std::vector<double> rowh(row_elems, 0.0);
  std::vector<float> rowhf(row_elems, 0.0f);
  for (int t = 0; t < kRowTables; ++t)
    for (size_t u = 0; u < rowt[t].size(); ++u) {
      rowh[row_off[t] + u] = rowt[t][u];
      rowhf[row_off[t] + u] = (float)rowt[t][u];
    }
  for (size_t u = 0; u < fact.size(); ++u) {
    rowh[fac_off + u] = fact[u];
    rowhf[fac_off + u] = (float)fact[u];
  }
  cudaMemcpyAsync(rowd, rowh.data(), row_elems * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(rowf, rowhf.data(), row_elems * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  c->xdev = (XEntry *)(base + off_x);
  double *devtab = (double *)(base + off_dev);
  c->norm = (double *)(base + off_norm);
  c->stage = (double *)(base + off_stage);
  cudaMemcpyAsync(metric, met.data(), met.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  size_t xo = 0;
  for (int k = 0; k < XNUM; ++k) {
    if (!xt[k].empty())
      cudaMemcpyAsync(c->xdev + xo, xt[k].data(), xt[k].size() * sizeof(XEntry), cudaMemcpyHostToDevice, c->stream);
    c->X.e[k] = c->xdev + xo;
    c->X.n[k] = (int)xt[k].size();
    xo += xt[k].size();
  }
  if (p->step4) {
    // Algorithm step 4: edge flux weights (outward normal x face area) of one
    // patch, their squares' sum and the whole boundary's area
    double wsq = 0.0, area = 0.0;
    for (int i = 0; i < p->Nr; ++i) {
      const double rc = G.rc(i), hc = G.hc(i);
      for (int side = 0; side < 2; ++side) {
        const double wt = rc * std::sin(G.th0 + (side ? p->Nth : 0) * G.ht) * hc * G.hp;
        const double wp = rc * hc * G.ht;
        wsq += p->Nph * wt * wt + p->Nth * wp * wp;
        area += p->Nph * wt + p->Nth * wp;
      }
    }
    for (int j = 0; j < p->Nth; ++j) {
      const double sc = std::sin(G.th0 + (j + 0.5) * G.ht);
      area += p->Nph * (p->R1 * p->R1 + p->R2 * p->R2) * sc * G.ht * G.hp;
    }
    c->s4_wsq = wsq;
    c->s4_alpha = 1.0 / (p->step4_eps * area * area);
  }
  Shell &S = c->S;
  S.L = L;
  S.hr = G.hr;
  S.ht = G.ht;
  S.hp = G.hp;
  S.R1 = p->R1;
  S.sin_theta1 = std::sin(G.th0);
  S.dt = p->dt;
  S.nu = p->Pr;
  S.kappa = 1.0;
  S.chi = p->chi;
  S.PrRa = p->Pr * p->Ra;
  S.rc = metric + 0 * len + pad;
  S.rf = metric + 1 * len + pad;
  S.sc = metric + 2 * len + pad;
  S.sf = metric + 3 * len + pad;
  S.cc = metric + 4 * len + pad;
  S.cf = metric + 5 * len + pad;
  S.irc = metric + 6 * len + pad;
  S.irf = metric + 7 * len + pad;
  S.isc = metric + 8 * len + pad;
  S.isf = metric + 9 * len + pad;
  S.hc = metric + 10 * len + pad;
  S.ihc = metric + 11 * len + pad;
  S.nrc = metric + 12 * len + pad;
  S.nrf = metric + 13 * len + pad;
  S.ihr = 1.0 / G.hr;
  S.iht = 1.0 / G.ht;
  S.ihp = 1.0 / G.hp;
  S.i2chi = 1.0 / (2.0 * p->chi);
  S.iR1sq = 1.0 / (p->R1 * p->R1);
  S.cphi = 1.0 / (p->R1 * p->R1 * S.sin_theta1 * S.sin_theta1 * G.hp * G.hp);
  S.T_in = p->T_inner;
  S.T_out = p->T_outer;
  {
    const double a[2] = {p->Tbc_inner_a, p->Tbc_outer_a}, b[2] = {p->Tbc_inner_b, p->Tbc_outer_b};
    shell_set_T_walls(S, a, b, G.hf(0), G.hf(p->Nr));
  }
  S.Tc_lap = nullptr;
  S.Tc_dr = nullptr;
  S.wall_ur = S.wall_ut = S.wall_up = nullptr;
  S.step7 = p->step7;
  shell_fill_fp64(S);
  for (int k = 0; k < kMetricTables; ++k) {
    S.ftab[k] = fmetric + k * len + pad;
    S.ltab[k] = fmetric + met.size() + k * len + pad;
  }
  for (int t = 0; t < kRowTables; ++t) {
    S.rowd[t] = rowd + row_off[t];
    S.rowf[t] = rowf + row_off[t];
  }
  S.facd = rowd + fac_off;
  S.facf = rowf + fac_off;
  if (deviation) {
    // device tables: [Tc at centres i = 0..Nr-1 | pc | Tc_lap | Tc_dr], each Nr + 2 long
    const size_t n = p->Nr + 2;
    std::vector<double> h(4 * n, 0.0);
    for (int i = 0; i < p->Nr; ++i) {
      h[0 * n + i] = Tc[i + 1];
      h[1 * n + i] = pc[i];
      h[2 * n + i] = Tlap[i];
      h[3 * n + i] = Tdr[i];
    }
    cudaMemcpyAsync(devtab, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    c->T_bg = devtab;
    c->p_bg = devtab + n;
    S.Tc_lap = devtab + 2 * n;
    S.Tc_dr = devtab + 3 * n;
    S.T_in = 0.0;   // the deviation has homogeneous reflection walls
    S.T_out = 0.0;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {   // also keeps the host tables alive until copied
    ys_destroy(c);
    return YS_ECUDA;
  }
  *out = c;
  return YS_OK;
}

static int set_fields_any(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                          const double *uph, const double *p, const double *aux, bool dev) {
  if (!c || (level != 0 && level != 1) || !T || !ur || !uth || !uph || !p) return YS_EINVAL;
  if (c->f32) return set_fields_t<float>(c, level, T, ur, uth, uph, p, aux, dev);
  return set_fields_t<double>(c, level, T, ur, uth, uph, p, aux, dev);
}

int ys_set_fields(ys_ctx *c, int level, const double *T, const double *ur, const double *uth, const double *uph,
                  const double *p) {
  return set_fields_any(c, level, T, ur, uth, uph, p, nullptr, false);
}

int ys_set_fields_ex(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                     const double *uph, const double *p, const double *aux) {
  return set_fields_any(c, level, T, ur, uth, uph, p, aux, false);
}

int ys_set_fields_dev(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                      const double *uph, const double *p, const double *aux) {
  return set_fields_any(c, level, T, ur, uth, uph, p, aux, true);
}

int ys_set_forcing(ys_ctx *c, int mode, int time_fn_id, const double *f_T, const double *f_r, const double *f_th,
                   const double *f_ph) {
  if (!c || mode < 0 || mode >= kMaxModes || time_fn_id < 0 || time_fn_id > 4) return YS_EINVAL;
  if (!f_T || !f_r || !f_th || !f_ph) return YS_EINVAL;
  int rc = c->f32 ? set_forcing_t<float>(c, mode, f_T, f_r, f_th, f_ph)
                  : set_forcing_t<double>(c, mode, f_T, f_r, f_th, f_ph);
  if (rc) return rc;
  c->mode_fn[mode] = time_fn_id;
  c->mode_set[mode] = 1;
  if (mode + 1 > c->nmodes_set) c->nmodes_set = mode + 1;
  return YS_OK;
}

int ys_set_wall_velocity(ys_ctx *c, const double *ur, const double *uth, const double *uph) {
  if (!c) return YS_EINVAL;
  const long Nt = c->L.Nt, Np = c->L.Np;
  const size_t n[3] = {(size_t)(4 * Nt * Np), (size_t)(4 * (Nt + 1) * Np), (size_t)(4 * Nt * (Np + 1))};
  const double *src[3] = {ur, uth, uph};
  if (!c->dwall && (ur || uth || uph)) {
    if (cudaMalloc(&c->dwall, (n[0] + n[1] + n[2]) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->dwall = nullptr;
      return YS_ENOMEM;
    }
    c->dbytes += (n[0] + n[1] + n[2]) * sizeof(double);
  }
  const double **dst[3] = {&c->S.wall_ur, &c->S.wall_ut, &c->S.wall_up};
  size_t off = 0;
  for (int m = 0; m < 3; ++m) {
    if (src[m]) {
      if (cudaMemcpyAsync(c->dwall + off, src[m], n[m] * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess)
        return YS_ECUDA;
      *dst[m] = c->dwall + off;
    } else {
      *dst[m] = nullptr;
    }
    off += n[m];
  }
  // Algorithm step 4: wall flux of each patch, sum of (outward) r_f^2 sin(theta_c) h_th h_ph u_r
  c->s4_cwall[0] = c->s4_cwall[1] = 0.0;
  if (ur) {
    const double R[2] = {c->prm.R1, c->prm.R2};
    for (int w = 0; w < 2; ++w)
      for (int p = 0; p < 2; ++p)
        for (long j = 0; j < Nt; ++j) {
          const double a = (w ? 1.0 : -1.0) * R[w] * R[w] * std::sin(c->geo.th0 + (j + 0.5) * c->geo.ht) *
                           c->geo.ht * c->geo.hp;
          for (long k = 0; k < Np; ++k) c->s4_cwall[p] += a * ur[((w * 2 + p) * Nt + j) * Np + k];
        }
  }
  // boundary values of the stored levels follow the new wall data
  if (c->f32)
    refresh_levels<float>(c);
  else
    refresh_levels<double>(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return YS_ECUDA;
  return YS_OK;
}

int ys_set_wall_data(ys_ctx *c, int time_fn_id, const double *T, const double *ur, const double *uth,
                     const double *uph) {
  if (!c || time_fn_id < 0 || time_fn_id > 4) return YS_EINVAL;
  const long Nt = c->L.Nt, Np = c->L.Np;
  const size_t n[4] = {(size_t)(4 * Nt * Np), (size_t)(4 * Nt * Np), (size_t)(4 * (Nt + 1) * Np),
                       (size_t)(4 * Nt * (Np + 1))};
  const double *src[4] = {T, ur, uth, uph};
  if (!c->dwall_t && (T || ur || uth || uph)) {
    if (cudaMalloc(&c->dwall_t, (n[0] + n[1] + n[2] + n[3]) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->dwall_t = nullptr;
      return YS_ENOMEM;
    }
    c->dbytes += (n[0] + n[1] + n[2] + n[3]) * sizeof(double);
  }
  const double **dst[4] = {&c->wall_t.T, &c->wall_t.ur, &c->wall_t.ut, &c->wall_t.up};
  size_t off = 0;
  for (int m = 0; m < 4; ++m) {
    if (src[m]) {
      if (cudaMemcpyAsync(c->dwall_t + off, src[m], n[m] * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess)
        return YS_ECUDA;
      *dst[m] = c->dwall_t + off;
    } else {
      *dst[m] = nullptr;
    }
    off += n[m];
  }
  c->wall_tfn = time_fn_id;
  // Algorithm step 4: wall flux of the time-dependent u_r per unit tau
  c->s4_cwall_t[0] = c->s4_cwall_t[1] = 0.0;
  if (ur) {
    const double R[2] = {c->prm.R1, c->prm.R2};
    for (int w = 0; w < 2; ++w)
      for (int p = 0; p < 2; ++p)
        for (long j = 0; j < Nt; ++j) {
          const double a = (w ? 1.0 : -1.0) * R[w] * R[w] * std::sin(c->geo.th0 + (j + 0.5) * c->geo.ht) *
                           c->geo.ht * c->geo.hp;
          for (long k = 0; k < Np; ++k) c->s4_cwall_t[p] += a * ur[((w * 2 + p) * Nt + j) * Np + k];
        }
  }
  // boundary values of the stored levels follow the new wall data
  if (c->f32)
    refresh_levels<float>(c);
  else
    refresh_levels<double>(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return YS_ECUDA;
  return YS_OK;
}

int ys_set_time(ys_ctx *c, double t) {
  if (!c) return YS_EINVAL;
  c->t = t;
  return YS_OK;
}

int ys_set_stream(ys_ctx *c, void *stream) {
  if (!c) return YS_EINVAL;
  cudaStreamSynchronize(c->stream);
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return YS_OK;
}

int ys_step(ys_ctx *c, int n_steps, int n_schwarz) {
  if (!c || n_steps < 0 || n_schwarz < 1) return YS_EINVAL;
  return c->f32 ? step_t<float>(c, n_steps, n_schwarz) : step_t<double>(c, n_steps, n_schwarz);
}

int ys_get_fields(ys_ctx *c, int level, double *T, double *ur, double *uth, double *uph, double *p, double *aux) {
  if (!c || (level != 0 && level != 1)) return YS_EINVAL;
  return c->f32 ? get_fields_t<float>(c, level, T, ur, uth, uph, p, aux)
                : get_fields_t<double>(c, level, T, ur, uth, uph, p, aux);
}

int ys_get_stats(ys_ctx *c, double *last_norm, double *t, long *steps) {
  if (!c) return YS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return YS_ECUDA;
  if (last_norm) {
    double mx = 0.0;
    for (int f = 0; f < YS_NFIELDS; ++f) mx = std::fmax(mx, c->norms_host[f]);
    *last_norm = mx;
  }
  if (t) *t = c->t;
  if (steps) *steps = c->steps_done;
  return YS_OK;
}

int ys_get_norms(ys_ctx *c, double *norms, int *iters) {
  if (!c) return YS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return YS_ECUDA;
  if (norms)
    for (int f = 0; f < YS_NFIELDS; ++f) norms[f] = c->norms_host[f];
  if (iters) *iters = c->iters_last;
  return YS_OK;
}

int ys_profile_enable(ys_ctx *c, int on) {
  if (!c) return YS_EINVAL;
  cudaStreamSynchronize(c->stream);
  c->prof_on = on ? 1 : 0;
  c->prof_used = 0;
  return YS_OK;
}

int ys_profile_read(ys_ctx *c, const char **names, double *ms, long *launches, int cap) {
  if (!c) return YS_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -YS_ECUDA;
  double tot[K_NUM] = {};
  long cnt[K_NUM] = {};
  for (size_t r = 0; r < c->prof_used; ++r) {
    float m = 0.f;
    cudaEventElapsedTime(&m, c->prof[r].a, c->prof[r].b);
    tot[c->prof[r].cls] += m;
    cnt[c->prof[r].cls] += 1;
  }
  for (int k = 0; k < K_NUM && k < cap; ++k) {
    if (names) names[k] = kClassNames[k];
    if (ms) ms[k] = tot[k];
    if (launches) launches[k] = cnt[k];
  }
  return K_NUM;
}

long ys_launch_count(ys_ctx *c) { return c ? c->launches : -1; }

int ys_measure_fp64_rate(double *tflops) {
  if (!tflops) return YS_EINVAL;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return YS_ECUDA;
  double *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return YS_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * kRateBlocksPerSM, iters = 8192;
  float ms = 0.f;
  k_fp64_rate<<<blocks, kRateThreads>>>(sink, 1.0, iters / 8);   // warm-up
  cudaEventRecord(e0);
  k_fp64_rate<<<blocks, kRateThreads>>>(sink, 1.0, iters);
  cudaEventRecord(e1);
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                  cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (!ok || !(ms > 0.f)) return YS_ECUDA;
  const double flops = 2.0 * kRateChains * (double)iters * blocks * kRateThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return YS_OK;
}

size_t ys_device_bytes(ys_ctx *c) { return c ? c->dbytes : 0; }

}  // extern "C"
