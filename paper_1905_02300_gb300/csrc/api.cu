// C ABI of the solver: context lifetime, field I/O and the AC time step
// (Sec. 3.3 artificial compressibility with bootstrapping, Sec. 4 Schwarz
// iteration with splitting-error reduction, Eq. er).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ys.h"
#include "geometry.h"
#include "kernels.cuh"

using namespace ys;

namespace {

// kernel classes for timing
enum KClass {
  K_EXTRAP = 0, K_FORCE, K_EXCH, K_WALLS, K_RING, K_RES_T, K_RES_U, K_SWEEP_R, K_SWEEP_T, K_SWEEP_P, K_PRES,
  K_PACK, K_FACTOR, K_NUM
};
const char *kClassNames[K_NUM] = {"extrapolate", "forcing",  "exchange", "walls",   "ring",     "resid_T",
                                  "resid_u",     "sweep_r",  "sweep_t",  "sweep_p", "pressure", "pack",
                                  "factorize"};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct ys_ctx {
  ys_params prm;
  GridGeo geo;
  Layout L;
  Shell S;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  // device memory
  void *dmem = nullptr;
  size_t dbytes = 0;
  double *fields = nullptr;   // 36 fields
  State<double> lev[3];       // level n, level n-1, iterate
  double *A[3];
  double *fcomb[4];
  double *B, *Cs;
  // per-step LU factors of the 12 (unknown, direction) line operators:
  // fac[loc][dir][0..2] = lo, 1/pivot, c'
  double *fac[4][3][3];
  double *metric = nullptr;
  XEntry *xdev = nullptr;
  XTables X;
  double *norm = nullptr;     // YS_NFIELDS accumulators
  double *stage = nullptr;    // host-layout staging (device)
  size_t stage_elems = 0;
  double *modes[kMaxModes][4] = {};
  int mode_fn[kMaxModes] = {};
  int nmodes_set = 0;
  // host state
  double t = 0.0;
  long steps_done = 0;
  int level1_set = 0;
  double norms_host[YS_NFIELDS] = {};
  int iters_last = 0;
  long launches = 0;
  // profiling
  int prof_on = 0;
  std::vector<ProfRec> prof;
  size_t prof_used = 0;
};

namespace {

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

int validate(const ys_params *p) {
  if (!p) return YS_EINVAL;
  if (!(p->R1 > 0.0) || !(p->R2 > p->R1) || !(p->dt > 0.0)) return YS_EINVAL;
  if (p->Nr < 8 || p->Nth < 8 || p->Nph < 8 || p->Nph < p->Nth) return YS_EINVAL;
  if (!(p->chi > 0.0) || p->overlap < 1) return YS_EINVAL;
  if (p->precision != YS_FP64 && p->precision != YS_MIXED) return YS_EINVAL;
  if (p->schwarz_mode != YS_ADDITIVE && p->schwarz_mode != YS_MULTIPLICATIVE) return YS_EINVAL;
  if (!(p->Pr > 0.0) || !(p->Ra >= 0.0) || !(p->schwarz_tol >= 0.0)) return YS_EINVAL;
  return YS_OK;
}

size_t user_elems(const Layout &L, int loc) {
  return 2ul * (L.Nr + (loc == LR)) * (L.Nt + (loc == LT)) * (L.Np + (loc == LP));
}

int copy_in(ys_ctx *c, int loc, const double *src, double *dst, bool device_src) {
  size_t n = user_elems(c->L, loc);
  cudaError_t e = cudaMemcpyAsync(c->stage, src, n * sizeof(double),
                                  device_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return YS_ECUDA;
  LAUNCH(c, K_PACK, 1, Launch<double>::unpack(c->L, loc, c->stage, dst, c->stream));
  return YS_OK;
}

int copy_out(ys_ctx *c, int loc, const double *src, double *dst) {
  size_t n = user_elems(c->L, loc);
  LAUNCH(c, K_PACK, 1, Launch<double>::pack(c->L, loc, src, c->stage, c->stream));
  cudaError_t e = cudaMemcpyAsync(dst, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return YS_ECUDA;
  return cuda_ok(cudaStreamSynchronize(c->stream));
}

// exchange + walls (+ pressure ring) of a whole state: boundary values as
// functions of the interior
void refresh(ys_ctx *c, State<double> s, int mask) {
  LAUNCH(c, K_EXCH, 4, Launch<double>::exchange(c->S, c->X, s, mask, c->stream));
  LAUNCH(c, K_WALLS, 1, Launch<double>::walls(c->S, s, mask, c->stream));
  if (c->prm.step7) LAUNCH(c, K_RING, 1, Launch<double>::ring(c->S, c->X, s, mask, c->stream));
}

const int kOrder[4][3] = {
    {DR, DT, DP},  // T (LC): r, theta, phi
    {DT, DP, DR},  // u_r: theta, phi, r
    {DP, DR, DT},  // u_theta: phi, r, theta
    {DR, DT, DP},  // u_phi: r, theta, phi
};
const int kSweepClass[3] = {K_SWEEP_R, K_SWEEP_T, K_SWEEP_P};

void solve_unknown(ys_ctx *c, int loc, int slot, int mask) {
  State<double> &it = c->lev[2];
  for (int s = 0; s < 3; ++s) {
    int dir = kOrder[loc][s];
    bool fin = (s == 2);
    double *const *F = c->fac[loc][dir];
    LAUNCH(c, kSweepClass[dir], 1,
           Launch<double>::solve(c->S, loc, dir, fin, F[0], F[1], F[2], c->B, it.f[slot], c->norm, slot, mask,
                                 c->stream));
  }
}

// LU factors of every line operator for this step (they depend only on a)
void factorize_all(ys_ctx *c, StepAux<double> ax) {
  for (int loc = LC; loc <= LP; ++loc)
    for (int dir = DR; dir <= DP; ++dir) {
      double *const *F = c->fac[loc][dir];
      LAUNCH(c, K_FACTOR, 1, Launch<double>::factorize(c->S, loc, dir, ax, F[0], F[1], F[2], 3, c->stream));
    }
}

// one defect-correction pass over T, u1, p1, u2, p2 on the masked patches
void iterate(ys_ctx *c, StepAux<double> ax, int mask) {
  State<double> &it = c->lev[2], &n = c->lev[0];
  LAUNCH(c, K_RES_T, 1, Launch<double>::resid_T(c->S, it, n, ax, c->B, mask, c->stream));
  solve_unknown(c, LC, F_T, mask);
  for (int sys = 1; sys <= 2; ++sys) {
    int o = (sys == 1) ? 0 : 4;
    for (int comp = 0; comp < 3; ++comp) {
      LAUNCH(c, K_RES_U, 1, Launch<double>::resid_u(c->S, sys, comp, it, n, ax, c->B, mask, c->stream));
      solve_unknown(c, LR + comp, F_U1R + comp + o, mask);
    }
    LAUNCH(c, K_PRES, 1, Launch<double>::pressure(c->S, sys, it, n, c->norm, mask, c->stream));
  }
}

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
}

const char *ys_strerror(int code) {
  switch (code) {
    case YS_OK: return "ok";
    case YS_EINVAL: return "invalid argument";
    case YS_ENOMEM: return "out of memory";
    case YS_ECUDA: return "CUDA error";
    case YS_EDIVERGED: return "diverged (NaN/Inf)";
    case YS_ETIMEOUT: return "timeout";
    case YS_EAGAIN: return "not ready";
    case YS_EBUSY: return "busy";
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
    if (c->modes[m][0]) cudaFree(c->modes[m][0]);
  if (c->dmem) cudaFree(c->dmem);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return YS_OK;
}

int ys_create_ex(const ys_params *p, ys_ctx **out) {
  if (!out) return YS_EINVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  if (p->precision != YS_FP64) return YS_EINVAL;   // mixed form: separate build step
  GridSpec gs{p->R1, p->R2, p->Nr, p->Nth, p->Nph, p->overlap};
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
  Layout &L = c->L;
  L.Nr = p->Nr;
  L.Nt = p->Nth;
  L.Np = p->Nph;
  L.NJ = p->Nth + 2;
  L.P = ((p->Nph + 2) + 7) / 8 * 8;
  L.SI = (long)L.NJ * L.P;
  long box = (long)(p->Nr + 2) * L.SI + 16;
  L.PS = (box + 31) / 32 * 32;
  L.total = 2 * L.PS;

  std::vector<double> met;
  int pad, len;
  make_metric(gs, G, met, pad, len);
  size_t nfields = 3 * NF + 3 + 4 + 2 + 36;
  size_t field_bytes = (size_t)L.total * sizeof(double);
  size_t xcount = 0;
  for (int k = 0; k < XNUM; ++k) xcount += xt[k].size();
  c->stage_elems = user_elems(L, LR);
  size_t se = user_elems(L, LT), sp = user_elems(L, LP);
  if (se > c->stage_elems) c->stage_elems = se;
  if (sp > c->stage_elems) c->stage_elems = sp;
  size_t off_metric = nfields * field_bytes;
  size_t off_x = off_metric + ((met.size() * sizeof(double) + 255) / 256) * 256;
  size_t off_norm = off_x + ((xcount * sizeof(XEntry) + 255) / 256) * 256;
  size_t off_stage = off_norm + 256;
  size_t total = off_stage + c->stage_elems * sizeof(double);

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
  c->fields = (double *)base;
  size_t fi = 0;
  for (int l = 0; l < 3; ++l)
    for (int f = 0; f < NF; ++f) c->lev[l].f[f] = c->fields + (fi++) * L.total;
  for (int a = 0; a < 3; ++a) c->A[a] = c->fields + (fi++) * L.total;
  for (int a = 0; a < 4; ++a) c->fcomb[a] = c->fields + (fi++) * L.total;
  c->B = c->fields + (fi++) * L.total;
  c->Cs = c->fields + (fi++) * L.total;
  for (int loc = 0; loc < 4; ++loc)
    for (int dir = 0; dir < 3; ++dir)
      for (int a = 0; a < 3; ++a) c->fac[loc][dir][a] = c->fields + (fi++) * L.total;
  c->metric = (double *)(base + off_metric);
  c->xdev = (XEntry *)(base + off_x);
  c->norm = (double *)(base + off_norm);
  c->stage = (double *)(base + off_stage);
  cudaMemcpyAsync(c->metric, met.data(), met.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  size_t xo = 0;
  for (int k = 0; k < XNUM; ++k) {
    if (!xt[k].empty())
      cudaMemcpyAsync(c->xdev + xo, xt[k].data(), xt[k].size() * sizeof(XEntry), cudaMemcpyHostToDevice, c->stream);
    c->X.e[k] = c->xdev + xo;
    c->X.n[k] = (int)xt[k].size();
    xo += xt[k].size();
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
  S.rc = c->metric + 0 * len + pad;
  S.rf = c->metric + 1 * len + pad;
  S.sc = c->metric + 2 * len + pad;
  S.sf = c->metric + 3 * len + pad;
  S.cc = c->metric + 4 * len + pad;
  S.cf = c->metric + 5 * len + pad;
  S.irc = c->metric + 6 * len + pad;
  S.irf = c->metric + 7 * len + pad;
  S.isc = c->metric + 8 * len + pad;
  S.isf = c->metric + 9 * len + pad;
  S.ihr = 1.0 / G.hr;
  S.iht = 1.0 / G.ht;
  S.ihp = 1.0 / G.hp;
  S.i2chi = 1.0 / (2.0 * p->chi);
  S.iR1sq = 1.0 / (p->R1 * p->R1);
  S.cphi = 1.0 / (p->R1 * p->R1 * S.sin_theta1 * S.sin_theta1 * G.hp * G.hp);
  S.T_in = p->T_inner;
  S.T_out = p->T_outer;
  S.step7 = p->step7;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    ys_destroy(c);
    return YS_ECUDA;
  }
  *out = c;
  return YS_OK;
}

static int set_fields_impl(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                           const double *uph, const double *p, const double *aux, bool dev) {
  if (!c || (level != 0 && level != 1) || !T || !ur || !uth || !uph || !p) return YS_EINVAL;
  State<double> &s = c->lev[level];
  const Layout &L = c->L;
  int rc = 0;
  rc |= copy_in(c, LC, T, s.f[F_T], dev);
  const double *u[3] = {ur, uth, uph};
  for (int m = 0; m < 3; ++m) {
    rc |= copy_in(c, LR + m, u[m], s.f[F_U2R + m], dev);
    if (!aux) rc |= copy_in(c, LR + m, u[m], s.f[F_U1R + m], dev);
  }
  rc |= copy_in(c, LC, p, s.f[F_P2], dev);
  if (aux) {
    size_t o = 0;
    for (int m = 0; m < 3; ++m) {
      rc |= copy_in(c, LR + m, aux + o, s.f[F_U1R + m], dev);
      o += user_elems(L, LR + m);
    }
    rc |= copy_in(c, LC, aux + o, s.f[F_P1], dev);
  } else {
    rc |= copy_in(c, LC, p, s.f[F_P1], dev);
  }
  if (rc) return YS_ECUDA;
  refresh(c, s, 3);
  if (level == 0 && !c->level1_set) {
    for (int f = 0; f < NF; ++f)
      cudaMemcpyAsync(c->lev[1].f[f], s.f[f], L.total * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  }
  if (level == 1) c->level1_set = 1;
  return cuda_ok(cudaStreamSynchronize(c->stream));
}

int ys_set_fields(ys_ctx *c, int level, const double *T, const double *ur, const double *uth, const double *uph,
                  const double *p) {
  return set_fields_impl(c, level, T, ur, uth, uph, p, nullptr, false);
}

int ys_set_fields_ex(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                     const double *uph, const double *p, const double *aux) {
  return set_fields_impl(c, level, T, ur, uth, uph, p, aux, false);
}

int ys_set_fields_dev(ys_ctx *c, int level, const double *T, const double *ur, const double *uth,
                      const double *uph, const double *p, const double *aux) {
  return set_fields_impl(c, level, T, ur, uth, uph, p, aux, true);
}

int ys_set_forcing(ys_ctx *c, int mode, int time_fn_id, const double *f_T, const double *f_r, const double *f_th,
                   const double *f_ph) {
  if (!c || mode < 0 || mode >= kMaxModes || time_fn_id < 0 || time_fn_id > 4) return YS_EINVAL;
  if (!f_T || !f_r || !f_th || !f_ph) return YS_EINVAL;
  if (!c->modes[mode][0]) {
    void *mem = nullptr;
    if (cudaMalloc(&mem, 4 * (size_t)c->L.total * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return YS_ENOMEM;
    }
    cudaMemsetAsync(mem, 0, 4 * (size_t)c->L.total * sizeof(double), c->stream);
    for (int a = 0; a < 4; ++a) c->modes[mode][a] = (double *)mem + a * c->L.total;
    c->dbytes += 4 * (size_t)c->L.total * sizeof(double);
  }
  c->mode_fn[mode] = time_fn_id;
  int rc = 0;
  rc |= copy_in(c, LC, f_T, c->modes[mode][0], false);
  rc |= copy_in(c, LR, f_r, c->modes[mode][1], false);
  rc |= copy_in(c, LT, f_th, c->modes[mode][2], false);
  rc |= copy_in(c, LP, f_ph, c->modes[mode][3], false);
  if (mode + 1 > c->nmodes_set) c->nmodes_set = mode + 1;
  if (rc) return YS_ECUDA;
  return cuda_ok(cudaStreamSynchronize(c->stream));
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
  const ys_params &prm = c->prm;
  for (int st = 0; st < n_steps; ++st) {
    State<double> n = c->lev[0], nm1 = c->lev[1], it = c->lev[2];
    LAUNCH(c, K_EXTRAP, 1, Launch<double>::extrapolate(c->L, it, n, nm1, c->A, c->stream));
    StepAux<double> ax;
    for (int a = 0; a < 3; ++a) ax.A[a] = c->A[a];
    ax.fT = ax.fr = ax.ft = ax.fp = nullptr;
    if (c->nmodes_set > 0) {
      // pointers and time weights of the modes at t_n + dt/2, passed by value
      Modes<double> md{};
      for (int m = 0; m < c->nmodes_set; ++m) {
        if (!c->modes[m][0]) continue;
        for (int a = 0; a < 4; ++a) md.F[md.n][a] = c->modes[m][a];
        md.tau[md.n] = time_fn(c->mode_fn[m], c->t + 0.5 * prm.dt);
        ++md.n;
      }
      LAUNCH(c, K_FORCE, 1, Launch<double>::combine_forcing(c->L.total, md, c->fcomb, c->stream));
      ax.fT = c->fcomb[0];
      ax.fr = c->fcomb[1];
      ax.ft = c->fcomb[2];
      ax.fp = c->fcomb[3];
    }
    factorize_all(c, ax);
    c->iters_last = 0;
    for (int k = 1; k <= n_schwarz; ++k) {
      cudaMemsetAsync(c->norm, 0, YS_NFIELDS * sizeof(double), c->stream);
      if (prm.schwarz_mode == YS_ADDITIVE) {
        LAUNCH(c, K_EXCH, 4, Launch<double>::exchange(c->S, c->X, it, 3, c->stream));
        LAUNCH(c, K_WALLS, 1, Launch<double>::walls(c->S, it, 3, c->stream));
        iterate(c, ax, 3);
        if (prm.step7) LAUNCH(c, K_RING, 1, Launch<double>::ring(c->S, c->X, it, 3, c->stream));
      } else {
        for (int p = 0; p < 2; ++p) {
          int m = 1 << p;
          LAUNCH(c, K_EXCH, 4, Launch<double>::exchange(c->S, c->X, it, m, c->stream));
          LAUNCH(c, K_WALLS, 1, Launch<double>::walls(c->S, it, m, c->stream));
          iterate(c, ax, m);
          if (prm.step7) LAUNCH(c, K_RING, 1, Launch<double>::ring(c->S, c->X, it, m, c->stream));
        }
      }
      c->iters_last = k;
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
    refresh(c, it, 3);
    // rotate time levels: n-1 <- n, n <- iterate, iterate <- old n-1
    c->lev[0] = it;
    c->lev[1] = n;
    c->lev[2] = nm1;
    c->t += prm.dt;
    c->steps_done++;
  }
  if (cudaGetLastError() != cudaSuccess) return YS_ECUDA;
  if (n_steps > 0) {
    double h[YS_NFIELDS];
    if (cudaMemcpyAsync(h, c->norm, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return YS_ECUDA;
    bool bad = false;
    for (int f = 0; f < YS_NFIELDS; ++f) {
      c->norms_host[f] = std::sqrt(h[f]);
      if (!std::isfinite(c->norms_host[f])) bad = true;
    }
    if (bad) return YS_EDIVERGED;
  }
  return YS_OK;
}

int ys_get_fields(ys_ctx *c, int level, double *T, double *ur, double *uth, double *uph, double *p, double *aux) {
  if (!c || (level != 0 && level != 1)) return YS_EINVAL;
  State<double> &s = c->lev[level];
  int rc = 0;
  if (T) rc |= copy_out(c, LC, s.f[F_T], T);
  if (ur) rc |= copy_out(c, LR, s.f[F_U2R], ur);
  if (uth) rc |= copy_out(c, LT, s.f[F_U2T], uth);
  if (uph) rc |= copy_out(c, LP, s.f[F_U2P], uph);
  if (p) rc |= copy_out(c, LC, s.f[F_P2], p);
  if (aux) {
    size_t o = 0;
    for (int m = 0; m < 3; ++m) {
      rc |= copy_out(c, LR + m, s.f[F_U1R + m], aux + o);
      o += user_elems(c->L, LR + m);
    }
    rc |= copy_out(c, LC, s.f[F_P1], aux + o);
  }
  return rc ? YS_ECUDA : YS_OK;
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

size_t ys_device_bytes(ys_ctx *c) { return c ? c->dbytes : 0; }

}  // extern "C"
