// Batched ensembles and the serving loop.
//
// A batch advances many independent shells of uneven sizes together: every
// kernel class of the AC step (Sec. 3.3, Sec. 4) is ONE persistent launch over
// all member shells.  Each launch walks a work map kept in device memory: per
// shell, the prefix sum of its block count and its grid width, so a CTA finds
// the shell and block it executes by binary search (only when its next block
// lies past the current shell's range: a CTA's blocks ascend).  Time-level rotation is a
// device kernel, so one step, captured once as a CUDA graph, stays valid while
// shells join and leave (only the device-resident maps and descriptors change).
// Per-shell arithmetic and block decomposition do not depend on the other
// members, so a shell's fields are the same alone and in any mix.
//
// The server admits requests by device-memory footprint and free slots,
// advances every admitted shell one batched step at a time, and retires shells
// whose step count is reached (continuous batching: admissions and
// retirements happen at every step boundary).
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bodies.cuh"
#include "ctx.h"

using namespace ys;

namespace ys {

template <typename R>
struct ShellDev {
  Shell S;
  State<R> lev[3];   // physical buffers; level n = lev[rot], n-1 = lev[rot+1], iterate = lev[rot+2] (mod 3)
  R *A[3];
  R *B, *W;          // right-hand side / forward-sweep scratch
  R *fac[4][3][3];
  double *norm;      // YS_NFIELDS accumulators of this shell
  XTables X;
  int rot;
  int step7;
};

// work maps: offs[cap + 1] prefix sums of per-shell block counts, gx[cap] grid widths
struct WorkMap {
  const int *offs;
  const int *gx;
};

enum MapId {
  M_EXTRAP = 0, M_EX0, M_EX1, M_EX2, M_EX3, M_WALLS, M_RING, M_RC, M_RR, M_RT, M_RP, M_LINE0,
  M_PSC0 = M_LINE0 + 12,   // warp-scan phi factorisations and solves (one line per warp), per unknown type
  M_VEC0 = M_PSC0 + 4,     // FP32 residuals, 4 phi-points per thread over flat groups, per unknown type
  M_PRES = M_VEC0 + 4,     // pressure updates over each shell's cells taken as one flat range
  M_FAC0 = M_PRES + 1,     // line factorisations (r, theta; phi in FP64), kFacTpb lines per block
  M_NUM = M_FAC0 + 12
};

namespace {

constexpr int kExtrapChunk = 4096;
constexpr int kMaxCap = 4096;

__device__ __forceinline__ int find_shell(const int *offs, int cap, int w) {
  int lo = 0, hi = cap;   // offs[lo] <= w < offs[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (offs[mid] <= w)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

template <typename R>
__device__ __forceinline__ void roles(const ShellDev<R> &D, State<R> &n, State<R> &nm1, State<R> &it) {
  int r = D.rot;
  n = D.lev[r];
  nm1 = D.lev[(r + 1) % 3];
  it = D.lev[(r + 2) % 3];
}

template <typename R>
__device__ __forceinline__ StepAux<R> aux_of(const ShellDev<R> &D) {
  StepAux<R> ax{};  // no sum tables: the bodies form the sums of a themselves
  for (int a = 0; a < 3; ++a) ax.A[a] = D.A[a];
  ax.fT = ax.fr = ax.ft = ax.fp = nullptr;
  return ax;
}

#define YS_BATCH_LOOP(map, cap)                               \
  const int total_w = (map).offs[cap];                       \
  int s_at = 0, s_beg = 0, s_end = 0, s_gx = 1;              \
  for (int w = blockIdx.x; w < total_w; w += gridDim.x) {    \
    if (w >= s_end) {                                        \
      s_at = find_shell((map).offs, cap, w);                 \
      s_beg = (map).offs[s_at];                              \
      s_end = (map).offs[s_at + 1];                          \
      s_gx = (map).gx[s_at];                                 \
    }                                                        \
    const int s = s_at;                                      \
    const int local = w - s_beg;                             \
    const int gxs = s_gx;                                    \
    const int bx = local % gxs, by = local / gxs;            \
    const ShellDev<R> &D = sh[s];                            \
    State<R> n, nm1, it;                                     \
    roles(D, n, nm1, it);

// the loop with a binary search for every block, for kernels at their
// register cap (the loop-carried shell range of YS_BATCH_LOOP made the
// velocity residuals spill more and run 7% slower)
#define YS_BATCH_LOOP_BS(map, cap)                            \
  const int total_w = (map).offs[cap];                       \
  for (int w = blockIdx.x; w < total_w; w += gridDim.x) {    \
    const int s = find_shell((map).offs, cap, w);            \
    const int local = w - (map).offs[s];                     \
    const int gxs = (map).gx[s];                             \
    const int bx = local % gxs, by = local / gxs;            \
    const ShellDev<R> &D = sh[s];                            \
    State<R> n, nm1, it;                                     \
    roles(D, n, nm1, it);

// the same loop for kernels that need only the iterate's fields
#define YS_BATCH_LOOP_IT(map, cap)                            \
  const int total_w = (map).offs[cap];                       \
  int s_at = 0, s_beg = 0, s_end = 0, s_gx = 1;              \
  for (int w = blockIdx.x; w < total_w; w += gridDim.x) {    \
    if (w >= s_end) {                                        \
      s_at = find_shell((map).offs, cap, w);                 \
      s_beg = (map).offs[s_at];                              \
      s_end = (map).offs[s_at + 1];                          \
      s_gx = (map).gx[s_at];                                 \
    }                                                        \
    const int s = s_at;                                      \
    const int local = w - s_beg;                             \
    const int gxs = s_gx;                                    \
    const int bx = local % gxs, by = local / gxs;            \
    const ShellDev<R> &D = sh[s];                            \
    R *const *itf = D.lev[(D.rot + 2) % 3].f;

template <typename R>
__global__ void kb_extrapolate(const ShellDev<R> *sh, WorkMap map, int cap) {
  YS_BATCH_LOOP(map, cap)
  (void)by;
  long q0 = (long)bx * kExtrapChunk, q1 = q0 + kExtrapChunk;
  if (q1 > D.S.L.total) q1 = D.S.L.total;
  bd::body_extrapolate(q0, q1, it, n, nm1, D.A[0], D.A[1], D.A[2]);
  }
}

template <typename R>
__global__ void kb_factorize(const ShellDev<R> *sh, WorkMap map, int cap, int loc, int dir) {
  YS_BATCH_LOOP(map, cap)
  R *const *F = D.fac[loc][dir];
  bd::body_factorize(D.S, loc, dir, aux_of(D), F[0], F[1], F[2], 3, bx, by);
  }
}

template <typename R>
__global__ void kb_solve(const ShellDev<R> *sh, WorkMap map, int cap, int loc, int dir, int final, int slot) {
  YS_BATCH_LOOP_IT(map, cap)
  R *const *F = D.fac[loc][dir];
  bd::body_solve(D.S, loc, dir, final, F[0], F[1], F[2], D.B, D.W, itf[slot], D.norm, slot, 3, bx, by);
  }
}

template <typename R>
__global__ void kb_factorize_phi(const ShellDev<R> *sh, WorkMap map, int cap, int loc) {
  YS_BATCH_LOOP(map, cap)
  (void)by;
  R *const *F = D.fac[loc][DP];
  bd::body_factorize_phi_scan(D.S, loc, aux_of(D), F[0], F[1], F[2], 3, bx);
  __syncwarp();
  }
}

template <typename R>
__global__ void kb_solve_phi(const ShellDev<R> *sh, WorkMap map, int cap, int loc, int final, int slot,
                             int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char phi_smem[];
  YS_BATCH_LOOP(map, cap)
  (void)by;
  R *const *F = D.fac[loc][DP];
  bd::body_solve_phi_scan(D.S, loc, final, F[0], F[1], F[2], D.B, D.W, it.f[slot], D.norm, slot, 3, bx,
                          (R *)phi_smem, smem_per_warp);
  __syncwarp();
  }
}

template <typename R>
__global__ void kb_resid_T(const ShellDev<R> *sh, WorkMap map, int cap) {
  YS_BATCH_LOOP(map, cap)
  bd::body_resid_T(D.S, it, n, aux_of(D), D.B, 3, bx, by);
  }
}

// FP32 storage: the residuals with 4 phi-points per thread (16-byte loads)
// over each shell's groups taken as one flat range; the sums of the advecting
// velocity are formed in the body (no per-step tables in a batch).
constexpr int kVecNV = 4;
template <typename R>
__global__ void __launch_bounds__(128, 4) kb_resid_T_vec(const ShellDev<R> *sh, WorkMap map, int cap) {
  YS_BATCH_LOOP(map, cap)
  bd::body_resid_T_vec<R, kVecNV, false, true>(D.S, it, n, aux_of(D), D.B, 3, bx, by);
  }
}

template <typename R>
__global__ void __launch_bounds__(128, 4)
    kb_resid_u_vec(const ShellDev<R> *sh, WorkMap map, int cap, int sys, int comp) {
  YS_BATCH_LOOP_BS(map, cap)
  if (comp == 0)
    bd::body_resid_ur_vec<R, kVecNV, false, true>(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  else if (comp == 1)
    bd::body_resid_ut_vec<R, kVecNV, false, true>(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  else
    bd::body_resid_up_vec<R, kVecNV, false, true>(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  }
}

template <typename R>
__global__ void kb_resid_u(const ShellDev<R> *sh, WorkMap map, int cap, int sys, int comp) {
  YS_BATCH_LOOP(map, cap)
  if (comp == 0)
    bd::body_resid_ur(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  else if (comp == 1)
    bd::body_resid_ut(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  else
    bd::body_resid_up(D.S, sys, it, n, aux_of(D), D.B, 3, bx, by);
  }
}

// Pressure updates; each block's norm shares are reduced in the CTA and
// written to parts[w] (w the block's index in the map, so a shell's blocks are
// the contiguous range offs[s] .. offs[s+1]); kb_norm_sum adds them up per
// shell.  No atomics here: a CTA's successive blocks belong to different
// shells, and per-shell atomics from every CTA piled up on a few addresses.
// A block is kPresPts x kPresTpb consecutive cells of the shell's flat range
// (phi fastest, rows one after another): short rows of small shells do not
// leave most of a block idle, and the block's set-up (work-map search, shell
// description) serves 4 cells a thread.
constexpr int kPresTpb = 128, kPresPts = 4;
template <typename R>
__global__ void __launch_bounds__(kPresTpb) kb_pressure(const ShellDev<R> *sh, WorkMap map, int cap, int sys,
                                                        double *parts) {
  using V = typename Cmp<R>::type;
  __shared__ V ws[kPresTpb];
  YS_BATCH_LOOP(map, cap)
  (void)by;
  const Layout &L = D.S.L;
  // 32-bit index arithmetic (a 64-bit division per index took more issue
  // slots than the update itself): a shell's cells number below 2^32, since
  // 2^32 cells of state would need more than a terabyte
  const unsigned ncell = 2u * L.Nr * L.Nt * L.Np;
  const unsigned np = L.Np, nt = L.Nt, nr = L.Nr;
  V acc = (V)0.0;
#pragma unroll
  for (int u = 0; u < kPresPts; ++u) {
    const unsigned f = ((unsigned)bx * kPresPts + u) * kPresTpb + threadIdx.x;
    if (f < ncell) {
      const int k = (int)(f % np);
      unsigned r = f / np;
      const int j = (int)(r % nt);
      r /= nt;
      const int i = (int)(r % nr), p = (int)(r / nr);
      acc += bd::body_pressure_at(D.S, sys, it, n, p, i, j, k);
    }
  }
  ws[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    V v = ws[threadIdx.x];
    for (int u = threadIdx.x + 32; u < kPresTpb; u += 32) v += ws[u];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) parts[w] = (double)v;
  }
  __syncthreads();
  }
}

// norm[s][slot] += CS_VOL(s) * sum of parts over shell s's blocks: one CTA a shell
template <typename R>
__global__ void kb_norm_sum(const ShellDev<R> *sh, WorkMap map, int cap, int slot, const double *parts) {
  __shared__ double ws[8];
  const int s = blockIdx.x;
  if (s >= cap) return;
  const int w0 = map.offs[s], w1 = map.offs[s + 1];
  double t = 0.0;
  for (int w = w0 + threadIdx.x; w < w1; w += blockDim.x) t += parts[w];
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0 && w1 > w0) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += ws[k];
    if (v != 0.0) atomicAdd(&sh[s].norm[slot], v * sh[s].S.dcs[CS_VOL]);
  }
}

template <typename R>
__global__ void kb_exchange(const ShellDev<R> *sh, WorkMap map, int cap, int kind) {
  YS_BATCH_LOOP(map, cap)
  if (kind == XP && !D.step7) continue;
  bd::body_exchange(D.S, D.X.e[kind], D.X.n[kind], kind, it, 3, bx, by);
  }
}

template <typename R>
__global__ void kb_walls(const ShellDev<R> *sh, WorkMap map, int cap) {
  YS_BATCH_LOOP(map, cap)
  bd::body_walls(D.S, WallData{}, it, 3, bx, by);
  }
}

// rotate time levels of every active shell: n-1 <- n, n <- iterate, iterate <- n-1
template <typename R>
__global__ void kb_rotate(ShellDev<R> *sh, const int *active, int cap) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < cap && active[s]) sh[s].rot = (sh[s].rot + 2) % 3;
}

int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// Lines per block of the batched line factorisations.  They keep their own
// width: the autotuned width of the solves (often 32 lines, best for the
// 128-register solves) made them 27% slower than 128 lines a block.
constexpr int kFacTpb = 128;

// per-shell block grid (gx, gy) of a map
void grid_of(const ys_ctx *c, int map, int tpb_line, int &gx, int &gy) {
  const Layout &L = c->L;
  gy = 1;
  if (map >= M_FAC0) {
    map = M_LINE0 + (map - M_FAC0);
    tpb_line = kFacTpb;
  }
  if (map == M_EXTRAP) {
    gx = cdiv(L.total, kExtrapChunk);
  } else if (map >= M_EX0 && map <= M_EX3) {
    int kind = map - M_EX0;
    int ni = (kind == XUR) ? L.Nr - 1 : L.Nr;
    gx = cdiv((long)c->X.n[kind] * ni, 256);
    gy = 2;
  } else if (map == M_WALLS) {
    gx = cdiv((long)(L.Nt + 2) * (L.Np + 2), 256);
    gy = 2;
  } else if (map == M_RING) {
    gx = cdiv((long)c->X.n[XP] * L.Nr, 256);
    gy = 2;
  } else if (map >= M_RC && map <= M_RP) {
    int loc = map - M_RC;
    int ni = L.Nr - (loc == LR), nj = L.Nt - (loc == LT), nk = L.Np - (loc == LP);
    gx = cdiv(nk, 128);
    gy = 2 * ni * nj;
  } else if (map == M_PRES) {
    gx = cdiv(2L * L.Nr * L.Nt * L.Np, (long)kPresTpb * kPresPts);
  } else if (map >= M_VEC0) {
    int loc = map - M_VEC0;
    int ni = L.Nr - (loc == LR), nj = L.Nt - (loc == LT);
    gx = cdiv((long)2 * ni * nj * cdiv(L.Np, kVecNV), 128);
  } else if (map >= M_PSC0) {
    gx = bd::phi_scan_ctas(L, map - M_PSC0);
  } else {
    int loc = (map - M_LINE0) / 3, dir = (map - M_LINE0) % 3;
    int ni = L.Nr - (loc == LR), nj = L.Nt - (loc == LT), nk = L.Np - (loc == LP);
    if (dir == DR) {
      gx = cdiv(nk, tpb_line);
      gy = 2 * nj;
    } else if (dir == DT) {
      gx = cdiv(nk, tpb_line);
      gy = 2 * ni;
    } else {
      gx = cdiv(nj, tpb_line);
      gy = 2 * ni;
    }
  }
}

}  // namespace

// per-member divergence watch words: previous norm, flag, first norm of the step
constexpr int kWatchSlots = 3;

// Divergence watch of every member after Schwarz iteration k (1-based) of a
// step (the single-shell norm_watch per slot): watch[kWatchSlots s] holds the
// largest squared increment norm of the member's previous iteration, the next
// its sticky flag, set by a non-finite norm or, for k >= 3, by a norm above
// kWatchGrowth times the previous iteration's and above the step's first
// (kept in the third).  Empty slots have zero norms and never set it.
__global__ void kb_norm_watch(const double *norms, double *watch, int cap, int k) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= cap) return;
  double cur = 0.0;
  bool bad = false;
  for (int f = 0; f < YS_NFIELDS; ++f) {
    const double v = norms[(size_t)s * YS_NFIELDS + f];
    if (!(v <= 1.79e308)) bad = true;
    else cur = fmax(cur, v);
  }
  double *w = watch + (size_t)kWatchSlots * s;
  if (k == 1) w[2] = cur;
  if (k >= 3 && cur > kWatchGrowth * kWatchGrowth * w[0] && cur > w[2]) bad = true;
  if (bad) w[1] = 1.0;
  w[0] = cur;
}

}  // namespace ys

// ---------------------------------------------------------------------------
// batch engine

struct ys_batch {
  int cap = 0, precision = 0, K = 3, tpb_line = 128;
  int dev = 0;
  cudaStream_t stream = nullptr;
  std::vector<ys_ctx *> slot;
  std::vector<int> rot;           // host mirror of the device rotation counters
  std::vector<long> steps;        // steps taken in the batch, per slot
  void *shells = nullptr;         // ShellDev<R>[cap] (device)
  int *maps = nullptr;            // M_NUM x (2 cap + 1) ints (device)
  int *active = nullptr;          // cap ints (device)
  double *norms = nullptr;        // cap x YS_NFIELDS (device)
  double *watch = nullptr;        // cap x kWatchSlots: divergence watch per member (device; kb_norm_watch)
  double *parts = nullptr;        // per-block pressure norm shares (device), parts_n doubles
  long parts_n = 0;
  std::vector<int> hmaps;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;              // maps / descriptors need upload
  // phi scans: shared-memory positions per warp, bytes per CTA, and the
  // persistent grids (as many CTAs as the SMs hold at once), set before a
  // step is captured or launched eagerly (phi_grids)
  int spw = 0;
  size_t spw_bytes = 0;
  int gp_solve = 0, gp_fact = 0;
  long launches = 0;
  // kernel-class timing (ys_batch_profile_*): profiled steps are launched
  // eagerly with an event pair around each launch instead of replaying the graph
  struct Prof {
    int cls;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<Prof> prof;
  size_t prof_used = 0;
};

namespace {

WorkMap map_of(ys_batch *b, int m) {
  WorkMap w;
  w.offs = b->maps + (size_t)m * (2 * b->cap + 1);
  w.gx = w.offs + b->cap + 1;
  return w;
}

int grid_size(int tpb) { return 152 * (2048 / tpb > 16 ? 16 : 2048 / tpb); }

template <typename R>
Fields<R> &FF(ys_ctx *c);
template <>
Fields<double> &FF<double>(ys_ctx *c) {
  return *c->f64;
}
template <>
Fields<float> &FF<float>(ys_ctx *c) {
  return *c->f32;
}

template <typename R>
ShellDev<R> describe(ys_batch *b, int s) {
  ys_ctx *c = b->slot[s];
  Fields<R> &D = FF<R>(c);
  ShellDev<R> d{};
  d.S = c->S;
  for (int l = 0; l < 3; ++l) d.lev[l] = D.lev[l];
  for (int a = 0; a < 3; ++a) d.A[a] = D.A[a];
  d.B = D.B;
  d.W = D.Cs;
  std::memcpy(d.fac, D.fac, sizeof(d.fac));
  d.norm = b->norms + (size_t)s * YS_NFIELDS;
  d.X = c->X;
  d.rot = b->rot[s];
  d.step7 = c->prm.step7;
  return d;
}

// upload descriptors, active flags and work maps (between steps only)
template <typename R>
int upload(ys_batch *b) {
  const int cap = b->cap;
  std::vector<ShellDev<R>> hd(cap);
  std::vector<int> act(cap, 0);
  for (int s = 0; s < cap; ++s)
    if (b->slot[s]) {
      hd[s] = describe<R>(b, s);
      act[s] = 1;
    }
  b->hmaps.assign((size_t)M_NUM * (2 * cap + 1), 0);
  for (int m = 0; m < M_NUM; ++m) {
    int *offs = b->hmaps.data() + (size_t)m * (2 * cap + 1);
    int *gx = offs + cap + 1;
    long acc = 0;
    for (int s = 0; s < cap; ++s) {
      offs[s] = (int)acc;
      int gxs = 1, gys = 0;
      if (b->slot[s]) grid_of(b->slot[s], m, b->tpb_line, gxs, gys);
      gx[s] = gxs;
      acc += (long)gxs * gys;
      if (acc > 0x7fffffffL) return YS_EINVAL;
    }
    offs[cap] = (int)acc;
  }
  // per-block pressure norm shares: grow the buffer to the pressure map's
  // blocks; the captured graph holds the old pointer, so drop it
  const long need = b->hmaps[(size_t)M_PRES * (2 * cap + 1) + cap];
  if (need > b->parts_n) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    cudaFree(b->parts);
    b->parts = nullptr;
    b->parts_n = 0;
    if (cudaMalloc(&b->parts, sizeof(double) * (size_t)need) != cudaSuccess) {
      cudaGetLastError();
      b->parts = nullptr;
      return YS_ENOMEM;
    }
    b->parts_n = need;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  cudaMemcpyAsync(b->shells, hd.data(), sizeof(ShellDev<R>) * cap, cudaMemcpyHostToDevice, b->stream);
  cudaMemcpyAsync(b->active, act.data(), sizeof(int) * cap, cudaMemcpyHostToDevice, b->stream);
  cudaMemcpyAsync(b->maps, b->hmaps.data(), sizeof(int) * b->hmaps.size(), cudaMemcpyHostToDevice, b->stream);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return YS_ECUDA;
  b->dirty = false;
  return YS_OK;
}

const int kOrderB[4][3] = {{DR, DT, DP}, {DT, DP, DR}, {DP, DR, DT}, {DR, DT, DP}};

// kernel classes of a batched step (timing names)
enum BClass {
  B_EXTRAP = 0, B_FACTOR, B_EXCH, B_WALLS, B_RING, B_RES_T, B_RES_U, B_SWEEP_R, B_SWEEP_T, B_SWEEP_P, B_PRES,
  B_WATCH, B_ROTATE, B_NUM
};
const char *kBClassNames[B_NUM] = {"extrapolate", "factorize", "exchange", "walls",    "ring",  "resid_T", "resid_u",
                                   "sweep_r",     "sweep_t",   "sweep_p",  "pressure", "watch", "rotate"};

// event pair around one launch of a profiled (eager) step
struct BMark {
  ys_batch *b;
  BMark(ys_batch *bb, int cls) : b(bb) {
    if (!b->prof_on) return;
    if (b->prof_used == b->prof.size()) {
      ys_batch::Prof r{cls, nullptr, nullptr};
      cudaEventCreate(&r.a);
      cudaEventCreate(&r.b);
      b->prof.push_back(r);
    }
    b->prof[b->prof_used].cls = cls;
    cudaEventRecord(b->prof[b->prof_used].a, b->stream);
  }
  ~BMark() {
    if (!b->prof_on) return;
    cudaEventRecord(b->prof[b->prof_used].b, b->stream);
    b->prof_used++;
  }
};

// CTAs of a persistent launch: as many as the SMs hold at once (at most 8 a
// SM; 4 a SM if the occupancy query fails)
template <typename K>
int resident_grid(K kernel, int threads, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 4;
  }
  return 152 * (nb > 8 ? 8 : nb);
}

// Shared memory and grids of the phi scans for the current members: the
// longest line of the batch that fits the per-warp buffer (shells with longer
// lines keep their forward results in W).  Called outside stream capture.
template <typename R>
void phi_grids(ys_batch *b) {
  static std::atomic<unsigned long long> attr_done{0};
  smem_attr_once(attr_done, kb_solve_phi<R>, bd::kScanSmemMax);
  int spw = 0;
  for (int s = 0; s < b->cap; ++s) {
    if (!b->slot[s]) continue;
    const int pad = bd::scan_pad(b->slot[s]->L.Np);
    if (pad > spw && (size_t)bd::kScanWarps * pad * sizeof(R) <= (size_t)bd::kScanSmemMax) spw = pad;
  }
  const size_t bytes = (size_t)bd::kScanWarps * spw * sizeof(R);
  if (b->gp_solve == 0 || bytes != b->spw_bytes) {
    b->gp_solve = resident_grid(kb_solve_phi<R>, 32 * bd::kScanWarps, bytes);
    b->gp_fact = resident_grid(kb_factorize_phi<R>, 32 * bd::kScanWarps, 0);
  }
  b->spw = spw;
  b->spw_bytes = bytes;
}

// one AC step of every member shell (additive Schwarz, K iterations)
template <typename R>
void enqueue_step(ys_batch *b) {
  const int cap = b->cap;
  const ShellDev<R> *sh = (const ShellDev<R> *)b->shells;
  cudaStream_t st = b->stream;
  const int g128 = grid_size(128), g256 = grid_size(256), gl = grid_size(b->tpb_line);
  long nl = 0;
  const int spw = b->spw, gp = b->gp_solve, gpf = b->gp_fact;
  const size_t spw_bytes = b->spw_bytes;
  {
    BMark m(b, B_EXTRAP);
    kb_extrapolate<R><<<g256, 256, 0, st>>>(sh, map_of(b, M_EXTRAP), cap);
  }
  ++nl;
  for (int loc = LC; loc <= LP; ++loc)
    for (int dir = DR; dir <= DP; ++dir) {
      BMark m(b, B_FACTOR);
      if (dir == DP && bd::use_phi_scan<R>())
        kb_factorize_phi<R><<<gpf, 32 * bd::kScanWarps, 0, st>>>(sh, map_of(b, M_PSC0 + loc), cap, loc);
      else
        kb_factorize<R><<<grid_size(kFacTpb), kFacTpb, 0, st>>>(sh, map_of(b, M_FAC0 + 3 * loc + dir), cap, loc,
                                                                dir);
      ++nl;
    }
  auto solve = [&](int loc, int slot) {
    for (int s = 0; s < 3; ++s) {
      int dir = kOrderB[loc][s];
      BMark m(b, dir == DR ? B_SWEEP_R : dir == DT ? B_SWEEP_T : B_SWEEP_P);
      if (dir == DP)
        kb_solve_phi<R><<<gp, 32 * bd::kScanWarps, spw_bytes, st>>>(sh, map_of(b, M_PSC0 + loc), cap, loc, s == 2,
                                                                   slot, spw);
      else
        kb_solve<R><<<gl, b->tpb_line, 0, st>>>(sh, map_of(b, M_LINE0 + 3 * loc + dir), cap, loc, dir, s == 2,
                                                 slot);
      ++nl;
    }
  };
  auto exchange = [&]() {
    for (int kind = XT; kind <= XUP; ++kind) {
      BMark m(b, B_EXCH);
      kb_exchange<R><<<g256, 256, 0, st>>>(sh, map_of(b, M_EX0 + kind), cap, kind);
      ++nl;
    }
    {
      BMark m(b, B_WALLS);
      kb_walls<R><<<g256, 256, 0, st>>>(sh, map_of(b, M_WALLS), cap);
    }
    ++nl;
  };
  for (int k = 0; k < b->K; ++k) {
    cudaMemsetAsync(b->norms, 0, sizeof(double) * YS_NFIELDS * cap, st);
    exchange();
    {
      BMark m(b, B_RES_T);
      if constexpr (sizeof(R) == sizeof(float))
        kb_resid_T_vec<R><<<g128, 128, 0, st>>>(sh, map_of(b, M_VEC0 + LC), cap);
      else
        kb_resid_T<R><<<g128, 128, 0, st>>>(sh, map_of(b, M_RC), cap);
    }
    ++nl;
    solve(LC, F_T);
    for (int sys = 1; sys <= 2; ++sys) {
      int o = (sys == 1) ? 0 : 4;
      for (int comp = 0; comp < 3; ++comp) {
        {
          BMark m(b, B_RES_U);
          if constexpr (sizeof(R) == sizeof(float))
            kb_resid_u_vec<R><<<g128, 128, 0, st>>>(sh, map_of(b, M_VEC0 + LR + comp), cap, sys, comp);
          else
            kb_resid_u<R><<<g128, 128, 0, st>>>(sh, map_of(b, M_RR + comp), cap, sys, comp);
        }
        ++nl;
        solve(LR + comp, F_U1R + comp + o);
      }
      {
        BMark m(b, B_PRES);
        kb_pressure<R><<<g128, kPresTpb, 0, st>>>(sh, map_of(b, M_PRES), cap, sys, b->parts);
        kb_norm_sum<R><<<cap, 256, 0, st>>>(sh, map_of(b, M_PRES), cap, sys == 1 ? 4 : 8, b->parts);
      }
      nl += 2;
    }
    {
      BMark m(b, B_RING);
      kb_exchange<R><<<g256, 256, 0, st>>>(sh, map_of(b, M_RING), cap, XP);
    }
    {
      BMark m(b, B_WATCH);
      kb_norm_watch<<<(cap + 127) / 128, 128, 0, st>>>(b->norms, b->watch, cap, k + 1);
    }
    nl += 2;
  }
  exchange();
  {
    BMark m(b, B_RING);
    kb_exchange<R><<<g256, 256, 0, st>>>(sh, map_of(b, M_RING), cap, XP);
  }
  {
    BMark m(b, B_ROTATE);
    kb_rotate<R><<<(cap + 127) / 128, 128, 0, st>>>((ShellDev<R> *)b->shells, b->active, cap);
  }
  nl += 2;
  b->launches = nl;
}

template <typename R>
int capture(ys_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaGraph_t g;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return YS_ECUDA;
  enqueue_step<R>(b);
  if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess) return YS_ECUDA;
  cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? YS_OK : YS_ECUDA;
}

template <typename R>
int batch_step(ys_batch *b, int n) {
  if (b->dirty) {
    int rc = upload<R>(b);
    if (rc) return rc;
  }
  if (b->prof_on) {
    // profiled steps: the same launches, eagerly, with events around each
    phi_grids<R>(b);
    for (int i = 0; i < n; ++i) enqueue_step<R>(b);
  } else {
    if (!b->exec) {
      phi_grids<R>(b);
      int rc = capture<R>(b);
      if (rc) return rc;
    }
    for (int i = 0; i < n; ++i)
      if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return YS_ECUDA;
  }
  for (int s = 0; s < b->cap; ++s)
    if (b->slot[s]) {
      b->rot[s] = (b->rot[s] + 2 * n) % 3;
      b->steps[s] += n;
    }
  return YS_OK;
}

// hand a context back: apply the device rotation to its host-side level order
template <typename R>
void give_back(ys_batch *b, int s) {
  ys_ctx *c = b->slot[s];
  Fields<R> &D = FF<R>(c);
  int r = b->rot[s];
  State<R> l[3] = {D.lev[r], D.lev[(r + 1) % 3], D.lev[(r + 2) % 3]};
  for (int k = 0; k < 3; ++k) D.lev[k] = l[k];
  c->t += b->steps[s] * c->prm.dt;
  c->steps_done += b->steps[s];
  c->iters_last = b->K;
  double h[YS_NFIELDS];
  cudaMemcpy(h, b->norms + (size_t)s * YS_NFIELDS, sizeof(h), cudaMemcpyDeviceToHost);
  for (int f = 0; f < YS_NFIELDS; ++f) c->norms_host[f] = std::sqrt(h[f]);
}

}  // namespace

extern "C" {

int ys_batch_create(int capacity, int precision, int n_schwarz, ys_batch **out) {
  if (!out || capacity < 1 || capacity > kMaxCap || n_schwarz < 1) return YS_EINVAL;
  if (precision != YS_FP64 && precision != YS_MIXED) return YS_EINVAL;
  *out = nullptr;
  ys_batch *b = new (std::nothrow) ys_batch();
  if (!b) return YS_ENOMEM;
  b->cap = capacity;
  b->precision = precision;
  b->K = n_schwarz;
  b->slot.assign(capacity, nullptr);
  b->rot.assign(capacity, 0);
  b->steps.assign(capacity, 0);
  cudaGetDevice(&b->dev);
  size_t shell_bytes = (precision == YS_MIXED ? sizeof(ShellDev<float>) : sizeof(ShellDev<double>)) * capacity;
  size_t map_bytes = sizeof(int) * (size_t)M_NUM * (2 * capacity + 1);
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&b->shells, shell_bytes) != cudaSuccess || cudaMalloc(&b->maps, map_bytes) != cudaSuccess ||
      cudaMalloc(&b->active, sizeof(int) * capacity) != cudaSuccess ||
      cudaMalloc(&b->norms, sizeof(double) * YS_NFIELDS * capacity) != cudaSuccess ||
      cudaMalloc(&b->watch, sizeof(double) * kWatchSlots * capacity) != cudaSuccess ||
      cudaMemsetAsync(b->watch, 0, sizeof(double) * kWatchSlots * capacity, b->stream) != cudaSuccess) {
    cudaGetLastError();
    ys_batch_destroy(b);
    return YS_ENOMEM;
  }
  *out = b;
  return YS_OK;
}

int ys_batch_add(ys_batch *b, ys_ctx *c, int *slot) {
  if (!b || !c || !slot) return YS_EINVAL;
  if ((c->prm.precision == YS_MIXED) != (b->precision == YS_MIXED)) return YS_EINVAL;
  if (c->prm.schwarz_mode != YS_ADDITIVE || c->nmodes_set > 0 || c->prm.step4) return YS_EINVAL;
  if (c->wall_t.T || c->wall_t.ur || c->wall_t.ut || c->wall_t.up) return YS_EINVAL;
  int s = -1;
  for (int i = 0; i < b->cap; ++i)
    if (!b->slot[i]) {
      s = i;
      break;
    }
  if (s < 0) return YS_EBUSY;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return YS_ECUDA;
  // a new member starts with a clear divergence watch (ordered after the
  // batch's queued steps, before its next one)
  if (cudaMemsetAsync(b->watch + (size_t)kWatchSlots * s, 0, kWatchSlots * sizeof(double), b->stream) != cudaSuccess)
    return YS_ECUDA;
  b->slot[s] = c;
  b->rot[s] = 0;
  b->steps[s] = 0;
  b->dirty = true;
  *slot = s;
  return YS_OK;
}

int ys_batch_remove(ys_batch *b, int s, ys_ctx **out) {
  if (!b || s < 0 || s >= b->cap || !b->slot[s]) return YS_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return YS_ECUDA;
  if (b->precision == YS_MIXED)
    give_back<float>(b, s);
  else
    give_back<double>(b, s);
  if (out) *out = b->slot[s];
  b->slot[s] = nullptr;
  b->dirty = true;
  return YS_OK;
}

int ys_batch_step(ys_batch *b, int n_steps) {
  if (!b || n_steps < 0) return YS_EINVAL;
  int rc = (b->precision == YS_MIXED) ? batch_step<float>(b, n_steps) : batch_step<double>(b, n_steps);
  if (rc) return rc;
  return cudaGetLastError() == cudaSuccess ? YS_OK : YS_ECUDA;
}

int ys_batch_sync(ys_batch *b) {
  if (!b) return YS_EINVAL;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? YS_OK : YS_ECUDA;
}

int ys_batch_norms(ys_batch *b, int s, double *norms) {
  if (!b || s < 0 || s >= b->cap || !b->slot[s] || !norms) return YS_EINVAL;
  double h[YS_NFIELDS], w[2];
  if (cudaMemcpyAsync(h, b->norms + (size_t)s * YS_NFIELDS, sizeof(h), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(w, b->watch + (size_t)kWatchSlots * s, sizeof(w), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return YS_ECUDA;
  bool bad = w[1] != 0.0;
  for (int f = 0; f < YS_NFIELDS; ++f) {
    norms[f] = std::sqrt(h[f]);
    if (!std::isfinite(norms[f])) bad = true;
  }
  return bad ? YS_EDIVERGED : YS_OK;
}

int ys_batch_profile_enable(ys_batch *b, int on) {
  if (!b) return YS_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return YS_ECUDA;
  b->prof_on = on != 0;
  b->prof_used = 0;
  return YS_OK;
}

int ys_batch_profile_read(ys_batch *b, const char **names, double *ms, long *launches, int cap) {
  if (!b) return -YS_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return -YS_ECUDA;
  double tot[B_NUM] = {};
  long cnt[B_NUM] = {};
  for (size_t r = 0; r < b->prof_used; ++r) {
    float m = 0.f;
    cudaEventElapsedTime(&m, b->prof[r].a, b->prof[r].b);
    tot[b->prof[r].cls] += m;
    cnt[b->prof[r].cls] += 1;
  }
  for (int k = 0; k < B_NUM && k < cap; ++k) {
    if (names) names[k] = kBClassNames[k];
    if (ms) ms[k] = tot[k];
    if (launches) launches[k] = cnt[k];
  }
  return B_NUM;
}

int ys_batch_set_line_threads(ys_batch *b, int tpb) {
  if (!b || (tpb != 32 && tpb != 64 && tpb != 128 && tpb != 256)) return YS_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return YS_ECUDA;
  if (tpb != b->tpb_line) {
    b->tpb_line = tpb;
    b->dirty = true;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  return YS_OK;
}

long ys_batch_launches_per_step(ys_batch *b) { return b ? b->launches : -1; }

void *ys_batch_stream(ys_batch *b) { return b ? (void *)b->stream : nullptr; }

int ys_batch_autotune(ys_batch *b, int trial_steps, int *chosen) {
  if (!b || trial_steps < 1) return YS_EINVAL;
  const int cand[4] = {32, 64, 128, 256};
  float best = 1e30f;
  int best_t = b->tpb_line;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // trial steps advance the member shells like ordinary steps
  for (int c = 0; c < 4; ++c) {
    int rc = ys_batch_set_line_threads(b, cand[c]);
    if (!rc) rc = ys_batch_step(b, 1);   // upload and capture outside the timing
    if (rc) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
    cudaEventRecord(e0, b->stream);
    rc = ys_batch_step(b, trial_steps);
    cudaEventRecord(e1, b->stream);
    if (rc || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc ? rc : YS_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_t = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = ys_batch_set_line_threads(b, best_t);
  if (chosen) *chosen = best_t;
  return rc;
}

int ys_batch_destroy(ys_batch *b) {
  if (!b) return YS_EINVAL;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto &r : b->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaFree(b->shells);
  cudaFree(b->maps);
  cudaFree(b->active);
  cudaFree(b->norms);
  cudaFree(b->watch);
  cudaFree(b->parts);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return YS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// serving loop

namespace {

struct Request {
  uint64_t ticket;
  ys_params prm;
  std::vector<double> init;     // packed [T | ur | uth | uph | p]
  std::vector<double> result;   // same layout, valid when DONE
  int n_steps = 0;
  int state = 0;                // 0 queued, 1 running, 2 done, 3 failed
  int error = 0;
  int slot = -1;
  long done_steps = 0;
  ys_ctx *ctx = nullptr;
  size_t bytes = 0;
  double deadline_s = 0.0;      // 0: none
  bool cancel = false;          // set under the server mutex by ys_cancel
  std::chrono::steady_clock::time_point t_submit, t_done;

  bool expired(std::chrono::steady_clock::time_point now) const {
    return deadline_s > 0.0 && std::chrono::duration<double>(now - t_submit).count() > deadline_s;
  }
};

size_t packed_len(const ys_params &p) {
  size_t c = 2ul * p.Nr * p.Nth * p.Nph;
  return 2 * c + 2ul * (p.Nr + 1) * p.Nth * p.Nph + 2ul * p.Nr * (p.Nth + 1) * p.Nph +
         2ul * p.Nr * p.Nth * (p.Nph + 1);
}

void unpack_fields(const ys_params &p, const double *buf, const double *f[5]) {
  size_t c = 2ul * p.Nr * p.Nth * p.Nph;
  f[0] = buf;
  f[1] = f[0] + c;
  f[2] = f[1] + 2ul * (p.Nr + 1) * p.Nth * p.Nph;
  f[3] = f[2] + 2ul * p.Nr * (p.Nth + 1) * p.Nph;
  f[4] = f[3] + 2ul * p.Nr * p.Nth * (p.Nph + 1);
}

}  // namespace

struct ys_server {
  size_t budget = 0, used = 0;
  int max_slots = 0, K = 0, precision = YS_MIXED;
  ys_batch *batch = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> queue;
  std::map<uint64_t, Request *> all;
  std::vector<Request *> running;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t max_queue = 4096;
  int dev = 0;
  std::thread worker;
  long steps_run = 0;
  double cell_updates = 0.0;
  int peak_running = 0;   // most requests ever resident together
};

namespace {

constexpr size_t kMaxQueue = 4096;

void server_loop(ys_server *S) {
  cudaSetDevice(S->dev);
  for (;;) {
    std::vector<Request *> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->running.empty(); });
      if (S->stop) return;
      // queued requests past their deadline fail without running
      const auto now = std::chrono::steady_clock::now();
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        if ((*it)->expired(now)) {
          (*it)->state = 3;
          (*it)->error = YS_ETIMEOUT;
          (*it)->t_done = now;
          (*it)->init.clear();
          (*it)->init.shrink_to_fit();
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
      // admission by free slots and device-memory budget, first come first served
      while (!S->queue.empty() && (int)(S->running.size() + admit.size()) < S->max_slots) {
        Request *r = S->queue.front();
        if (S->used + r->bytes > S->budget) break;
        S->queue.pop_front();
        S->used += r->bytes;
        admit.push_back(r);
      }
    }
    for (Request *r : admit) {
      const double *f[5];
      unpack_fields(r->prm, r->init.data(), f);
      int rc = ys_create_ex(&r->prm, &r->ctx);
      if (!rc) rc = ys_set_fields(r->ctx, 0, f[0], f[1], f[2], f[3], f[4]);
      if (!rc) rc = ys_batch_add(S->batch, r->ctx, &r->slot);
      std::lock_guard<std::mutex> lk(S->mu);
      if (rc) {
        if (r->ctx) ys_destroy(r->ctx);
        r->ctx = nullptr;
        r->state = 3;
        r->error = rc;
        S->used -= r->bytes;
        r->t_done = std::chrono::steady_clock::now();
      } else {
        r->state = 1;
        S->running.push_back(r);
        if ((int)S->running.size() > S->peak_running) S->peak_running = (int)S->running.size();
      }
    }
    std::vector<Request *> run;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      run = S->running;
    }
    if (run.empty()) continue;
    int rc = ys_batch_step(S->batch, 1);
    if (!rc) rc = ys_batch_sync(S->batch);
    // requests cancelled, or past their deadline, leave at this step boundary
    std::vector<int> stop_code(run.size(), 0);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const auto now = std::chrono::steady_clock::now();
      for (size_t i = 0; i < run.size(); ++i)
        stop_code[i] = run[i]->cancel ? YS_ECANCELED : run[i]->expired(now) ? YS_ETIMEOUT : 0;
    }
    double step_cells = 0.0;   // counters are published under the lock below (ys_server_stats reads them)
    std::vector<Request *> finished;
    for (size_t i = 0; i < run.size(); ++i) {
      Request *r = run[i];
      r->done_steps++;
      step_cells += 2.0 * r->prm.Nr * r->prm.Nth * r->prm.Nph;
      if (stop_code[i]) {
        ys_ctx *c = nullptr;
        ys_batch_remove(S->batch, r->slot, &c);
        ys_destroy(c);
        r->ctx = nullptr;
        r->error = stop_code[i];
        finished.push_back(r);
        continue;
      }
      double nrm[YS_NFIELDS];
      bool bad = rc != 0;
      // non-finite norms or a tripped divergence watch fail this request alone
      const int nrc = bad ? YS_OK : ys_batch_norms(S->batch, r->slot, nrm);
      if (nrc != YS_OK) bad = true;
      if (bad || r->done_steps >= r->n_steps) {
        ys_ctx *c = nullptr;
        ys_batch_remove(S->batch, r->slot, &c);
        int err = bad ? (rc ? rc : nrc) : 0;
        if (!bad) {
          r->result.resize(packed_len(r->prm));
          const double *f[5];
          unpack_fields(r->prm, r->result.data(), f);
          err = ys_get_fields(c, 0, (double *)f[0], (double *)f[1], (double *)f[2], (double *)f[3], (double *)f[4],
                              nullptr);
        }
        ys_destroy(c);
        r->ctx = nullptr;
        r->error = err;
        finished.push_back(r);
      }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->steps_run++;
    S->cell_updates += step_cells;
    for (Request *r : finished) {
      r->state = r->error ? 3 : 2;
      r->t_done = std::chrono::steady_clock::now();
      r->init.clear();
      r->init.shrink_to_fit();
      S->used -= r->bytes;
      for (size_t i = 0; i < S->running.size(); ++i)
        if (S->running[i] == r) {
          S->running.erase(S->running.begin() + i);
          break;
        }
    }
  }
}

size_t footprint(const ys_params &p) {
  // the shell's own device allocation (exactly what ys_create_ex takes) plus
  // a margin for its share of the batch's member buffers (maps, norms,
  // pressure parts); served shells use no forcing modes; 0: invalid
  const size_t b = ys_shell_device_bytes(&p);
  return b ? b + (1u << 20) : 0;
}

}  // namespace

extern "C" {

int ys_server_create(size_t hbm_budget_bytes, int max_slots, ys_server **out) {
  if (!out || max_slots < 1 || max_slots > kMaxCap || hbm_budget_bytes == 0) return YS_EINVAL;
  *out = nullptr;
  ys_server *S = new (std::nothrow) ys_server();
  if (!S) return YS_ENOMEM;
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  cudaGetDevice(&S->dev);
  *out = S;
  return YS_OK;
}

int ys_submit(ys_server *S, const ys_params *p, const double *init_fields, int n_steps, int n_schwarz,
              uint64_t *ticket) {
  return ys_submit_ex(S, p, init_fields, n_steps, n_schwarz, 0.0, ticket);
}

int ys_submit_ex(ys_server *S, const ys_params *p, const double *init_fields, int n_steps, int n_schwarz,
                 double deadline_s, uint64_t *ticket) {
  if (!S || !p || !init_fields || n_steps < 1 || n_schwarz < 1 || !ticket) return YS_EINVAL;
  if (!(deadline_s >= 0.0)) return YS_EINVAL;
  if (p->schwarz_mode != YS_ADDITIVE || p->schwarz_tol != 0.0) return YS_EINVAL;
  if (p->r_half) return YS_EINVAL;   // queued requests keep no copy of the radii: uniform grids only
  const size_t bytes = footprint(*p);
  if (!bytes || bytes > S->budget) return YS_EINVAL;   // invalid, or can never be admitted
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->batch) {
    // the first request fixes the batch precision and iteration count
    int rc = ys_batch_create(S->max_slots, p->precision, n_schwarz, &S->batch);
    if (rc) return rc;
    S->K = n_schwarz;
    S->precision = p->precision;
    S->worker = std::thread(server_loop, S);
  }
  if (n_schwarz != S->K || p->precision != S->precision) return YS_EINVAL;
  if (S->queue.size() >= S->max_queue) return YS_EBUSY;
  Request *r = new (std::nothrow) Request();
  if (!r) return YS_ENOMEM;
  r->prm = *p;
  r->init.assign(init_fields, init_fields + packed_len(*p));
  r->n_steps = n_steps;
  r->bytes = bytes;
  r->deadline_s = deadline_s;
  r->ticket = S->next_ticket++;
  r->t_submit = std::chrono::steady_clock::now();
  S->queue.push_back(r);
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  lk.unlock();
  S->cv.notify_one();
  return YS_OK;
}

int ys_poll(ys_server *S, uint64_t ticket, int *state, double *out_fields, double *latency_s) {
  if (!S) return YS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return YS_EINVAL;
  Request *r = it->second;
  if (state) *state = r->state;
  if (r->state < 2) return YS_EAGAIN;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (r->state == 3) return r->error ? r->error : YS_ECUDA;
  if (out_fields) std::memcpy(out_fields, r->result.data(), r->result.size() * sizeof(double));
  return YS_OK;
}

int ys_cancel(ys_server *S, uint64_t ticket) {
  if (!S) return YS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return YS_EINVAL;
  Request *r = it->second;
  if (r->state >= 2) return YS_EINVAL;
  if (r->state == 0) {
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
      if (*q == r) {
        S->queue.erase(q);
        r->state = 3;
        r->error = YS_ECANCELED;
        r->t_done = std::chrono::steady_clock::now();
        r->init.clear();
        r->init.shrink_to_fit();
        return YS_OK;
      }
  }
  // admitted (or being admitted): the worker retires it at the next step boundary
  r->cancel = true;
  return YS_OK;
}

int ys_server_set_queue_limit(ys_server *S, int max_queued) {
  if (!S || max_queued < 1 || max_queued > (int)kMaxQueue) return YS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_queue = (size_t)max_queued;
  return YS_OK;
}

int ys_server_stats(ys_server *S, long *steps_run, double *cell_updates, int *running, int *queued,
                    int *peak_running) {
  if (!S) return YS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (steps_run) *steps_run = S->steps_run;
  if (cell_updates) *cell_updates = S->cell_updates;
  if (running) *running = (int)S->running.size();
  if (queued) *queued = (int)S->queue.size();
  if (peak_running) *peak_running = S->peak_running;
  return YS_OK;
}

int ys_server_destroy(ys_server *S) {
  if (!S) return YS_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Request *r : S->running) {
    ys_ctx *c = nullptr;
    ys_batch_remove(S->batch, r->slot, &c);
    if (c) ys_destroy(c);
  }
  if (S->batch) ys_batch_destroy(S->batch);
  for (auto &kv : S->all) delete kv.second;
  delete S;
  return YS_OK;
}

}  // extern "C"
