// Internal definition of the single-shell context (shared by api.cu and the
// batch / serving translation unit).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/ys.h"
#include "geometry.h"
#include "kernels.cuh"

namespace ys {

// kernel classes for timing
enum KClass {
  K_EXTRAP = 0, K_FORCE, K_EXCH, K_WALLS, K_RING, K_RES_T, K_RES_U, K_SWEEP_R, K_SWEEP_T, K_SWEEP_P, K_PRES,
  K_PACK, K_FACTOR, K_WATCH, K_SUMS, K_NUM
};

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

// FP64 LevelSums fields of a shell: the iterated system's three velocity
// components, T, and the bootstrapped momentum pressure P2
constexpr int kLevelSums = 5;

// Typed device state of one shell.
template <typename R>
struct Fields {
  State<R> lev[3];           // level n, level n-1, iterate
  R *A[3];                   // advecting velocity
  R *fcomb[4];               // forcing at t_n + dt/2
  R *B, *Cs;                 // right-hand-side work field, forward-sweep scratch of the line solves
  R *fac[4][3][3];           // per-step LU factors: fac[loc][dir] = {lo, 1/pivot, c'}
  R *As[4][3];               // per-step sums of the advecting velocity (StepAux::As)
  R *Sv[kLevelSums];         // FP64: LevelSums fields (velocity of the iterated system, T, P2), else null
  R *seg[4][2];              // FP64: lane-segment products of each unknown's phi factor (a, g), else null
  R *modes[kMaxModes][4];    // forcing modes
};

}  // namespace ys

struct ys_ctx {
  ys_params prm;
  ys::GridGeo geo;
  ys::Layout L;
  ys::Shell S;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  void *dmem = nullptr;
  size_t dbytes = 0;
  void *modes_mem[ys::kMaxModes] = {};
  ys::Fields<double> *f64 = nullptr;
  ys::Fields<float> *f32 = nullptr;
  ys::XEntry *xdev = nullptr;
  ys::XTables X;
  double *norm = nullptr;     // YS_NFIELDS accumulators
  double *stage = nullptr;    // host-layout staging (device); per-block norm shares of k_pressure during a step
  double *dwall = nullptr;    // Dirichlet wall velocity (device, ys_set_wall_velocity), or null
  double *dwall_t = nullptr;  // time-dependent wall data (device, ys_set_wall_data), or null
  ys::WallData wall_t = {};   // its parts (pointers into dwall_t)
  int wall_tfn = 0;           // its time function
  double s4_cwall_t[2] = {0.0, 0.0};   // wall flux of the time-dependent wall velocity per unit tau
  // Algorithm step 4: alpha = 1 / (eps |dOmega|^2), w.w of the edge flux
  // weights, and the wall flux c of each patch (from the wall velocity)
  double s4_alpha = 0.0, s4_wsq = 0.0, s4_cwall[2] = {0.0, 0.0};
  double *T_bg = nullptr;     // deviation backgrounds per radial index (mixed form), else null
  double *p_bg = nullptr;
  int mode_fn[ys::kMaxModes] = {};
  int mode_set[ys::kMaxModes] = {};
  int nmodes_set = 0;
  double t = 0.0;
  long steps_done = 0;
  int level1_set = 0;
  double norms_host[YS_NFIELDS] = {};
  int iters_last = 0;
  long launches = 0;
  int prof_on = 0;
  std::vector<ys::ProfRec> prof;
  size_t prof_used = 0;
};
