// Kernel launchers of the solver (host-callable, C++ linkage, namespace ys).
#pragma once
#include "ys_internal.cuh"

#include <atomic>

namespace ys {

// Field slots of one time level / iterate.
enum FieldSlot { F_T = 0, F_U1R, F_U1T, F_U1P, F_P1, F_U2R, F_U2T, F_U2P, F_P2, NF = 9 };

// One time level or iterate.  Bulk fields (T, u1, u2) are stored in R;
// pressures are always FP64 (p[0] = p1, p[1] = p2).  The slots F_P1 / F_P2 of f
// are not used by the kernels.
template <typename R>
struct State {
  R *f[NF];
  double *p[2];
};

// Arithmetic type of the bulk stencils and sweeps: the storage type.
template <typename R>
struct Cmp {
  using type = R;
};

// Raise a kernel's dynamic shared-memory limit to `bytes` once per device: a
// bit per device in `done` (the call site's own flag word), set after the
// attribute took, so that concurrent first calls merely repeat it.
template <typename K>
inline void smem_attr_once(std::atomic<unsigned long long> &done, K kernel, int bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
    done.fetch_or(bit, std::memory_order_acq_rel);
}

// Advecting velocity and forcing pointers of one step.
template <typename R>
struct StepAux {
  const R *A[3];   // a = 1.5 u2^n - 0.5 u2^{n-1} at r-, theta-, phi-faces
  const R *fT, *fr, *ft, *fp;   // forcing at t_n + dt/2 (nullptr = none)
  // As[loc][dir]: per-step sums of the advecting component `dir` over its
  // nearest stored values around the points of `loc` (2 values at cell
  // centres, 4 at the other faces), summed in the order the stencils use;
  // nullptr for a face's own component, and all nullptr where a launch
  // forms the sums itself (batched shells, the allocation-free solve).  The
  // FP32-storage residual kernels k_resid_* require them.
  const R *As[4][3];
};

// Two-level sums S = psi + psi^n, whole padded fields: S[0..2] the velocity
// components (r, theta, phi) of the system being iterated, S[3] the
// temperature; S[4] the pressure entering that system's momentum rows
// (P_1 = p_1^n, or the field P_2 = p_2^n + (p_1 - p_1^n)/2).  The FP64
// single-shell residuals and pressure updates read them instead of forming
// them at every stencil point.
template <typename R>
struct LevelSums {
  const R *S[5];
};
// up to four whole-field sums s[f] = a[f] + b[f] (null s[f]: unused)
template <typename R>
struct SumJob {
  const R *a[4], *b[4];
  R *s[4];
};

// Separable forcing modes, passed by value: out_c = sum_m tau[m] F[m][c].
constexpr int kMaxModes = 8;
template <typename R>
struct Modes {
  const R *F[kMaxModes][4];
  double tau[kMaxModes];
  int n;
};

struct XTables {
  const XEntry *e[XNUM];
  int n[XNUM];
};

template <typename R>
struct Launch {
  // extrapolation: it = 2 n - nm1 (all slots), A = 1.5 n.u2 - 0.5 nm1.u2
  static void extrapolate(const Layout &L, State<R> it, State<R> n, State<R> nm1, R *A[3],
                          cudaStream_t st);
  // the per-step sums of the advecting velocity (StepAux::As) from A
  static void adv_sums(const Layout &L, R *const A[3], R *const As[4][3], cudaStream_t st);
  // forcing f = sum_m tau_m F_m for the four forcing fields
  static void combine_forcing(long total, Modes<R> modes, R *out[4], cudaStream_t st);
  // Schwarz exchange into the listed patches (mask bit p) of state s
  static void exchange(const Shell &S, const XTables &X, State<R> s, int patch_mask, cudaStream_t st);
  static void walls(const Shell &S, const WallData &wt, State<R> s, int patch_mask, cudaStream_t st);
  static void ring(const Shell &S, const XTables &X, State<R> s, int patch_mask, cudaStream_t st);
  // residual -F into B
  static void resid_T(const Shell &S, State<R> it, State<R> n, StepAux<R> ax, R *B, int patch_mask,
                      cudaStream_t st, LevelSums<R> ls = {});
  // (FP64: ls holds the system's two-level sums, formed by sum_levels)
  static void resid_u(const Shell &S, int sys, int comp, State<R> it, State<R> n, StepAux<R> ax, R *B,
                      int patch_mask, cudaStream_t st, LevelSums<R> ls = {});
  // the whole-field sums of `job` (LevelSums)
  static void sum_levels(const Layout &L, SumJob<R> job, cudaStream_t st);
  // P2 = p2n + (p1 - p1n) / 2 over the whole padded field (LevelSums::S[4])
  static void bootstrap_pressure(const Layout &L, const double *p2n, const double *p1, const double *p1n,
                                 double *P2, cudaStream_t st);
  // one line sweep of the factor (loc, dir); final sweeps add into dst and
  // accumulate the weighted squared increment into norm[slot]
  static void sweep(const Shell &S, int loc, int dir, bool final, StepAux<R> ax, R *B, R *Cs, R *dst,
                    double *norm, int slot, int patch_mask, cudaStream_t st);
  // per-step LU factorisation of the factor (loc, dir) into (Lo, Iv, Cp)
  // (FP64 phi factors given seg = {products of a, of g}: also their
  // lane-segment products, and Lo then holds a = -iv lo)
  static void factorize(const Shell &S, int loc, int dir, StepAux<R> ax, R *Lo, R *Iv, R *Cp, int patch_mask,
                        cudaStream_t st, R *const *seg = nullptr);
  // line solve with a stored factorisation (same conventions as sweep)
  // W: scratch for the forward sweep (distinct from B and dst)
  // FP64 final factors given Sout: also Sout = new dst + Pn (LevelSums);
  // FP64 phi factors given seg: the solves with the lane-segment products
  static void solve(const Shell &S, int loc, int dir, bool final, const R *Lo, const R *Iv, const R *Cp, R *B,
                    R *W, R *dst, double *norm, int slot, int patch_mask, cudaStream_t st, const R *Pn = nullptr,
                    R *Sout = nullptr, R *const *seg = nullptr);
  // pressure update of system sys; part: scratch of one FP64 per cell block
  // (partial norms, summed into norm[4] or norm[8] by a second kernel)
  // Algorithm step 4 on the edge velocity of both systems (acc: 4 FP64 scratch)
  static void mass_flux(const Shell &S, State<R> s, int patch_mask, double *acc, double alpha, double wsq,
                        double cw0, double cw1, double tol, cudaStream_t st);
  static void pressure(const Shell &S, int sys, State<R> it, State<R> n, double *norm, double *part,
                       int patch_mask, cudaStream_t st, LevelSums<R> ls = {});
  // host layout <-> device layout; bg (FP64 per radial index, may be null) is
  // subtracted on the way in and added on the way out
  // user layout (device or mapped pinned host memory) -> padded field dst and,
  // when given, dst2 (src read once)
  static void unpack(const Layout &L, int loc, const double *src, R *dst, const double *bg, cudaStream_t st,
                     R *dst2 = nullptr);
  static void pack(const Layout &L, int loc, const R *src, double *dst, const double *bg, cudaStream_t st);
};

// length of one FP64 lane-segment product array of the phi factors
// (Launch::factorize / solve with seg): 2 Nr Nt lines x 32 lanes per chunk
long phi_seg_elems(const Layout &L);

// FP64 pressure fields: host layout <-> device layout
void unpack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st,
              double *dst2 = nullptr);
void pack_p(const Layout &L, const double *src, double *dst, const double *bg, cudaStream_t st);
// After Schwarz iteration k (1-based) of a step: set norm[kWatchFlag] when
// the iteration's squared increment norms norm[0..NF) are not finite or, for
// k >= 3, the largest exceeds kWatchGrowth^2 times norm[kWatchPrev], the
// previous iteration's; then store it there.
void norm_watch(double *norm, int k, cudaStream_t st);

}  // namespace ys
