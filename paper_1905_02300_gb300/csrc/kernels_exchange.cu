// Yin <-> Yang Schwarz boundary exchange (Sec. 4; Algorithm steps 1, 3, 4, 7).
//
// Each patch's boundary values are interpolated from the other patch at the
// same radius (the patches share the radial grid): tensor bilinear
// interpolation in the donor's local (theta, phi), one stencil per donor
// component, then the 2x2 rotation of the tangential components between the
// two local bases.  Radial components need no rotation.  Donor stencils only
// touch the donor's unknowns (never boundary values), which the host checks
// when it builds the tables, so both patches are filled in one launch without
// a snapshot.  Radial ghosts of cell-centred quantities are reflections about
// the wall value.
#include "bodies.cuh"

namespace ys {

namespace {


// threads over (entry, i) pairs, blockIdx.y = target patch
template <typename R>
__global__ void k_exchange(Shell S, const XEntry *__restrict__ e, int n, int kind, State<R> s, int patch_mask) {
  bd::body_exchange(S, e, n, kind, s, patch_mask, blockIdx.x, blockIdx.y);
}

// radial wall data: threads over the padded (j, k) plane, blockIdx.y = patch
template <typename R>
__global__ void k_walls(Shell S, WallData wt, State<R> s, int patch_mask) {
  bd::body_walls(S, wt, s, patch_mask, blockIdx.x, blockIdx.y);
}

// Algorithm step 4 (mass-flux correction).  Edge faces of a patch: theta
// faces j = 0, Nth for every (i, k) and phi faces k = 0, Nph for every (i, j);
// flux weight w = outward normal x face area from the discrete Gauss theorem
// of the divergence: r_c sin(theta_f) h_c h_phi (theta faces), r_c h_c h_theta
// (phi faces), h_c the radial cell width.  Thread e of the y = patch plane handles one edge face.
__device__ __forceinline__ bool edge_face(const Shell &S, int p, long e, long &q, bool &theta, double &w) {
  const Layout &L = S.L;
  const long nt = 2L * L.Nr * L.Np, np = 2L * L.Nr * L.Nt;
  if (e < nt) {
    const int side = (int)(e / ((long)L.Nr * L.Np));
    const long rem = e % ((long)L.Nr * L.Np);
    const int i = (int)(rem / L.Np), k = (int)(rem % L.Np), j = side ? L.Nt : 0;
    q = lidx(L, p, i, j, k);
    theta = true;
    w = (side ? 1.0 : -1.0) * S.rc[i] * S.sf[j] * S.hc[i] * S.hp;
    return true;
  }
  e -= nt;
  if (e >= np) return false;
  const int side = (int)(e / ((long)L.Nr * L.Nt));
  const long rem = e % ((long)L.Nr * L.Nt);
  const int i = (int)(rem / L.Nt), j = (int)(rem % L.Nt), k = side ? L.Np : 0;
  q = lidx(L, p, i, j, k);
  theta = false;
  w = (side ? 1.0 : -1.0) * S.rc[i] * S.hc[i] * S.ht;
  return true;
}

// acc[2 p + s - 1] += sum over patch p's edge faces of w u_s (systems s = 1, 2)
template <typename R>
__global__ void k_edge_flux(Shell S, State<R> st, int patch_mask, double *acc) {
  const int p = blockIdx.y;
  if (!((patch_mask >> p) & 1)) return;
  long q;
  bool theta;
  double w, a1 = 0.0, a2 = 0.0;
  if (edge_face(S, p, blockIdx.x * (long)blockDim.x + threadIdx.x, q, theta, w)) {
    a1 = w * (double)(theta ? st.f[F_U1T] : st.f[F_U1P])[q];
    a2 = w * (double)(theta ? st.f[F_U2T] : st.f[F_U2P])[q];
  }
  for (int off = 16; off > 0; off >>= 1) {
    a1 += __shfl_down_sync(0xffffffffu, a1, off);
    a2 += __shfl_down_sync(0xffffffffu, a2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (a1 != 0.0) atomicAdd(&acc[2 * p], a1);
    if (a2 != 0.0) atomicAdd(&acc[2 * p + 1], a2);
  }
}

// u <- u - alpha F / (1 + alpha w.w) w on the edge faces, F = acc + wall flux,
// when |F| >= tol: the minimiser of J
template <typename R>
__global__ void k_edge_fix(Shell S, State<R> st, int patch_mask, const double *acc, double alpha, double wsq,
                           double cw0, double cw1, double tol) {
  const int p = blockIdx.y;
  if (!((patch_mask >> p) & 1)) return;
  long q;
  bool theta;
  double w;
  if (!edge_face(S, p, blockIdx.x * (long)blockDim.x + threadIdx.x, q, theta, w)) return;
  const double cw = p ? cw1 : cw0;
  for (int s = 0; s < 2; ++s) {
    const double F = acc[2 * p + s] + cw;
    if (!(fabs(F) >= tol)) continue;
    const double beta = alpha * F / (1.0 + alpha * wsq);
    R *u = theta ? st.f[s ? F_U2T : F_U1T] : st.f[s ? F_U2P : F_U1P];
    u[q] = (R)((double)u[q] - beta * w);
  }
}

}  // namespace

template <typename R>
void Launch<R>::mass_flux(const Shell &S, State<R> s, int pm, double *acc, double alpha, double wsq, double cw0,
                          double cw1, double tol, cudaStream_t st) {
  const long E = 2L * S.L.Nr * S.L.Np + 2L * S.L.Nr * S.L.Nt;
  const dim3 g((unsigned)((E + 255) / 256), 2);
  cudaMemsetAsync(acc, 0, 4 * sizeof(double), st);
  k_edge_flux<R><<<g, 256, 0, st>>>(S, s, pm, acc);
  k_edge_fix<R><<<g, 256, 0, st>>>(S, s, pm, acc, alpha, wsq, cw0, cw1, tol);
}

template <typename R>
void Launch<R>::exchange(const Shell &S, const XTables &X, State<R> s, int pm, cudaStream_t st) {
  for (int kind = XT; kind <= XUP; ++kind) {
    int ni = (kind == XUR) ? S.L.Nr - 1 : S.L.Nr;
    long n = (long)X.n[kind] * ni;
    if (n <= 0) continue;
    k_exchange<R><<<dim3((unsigned)((n + 255) / 256), 2), 256, 0, st>>>(S, X.e[kind], X.n[kind], kind, s, pm);
  }
}

template <typename R>
void Launch<R>::walls(const Shell &S, const WallData &wt, State<R> s, int pm, cudaStream_t st) {
  long plane = (long)(S.L.Nt + 2) * (S.L.Np + 2);
  k_walls<R><<<dim3((unsigned)((plane + 255) / 256), 2), 256, 0, st>>>(S, wt, s, pm);
}

template <typename R>
void Launch<R>::ring(const Shell &S, const XTables &X, State<R> s, int pm, cudaStream_t st) {
  long n = (long)X.n[XP] * S.L.Nr;
  k_exchange<R><<<dim3((unsigned)((n + 255) / 256), 2), 256, 0, st>>>(S, X.e[XP], X.n[XP], XP, s, pm);
}

#define YS_INST_EXCHANGE(R)                                                                 \
  template void Launch<R>::exchange(const Shell &, const XTables &, State<R>, int, cudaStream_t); \
  template void Launch<R>::walls(const Shell &, const WallData &, State<R>, int, cudaStream_t);                   \
  template void Launch<R>::ring(const Shell &, const XTables &, State<R>, int, cudaStream_t);       \
  template void Launch<R>::mass_flux(const Shell &, State<R>, int, double *, double, double, double, double, \
                                     double, cudaStream_t);
YS_INST_EXCHANGE(double)
YS_INST_EXCHANGE(float)

}  // namespace ys
