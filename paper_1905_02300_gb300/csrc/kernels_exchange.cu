// Yin <-> Yang Schwarz boundary exchange (Sec. 4; Algorithm steps 1, 3, 7).
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
__global__ void k_walls(Shell S, State<R> s, int patch_mask) {
  bd::body_walls(S, s, patch_mask, blockIdx.x, blockIdx.y);
}

}  // namespace

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
void Launch<R>::walls(const Shell &S, State<R> s, int pm, cudaStream_t st) {
  long plane = (long)(S.L.Nt + 2) * (S.L.Np + 2);
  k_walls<R><<<dim3((unsigned)((plane + 255) / 256), 2), 256, 0, st>>>(S, s, pm);
}

template <typename R>
void Launch<R>::ring(const Shell &S, const XTables &X, State<R> s, int pm, cudaStream_t st) {
  long n = (long)X.n[XP] * S.L.Nr;
  k_exchange<R><<<dim3((unsigned)((n + 255) / 256), 2), 256, 0, st>>>(S, X.e[XP], X.n[XP], XP, s, pm);
}

#define YS_INST_EXCHANGE(R)                                                                 \
  template void Launch<R>::exchange(const Shell &, const XTables &, State<R>, int, cudaStream_t); \
  template void Launch<R>::walls(const Shell &, State<R>, int, cudaStream_t);                   \
  template void Launch<R>::ring(const Shell &, const XTables &, State<R>, int, cudaStream_t);
YS_INST_EXCHANGE(double)
YS_INST_EXCHANGE(float)

}  // namespace ys
