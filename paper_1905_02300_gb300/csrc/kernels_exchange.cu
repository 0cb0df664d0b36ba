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
#include "kernels.cuh"

namespace ys {

namespace {

template <typename R>
__device__ __forceinline__ double bilin(const R *a, const Layout &L, int p, int i, int j0, int k0, double wj,
                                        double wk) {
  long q = lidx(L, p, i, j0, k0);
  return (1 - wj) * (1 - wk) * (double)a[q] + (1 - wj) * wk * (double)a[q + 1] + wj * (1 - wk) * (double)a[q + L.P] +
         wj * wk * (double)a[q + L.P + 1];
}

// threads over (entry, i) pairs, blockIdx.y = target patch
template <typename R>
__global__ void k_exchange(Shell S, const XEntry *__restrict__ e, int n, int kind, State<R> s, int patch_mask) {
  const Layout &L = S.L;
  int p = blockIdx.y;
  if (!((patch_mask >> p) & 1)) return;
  int d = 1 - p;
  int ni = (kind == XUR) ? L.Nr - 1 : L.Nr;
  int i0 = (kind == XUR) ? 1 : 0;
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)n * ni) return;
  int ent = (int)(t % n);
  int i = i0 + (int)(t / n);
  const XEntry E = e[ent];
  long qt = lidx(L, p, i, E.tj, E.tk);
  if (kind == XT) {
    s.f[F_T][qt] = (R)bilin(s.f[F_T], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else if (kind == XUR) {
    s.f[F_U1R][qt] = (R)bilin(s.f[F_U1R], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
    s.f[F_U2R][qt] = (R)bilin(s.f[F_U2R], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else if (kind == XP) {
    s.p[0][qt] = bilin(s.p[0], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
    s.p[1][qt] = bilin(s.p[1], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
  } else {
    int slot = (kind == XUT) ? F_U1T : F_U1P;
    for (int o = 0; o <= 4; o += 4) {
      double vt = bilin(s.f[F_U1T + o], L, d, i, E.j0a, E.k0a, E.wja, E.wka);
      double vp = bilin(s.f[F_U1P + o], L, d, i, E.j0b, E.k0b, E.wjb, E.wkb);
      s.f[slot + o][qt] = (R)(E.ra * vt + E.rb * vp);
    }
  }
}

// radial wall data: threads over the padded (j, k) plane, blockIdx.y = patch
template <typename R>
__global__ void k_walls(Shell S, State<R> s, int patch_mask) {
  const Layout &L = S.L;
  int p = blockIdx.y;
  if (!((patch_mask >> p) & 1)) return;
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long plane = (long)(L.Nt + 2) * (L.Np + 2);
  if (t >= plane) return;
  int j = (int)(t / (L.Np + 2)) - 1;
  int k = (int)(t % (L.Np + 2)) - 1;
  const int Nr = L.Nr, Nt = L.Nt, Np = L.Np;
  long lo = lidx(L, p, -1, j, k), l0 = lidx(L, p, 0, j, k);
  long hi = lidx(L, p, Nr, j, k), h0 = lidx(L, p, Nr - 1, j, k);
  // u_r on the wall faces i = 0 and i = Nr, the whole plane
  s.f[F_U1R][l0] = (R)0.0;
  s.f[F_U2R][l0] = (R)0.0;
  s.f[F_U1R][hi] = (R)0.0;
  s.f[F_U2R][hi] = (R)0.0;
  if (j >= 0 && j < Nt && k >= 0 && k < Np) {
    s.f[F_T][lo] = (R)(2.0 * S.T_in - (double)s.f[F_T][l0]);
    s.f[F_T][hi] = (R)(2.0 * S.T_out - (double)s.f[F_T][h0]);
  }
  if (j >= 1 && j < Nt && k >= 0 && k < Np) {
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1T + o];
      u[lo] = (R)(-(double)u[l0]);
      u[hi] = (R)(-(double)u[h0]);
    }
  }
  if (j >= 0 && j < Nt && k >= 1 && k < Np) {
    for (int o = 0; o <= 4; o += 4) {
      R *u = s.f[F_U1P + o];
      u[lo] = (R)(-(double)u[l0]);
      u[hi] = (R)(-(double)u[h0]);
    }
  }
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
