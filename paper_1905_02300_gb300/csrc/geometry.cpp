// Host-side geometry of one shell: grid spacings, FP64 metric tables and the
// Schwarz exchange tables (Sec. 2 Yin/Yang maps, Sec. 4 MAC placement and
// interpolated boundary data).
#include "geometry.h"

#include <cmath>
#include <vector>

namespace ys {

static const double kPi = 3.14159265358979323846;

int make_grid(const GridSpec &g, GridGeo &out) {
  if (!(g.R1 > 0.0) || !(g.R2 > g.R1)) return 1;
  if (g.overlap < 1 || g.Nth <= 2 * g.overlap + 4) return 1;
  out.hr = (g.R2 - g.R1) / g.Nr;
  out.ht = (kPi / 2) / (g.Nth - 2 * g.overlap);
  out.delta = g.overlap * out.ht;
  out.hp = (1.5 * kPi + 2 * out.delta) / g.Nph;
  out.th0 = kPi / 4 - out.delta;
  out.ph0 = -0.75 * kPi - out.delta;
  if (!(out.th0 > 0.0)) return 1;
  return 0;
}

void make_metric(const GridSpec &g, const GridGeo &G, std::vector<double> &tab, int &pad, int &len) {
  // kMetricTables tables (rc, rf, sc, sf, cc, cf and the reciprocals of rc,
  // rf, sc, sf), each indexed by logical index with `pad` slots below 0
  pad = 2;
  int n = (g.Nr > g.Nth ? g.Nr : g.Nth) + 2 * pad + 2;
  len = n;
  tab.assign(kMetricTables * (size_t)n, 0.0);
  auto inv = [](double v) { return v != 0.0 ? 1.0 / v : 0.0; };
  for (int t = 0; t < n; ++t) {
    int i = t - pad;
    double rc = g.R1 + (i + 0.5) * G.hr, rf = g.R1 + i * G.hr;
    double thc = G.th0 + (i + 0.5) * G.ht, thf = G.th0 + i * G.ht;
    tab[0 * n + t] = rc;
    tab[1 * n + t] = rf;
    tab[2 * n + t] = std::sin(thc);
    tab[3 * n + t] = std::sin(thf);
    tab[4 * n + t] = std::cos(thc);
    tab[5 * n + t] = std::cos(thf);
    tab[6 * n + t] = inv(rc);
    tab[7 * n + t] = inv(rf);
    tab[8 * n + t] = inv(std::sin(thc));
    tab[9 * n + t] = inv(std::sin(thf));
  }
}

namespace {

struct V3 {
  double x, y, z;
};
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// M(x, y, z) = (-x, z, y): Yin <-> Yang local Cartesian coordinates
inline V3 Mmap(V3 a) { return V3{-a.x, a.z, a.y}; }
inline V3 unit(double th, double ph) {
  return V3{std::sin(th) * std::cos(ph), std::sin(th) * std::sin(ph), std::cos(th)};
}
inline V3 e_th(double th, double ph) {
  return V3{std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph), -std::sin(th)};
}
inline V3 e_ph(double, double ph) { return V3{-std::sin(ph), std::cos(ph), 0.0}; }

// bilinear stencil of a donor quantity staggered (face_t, face_p) at donor
// angles; checks that the 2x2 stencil lies within [jlo, jhi] x [klo, khi]
bool stencil(const GridSpec &g, const GridGeo &G, bool face_t, bool face_p, double th, double ph, int shrink,
             int &j0, int &k0, double &wj, double &wk) {
  double jf = (th - G.th0) / G.ht - (face_t ? 0.0 : 0.5);
  double kf = (ph - G.ph0) / G.hp - (face_p ? 0.0 : 0.5);
  j0 = (int)std::floor(jf);
  k0 = (int)std::floor(kf);
  wj = jf - j0;
  wk = kf - k0;
  int jlo = face_t ? 1 : 0, jhi = face_t ? g.Nth - 1 : g.Nth - 1;
  int klo = face_p ? 1 : 0, khi = face_p ? g.Nph - 1 : g.Nph - 1;
  jlo += shrink;
  jhi -= shrink;
  klo += shrink;
  khi -= shrink;
  return j0 >= jlo && j0 + 1 <= jhi && k0 >= klo && k0 + 1 <= khi;
}

}  // namespace

int make_exchange(const GridSpec &g, const GridGeo &G, std::vector<XEntry> tabs[XNUM]) {
  const int Nt = g.Nth, Np = g.Nph;
  for (int kind = 0; kind < XNUM; ++kind) {
    std::vector<XEntry> &T = tabs[kind];
    T.clear();
    std::vector<std::pair<int, int>> pts;
    if (kind == XT || kind == XUR) {
      for (int j : {-1, Nt})
        for (int k = 0; k < Np; ++k) pts.push_back({j, k});
      for (int k : {-1, Np})
        for (int j = 0; j < Nt; ++j) pts.push_back({j, k});
    } else if (kind == XUT) {
      for (int j : {0, Nt})
        for (int k = 0; k < Np; ++k) pts.push_back({j, k});
      for (int k : {-1, Np})
        for (int j = 1; j < Nt; ++j) pts.push_back({j, k});
    } else if (kind == XUP) {
      for (int k : {0, Np})
        for (int j = 0; j < Nt; ++j) pts.push_back({j, k});
      for (int j : {-1, Nt})
        for (int k = 1; k < Np; ++k) pts.push_back({j, k});
    } else {  // pressure ring: outermost interior cells
      for (int j = 0; j < Nt; ++j)
        for (int k = 0; k < Np; ++k)
          if (j == 0 || j == Nt - 1 || k == 0 || k == Np - 1) pts.push_back({j, k});
    }
    for (auto &pt : pts) {
      XEntry e{};
      e.tj = pt.first;
      e.tk = pt.second;
      double th = G.th0 + (pt.first + (kind == XUT ? 0.0 : 0.5)) * G.ht;
      double ph = G.ph0 + (pt.second + (kind == XUP ? 0.0 : 0.5)) * G.hp;
      V3 xd = Mmap(unit(th, ph));
      double thd = std::acos(xd.z < -1 ? -1 : (xd.z > 1 ? 1 : xd.z));
      double phd = std::atan2(xd.y, xd.x);
      if (kind == XT || kind == XUR || kind == XP) {
        if (!stencil(g, G, false, false, thd, phd, kind == XP ? 1 : 0, e.j0a, e.k0a, e.wja, e.wka)) return 1;
        e.ra = 1.0;
        e.rb = 0.0;
      } else {
        if (!stencil(g, G, true, false, thd, phd, 0, e.j0a, e.k0a, e.wja, e.wka)) return 1;
        if (!stencil(g, G, false, true, thd, phd, 0, e.j0b, e.k0b, e.wjb, e.wkb)) return 1;
        V3 et = (kind == XUT) ? e_th(th, ph) : e_ph(th, ph);
        e.ra = dot(et, Mmap(e_th(thd, phd)));
        e.rb = dot(et, Mmap(e_ph(thd, phd)));
      }
      T.push_back(e);
    }
  }
  return 0;
}

}  // namespace ys
