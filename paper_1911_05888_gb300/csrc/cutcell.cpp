// Cut cells of an embedded circle on a Cartesian grid (host): the setup step
// of the embedded-interface problems (Section 5, the circular interface of
// the multi-phase tests).  The paper takes the quadrature from external
// implicit-quadrature work; this is quadrature by dimension reduction written
// from that idea:
//  * in each cell crossed by phi(x) = |x - c| - r the height direction is the
//    axis of the larger normal component at the cell centre, so that the
//    circle is a smooth graph over the tangential axis inside the cell;
//  * the tangential interval is split where the circle crosses the cell's
//    height-direction faces, a q-point Gauss rule runs on each part, and at
//    each node the circle's chord (found analytically) splits the height
//    interval into the inside (phase 1) and outside (phase 2) parts, each with
//    its own q-point Gauss rule;
//  * the interface rule uses the same tangential nodes on the branch of the
//    circle inside the cell, weighted by ds = sqrt(1 + (dh/dt)^2) dt.
// A piece below a quarter of its cell joins the same-phase piece across the
// cell face it shares most with (the longest same-phase part of the face),
// among the neighbours that are not small themselves.  The merged elements
// are coloured greedily over the reach of the couplings.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <limits>
#include <set>
#include <string>
#include <vector>

#include "stk_internal.h"
#include "../../include/stokes_mg.h"

namespace stk {

namespace {

struct Circ {
  double c[2], r;
  double phi(double x, double y) const { return std::sqrt((x - c[0]) * (x - c[0]) + (y - c[1]) * (y - c[1])) - r; }
};

// -1 inside, +1 outside, 0 cut
int classify(const Circ& C, const double* lo, const double* hi) {
  double nx = std::min(std::max(C.c[0], lo[0]), hi[0]), ny = std::min(std::max(C.c[1], lo[1]), hi[1]);
  const double dmin = std::sqrt((nx - C.c[0]) * (nx - C.c[0]) + (ny - C.c[1]) * (ny - C.c[1]));
  double dmax = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double x = a ? hi[0] : lo[0], y = b ? hi[1] : lo[1];
      dmax = std::max(dmax, std::sqrt((x - C.c[0]) * (x - C.c[0]) + (y - C.c[1]) * (y - C.c[1])));
    }
  if (dmax <= C.r) return -1;
  if (dmin >= C.r) return 1;
  return 0;
}

// Gauss rule of q points on [a, b], appended to (t, w).
void gauss_on(double a, double b, const std::vector<double>& gx, const std::vector<double>& gw,
              std::vector<double>& t, std::vector<double>& w) {
  for (size_t k = 0; k < gx.size(); ++k) {
    t.push_back(0.5 * (a + b) + 0.5 * (b - a) * gx[k]);
    w.push_back(0.5 * (b - a) * gw[k]);
  }
}

// Volume rules of the inside and outside pieces of a cut cell and its
// interface rule (points, weights, normals out of the circle).
void cut_cell_rules(const Circ& C, const double* lo, const double* hi, const std::vector<double>& gx,
                    const std::vector<double>& gw, CutPiece& in, CutPiece& out, CutArc& arc) {
  const double cx = 0.5 * (lo[0] + hi[0]) - C.c[0], cy = 0.5 * (lo[1] + hi[1]) - C.c[1];
  const int h_ax = std::fabs(cy) > std::fabs(cx) ? 1 : 0, t_ax = 1 - h_ax;
  const double c_t = C.c[t_ax], c_h = C.c[h_ax], r = C.r;
  const double t0 = lo[t_ax], t1 = hi[t_ax], h0 = lo[h_ax], h1 = hi[h_ax];
  std::set<double> brk = {t0, t1};
  for (double hh : {h0, h1}) {
    const double disc = r * r - (hh - c_h) * (hh - c_h);
    if (disc > 0)
      for (double s : {-1.0, 1.0}) {
        const double t = c_t + s * std::sqrt(disc);
        if (t0 < t && t < t1) brk.insert(t);
      }
  }
  for (double s : {-1.0, 1.0}) {
    const double t = c_t + s * r;
    if (t0 < t && t < t1) brk.insert(t);
  }
  auto put = [&](CutPiece& P, double t, double wt, double a, double b) {
    std::vector<double> hs, wh;
    gauss_on(a, b, gx, gw, hs, wh);
    for (size_t k = 0; k < hs.size(); ++k) {
      double x[2];
      x[t_ax] = t;
      x[h_ax] = hs[k];
      P.x.push_back(x[0]);
      P.x.push_back(x[1]);
      P.w.push_back(wt * wh[k]);
    }
  };
  std::vector<double> bs(brk.begin(), brk.end());
  // Each interval graded by halving toward an end that one of the circle's
  // extreme points (square-root branch points of the chord's half-width and
  // of the arc's ds / dt) lies beyond or at, closer than the interval's length
  // (at most 40 halvings): the Gauss rules of the pieces then converge
  // exponentially.
  const double sing[2] = {c_t - r, c_t + r};
  std::vector<std::pair<double, double>> pieces;
  for (size_t m = 0; m + 1 < bs.size(); ++m) {
    const double a = bs[m], b = bs[m + 1];
    if (b - a <= 0) continue;
    const double L = b - a;
    std::set<double> cuts = {a, b};
    const double ends[2] = {a, b}, inward[2] = {1.0, -1.0};
    for (int side = 0; side < 2; ++side) {
      double d = std::numeric_limits<double>::infinity();
      for (double e : sing)
        if ((e - ends[side]) * inward[side] <= 0.0) d = std::min(d, std::fabs(e - ends[side]));
      if (d >= L) continue;
      double step = L;
      for (int lev = 0; lev < 40; ++lev) {
        step *= 0.5;
        cuts.insert(ends[side] + inward[side] * step);
        if (step <= d) break;
      }
    }
    std::vector<double> cv(cuts.begin(), cuts.end());
    for (size_t j = 0; j + 1 < cv.size(); ++j)
      if (cv[j + 1] > cv[j]) pieces.emplace_back(cv[j], cv[j + 1]);
  }
  for (const auto& pc : pieces) {
    const double a = pc.first, b = pc.second;
    std::vector<double> ts, wts;
    gauss_on(a, b, gx, gw, ts, wts);
    for (size_t k = 0; k < ts.size(); ++k) {
      const double t = ts[k], wt = wts[k];
      const double disc = r * r - (t - c_t) * (t - c_t);
      double lo_in = 0.0, hi_in = 0.0, w = 0.0;
      if (disc > 0) {
        w = std::sqrt(disc);
        lo_in = std::max(h0, c_h - w);
        hi_in = std::min(h1, c_h + w);
      }
      if (hi_in > lo_in) {
        put(in, t, wt, lo_in, hi_in);
        if (lo_in > h0) put(out, t, wt, h0, lo_in);
        if (h1 > hi_in) put(out, t, wt, hi_in, h1);
      } else {
        put(out, t, wt, h0, h1);
      }
      if (disc > 0)
        for (double s : {-1.0, 1.0}) {
          const double hv = c_h + s * w;
          if (h0 <= hv && hv <= h1) {
            const double dh = -s * (t - c_t) / w;
            double x[2];
            x[t_ax] = t;
            x[h_ax] = hv;
            const double vx = x[0] - C.c[0], vy = x[1] - C.c[1], nv = std::sqrt(vx * vx + vy * vy);
            arc.x.push_back(x[0]);
            arc.x.push_back(x[1]);
            arc.w.push_back(wt * std::sqrt(1.0 + dh * dh));
            arc.nrm.push_back(vx / nv);
            arc.nrm.push_back(vy / nv);
          }
        }
    }
  }
}

// Bounding box of the phase-ph piece of the cut cell [lo, hi]: along axis k
// the inside piece spans the coordinates whose line across the cell meets
// the disk, |x_k - c_k| < sqrt(r^2 - d^2) with d the distance from c to the
// cell's range on the other axis; the outside piece loses the coordinates
// whose whole line lies in the disk, |x_k - c_k| < sqrt(r^2 - D^2) with D the
// largest distance to that range, and keeps the hull of the rest.
void piece_box(const Circ& C, const double* lo, const double* hi, int ph, double* blo, double* bhi) {
  for (int k = 0; k < 2; ++k) {
    const int o = 1 - k;
    blo[k] = lo[k];
    bhi[k] = hi[k];
    if (ph == 1) {
      const double d = std::max(0.0, std::max(lo[o] - C.c[o], C.c[o] - hi[o]));
      const double a = std::sqrt(std::max(C.r * C.r - d * d, 0.0));
      blo[k] = std::max(lo[k], C.c[k] - a);
      bhi[k] = std::min(hi[k], C.c[k] + a);
    } else {
      const double D = std::max(std::fabs(lo[o] - C.c[o]), std::fabs(hi[o] - C.c[o]));
      if (C.r * C.r > D * D) {
        const double a = std::sqrt(C.r * C.r - D * D);
        if (C.c[k] - a <= lo[k] && lo[k] < C.c[k] + a) blo[k] = C.c[k] + a;
        if (C.c[k] - a < hi[k] && hi[k] <= C.c[k] + a) bhi[k] = C.c[k] - a;
      }
    }
  }
}

double sum_of(const std::vector<double>& w) {
  double a = 0.0;
  for (double v : w) a += v;
  return a;
}

}  // namespace

void cut_face_parts(const CutGeometry& G, double a, double b, int axis, double fixed, std::vector<double>* x,
                    std::vector<double>* w) {
  const Circ C{{G.c[0], G.c[1]}, G.r};
  std::vector<double> gx, gw;
  gauss_rule(G.q, gx, gw);
  const int o = 1 - axis;
  std::set<double> cuts = {a, b};
  const double disc = C.r * C.r - (fixed - C.c[axis]) * (fixed - C.c[axis]);
  if (disc > 0)
    for (double s : {-1.0, 1.0}) {
      const double v = C.c[o] + s * std::sqrt(disc);
      if (a < v && v < b) cuts.insert(v);
    }
  for (int ph = 0; ph < 2; ++ph) {
    x[ph].clear();
    w[ph].clear();
  }
  std::vector<double> cs(cuts.begin(), cuts.end());
  for (size_t m = 0; m + 1 < cs.size(); ++m) {
    const double u = cs[m], v = cs[m + 1];
    if (v <= u) continue;
    double mid[2];
    mid[axis] = fixed;
    mid[o] = 0.5 * (u + v);
    const int ph = C.phi(mid[0], mid[1]) < 0 ? 0 : 1;
    std::vector<double> ts, ws;
    gauss_on(u, v, gx, gw, ts, ws);
    for (size_t k = 0; k < ts.size(); ++k) {
      double p[2];
      p[axis] = fixed;
      p[o] = ts[k];
      x[ph].push_back(p[0]);
      x[ph].push_back(p[1]);
      w[ph].push_back(ws[k]);
    }
  }
}

void build_cut_geometry(CutGeometry& G, int n, const double* lo, const double* hi, double cx, double cy, double r,
                        int q, double frac, bool inside_only) {
  G = CutGeometry();
  G.inside_only = inside_only;
  G.n = n;
  G.q = q;
  G.frac = frac;
  G.c[0] = cx;
  G.c[1] = cy;
  G.r = r;
  for (int k = 0; k < 2; ++k) {
    G.lo[k] = lo[k];
    G.hi[k] = hi[k];
    G.h[k] = (hi[k] - lo[k]) / n;
  }
  const Circ C{{cx, cy}, r};
  std::vector<double> gx, gw;
  gauss_rule(q, gx, gw);
  auto add = [&](CutPiece&& P) {
    if (inside_only && P.ph != 1) return;
    P.area = sum_of(P.w);
    G.piece_of[((int64_t)P.j * n + P.i) * 4 + P.ph] = (int)G.pieces.size();
    G.pieces.push_back(std::move(P));
  };
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const double clo[2] = {lo[0] + G.h[0] * i, lo[1] + G.h[1] * j};
      const double chi[2] = {clo[0] + G.h[0], clo[1] + G.h[1]};
      const int k = classify(C, clo, chi);
      if (k != 0) {
        // the full cell: tensor Gauss rule, x fastest
        CutPiece P;
        P.i = i;
        P.j = j;
        P.ph = k < 0 ? 1 : 2;
        for (int a = 0; a < 2; ++a) {
          P.blo[a] = clo[a];
          P.bhi[a] = chi[a];
        }
        std::vector<double> xs, wx, ys, wy;
        gauss_on(clo[0], chi[0], gx, gw, xs, wx);
        gauss_on(clo[1], chi[1], gx, gw, ys, wy);
        for (int v = 0; v < q; ++v)
          for (int u = 0; u < q; ++u) {
            P.x.push_back(xs[u]);
            P.x.push_back(ys[v]);
            P.w.push_back(wy[v] * wx[u]);
          }
        add(std::move(P));
        continue;
      }
      CutPiece in, out;
      CutArc arc;
      in.i = out.i = arc.i = i;
      in.j = out.j = arc.j = j;
      in.ph = 1;
      out.ph = 2;
      cut_cell_rules(C, clo, chi, gx, gw, in, out, arc);
      piece_box(C, clo, chi, 1, in.blo, in.bhi);
      piece_box(C, clo, chi, 2, out.blo, out.bhi);
      add(std::move(in));
      add(std::move(out));
      G.arcs.push_back(std::move(arc));
    }
  // merging: a small piece joins the same-phase piece across the cell face
  // with the longest same-phase part, among neighbours not small themselves
  const int np = (int)G.pieces.size();
  const double cell_area = G.h[0] * G.h[1];
  G.element.resize(np);
  for (int k = 0; k < np; ++k) G.element[k] = k;
  std::vector<char> small(np);
  for (int k = 0; k < np; ++k) small[k] = G.pieces[k].area < frac * cell_area;
  for (int k = 0; k < np; ++k) {
    if (!small[k]) continue;
    const CutPiece& p = G.pieces[k];
    int best = -1;
    double best_len = -1.0;
    const int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (auto& dv : dd) {
      const int ii = p.i + dv[0], jj = p.j + dv[1];
      if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
      const int nb = G.find(ii, jj, p.ph);
      if (nb < 0 || small[nb]) continue;
      const double clo[2] = {lo[0] + G.h[0] * p.i, lo[1] + G.h[1] * p.j};
      std::vector<double> fx[2], fw[2];
      if (dv[0] != 0)
        cut_face_parts(G, clo[1], clo[1] + G.h[1], 0, clo[0] + (dv[0] > 0 ? G.h[0] : 0.0), fx, fw);
      else
        cut_face_parts(G, clo[0], clo[0] + G.h[0], 1, clo[1] + (dv[1] > 0 ? G.h[1] : 0.0), fx, fw);
      const double L = sum_of(fw[p.ph - 1]);
      if (L > best_len) {
        best = nb;
        best_len = L;
      }
    }
    if (best >= 0) G.element[k] = best;
  }
}

}  // namespace stk

using namespace stk;

extern "C" int stk_cut_cells(int n, const double* lo, const double* hi, double cx, double cy, double r, int q,
                             double merge_fraction, int64_t* npieces, int* cell, int* phase, double* area,
                             int* element, int* colour, double* interface_length) {
  if (n < 1 || n > 4096 || !lo || !hi || !(r > 0) || q < 1 || q > 32 || !(merge_fraction >= 0) || !npieces)
    return STK_ERR_INVALID_ARG;
  if (!(hi[0] > lo[0]) || !(hi[1] > lo[1])) return STK_ERR_INVALID_ARG;
  CutGeometry G;
  build_cut_geometry(G, n, lo, hi, cx, cy, r, q, merge_fraction);
  struct Piece {
    int i, j, ph;
    double area;
  };
  std::vector<Piece> pieces;
  for (const CutPiece& P : G.pieces) pieces.push_back({P.i, P.j, P.ph, P.area});
  double arc_total = 0.0;
  for (const CutArc& A : G.arcs) arc_total += sum_of(A.w);
  const int np = (int)pieces.size();
  const std::vector<int>& elem = G.element;
  // greedy colours of the elements (representatives in increasing order)
  std::vector<int> reps;
  for (int k = 0; k < np; ++k)
    if (elem[k] == k) reps.push_back(k);
  std::map<int, std::vector<std::pair<int, int>>> cells;      // rep -> host cells
  std::map<int64_t, std::vector<int>> owner;                   // cell -> reps
  for (int k = 0; k < np; ++k) {
    cells[elem[k]].push_back({pieces[k].i, pieces[k].j});
    owner[(int64_t)pieces[k].j * n + pieces[k].i].push_back(elem[k]);
  }
  const int stencil[13][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 0}, {0, 1}, {1, -1},
                              {1, 0},   {1, 1},  {2, 0},  {-2, 0}, {0, 2}, {0, -2}};
  std::map<int, int> col;
  for (int rep : reps) {
    std::set<int> used;
    for (auto& c : cells[rep])
      for (auto& o : stencil) {
        const int ii = c.first + o[0], jj = c.second + o[1];
        if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
        for (int other : owner[(int64_t)jj * n + ii])
          if (other != rep && col.count(other)) used.insert(col[other]);
      }
    int cc = 0;
    while (used.count(cc)) ++cc;
    col[rep] = cc;
  }
  const int64_t cap = *npieces;
  *npieces = np;
  if (interface_length) *interface_length = arc_total;
  if (cap < np) return STK_OK;   // sizes only
  for (int k = 0; k < np; ++k) {
    if (cell) {
      cell[2 * k] = pieces[k].i;
      cell[2 * k + 1] = pieces[k].j;
    }
    if (phase) phase[k] = pieces[k].ph;
    if (area) area[k] = pieces[k].area;
    if (element) element[k] = elem[k];
    if (colour) colour[k] = col[elem[k]];
  }
  return STK_OK;
}
