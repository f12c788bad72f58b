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

// Areas of the two pieces of a cut cell and the length of its interface arc.
void cut_cell(const Circ& C, const double* lo, const double* hi, const std::vector<double>& gx,
              const std::vector<double>& gw, double& a_in, double& a_out, double& arc) {
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
  const int q = (int)gx.size();
  auto interval = [&](double a, double b) {
    double sum = 0.0;   // length via the same Gauss weights as the oracle
    for (int k = 0; k < q; ++k) sum += 0.5 * (b - a) * gw[k];
    return sum;
  };
  a_in = a_out = arc = 0.0;
  std::vector<double> bs(brk.begin(), brk.end());
  for (size_t m = 0; m + 1 < bs.size(); ++m) {
    const double a = bs[m], b = bs[m + 1];
    if (b - a <= 0) continue;
    for (int k = 0; k < q; ++k) {
      const double t = 0.5 * (a + b) + 0.5 * (b - a) * gx[k], wt = 0.5 * (b - a) * gw[k];
      const double disc = r * r - (t - c_t) * (t - c_t);
      double lo_in = 0.0, hi_in = 0.0, w = 0.0;
      if (disc > 0) {
        w = std::sqrt(disc);
        lo_in = std::max(h0, c_h - w);
        hi_in = std::min(h1, c_h + w);
      }
      if (hi_in > lo_in) {
        a_in += wt * interval(lo_in, hi_in);
        if (lo_in > h0) a_out += wt * interval(h0, lo_in);
        if (h1 > hi_in) a_out += wt * interval(hi_in, h1);
      } else {
        a_out += wt * interval(h0, h1);
      }
      if (disc > 0)
        for (double s : {-1.0, 1.0}) {
          const double hv = c_h + s * w;
          if (h0 <= hv && hv <= h1) {
            const double dh = -s * (t - c_t) / w;
            arc += wt * std::sqrt(1.0 + dh * dh);
          }
        }
    }
  }
}

// Length of the phase-ph part of the face {x_axis = fixed, other in [a, b]}.
double face_part_length(const Circ& C, double a, double b, int axis, double fixed, int ph,
                        const std::vector<double>& gw) {
  const int o = 1 - axis;
  std::set<double> cuts = {a, b};
  const double disc = C.r * C.r - (fixed - C.c[axis]) * (fixed - C.c[axis]);
  if (disc > 0)
    for (double s : {-1.0, 1.0}) {
      const double v = C.c[o] + s * std::sqrt(disc);
      if (a < v && v < b) cuts.insert(v);
    }
  std::vector<double> cs(cuts.begin(), cuts.end());
  double len = 0.0;
  for (size_t m = 0; m + 1 < cs.size(); ++m) {
    const double u = cs[m], v = cs[m + 1];
    if (v <= u) continue;
    double mid[2];
    mid[axis] = fixed;
    mid[o] = 0.5 * (u + v);
    const int p = C.phi(mid[0], mid[1]) < 0 ? 1 : 2;
    if (p != ph) continue;
    for (double w : gw) len += 0.5 * (v - u) * w;
  }
  return len;
}

}  // namespace

}  // namespace stk

using namespace stk;

extern "C" int stk_cut_cells(int n, const double* lo, const double* hi, double cx, double cy, double r, int q,
                             double merge_fraction, int64_t* npieces, int* cell, int* phase, double* area,
                             int* element, int* colour, double* interface_length) {
  if (n < 1 || n > 4096 || !lo || !hi || !(r > 0) || q < 1 || q > 32 || !(merge_fraction >= 0) || !npieces)
    return STK_ERR_INVALID_ARG;
  if (!(hi[0] > lo[0]) || !(hi[1] > lo[1])) return STK_ERR_INVALID_ARG;
  const Circ C{{cx, cy}, r};
  std::vector<double> gx, gw;
  gauss_rule(q, gx, gw);
  const double hx = (hi[0] - lo[0]) / n, hy = (hi[1] - lo[1]) / n, cell_area = hx * hy;
  struct Piece {
    int i, j, ph;
    double area;
  };
  std::vector<Piece> pieces;
  std::map<int64_t, int> piece_of;   // (cell, phase) -> piece
  double arc_total = 0.0;
  auto key = [n](int i, int j, int ph) { return ((int64_t)j * n + i) * 4 + ph; };
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const double clo[2] = {lo[0] + hx * i, lo[1] + hy * j}, chi[2] = {clo[0] + hx, clo[1] + hy};
      const int k = classify(C, clo, chi);
      if (k != 0) {
        // the full cell: the tensor rule's weights sum to the cell's area
        double a = 0.0;
        for (int u = 0; u < q; ++u)
          for (int v = 0; v < q; ++v) a += 0.5 * hx * gw[v] * 0.5 * hy * gw[u];
        piece_of[key(i, j, k < 0 ? 1 : 2)] = (int)pieces.size();
        pieces.push_back({i, j, k < 0 ? 1 : 2, a});
        continue;
      }
      double a_in, a_out, arc;
      cut_cell(C, clo, chi, gx, gw, a_in, a_out, arc);
      arc_total += arc;
      piece_of[key(i, j, 1)] = (int)pieces.size();
      pieces.push_back({i, j, 1, a_in});
      piece_of[key(i, j, 2)] = (int)pieces.size();
      pieces.push_back({i, j, 2, a_out});
    }
  const int np = (int)pieces.size();
  // merging
  std::vector<int> elem(np);
  for (int k = 0; k < np; ++k) elem[k] = k;
  std::vector<char> small(np);
  for (int k = 0; k < np; ++k) small[k] = pieces[k].area < merge_fraction * cell_area;
  for (int k = 0; k < np; ++k) {
    if (!small[k]) continue;
    const Piece& p = pieces[k];
    int best = -1;
    double best_len = -1.0;
    const int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (auto& dv : dd) {
      const int ii = p.i + dv[0], jj = p.j + dv[1];
      if (ii < 0 || ii >= n || jj < 0 || jj >= n) continue;
      auto it = piece_of.find(key(ii, jj, p.ph));
      if (it == piece_of.end() || small[it->second]) continue;
      const double clo[2] = {lo[0] + hx * p.i, lo[1] + hy * p.j};
      double L;
      if (dv[0] != 0)
        L = face_part_length(C, clo[1], clo[1] + hy, 0, clo[0] + (dv[0] > 0 ? hx : 0.0), p.ph, gw);
      else
        L = face_part_length(C, clo[0], clo[0] + hx, 1, clo[1] + (dv[1] > 0 ? hy : 0.0), p.ph, gw);
      if (L > best_len) {
        best = it->second;
        best_len = L;
      }
    }
    if (best >= 0) elem[k] = best;
  }
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
