// Cut-cell problems of an embedded circle (host setup): the LDG operators of
// Appendix A on the merged cut-cell elements (Section 5's circular interface),
// the multigrid hierarchy by same-phase agglomeration with Algorithm 2
// (steady) or Algorithm 3 (unsteady) on every level, the Stokes blocks of eq.
// (blockform) / (timedep2) with the Section 5.6 scaling, the smoother
// colouring, the sample points of the data and the right-hand side.
//
//  * Element basis: the tensor Legendre basis Q_p on the element's bounding
//    box (the hull of its pieces' bounding boxes); the element mass matrix
//    M_E = int_E phi_a phi_b is a dense block.  Every integral runs on the
//    cut-cell rules of cutcell.cpp.
//  * G_k = M^{-1}(B_k + L_k): the broken derivative plus the lift of eq.
//    (gsum) -- on an intraphase face (normal +e_k from the left element to the
//    right one) into the right element's rows; -int u v n_k on the Dirichlet
//    box; on the circle (normal out of it, from phase 1 into phase 2) split
//    (1 - lambda) into the phase-1 element and lambda into the phase-2
//    element with lambda of eq. (viscosityupwind).
//  * Penalties: tau_bdry = c_bdry p mu / h on the box and
//    tau_ij = 3 p min(mu-, mu+) / h on the circle (E~, eq. Epenalty); the
//    pressure penalty tau h / mu (eq. eop) on intraphase faces, or eq.
//    (taupgeneral) 1 / (h rho / (tau0 delta) + mu / (tau h)) for an unsteady
//    problem with its two limits kept for Algorithm 3.
//  * Coarse elements: the elements of a level grouped by the parent cell
//    (halved grid) of their anchor cell and by phase (the anchor of a merged
//    element is the host cell of its representative piece); the coarse basis
//    lives on the union of the members' boxes, and the injection onto a member
//    f re-expands the coarse polynomial in the member's basis (the L2
//    projection over the member's box, exact for Q_p).
//  * Colouring: greedy, elements in index order, each the smallest colour not
//    used by an already coloured element it is structurally coupled with:
//    the level's field operators couple elements one face / interface step
//    apart (on a coarse level, groups with members one step apart) and
//    G^T M G reaches two steps, so the graph is the square of the one-step
//    graph.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <functional>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "stk_internal.h"
#include "../../include/stokes_mg.h"

namespace stk {

namespace {

using Blk = std::vector<double>;

// Sparse matrix of s x s blocks (row-major blocks), rows of element blocks.
struct BMat {
  int ne = 0, s = 0;
  std::vector<std::map<int, Blk>> row;
  BMat() = default;
  BMat(int n, int s_) : ne(n), s(s_), row(n) {}
  double* at(int i, int j) {
    auto it = row[i].find(j);
    if (it == row[i].end()) it = row[i].emplace(j, Blk((size_t)s * s, 0.0)).first;
    return it->second.data();
  }
  const double* get(int i, int j) const {
    auto it = row[i].find(j);
    return it == row[i].end() ? nullptr : it->second.data();
  }
};

// C += alpha op(A) B with op(A) = A or A^T (s x s row-major)
void mm(int s, double alpha, const double* A, bool ta, const double* B, double* C) {
  for (int i = 0; i < s; ++i)
    for (int k = 0; k < s; ++k) {
      const double a = alpha * (ta ? A[k * s + i] : A[i * s + k]);
      const double* b = B + (size_t)k * s;
      double* c = C + (size_t)i * s;
      for (int j = 0; j < s; ++j) c[j] += a * b[j];
    }
}

// C += alpha A op(B) with op(B) = B or B^T
void mm_r(int s, double alpha, const double* A, const double* B, bool tb, double* C) {
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int k = 0; k < s; ++k) acc += A[i * s + k] * (tb ? B[j * s + k] : B[k * s + j]);
      C[i * s + j] += alpha * acc;
    }
}

// X^T diag(w) Y for point tables X [m][s], Y [m][s]
void weighted(int m, int s, const double* X, const double* Y, const double* w, double alpha, double* out) {
  for (int k = 0; k < m; ++k) {
    const double wk = alpha * w[k];
    for (int a = 0; a < s; ++a) {
      const double xa = wk * X[(size_t)k * s + a];
      for (int b = 0; b < s; ++b) out[(size_t)a * s + b] += xa * Y[(size_t)k * s + b];
    }
  }
}

BMat transpose(const BMat& A) {
  BMat T(A.ne, A.s);
  for (int i = 0; i < A.ne; ++i)
    for (auto& kv : A.row[i]) {
      double* t = T.at(kv.first, i);
      for (int a = 0; a < A.s; ++a)
        for (int b = 0; b < A.s; ++b) t[b * A.s + a] = kv.second[a * A.s + b];
    }
  return T;
}

// out(i, j) = Dg[i] A(i, j) (left) or A(i, j) Dg[j] (right), Dg block diagonal
BMat diag_mul(const std::vector<Blk>& Dg, const BMat& A, bool left) {
  BMat C(A.ne, A.s);
  parallel_for(A.ne, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      for (auto& kv : A.row[i]) {
        Blk out((size_t)A.s * A.s, 0.0);
        if (left)
          mm(A.s, 1.0, Dg[i].data(), false, kv.second.data(), out.data());
        else
          mm(A.s, 1.0, kv.second.data(), false, Dg[kv.first].data(), out.data());
        C.row[i].emplace(kv.first, std::move(out));
      }
  });
  return C;
}

std::vector<Blk> diag_blocks(const BMat& A) {
  std::vector<Blk> D(A.ne, Blk((size_t)A.s * A.s, 0.0));
  for (int i = 0; i < A.ne; ++i) {
    const double* d = A.get(i, i);
    if (d) std::copy(d, d + (size_t)A.s * A.s, D[i].begin());
  }
  return D;
}

std::vector<Blk> diag_inverse(const BMat& A) {
  std::vector<Blk> D = diag_blocks(A);
  std::vector<double> in((size_t)A.ne * A.s * A.s), out(in.size());
  for (int i = 0; i < A.ne; ++i) std::copy(D[i].begin(), D[i].end(), in.begin() + (size_t)i * A.s * A.s);
  std::string err;
  if (invert_blocks(A.s, A.ne, in.data(), out.data(), err) != STK_OK) throw std::runtime_error("mass matrix: " + err);
  for (int i = 0; i < A.ne; ++i) std::copy(out.begin() + (size_t)i * A.s * A.s, out.begin() + (size_t)(i + 1) * A.s * A.s, D[i].begin());
  return D;
}

// Coarse operator I^T A I with I block diagonal per fine element:
// (I^T A I)(parent(i), parent(j)) += I_i^T A(i, j) I_j.
BMat galerkin(const BMat& A, const std::vector<int>& parent, const std::vector<double>& Ib,
              const std::vector<std::vector<int>>& children, double alpha) {
  const int s = A.s, ss = s * s, nc = (int)children.size();
  BMat C(nc, s);
  parallel_for(nc, [&](int64_t c0, int64_t c1) {
    Blk tmp(ss);
    for (int64_t c = c0; c < c1; ++c)
      for (int f : children[c])
        for (auto& kv : A.row[f]) {
          std::fill(tmp.begin(), tmp.end(), 0.0);
          mm(s, 1.0, &Ib[(size_t)f * ss], true, kv.second.data(), tmp.data());   // I_f^T A
          auto it = C.row[c].find(parent[kv.first]);
          if (it == C.row[c].end()) it = C.row[c].emplace(parent[kv.first], Blk(ss, 0.0)).first;
          mm_r(s, alpha, tmp.data(), &Ib[(size_t)kv.first * ss], false, it->second.data());
        }
  });
  return C;
}

// The LDG operators of one level (field blocks per element pair).
struct Ops {
  int ne = 0, s = 0;
  bool unsteady = false;
  BMat M, Mmu, Mrho, Et, E, Emu, Erho;
  BMat G[2];
  std::vector<Blk> Minv;
};

// eq. (Etimedep): per element pair, E = (|Erho| / (|Emu| + |Erho|))^2 Emu +
// (|Emu| / (|Emu| + |Erho|))^2 Erho with Frobenius norms.
BMat combine_penalty(const BMat& Emu, const BMat& Erho) {
  const int s = Emu.s, ss = s * s;
  BMat E(Emu.ne, s);
  for (int i = 0; i < Emu.ne; ++i) {
    std::set<int> cols;
    for (auto& kv : Emu.row[i]) cols.insert(kv.first);
    for (auto& kv : Erho.row[i]) cols.insert(kv.first);
    for (int j : cols) {
      const double* a = Emu.get(i, j);
      const double* b = Erho.get(i, j);
      double fm = 0, fr = 0;
      for (int k = 0; k < ss; ++k) {
        if (a) fm += a[k] * a[k];
        if (b) fr += b[k] * b[k];
      }
      fm = std::sqrt(fm);
      fr = std::sqrt(fr);
      const double tot = fm + fr;
      const double wm = tot > 0 ? (fr / tot) * (fr / tot) : 0.0, wr = tot > 0 ? (fm / tot) * (fm / tot) : 0.0;
      double* e = E.at(i, j);
      for (int k = 0; k < ss; ++k) e[k] = (a ? wm * a[k] : 0.0) + (b ? wr * b[k] : 0.0);
    }
  }
  return E;
}

struct Face {
  int ea, eb, axis, side;                 // intra: left, right element; boundary: element, -, axis, side
  std::vector<double> x, w, nrm;
};

}  // namespace

// Cut-cell state kept between setup and the right-hand side: elements,
// faces and the finest level's operators.
struct CutState {
  int ne = 0, s = 0, p = 0;
  std::vector<int> reps, of_piece, phase;
  std::vector<std::vector<int>> pieces;   // element -> pieces
  std::vector<double> box_lo, box_hi;     // [ne][2]
  std::vector<Face> intra, bdry, arcs;    // arcs: ea phase-1 element, eb phase-2 element
  Ops fine;
};

namespace {

void box_basis(int p, const double* a, const double* b, const double* x, int m, double* Phi, double* Dx,
               double* Dy) {
  const int p1 = p + 1, s = p1 * p1;
  const double sx = 2.0 / (b[0] - a[0]), sy = 2.0 / (b[1] - a[1]);
  for (int k = 0; k < m; ++k) {
    double v0[16], d0[16], v1[16], d1[16];
    psi_eval(p, (2 * x[2 * k] - (a[0] + b[0])) / (b[0] - a[0]), v0, d0);
    psi_eval(p, (2 * x[2 * k + 1] - (a[1] + b[1])) / (b[1] - a[1]), v1, d1);
    for (int a1 = 0; a1 < p1; ++a1)
      for (int a0 = 0; a0 < p1; ++a0) {
        const int md = a0 + p1 * a1;
        Phi[(size_t)k * s + md] = v0[a0] * v1[a1];
        if (Dx) Dx[(size_t)k * s + md] = d0[a0] * sx * v1[a1];
        if (Dy) Dy[(size_t)k * s + md] = v0[a0] * d1[a1] * sy;
      }
  }
}

void elements_of(const CutGeometry& G, int p, CutState& S) {
  S.p = p;
  S.s = (p + 1) * (p + 1);
  std::set<int> rs(G.element.begin(), G.element.end());
  S.reps.assign(rs.begin(), rs.end());
  std::map<int, int> index;
  for (size_t e = 0; e < S.reps.size(); ++e) index[S.reps[e]] = (int)e;
  S.ne = (int)S.reps.size();
  S.of_piece.resize(G.pieces.size());
  S.pieces.assign(S.ne, {});
  for (size_t k = 0; k < G.pieces.size(); ++k) {
    S.of_piece[k] = index[G.element[k]];
    S.pieces[S.of_piece[k]].push_back((int)k);
  }
  S.phase.resize(S.ne);
  S.box_lo.resize(2 * S.ne);
  S.box_hi.resize(2 * S.ne);
  for (int e = 0; e < S.ne; ++e) {
    S.phase[e] = G.pieces[S.reps[e]].ph;
    // the hull of the pieces' bounding boxes
    for (int a = 0; a < 2; ++a) {
      S.box_lo[2 * e + a] = 1e300;
      S.box_hi[2 * e + a] = -1e300;
    }
    for (int k : S.pieces[e])
      for (int a = 0; a < 2; ++a) {
        S.box_lo[2 * e + a] = std::min(S.box_lo[2 * e + a], G.pieces[k].blo[a]);
        S.box_hi[2 * e + a] = std::max(S.box_hi[2 * e + a], G.pieces[k].bhi[a]);
      }
  }
}

std::vector<double> side_normals(int axis, int side, size_t m) {
  std::vector<double> nrm(2 * m, 0.0);
  for (size_t k = 0; k < m; ++k) nrm[2 * k + axis] = side;
  return nrm;
}

// Intraphase faces, Dirichlet faces (box sides with their outward normals, and
// the circle with its outward normal when it bounds the domain: axis -1) and
// interface arcs, cells in order.
void faces_of(const CutGeometry& G, CutState& S) {
  const int n = G.n;
  S.intra.clear();
  S.bdry.clear();
  S.arcs.clear();
  size_t arc_i = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const double clo[2] = {G.lo[0] + G.h[0] * i, G.lo[1] + G.h[1] * j};
      for (int axis = 0; axis < 2; ++axis) {
        const int o = 1 - axis;
        const int ii = axis == 0 ? i + 1 : i, jj = axis == 0 ? j : j + 1;
        std::vector<double> px[2], pw[2];
        cut_face_parts(G, clo[o], clo[o] + G.h[o], axis, clo[axis] + G.h[axis], px, pw);
        for (int ph = 1; ph <= 2; ++ph) {
          if (pw[ph - 1].empty()) continue;
          if (ii < n && jj < n) {
            const int a = G.find(i, j, ph), b = G.find(ii, jj, ph);
            if (a < 0 || b < 0) continue;
            const int ea = S.of_piece[a], eb = S.of_piece[b];
            if (ea != eb) S.intra.push_back({ea, eb, axis, 0, px[ph - 1], pw[ph - 1], {}});
          } else {
            const int a = G.find(i, j, ph);
            if (a < 0) {
              if (G.inside_only) continue;
              throw std::runtime_error("boundary face part without a piece");
            }
            S.bdry.push_back({S.of_piece[a], -1, axis, 1, px[ph - 1], pw[ph - 1], side_normals(axis, 1, pw[ph - 1].size())});
          }
        }
        if ((axis == 0 && i == 0) || (axis == 1 && j == 0)) {
          cut_face_parts(G, clo[o], clo[o] + G.h[o], axis, clo[axis], px, pw);
          for (int ph = 1; ph <= 2; ++ph) {
            if (pw[ph - 1].empty()) continue;
            const int a = G.find(i, j, ph);
            if (a < 0) {
              if (G.inside_only) continue;
              throw std::runtime_error("boundary face part without a piece");
            }
            S.bdry.push_back({S.of_piece[a], -1, axis, -1, px[ph - 1], pw[ph - 1],
                              side_normals(axis, -1, pw[ph - 1].size())});
          }
        }
      }
      if (arc_i < G.arcs.size() && G.arcs[arc_i].i == i && G.arcs[arc_i].j == j) {
        const CutArc& A = G.arcs[arc_i++];
        if (!A.w.empty()) {
          const int in = S.of_piece[G.find(i, j, 1)];
          const int out = G.find(i, j, 2);
          if (out < 0)   // the circle bounds the domain: a Dirichlet face of the inside element
            S.bdry.push_back({in, -1, -1, 0, A.x, A.w, A.nrm});
          else
            S.arcs.push_back({in, S.of_piece[out], -1, 0, A.x, A.w, A.nrm});
        }
      }
    }
}

// Appendix A on the merged elements.
void fine_operators(const Ctx& c, const CutGeometry& G, CutState& S) {
  const int ne = S.ne, s = S.s, p = S.p, ss = s * s;
  const double hk = G.h[0];
  const bool unsteady = c.cut_delta > 0;
  auto mu = [&](int e) { return c.mu_phase[S.phase[e] - 1]; };
  auto rho = [&](int e) { return unsteady ? c.rho_phase[S.phase[e] - 1] : 1.0; };
  Ops& O = S.fine;
  O.ne = ne;
  O.s = s;
  O.unsteady = unsteady;
  O.M = BMat(ne, s);
  O.Mmu = BMat(ne, s);
  O.Mrho = BMat(ne, s);
  O.Et = BMat(ne, s);
  O.E = BMat(ne, s);
  O.Emu = BMat(ne, s);
  O.Erho = BMat(ne, s);
  BMat g[2] = {BMat(ne, s), BMat(ne, s)};
  auto phi = [&](int e, const std::vector<double>& x, std::vector<double>& Phi, std::vector<double>* D) {
    const int m = (int)x.size() / 2;
    Phi.assign((size_t)m * s, 0.0);
    if (D) {
      D[0].assign((size_t)m * s, 0.0);
      D[1].assign((size_t)m * s, 0.0);
    }
    box_basis(p, &S.box_lo[2 * e], &S.box_hi[2 * e], x.data(), m, Phi.data(), D ? D[0].data() : nullptr,
              D ? D[1].data() : nullptr);
  };
  // element mass matrices and broken derivatives
  for (int e = 0; e < ne; ++e) {
    Blk M(ss, 0.0), B0(ss, 0.0), B1(ss, 0.0);
    for (int k : S.pieces[e]) {
      const CutPiece& P = G.pieces[k];
      std::vector<double> Phi, D[2];
      phi(e, P.x, Phi, D);
      const int m = (int)P.w.size();
      weighted(m, s, Phi.data(), Phi.data(), P.w.data(), 1.0, M.data());
      weighted(m, s, Phi.data(), D[0].data(), P.w.data(), 1.0, B0.data());
      weighted(m, s, Phi.data(), D[1].data(), P.w.data(), 1.0, B1.data());
    }
    std::copy(M.begin(), M.end(), O.M.at(e, e));
    double* mm_ = O.Mmu.at(e, e);
    for (int k = 0; k < ss; ++k) mm_[k] = mu(e) * M[k];
    if (unsteady) {
      double* mr = O.Mrho.at(e, e);
      for (int k = 0; k < ss; ++k) mr[k] = rho(e) * M[k];
    }
    double* g0 = g[0].at(e, e);
    double* g1 = g[1].at(e, e);
    for (int k = 0; k < ss; ++k) {
      g0[k] += B0[k];
      g1[k] += B1[k];
    }
  }
  auto add = [&](BMat& A, int i, int j, double alpha, const std::vector<double>& X, const std::vector<double>& Y,
                 const std::vector<double>& w) {
    weighted((int)w.size(), s, X.data(), Y.data(), w.data(), alpha, A.at(i, j));
  };
  for (const Face& F : S.intra) {
    std::vector<double> Pa, Pb;
    phi(F.ea, F.x, Pa, nullptr);
    phi(F.eb, F.x, Pb, nullptr);
    // lift into the right (+) element: int (u+ - u-) v+
    add(g[F.axis], F.eb, F.eb, 1.0, Pb, Pb, F.w);
    add(g[F.axis], F.eb, F.ea, -1.0, Pb, Pa, F.w);
    std::vector<std::pair<BMat*, double>> coefs;
    if (unsteady) {
      const double m_ = mu(F.ea), r_ = rho(F.ea);
      coefs.push_back({&O.E, 1.0 / (hk * r_ / (c.tau0 * c.cut_delta) + m_ / (c.tau * hk))});
      coefs.push_back({&O.Emu, c.tau * hk / m_});
      coefs.push_back({&O.Erho, c.tau0 * c.cut_delta / (hk * r_)});
    } else {
      coefs.push_back({&O.E, c.tau * hk / mu(F.ea)});
    }
    for (auto& cf : coefs) {
      add(*cf.first, F.ea, F.ea, cf.second, Pa, Pa, F.w);
      add(*cf.first, F.eb, F.eb, cf.second, Pb, Pb, F.w);
      add(*cf.first, F.ea, F.eb, -cf.second, Pa, Pb, F.w);
      add(*cf.first, F.eb, F.ea, -cf.second, Pb, Pa, F.w);
    }
  }
  for (const Face& F : S.bdry) {
    std::vector<double> P;
    phi(F.ea, F.x, P, nullptr);
    if (F.axis >= 0) {
      add(g[F.axis], F.ea, F.ea, -(double)F.side, P, P, F.w);
    } else {
      // curved Dirichlet boundary: -int u v n_k with the outward normal
      for (int k = 0; k < 2; ++k) {
        std::vector<double> wn(F.w.size());
        for (size_t q = 0; q < F.w.size(); ++q) wn[q] = F.w[q] * F.nrm[2 * q + k];
        add(g[k], F.ea, F.ea, -1.0, P, P, wn);
      }
    }
    add(O.Et, F.ea, F.ea, c.c_bdry * p * mu(F.ea) / hk, P, P, F.w);
  }
  for (const Face& F : S.arcs) {
    std::vector<double> Pm, Pp;
    phi(F.ea, F.x, Pm, nullptr);
    phi(F.eb, F.x, Pp, nullptr);
    const double mum = mu(F.ea), mup = mu(F.eb);
    const double lam = mum < mup ? 0.0 : (mum > mup ? 1.0 : 0.5);
    for (int axis = 0; axis < 2; ++axis) {
      std::vector<double> wn(F.w.size());
      for (size_t k = 0; k < F.w.size(); ++k) wn[k] = F.w[k] * F.nrm[2 * k + axis];
      add(g[axis], F.ea, F.eb, 1.0 - lam, Pm, Pp, wn);
      add(g[axis], F.ea, F.ea, -(1.0 - lam), Pm, Pm, wn);
      add(g[axis], F.eb, F.eb, lam, Pp, Pp, wn);
      add(g[axis], F.eb, F.ea, -lam, Pp, Pm, wn);
    }
    const double tij = 3.0 * p * std::min(mum, mup) / hk;
    add(O.Et, F.ea, F.ea, tij, Pm, Pm, F.w);
    add(O.Et, F.ea, F.eb, -tij, Pm, Pp, F.w);
    add(O.Et, F.eb, F.ea, -tij, Pp, Pm, F.w);
    add(O.Et, F.eb, F.eb, tij, Pp, Pp, F.w);
  }
  O.Minv = diag_inverse(O.M);
  for (int k = 0; k < 2; ++k) O.G[k] = diag_mul(O.Minv, g[k], true);
}

// Algorithm 2 (steady) / Algorithm 3 (unsteady) applied once.
Ops coarsen(const Ops& F, const std::vector<int>& parent, const std::vector<double>& Ib,
            const std::vector<std::vector<int>>& children) {
  Ops C;
  C.ne = (int)children.size();
  C.s = F.s;
  C.unsteady = F.unsteady;
  C.M = galerkin(F.M, parent, Ib, children, 1.0);
  C.Minv = diag_inverse(C.M);
  C.Mmu = galerkin(F.Mmu, parent, Ib, children, 1.0);
  const std::vector<Blk> Mf = diag_blocks(F.M);
  for (int k = 0; k < 2; ++k) {
    BMat Y = diag_mul(Mf, F.G[k], true);
    C.G[k] = diag_mul(C.Minv, galerkin(Y, parent, Ib, children, 1.0), true);
  }
  C.Et = galerkin(F.Et, parent, Ib, children, 0.5);
  if (F.unsteady) {
    C.Mrho = galerkin(F.Mrho, parent, Ib, children, 1.0);
    C.Emu = galerkin(F.Emu, parent, Ib, children, 2.0);
    C.Erho = galerkin(F.Erho, parent, Ib, children, 0.5);
    C.E = combine_penalty(C.Emu, C.Erho);
  } else {
    C.Mrho = BMat(C.ne, C.s);
    C.Emu = BMat(C.ne, C.s);
    C.Erho = BMat(C.ne, C.s);
    C.E = galerkin(F.E, parent, Ib, children, 2.0);
  }
  return C;
}

// The Stokes operator of eq. (blockform) / (timedep2) of one level, element
// by element, with the sqrt(mu) scaling when enabled, into the general
// block-sparse form of HostLevel (diagonal blocks D, coupling tasks).
void stokes_blocks(const Ctx& c, const Ops& O, HostLevel& L) {
  const int ne = O.ne, s = O.s, ss = s * s, nb = 3 * s;
  const double gam = c.gamma;
  const std::vector<Blk> Md = diag_blocks(O.M);
  const std::vector<Blk> Mmud = diag_blocks(O.Mmu);
  BMat Gt[2] = {transpose(O.G[0]), transpose(O.G[1])};
  BMat H[2] = {diag_mul(Mmud, O.G[0], true), diag_mul(Mmud, O.G[1], true)};   // Mmu G_i
  L.ne = ne;
  // scaling D (Section 5.6): mu_E = Mmu(E)[0][0] / M(E)[0][0]
  L.Dscale.clear();
  if (c.scale_mu) {
    L.Dscale.resize((size_t)ne * nb);
    for (int e = 0; e < ne; ++e) {
      const double mue = Mmud[e][0] / Md[e][0];
      for (int r = 0; r < nb; ++r) L.Dscale[(size_t)e * nb + r] = r < 2 * s ? 1.0 / std::sqrt(mue) : std::sqrt(mue);
    }
  }
  // rows in parallel: per element row, a map neighbour -> 3 x 3 sub-blocks
  std::vector<std::vector<int>> nbrs(ne);
  std::vector<std::vector<std::array<Blk, 9>>> blocks(ne);   // per neighbour: 3 x 3 sub-blocks (empty = absent)
  parallel_for(ne, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      std::map<int, std::array<Blk, 9>> row;
      auto sub = [&](int f, int rv, int cv) -> double* {
        Blk& b = row[f][rv * 3 + cv];
        if (b.empty()) b.assign(ss, 0.0);
        return b.data();
      };
      // velocity-velocity: gamma G_j^T Mmu G_i (rv = i, cv = j) plus, on the
      // diagonal variable blocks, sum_k G_k^T Mmu G_k + E~ (+ Mrho / delta)
      Blk prod(ss);
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (auto& a : Gt[j].row[e])           // G_j^T(e, m)
            for (auto& b : H[i].row[a.first]) {   // Mmu G_i(m, f)
              std::fill(prod.begin(), prod.end(), 0.0);
              mm(s, 1.0, a.second.data(), false, b.second.data(), prod.data());
              if (gam != 0.0) {
                double* t = sub(b.first, i, j);
                for (int k = 0; k < ss; ++k) t[k] += gam * prod[k];
              }
              // the Laplacian sum_k G_k^T Mmu G_k on both velocity diagonal blocks
              if (i == j)
                for (int v = 0; v < 2; ++v) {
                  double* t = sub(b.first, v, v);
                  for (int k = 0; k < ss; ++k) t[k] += prod[k];
                }
            }
      auto add_all = [&](const BMat& A, double alpha, int rv, int cv) {
        for (auto& kv : A.row[e]) {
          double* t = sub(kv.first, rv, cv);
          for (int k = 0; k < ss; ++k) t[k] += alpha * kv.second[k];
        }
      };
      for (int v = 0; v < 2; ++v) {
        add_all(O.Et, 1.0, v, v);
        if (O.unsteady) add_all(O.Mrho, 1.0 / c.cut_delta, v, v);
      }
      // velocity-pressure: -G_i^T M ; pressure-velocity: -M G_j ; pressure: -E
      for (int i = 0; i < 2; ++i) {
        for (auto& kv : Gt[i].row[e]) {
          double* t = sub(kv.first, i, 2);
          mm(s, -1.0, kv.second.data(), false, Md[kv.first].data(), t);
        }
        for (auto& kv : O.G[i].row[e]) {
          double* t = sub(kv.first, 2, i);
          mm(s, -1.0, Md[e].data(), false, kv.second.data(), t);
        }
      }
      add_all(O.E, -1.0, 2, 2);
      for (auto& kv : row) {
        nbrs[e].push_back(kv.first);
        blocks[e].push_back(std::move(kv.second));
      }
    }
  });
  // element-major assembly, scaling, tasks: scale and count in parallel,
  // then place every element's tasks at its prefix offset
  L.D.assign((size_t)ne * nb * nb, 0.0);
  std::vector<int> count(ne, 0);
  parallel_for(ne, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      for (size_t k = 0; k < nbrs[e].size(); ++k) {
        const int f = nbrs[e][k];
        for (int v = 0; v < 9; ++v) {
          Blk& B = blocks[e][k][v];
          if (B.empty()) continue;
          const int rv = v / 3, cv = v % 3;
          if (!L.Dscale.empty())
            for (int a = 0; a < s; ++a)
              for (int bb = 0; bb < s; ++bb)
                B[a * s + bb] *= L.Dscale[(size_t)e * nb + rv * s + a] * L.Dscale[(size_t)f * nb + cv * s + bb];
          if (f == e) {
            for (int a = 0; a < s; ++a)
              for (int bb = 0; bb < s; ++bb) L.D[((size_t)e * nb + rv * s + a) * nb + cv * s + bb] = B[a * s + bb];
            Blk().swap(B);
            continue;
          }
          bool nz = false;
          for (int q = 0; q < ss && !nz; ++q) nz = B[q] != 0.0;
          if (nz)
            ++count[e];
          else
            Blk().swap(B);
        }
      }
  });
  L.tptr.assign(ne + 1, 0);
  for (int e = 0; e < ne; ++e) L.tptr[e + 1] = L.tptr[e] + count[e];
  const size_t nt = (size_t)L.tptr[ne];
  L.tnbr.assign(nt, 0);
  L.tvar.assign(nt, 0);
  L.C.assign(nt * ss, 0.0);
  parallel_for(ne, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      size_t t = (size_t)L.tptr[e];
      for (size_t k = 0; k < nbrs[e].size(); ++k)
        for (int v = 0; v < 9; ++v) {
          Blk& B = blocks[e][k][v];
          if (B.empty()) continue;
          L.tnbr[t] = nbrs[e][k];
          L.tvar[t] = (v / 3) * 4 + v % 3;
          std::copy(B.begin(), B.end(), L.C.begin() + t * ss);
          ++t;
          Blk().swap(B);
        }
    }
  });
}

std::vector<int> greedy(const std::vector<std::set<int>>& S) {
  const int ne = (int)S.size();
  std::vector<int> col(ne, -1);
  for (int e = 0; e < ne; ++e) {
    std::set<int> used;
    for (int j : S[e])
      if (j != e && col[j] >= 0) used.insert(col[j]);
    int cc = 0;
    while (used.count(cc)) ++cc;
    col[e] = cc;
  }
  return col;
}

bool same_geometry(const CutGeometry& G, const Ctx& c) {
  return G.n == c.n[0] && G.q == c.q && G.lo[0] == c.lo[0] && G.lo[1] == c.lo[1] && G.hi[0] == c.hi[0] &&
         G.hi[1] == c.hi[1] && G.c[0] == c.cut_c[0] && G.c[1] == c.cut_c[1] && G.r == c.cut_r && G.frac == c.cut_frac &&
         G.inside_only == (c.cut_inside != 0);
}

}  // namespace

const CutGeometry& cut_geometry(Ctx& c) {
  if (!c.cutg || !same_geometry(*c.cutg, c)) {
    auto G = std::make_shared<CutGeometry>();
    build_cut_geometry(*G, c.n[0], c.lo, c.hi, c.cut_c[0], c.cut_c[1], c.cut_r, c.q, c.cut_frac, c.cut_inside != 0);
    c.cutg = G;
    c.cuts.reset();
  }
  return *c.cutg;
}

int setup_cut(Ctx& c, std::string& err) {
  const CutGeometry& G = cut_geometry(c);
  auto S = std::make_shared<CutState>();
  elements_of(G, c.p, *S);
  faces_of(G, *S);
  fine_operators(c, G, *S);
  const int s = S->s, ss = s * s;
  c.host.clear();
  // structural coupling graph of the finest level: pairs within two face /
  // interface steps
  const int ne0 = S->ne;
  std::vector<std::set<int>> G1(ne0);
  for (int e = 0; e < ne0; ++e) G1[e].insert(e);
  for (const Face& F : S->intra) {
    G1[F.ea].insert(F.eb);
    G1[F.eb].insert(F.ea);
  }
  for (const Face& F : S->arcs) {
    G1[F.ea].insert(F.eb);
    G1[F.eb].insert(F.ea);
  }
  auto square = [](const std::vector<std::set<int>>& g) {
    std::vector<std::set<int>> out(g.size());
    for (size_t e = 0; e < g.size(); ++e)
      for (int m : g[e]) out[e].insert(g[m].begin(), g[m].end());
    return out;
  };
  std::vector<std::set<int>> structure = square(G1);
  // level state for the coarsening: anchors, boxes, phases, level-0 pieces
  int ne = ne0;
  std::vector<int> anchor(2 * ne), phase = S->phase;
  for (int e = 0; e < ne; ++e) {
    anchor[2 * e] = G.pieces[S->reps[e]].i;
    anchor[2 * e + 1] = G.pieces[S->reps[e]].j;
  }
  std::vector<double> box_lo = S->box_lo, box_hi = S->box_hi;
  Ops ops = S->fine;
  int n = G.n;
  for (;;) {
    HostLevel L;
    L.n[0] = L.n[1] = n;
    stokes_blocks(c, ops, L);
    L.colour = greedy(structure);
    c.host.push_back(std::move(L));
    if (n <= 2) break;
    // an earlier bottom: this level (not level 0) is small enough for the
    // dense pseudo-inverse (stk_set_bottom)
    if (c.host.size() > 1 && c.bottom_max > 0 && (int64_t)ne * 3 * s <= c.bottom_max) break;
    n /= 2;
    // same-phase agglomeration by the parent of the anchor cell
    std::map<std::array<int, 3>, int> keys;
    for (int e = 0; e < ne; ++e) keys[{anchor[2 * e + 1] / 2, anchor[2 * e] / 2, phase[e]}] = 0;
    int nc = 0;
    for (auto& kv : keys) kv.second = nc++;          // (cy, cx, phase) lexicographic
    std::vector<int> parent(ne);
    for (int e = 0; e < ne; ++e) parent[e] = keys[{anchor[2 * e + 1] / 2, anchor[2 * e] / 2, phase[e]}];
    std::vector<int> c_anchor(2 * nc), c_phase(nc);
    for (auto& kv : keys) {
      c_anchor[2 * kv.second] = kv.first[1];
      c_anchor[2 * kv.second + 1] = kv.first[0];
      c_phase[kv.second] = kv.first[2];
    }
    std::vector<double> c_lo(2 * nc, 1e300), c_hi(2 * nc, -1e300);
    std::vector<std::vector<int>> children(nc);
    for (int e = 0; e < ne; ++e) {
      children[parent[e]].push_back(e);
      for (int a = 0; a < 2; ++a) {
        c_lo[2 * parent[e] + a] = std::min(c_lo[2 * parent[e] + a], box_lo[2 * e + a]);
        c_hi[2 * parent[e] + a] = std::max(c_hi[2 * parent[e] + a], box_hi[2 * e + a]);
      }
    }
    // injection: the coarse Q_p function restricted to the member is a Q_p
    // polynomial on the member's box, re-expanded in the member's basis by
    // the L2 projection over that box, I_f = M_B^{-1} int_B phi_f phi_c^T
    // (tensor Gauss, p + 1 points per axis; well conditioned, unlike the
    // projection over a small cut piece)
    std::vector<double> Ib((size_t)ne * ss);
    std::atomic<int> bad(-1);
    std::vector<double> gx, gw;
    gauss_rule(c.p + 1, gx, gw);
    const int q1 = c.p + 1, m = q1 * q1;
    parallel_for(ne, [&](int64_t f0, int64_t f1) {
      for (int64_t f = f0; f < f1; ++f) {
        Blk Mf(ss, 0.0), Bf(ss, 0.0), inv(ss);
        std::vector<double> x((size_t)2 * m), w(m);
        const double* a = &box_lo[2 * f];
        const double* b = &box_hi[2 * f];
        for (int v = 0; v < q1; ++v)
          for (int u = 0; u < q1; ++u) {
            x[2 * (v * q1 + u)] = 0.5 * (a[0] + b[0]) + 0.5 * (b[0] - a[0]) * gx[u];
            x[2 * (v * q1 + u) + 1] = 0.5 * (a[1] + b[1]) + 0.5 * (b[1] - a[1]) * gx[v];
            w[v * q1 + u] = gw[v] * gw[u] * 0.25 * (b[0] - a[0]) * (b[1] - a[1]);
          }
        std::vector<double> Pf((size_t)m * s), Pc((size_t)m * s);
        box_basis(c.p, a, b, x.data(), m, Pf.data(), nullptr, nullptr);
        box_basis(c.p, &c_lo[2 * parent[f]], &c_hi[2 * parent[f]], x.data(), m, Pc.data(), nullptr, nullptr);
        weighted(m, s, Pf.data(), Pf.data(), w.data(), 1.0, Mf.data());
        weighted(m, s, Pf.data(), Pc.data(), w.data(), 1.0, Bf.data());
        std::string e2;
        if (invert_blocks(s, 1, Mf.data(), inv.data(), e2) != STK_OK) {
          bad = (int)f;
          continue;
        }
        double* out = &Ib[(size_t)f * ss];
        std::fill(out, out + ss, 0.0);
        mm(s, 1.0, inv.data(), false, Bf.data(), out);
      }
    });
    if (bad >= 0) {
      err = "cut-cell element mass matrix is singular";
      return STK_ERR_SINGULAR_BLOCK;
    }
    HostLevel& Lf = c.host.back();
    Lf.parent = parent;
    Lf.Ib = Ib;
    ops = coarsen(ops, parent, Ib, children);
    std::vector<std::set<int>> g1(nc);
    for (int e = 0; e < ne; ++e)
      for (int j : G1[e]) g1[parent[e]].insert(parent[j]);
    G1.swap(g1);
    structure = square(G1);
    ne = nc;
    anchor.swap(c_anchor);
    phase.swap(c_phase);
    box_lo.swap(c_lo);
    box_hi.swap(c_hi);
  }
  c.cuts = S;
  return STK_OK;
}

int64_t cut_count_points(Ctx& c, int kind) {
  std::vector<double> x;
  cut_points(c, kind, x, nullptr, nullptr);
  return (int64_t)x.size() / 2;
}

void cut_points(Ctx& c, int kind, std::vector<double>& xyz, std::vector<double>* nrm, std::vector<int>* phase) {
  const CutGeometry& G = cut_geometry(c);
  xyz.clear();
  if (nrm) nrm->clear();
  if (phase) phase->clear();
  if (kind == STK_PTS_VOLUME) {
    for (const CutPiece& P : G.pieces) {
      xyz.insert(xyz.end(), P.x.begin(), P.x.end());
      if (phase) phase->insert(phase->end(), P.w.size(), P.ph);
    }
    return;
  }
  if (kind == STK_PTS_INTERIOR_FACE) return;   // intraphase faces carry no data
  CutState tmp;
  const CutState* S = c.cuts ? c.cuts.get() : nullptr;
  if (!S) {
    elements_of(G, c.p, tmp);
    faces_of(G, tmp);
    S = &tmp;
  }
  const std::vector<Face>& list = kind == STK_PTS_BOUNDARY_FACE ? S->bdry : S->arcs;
  for (const Face& F : list) {
    xyz.insert(xyz.end(), F.x.begin(), F.x.end());
    const size_t m = F.w.size();
    if (nrm) nrm->insert(nrm->end(), F.nrm.begin(), F.nrm.end());
    if (phase) phase->insert(phase->end(), m, kind == STK_PTS_BOUNDARY_FACE ? S->phase[F.ea] : 1);
  }
}

// Right-hand side (eqs. appstokes1 / appstokes2 times M) on the merged
// elements: volume data (f_1, f_2, fdiv) at the volume points, Dirichlet
// data at the boundary-face points, and at the interface points the jumps
// g = u(1) - u(2) and h = sigma(1) n - sigma(2) n, weighted like the lift.
int cut_assemble_rhs(Ctx& c, const double* f_vol, const double* bdata, const double* idata, double* b,
                     std::string& err) {
  const CutGeometry& G = cut_geometry(c);
  if (!c.cuts) {
    err = "call stk_setup first";
    return STK_ERR_NOT_SETUP;
  }
  const CutState& S = *c.cuts;
  const int ne = S.ne, s = S.s, p = S.p, nb = 3 * s;
  const double hk = G.h[0];
  auto mu = [&](int e) { return c.mu_phase[S.phase[e] - 1]; };
  std::vector<double> bu[2] = {std::vector<double>((size_t)ne * s, 0.0), std::vector<double>((size_t)ne * s, 0.0)};
  std::vector<double> bp((size_t)ne * s, 0.0);
  std::vector<double> jg[2][2];
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 2; ++k) jg[i][k].assign((size_t)ne * s, 0.0);
  auto phi = [&](int e, const std::vector<double>& x, std::vector<double>& Phi) {
    const int m = (int)x.size() / 2;
    Phi.assign((size_t)m * s, 0.0);
    box_basis(p, &S.box_lo[2 * e], &S.box_hi[2 * e], x.data(), m, Phi.data(), nullptr, nullptr);
  };
  auto acc = [&](std::vector<double>& out, int e, const std::vector<double>& Phi, const std::vector<double>& w,
                 const double* val, int stride, double alpha) {
    const int m = (int)w.size();
    for (int k = 0; k < m; ++k) {
      const double v = alpha * w[k] * val[(size_t)k * stride];
      for (int a = 0; a < s; ++a) out[(size_t)e * s + a] += Phi[(size_t)k * s + a] * v;
    }
  };
  // volume data, pieces in order
  size_t off = 0;
  std::vector<size_t> piece_off(G.pieces.size());
  for (size_t k = 0; k < G.pieces.size(); ++k) {
    piece_off[k] = off;
    off += G.pieces[k].w.size();
  }
  for (int e = 0; e < ne; ++e)
    for (int k : S.pieces[e]) {
      const CutPiece& P = G.pieces[k];
      std::vector<double> Phi;
      phi(e, P.x, Phi);
      const double* f = f_vol + piece_off[k] * 3;
      acc(bu[0], e, Phi, P.w, f + 0, 3, 1.0);
      acc(bu[1], e, Phi, P.w, f + 1, 3, 1.0);
      acc(bp, e, Phi, P.w, f + 2, 3, 1.0);
    }
  off = 0;
  for (const Face& F : S.bdry) {
    std::vector<double> Phi;
    phi(F.ea, F.x, Phi);
    const double* g = bdata + off * 2;
    const double tau_d = c.c_bdry * p * mu(F.ea) / hk;
    for (int i = 0; i < 2; ++i) {
      acc(bu[i], F.ea, Phi, F.w, g + i, 2, tau_d);
      if (F.axis >= 0) {
        acc(jg[i][F.axis], F.ea, Phi, F.w, g + i, 2, (double)F.side);
      } else {
        for (int k = 0; k < 2; ++k) {
          std::vector<double> ng(F.w.size());
          for (size_t q = 0; q < F.w.size(); ++q) ng[q] = F.nrm[2 * q + k] * g[q * 2 + i];
          acc(jg[i][k], F.ea, Phi, F.w, ng.data(), 1, 1.0);
        }
      }
    }
    off += F.w.size();
  }
  off = 0;
  for (const Face& F : S.arcs) {
    const size_t m = F.w.size();
    if (idata) {
      std::vector<double> Pm, Pp;
      phi(F.ea, F.x, Pm);
      phi(F.eb, F.x, Pp);
      const double mum = mu(F.ea), mup = mu(F.eb);
      const double lam = mum < mup ? 0.0 : (mum > mup ? 1.0 : 0.5);
      const double tij = 3.0 * p * std::min(mum, mup) / hk;
      const double* d = idata + off * 4;
      for (int i = 0; i < 2; ++i) {
        for (int k = 0; k < 2; ++k) {
          std::vector<double> ng(m);
          for (size_t t = 0; t < m; ++t) ng[t] = F.nrm[2 * t + k] * d[t * 4 + i];
          acc(jg[i][k], F.ea, Pm, F.w, ng.data(), 1, 1.0 - lam);
          acc(jg[i][k], F.eb, Pp, F.w, ng.data(), 1, lam);
        }
        acc(bu[i], F.ea, Pm, F.w, d + 2 + i, 4, lam);
        acc(bu[i], F.ea, Pm, F.w, d + i, 4, tij);
        acc(bu[i], F.eb, Pp, F.w, d + 2 + i, 4, 1.0 - lam);
        acc(bu[i], F.eb, Pp, F.w, d + i, 4, -tij);
      }
    }
    off += m;
  }
  // bu_i -= sum_j G_j^T Mmu M^{-1} (jg[i][j] + gamma jg[j][i]); bp += jg[0][0] + jg[1][1]
  const Ops& O = S.fine;
  const std::vector<Blk> Mmud = diag_blocks(O.Mmu);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      std::vector<double> t((size_t)ne * s);
      bool any = false;
      for (size_t k = 0; k < t.size(); ++k) {
        t[k] = jg[i][j][k] + c.gamma * jg[j][i][k];
        any = any || t[k] != 0.0;
      }
      if (!any) continue;
      std::vector<double> y((size_t)ne * s, 0.0);
      for (int e = 0; e < ne; ++e) {
        double u[16] = {0};
        for (int a = 0; a < s; ++a)
          for (int bb = 0; bb < s; ++bb) u[a] += O.Minv[e][a * s + bb] * t[(size_t)e * s + bb];
        for (int a = 0; a < s; ++a)
          for (int bb = 0; bb < s; ++bb) y[(size_t)e * s + a] += Mmud[e][a * s + bb] * u[bb];
      }
      // G_j^T y: G_j(e, f) contributes G_j(e, f)^T y_e to row f
      for (int e = 0; e < ne; ++e)
        for (auto& kv : O.G[j].row[e])
          for (int a = 0; a < s; ++a)
            for (int bb = 0; bb < s; ++bb)
              bu[i][(size_t)kv.first * s + bb] -= kv.second[a * s + bb] * y[(size_t)e * s + a];
    }
  for (size_t k = 0; k < bp.size(); ++k) bp[k] += jg[0][0][k] + jg[1][1][k];
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < s; ++a) {
      b[(size_t)e * nb + a] = bu[0][(size_t)e * s + a];
      b[(size_t)e * nb + s + a] = bu[1][(size_t)e * s + a];
      b[(size_t)e * nb + 2 * s + a] = bp[(size_t)e * s + a];
    }
  return STK_OK;
}

void cut_face_neighbours(Ctx& c, std::vector<int>& nbr, std::vector<double>& ctr) {
  const CutGeometry& G = cut_geometry(c);
  if (!c.cuts) throw std::runtime_error("cut-cell problem not set up");
  const CutState& S = *c.cuts;
  nbr.assign((size_t)S.ne * 4, -1);
  ctr.assign((size_t)S.ne * 2, 0.0);
  const int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  for (int e = 0; e < S.ne; ++e) {
    const CutPiece& rep = G.pieces[S.reps[e]];
    for (int k = 0; k < 4; ++k) {
      const int ii = rep.i + dd[k][0], jj = rep.j + dd[k][1];
      if (ii < 0 || ii >= G.n || jj < 0 || jj >= G.n) continue;
      const int piece = G.find(ii, jj, S.phase[e]);
      if (piece >= 0 && S.of_piece[piece] != e) nbr[(size_t)e * 4 + k] = S.of_piece[piece];
    }
    for (int a = 0; a < 2; ++a)
      ctr[(size_t)e * 2 + a] = (0.5 * (S.box_lo[2 * e + a] + S.box_hi[2 * e + a]) - G.lo[a]) / (G.hi[a] - G.lo[a]);
  }
}

}  // namespace stk
