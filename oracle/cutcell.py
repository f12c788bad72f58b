"""Cut cells of an embedded circle on a Cartesian grid (oracle): quadrature by
dimension reduction and the merging of small pieces.

Section 5 (curved domains, the circular interface of the multi-phase tests)
takes its quadrature from external implicit-quadrature work that is not part
of the paper; the reading here is written from the idea of dimension
reduction.  The circle phi(x) = |x - c| - r splits every cell it crosses into
an inside piece (phi < 0, phase 1) and an outside piece (phase 2).

* Height direction: in each cut cell, the axis along which the circle's
  normal at the cell centre has the larger component.  Over the other
  (tangential) axis the circle is then a smooth graph inside the cell (the
  points where it is vertical lie in cells that chose the other axis).
* Volume rule: the tangential interval is split at every crossing of the
  circle with the cell's two height-direction faces; on each sub-interval a
  q-point Gauss rule gives the tangential nodes, and at each node the chord of
  the circle (found analytically) splits the height interval into inside and
  outside parts, each with its own q-point Gauss rule.
* Interface rule: the same tangential nodes on the branch of the circle that
  lies in the cell, weighted by ds = sqrt(1 + (dh/dt)^2) dt; the normal points
  out of the circle (from phase 1 into phase 2).
* Face rule: a cell face is split at its crossings with the circle; each part
  belongs to the phase of its midpoint.

Merging: a piece whose area is below 1/4 of its cell's joins the piece of the
same phase across the cell face with which it shares the longest same-phase
segment; pieces that are large enough stay elements of their own.
"""
import numpy as np

from .basis import gauss


class Circle:
    def __init__(self, centre, radius):
        self.c = np.asarray(centre, dtype=np.float64)
        self.r = float(radius)

    def phi(self, x):
        x = np.asarray(x, dtype=np.float64)
        return np.sqrt(((x - self.c) ** 2).sum(axis=-1)) - self.r

    def normal(self, x):
        x = np.asarray(x, dtype=np.float64)
        v = x - self.c
        return v / np.sqrt((v ** 2).sum(axis=-1, keepdims=True))


def _gauss_on(a, b, q):
    x, w = gauss(q)
    return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w


def graded_cuts(a, b, sing, levels=40):
    """Cut points of [a, b]: its ends, plus halvings toward an end that one of
    the branch points sing (the circle's extreme points, where the chord's
    half-width and the arc's ds / dt have square-root singularities) lies
    beyond or at, closer than b - a: a + L / 2^j (or b - L / 2^j), j = 1, 2, ...
    until the step is no longer than the distance (at most `levels` halvings).
    Each piece then sees the singularity at a relative distance of order one,
    so its Gauss rule converges exponentially."""
    L = b - a
    cuts = {a, b}
    for end, inward in ((a, 1.0), (b, -1.0)):
        d = min((abs(e - end) for e in sing if (e - end) * inward <= 0.0), default=np.inf)
        if d >= L:
            continue
        step = L
        for _ in range(levels):
            step *= 0.5
            cuts.add(end + inward * step)
            if step <= d:
                break
    return sorted(cuts)


def classify(circle, lo, hi):
    """-1 inside, +1 outside, 0 cut, for the cell [lo, hi] (2D)."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    near = np.clip(circle.c, lo, hi)
    dmin = np.sqrt(((near - circle.c) ** 2).sum())
    corners = np.array([[lo[0], lo[1]], [hi[0], lo[1]], [lo[0], hi[1]], [hi[0], hi[1]]])
    dmax = np.sqrt(((corners - circle.c) ** 2).sum(axis=1)).max()
    if dmax <= circle.r:
        return -1
    if dmin >= circle.r:
        return 1
    return 0


def piece_box(circle, lo, hi, ph):
    """Bounding box (lo, hi) of the phase-ph piece of the cut cell [lo, hi].
    Along axis k the inside piece (cell and disk) spans the coordinates whose
    line across the cell meets the disk: |x_k - c_k| < sqrt(r^2 - d^2), d the
    distance from c to the cell's range on the other axis.  The outside piece
    loses the coordinates whose whole line lies in the disk, |x_k - c_k| <
    sqrt(r^2 - D^2) with D the largest distance to that range; its box is the
    hull of what remains."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    blo, bhi = lo.copy(), hi.copy()
    c, r = circle.c, circle.r
    for k in range(2):
        o = 1 - k
        if ph == 1:
            d = max(0.0, lo[o] - c[o], c[o] - hi[o])
            a = np.sqrt(max(r * r - d * d, 0.0))
            blo[k] = max(lo[k], c[k] - a)
            bhi[k] = min(hi[k], c[k] + a)
        else:
            D = max(abs(lo[o] - c[o]), abs(hi[o] - c[o]))
            if r * r > D * D:
                a = np.sqrt(r * r - D * D)
                if c[k] - a <= lo[k] < c[k] + a:
                    blo[k] = c[k] + a
                if c[k] - a < hi[k] <= c[k] + a:
                    bhi[k] = c[k] - a
    return blo, bhi


def cell_rules(circle, lo, hi, q):
    """Gauss rules of a cut cell [lo, hi]: (x_in, w_in), (x_out, w_out),
    (x_if, w_if, n_if).  Points [m, 2]."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    ctr = 0.5 * (lo + hi)
    n = circle.normal(ctr)
    h_ax = int(np.argmax(np.abs(n)))
    t_ax = 1 - h_ax
    c_t, c_h, r = circle.c[t_ax], circle.c[h_ax], circle.r
    t0, t1, h0, h1 = lo[t_ax], hi[t_ax], lo[h_ax], hi[h_ax]
    brk = {t0, t1}
    for hh in (h0, h1):
        disc = r * r - (hh - c_h) ** 2
        if disc > 0:
            for s in (-1.0, 1.0):
                t = c_t + s * np.sqrt(disc)
                if t0 < t < t1:
                    brk.add(t)
    for s in (-1.0, 1.0):
        t = c_t + s * r
        if t0 < t < t1:
            brk.add(t)
    brk = sorted(brk)
    xin, win, xout, wout, xif, wif, nif = [], [], [], [], [], [], []

    def put(lst, t, hvals):
        p = np.zeros((len(hvals), 2))
        p[:, t_ax] = t
        p[:, h_ax] = hvals
        lst.append(p)

    pieces = []
    for a, b in zip(brk[:-1], brk[1:]):
        if b - a > 0:
            cuts = graded_cuts(a, b, (c_t - r, c_t + r))
            pieces += [(u, v) for u, v in zip(cuts[:-1], cuts[1:]) if v > u]
    for a, b in pieces:
        ts, wts = _gauss_on(a, b, q)
        for t, wt in zip(ts, wts):
            disc = r * r - (t - c_t) ** 2
            if disc > 0:
                w = np.sqrt(disc)
                lo_in, hi_in = max(h0, c_h - w), min(h1, c_h + w)
            else:
                w, lo_in, hi_in = 0.0, 0.0, 0.0
            if hi_in > lo_in:
                hs, wh = _gauss_on(lo_in, hi_in, q)
                put(xin, t, hs)
                win.append(wt * wh)
                outs = [(h0, lo_in), (hi_in, h1)]
            else:
                outs = [(h0, h1)]
            for oa, ob in outs:
                if ob > oa:
                    hs, wh = _gauss_on(oa, ob, q)
                    put(xout, t, hs)
                    wout.append(wt * wh)
            if disc > 0:
                for s in (-1.0, 1.0):
                    hv = c_h + s * w
                    if h0 <= hv <= h1:
                        dh = -s * (t - c_t) / w
                        put(xif, t, np.array([hv]))
                        wif.append(np.array([wt * np.sqrt(1.0 + dh * dh)]))
    cat = lambda L, k: np.concatenate(L) if L else np.zeros((0, 2) if k else 0)
    x_if = cat(xif, 1)
    n_if = circle.normal(x_if) if len(x_if) else np.zeros((0, 2))
    return (cat(xin, 1), cat(win, 0)), (cat(xout, 1), cat(wout, 0)), (x_if, cat(wif, 0), n_if)


def face_parts(circle, a, b, fixed_axis, fixed, q):
    """Gauss rules of the inside and outside parts of the face segment
    {x_fixed_axis = fixed, other coordinate in [a, b]}: dict phase ->
    (points [m, 2], weights)."""
    o = 1 - fixed_axis
    cuts = {a, b}
    disc = circle.r ** 2 - (fixed - circle.c[fixed_axis]) ** 2
    if disc > 0:
        for s in (-1.0, 1.0):
            v = circle.c[o] + s * np.sqrt(disc)
            if a < v < b:
                cuts.add(v)
    cuts = sorted(cuts)
    out = {1: ([], []), 2: ([], [])}
    for u, v in zip(cuts[:-1], cuts[1:]):
        if v <= u:
            continue
        mid = np.zeros(2)
        mid[fixed_axis] = fixed
        mid[o] = 0.5 * (u + v)
        ph = 1 if circle.phi(mid) < 0 else 2
        s, w = _gauss_on(u, v, q)
        p = np.zeros((q, 2))
        p[:, fixed_axis] = fixed
        p[:, o] = s
        out[ph][0].append(p)
        out[ph][1].append(w)
    return {ph: (np.concatenate(P) if P else np.zeros((0, 2)), np.concatenate(W) if W else np.zeros(0))
            for ph, (P, W) in out.items()}


class CutMesh:
    """The pieces of an n x n grid on [lo, hi]^2 cut by a circle: one piece per
    uncut cell, two per cut cell; each piece with its phase, area and volume
    rule; and the merged elements.  inside_only keeps the phase-1 pieces only:
    the disc as a curved domain (Section 5's curved-geometry problems), whose
    boundary is the circle."""

    def __init__(self, circle, n, lo=(0.0, 0.0), hi=(1.0, 1.0), q=8, merge_fraction=0.25, inside_only=False):
        self.circle, self.n, self.q = circle, int(n), q
        self.inside_only = bool(inside_only)
        self.lo, self.hi = np.asarray(lo, float), np.asarray(hi, float)
        self.h = (self.hi - self.lo) / self.n
        self.pieces = []           # dicts: cell (i, j), phase, area, rule (points, weights)
        self.piece_of = {}         # (i, j, phase) -> piece index
        self.interface = {}        # (i, j) -> (points, weights, normals)
        x, w = gauss(q)
        for j in range(self.n):
            for i in range(self.n):
                clo = self.lo + self.h * np.array([i, j])
                chi = clo + self.h
                k = classify(circle, clo, chi)
                if k != 0:
                    ph = 1 if k < 0 else 2
                    px, pw = self._full_rule(clo, chi)
                    self._add(i, j, ph, px, pw, (clo, chi))
                    continue
                (xi, wi), (xo, wo), ifr = cell_rules(circle, clo, chi, q)
                self._add(i, j, 1, xi, wi, piece_box(circle, clo, chi, 1))
                self._add(i, j, 2, xo, wo, piece_box(circle, clo, chi, 2))
                self.interface[(i, j)] = ifr
        self.cell_area = float(np.prod(self.h))
        self._merge(merge_fraction)

    def _full_rule(self, clo, chi):
        xs, wx = _gauss_on(clo[0], chi[0], self.q)
        ys, wy = _gauss_on(clo[1], chi[1], self.q)
        X, Y = np.meshgrid(xs, ys, indexing="xy")
        return np.stack([X.ravel(), Y.ravel()], axis=1), np.outer(wy, wx).ravel()

    def _add(self, i, j, ph, px, pw, box):
        if self.inside_only and ph != 1:
            return
        self.piece_of[(i, j, ph)] = len(self.pieces)
        self.pieces.append(dict(cell=(i, j), phase=ph, area=float(pw.sum()), points=px, weights=pw,
                                box=(np.asarray(box[0], float), np.asarray(box[1], float))))

    def shared_face_length(self, i, j, di, dj, ph):
        """Length of the phase-ph part of the face between cell (i, j) and
        cell (i + di, j + dj)."""
        clo = self.lo + self.h * np.array([i, j])
        if di != 0:
            fixed = clo[0] + (self.h[0] if di > 0 else 0.0)
            parts = face_parts(self.circle, clo[1], clo[1] + self.h[1], 0, fixed, self.q)
        else:
            fixed = clo[1] + (self.h[1] if dj > 0 else 0.0)
            parts = face_parts(self.circle, clo[0], clo[0] + self.h[0], 1, fixed, self.q)
        return float(parts[ph][1].sum())

    def _merge(self, frac):
        """element[p]: the element (a representative piece index) of every
        piece.  A piece below frac of its cell joins the same-phase piece across
        the face it shares most with (longest same-phase segment), among
        neighbours that are not small themselves."""
        self.element = list(range(len(self.pieces)))
        small = [p["area"] < frac * self.cell_area for p in self.pieces]
        self.merged_into = {}
        for k, p in enumerate(self.pieces):
            if not small[k]:
                continue
            i, j = p["cell"]
            best, best_len = None, -1.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if not (0 <= ii < self.n and 0 <= jj < self.n):
                    continue
                nb = self.piece_of.get((ii, jj, p["phase"]))
                if nb is None or small[nb]:
                    continue
                L = self.shared_face_length(i, j, di, dj, p["phase"])
                if L > best_len:
                    best, best_len = nb, L
            if best is not None:
                self.element[k] = best
                self.merged_into[k] = best

    def element_area(self, rep):
        return sum(p["area"] for k, p in enumerate(self.pieces) if self.element[k] == rep)


def greedy_colours(mesh):
    """Colours of the merged elements (Section 3 asks only for a valid
    multi-colouring).  Elements in the order of their representative piece
    (cells lexicographic, x fastest; the inside piece first), each taking the
    smallest colour not taken by an already coloured element that it may
    couple with: some host cell of one lies at an offset of the coupling
    stencil {|o_x|, |o_y| <= 1} or +-2 e_k of some host cell of the other (the
    reach of the viscous-stress and interphase couplings, reading 18).
    Returns (representatives in order, colour of each)."""
    reps = sorted(set(mesh.element))
    cells = {rep: set() for rep in reps}
    for k, p in enumerate(mesh.pieces):
        cells[mesh.element[k]].add(p["cell"])
    stencil = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)] + [(2, 0), (-2, 0), (0, 2), (0, -2)]
    owner = {}
    for rep in reps:
        for c in cells[rep]:
            owner.setdefault(c, []).append(rep)
    colour = {}
    for rep in reps:
        used = set()
        for (i, j) in cells[rep]:
            for di, dj in stencil:
                for other in owner.get((i + di, j + dj), []):
                    if other != rep and other in colour:
                        used.add(colour[other])
        c = 0
        while c in used:
            c += 1
        colour[rep] = c
    return reps, np.array([colour[r] for r in reps], dtype=np.int64)
