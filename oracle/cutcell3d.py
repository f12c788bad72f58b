"""Cut cells of an embedded sphere on a Cartesian grid: volume, surface and face
quadrature by dimension reduction (oracle; test infrastructure only).

Section 5's curved domains include the sphere (Dirichlet data on it) and
Section 6's bubble is also run in 3D; their quadrature comes from external
implicit-quadrature work, not part of the paper.  This is a reading written
from the idea of dimension reduction, one dimension at a time, on top of the
2D rules of oracle/cutcell.py:

* Height direction k: the axis whose tangential rectangle R (axes i, j)
  stays farthest inside the silhouette circle |t - c'| = r, c' the centre's
  projection, relative to R's diagonal; below half a diagonal on every axis
  the cell is split into eight and each part treated alike.
* Over a tangential point t the sphere has the heights z(t) = c_k +- sqrt(D),
  D = r^2 - |t - c'|^2.  The order of {z-, z+, h0, h1} (the cell's height
  range) changes only where |t - c'| equals r (the silhouette) or
  sqrt(r^2 - (h - c_k)^2) for h = h0, h1: concentric circles about c'.
  Between consecutive such radii (only the circles that cross R count) the
  inside segment [L(t), U(t)] (L = z- or h0, U = z+ or h1) has a fixed
  formula and the height integral F(t) is smooth in t.
* The tangential integral over R intersected with the annulus
  rho_a < |t - c'| < rho_b is the 2D rule of R intersected with the disc of
  radius rho_b minus the one of radius rho_a (cutcell.cell_rules): exact for
  the smooth extension of F into the inner disc, which the fixed formula
  provides (D only grows inward).  The resulting weights can be negative.
* The surface rule uses the same tangential nodes at z+ or z- with the graph's
  area element r / sqrt(D), bounded since the silhouette stays away from R.
* The 2D rules of rectangle and disc split the outer variable at the circle's
  crossings with the rectangle and at its extreme points, and grade each piece
  geometrically toward an extreme point lying just beyond it (the chord's
  half-width has a square-root branch point there).
* A cell face (x_a = const) meets the sphere in a circle of radius
  sqrt(r^2 - (x_a - c_a)^2): its inside and outside parts are the 2D rules of
  that face.

Phase 1 is inside the sphere, phase 2 outside; the surface normal points out
of the sphere.
"""
import numpy as np

from .basis import gauss


def _gauss_on(a, b, q):
    x, w = gauss(q)
    return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w


class Sphere:
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


def classify(sphere, lo, hi):
    """-1 inside, +1 outside, 0 cut, for the cell [lo, hi] (3D)."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    near = np.clip(sphere.c, lo, hi)
    dmin = np.sqrt(((near - sphere.c) ** 2).sum())
    far = np.where(np.abs(lo - sphere.c) > np.abs(hi - sphere.c), lo, hi)
    dmax = np.sqrt(((far - sphere.c) ** 2).sum())
    if dmax <= sphere.r:
        return -1
    if dmin >= sphere.r:
        return 1
    return 0


def _rect_distances(c2, lo2, hi2):
    """Smallest and largest distance from c2 to the rectangle [lo2, hi2]."""
    near = np.clip(c2, lo2, hi2)
    far = np.where(np.abs(lo2 - c2) > np.abs(hi2 - c2), lo2, hi2)
    return np.sqrt(((near - c2) ** 2).sum()), np.sqrt(((far - c2) ** 2).sum())


def _circle_crosses_rect(c2, rho, lo2, hi2):
    """Whether the circle |t - c2| = rho passes through the open rectangle."""
    dmin, dmax = _rect_distances(c2, lo2, hi2)
    return dmin < rho < dmax


def _graded(a, b, sing, ratio=0.5, levels=60):
    """[a, b] split geometrically toward an end near which one of the branch
    points sing lies (closer than b - a, outside or at the end), so that the
    Gauss rules of the pieces see the square-root singularity only at a
    relative distance of order one: exponential instead of algebraic
    convergence."""
    L = b - a
    cuts = {a, b}
    for end, inward in ((a, 1.0), (b, -1.0)):
        d = min((abs(e - end) for e in sing if (e - end) * inward <= 0.0), default=np.inf)
        if d >= L:
            continue
        for j in range(1, levels + 1):
            step = L * ratio ** j
            cuts.add(end + inward * step)
            if step <= d:
                break
    return sorted(cuts)


def _disc_rule(c2, rho, lo2, hi2, q):
    """2D rule of the rectangle [lo2, hi2] intersected with the disc of radius
    rho about c2 (rho = inf: the whole rectangle).  Outer variable along the
    second axis, split at the circle's crossings with the first axis's edges
    and at its extreme points, each piece graded toward the extreme points
    (the branch points of the chord's half-width) that lie near it; inner
    Gauss rules on the chord within the rectangle."""
    if np.isinf(rho):
        s0, w0 = _gauss_on(lo2[0], hi2[0], q)
        s1, w1 = _gauss_on(lo2[1], hi2[1], q)
        pts = np.stack(np.meshgrid(s0, s1, indexing="ij"), axis=-1).reshape(-1, 2)
        return pts, np.outer(w0, w1).ravel()
    if rho <= 0:
        return np.zeros((0, 2)), np.zeros(0)
    ch, ct = c2
    y0, y1, t0, t1 = lo2[0], hi2[0], lo2[1], hi2[1]
    sing = (ct - rho, ct + rho)
    brk = {t0, t1}
    for yy in (y0, y1):
        d = rho * rho - (yy - ch) ** 2
        if d > 0:
            for sg in (-1.0, 1.0):
                tt = ct + sg * np.sqrt(d)
                if t0 < tt < t1:
                    brk.add(tt)
    for e in sing:
        if t0 < e < t1:
            brk.add(e)
    brk = sorted(brk)
    P, W = [], []
    for a, b in zip(brk[:-1], brk[1:]):
        if b <= a:
            continue
        cuts = _graded(a, b, sing)
        for u, v in zip(cuts[:-1], cuts[1:]):
            if v <= u:
                continue
            ts, wts = _gauss_on(u, v, q)
            d = rho * rho - (ts - ct) ** 2
            keep = d > 0
            w = np.sqrt(np.where(keep, d, 0.0))
            lo_y, hi_y = np.maximum(y0, ch - w), np.minimum(y1, ch + w)
            keep &= hi_y > lo_y
            if not keep.any():
                continue
            ts, wts, lo_y, hi_y = ts[keep], wts[keep], lo_y[keep], hi_y[keep]
            g, gw = gauss(q)
            ys = 0.5 * (lo_y + hi_y)[:, None] + 0.5 * (hi_y - lo_y)[:, None] * g[None, :]
            P.append(np.stack([ys.ravel(), np.repeat(ts, q)], 1))
            W.append(((wts * 0.5 * (hi_y - lo_y))[:, None] * gw[None, :]).ravel())
    if not P:
        return np.zeros((0, 2)), np.zeros(0)
    return np.concatenate(P), np.concatenate(W)


kSilhouetteMargin = 0.5   # cells split until r - max |t - c'| >= 0.5 x the rectangle's diagonal


def _box_rule(lo, hi, q):
    g = [_gauss_on(lo[a], hi[a], q) for a in range(3)]
    pts = np.stack(np.meshgrid(g[0][0], g[1][0], g[2][0], indexing="ij"), axis=-1).reshape(-1, 3)
    w = (g[0][1][:, None, None] * g[1][1][None, :, None] * g[2][1][None, None, :]).ravel()
    return pts, w


def cell_rules(sphere, lo, hi, q, depth=0):
    """Rules of the cell [lo, hi] cut by the sphere: (x_in, w_in),
    (x_out, w_out), (x_if, w_if, n_if); points [m, 3].  When no axis keeps
    its tangential rectangle well inside the silhouette circle the cell is
    split into eight and the rules of the parts are joined."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    c, r = sphere.c, sphere.r
    # height direction: the axis whose tangential rectangle stays farthest
    # inside the silhouette circle, relative to its diagonal (the height
    # integrals carry sqrt(r^2 - |t - c'|^2), singular on the silhouette)
    best, k = -np.inf, None
    for a in range(3):
        ta = [b for b in range(3) if b != a]
        dmax = _rect_distances(c[ta], lo[ta], hi[ta])[1]
        margin = (r - dmax) / np.sqrt(((hi[ta] - lo[ta]) ** 2).sum())
        if margin > best:
            best, k = margin, a
    if best < kSilhouetteMargin:
        if depth > 8:
            raise ValueError("no height direction found for the cell")
        mid = 0.5 * (lo + hi)
        parts = ([], []), ([], []), ([], [], [])
        for o in range(8):
            slo = np.where([(o >> a) & 1 for a in range(3)], mid, lo)
            shi = np.where([(o >> a) & 1 for a in range(3)], hi, mid)
            cl = classify(sphere, slo, shi)
            if cl == 0:
                sub = cell_rules(sphere, slo, shi, q, depth + 1)
            else:
                box = _box_rule(slo, shi, q)
                empty = (np.zeros((0, 3)), np.zeros(0))
                sub = (box, empty) if cl < 0 else (empty, box)
                sub = sub + ((np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3))),)
            for dst, src in zip(parts, sub):
                for lst, arr in zip(dst, src):
                    lst.append(arr)
        return tuple(tuple(np.concatenate(lst) for lst in part) for part in parts)
    tang = [a for a in range(3) if a != k]
    c2, lo2, hi2 = c[tang], lo[tang], hi[tang]
    h0, h1, ck = lo[k], hi[k], c[k]
    radii = sorted({np.sqrt(r * r - (h - ck) ** 2) for h in (h0, h1) if r * r > (h - ck) ** 2
                    if _circle_crosses_rect(c2, np.sqrt(r * r - (h - ck) ** 2), lo2, hi2)})
    bounds = [0.0] + radii + [np.inf]
    dmin, dmax = _rect_distances(c2, lo2, hi2)
    xin, win, xout, wout, xif, wif = [], [], [], [], [], []

    for ra, rb in zip(bounds[:-1], bounds[1:]):
        # the configuration of the annulus, at a radius of it that occurs in R
        rm = 0.5 * (max(ra, dmin) + min(rb, dmax))
        Dm = r * r - rm * rm
        if Dm > 0:
            sm = np.sqrt(Dm)
            low_root, high_root = h0 < ck - sm < h1, h0 < ck + sm < h1
            inside = max(h0, ck - sm) < min(h1, ck + sm)
        else:
            low_root = high_root = inside = False
        # signed tangential rule of the annulus within R
        pb, wb = _disc_rule(c2, rb, lo2, hi2, q)
        pa, wa = _disc_rule(c2, ra, lo2, hi2, q)
        pts = np.concatenate([pb, pa])
        wts = np.concatenate([wb, -wa])
        if not len(wts):
            continue
        g, gw = gauss(q)
        D = r * r - ((pts - c2) ** 2).sum(1)
        sq = np.sqrt(np.maximum(D, 0.0)) if (inside or low_root or high_root) else np.zeros(len(D))
        L = ck - sq if low_root else np.full(len(D), h0)
        U = ck + sq if high_root else np.full(len(D), h1)

        def seg(a, b):
            hs = 0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * g[None, :]
            ww = (wts * 0.5 * (b - a))[:, None] * gw[None, :]
            p = np.zeros((hs.size, 3))
            p[:, tang[0]] = np.repeat(pts[:, 0], q)
            p[:, tang[1]] = np.repeat(pts[:, 1], q)
            p[:, k] = hs.ravel()
            return p, ww.ravel()
        if inside:
            p, ww = seg(L, U)
            xin.append(p)
            win.append(ww)
            segs = ([(np.full(len(D), h0), L)] if low_root else []) + ([(U, np.full(len(D), h1))] if high_root else [])
        else:
            segs = [(np.full(len(D), h0), np.full(len(D), h1))]
        for a, b in segs:
            p, ww = seg(a, b)
            xout.append(p)
            wout.append(ww)
        for on, z in ((low_root, ck - sq), (high_root, ck + sq)):
            if on:
                p = np.zeros((len(D), 3))
                p[:, tang[0]], p[:, tang[1]], p[:, k] = pts[:, 0], pts[:, 1], z
                xif.append(p)
                wif.append(wts * r / sq)
    cat = lambda L, d: np.concatenate(L) if L else np.zeros((0, 3) if d else 0)
    x_if = cat(xif, 1)
    n_if = sphere.normal(x_if) if len(x_if) else np.zeros((0, 3))
    return (cat(xin, 1), cat(win, 0)), (cat(xout, 1), cat(wout, 0)), (x_if, cat(wif, 0), n_if)


def face_parts(sphere, lo, hi, axis, value, q):
    """Rules of the inside (phase 1) and outside (phase 2) parts of the cell
    face {x_axis = value} of [lo, hi]: dict phase -> (points [m, 3], weights).
    The face meets the sphere in the circle of radius sqrt(r^2 - d^2), d the
    distance of the face's plane from the centre."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    c, r = sphere.c, sphere.r
    tang = [a for a in range(3) if a != axis]
    c2, lo2, hi2 = c[tang], lo[tang], hi[tang]
    d2 = r * r - (value - c[axis]) ** 2
    xf, wf = _disc_rule(c2, np.inf, lo2, hi2, q)
    if d2 > 0:
        xi, wi = _disc_rule(c2, np.sqrt(d2), lo2, hi2, q)
        xo, wo = np.concatenate([xf, xi]), np.concatenate([wf, -wi])   # the face minus the disc
    else:
        xi, wi = np.zeros((0, 2)), np.zeros(0)
        xo, wo = xf, wf

    def lift(p2):
        p = np.zeros((len(p2), 3))
        p[:, tang[0]], p[:, tang[1]] = p2[:, 0], p2[:, 1]
        p[:, axis] = value
        return p
    return {1: (lift(xi), wi), 2: (lift(xo), wo)}


class CutMesh3D:
    """The pieces of an n^3 grid on [lo, hi]^3 cut by a sphere: one piece per
    uncut cell, two per cut cell (phase 1 inside, 2 outside), each with its
    volume and rule; and the merged elements, by the same reading as the 2D
    mesh: a piece below merge_fraction of its cell's volume joins the
    same-phase piece across the cell face whose same-phase part has the
    largest area, among neighbours that are not small themselves."""

    def __init__(self, sphere, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), q=6, merge_fraction=0.25):
        self.sphere, self.n, self.q = sphere, int(n), q
        self.lo, self.hi = np.asarray(lo, float), np.asarray(hi, float)
        self.h = (self.hi - self.lo) / self.n
        self.cell_volume = float(np.prod(self.h))
        self.pieces = []
        self.piece_of = {}
        self.interface = {}
        for kk in range(self.n):
            for j in range(self.n):
                for i in range(self.n):
                    clo = self.lo + self.h * np.array([i, j, kk])
                    chi = clo + self.h
                    cl = classify(sphere, clo, chi)
                    if cl != 0:
                        self._add((i, j, kk), 1 if cl < 0 else 2, *_box_rule(clo, chi, q))
                        continue
                    (xi, wi), (xo, wo), ifr = cell_rules(sphere, clo, chi, q)
                    self._add((i, j, kk), 1, xi, wi)
                    self._add((i, j, kk), 2, xo, wo)
                    self.interface[(i, j, kk)] = ifr
        self._merge(merge_fraction)

    def _add(self, cell, ph, px, pw):
        self.piece_of[cell + (ph,)] = len(self.pieces)
        self.pieces.append(dict(cell=cell, phase=ph, volume=float(pw.sum()), points=px, weights=pw))

    def shared_face_area(self, cell, axis, sign, ph):
        """Area of the phase-ph part of the face of `cell` toward its neighbour
        at +-e_axis (sign +1 or -1)."""
        clo = self.lo + self.h * np.array(cell)
        chi = clo + self.h
        value = chi[axis] if sign > 0 else clo[axis]
        return float(face_parts(self.sphere, clo, chi, axis, value, self.q)[ph][1].sum())

    def _merge(self, frac):
        """element[p]: the element (a representative piece) of every piece.
        A small piece joins the same-phase face neighbour whose shared
        same-phase face part is largest, non-small neighbours first; if all of
        them are small (a sliver near an edge or corner of the cell, where the
        sphere enters it only slightly, a case the 2D mesh does not have) it
        joins the largest-sharing small one, and the joins are followed
        transitively.  The representative of an element is its non-small
        piece, else its first piece."""
        npc = len(self.pieces)
        parent = list(range(npc))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        small = [p["volume"] < frac * self.cell_volume for p in self.pieces]
        self.merged_into = {}
        for k, p in enumerate(self.pieces):
            if not small[k]:
                continue
            cand = []
            for axis in range(3):
                for sign in (-1, 1):
                    nc = list(p["cell"])
                    nc[axis] += sign
                    if not 0 <= nc[axis] < self.n:
                        continue
                    nb = self.piece_of.get(tuple(nc) + (p["phase"],))
                    if nb is None:
                        continue
                    A = self.shared_face_area(p["cell"], axis, sign, p["phase"])
                    if A > 0:
                        cand.append((not small[nb], A, -nb, nb))
            if cand:
                best = max(cand)[3]
                self.merged_into[k] = best
                ra, rb = find(k), find(best)
                if ra != rb:
                    parent[ra] = rb
        groups = {}
        for k in range(npc):
            groups.setdefault(find(k), []).append(k)
        self.element = [0] * npc
        for members in groups.values():
            big = [k for k in members if not small[k]]
            rep = big[0] if big else members[0]
            for k in members:
                self.element[k] = rep

    def element_volume(self, rep):
        return sum(p["volume"] for k, p in enumerate(self.pieces) if self.element[k] == rep)
