"""Learned element-local post-smoother: the plain definition of its features,
two-layer perceptron, mean-squared-error loss and gradient, and the outer
iteration that judges the correction (oracle).

Not a step of the paper: the correction is an addition on top of the V-cycle.
Features of element i: [r_i, r_{i-e_0}, r_{i+e_0}, ..., r_{i+e_{d-1}}] / ||r_i||
(zeros where the neighbour is outside a non-periodic box); the network is
y = tanh(F W1 + b1) W2 + b2; the loss over a set of rows is
sum_rows ||y - t||^2 / rows.

Acceptance (the reading of "kept only in cycles where its measured residual
contraction beats plain block Gauss-Seidel"): the outer iteration is
x <- x + V(0, b - A x); its first two iterations use the plain cycle and
measure kappa = (||r_2|| / ||r_0||)^(1/2); every later iteration adds the
correction delta computed from the cycle's own residual after post-smoothing
and keeps it only if ||r_new|| < kappa ||r_old||, else returns to the plain
cycle's result; two consecutive rejections switch the correction off.
"""
import numpy as np


def face_neighbours(mesh):
    """[ne, 2d] neighbour index at -e_0, +e_0, -e_1, ... (-1 outside)."""
    d = mesh.d
    out = np.full((mesh.ne, 2 * d), -1, dtype=np.int64)
    for k in range(d):
        for j, step in enumerate((-1, 1)):
            idx = mesh.idx.copy()
            idx[:, k] += step
            ok = (idx[:, k] >= 0) & (idx[:, k] < mesh.n[k])
            if mesh.periodic(k):
                idx[:, k] %= mesh.n[k]
                ok[:] = True
            e = (idx * np.asarray(mesh.stride)).sum(axis=1)
            out[:, 2 * k + j] = np.where(ok, e, -1)
    return out


def cut_face_neighbours(mesh, els):
    """[ne, 4] neighbours of the merged cut-cell elements (cutcell.CutMesh,
    cutldg.CutElements) at -e_0, +e_0, -e_1, +e_1: the element of the piece of
    the element's own phase in the cell next to its anchor cell (the host cell
    of its representative piece); -1 where that cell is outside the box, holds
    no piece of that phase, or belongs to the element itself."""
    out = np.full((els.ne, 4), -1, dtype=np.int64)
    for e in range(els.ne):
        i, j = mesh.pieces[els.reps[e]]["cell"]
        for k, (di, dj) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
            ii, jj = i + di, j + dj
            if not (0 <= ii < mesh.n and 0 <= jj < mesh.n):
                continue
            piece = mesh.piece_of.get((ii, jj, int(els.phase[e])))
            if piece is None:
                continue
            f = int(els.of_piece[piece])
            if f != e:
                out[e, k] = f
    return out


def features(r, nbrs):
    """r [ne, nb] -> (F [ne, (2d+1) nb], ||r_i||)."""
    ne, nb = r.shape
    nrm = np.sqrt((r * r).sum(axis=1))
    inv = 1.0 / (nrm + 1e-30)
    cols = [r]
    for f in range(nbrs.shape[1]):
        j = nbrs[:, f]
        cols.append(np.where((j >= 0)[:, None], r[np.maximum(j, 0)], 0.0))
    return np.concatenate(cols, axis=1) * inv[:, None], nrm


def unpack(w, nin, hid, nout):
    i = 0
    W1 = w[i:i + nin * hid].reshape(nin, hid); i += nin * hid
    b1 = w[i:i + hid]; i += hid
    W2 = w[i:i + hid * nout].reshape(hid, nout); i += hid * nout
    b2 = w[i:i + nout]
    return W1, b1, W2, b2


def forward(F, w, nin, hid, nout):
    W1, b1, W2, b2 = unpack(w, nin, hid, nout)
    H = np.tanh(F[:, :nin] @ W1 + b1)
    return H @ W2 + b2, H


def loss_and_grad(F, T, w, nin, hid, nout):
    """Mean over rows of ||y - t||^2 and its gradient (back-propagation)."""
    W1, b1, W2, b2 = unpack(w, nin, hid, nout)
    X = F[:, :nin]
    Y, H = forward(F, w, nin, hid, nout)
    rows = X.shape[0]
    D = Y - T
    loss = (D * D).sum() / rows
    dY = 2.0 * D / rows
    gW2 = H.T @ dY
    gb2 = dY.sum(axis=0)
    dZ = (dY @ W2.T) * (1.0 - H * H)
    gW1 = X.T @ dZ
    gb1 = dZ.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def residual_loss_and_grad(A, r, nbrs, w, nin, hid, nout):
    """Training objective of the correction: L = ||r - A delta||^2 / ||r||^2
    with delta_i = ||r_i|| y_i(features of r), and dL/dw by back-propagation
    (A symmetric, so dL/d delta = -2 A q / ||r||^2 with q = r - A delta)."""
    ne, nb = r.shape
    W1, b1, W2, b2 = unpack(w, nin, hid, nout)
    F, nrm = features(r, nbrs)
    Y, H = forward(F, w, nin, hid, nout)
    delta = nrm[:, None] * Y
    q = r.ravel() - A @ delta.ravel()
    rr = float(r.ravel() @ r.ravel())
    loss = float(q @ q) / rr
    g = (-2.0 * (A @ q) / rr).reshape(ne, nb)
    dY = nrm[:, None] * g
    gW2 = H.T @ dY
    gb2 = dY.sum(axis=0)
    dZ = (dY @ W2.T) * (1.0 - H * H)
    gW1 = F[:, :nin].T @ dZ
    gb1 = dZ.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])


def correction(mg, c, r, w, nin, hid, nout, nbrs):
    """delta = ||r_c,i|| y_i with y the network on the features of the
    cycle's own residual r_c = r - A c after its post-smoothing (from the
    smoother's stored blocks, as the cycle forms its residuals)."""
    ne = mg.levels[0].ne
    rc = mg.cycle_residual(0, c, r).reshape(ne, -1)
    F, nrm = features(rc, nbrs)
    y, _ = forward(F, w, nin, hid, nout)
    return (nrm[:, None] * y).ravel()


def solve_with_correction(mg, b, w, nin, hid, nout, nbrs, rtol=1e-10, maxit=100):
    """Outer iteration x <- x + V(0, b - A x) from x = 0 with the learned
    correction judged by the acceptance rule above.  Returns (x, relative
    residual history, decisions, ratios, kappa): decision -1 for a plain
    iteration, 1 kept, 0 undone; ratio = ||r_new|| / (kappa ||r_old||) for the
    judged iterations (0 otherwise)."""
    A = mg.A
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    bn = bn if bn > 0 else 1.0
    r = b - A @ x
    rel0 = rel = np.linalg.norm(r) / bn
    hist, dec, ratios = [rel], [], []
    kappa, active, consecutive, it = None, True, 0, 0
    while rel > rtol and it < maxit:
        c = mg.precondition(r)
        if active and it >= 2:
            delta = correction(mg, c, r, w, nin, hid, nout, nbrs)
            x_new = x + c + delta
            r_new = b - A @ x_new
            ratio = (np.linalg.norm(r_new) / bn) / (kappa * rel)
            ratios.append(ratio)
            if ratio < 1.0:
                x, r = x_new, r_new
                dec.append(1)
                consecutive = 0
            else:
                x = x + c
                r = b - A @ x
                dec.append(0)
                consecutive += 1
                if consecutive >= 2:
                    active = False
        else:
            x = x + c
            r = b - A @ x
            dec.append(-1)
            ratios.append(0.0)
        rel = np.linalg.norm(r) / bn
        it += 1
        hist.append(rel)
        if it == 2:
            kappa = np.sqrt(rel / rel0)
    return x, hist, dec, ratios, kappa
