"""Learned element-local post-smoother: the plain definition of its features,
two-layer perceptron, mean-squared-error loss and gradient (oracle).

Not a step of the paper: the correction is an addition on top of the V-cycle.
Features of element i: [r_i, r_{i-e_0}, r_{i+e_0}, ..., r_{i+e_{d-1}}] / ||r_i||
(zeros where the neighbour is outside a non-periodic box); the network is
y = tanh(F W1 + b1) W2 + b2; the loss over a set of rows is
sum_rows ||y - t||^2 / rows.
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
