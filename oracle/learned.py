"""FP64 oracle of the learned force correction.

TEST INFRASTRUCTURE ONLY: the plain reference the CUDA feature stencil and the
CUDA MLP kernels are checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It imports nothing from the CUDA package and shares no
code with it.

The paper has no learned component.  This follows the extension's contract
(stated in the library's header): a 512-feature near-surface stencil of a
sphere -> MLP 512-64-64-6 with tanh -> correction of the hydrodynamic force
and torque, trained by full-batch Adam on
L = 1/(2n) sum_s sum_k w_k (y^_sk - t_sk/s_k)^2 with w_k = (s_k / max_j s_j)^2.
Everything here is NumPy in float64, one operation per line of the
definition, no blocking or fusion.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 512, 64, 6
N_PTS = 125
N_PARAMS = N_IN * N_H + N_H + N_H * N_H + N_H + N_H * N_OUT + N_OUT
N_NORM = 2 * N_IN + N_OUT


# ---- parameters ---------------------------------------------------------------------
def unpack(P):
    """Flat parameter vector -> (W1 [512,64], b1, W2 [64,64], b2, W3 [64,6], b3);
    weights are stored [input][output], the output index fastest."""
    P = np.asarray(P, dtype=np.float64)
    assert P.size == N_PARAMS
    o = 0
    W1 = P[o:o + N_IN * N_H].reshape(N_IN, N_H); o += N_IN * N_H
    b1 = P[o:o + N_H]; o += N_H
    W2 = P[o:o + N_H * N_H].reshape(N_H, N_H); o += N_H * N_H
    b2 = P[o:o + N_H]; o += N_H
    W3 = P[o:o + N_H * N_OUT].reshape(N_H, N_OUT); o += N_H * N_OUT
    b3 = P[o:o + N_OUT]; o += N_OUT
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3])


def split_norm(norm):
    norm = np.asarray(norm, dtype=np.float64)
    return norm[:N_IN], norm[N_IN:2 * N_IN], norm[2 * N_IN:]


# ---- network ------------------------------------------------------------------------
def forward(P, norm, X):
    """Activations of the network for samples X [n, 512]."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    mu, inv_sigma, s_out = split_norm(norm)
    xh = (np.asarray(X, dtype=np.float64) - mu) * inv_sigma
    z1 = xh @ W1 + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2 + b2
    h2 = np.tanh(z2)
    yh = h2 @ W3 + b3
    return {"xh": xh, "h1": h1, "h2": h2, "yh": yh, "y": yh * s_out}


def loss_weights(s_out):
    """w_k = (s_k / max_j s_j)^2: the loss of output k in the physical units
    of the largest target (the targets are dimensionless already), while each
    output keeps its own scale s_k."""
    s_out = np.asarray(s_out, dtype=np.float64)
    return (s_out / s_out.max()) ** 2


def loss(P, norm, X, T):
    """L = 1/(2n) sum_s sum_k w_k (y^_sk - t_sk / s_k)^2."""
    _, _, s_out = split_norm(norm)
    a = forward(P, norm, X)
    e = a["yh"] - np.asarray(T, dtype=np.float64) / s_out
    return 0.5 * np.sum(loss_weights(s_out) * e * e) / e.shape[0]


def gradient(P, norm, X, T):
    """dL/dP by the chain rule, written out layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(P)
    _, _, s_out = split_norm(norm)
    a = forward(P, norm, X)
    n = a["yh"].shape[0]
    d3 = loss_weights(s_out) * (a["yh"] - np.asarray(T, dtype=np.float64) / s_out) / n  # dL/dy^
    gW3 = a["h2"].T @ d3
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ W3.T) * (1.0 - a["h2"] ** 2)  # dL/dz2 (tanh' = 1 - tanh^2)
    gW2 = a["h1"].T @ d2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2.T) * (1.0 - a["h1"] ** 2)  # dL/dz1
    gW1 = a["xh"].T @ d1
    gb1 = d1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam(P, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at step count t >= 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return P - lr * mh / (np.sqrt(vh) + eps), m, v


def fit_normalization(X, T):
    """mu and 1/sigma per input (sigma < 1e-6 -> 1); output scale s_k = RMS of
    target k (>= 1e-12).  Each output is scaled to its own target, so a
    near-zero lateral target is predicted near zero; the loss weights
    (loss_weights) keep such components from dominating the fit."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    inv = np.where(sd > 1e-6, 1.0 / np.where(sd > 1e-6, sd, 1.0), 1.0)
    rms = np.sqrt((T * T).mean(axis=0))
    return np.concatenate([mu, inv, np.maximum(rms, 1e-12)])


# ---- feature stencil ----------------------------------------------------------------
def body_velocity(p, xc, shape, bc_z):
    """U + Omega x r at point xc, r the minimum-image offset from the centre."""
    r = np.array(xc, dtype=np.float64) - np.asarray(p["x"], dtype=np.float64)
    for a in range(3):
        if a == 2 and bc_z:
            continue
        L = shape[a]
        if r[a] > 0.5 * L:
            r[a] -= L
        elif r[a] < -0.5 * L:
            r[a] += L
    return np.asarray(p["u"], dtype=np.float64) + np.cross(np.asarray(p["omega"], dtype=np.float64), r)


def features(pdf, indicator, owner, particles, p_index, F, T, u_ref, rho0, bc_z, lattice_c):
    """The 512 features of particle p_index.

    pdf        stored post-collision PDFs (19, nz, ny, nx)
    indicator  solid indicator per cell (nz, ny, nx): PSM min(sum eps, 1), MEM 0/1
    owner      MEM owner per cell (0 fluid, s+1 solid) or None (PSM)
    particles  particle dicts of the state the step used
    F, T       the step's hydrodynamic force and torque of the particle
    lattice_c  (19, 3) lattice velocities
    """
    nq, nz, ny, nx = pdf.shape
    shape = (nx, ny, nz)
    c = np.asarray(lattice_c, dtype=np.float64)
    P = particles[p_index]
    X = np.asarray(P["x"], dtype=np.float64)
    U = np.asarray(P["u"], dtype=np.float64)
    R = 0.5 * P["diameter"]
    h = 0.5 * (R + 2.0)
    out = np.zeros(N_IN)

    def cell_value(ix, iy, iz):
        """(indicator, velocity) of one cell; None beyond a closed wall."""
        x = ix % nx
        y = iy % ny
        if bc_z:
            if iz < 0 or iz >= nz:
                return None
            z = iz
        else:
            z = iz % nz
        e = float(indicator[z, y, x])
        if owner is not None and owner[z, y, x] > 0:
            v = body_velocity(particles[owner[z, y, x] - 1], (x + 0.5, y + 0.5, z + 0.5), shape, bc_z)
        else:
            f = pdf[:, z, y, x]
            v = (f[:, None] * c).sum(axis=0) / rho0
        return e, v

    for k in range(5):
        for j in range(5):
            for i in range(5):
                s = i + 5 * j + 25 * k
                pos = X + h * np.array([i - 2, j - 2, k - 2], dtype=np.float64)
                cc = pos - 0.5  # in cell-centre coordinates
                base = np.floor(cc).astype(int)
                fr = cc - base
                eps = 0.0
                u = np.zeros(3)
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            w = ((fr[0] if dx else 1 - fr[0]) * (fr[1] if dy else 1 - fr[1])
                                 * (fr[2] if dz else 1 - fr[2]))
                            cv = cell_value(base[0] + dx, base[1] + dy, base[2] + dz)
                            if cv is None:
                                continue
                            eps += w * cv[0]
                            u += w * cv[1]
                out[s] = eps
                for a in range(3):
                    out[N_PTS * (1 + a) + s] = (u[a] - U[a]) / u_ref
    D = P["diameter"]
    fs = rho0 * u_ref ** 2 * D ** 2
    out[500:503] = U / u_ref
    out[503:506] = np.asarray(P["omega"], dtype=np.float64) * R / u_ref
    out[506:509] = np.asarray(F, dtype=np.float64) / fs
    out[509:512] = np.asarray(T, dtype=np.float64) / (fs * D)
    return out
