"""Second CPU loop, in the reduced (x, z, delta, lambda) form -- TEST INFRASTRUCTURE ONLY.

Its one job is to check, against the literal Algorithm 1 in ``mfs_oracle.c``, the identity that
lets a sweep keep only n- and m-length vectors. After any iteration of Algorithm 1 the lambda- and
gamma-updates together with the y-step give gamma = -U^T lambda and y = V^T x + U^T rho with
rho = F_U (b - A x). Substituting into the x-step (eq. vvt) and the lambda-update yields

    v       = rho - lambda/mu                                (m)
    x+      = F_V (d * x + A^T v + z + (delta - c)/mu)       (d_j = nonzeros in column j)
    z+      = proj_K(x+ - delta/mu)
    delta+  = delta + mu (z+ - x+)
    rho+    = F_U (b - A x+)
    lambda+ = lambda - mu rho+

The literal zero start (y = gamma = lambda = 0, z = delta = 0) corresponds to x = 0, v = 0 here.
FP64, numpy + scipy.sparse matrix-vector products; written separately from the C oracle and
sharing no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def proj_lorentz_rows(w):
    """Projection onto one Lorentz cone (eq. proj), written out for one vector."""
    w1 = w[0]
    a = np.linalg.norm(w[1:])
    if a <= -w1:
        return np.zeros_like(w)
    if a <= w1:
        return w.copy()
    out = 0.5 * w
    out[0] += 0.5 * a
    out[1:] += w1 * w[1:] / (2.0 * a)
    return out


def proj_K(cones, w):
    out = np.empty_like(w)
    off = 0
    for kind, s in cones:
        s = int(s)
        if kind == 1:
            out[off:off + s] = proj_lorentz_rows(w[off:off + s])
        else:
            out[off:off + s] = np.maximum(w[off:off + s], 0.0)
        off += s
    return out


class Reduced:
    def __init__(self, prob, mu=1.0):
        m, n = prob["m"], prob["n"]
        A = sp.coo_matrix((np.asarray(prob["val"], np.float64), (prob["row"], prob["col"])),
                          shape=(m, n)).tocsr()
        A.sum_duplicates()
        A.eliminate_zeros()
        self.A = A
        self.AT = A.T.tocsr()
        self.d = np.diff(A.tocsc().indptr).astype(np.float64)
        self.r = np.asarray(A.multiply(A).sum(axis=1)).ravel()
        self.b = np.asarray(prob["b"], np.float64)
        self.c = np.asarray(prob["c"], np.float64)
        self.cones = [(int(k), int(s)) for k, s in prob["cones"]]
        self.mu = float(mu)
        self.x = np.zeros(n)
        self.z = np.zeros(n)
        self.delta = np.zeros(n)
        self.lam = np.zeros(m)
        self.v = np.zeros(m)

    def iterate(self, k):
        mu = self.mu
        for _ in range(int(k)):
            x = (self.d * self.x + self.AT @ self.v + self.z + (self.delta - self.c) / mu) / (1.0 + self.d)
            z = proj_K(self.cones, x - self.delta / mu)
            self.delta = self.delta + mu * (z - x)
            rho = (self.b - self.A @ x) / (1.0 + self.r)
            self.lam = self.lam - mu * rho
            self.v = rho - self.lam / mu
            self.x, self.z = x, z
