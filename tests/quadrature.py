"""Brute-force quadrature of Gaussian integrals, for pinning the oracle on tiny inputs.

Independent of the oracle's Obara-Saika recursions: every integral here is evaluated by
Gauss-Hermite quadrature of polynomial-times-Gaussian integrands (exact for the polynomial
degrees involved), and the Coulomb operator by its Gaussian transform
    1/r = (2/sqrt(pi)) int_0^inf exp(-u^2 r^2) du,
with u mapped to t in [0, 1) by u = sqrt(s) t / sqrt(1 - t^2) and Gauss-Legendre nodes in t.
Kinetic energy uses the gradient form T = (1/2) <grad mu | grad nu>, a different formula from the
oracle's second-derivative form.

Pure NumPy, slow; use only for a handful of shells.
"""
from __future__ import annotations

import math

import numpy as np

GH_X, GH_W = np.polynomial.hermite.hermgauss(12)   # exact for degree <= 23
GL_X, GL_W = np.polynomial.legendre.leggauss(120)
GL_T = 0.5 * (GL_X + 1.0)
GL_WT = 0.5 * GL_W


def cartesians(l):
    out = []
    for x in range(l, -1, -1):
        for y in range(l - x, -1, -1):
            out.append((x, y, l - x - y))
    return out


class QShells:
    """Contracted Cartesian shells: list of (centre bohr, l, exps, raw coefs)."""

    def __init__(self, shells):
        self.shells = shells
        self.aos = []  # (centre, (lx,ly,lz), exps, coefs incl. shell-level primitive norm)
        for C, l, ex, co in shells:
            ex = np.asarray(ex, float)
            co = np.asarray(co, float) * (2 * ex / np.pi) ** 0.75 * (4 * ex) ** (l / 2)
            for c in cartesians(l):
                self.aos.append((np.asarray(C, float), c, ex, co))
        self.scale = np.ones(len(self.aos))
        S = overlap(self)
        self.scale = 1.0 / np.sqrt(np.diag(S))

    @property
    def n(self):
        return len(self.aos)


def _gauss1d_poly(i, A, j, B, a, b, extra=None):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2 [- g (x-C)^2]) dx by Gauss-Hermite.

    extra: optional (g, C) third Gaussian factor (vectorised over g arrays)."""
    if extra is None:
        p = a + b
        P = (a * A + b * B) / p
        c = a * A * A + b * B * B - p * P * P
        x = P + GH_X / math.sqrt(p)
        return np.sum(GH_W * (x - A) ** i * (x - B) ** j) * math.exp(-c) / math.sqrt(p)
    g, C = extra
    g = np.asarray(g, float)[:, None]
    p = a + b + g
    P = (a * A + b * B + g * C) / p
    c = a * A * A + b * B * B + g * C * C - p * P * P
    x = P + GH_X[None, :] / np.sqrt(p)
    val = np.sum(GH_W[None, :] * (x - A) ** i * (x - B) ** j, axis=1)
    return val * np.exp(-c[:, 0]) / np.sqrt(p[:, 0])


def overlap(q: QShells):
    n = q.n
    S = np.zeros((n, n))
    for m, (A, ca, ea, wa) in enumerate(q.aos):
        for k, (B, cb, eb, wb) in enumerate(q.aos):
            v = 0.0
            for a, x in zip(ea, wa):
                for b, y in zip(eb, wb):
                    v += x * y * np.prod([_gauss1d_poly(ca[d], A[d], cb[d], B[d], a, b) for d in range(3)])
            S[m, k] = v * q.scale[m] * q.scale[k]
    return S


def _d1(i, A, a):
    """d/dx [(x-A)^i exp(-a (x-A)^2)] as a list of (coef, power) terms."""
    t = [(-2.0 * a, i + 1)]
    if i > 0:
        t.append((float(i), i - 1))
    return t


def kinetic(q: QShells):
    n = q.n
    T = np.zeros((n, n))
    for m, (A, ca, ea, wa) in enumerate(q.aos):
        for k, (B, cb, eb, wb) in enumerate(q.aos):
            v = 0.0
            for a, x in zip(ea, wa):
                for b, y in zip(eb, wb):
                    s1 = [_gauss1d_poly(ca[d], A[d], cb[d], B[d], a, b) for d in range(3)]
                    tot = 0.0
                    for d in range(3):
                        g = 0.0
                        for c1, p1 in _d1(ca[d], A[d], a):
                            for c2, p2 in _d1(cb[d], B[d], b):
                                g += c1 * c2 * _gauss1d_poly(p1, A[d], p2, B[d], a, b)
                        prod = g
                        for e in range(3):
                            if e != d:
                                prod *= s1[e]
                        tot += prod
                    v += x * y * 0.5 * tot
            T[m, k] = v * q.scale[m] * q.scale[k]
    return T


def nuclear(q: QShells, charges_xyz, charges_Z):
    """V_mu nu = -sum_C Z_C <mu|1/|r-C||nu> by the Gaussian transform of 1/r."""
    n = q.n
    V = np.zeros((n, n))
    for m, (A, ca, ea, wa) in enumerate(q.aos):
        for k, (B, cb, eb, wb) in enumerate(q.aos):
            v = 0.0
            for a, x in zip(ea, wa):
                for b, y in zip(eb, wb):
                    p = a + b
                    t = GL_T
                    u2 = p * t * t / (1 - t * t)
                    du = math.sqrt(p) * (1 - t * t) ** -1.5
                    for C, Z in zip(charges_xyz, charges_Z):
                        f = np.ones_like(t)
                        for d in range(3):
                            f = f * _gauss1d_poly(ca[d], A[d], cb[d], B[d], a, b, extra=(u2, C[d]))
                        v -= Z * x * y * (2 / math.sqrt(math.pi)) * np.sum(GL_WT * du * f)
            V[m, k] = v * q.scale[m] * q.scale[k]
    return V


def _gauss2d(i, A, j, B, k, C, l, D, p, P, q, Q, u2):
    """int int (x1-A)^i (x1-B)^j (x2-C)^k (x2-D)^l exp(-p(x1-P)^2 - q(x2-Q)^2 - u2 (x1-x2)^2) dx1 dx2
    for an array of u2, by a 2D Gauss-Hermite grid after completing the square (M = L L^T)."""
    g = np.asarray(u2, float)
    m11, m12, m22 = p + g, -g, q + g
    det = m11 * m22 - m12 * m12
    r1, r2 = p * P, q * Q
    c1 = (m22 * r1 - m12 * r2) / det
    c2 = (m11 * r2 - m12 * r1) / det
    const = p * P * P + q * Q * Q - (c1 * r1 + c2 * r2)
    L11 = np.sqrt(m11)
    L21 = m12 / L11
    L22 = np.sqrt(m22 - L21 * L21)
    # x = c + L^{-T} y, L^{-T} = [[1/L11, -L21/(L11 L22)], [0, 1/L22]]
    Y1 = GH_X[None, :, None]
    Y2 = GH_X[None, None, :]
    x1 = c1[:, None, None] + Y1 / L11[:, None, None] - (L21 / (L11 * L22))[:, None, None] * Y2
    x2 = c2[:, None, None] + Y2 / L22[:, None, None]
    f = (x1 - A) ** i * (x1 - B) ** j * (x2 - C) ** k * (x2 - D) ** l
    W = np.outer(GH_W, GH_W)[None]
    return np.sum(W * f, axis=(1, 2)) * np.exp(-const) / (L11 * L22)


def _eri_element(ao1, ao2, ao3, ao4):
    """(mu nu|lambda sigma) of four unscaled contracted Cartesian AOs by quadrature."""
    (A, ca, ea, wa), (B, cb, eb, wb), (C, cc, ec, wc), (D, cd, ed, wd) = ao1, ao2, ao3, ao4
    v = 0.0
    for a, xa in zip(ea, wa):
        for b, xb in zip(eb, wb):
            p = a + b
            P = (a * A + b * B) / p
            Kab = math.exp(-a * b / p * np.sum((A - B) ** 2))
            for c, xc in zip(ec, wc):
                for d, xd in zip(ed, wd):
                    qq = c + d
                    Q = (c * C + d * D) / qq
                    Kcd = math.exp(-c * d / qq * np.sum((C - D) ** 2))
                    rho = p * qq / (p + qq)
                    t = GL_T
                    u2 = rho * t * t / (1 - t * t)
                    du = math.sqrt(rho) * (1 - t * t) ** -1.5
                    f = np.ones_like(t)
                    for dd in range(3):
                        f = f * _gauss2d(ca[dd], A[dd], cb[dd], B[dd], cc[dd], C[dd], cd[dd], D[dd],
                                         p, P[dd], qq, Q[dd], u2)
                    v += xa * xb * xc * xd * Kab * Kcd * (2 / math.sqrt(math.pi)) * np.sum(GL_WT * du * f)
    return v


def eri(q1: QShells, q2: QShells):
    """(mu nu|lambda sigma), mu nu in q1, lambda sigma in q2, by quadrature."""
    n1, n2 = q1.n, q2.n
    out = np.zeros((n1, n1, n2, n2))
    for m1, o1 in enumerate(q1.aos):
        for m2, o2 in enumerate(q1.aos):
            for m3, o3 in enumerate(q2.aos):
                for m4, o4 in enumerate(q2.aos):
                    v = _eri_element(o1, o2, o3, o4)
                    out[m1, m2, m3, m4] = v * q1.scale[m1] * q1.scale[m2] * q2.scale[m3] * q2.scale[m4]
    return out


def eri_diagonal(q: QShells):
    """(mu nu|mu nu) for every AO pair of q, shape (n, n), by quadrature."""
    out = np.zeros((q.n, q.n))
    for m1, o1 in enumerate(q.aos):
        for m2, o2 in enumerate(q.aos):
            out[m1, m2] = _eri_element(o1, o2, o1, o2) * (q.scale[m1] * q.scale[m2]) ** 2
    return out


def dipole(q: QShells, origin=(0.0, 0.0, 0.0)):
    """<mu| r - origin |nu>, shape (3, n, n)."""
    n = q.n
    M = np.zeros((3, n, n))
    o = np.asarray(origin, float)
    for m, (A, ca, ea, wa) in enumerate(q.aos):
        for k, (B, cb, eb, wb) in enumerate(q.aos):
            for comp in range(3):
                v = 0.0
                for a, x in zip(ea, wa):
                    for b, y in zip(eb, wb):
                        prod = 1.0
                        for d in range(3):
                            if d == comp:
                                # (x - o) = (x - A) + (A - o)
                                s = (_gauss1d_poly(ca[d] + 1, A[d], cb[d], B[d], a, b)
                                     + (A[d] - o[d]) * _gauss1d_poly(ca[d], A[d], cb[d], B[d], a, b))
                            else:
                                s = _gauss1d_poly(ca[d], A[d], cb[d], B[d], a, b)
                            prod *= s
                        v += x * y * prod
                M[comp, m, k] = v * q.scale[m] * q.scale[k]
    return M
