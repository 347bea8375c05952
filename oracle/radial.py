"""Closed-form convolutions of the Helmholtz kernel with a radial bump (oracle pin).

TEST INFRASTRUCTURE ONLY.  For rho(y) = phi(|y - c|) with
phi(s) = exp(-1/(1 - (s/R)^2)) on s < R, the only surviving term of the Helmholtz
addition theorem e^{ik|x-y|}/(4 pi |x-y|) = ik sum_l j_l(k r<) h_l(k r>) sum_m Y Y*
is l = 0, which gives, with r = |x - c|,
    u(r)  = (G * rho)(x) = (e^{ikr}/r) I1(r) + j0(kr) I2(r),
    I1(r) = int_0^r s^2 phi(s) j0(ks) ds,   I2(r) = int_r^R s phi(s) e^{iks} ds,
and (G^d * rho)(x) = u'(r) (x_d - c_d)/r with
    u'(r) = (ik - 1/r)(e^{ikr}/r) I1(r) + k j0'(kr) I2(r).
G = e^{ik|x|}/(4 pi |x|) is the kernel of the volume integral equation (Section 2);
G^d = dG/dx_d.  The integrals are evaluated by composite Gauss-Legendre quadrature.
"""
from __future__ import annotations

import numpy as np


def phi(s, R):
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros_like(s)
    inside = s < R
    q = (s[inside] / R) ** 2
    out[inside] = np.exp(-1.0 / (1.0 - q))
    return out


def _gl_panels(a, b, panels=64, order=24):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, panels + 1)
    c = 0.5 * (edges[1:] + edges[:-1])
    r = 0.5 * (edges[1:] - edges[:-1])
    nodes = (c[:, None] + r[:, None] * x[None, :]).ravel()
    weights = (r[:, None] * w[None, :]).ravel()
    return nodes, weights


def _j0(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.ones_like(z)
    nz = np.abs(z) > 1e-8
    out[nz] = np.sin(z[nz]) / z[nz]
    out[~nz] = 1.0 - z[~nz] ** 2 / 6.0
    return out


def _dj0(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    nz = np.abs(z) > 1e-4
    out[nz] = (z[nz] * np.cos(z[nz]) - np.sin(z[nz])) / z[nz] ** 2
    out[~nz] = -z[~nz] / 3.0 + z[~nz] ** 3 / 30.0
    return out


def radial_fields(r, k, R=0.4, panels=64, order=24):
    """u(r) and u'(r) for an array of radii r (> 0)."""
    r = np.asarray(r, dtype=np.float64)
    u = np.zeros(r.shape, np.complex128)
    du = np.zeros(r.shape, np.complex128)
    for idx, rv in np.ndenumerate(r):
        rr = min(rv, R)
        if rr > 0:
            s, w = _gl_panels(0.0, rr, panels, order)
            I1 = np.sum(w * s * s * phi(s, R) * _j0(k * s))
        else:
            I1 = 0.0
        if rv < R:
            s, w = _gl_panels(rv, R, panels, order)
            I2 = np.sum(w * s * phi(s, R) * np.exp(1j * k * s))
        else:
            I2 = 0.0
        if rv == 0.0:
            u[idx] = I2  # I1(r)/r -> 0 and j0(0) = 1 at the centre
            du[idx] = 0.0
            continue
        e = np.exp(1j * k * rv)
        u[idx] = e / rv * I1 + _j0(k * rv) * I2
        du[idx] = (1j * k - 1.0 / rv) * e / rv * I1 + k * _dj0(k * rv) * I2
    return u, du


def bump_on_grid(n, R=0.4, c=(0.5, 0.5, 0.5)):
    """rho sampled at the grid nodes x_i = i/(n+1), shape (n,n,n) [i3][i2][i1]."""
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X1 - c[0]) ** 2 + (X2 - c[1]) ** 2 + (X3 - c[2]) ** 2)
    return phi(r, R).astype(np.complex128)


def exact_on_points(points, k, R=0.4, c=(0.5, 0.5, 0.5)):
    """(G*rho, G^1*rho, G^2*rho, G^3*rho) at the given points (P,3)."""
    P = np.asarray(points, dtype=np.float64)
    dx = P - np.asarray(c)[None, :]
    r = np.sqrt(np.sum(dx * dx, axis=1))
    u, du = radial_fields(r, k, R)
    out = np.zeros((4, P.shape[0]), np.complex128)
    out[0] = u
    safe = np.where(r > 0, r, 1.0)
    for d in range(3):
        out[1 + d] = np.where(r > 0, du * dx[:, d] / safe, 0.0)
    return out
