"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module produces input DATA only: the permittivity on the grid, its analytic
gradient, incident plane waves and random test vectors.  It holds none of the
method's arithmetic (no contrast, no kernels, no FFTs, no stencils); the oracle and
the CUDA library each turn these arrays into the operator on their own.

Grid convention (Section 2 of the paper): Omega = (0,1)^3, n points per dimension,
h = 1/(n+1), node i = (i1,i2,i3) in {1..n}^3 sits at x = i*h.  Arrays are C-ordered
[i3][i2][i1] (i1 fastest); vector fields are [d][i3][i2][i1].

Media (the paper describes its media only in words, so these Gaussian-bump media
stand in for them):
  * ``gaussian``  eps = 1 + a*exp(-|x-c|^2/(2 w^2)) * T(x), c = (1/2,1/2,1/2)
  * ``bumps``     eps = 1 + T(x) * sum_b a_b exp(-|x-c_b|^2/(2 w_b^2)),
                  a_b ~ U[0.1,0.5], w_b ~ U[0.05,0.12], c_b ~ U[0.2,0.8]^3
with the smooth taper T(x) = prod_d s(x_d), s(t) = S(t/delta) S((1-t)/delta),
S(u) = psi(u)/(psi(u)+psi(1-u)), psi(u) = exp(-1/u) for u>0 else 0, delta = 0.15.
T and all its derivatives vanish on the boundary of Omega, so eps - 1 extends by
zero to a smooth function of R^3, as the volume integral equation assumes.
Random draws come from splitmix64 (published by Steele, Lea and Flood, 2014),
drawn per bump in the order a, w, c_x, c_y, c_z.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 counter-based generator; ``uniform()`` gives doubles in [0,1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def grid_coords(n: int):
    """Node coordinates x_i = i*h, i = 1..n, h = 1/(n+1); returns (x, h)."""
    h = 1.0 / (n + 1)
    return np.arange(1, n + 1, dtype=np.float64) * h, h


def wavenumber_for_grid(n: int) -> float:
    """omega = k = pi*n/4: n/8 wavelengths across the unit cube, about 8 points per wavelength."""
    return math.pi * n / 4.0


# ---------------------------------------------------------------- taper ----

def _psi(u):
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    pos = u > 0
    out[pos] = np.exp(-1.0 / u[pos])
    return out


def _dpsi(u):
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    pos = u > 0
    out[pos] = np.exp(-1.0 / u[pos]) / (u[pos] * u[pos])
    return out


def _step(u):
    a, b = _psi(u), _psi(1.0 - u)
    return a / (a + b)


def _dstep(u):
    a, b = _psi(u), _psi(1.0 - u)
    da, db = _dpsi(u), -_dpsi(1.0 - u)
    return (da * (a + b) - a * (da + db)) / (a + b) ** 2


def taper_1d(t, delta: float = 0.15):
    """s(t) and s'(t) of the 1-D taper that is 1 in the middle and 0 at t=0 and t=1."""
    u, v = t / delta, (1.0 - t) / delta
    s = _step(u) * _step(v)
    ds = _dstep(u) * _step(v) / delta - _step(u) * _dstep(v) / delta
    return s, ds


# ---------------------------------------------------------------- media ----

def _bump_field(n, bumps, delta=0.15):
    """eps and grad eps for eps = 1 + T(x) * sum_b a_b exp(-|x-c_b|^2/(2 w_b^2))."""
    x, _ = grid_coords(n)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    P = [X1, X2, X3]
    g = np.zeros((n, n, n))
    dg = [np.zeros((n, n, n)) for _ in range(3)]
    for (a, w, c) in bumps:
        r2 = sum((P[d] - c[d]) ** 2 for d in range(3))
        e = a * np.exp(-r2 / (2.0 * w * w))
        g += e
        for d in range(3):
            dg[d] += -e * (P[d] - c[d]) / (w * w)
    s = [taper_1d(P[d], delta) for d in range(3)]
    T = s[0][0] * s[1][0] * s[2][0]
    dT = [s[0][1] * s[1][0] * s[2][0], s[0][0] * s[1][1] * s[2][0], s[0][0] * s[1][0] * s[2][1]]
    eps = 1.0 + T * g
    grad = np.stack([dT[d] * g + T * dg[d] for d in range(3)])
    return eps.astype(np.complex128), grad.astype(np.complex128)


def medium_gaussian(n: int, amplitude: float = 0.5, width: float = 0.15):
    """Centred Gaussian lens eps = 1 + a exp(-|x-c|^2/(2 w^2)) T(x); returns (eps, grad_eps)."""
    return _bump_field(n, [(amplitude, width, (0.5, 0.5, 0.5))])


def medium_gaussian_untapered(n: int, amplitude: float = 0.5, width: float = 0.08):
    """Narrow centred Gaussian without the taper, eps = 1 + a exp(-|x-c|^2/(2 w^2)),
    with its analytic gradient.  At w = 0.08 eps - 1 is below 3e-9 of its peak on
    the boundary of the unit cube, and its derivatives stay moderate, so finite
    differences of eps reach their asymptotic order already at n = 32."""
    x, _ = grid_coords(n)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    P = [X1, X2, X3]
    r2 = sum((P[d] - 0.5) ** 2 for d in range(3))
    e = amplitude * np.exp(-r2 / (2.0 * width * width))
    grad = np.stack([-e * (P[d] - 0.5) / (width * width) for d in range(3)])
    return (1.0 + e).astype(np.complex128), grad.astype(np.complex128)


def draw_bumps(seed: int, count: int):
    rng = SplitMix64(seed)
    bumps = []
    for _ in range(count):
        a = 0.1 + 0.4 * rng.uniform()
        w = 0.05 + 0.07 * rng.uniform()
        c = tuple(0.2 + 0.6 * rng.uniform() for _ in range(3))
        bumps.append((a, w, c))
    return bumps


def medium_bumps(n: int, seed: int, count: int):
    """Sum of ``count`` seeded Gaussian bumps, tapered; returns (eps, grad_eps)."""
    return _bump_field(n, draw_bumps(seed, count))


def medium_lossy(n: int, seed: int, count: int, sigma_over_omega: float):
    """Bump medium with a conductivity term: eps_c = eps + i*(sigma/omega)*T(x)."""
    eps, grad = medium_bumps(n, seed, count)
    x, _ = grid_coords(n)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    P = [X1, X2, X3]
    s = [taper_1d(P[d]) for d in range(3)]
    T = s[0][0] * s[1][0] * s[2][0]
    dT = [s[0][1] * s[1][0] * s[2][0], s[0][0] * s[1][1] * s[2][0], s[0][0] * s[1][0] * s[2][1]]
    eps = eps + 1j * sigma_over_omega * T
    grad = grad + 1j * sigma_over_omega * np.stack(dT)
    return eps, grad


# ------------------------------------------------------ incident fields ----

def plane_wave(n: int, k: float, direction, polarisation):
    """E^i = p exp(i k d.x) on the grid, shape (3, n, n, n) complex128."""
    x, _ = grid_coords(n)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(polarisation, dtype=np.float64)
    phase = np.exp(1j * k * (d[0] * X1 + d[1] * X2 + d[2] * X3))
    return np.stack([p[c] * phase for c in range(3)])


def fibonacci_directions(count: int):
    """``count`` unit directions on a Fibonacci sphere: z_j = 1-(2j+1)/count, phi_j = j*pi*(3-sqrt 5)."""
    out = []
    ga = math.pi * (3.0 - math.sqrt(5.0))
    for j in range(count):
        z = 1.0 - (2.0 * j + 1.0) / count
        r = math.sqrt(max(0.0, 1.0 - z * z))
        out.append((r * math.cos(j * ga), r * math.sin(j * ga), z))
    return out


def polarisations(d):
    """Two unit polarisations orthogonal to d: p1 = normalise(d x a), p2 = d x p1."""
    d = np.asarray(d, dtype=np.float64)
    a = np.array([1.0, 0.0, 0.0]) if abs(d[2]) > 0.9 else np.array([0.0, 0.0, 1.0])
    p1 = np.cross(d, a)
    p1 /= np.linalg.norm(p1)
    p2 = np.cross(d, p1)
    return p1, p2


def plane_wave_block(n: int, k: float, count: int):
    """``count`` incident fields: Fibonacci directions x 2 polarisations, shape (count, 3, n, n, n)."""
    ndir = (count + 1) // 2
    fields = []
    for d in fibonacci_directions(ndir):
        p1, p2 = polarisations(d)
        fields.append(plane_wave(n, k, d, p1))
        fields.append(plane_wave(n, k, d, p2))
    return np.stack(fields[:count])


def random_field(n: int, seed: int, nrhs: int | None = None):
    """Standard complex normal test vector of shape (3,n,n,n) or (nrhs,3,n,n,n)."""
    rng = np.random.default_rng(seed)
    shape = (3, n, n, n) if nrhs is None else (nrhs, 3, n, n, n)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


def random_medium(n: int, seed: int, amplitude: float = 0.3):
    """Rough random complex eps with a matching random gradient (for algebraic tests only)."""
    rng = np.random.default_rng(seed)
    eps = 1.0 + amplitude * (rng.uniform(0, 1, (n, n, n)) + 0.2j * rng.uniform(0, 1, (n, n, n)))
    grad = amplitude * (rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n)))
    return eps.astype(np.complex128), grad.astype(np.complex128)


# ------------------------------------------------------- named workloads ----

def workload(name: str):
    """The named synthetic workloads: returns dict(n, omega, eps, grad, einc)."""
    if name == "n16_gaussian":
        n = 16
        k = wavenumber_for_grid(n)
        eps, grad = medium_gaussian(n)
        einc = plane_wave(n, k, (0, 0, 1), (1, 0, 0))[None]
    elif name == "n64_bumps8":
        n = 64
        k = wavenumber_for_grid(n)
        eps, grad = medium_bumps(n, seed=2, count=8)
        einc = plane_wave(n, k, (0, 0, 1), (1, 0, 0))[None]
    elif name == "n64_bumps8_rhs64":
        n = 64
        k = wavenumber_for_grid(n)
        eps, grad = medium_bumps(n, seed=2, count=8)
        einc = plane_wave_block(n, k, 64)
    elif name == "n128_bumps32_rhs8":
        n = 128
        k = wavenumber_for_grid(n)
        eps, grad = medium_bumps(n, seed=5, count=32)
        einc = plane_wave_block(n, k, 8)
    elif name in ("n256_bumps32", "n256_bumps32_rhs8"):
        n = 256
        k = wavenumber_for_grid(n)
        eps, grad = medium_bumps(n, seed=6, count=32)
        einc = plane_wave(n, k, (0, 0, 1), (1, 0, 0))[None] if name == "n256_bumps32" else plane_wave_block(n, k, 8)
    else:
        raise KeyError(name)
    return dict(n=n, omega=k, eps=eps, grad=grad, einc=einc)


def uneven_batch(count: int = 32, sizes=(32, 48, 64, 96), base_seed: int = 100):
    """``count`` independent problems: problem q draws n from ``sizes`` (splitmix64,
    seed base_seed + q), k = pi n/4, its own 8-bump medium (same seed) and one
    plane wave along +z polarised along x."""
    out = []
    for q in range(count):
        rng = SplitMix64(base_seed + q)
        n = sizes[min(int(rng.uniform() * len(sizes)), len(sizes) - 1)]
        k = wavenumber_for_grid(n)
        eps, grad = medium_bumps(n, seed=base_seed + q, count=8)
        einc = plane_wave(n, k, (0, 0, 1), (1, 0, 0))
        out.append(dict(n=n, omega=k, eps=eps, grad=grad, einc=einc))
    return out


# ------------------------------------------------------------- 2-D inputs ----
# The 2-D variant (Sections 2 and 4): Omega = (0,1)^2, n points per dimension,
# h = 1/(n+1), arrays [i2][i1], vector fields [d][i2][i1] with two components.
# Media stand in for the three 2-D examples of Section 4, which are given only in
# words (a converging Gaussian lens, a square obstacle with smooth boundary, a
# random perturbation of that obstacle).

def wavenumber_for_grid_2d(n: int) -> float:
    """k = 2 pi (n+1)/6: six points per background wavelength, as in Section 4
    (n = 119 gives k/2pi = 20, the first row of Tables 1-3)."""
    return 2.0 * math.pi * (n + 1) / 6.0


def _window_1d(t, lo, hi, delta):
    """b(t) = S((t-lo)/delta) S((hi-t)/delta) and b'(t): 1 on [lo+delta, hi-delta], 0 outside (lo, hi)."""
    u, v = (t - lo) / delta, (hi - t) / delta
    b = _step(u) * _step(v)
    db = _dstep(u) * _step(v) / delta - _step(u) * _dstep(v) / delta
    return b, db


def medium2_lens(n: int, amplitude: float = 0.5, width: float = 0.12):
    """Converging Gaussian lens eps = 1 + a exp(-|x-c|^2/(2 w^2)) T(x), c = (1/2,1/2),
    T(x) = s(x1) s(x2) the taper; returns (eps (n,n), grad_eps (2,n,n))."""
    x, _ = grid_coords(n)
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    e = amplitude * np.exp(-((X1 - 0.5) ** 2 + (X2 - 0.5) ** 2) / (2.0 * width * width))
    s1, ds1 = taper_1d(X1)
    s2, ds2 = taper_1d(X2)
    T = s1 * s2
    g1 = -e * (X1 - 0.5) / (width * width)
    g2 = -e * (X2 - 0.5) / (width * width)
    eps = 1.0 + T * e
    grad = np.stack([ds1 * s2 * e + T * g1, s1 * ds2 * e + T * g2])
    return eps.astype(np.complex128), grad.astype(np.complex128)


def _square_profile(n, lo=0.3, hi=0.7, delta=0.06):
    x, _ = grid_coords(n)
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    b1, db1 = _window_1d(X1, lo, hi, delta)
    b2, db2 = _window_1d(X2, lo, hi, delta)
    return X1, X2, b1 * b2, db1 * b2, b1 * db2


def medium2_square(n: int, amplitude: float = 0.4):
    """Square obstacle with smooth boundary: eps = 1 + a b(x1) b(x2), b the smooth
    window that is 1 on [0.36, 0.64] and 0 outside (0.3, 0.7)."""
    _, _, B, dB1, dB2 = _square_profile(n)
    eps = 1.0 + amplitude * B
    grad = np.stack([amplitude * dB1, amplitude * dB2])
    return eps.astype(np.complex128), grad.astype(np.complex128)


def medium2_random(n: int, seed: int = 7, amplitude: float = 0.4, count: int = 24):
    """Random perturbation of the square obstacle: eps = 1 + b(x1) b(x2) (a + rho(x)),
    rho = sum of ``count`` Gaussian bumps with amplitude U[-0.15,0.15], width
    U[0.02,0.05], centre U[0.3,0.7]^2 (splitmix64, drawn in that order)."""
    X1, X2, B, dB1, dB2 = _square_profile(n)
    rng = SplitMix64(seed)
    rho = np.zeros_like(X1)
    dr1 = np.zeros_like(X1)
    dr2 = np.zeros_like(X1)
    for _ in range(count):
        a = -0.15 + 0.3 * rng.uniform()
        w = 0.02 + 0.03 * rng.uniform()
        c1 = 0.3 + 0.4 * rng.uniform()
        c2 = 0.3 + 0.4 * rng.uniform()
        e = a * np.exp(-((X1 - c1) ** 2 + (X2 - c2) ** 2) / (2.0 * w * w))
        rho += e
        dr1 += -e * (X1 - c1) / (w * w)
        dr2 += -e * (X2 - c2) / (w * w)
    q = amplitude + rho
    eps = 1.0 + B * q
    grad = np.stack([dB1 * q + B * dr1, dB2 * q + B * dr2])
    return eps.astype(np.complex128), grad.astype(np.complex128)


def plane_wave_2d(n: int, k: float):
    """The incident field of Section 4 (2-D): E^i = (0, e^{i k x1}), shape (2, n, n)."""
    x, _ = grid_coords(n)
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    return np.stack([np.zeros_like(X1, dtype=np.complex128), np.exp(1j * k * X1)])


def random_field_2d(n: int, seed: int, nrhs: int | None = None):
    """Standard complex normal test vector of shape (2,n,n) or (nrhs,2,n,n)."""
    rng = np.random.default_rng(seed)
    shape = (2, n, n) if nrhs is None else (nrhs, 2, n, n)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


def random_medium_2d(n: int, seed: int, amplitude: float = 0.3):
    """Rough random complex eps with a random gradient (algebraic tests only)."""
    rng = np.random.default_rng(seed)
    eps = 1.0 + amplitude * (rng.uniform(0, 1, (n, n)) + 0.2j * rng.uniform(0, 1, (n, n)))
    grad = amplitude * (rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n)))
    return eps.astype(np.complex128), grad.astype(np.complex128)


def workload_2d(name: str):
    """'<medium>2d_n<n>' with medium lens | square | random, e.g. 'lens2d_n119':
    returns dict(n, omega, eps, grad, einc) with einc of shape (1, 2, n, n)."""
    med, _, size = name.partition("2d_n")
    n = int(size)
    k = wavenumber_for_grid_2d(n)
    if med == "lens":
        eps, grad = medium2_lens(n)
    elif med == "square":
        eps, grad = medium2_square(n)
    elif med == "random":
        eps, grad = medium2_random(n)
    else:
        raise KeyError(name)
    return dict(n=n, omega=k, eps=eps, grad=grad, einc=plane_wave_2d(n, k)[None])
