"""Mie series for a homogeneous dielectric sphere (test infrastructure).

Bohren & Huffman, "Absorption and Scattering of Light by Small Particles"
(1983), Section 4.4 and Appendix A: e^{-i omega t}, relative index
m = sqrt(eps_r) (mu_r = 1), size parameter x = k_e a. Coefficients a_n, b_n
from Riccati–Bessel functions with the logarithmic derivative D_n(mx)
computed by downward recurrence; amplitude functions S1, S2 from the angle
functions pi_n, tau_n.

For the incident field E = x_hat e^{ikz} the scattered field is
E_s ~ e^{ikr}/(-ikr) [cos(phi) S2(theta) theta_hat - sin(phi) S1(theta) phi_hat],
so the far-field pattern (coefficient of e^{ikr}/r) is
E_inf = (i/k) [cos(phi) S2 theta_hat - sin(phi) S1 phi_hat].
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(x: float, m: complex, nmax: int | None = None):
    """a_n, b_n for n = 1..nmax (Bohren & Huffman eq. 4.88 with D_n, Appendix A)."""
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1 / 3) + 2))
    mx = m * x
    nstart = int(max(nmax, abs(mx))) + 16
    D = np.zeros(nstart + 1, dtype=np.complex128)
    for n in range(nstart, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    n = np.arange(0, nmax + 1)
    psi = x * spherical_jn(n, x)                           # psi_n(x)
    xi = x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))  # xi_n(x)
    nn = np.arange(1, nmax + 1)
    Dn = D[1:nmax + 1]
    ta = Dn / m + nn / x
    tb = m * Dn + nn / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return a, b


def amplitudes(x: float, m: complex, theta):
    """S1(theta), S2(theta) (Bohren & Huffman eq. 4.74)."""
    a, b = coefficients(x, m)
    nmax = len(a)
    mu = np.cos(np.asarray(theta, dtype=np.float64))
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    pi_prev = np.zeros_like(mu)
    pi_n = np.ones_like(mu)
    for n in range(1, nmax + 1):
        tau_n = n * mu * pi_n - (n + 1) * pi_prev
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_n + b[n - 1] * tau_n)
        S2 += f * (a[n - 1] * tau_n + b[n - 1] * pi_n)
        pi_next = ((2 * n + 1) * mu * pi_n - (n + 1) * pi_prev) / n
        pi_prev, pi_n = pi_n, pi_next
    return S1, S2


def efficiencies(x: float, m: complex):
    """Q_ext, Q_sca (Bohren & Huffman eqs. 4.61, 4.62)."""
    a, b = coefficients(x, m)
    n = np.arange(1, len(a) + 1)
    qext = 2.0 / x ** 2 * np.sum((2 * n + 1) * (a + b).real)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (abs(a) ** 2 + abs(b) ** 2))
    return qext, qsca


def far_field(k: float, radius: float, eps_r: complex, dirs):
    """Cartesian far-field pattern E_inf(x_hat) for E_inc = x_hat e^{ikz}: [n, 3] complex."""
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    m = np.sqrt(complex(eps_r))
    if m.imag < 0:
        m = -m
    theta = np.arccos(np.clip(dirs[:, 2], -1.0, 1.0))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    S1, S2 = amplitudes(k * radius, m, theta)
    th_hat = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], 1)
    ph_hat = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], 1)
    E = (1j / k) * (np.cos(phi)[:, None] * S2[:, None] * th_hat
                    - np.sin(phi)[:, None] * S1[:, None] * ph_hat)
    return E
