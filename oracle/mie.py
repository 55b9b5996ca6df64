"""Mie series for plane-wave scattering by a perfectly conducting sphere.

Pins the EFIE inputs (Sec. 2, Eq. 7 and the RWG discretisation), not the
preconditioner: the textbook closed form with Riccati-Bessel functions
psi_n(x) = x j_n(x), xi_n(x) = x h_n^(2)(x) (the e^{+j w t} convention), coefficients
a_n = psi_n'(x)/xi_n'(x), b_n = psi_n(x)/xi_n(x), amplitude functions

    S1(th) = sum (2n+1)/(n(n+1)) [a_n pi_n + b_n tau_n],
    S2(th) = sum (2n+1)/(n(n+1)) [a_n tau_n + b_n pi_n],

pi_n = P_n^1(cos th)/sin th, tau_n = d P_n^1(cos th)/d th, th = scattering angle from
the forward direction.  Bistatic RCS: E-plane (the plane of the incident E-field)
sigma = lambda^2/pi |S2|^2, H-plane sigma = lambda^2/pi |S1|^2.  The sum runs to
n_max = x + 4 x^{1/3} + 2.  |S| is convention independent.
"""
import numpy as np
import scipy.special as sp


def _coeffs(x):
    nmax = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    jn = sp.spherical_jn(n, x)
    jnp = sp.spherical_jn(n, x, derivative=True)
    yn = sp.spherical_yn(n, x)
    ynp = sp.spherical_yn(n, x, derivative=True)
    hn = jn - 1j * yn
    hnp = jnp - 1j * ynp
    psi, dpsi = x * jn, jn + x * jnp
    xi, dxi = x * hn, hn + x * hnp
    return n, dpsi / dxi, psi / xi


def _pitau(n, th):
    mu = np.cos(th)
    N = len(n)
    pi = np.zeros((N, len(th)))
    tau = np.zeros((N, len(th)))
    p0 = np.zeros_like(mu)                 # pi_{n-2}
    p1 = np.zeros_like(mu)                 # pi_{n-1}; pi_0 = 0
    for i in range(N):                     # pi_1 = 1, pi_n recurrence (Bohren & Huffman)
        k = i + 1
        if k == 1:
            pk = np.ones_like(mu)
        else:
            pk = ((2 * k - 1) / (k - 1)) * mu * p1 - (k / (k - 1)) * p0
        pi[i] = pk
        tau[i] = k * mu * pk - (k + 1) * p1
        p0, p1 = p1, pk
    return pi, tau


def amplitudes(ka, th):
    n, a, b = _coeffs(ka)
    pi, tau = _pitau(n, np.atleast_1d(th))
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(f * (a[:, None] * pi + b[:, None] * tau), axis=0)
    S2 = np.sum(f * (a[:, None] * tau + b[:, None] * pi), axis=0)
    return S1, S2


def bistatic(ka, th, wavelength=1.0):
    """(sigma_E, sigma_H) in m^2 at scattering angles th (radians)."""
    S1, S2 = amplitudes(ka, th)
    c = wavelength ** 2 / np.pi
    return c * np.abs(S2) ** 2, c * np.abs(S1) ** 2


def monostatic(ka, wavelength=1.0):
    n, a, b = _coeffs(ka)
    s = np.sum((-1.0) ** n * (2 * n + 1) * (a - b))
    return wavelength ** 2 / (4.0 * np.pi) * abs(s) ** 2
