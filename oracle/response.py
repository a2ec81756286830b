"""Fourier response of a drifting sinusoid and the f-fdot power plane.

The paper runs accelsearch with zmax = 0 or 50 (Sect. 3.2, Table 4) and
cites Ransom et al. (2002) for the method without stating it.  The
definitions here are derived from first principles:

* A unit-amplitude signal whose frequency (in bins of the series span)
  moves linearly from r - z/2 to r + z/2 over the span has the phase
  (r - z/2) u + z u^2 / 2 cycles at fractional time u in [0, 1).  Its DFT
  at bin k is N * rho(r - k, z) with
      rho(q, z) = integral_0^1 exp(2 pi i [(q - z/2) u + z u^2 / 2]) du.
* The plane value at (r, z) correlates the spectrum with that template
  over the 2m bins nearest r, normalised to unit energy:
      A(r, z) = sum_{k = floor(r)-m+1}^{floor(r)+m} A'_k conj(rho(r - k, z)) / sqrt(E),
      E = sum over the same 2m taps of |rho|^2,
  with bins outside [0, nfft/2) contributing 0.  The plane is sampled at
  half-bin spacing r = h/2 and at z_j = -zmax + j*dz.
* Readings: half-width m(z) = ceil(|z|/2) + extra (extra = 16); unit-energy
  normalisation so that noise powers stay Exp(1); half-bin spacing.

rho is evaluated here by composite Gauss-Legendre quadrature of its
defining integral (not by a closed form), so this module is independent of
any Fresnel-integral implementation.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

_GL_NODES = 20
_gl_x, _gl_w = np.polynomial.legendre.leggauss(_GL_NODES)


def rho_quad(q: float, z: float) -> complex:
    """rho(q, z) by composite Gauss-Legendre quadrature on [0, 1].

    The integrand's instantaneous frequency is bounded by |q| + |z|/2 cycles
    per unit; one 20-node panel per cycle (plus two) gives ~1e-14
    accuracy."""
    q = float(q)
    z = float(z)
    panels = int(math.ceil(abs(q) + 0.5 * abs(z))) + 2
    edges = np.linspace(0.0, 1.0, panels + 1)
    a = edges[:-1][:, None]
    b = edges[1:][:, None]
    u = 0.5 * (b - a) * _gl_x[None, :] + 0.5 * (a + b)
    w = 0.5 * (b - a) * _gl_w[None, :]
    ph = 2.0 * math.pi * ((q - 0.5 * z) * u + 0.5 * z * u * u)
    return complex(np.sum(w * np.cos(ph)), np.sum(w * np.sin(ph)))


def rho(q: float, z: float) -> complex:
    """rho(q, z): the sinc closed form at z = 0 (pinned to the quadrature by
    the tests), the quadrature of the defining integral otherwise."""
    if z == 0.0:
        q = float(q)
        if q == 0.0:
            return 1.0 + 0.0j
        return complex(math.cos(math.pi * q), math.sin(math.pi * q)) * (math.sin(math.pi * q) / (math.pi * q))
    return rho_quad(q, z)


def halfwidth(z: float, extra: int = 16) -> int:
    return int(math.ceil(abs(z) / 2.0)) + int(extra)


def z_values(zmax: int, dz: float) -> np.ndarray:
    """z_j = -zmax + j*dz for j = 0 .. 2*zmax/dz (row Z = zmax/dz is z = 0)."""
    if zmax == 0:
        return np.zeros(1)
    nz = int(round(2 * zmax / dz)) + 1
    return -float(zmax) + np.arange(nz, dtype=np.float64) * float(dz)


@lru_cache(maxsize=4096)
def taps(z: float, parity: int, extra: int = 16):
    """(t offsets, conj(rho) coefficients, E) for plane points r = k0 + parity/2:
    tap t in [-m+1, m] multiplies A'_{k0+t} by conj(rho(parity/2 - t, z))."""
    m = halfwidth(z, extra)
    t = np.arange(-m + 1, m + 1)
    frac = 0.5 * parity
    rho = np.array([rho_quad(frac - ti, z) for ti in t], dtype=np.complex128)
    E = float(np.sum(rho.real ** 2 + rho.imag ** 2))
    return t, np.conj(rho), E


def plane_row_direct(Ap: np.ndarray, z: float, extra: int = 16) -> np.ndarray:
    """FP64 [nfft] powers |A(h/2, z)|^2 for h = 0 .. nfft-1, by the direct sum."""
    M = Ap.shape[0]
    out = np.empty(2 * M, dtype=np.float64)
    for parity in (0, 1):
        t, g, E = taps(float(z), parity, extra)
        acc = np.zeros(M, dtype=np.complex128)
        for ti, gi in zip(t, g):
            lo = max(0, -int(ti))
            hi = min(M, M - int(ti))
            if hi > lo:
                acc[lo:hi] += Ap[lo + ti: hi + ti] * gi
        out[parity::2] = (acc.real ** 2 + acc.imag ** 2) / E
    return out


def plane_row_fftconv(Ap: np.ndarray, z: float, extra: int = 16) -> np.ndarray:
    """Same values as plane_row_direct, with the correlation computed by
    scipy's FFT convolution (a library step; checked against the direct
    sum in the tests).  Used to keep full-size acceleration cases fast."""
    from scipy.signal import fftconvolve
    M = Ap.shape[0]
    out = np.empty(2 * M, dtype=np.float64)
    for parity in (0, 1):
        t, g, E = taps(float(z), parity, extra)
        m = int(t[-1])
        kern = g[::-1]  # kern[v] = g at t = m - v
        full = fftconvolve(Ap, kern)
        acc = full[m: m + M]
        out[parity::2] = (acc.real ** 2 + acc.imag ** 2) / E
    return out


def power_plane(Ap: np.ndarray, zmax: int, dz: float, extra: int = 16,
                method: str = "direct") -> np.ndarray:
    """FP64 [n_z][nfft] plane of normalised powers."""
    zs = z_values(zmax, dz)
    fn = plane_row_direct if method == "direct" else plane_row_fftconv
    return np.stack([fn(Ap, float(z), extra) for z in zs])
