"""Pins for the drifting-sinusoid response and the f-fdot plane."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import response as R


def _rho_fresnel(q, z):
    # Completing the square: (q - z/2) u + z u^2/2 = (z/2)(u + b)^2 - (q - z/2)^2/(2z),
    # b = (q - z/2)/z; substitute w = sqrt(2|z|)(u + b) and use scipy's Fresnel
    # integrals S(x) = int_0^x sin(pi t^2/2), C(x) = int_0^x cos(pi t^2/2).
    b = (q - z / 2) / z
    s = math.sqrt(2 * abs(z))
    S0, C0 = special.fresnel(s * b)
    S1, C1 = special.fresnel(s * (1 + b))
    val = complex(C1 - C0, math.copysign(1.0, z) * (S1 - S0)) / s
    return val * complex(math.cos(-math.pi * (q - z / 2) ** 2 / z), math.sin(-math.pi * (q - z / 2) ** 2 / z))


@pytest.mark.parametrize("q", [0.0, 0.5, -3.25, 7.5, 20.0])
def test_z0_is_sinc(q):
    ref = complex(math.cos(math.pi * q), math.sin(math.pi * q)) * (np.sinc(q))
    assert abs(R.rho_quad(q, 0.0) - ref) < 1e-13
    # the closed form rho() takes at z = 0 is the same function as the quadrature
    assert abs(R.rho(q, 0.0) - R.rho_quad(q, 0.0)) < 1e-13
    assert abs(R.rho(q + 0.25, 0.0) - R.rho_quad(q + 0.25, 0.0)) < 1e-13


@pytest.mark.parametrize("q,z", [(0.0, 1.0), (0.5, -2.0), (3.5, 10.0), (-40.0, 150.0), (60.5, -200.0), (116.0, 200.0)])
def test_quadrature_matches_fresnel_form(q, z):
    assert abs(R.rho_quad(q, z) - _rho_fresnel(q, z)) < 1e-10


@pytest.mark.parametrize("z", [0.0, 4.0, -37.0, 151.0])
def test_parseval_and_truncated_energy(z):
    # sum over all integer k of |rho(q - k, z)|^2 = int_0^1 |.|^2 du = 1.
    q0 = 0.5
    ks = np.arange(-int(abs(z)) - 400, int(abs(z)) + 401)
    e = sum(abs(R.rho_quad(q0 - k, z)) ** 2 for k in ks)
    assert abs(e - 1.0) < 2e-3
    _, _, E = R.taps(z, 1)
    assert E >= 0.98
    if z == 0.0:
        # half-integer sinc taps |q| <= 15.5: E = 1 - (2/pi^2) * trigamma(16.5)
        assert abs(E - (1.0 - 2.0 / math.pi ** 2 * special.polygamma(1, 16.5))) < 1e-12


def _chirp_spectrum(N, r0, z0, a=1.0):
    u = np.arange(N) / N
    y = a * np.cos(2 * np.pi * ((r0 - z0 / 2) * u + z0 * u * u / 2))
    return np.fft.rfft(y)[: N // 2]


@pytest.mark.parametrize("r0,z0", [(400.0, 0.0), (400.5, 0.0), (1000.0, 20.0), (1500.5, -36.0)])
def test_matched_filter_recovers_chirp_power(r0, z0):
    # A real chirp's spectrum near r0 is (N a / 2) rho(r0 - k, z0); the plane at
    # (r0, z0) collects all its energy in the 2m taps: |A|^2 = (N a/2)^2 E.
    N = 1 << 13
    A = _chirp_spectrum(N, r0, z0)
    row = R.plane_row_direct(A, z0)
    h = int(round(2 * r0))
    _, _, E = R.taps(z0, h % 2)
    expect = (N / 2) ** 2 * E
    assert abs(row[h] - expect) < 2e-3 * expect
    # and it is the maximum of the row
    assert int(np.argmax(row)) == h


def test_z0_integer_half_bins_are_raw_powers():
    rng = np.random.default_rng(0)
    A = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    row = R.plane_row_direct(A, 0.0)
    np.testing.assert_allclose(row[0::2], np.abs(A) ** 2, rtol=1e-12)


def test_direct_equals_fftconv():
    rng = np.random.default_rng(7)
    A = rng.standard_normal(2048) + 1j * rng.standard_normal(2048)
    for z in (0.0, 6.0, -30.0):
        np.testing.assert_allclose(R.plane_row_fftconv(A, z), R.plane_row_direct(A, z), rtol=1e-9, atol=1e-9)


def test_direct_sum_brute_tiny():
    # Plane value straight from the definition with Python loops.
    rng = np.random.default_rng(8)
    M = 40
    A = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    z = 5.0
    m = R.halfwidth(z)
    row = R.plane_row_direct(A, z)
    for h in (0, 1, 17, 38, 79):
        r = h / 2.0
        acc, E = 0j, 0.0
        for k in range(int(math.floor(r)) - m + 1, int(math.floor(r)) + m + 1):
            rho = R.rho_quad(r - k, z)
            E += abs(rho) ** 2
            if 0 <= k < M:
                acc += A[k] * rho.conjugate()
        assert abs(row[h] - abs(acc) ** 2 / E) < 1e-9 * max(1.0, row[h])


def test_z_values():
    assert R.z_values(0, 2.0).tolist() == [0.0]
    zs = R.z_values(200, 2.0)
    assert zs.shape[0] == 201 and zs[0] == -200 and zs[100] == 0 and zs[-1] == 200
