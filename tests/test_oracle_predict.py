"""Pins of the FP64 oracle of the subgrid producer (oracle/predict.py).

The producer's sum is fixed by the improved w-stacking method: a w-plane
grid is the Fourier transform of the corrected sky image times the w-phase
screen of the plane.  The oracle evaluates it with an FFT; these checks tie
it to things other than itself:
  * brute force: the sum over pixels taken term by term here, from the
    physical quantities (u, v, w in wavelengths, l, m, n direction cosines);
  * a point source: the grid is the analytic visibility of one source,
    V(u, v, w) = flux exp(-2 pi i (u l0 + v m0 + w (n0 - 1)));
  * Parseval: the energy of a plane is N^2 times that of its screened image;
  * an integer cell offset shifts the window over the same grid;
  * a real image with no w term gives a Hermitian grid, V(-u, -v) = conj V(u, v);
  * plane c of a stack is the single plane at w0 + c dw.
"""
import numpy as np
import pytest

from oracle import predict as P


def _image(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))


def _brute(image, taper, theta, u0, v0, w):
    """sum_{l,m} I T exp(-2 pi i (u l + v m + w (n - 1))) over every cell."""
    N = image.shape[0]
    l = (np.arange(N) - N // 2) * theta / N
    L, M = np.meshgrid(l, l)                    # M[b][a] = m_b, L[b][a] = l_a
    r2 = L ** 2 + M ** 2
    n = np.sqrt(np.clip(1 - r2, 0, None))
    inside = r2 < 1
    out = np.zeros((N, N), dtype=np.complex128)
    for y in range(N):
        for x in range(N):
            u = (x - N // 2 + u0) / theta
            v = (y - N // 2 + v0) / theta
            term = image * taper * np.exp(-2j * np.pi * (u * L + v * M + w * (n - 1)))
            out[y, x] = term[inside].sum()
    return out


@pytest.mark.parametrize("N,theta", [(8, 0.5), (6, 1.9), (10, 0.05)])
def test_fft_form_equals_the_sum_taken_term_by_term(N, theta):
    img = _image(N, 1)
    T = np.random.default_rng(2).uniform(0.5, 2.0, (N, N))
    offs = [(0, 0, 0.0, 1.0), (3, -2, 17.5, 2.25), (-5, 7, -40.0, -0.5)]
    got = P.predict(img, theta, offs, nz=3, taper=T)
    for s, (u0, v0, w0, dw) in enumerate(offs):
        for c in range(3):
            want = _brute(img, T, theta, u0, v0, w0 + c * dw)
            assert np.max(np.abs(got[s, :, :, c] - want)) <= 1e-12 * np.max(np.abs(want))
    # the oracle's own term-by-term form agrees too
    np.testing.assert_allclose(P.predict_direct(img, theta, offs[:2], nz=2, taper=T), got[:2, :, :, :2],
                               rtol=0, atol=1e-11)


def test_point_source_is_its_analytic_visibility():
    N, theta = 16, 0.4
    a0, b0, flux = 11, 5, 2.5 - 1.0j
    img = np.zeros((N, N), dtype=np.complex128)
    img[b0, a0] = flux
    l0 = (a0 - N // 2) * theta / N
    m0 = (b0 - N // 2) * theta / N
    n0 = np.sqrt(1 - l0 ** 2 - m0 ** 2)
    u0, v0, w0, dw = 4, -3, 123.25, 7.5
    got = P.predict(img, theta, [(u0, v0, w0, dw)], nz=4)[0]
    for y, x, c in [(0, 0, 0), (7, 3, 1), (15, 15, 3), (8, 8, 2)]:
        u = (x - N // 2 + u0) / theta
        v = (y - N // 2 + v0) / theta
        w = w0 + c * dw
        want = flux * np.exp(-2j * np.pi * (u * l0 + v * m0 + w * (n0 - 1)))
        assert abs(got[y, x, c] - want) <= 1e-12


def test_parseval():
    N, theta = 32, 0.8
    img = _image(N, 3)
    T = np.random.default_rng(4).uniform(0.1, 1.0, (N, N))
    got = P.predict(img, theta, [(2, 9, 31.0, 3.0)], nz=4, taper=T)[0]
    _, inside = P.n_minus_one(N, theta)
    energy = np.sum(np.abs(img * T)[inside] ** 2)
    for c in range(4):
        assert abs(np.sum(np.abs(got[:, :, c]) ** 2) - N * N * energy) <= 1e-12 * N * N * energy


def test_integer_offsets_shift_the_window():
    N, theta = 16, 0.6
    img = _image(N, 5)
    g0 = P.predict(img, theta, [(0, 0, 10.0, 1.0)], nz=2)[0]
    gu = P.predict(img, theta, [(1, 0, 10.0, 1.0)], nz=2)[0]
    gv = P.predict(img, theta, [(0, 3, 10.0, 1.0)], nz=2)[0]
    np.testing.assert_allclose(gu[:, :-1], g0[:, 1:], rtol=0, atol=1e-11)
    np.testing.assert_allclose(gv[:-3, :], g0[3:, :], rtol=0, atol=1e-11)


def test_real_image_without_w_term_is_hermitian():
    N, theta = 16, 0.5
    img = np.random.default_rng(6).standard_normal((N, N))
    g = P.predict(img, theta, [(0, 0, 0.0, 0.0)], nz=1)[0, :, :, 0]
    # cell x <-> u = (x - N/2) / theta, so -u is cell N - x
    for y in range(1, N):
        for x in range(1, N):
            assert abs(g[N - y, N - x] - np.conj(g[y, x])) <= 1e-12 * np.max(np.abs(g))
    # with a w term the screen breaks the symmetry
    gw = P.predict(img, theta, [(0, 0, 50.0, 0.0)], nz=1)[0, :, :, 0]
    assert abs(gw[N - 3, N - 5] - np.conj(gw[3, 5])) > 1e-6


def test_plane_c_is_the_single_plane_at_its_w():
    N, theta = 16, 0.7
    img = _image(N, 7)
    stack = P.predict(img, theta, [(1, 2, -20.0, 4.5)], nz=4)[0]
    for c in range(4):
        single = P.predict(img, theta, [(1, 2, -20.0 + 4.5 * c, 0.0)], nz=1)[0, :, :, 0]
        np.testing.assert_allclose(stack[:, :, c], single, rtol=0, atol=1e-12)


def test_pixels_outside_the_unit_circle_contribute_nothing():
    N, theta = 8, 2.4                           # the corners lie outside l^2 + m^2 < 1
    nm1, inside = P.n_minus_one(N, theta)
    assert not inside.all() and inside.any()
    img = np.zeros((N, N), dtype=np.complex128)
    img[~inside] = 1.0
    assert np.all(P.predict(img, theta, [(0, 0, 3.0, 1.0)], nz=2) == 0)
    # n - 1 from the cancellation-free form agrees with the plain one
    l = (np.arange(N) - N // 2) * theta / N
    L, M = np.meshgrid(l, l)
    plain = np.sqrt(np.clip(1 - L ** 2 - M ** 2, 0, None)) - 1
    np.testing.assert_allclose(nm1[inside], plain[inside], rtol=0, atol=1e-15)
