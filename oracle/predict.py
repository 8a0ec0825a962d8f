"""FP64 oracle of the step upstream of degridding -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the library never imports it.

The degridding paper takes its stack of 512 x 512 x 4 subgrids as given: they
are "pre-computed grid data" of the improved w-stacking method (paper,
Introduction), which it does not describe.  The reading used here follows
the published improved w-stacking method (Ye, Gull, Tan & Nikolic 2020,
MNRAS 491, 1146; Ye 2019, PhD thesis, Cambridge): the grid at a w-plane w_c
is the Fourier transform of the sky image after the image-plane correction
of the gridding kernels and the w-phase screen of that plane,

    G_c(u, v) = sum_{l, m} I(l, m) T(l, m) exp(-2 pi i (u l + v m + w_c (n - 1))),
    n = sqrt(1 - l^2 - m^2),

and a subgrid is a window of nx x ny uv cells of that grid at nz consecutive
w-planes, stored C-order [y = v][x = u][z = w-plane] like the stack the
degridding kernels read.  The discretisation (a reading where the method
leaves freedom; restated in the design notes):

  * image: N x N pixels, row b <-> m, column a <-> l, l_a = (a - N/2) dl and
    m_b = (b - N/2) dl with dl = theta / N (theta: image width in direction
    cosines); pixels with l^2 + m^2 >= 1 (no sky there) contribute nothing;
  * subgrid cell (x, y) of subgrid s: u = (x - N/2 + u0_s) / theta,
    v = (y - N/2 + v0_s) / theta (integer cell offsets u0_s, v0_s), so that
    u l_a = (x - N/2 + u0_s)(a - N/2) / N;
  * w-planes w_c = w0_s + c dw_s (wavelengths), c = 0 .. nz - 1;
  * T: the image-plane correction (a real taper), an input like the image.

predict() evaluates it with numpy's FP64 FFT (a library primitive for the
sum over pixels); predict_direct() takes the sum term by term (tiny sizes
only).  The tests pin both against closed forms and each other.
"""
from __future__ import annotations

import numpy as np


def n_minus_one(N: int, theta: float):
    """(n - 1) per pixel, float64 [N][N], and the mask of pixels inside the
    unit circle (outside: n - 1 is set to 0 and the pixel is masked)."""
    idx = (np.arange(N, dtype=np.float64) - N // 2) * (theta / N)
    l = idx[None, :]
    m = idx[:, None]
    r2 = l * l + m * m
    inside = r2 < 1.0
    nm1 = np.zeros((N, N), dtype=np.float64)
    # n - 1 = -r^2 / (1 + sqrt(1 - r^2)): no cancellation near the centre
    nm1[inside] = -(r2[inside]) / (1.0 + np.sqrt(1.0 - r2[inside]))
    return nm1, inside


def _screen(N, theta, u0, v0, w):
    """exp(-2 pi i (u0 (a - N/2) / N + v0 (b - N/2) / N + w (n - 1))) on the
    pixels inside the unit circle, 0 outside; complex128 [N][N]."""
    nm1, inside = n_minus_one(N, theta)
    a = np.arange(N, dtype=np.int64) - N // 2
    # the uv offset phase in exact integer turns modulo N
    turns_uv = ((u0 * a[None, :] + v0 * a[:, None]) % N).astype(np.float64) / N
    ph = np.exp(-2j * np.pi * (turns_uv + w * nm1))
    return np.where(inside, ph, 0.0)


def predict(image, theta, offsets, nz=4, taper=None):
    """Subgrids [S][N][N][nz] complex128 of the N x N image.

    offsets: [S][4] rows (u0, v0, w0, dw); u0, v0 integer cell offsets,
    w0, dw in wavelengths.  taper: real [N][N] or None (all ones).
    """
    img = np.asarray(image, dtype=np.complex128)
    N = img.shape[0]
    assert img.shape == (N, N) and N % 2 == 0
    T = np.ones((N, N)) if taper is None else np.asarray(taper, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.float64).reshape(-1, 4)
    out = np.empty((off.shape[0], N, N, nz), dtype=np.complex128)
    for s, (u0, v0, w0, dw) in enumerate(off):
        assert u0 == int(u0) and v0 == int(v0)
        for c in range(nz):
            J = img * T * _screen(N, theta, int(u0), int(v0), w0 + c * dw)
            # sum_{a,b} J[b][a] exp(-2 pi i ((x - N/2)(a - N/2) + (y - N/2)(b - N/2)) / N)
            out[s, :, :, c] = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(J)))
    return out


def predict_direct(image, theta, offsets, nz=4, taper=None):
    """The same sum taken term by term from its definition (tiny N only)."""
    img = np.asarray(image, dtype=np.complex128)
    N = img.shape[0]
    T = np.ones((N, N)) if taper is None else np.asarray(taper, dtype=np.float64)
    off = np.asarray(offsets, dtype=np.float64).reshape(-1, 4)
    dl = theta / N
    out = np.zeros((off.shape[0], N, N, nz), dtype=np.complex128)
    for s, (u0, v0, w0, dw) in enumerate(off):
        for c in range(nz):
            w = w0 + c * dw
            for y in range(N):
                v = (y - N // 2 + v0) / theta
                for x in range(N):
                    u = (x - N // 2 + u0) / theta
                    acc = 0j
                    for b in range(N):
                        m = (b - N // 2) * dl
                        for a in range(N):
                            l = (a - N // 2) * dl
                            if l * l + m * m >= 1.0:
                                continue
                            n = np.sqrt(1.0 - l * l - m * m)
                            acc += img[b, a] * T[b, a] * np.exp(-2j * np.pi * (u * l + v * m + w * (n - 1.0)))
                    out[s, y, x, c] = acc
    return out
