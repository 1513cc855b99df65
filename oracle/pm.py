"""FP64 CPU oracle of the long-range particle-mesh force of the TreePM split (TEST
INFRASTRUCTURE ONLY: only tests/, the smoke check and the bench's CPU-baseline leg use it).

The steps are those of Sec. 2.3 ("TreePM approach"), in the paper's order:
  1. clouds-in-cell (CIC) assignment of the particle masses to a periodic N^3 mesh (mesh
     points at i * Delta, Delta = L / N);
  2. discrete Fourier transform of the density;
  3. multiplication with the Green's function -4 pi G exp(-k^2 r_s^2) / k^2 (the long-range
     part of Eq. eqnksum), divided by the Fourier transforms of the CIC assignment and of the
     CIC interpolation, sinc^2(k_i Delta / 2) per axis each (the deconvolution "in the mean");
  4. inverse transform: the long-range potential on the mesh;
  5. forces on the mesh by the fourth-order finite difference
       d phi / dx ~ [8 (phi_{i+1} - phi_{i-1}) - (phi_{i+2} - phi_{i-2})] / (12 Delta);
  6. CIC interpolation of forces and potential to the particle positions.
numpy's FFT serves as the transform (a library primitive); everything else is written out.
Readings: the sign of Eq. (eqnksum) is taken so that the long-range and short-range
potentials add up to the periodic potential of Eq. (eqnpo1) (phi_lr is negative around a
particle); the k = 0 mode is zero (neutralising background).  Pins: tests/test_oracle_pm.py
(Ewald sums, momentum conservation, symmetric lattices).
"""
from __future__ import annotations

import numpy as np

TWO32 = 4294967296.0


def _cic_weights(pos_int: np.ndarray, n_grid: int):
    """Mesh index i and fraction d of every particle along each axis: x / Delta = i + d
    (exact in FP64: x_int * N / 2^32 with N a power of two)."""
    u = pos_int.astype(np.float64) * (n_grid / TWO32)
    i = np.floor(u).astype(np.int64)
    return i, u - i


def cic_assign(pos_int: np.ndarray, mass: np.ndarray, n_grid: int, L: float) -> np.ndarray:
    """Step 1: mass density on the mesh (mass / Delta^3 per point)."""
    i, d = _cic_weights(pos_int, n_grid)
    rho = np.zeros((n_grid, n_grid, n_grid))
    for ox in (0, 1):
        wx = d[0] if ox else 1.0 - d[0]
        for oy in (0, 1):
            wy = d[1] if oy else 1.0 - d[1]
            for oz in (0, 1):
                wz = d[2] if oz else 1.0 - d[2]
                np.add.at(rho, ((i[0] + ox) % n_grid, (i[1] + oy) % n_grid, (i[2] + oz) % n_grid),
                          mass * wx * wy * wz)
    return rho / (L / n_grid) ** 3


def green(n_grid: int, L: float, r_s: float, G: float = 1.0) -> np.ndarray:
    """Step 3: -4 pi G exp(-k^2 r_s^2) / k^2 / (W_assign W_interp), W = prod_i sinc^2(k_i Delta/2),
    on the numpy FFT frequency layout; zero at k = 0."""
    n = np.fft.fftfreq(n_grid, d=1.0 / n_grid)          # integer wave numbers
    k1 = 2.0 * np.pi * n / L
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    delta = L / n_grid

    def sinc(k):
        x = 0.5 * k * delta
        return np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))

    w = (sinc(kx) * sinc(ky) * sinc(kz)) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        g = -4.0 * np.pi * G * np.exp(-k2 * r_s * r_s) / k2 / (w * w)
    g[0, 0, 0] = 0.0
    return g


def potential_mesh(rho: np.ndarray, L: float, r_s: float, G: float = 1.0) -> np.ndarray:
    """Steps 2-4: the long-range potential on the mesh."""
    n_grid = rho.shape[0]
    return np.fft.ifftn(np.fft.fftn(rho) * green(n_grid, L, r_s, G)).real


def force_mesh(phi: np.ndarray, L: float) -> np.ndarray:
    """Step 5: a = -grad phi on the mesh, fourth-order differences, shape (3, N, N, N)."""
    delta = L / phi.shape[0]
    out = np.empty((3,) + phi.shape)
    for ax in range(3):
        d1 = np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)
        d2 = np.roll(phi, -2, axis=ax) - np.roll(phi, 2, axis=ax)
        out[ax] = -(8.0 * d1 - d2) / (12.0 * delta)
    return out


def cic_interp(field: np.ndarray, pos_int: np.ndarray) -> np.ndarray:
    """Step 6: CIC interpolation of a mesh field (..., N, N, N) to the particles."""
    n_grid = field.shape[-1]
    i, d = _cic_weights(pos_int, n_grid)
    out = np.zeros(field.shape[:-3] + (pos_int.shape[1],))
    for ox in (0, 1):
        wx = d[0] if ox else 1.0 - d[0]
        for oy in (0, 1):
            wy = d[1] if oy else 1.0 - d[1]
            for oz in (0, 1):
                wz = d[2] if oz else 1.0 - d[2]
                out += field[..., (i[0] + ox) % n_grid, (i[1] + oy) % n_grid, (i[2] + oz) % n_grid] \
                    * (wx * wy * wz)
    return out


def long_range(pos_int: np.ndarray, mass: np.ndarray, n_grid: int, L: float, r_s: float,
               G: float = 1.0, sinks: np.ndarray | None = None):
    """Long-range accelerations (n, 3) and potentials (n,) of the particles (integer
    coordinates, 3 x n; unit L / 2^32), or of the sinks' positions if given (3 x ns)."""
    pos_int = np.ascontiguousarray(pos_int, np.uint32)
    rho = cic_assign(pos_int, np.asarray(mass, np.float64), n_grid, L)
    phi = potential_mesh(rho, L, r_s, G)
    acc = force_mesh(phi, L)
    at = pos_int if sinks is None else np.ascontiguousarray(sinks, np.uint32)
    return cic_interp(acc, at).T, cic_interp(phi, at)
