"""Seeded synthetic particle sets shared by the CUDA path, the oracle, the tests and the bench.

This module only draws inputs: it holds none of the gravity method's arithmetic (no
integer coordinates, keys, trees, multipoles or force kernels).  Every generator is
deterministic for a given seed (numpy PCG64), so the CPU oracle and the GPU path see
bit-identical inputs on any machine.

Workloads (stand-ins for the paper's test problems, none of whose data is used):

* ``plummer``   -- isolated Plummer sphere, the stand-in for the isolated halo test of
                   Sec. 3.2 (the paper uses a 1M-particle Hernquist halo).
* ``zeldovich`` -- periodic lattice displaced by a Gaussian random field with P(k) ~ k^-2
                   (Zel'dovich approximation), the stand-in for the cosmological boxes of
                   Sec. 3.3/3.4.
* ``zoom``      -- periodic box with a central high-resolution sphere of 64x number density
                   and 1/64 particle mass, the stand-in for the zoom runs of Sec. 3.5.
* ``multi_plummer`` -- many independent Plummer spheres of log-uniform size.
* ``lattice``   -- a perfect cubic lattice (zero net force by symmetry).
* ``sparse_pairs`` -- isolated particle pairs just inside a cutoff, scattered sparsely (every
                   group of consecutive particles spans many cutoff radii).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class ParticleSet:
    pos: np.ndarray          # (N, 3) float64 physical positions
    mass: np.ndarray         # (N,) float64
    eps_class: np.ndarray    # (N,) uint8 softening class index
    eps_table: np.ndarray    # (n_classes,) float64 softening lengths eps_0
    box_size: float          # L for periodic sets; 0.0 for isolated sets
    periodic: bool

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def plummer_mass_fraction(r: np.ndarray | float, a: float = 1.0) -> np.ndarray | float:
    """Untruncated Plummer enclosed mass fraction M(<r)/M = r^3 / (r^2 + a^2)^(3/2)."""
    r = np.asarray(r, dtype=np.float64)
    return r ** 3 / (r * r + a * a) ** 1.5


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0,
            r_trunc: float = 20.0, eps: float = 0.01) -> ParticleSet:
    """Equal-mass Plummer sphere truncated at ``r_trunc``.

    Radii come from the inverse cumulative mass profile r = a (X^(-2/3) - 1)^(-1/2) with
    X ~ U(0, M(r_trunc)); directions are isotropic.
    """
    g = _rng(seed)
    xmax = float(plummer_mass_fraction(r_trunc, a))
    x = g.uniform(0.0, xmax, size=n)
    x = np.maximum(x, 1e-300)
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    mu = g.uniform(-1.0, 1.0, size=n)
    phi = g.uniform(0.0, 2.0 * math.pi, size=n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    pos = np.stack([r * s * np.cos(phi), r * s * np.sin(phi), r * mu], axis=1)
    mass = np.full(n, total_mass / n, dtype=np.float64)
    return ParticleSet(pos=pos, mass=mass, eps_class=np.zeros(n, np.uint8),
                       eps_table=np.array([eps], np.float64), box_size=0.0, periodic=False)


def _gaussian_displacement(n: int, L: float, g: np.random.Generator) -> np.ndarray:
    """Zel'dovich displacement field psi on an n^3 grid for P(k) ~ k^-2 (unnormalised).

    White noise is drawn in real space and coloured in Fourier space, which keeps the
    field Hermitian.  psi(k) = i k delta(k) / k^2; the Nyquist planes are zeroed.
    Returns an array of shape (3, n, n, n), float64.
    """
    try:
        import scipy.fft as sfft
        fwd = lambda a: sfft.rfftn(a, workers=-1)
        inv = lambda a: sfft.irfftn(a, s=(n, n, n), workers=-1)
    except Exception:  # pragma: no cover
        fwd = np.fft.rfftn
        inv = lambda a: np.fft.irfftn(a, s=(n, n, n))
    white = g.standard_normal((n, n, n))
    dk = fwd(white)
    del white
    kf = 2.0 * math.pi / L
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz1 = np.fft.rfftfreq(n, d=1.0 / n)
    kx = k1[:, None, None]
    ky = k1[None, :, None]
    kz = kz1[None, None, :]
    k2 = (kx * kx + ky * ky + kz * kz) * kf * kf
    k2[0, 0, 0] = 1.0
    amp = np.sqrt(1.0 / k2)            # sqrt(P(k)) with P ~ k^-2
    nyq = n // 2
    mask = (np.abs(kx) == nyq) | (np.abs(ky) == nyq) | (kz == nyq)
    amp = np.where(mask, 0.0, amp)
    amp[0, 0, 0] = 0.0
    dk *= amp
    del amp
    psi = np.empty((3, n, n, n), dtype=np.float64)
    for ax, kk in enumerate((kx, ky, kz)):
        psi[ax] = inv(dk * (1j * kk * kf) / k2)
    return psi


def zeldovich(n_side: int, L: float, rms_in_spacing: float, seed: int,
              eps_in_spacing: float = 1.0 / 30.0, mass: float = 1.0) -> ParticleSet:
    """Periodic lattice q = (i + 1/2) Delta displaced by a k^-2 Zel'dovich field.

    The 3-D rms displacement |psi| is rescaled to ``rms_in_spacing`` lattice spacings.
    Softening eps_0 = eps_in_spacing * Delta.  All particles have mass ``mass``.
    """
    g = _rng(seed)
    delta = L / n_side
    psi = _gaussian_displacement(n_side, L, g)
    rms = math.sqrt(float(np.mean(psi[0] ** 2 + psi[1] ** 2 + psi[2] ** 2)))
    scale = (rms_in_spacing * delta / rms) if rms > 0 else 0.0
    idx = (np.arange(n_side, dtype=np.float64) + 0.5) * delta
    pos = np.empty((n_side ** 3, 3), dtype=np.float64)
    qx = np.broadcast_to(idx[:, None, None], (n_side,) * 3)
    qy = np.broadcast_to(idx[None, :, None], (n_side,) * 3)
    qz = np.broadcast_to(idx[None, None, :], (n_side,) * 3)
    for ax, q in enumerate((qx, qy, qz)):
        pos[:, ax] = (q + scale * psi[ax]).reshape(-1)
    del psi
    pos = np.mod(pos, L)
    pos[pos >= L] -= L
    n = n_side ** 3
    return ParticleSet(pos=pos, mass=np.full(n, mass, np.float64),
                       eps_class=np.zeros(n, np.uint8),
                       eps_table=np.array([eps_in_spacing * delta], np.float64),
                       box_size=float(L), periodic=True)


def zoom(n_lo_side: int, L: float, seed: int, density_contrast: int = 64,
         radius_frac: float = 0.125, rms_in_spacing: float = 0.5) -> ParticleSet:
    """Zoom-like periodic box: a central sphere of radius ``radius_frac*L`` holds
    ``density_contrast`` times the number density of the surroundings with particle mass
    1/density_contrast (mass density stays uniform).  Both sets are lattices displaced by a
    Gaussian field with rms ``rms_in_spacing`` of their own spacing.  Class 0 = low-res
    (eps = Delta_lo/30), class 1 = high-res (eps = Delta_hi/30).
    """
    g = _rng(seed)
    d_lo = L / n_lo_side
    refine = round(density_contrast ** (1.0 / 3.0))
    d_hi = d_lo / refine
    c = 0.5 * L
    R = radius_frac * L
    # low-res lattice outside the sphere
    psi = _gaussian_displacement(n_lo_side, L, g)
    rms = math.sqrt(float(np.mean(psi[0] ** 2 + psi[1] ** 2 + psi[2] ** 2)))
    s = rms_in_spacing * d_lo / rms
    q1 = (np.arange(n_lo_side) + 0.5) * d_lo
    qx, qy, qz = np.meshgrid(q1, q1, q1, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)
    keep = np.sum((q - c) ** 2, axis=1) >= R * R
    lo = q[keep] + s * np.stack([psi[0].ravel()[keep], psi[1].ravel()[keep],
                                 psi[2].ravel()[keep]], axis=1)
    del psi, qx, qy, qz, q
    # high-res lattice inside the sphere (field drawn on the sphere's bounding cube)
    n_hi = int(math.ceil(2 * R / d_hi))
    psi = _gaussian_displacement(n_hi, n_hi * d_hi, g)
    rms = math.sqrt(float(np.mean(psi[0] ** 2 + psi[1] ** 2 + psi[2] ** 2)))
    s = rms_in_spacing * d_hi / rms
    h1 = c - 0.5 * n_hi * d_hi + (np.arange(n_hi) + 0.5) * d_hi
    hx, hy, hz = np.meshgrid(h1, h1, h1, indexing="ij")
    h = np.stack([hx.ravel(), hy.ravel(), hz.ravel()], axis=1)
    inside = np.sum((h - c) ** 2, axis=1) < R * R
    hi = h[inside] + s * np.stack([psi[0].ravel()[inside], psi[1].ravel()[inside],
                                   psi[2].ravel()[inside]], axis=1)
    del psi, hx, hy, hz, h
    pos = np.concatenate([lo, hi], axis=0)
    pos = np.mod(pos, L)
    pos[pos >= L] -= L
    mass = np.concatenate([np.ones(len(lo)), np.full(len(hi), 1.0 / density_contrast)])
    cls = np.concatenate([np.zeros(len(lo), np.uint8), np.ones(len(hi), np.uint8)])
    return ParticleSet(pos=pos, mass=mass, eps_class=cls,
                       eps_table=np.array([d_lo / 30.0, d_hi / 30.0]),
                       box_size=float(L), periodic=True)


def multi_plummer(n_systems: int, seed: int, n_min: int = 1024, n_max: int = 65536,
                  eps: float = 0.01) -> list[ParticleSet]:
    """Independent Plummer spheres with N log-uniform in [n_min, n_max]."""
    g = _rng(seed)
    ns = np.rint(np.exp(g.uniform(math.log(n_min), math.log(n_max), size=n_systems)))
    seeds = g.integers(1, 2 ** 31 - 1, size=n_systems)
    return [plummer(int(k), int(sd), eps=eps) for k, sd in zip(ns, seeds)]


def lattice(n_side: int, L: float, eps_in_spacing: float = 1.0 / 30.0) -> ParticleSet:
    """Perfect periodic cubic lattice with points at (i + 1/2) Delta."""
    d = L / n_side
    q1 = (np.arange(n_side) + 0.5) * d
    qx, qy, qz = np.meshgrid(q1, q1, q1, indexing="ij")
    pos = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)
    n = pos.shape[0]
    return ParticleSet(pos=pos, mass=np.ones(n), eps_class=np.zeros(n, np.uint8),
                       eps_table=np.array([eps_in_spacing * d]), box_size=float(L),
                       periodic=True)


def sparse_pairs(n_pairs: int, L: float, sep: float, seed: int,
                 eps: float | None = None) -> ParticleSet:
    """Periodic box holding n_pairs particle pairs: pair centres uniform in the box, the two
    members sep apart along a uniformly random direction.  With sep just below a cutoff radius
    and few pairs per cutoff volume, most particles have exactly one neighbour inside the
    cutoff, close to it, and groups of consecutive particles spread far apart (a sparse
    active subset)."""
    g = _rng(seed)
    c = g.uniform(0.0, L, size=(n_pairs, 3))
    u = g.normal(size=(n_pairs, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pos = np.concatenate([c - 0.5 * sep * u, c + 0.5 * sep * u])
    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0
    n = pos.shape[0]
    return ParticleSet(pos=pos, mass=np.ones(n), eps_class=np.zeros(n, np.uint8),
                       eps_table=np.array([sep / 100.0 if eps is None else eps]),
                       box_size=float(L), periodic=True)


def subset(n: int, k: int, seed: int) -> np.ndarray:
    """Sorted random subset of k distinct indices out of n."""
    if k >= n:
        return np.arange(n, dtype=np.int64)
    g = _rng(seed)
    return np.sort(g.choice(n, size=k, replace=False)).astype(np.int64)


# ---- the five workload recipes (sizes, splits and seeds) ------------------------------------

def plummer_16k() -> ParticleSet:
    """Isolated Plummer sphere, N = 16384, eps = 0.01, seed 1001."""
    return plummer(16384, 1001)


def zeldovich_gpu(n_side: int, L: float, rms_in_spacing: float, seed: int):
    """The ``zeldovich`` recipe drawn on the GPU with torch (seeded torch generator, cuFFT), for
    sizes whose host FFTs would take minutes (512^3).  Same lattice, spectrum, Nyquist planes
    and rms rescaling as ``zeldovich``; the numbers differ from the numpy generator's (another
    random stream).  Returns a (N, 3) float64 CUDA tensor of positions in [0, L).  Masses are 1
    and eps_0 = Delta / 30, as in ``zeldovich``.
    """
    import torch
    n = n_side
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(seed)
    dk = torch.fft.rfftn(torch.randn((n, n, n), generator=gen, dtype=torch.float64, device=dev))
    kf = 2.0 * math.pi / L
    k1 = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=dev)
    kz1 = torch.fft.rfftfreq(n, d=1.0 / n, dtype=torch.float64, device=dev)
    kx, ky, kz = k1[:, None, None], k1[None, :, None], kz1[None, None, :]
    k2 = (kx * kx + ky * ky + kz * kz) * kf * kf
    k2[0, 0, 0] = 1.0
    nyq = n // 2
    mask = (kx.abs() == nyq) | (ky.abs() == nyq) | (kz == nyq)
    amp = torch.where(mask, torch.zeros((), dtype=torch.float64, device=dev), k2.rsqrt())
    amp[0, 0, 0] = 0.0
    dk = dk * amp / k2
    del amp, mask
    delta = L / n
    idx = (torch.arange(n, dtype=torch.float64, device=dev) + 0.5) * delta
    pos = torch.empty((n ** 3, 3), dtype=torch.float64, device=dev)
    ss = 0.0
    for ax, kk in enumerate((kx, ky, kz)):
        psi = torch.fft.irfftn(dk * (1j * kk * kf), s=(n, n, n))
        ss += float((psi * psi).sum().item())
        pos[:, ax] = psi.reshape(-1)
        del psi
    rms = math.sqrt(ss / n ** 3)
    scale = (rms_in_spacing * delta / rms) if rms > 0 else 0.0
    lat = (idx[:, None, None].expand(n, n, n), idx[None, :, None].expand(n, n, n),
           idx[None, None, :].expand(n, n, n))
    for ax in range(3):
        pos[:, ax] = torch.remainder(lat[ax].reshape(-1) + scale * pos[:, ax], L)
    pos[pos >= L] -= L
    return pos


def zeldovich_box(n_side: int, L: float, rms_in_spacing: float, seed: int) -> ParticleSet:
    return zeldovich(n_side, L, rms_in_spacing, seed)


def treepm_params_for(n_side: int, L: float) -> dict:
    """Split scale r_s = 1.25 L / (2 n_side) (mesh of twice the particle grid) and
    R_cut = 4.5, as used by the periodic workloads."""
    return {"r_s": 1.25 * L / (2 * n_side), "r_cut_factor": 4.5}
