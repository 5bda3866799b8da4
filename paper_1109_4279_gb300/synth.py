"""Seeded synthetic inputs: gauge fields, sources, gauge transforms, directions.

This module holds input generation only -- none of the solver's arithmetic --
so that the CUDA path's tests and the CPU oracle can draw identical inputs.
The paper's beta = 5.29 ensembles (Sec. 4 Fig. 1, Sec. 6) are not available;
links are drawn as U = exp(i eps sum_a g_a lambda_a / 2) with g_a ~ N(0, 1),
which spreads plaquettes around the identity like a smooth gauge field.

Generation order (fixed, so that every consumer sees the same numbers):
``rng = numpy.random.default_rng(seed)``; ``g = rng.standard_normal((V, 4, 8))``
in lexicographic site order, mu = 0..3, a = 1..8; then the right-hand side
``rng.standard_normal((V, 4, 3, 2))`` -> re + i im.
"""
from __future__ import annotations

import numpy as np

# Gell-Mann matrices lambda_1 .. lambda_8
GELL_MANN = np.zeros((8, 3, 3), np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1], GELL_MANN[1][1, 0] = -1j, 1j
GELL_MANN[2][0, 0], GELL_MANN[2][1, 1] = 1, -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2], GELL_MANN[4][2, 0] = -1j, 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2], GELL_MANN[6][2, 1] = -1j, 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def volume(dims) -> int:
    return int(np.prod(dims))


def su3_exp(H: np.ndarray) -> np.ndarray:
    """exp(i H) for Hermitian (..., 3, 3) H via eigh, then re-unitarised."""
    w, v = np.linalg.eigh(H)
    U = np.einsum("...ab,...b,...cb->...ac", v, np.exp(1j * w), np.conj(v))
    return reunitarise(U)


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt rows 0 and 1; row 2 = conj(row0 x row1), so det U = 1."""
    U = np.array(U, np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    U[..., 0, :] = r0
    U[..., 1, :] = r1
    U[..., 2, :] = np.conj(np.cross(r0, r1))
    return U


def algebra(theta: np.ndarray) -> np.ndarray:
    """sum_a theta_a lambda_a / 2 for theta of shape (..., 8)."""
    return np.einsum("...a,aij->...ij", theta, GELL_MANN) / 2.0


def gauge_field(dims, eps: float, seed: int, rng=None):
    """(V, 4, 3, 3) complex128 links exp(i eps sum_a g_a lambda_a / 2).

    Returns (U, rng) so that callers can continue drawing from the same
    generator (the right-hand side is drawn next).
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    V = volume(dims)
    g = rng.standard_normal((V, 4, 8))
    U = su3_exp(eps * algebra(g))
    return U, rng


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gaussian_spinor(dims, rng, nrhs: int | None = None) -> np.ndarray:
    """(V, 4, 3) (or (nrhs, V, 4, 3)) complex Gaussian, re and im ~ N(0, 1)."""
    V = volume(dims)
    shape = (V, 4, 3, 2) if nrhs is None else (nrhs, V, 4, 3, 2)
    r = rng.standard_normal(shape)
    return r[..., 0] + 1j * r[..., 1]


def point_sources(dims, site: int = 0) -> np.ndarray:
    """12 spin-colour point sources at one site: (12, V, 4, 3), source s*3+c."""
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), np.complex128)
    for s in range(4):
        for c in range(3):
            b[s * 3 + c, site, s, c] = 1.0
    return b


def random_su3(n: int, rng) -> np.ndarray:
    """n Haar-ish random SU(3) matrices (QR of a complex Gaussian, det fixed to 1)."""
    z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return reunitarise(q)


def link_directions(dims, n: int, seed: int):
    """n random link directions: (site, mu, theta in R^8 with |theta| = 1)."""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    sites = rng.integers(0, V, size=n)
    mus = rng.integers(0, 4, size=n)
    th = rng.standard_normal((n, 8))
    th /= np.linalg.norm(th, axis=1, keepdims=True)
    return sites, mus, th


# The five workloads (sizes, link spread, masses, solver shapes).  dims are
# (L0 = T, L1, L2, L3).
WORKLOADS = {
    "4^4 fp64": dict(dims=(4, 4, 4, 4), eps=0.3, seed=1, m0=0.1, csw=1.0, block=(2, 2, 2, 2),
                     nmr=4, ncy=4, nkv=16),
    "16^3x32 fp32": dict(dims=(32, 16, 16, 16), eps=0.5, seed=2, m0=0.0, csw=1.5,
                         block=(4, 4, 4, 4), nmr=4, ncy=4, nkv=16),
    "32^3x64 fp16": dict(dims=(64, 32, 32, 32), eps=0.5, seed=3, m0=-0.05, csw=1.5,
                         block=(4, 4, 4, 4), nmr=4, ncy=4, nkv=16),
    "24^3x48 12 point sources": dict(dims=(48, 24, 24, 24), eps=0.5, seed=4, m0=0.0, csw=1.5,
                                     block=(4, 4, 4, 4), nmr=4, ncy=4, nkv=16),
    "16^3x32 gradient": dict(dims=(32, 16, 16, 16), eps=0.5, seed=5, m0=0.0, csw=1.5,
                             block=(4, 4, 4, 4), nmr=4, ncy=4, nkv=16),
}

# Ten lattices of uneven sizes for the batched solve (seeds 10..19 in order).
UNEVEN_LATTICES = ([(8, 8, 8, 8)] * 2 + [(16, 8, 8, 8)] * 2 + [(24, 12, 12, 12)] * 3
                   + [(32, 16, 16, 16)] * 3)

ANTIPERIODIC_T = (-1.0, 1.0, 1.0, 1.0)
