"""Small shared helpers for the tests (norms, gamma_5, chiral basis)."""
import numpy as np

# Chiral basis written out entry by entry (the basis the library and oracle use).
G = np.zeros((4, 4, 4), complex)
G[0] = [[0, 0, -1, 0], [0, 0, 0, -1], [-1, 0, 0, 0], [0, -1, 0, 0]]
G[1] = [[0, 0, 0, -1j], [0, 0, -1j, 0], [0, 1j, 0, 0], [1j, 0, 0, 0]]
G[2] = [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]
G[3] = [[0, 0, -1j, 0], [0, 0, 0, 1j], [1j, 0, 0, 0], [0, -1j, 0, 0]]
G5 = np.diag([1, 1, -1, -1]).astype(complex)


def rel(a, b):
    """Norm-wise relative difference |a - b| / |b| over the whole field."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def g5(psi):
    """gamma_5 psi for spinor fields (..., 4, 3)."""
    out = np.array(psi, copy=True)
    out[..., 2:, :] *= -1
    return out


def vdot(a, b):
    return np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())
