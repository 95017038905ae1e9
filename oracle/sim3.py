"""Sim(3) algebra for the oracle (Sec. III-E of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

A similarity T = (s, R, t) acts as x -> s R x + t and is stored as a tuple of
float64 numpy values.  Its 4x4 matrix is [[sR, t], [0, 1]].  The paper maps a
transform to "a minimal representation in R^7 of the associated Lie algebra"
through log_Sim(3) and says nothing more; the coordinate order used here is a
reading: xi = (rho[3], phi[3], sigma) with generator

    xi^ = [[phi^ + sigma I, rho], [0, 0]]

so that Exp(xi) is the matrix exponential of xi^ (the plain definition, via
``scipy.linalg.expm``).  Log inverts it: sigma = ln s, phi = the rotation
vector of R, rho = V^-1 t where V is the upper-right block of
expm([[phi^ + sigma I, I], [0, 0]]) (Van Loan's block-exponential identity),
which is exactly the matrix that Exp applies to rho.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm
from scipy.spatial.transform import Rotation


def hat(v):
    v = np.asarray(v, dtype=np.float64)
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def identity():
    return (1.0, np.eye(3), np.zeros(3))


def matrix(T):
    s, R, t = T
    M = np.eye(4)
    M[:3, :3] = s * np.asarray(R)
    M[:3, 3] = t
    return M


def from_matrix(M):
    A = M[:3, :3]
    s = float(np.cbrt(np.linalg.det(A)))
    return (s, A / s, M[:3, 3].copy())


def compose(A, B):
    """(A B)(x) = A(B(x))."""
    sa, Ra, ta = A
    sb, Rb, tb = B
    return (sa * sb, Ra @ Rb, sa * (Ra @ tb) + ta)


def inverse(T):
    s, R, t = T
    return (1.0 / s, R.T.copy(), -(R.T @ t) / s)


def act(T, X):
    """Apply T to points X [N,3]."""
    s, R, t = T
    return s * (np.asarray(X, dtype=np.float64) @ R.T) + t


def generator(xi):
    xi = np.asarray(xi, dtype=np.float64)
    G = np.zeros((4, 4))
    G[:3, :3] = hat(xi[3:6]) + xi[6] * np.eye(3)
    G[:3, 3] = xi[0:3]
    return G


def exp(xi):
    return from_matrix(expm(generator(xi)))


def log(T):
    s, R, t = T
    sigma = float(np.log(s))
    phi = Rotation.from_matrix(R).as_rotvec()
    B = np.zeros((6, 6))
    B[:3, :3] = hat(phi) + sigma * np.eye(3)
    B[:3, 3:] = np.eye(3)
    V = expm(B)[:3, 3:]
    rho = np.linalg.solve(V, t)
    return np.concatenate([rho, phi, [sigma]])


def geodesic_sq(A, B):
    """||log(A^-1 B)||^2."""
    e = log(compose(inverse(A), B))
    return float(e @ e)


def rotation_angle(Ra, Rb):
    """Angle of Ra Rb^T in radians."""
    return float(np.linalg.norm(Rotation.from_matrix(Ra @ Rb.T).as_rotvec()))
