"""Stored-energy densities written directly from the paper's formulas, for pinning
the oracle.  Derivatives are taken numerically here (complex step for W_F,
central differences of that for W_FF), so the oracle's hand-derived P and C are
checked against an independent route rather than retyped.

All functions act on ONE voxel: F is a (d, d) array (real or complex).
"""
import numpy as np


def _det(F):
    if F.shape == (2, 2):
        return F[0, 0] * F[1, 1] - F[0, 1] * F[1, 0]
    return (F[0, 0] * (F[1, 1] * F[2, 2] - F[1, 2] * F[2, 1])
            - F[0, 1] * (F[1, 0] * F[2, 2] - F[1, 2] * F[2, 0])
            + F[0, 2] * (F[1, 0] * F[2, 1] - F[1, 1] * F[2, 0]))


def w_mooney_rivlin_2d(F, mu, kappa):
    """Section 4.1: W = mu/2 (I1 - ln I2 - 2) + kappa/2 (sqrt(I2) - 1)^2, C = F^T F,
    I1 = tr C, I2 = det C (2x2)."""
    C = F.T @ F
    I1 = C[0, 0] + C[1, 1]
    I2 = _det(C)
    return 0.5 * mu * (I1 - np.log(I2) - 2.0) + 0.5 * kappa * (np.sqrt(I2) - 1.0) ** 2


def w_neohooke_3d(F, mu, lam):
    """Compressible neo-Hookean in 3D, mu/2 (tr C - 3 - ln det C) + lam/2 (sqrt(det C) - 1)^2;
    plane strain F = diag(F2, 1) gives back the 2D Mooney-Rivlin form."""
    C = F.T @ F
    I1 = C[0, 0] + C[1, 1] + C[2, 2]
    I3 = _det(C)
    return 0.5 * mu * (I1 - np.log(I3) - 3.0) + 0.5 * lam * (np.sqrt(I3) - 1.0) ** 2


def w_neohooke(F, mu, lam):
    return w_mooney_rivlin_2d(F, mu, lam) if F.shape[0] == 2 else w_neohooke_3d(F, mu, lam)


def w_linear(F, mu, lam):
    """Isotropic linear elasticity in H = F - I: mu |sym H|^2 + lam/2 (tr H)^2."""
    d = F.shape[0]
    H = F - np.eye(d)
    E = 0.5 * (H + H.T)
    return mu * np.sum(E * E) + 0.5 * lam * np.trace(H) ** 2


ENERGIES = {"neohookean": w_neohooke, "linear": w_linear}


def stress_cs(w, F, *args, h=1e-30):
    """W_F by the complex-step derivative: P_kl = Im W(F + i h e_k e_l^T) / h."""
    d = F.shape[0]
    P = np.zeros((d, d))
    for k in range(d):
        for l in range(d):
            E = np.zeros((d, d), dtype=np.complex128)
            E[k, l] = 1j * h
            P[k, l] = np.imag(w(F.astype(np.complex128) + E, *args)) / h
    return P


def tangent_fd(w, F, *args, eps=1e-6):
    """W_FF by central differences of the complex-step W_F: C[i,j,k,l] = dP_ij/dF_kl."""
    d = F.shape[0]
    C = np.zeros((d, d, d, d))
    for k in range(d):
        for l in range(d):
            E = np.zeros((d, d))
            E[k, l] = eps
            C[:, :, k, l] = (stress_cs(w, F + E, *args) - stress_cs(w, F - E, *args)) / (2 * eps)
    return C


# ----------------------------------------------------------------- real-space central differences

def grad_stencil(u):
    """(D u)_ij = (u_i(x + h e_j) - u_i(x - h e_j)) / (2h), h = 1/N, for u of shape (d, *grid)
    with the last grid axis along e_1."""
    d = u.shape[0]
    n = u.shape[-1]
    out = np.empty((d, d) + u.shape[1:])
    for i in range(d):
        for j in range(d):
            ax = d - 1 - j
            out[i, j] = (np.roll(u[i], -1, axis=ax) - np.roll(u[i], 1, axis=ax)) * (n / 2.0)
    return out


def div_stencil(T):
    """Central-difference divergence (D^T is minus this): (div T)_i = sum_j (T_ij(x+he_j) - T_ij(x-he_j))/(2h)."""
    d = T.shape[0]
    n = T.shape[-1]
    out = np.zeros((d,) + T.shape[2:])
    for i in range(d):
        for j in range(d):
            ax = d - 1 - j
            out[i] += (np.roll(T[i, j], -1, axis=ax) - np.roll(T[i, j], 1, axis=ax)) * (n / 2.0)
    return out


# ----------------------------------------------------------------- liquid crystal elastomer (Section 5.1)

def w_lce(F, n, mu, lam, r, alpha, n0):
    """Compressible network + non-ideality, literally from Section 5.1's formulas with
    l = r^{-1/3}(I + (r-1) n n^T) (positive-definite sign):
    mu/2 (tr(F^T l^{-1} F) - 3 - ln det C) + lam/2 (sqrt(det C) - 1)^2
    + mu alpha/2 tr((I - n0 n0^T) F^T (n n^T) F).  n is used as given (not normalised)."""
    ell = r ** (-1.0 / 3.0) * (np.eye(3) + (r - 1.0) * np.outer(n, n))
    ell_inv = np.linalg.inv(ell) if not np.iscomplexobj(n) else _inv3(ell)
    C = F.T @ F
    I3 = _det(C)
    W_el = 0.5 * mu * (np.trace(F.T @ ell_inv @ F) - 3.0 - np.log(I3)) + 0.5 * lam * (np.sqrt(I3) - 1.0) ** 2
    W_ni = 0.5 * mu * alpha * np.trace((np.eye(3) - np.outer(n0, n0)) @ F.T @ np.outer(n, n) @ F)
    return W_el + W_ni


def _inv3(M):
    c = np.array([[M[1, 1] * M[2, 2] - M[1, 2] * M[2, 1], M[0, 2] * M[2, 1] - M[0, 1] * M[2, 2],
                   M[0, 1] * M[1, 2] - M[0, 2] * M[1, 1]],
                  [M[1, 2] * M[2, 0] - M[1, 0] * M[2, 2], M[0, 0] * M[2, 2] - M[0, 2] * M[2, 0],
                   M[0, 2] * M[1, 0] - M[0, 0] * M[1, 2]],
                  [M[1, 0] * M[2, 1] - M[1, 1] * M[2, 0], M[0, 1] * M[2, 0] - M[0, 0] * M[2, 1],
                   M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]]], dtype=M.dtype)
    return c / _det(M)


def lce_grad_cs(F, n, args, h=1e-30):
    """(W_F, W_n) of w_lce by complex steps in each component of F and of n."""
    gF = np.zeros((3, 3))
    gn = np.zeros(3)
    Fc = F.astype(np.complex128)
    nc = n.astype(np.complex128)
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3), dtype=np.complex128)
            E[k, l] = 1j * h
            gF[k, l] = np.imag(w_lce(Fc + E, nc, *args)) / h
        e = np.zeros(3, dtype=np.complex128)
        e[k] = 1j * h
        gn[k] = np.imag(w_lce(Fc, nc + e, *args)) / h
    return gF, gn
