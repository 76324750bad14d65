"""Stored-energy densities for the FP64 oracle: W, its first derivative P = W_F and
its second derivative C = W_FF, batched over voxels.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle that checks the
CUDA path; only the test suite, the package's smoke check and the bench's CPU
baseline may import it.  It shares no code with the CUDA library.

Array conventions: F has shape (V, d, d) (row-major F_ij), per-voxel material
parameters have shape (V,).  P has shape (V, d, d); C has shape (V, d, d, d, d)
with C[v, i, j, k, l] = d P_ij / d F_kl.
"""
from __future__ import annotations

import numpy as np


def _inv_t(F):
    """F^{-T} and J = det F, batched."""
    J = np.linalg.det(F)
    A = np.linalg.inv(F).transpose(0, 2, 1)
    return A, J


class NeoHookean:
    """Compressible neo-Hookean density, Section 4.1 (Mooney-Rivlin form with
    I_2 = det C = J^2), written for d = 2 (plane strain) and d = 3:

        W = mu/2 (|F|^2 - d - 2 ln J) + lam/2 (J - 1)^2.

    For d = 2 this is mu/2 (I_1 - ln I_2 - 2) + kappa/2 (sqrt(I_2) - 1)^2 with
    kappa = lam.  For d = 3 the same expression restricted to F = diag(F_2D, 1)
    gives back the 2D one (plane strain).
    """

    nparam = 2

    def __init__(self, mu, lam):
        self.mu = np.asarray(mu, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)

    def subset(self, idx):
        return type(self)(self.mu[idx], self.lam[idx])

    def W(self, F):
        d = F.shape[-1]
        J = np.linalg.det(F)
        with np.errstate(invalid="ignore", divide="ignore"):
            lnJ = np.log(J)
        return (0.5 * self.mu * (np.einsum("vij,vij->v", F, F) - d - 2.0 * lnJ)
                + 0.5 * self.lam * (J - 1.0) ** 2)

    def P(self, F):
        A, J = _inv_t(F)
        c = self.lam * J * (J - 1.0) - self.mu
        return self.mu[:, None, None] * F + c[:, None, None] * A

    def C(self, F):
        d = F.shape[-1]
        A, J = _inv_t(F)
        c = self.lam * J * (J - 1.0) - self.mu
        b = self.lam * (2.0 * J - 1.0) * J
        I = np.eye(d)
        out = self.mu[:, None, None, None, None] * np.einsum("ik,jl->ijkl", I, I)[None]
        out = out + b[:, None, None, None, None] * np.einsum("vij,vkl->vijkl", A, A)
        out = out - c[:, None, None, None, None] * np.einsum("vil,vkj->vijkl", A, A)
        return out


class LinearElastic:
    """Isotropic linear elasticity in the displacement gradient H = F - I:

        W = mu |sym H|^2 + lam/2 (tr H)^2.

    Quadratic, so the local problem is linear and W is convex; used for the closed
    form laminate and the monotone-residual checks (Section 2.2 quadratic case).
    """

    nparam = 2

    def __init__(self, mu, lam):
        self.mu = np.asarray(mu, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)

    def subset(self, idx):
        return type(self)(self.mu[idx], self.lam[idx])

    def W(self, F):
        d = F.shape[-1]
        H = F - np.eye(d)[None]
        E = 0.5 * (H + H.transpose(0, 2, 1))
        tr = np.trace(H, axis1=1, axis2=2)
        return self.mu * np.einsum("vij,vij->v", E, E) + 0.5 * self.lam * tr * tr

    def P(self, F):
        d = F.shape[-1]
        H = F - np.eye(d)[None]
        E = 0.5 * (H + H.transpose(0, 2, 1))
        tr = np.trace(H, axis1=1, axis2=2)
        return 2.0 * self.mu[:, None, None] * E + (self.lam * tr)[:, None, None] * np.eye(d)[None]

    def C(self, F):
        d = F.shape[-1]
        I = np.eye(d)
        sym = np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I)
        vol = np.einsum("ij,kl->ijkl", I, I)
        return (self.mu[:, None, None, None, None] * sym[None]
                + self.lam[:, None, None, None, None] * vol[None])


MODELS = {"neohookean": NeoHookean, "linear": LinearElastic}


def make_material(model: str, phase: np.ndarray, params: np.ndarray):
    """Per-voxel material for a phase map (any grid shape) and a per-phase table
    params[p] = (mu, lam).  Voxels are taken in C order of ``phase``."""
    ph = np.asarray(phase).reshape(-1).astype(np.int64)
    tab = np.asarray(params, dtype=np.float64)
    return MODELS[model](tab[ph, 0], tab[ph, 1])
