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


class LCE:
    """Liquid crystal elastomer of Section 5.1 (3D), compressible network:

        W(F, n; x) = mu/2 (tr(F^T l^{-1} F) - 3 - 2 ln J) + lam/2 (J - 1)^2        (network)
                     + mu alpha/2 tr((I - n0 (x) n0) F^T (n (x) n) F)                 (non-ideality)

    with the step-length tensor l = r^{-1/3} (I + (r - 1) n (x) n) (the sign that makes
    l positive definite and elongates the material along n by r^{1/3}), so
    l^{-1} = r^{1/3} (I - (1 - 1/r) n (x) n).  The Frank energy is not part of W here;
    the iteration adds its explicit force (see admm.local_newton_lce).

    In terms of m = F^T n:  W = mu r^{1/3}/2 |F|^2 + 1/2 m.M m - mu ln J + lam/2 (J-1)^2
    - 3 mu/2 with M = mu (alpha - r^{1/3}(1 - 1/r)) I - mu alpha n0 (x) n0; the
    derivatives below are taken from that form.  Arrays: F (V,3,3), n (V,3).
    """

    nparam = 5

    def __init__(self, mu, lam, r, alpha, kappa, n0, cF=None, cn=None, incompressible=False):
        self.mu = np.asarray(mu, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)
        self.r = np.asarray(r, dtype=np.float64)
        self.alpha = np.asarray(alpha, dtype=np.float64)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        self.n0 = np.asarray(n0, dtype=np.float64)
        # dissipation weights of one implicit time step (Section 5.1's potential
        # D = nu_F/2 |F'|^2 + nu_n/2 |n'|^2): cF = nu_F/dt, cn = nu_n/dt
        self.cF = np.zeros_like(self.mu) if cF is None else np.asarray(cF, dtype=np.float64)
        self.cn = np.zeros_like(self.mu) if cn is None else np.asarray(cn, dtype=np.float64)
        # incompressible network (Section 5.1 as printed): W = mu/2 (tr(F^T l^-1 F) - 3) +
        # non-ideality, det F = 1 enforced by the local step's multiplier; no volumetric terms
        self.incompressible = bool(incompressible)

    def subset(self, idx):
        return LCE(self.mu[idx], self.lam[idx], self.r[idx], self.alpha[idx], self.kappa[idx], self.n0[idx],
                   self.cF[idx], self.cn[idx], self.incompressible)

    def ell_inv(self, n):
        r13 = np.cbrt(self.r)
        s = 1.0 - 1.0 / self.r
        return r13[:, None, None] * (np.eye(3)[None] - s[:, None, None] * np.einsum("vi,vj->vij", n, n))

    def W(self, F, n):
        J = np.linalg.det(F)
        with np.errstate(invalid="ignore", divide="ignore"):
            lnJ = np.log(J)
        tr_el = np.einsum("vji,vjk,vki->v", F, self.ell_inv(n), F)
        P0 = np.eye(3)[None] - np.einsum("vi,vj->vij", self.n0, self.n0)
        FtnnF = np.einsum("vji,vj,vk,vkl->vil", F, n, n, F)
        tr_ni = np.einsum("vij,vji->v", P0, FtnnF)
        vol = 0.0 if self.incompressible else -self.mu * lnJ + 0.5 * self.lam * (J - 1.0) ** 2
        return 0.5 * self.mu * (tr_el - 3.0) + vol + 0.5 * self.mu * self.alpha * tr_ni

    def _M(self):
        r13 = np.cbrt(self.r)
        c1 = self.mu * (self.alpha - r13 * (1.0 - 1.0 / self.r))
        c2 = self.mu * self.alpha
        return c1[:, None, None] * np.eye(3)[None] - c2[:, None, None] * np.einsum("vi,vj->vij", self.n0, self.n0)

    def derivatives(self, F, n):
        """Gradients and Hessian blocks of W: (P = W_F, W_n, W_FF (V,3,3,3,3), W_Fn (V,3,3,3), W_nn (V,3,3))."""
        A = np.linalg.inv(F).transpose(0, 2, 1)
        J = np.linalg.det(F)
        r13 = np.cbrt(self.r)
        M = self._M()
        m = np.einsum("vij,vi->vj", F, n)
        Mm = np.einsum("vjl,vl->vj", M, m)
        c = self.lam * J * (J - 1.0) - self.mu
        b = self.lam * (2.0 * J - 1.0) * J
        if self.incompressible:
            c = np.zeros_like(c)
            b = np.zeros_like(b)
        P = (self.mu * r13)[:, None, None] * F + np.einsum("vk,vl->vkl", n, Mm) + c[:, None, None] * A
        Wn = np.einsum("vkj,vj->vk", F, Mm)
        I = np.eye(3)
        WFF = ((self.mu * r13)[:, None, None, None, None] * np.einsum("ik,jl->ijkl", I, I)[None]
               + np.einsum("vk,vp,vlq->vklpq", n, n, M)
               + b[:, None, None, None, None] * np.einsum("vij,vkl->vijkl", A, A)
               - c[:, None, None, None, None] * np.einsum("vil,vkj->vijkl", A, A))
        MFt = np.einsum("vlj,vpj->vlp", M, F)
        WFn = np.einsum("kp,vl->vklp", I, Mm) + np.einsum("vk,vlp->vklp", n, MFt)
        Wnn = np.einsum("vkj,vjl,vpl->vkp", F, M, F)
        return P, Wn, WFF, WFn, Wnn

    def P(self, F, n):
        return self.derivatives(F, n)[0]


def make_lce(phase: np.ndarray, params: np.ndarray, n0: np.ndarray, incompressible: bool = False):
    """Per-voxel LCE material: params[p] = (mu, lam, r, alpha, kappa_F[, nu_F/dt, nu_n/dt]);
    n0 of shape (3, *grid) (component-major, like the fields)."""
    ph = np.asarray(phase).reshape(-1).astype(np.int64)
    tab = np.asarray(params, dtype=np.float64)
    n0v = np.asarray(n0, dtype=np.float64).reshape(3, -1).T
    cF = tab[ph, 5] if tab.shape[1] > 5 else None
    cn = tab[ph, 6] if tab.shape[1] > 6 else None
    return LCE(tab[ph, 0], tab[ph, 1], tab[ph, 2], tab[ph, 3], tab[ph, 4], n0v, cF, cn, incompressible)
