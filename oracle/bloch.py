"""FP64 CPU oracle for the Bloch-wave ADMM (Section 2.4, Steps 1'-4'): the modulus of
stability beta_k of a periodic tangent field L(x) over Bloch waves.

TEST INFRASTRUCTURE ONLY.  Plain numpy; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library and never imports the solver package.

Discrete setting (the grid and central differences of the periodic problem,
Section 2.3; h = 1/N, direction j is array axis d-1-j, x last).  A Bloch wave is
v = p(x) exp(i omega.x) with p periodic, omega_j = 2 pi / k_j.  The central
difference of v is exp(i omega.x) (D p) with

    (D p)_ij(x) = (p_i(x + h e_j) e^{i theta_j} - p_i(x - h e_j) e^{-i theta_j}) / (2h),

theta_j = omega_j h, whose Fourier symbol (unnormalised DFT, frequency index m) is
i s_j(m), s_j(m) = N sin(2 pi (m_j + 1/k_j) / N).  The modulus is the eigenvalue
form of the definition,

    beta_k = min over ||p|| = 1 of <D p, L D p>,   ||p||^2 = mean over voxels of |p|^2,

i.e. the smallest eigenvalue of D^* L D.  Steps of one iteration i -> i + 1:

 1'. G_{i+1} = (L + rho I)^{-1} (g_i + rho D p_i)                      (per voxel)
 2'. p_{i+1} = argmin over ||p|| = 1 of rho/2 ||D p - Q||^2, Q = G_{i+1} - g_i/rho.
     In Fourier p^(m) = rho b^(m) / (rho kappa(m) - sigma), b = D^* Q,
     kappa = sum_j s_j^2, with sigma < rho min kappa the root of ||p(sigma)|| = 1
     (the secular equation of a trust-region subproblem; unique on that interval).
 3'. g_{i+1} = g_i + rho (D p_{i+1} - G_{i+1})
 4'. r_p = ||D p_{i+1} - G_{i+1}||,  r_d = rho / mu_ref ||D (p_{i+1} - p_i)||.

At a fixed point D p = G, L G = g and D^* L D p = sigma p: sigma is the eigenvalue
(and the minimum of the augmented Lagrangian is reached at the smallest one).
Start: p_0 = the given field normalised, g_0 = L D p_0.

Penalty: fixed, or Section 2.1's residual balancing after every Step 4' (rho <- kappa rho
if r_p > tau r_d, rho <- max(rho / kappa, rho_floor) if r_d > tau r_p), with
rho_floor = max(rho_min (default mu_ref), 2 max(0, -lambda_min(L))): L + rho I must stay
positive definite for Step 1', and below about twice the most negative eigenvalue of L
the iteration was seen to diverge.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

from .materials import make_material


def bloch_symbols(n: int, dim: int, k):
    """s_j(m) = N sin(2 pi (m + 1/k_j) / N), m = 0..N-1 (FFT order), shaped to broadcast
    along direction j (array axis dim-1-j)."""
    m = np.arange(n, dtype=np.float64)
    out = []
    for j in range(dim):
        s = n * np.sin(2.0 * np.pi * (m + 1.0 / k[j]) / n)
        shape = [1] * dim
        shape[dim - 1 - j] = n
        out.append(s.reshape(shape))
    return out


def _axes(dim, lead):
    return tuple(range(lead, lead + dim))


def bloch_grad(p: np.ndarray, k) -> np.ndarray:
    """D p through the spectrum: (D p)_ij = IFFT(i s_j p^_i); p (d, *grid) complex."""
    d = p.shape[0]
    s = bloch_symbols(p.shape[-1], d, k)
    ph = np.fft.fftn(p, axes=_axes(d, 1))
    return np.stack([np.stack([np.fft.ifftn(1j * s[j] * ph[i], axes=_axes(d, 0)) for j in range(d)])
                     for i in range(d)])


def norm(f: np.ndarray) -> float:
    """sqrt(mean over voxels of the squared Frobenius norm), for p (d, *grid) or G (d, d, *grid)."""
    return float(np.sqrt(np.sum(np.abs(f) ** 2) / _nvox(f)))


def _nvox(f):
    # the grid is the trailing dims: p has d + 1 dims, tensor fields d + 2
    d = f.shape[0]
    return int(np.prod(f.shape[-d:]))


def tangent_field(model, phase, params, F):
    """L(x) = W_FF(F(x)) of the per-voxel material, shape (V, d, d, d, d)."""
    d = F.shape[0]
    mat = make_material(model, phase, params)
    Fv = F.reshape(d, d, -1).transpose(2, 0, 1)
    return mat.C(Fv)


def constrained_step(b_hat: np.ndarray, kappa: np.ndarray, rho: float, nvox: int):
    """Step 2' in Fourier: sigma and p^ = rho b^ / (rho kappa - sigma) with ||p|| = 1.
    ||p||^2 = sum |p^|^2 / V^2 (Parseval for the unnormalised DFT)."""
    W = np.sum(np.abs(b_hat) ** 2, axis=0)
    pole = rho * float(np.min(kappa))
    total = float(np.sum(W))

    def psi(sig):  # 1/||p(sigma)|| - 1, decreasing on (-inf, pole)
        S = np.sum(rho * rho * W / (rho * kappa - sig) ** 2) / (nvox * nvox)
        return 1.0 / np.sqrt(S) - 1.0

    lo = pole - 2.0 * rho * np.sqrt(total) / nvox  # ||p(lo)|| <= 1/2
    hi = pole
    if not (np.isfinite(total) and total > 0.0):
        raise FloatingPointError("Step 2': b is zero or not finite (the iteration diverged?)")
    if not psi(np.nextafter(hi, -np.inf)) < 0.0:
        raise FloatingPointError("Step 2': no root below the pole (hard case)")
    sigma = brentq(psi, lo, np.nextafter(hi, -np.inf), xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    return sigma, rho * b_hat / (rho * kappa - sigma)


def rho_floor(L: np.ndarray, mu_ref: float, rho_min=None) -> float:
    """max(rho_min (default mu_ref), 2 max(0, -lambda_min)) over the voxels' L."""
    d2 = L.shape[1] * L.shape[2]
    lmin = float(np.min(np.linalg.eigvalsh(L.reshape(-1, d2, d2))))
    return max(rho_min if rho_min else mu_ref, 2.0 * max(0.0, -lmin))


def bloch_solve(L: np.ndarray, p0: np.ndarray, k, rho: float, tol: float, max_iter: int, mu_ref: float,
                rho_policy: str = "fixed", kappa: float = 1.3, tau: float = 10.0, rho_min=None):
    """Steps 1'-4' from p_0 (normalised here) until r_p <= tol and r_d <= tol or max_iter.

    L: (V, d, d, d, d) tangent field (voxels in C order of the grid); p0: (d, *grid)
    complex.  Returns dict with p, G, g, sigma (Step 2's multiplier of the last
    iteration), history [(r_p, r_d)], rhos (the penalty of every iteration),
    iterations, converged, rayleigh = <Dp, L Dp>."""
    d = p0.shape[0]
    grid = p0.shape[1:]
    V = int(np.prod(grid))
    n = grid[-1]
    s = bloch_symbols(n, d, k)
    kap = sum(sj * sj for sj in s) * np.ones(grid)  # |s|^2 per frequency
    Lm = L.reshape(V, d * d, d * d)
    floor = rho_floor(L, mu_ref, rho_min) if rho_policy == "adaptive" else None

    def apply(M, T):  # per-voxel (d*d, d*d) matrix on a (d, d, *grid) field
        Tv = T.reshape(d * d, V).T
        return np.einsum("vab,vb->va", M, Tv).T.reshape((d, d) + grid)

    def solve(T):
        Tv = T.reshape(d * d, V).T
        A = Lm + rho * np.eye(d * d)[None]
        return np.linalg.solve(A, Tv[..., None])[..., 0].T.reshape((d, d) + grid)

    p = np.array(p0, dtype=np.complex128)
    p = p / norm(p)
    Dp = bloch_grad(p, k)
    g = apply(Lm, Dp)
    hist = []
    rhos = []
    sigma = np.nan
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        G = solve(g + rho * Dp)                                        # Step 1'
        Q = G - g / rho                                                # Step 2'
        Qh = np.fft.fftn(Q, axes=_axes(d, 2))
        b_hat = np.stack([sum(-1j * s[j] * Qh[i, j] for j in range(d)) for i in range(d)])
        sigma, p_hat = constrained_step(b_hat, kap, rho, V)
        p_new = np.fft.ifftn(p_hat, axes=_axes(d, 1))
        Dp_new = bloch_grad(p_new, k)
        g = g + rho * (Dp_new - G)                                     # Step 3'
        r_p = norm(Dp_new - G)                                         # Step 4'
        r_d = rho / mu_ref * norm(Dp_new - Dp)
        hist.append((r_p, r_d))
        rhos.append(rho)
        p, Dp = p_new, Dp_new
        if r_p <= tol and r_d <= tol:
            converged = True
            break
        if rho_policy == "adaptive":
            if r_d > 0.0 and r_p / r_d > tau:
                rho = kappa * rho
            elif r_p > 0.0 and r_d / r_p > tau:
                rho = max(rho / kappa, floor)
    rq = float(np.real(np.sum(np.conj(Dp) * apply(Lm, Dp))) / V)
    return {"p": p, "G": G if max_iter > 0 else None, "g": g, "sigma": sigma, "history": hist, "rhos": rhos,
            "iterations": it if max_iter > 0 else 0, "converged": converged, "rayleigh": rq}
