"""FP64 CPU oracle for the ADMM iteration of Zhou & Bhattacharya (Section 2.1,
Steps 1-4; Section 2.3 for the periodic cell and the discrete derivative symbols).

TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference the CUDA path is
checked against.  Only the test suite, the package's smoke check and the bench's
CPU-baseline leg may import it; the product path never does, and this module
shares no code with the CUDA library.

What it computes, in the paper's order.  State (F, Lambda, u~) on a periodic N^d
grid of the unit cell, h = 1/N, with <F> = Fbar prescribed (strain control).
One iteration i -> i+1:

  Step 1 (local problem, eq. eq):   at every voxel
        F_{i+1} = argmin_F  W(F;x) - Lambda_i : F + rho/2 |F - G_i|^2,
        G_i = Fbar + D u~_i,
    i.e. W_F(F_{i+1}) - Lambda_i - rho (G_i - F_{i+1}) = 0, solved by damped
    Newton with backtracking (the converged minimiser is what matters; the paper's
    own local solver is steepest descent, any convergent one reaches the same point).
  Step 2 (Helmholtz projection, eq. helm / helmf):
        u^_i(xi) = - sum_j (F^ - Lambda^/rho)_ij  i k_j / |k|^2,
    with the central-difference symbol k_j = sin(h xi_j)/h in the numerator and
    |k|^2 = sum_j k_j^2 in the denominator (one discrete gradient D, Laplacian
    D^T D; u^ = 0 where |k|^2 = 0).  Computed with a library FFT of all d^2
    components of F - Lambda/rho.
  Step 3 (multiplier, eq. update):  Lambda_{i+1} = Lambda_i + rho (G_{i+1} - F_{i+1}).
  Step 4 (check, eq. check):  r_p = ||G_{i+1} - F_{i+1}||,
        r_d = (rho/mu_ref) ||G_{i+1} - G_i||,   ||f||^2 = mean_x |f(x)|^2_Frobenius.
  Optional penalty update (eq. rho-update, He-Yang-Wang):
        rho <- kappa rho if r_p/r_d > tau;  max(rho/kappa, rho_min) if r_d/r_p > tau.

The derivative D u~ in G is evaluated spectrally (multiply u^ by i k_j), not with
real-space stencils; that is the same operator written another way.

Initial state (the paper gives none for the first load step): F_0 = Fbar,
u~_0 = 0 and Lambda_0 = W_F(Fbar; x) (the multiplier converges to the stress), or
Lambda_0 = 0 on request.

Field layout: F and Lambda have shape (d, d, *grid), u~ has shape (d, *grid),
with grid = (N,)*d in C order and the LAST grid axis along e_1 (x); direction j
(0-based) is grid axis d-1-j.
"""
from __future__ import annotations

import numpy as np

from .materials import make_material

# --------------------------------------------------------------------------- discrete symbols


def wavenumbers(n: int, dim: int):
    """Central-difference symbols k_j = sin(h xi_j)/h, xi_j = 2 pi m_j, m_j in [-n/2, n/2),
    h = 1/n, one array per direction j, each broadcastable to the grid shape.

    k_j is set to exactly 0 at m_j = 0 and m_j = -n/2, where sin(h xi_j) vanishes.
    """
    m = np.fft.fftfreq(n) * n
    k = n * np.sin(2.0 * np.pi * m / n)
    k[(m == 0) | (m == -n // 2)] = 0.0
    out = []
    for j in range(dim):
        shape = [1] * dim
        shape[dim - 1 - j] = n
        out.append(k.reshape(shape))
    return out


def _grid_axes(dim: int, lead: int):
    return tuple(range(lead, lead + dim))


# --------------------------------------------------------------------------- Step 2: Helmholtz projection


def u_step(F: np.ndarray, Lam: np.ndarray, rho: float):
    """Step 2 (eq. helmf with discrete symbols): returns (u^ complex (d,*grid), u~ real (d,*grid))."""
    d = F.shape[0]
    n = F.shape[-1]
    k = wavenumbers(n, d)
    k2 = sum(kj * kj for kj in k)
    Qh = np.fft.fftn(F - Lam / rho, axes=_grid_axes(d, 2))
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0.0, 1.0 / np.where(k2 > 0.0, k2, 1.0), 0.0)
    uh = np.zeros((d,) + F.shape[2:], dtype=np.complex128)
    for i in range(d):
        acc = np.zeros(F.shape[2:], dtype=np.complex128)
        for j in range(d):
            acc = acc + (-1j * k[j]) * Qh[i, j]
        uh[i] = acc * inv
    u = np.fft.ifftn(uh, axes=_grid_axes(d, 1)).real
    return uh, u


def grad_from_spectrum(uh: np.ndarray) -> np.ndarray:
    """D u~ from u^: (D u~)_ij = IFFT(i k_j u^_i), shape (d, d, *grid)."""
    d = uh.shape[0]
    n = uh.shape[-1]
    k = wavenumbers(n, d)
    out = np.empty((d, d) + uh.shape[1:], dtype=np.float64)
    for i in range(d):
        for j in range(d):
            out[i, j] = np.fft.ifftn(1j * k[j] * uh[i], axes=_grid_axes(d, 0)).real
    return out


def grad_u(u: np.ndarray) -> np.ndarray:
    """D u~ for a real-space periodic field u~ (d, *grid), through its spectrum."""
    d = u.shape[0]
    uh = np.fft.fftn(u, axes=_grid_axes(d, 1))
    return grad_from_spectrum(uh)


# --------------------------------------------------------------------------- Step 1: local problem


def _to_voxels(T: np.ndarray) -> np.ndarray:
    d = T.shape[0]
    return T.reshape(d, d, -1).transpose(2, 0, 1)


def _to_field(Tv: np.ndarray, grid_shape) -> np.ndarray:
    d = Tv.shape[1]
    return Tv.transpose(1, 2, 0).reshape((d, d) + tuple(grid_shape))


def local_newton(mat, F0, Lam, G, rho, step_tol=1e-10, cap=50, armijo=1e-4, small_step=1e-7):
    """Step 1 at every voxel: minimise phi(F) = W(F) - Lam:F + rho/2 |F - G|^2.

    Damped Newton from F0 with the analytic Hessian W_FF + rho I.  When the Newton
    direction is not a descent direction the steepest-descent direction -grad phi
    is used (the paper's local method).  Backtracking halves the step until
    J = det F > 0 and the Armijo decrease holds (steps below ``small_step`` are
    accepted on J > 0 alone, since phi's rounding noise exceeds the decrease there).
    A voxel stops after a full step with max |step| <= step_tol.

    All arrays are per voxel: F0, Lam, G of shape (V, d, d).  Returns (F, iters).
    """
    V, d, _ = F0.shape
    n2 = d * d
    F = F0.copy()
    iters = np.zeros(V, dtype=np.int64)
    active = np.ones(V, dtype=bool)

    def phi(sub, Fs, Lam_s, G_s):
        return (sub.W(Fs) - np.einsum("vij,vij->v", Lam_s, Fs)
                + 0.5 * rho * np.einsum("vij,vij->v", Fs - G_s, Fs - G_s))

    for _ in range(cap):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        sub = mat.subset(idx)
        Fa = F[idx]
        Lam_s = Lam[idx]
        G_s = G[idx]
        g = sub.P(Fa) - Lam_s + rho * (Fa - G_s)
        H = sub.C(Fa).reshape(-1, n2, n2) + rho * np.eye(n2)[None]
        delta = -np.linalg.solve(H, g.reshape(-1, n2, 1))[..., 0].reshape(-1, d, d)
        slope = np.einsum("vij,vij->v", g, delta)
        bad = ~(slope < 0.0) | ~np.all(np.isfinite(delta), axis=(1, 2))
        if np.any(bad):
            delta[bad] = -g[bad]
            slope[bad] = -np.einsum("vij,vij->v", g[bad], g[bad])
        phi0 = phi(sub, Fa, Lam_s, G_s)
        t = np.ones(idx.size)
        accepted = np.zeros(idx.size, dtype=bool)
        size = np.max(np.abs(delta), axis=(1, 2))
        for _ls in range(60):
            pend = ~accepted
            if not np.any(pend):
                break
            Ft = Fa + t[:, None, None] * delta
            J = np.linalg.det(Ft)
            ok = J > 0.0
            with np.errstate(invalid="ignore", divide="ignore"):
                ph = phi(sub, Ft, Lam_s, G_s)
            dec = ph <= phi0 + armijo * t * slope
            acc = pend & ok & (dec | (t * size <= small_step))
            accepted |= acc
            t = np.where(pend & ~acc, 0.5 * t, t)
        t = np.where(accepted, t, 0.0)
        F[idx] = Fa + t[:, None, None] * delta
        iters[idx] += 1
        done = accepted & (t == 1.0) & (size <= step_tol)
        active[idx[done]] = False
    return F, iters


# --------------------------------------------------------------------------- Steps 3 and 4


def multiplier_update(Lam, G_new, F, rho):
    """Step 3 (eq. update): Lambda_{i+1} = Lambda_i + rho (grad u_{i+1} - F_{i+1})."""
    return Lam + rho * (G_new - F)


# --------------------------------------------------------------------------- the iteration


def rms(T: np.ndarray) -> float:
    """Unit-cell L2 norm: sqrt(mean over voxels of the squared Frobenius norm)."""
    d = T.shape[0]
    return float(np.sqrt(np.sum(T * T) / T[0, 0].size))


def initial_state(mat, Fbar_d: np.ndarray, grid_shape, lambda0: str = "stress"):
    d = Fbar_d.shape[0]
    V = int(np.prod(grid_shape))
    Fv = np.broadcast_to(Fbar_d, (V, d, d)).copy()
    F = _to_field(Fv, grid_shape)
    if lambda0 == "stress":
        Lam = _to_field(mat.P(Fv), grid_shape)
    elif lambda0 == "zero":
        Lam = np.zeros_like(F)
    else:
        raise ValueError(lambda0)
    u = np.zeros((d,) + tuple(grid_shape))
    return {"F": F, "Lam": Lam, "u": u}


def admm_solve(phase, params, Fbar, rho, tol, max_iter, model="neohookean", mu_ref=None,
               lambda0="stress", state=None, rho_policy="fixed", kappa=1.3, tau=10.0,
               rho_min=None, local_cap=50, step_tol=1e-10):
    """Run the ADMM iteration (Steps 1-4) until r_p <= tol and r_d <= tol, or max_iter.

    phase: uint8 grid (N,)*d; params: per-phase (mu, lam); Fbar: 3x3 (the upper-left
    d x d block is used).  Returns a dict with F, Lam, u (final state), iters,
    converged, history (list of (r_p, r_d, rho_used)), rho (next rho) and the
    homogenised first Piola-Kirchhoff stress <W_F(F)> (d x d).
    """
    phase = np.asarray(phase)
    d = phase.ndim
    grid = phase.shape
    mat = make_material(model, phase, params)
    Fbar_d = np.asarray(Fbar, dtype=np.float64)[:d, :d]
    if mu_ref is None:
        mu_ref = float(np.mean(mat.mu))
    if rho_min is None:
        rho_min = mu_ref
    st = initial_state(mat, Fbar_d, grid, lambda0) if state is None else {
        k: np.array(v, dtype=np.float64, copy=True) for k, v in state.items()}
    F, Lam, u = st["F"], st["Lam"], st["u"]
    G = Fbar_d.reshape((d, d) + (1,) * d) + grad_u(u)
    history = []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        # Step 1
        Fv, _ = local_newton(mat, _to_voxels(F), _to_voxels(Lam), _to_voxels(G), rho,
                             step_tol=step_tol, cap=local_cap)
        F = _to_field(Fv, grid)
        # Step 2
        uh, u = u_step(F, Lam, rho)
        G_new = Fbar_d.reshape((d, d) + (1,) * d) + grad_from_spectrum(uh)
        # Step 3
        Lam = multiplier_update(Lam, G_new, F, rho)
        # Step 4
        r_p = rms(G_new - F)
        r_d = rho / mu_ref * rms(G_new - G)
        history.append((r_p, r_d, rho))
        G = G_new
        if r_p <= tol and r_d <= tol:
            converged = True
            break
        if not (np.isfinite(r_p) and np.isfinite(r_d)):
            break
        if rho_policy == "adaptive":
            if r_d > 0.0 and r_p / r_d > tau:
                rho = kappa * rho
            elif r_p > 0.0 and r_d / r_p > tau:
                rho = max(rho / kappa, rho_min)
    stress = np.mean(mat.P(_to_voxels(F)), axis=0)
    return {"F": F, "Lam": Lam, "u": u, "iters": it if max_iter > 0 else 0,
            "converged": converged, "history": history, "rho": rho,
            "stress": stress, "mu_ref": mu_ref}


def homogenised_stress(phase, params, F, model="neohookean"):
    """<W_F(F)> over the cell (first Piola-Kirchhoff), shape (d, d)."""
    mat = make_material(model, phase, params)
    return np.mean(mat.P(_to_voxels(F)), axis=0)
