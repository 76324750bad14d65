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

from .materials import make_lce, make_material

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


def local_newton(mat, F0, Lam, G, rho, step_tol=1e-10, cap=50, armijo=1e-4, small_step=1e-7,
                 return_conv=False):
    """Step 1 at every voxel: minimise phi(F) = W(F) - Lam:F + rho/2 |F - G|^2.

    Damped Newton from F0 with the analytic Hessian W_FF + rho I.  When the Newton
    direction is not a descent direction the steepest-descent direction -grad phi
    is used (the paper's local method).  Backtracking halves the step until
    J = det F > 0 and the Armijo decrease holds (steps below ``small_step`` are
    accepted on J > 0 alone, since phi's rounding noise exceeds the decrease there).
    A voxel stops after a full step with max |step| <= step_tol (its pointwise
    convergence test); ``cap`` bounds the Newton iterations of this call, so that
    calling it again from the returned F continues the same iteration (the rounds
    of local_step_rounds).

    All arrays are per voxel: F0, Lam, G of shape (V, d, d).  Returns (F, iters), and
    with return_conv=True also the mask of voxels that met the convergence test.
    """
    V, d, _ = F0.shape
    n2 = d * d
    F = F0.copy()
    iters = np.zeros(V, dtype=np.int64)
    active = np.ones(V, dtype=bool)
    conv = np.zeros(V, dtype=bool)

    def phi(sub, Fs, Lam_s, G_s):
        return (sub.W(Fs) - np.einsum("vij,vij->v", Lam_s, Fs)
                + 0.5 * rho * np.einsum("vij,vij->v", Fs - G_s, Fs - G_s))

    for _ in range(cap + 1):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        sub = mat.subset(idx)
        Fa = F[idx]
        Lam_s = Lam[idx]
        G_s = G[idx]
        g = sub.P(Fa) - Lam_s + rho * (Fa - G_s)
        keep = iters[idx] < cap
        if not np.all(keep):
            active[idx[~keep]] = False
            idx, Fa, Lam_s, G_s, g = idx[keep], Fa[keep], Lam_s[keep], G_s[keep], g[keep]
            if idx.size == 0:
                break
            sub = mat.subset(idx)
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
        conv[idx[done]] = True
    return (F, iters, conv) if return_conv else (F, iters)


def local_step_rounds(run, V, cap, round_len, enough, check_first):
    """Step 1 solved approximately in the manner of Algorithm 1's inner loop and of
    Section 4.2: the local iterations run in rounds of ``round_len`` iterations at
    every point that has not yet met its pointwise convergence test, and after each
    round a global check ``enough(conv)`` decides whether to proceed to Step 2.

      run(idx, k)  advances the local iteration at voxels idx by up to k iterations
                   from their current state and returns (iters_done, conv) for idx;
      enough(conv) the global check (r_l <= f r_d, or the converged fraction >= p);
      check_first  evaluate the check once before the first round (the while loop of
                   Algorithm 1 tests r_l before iterating).

    Stops at the check, when every point has converged, or after ``cap`` local
    iterations.  Returns (iters, conv, rounds) per voxel / in total."""
    iters = np.zeros(V, dtype=np.int64)
    conv = np.zeros(V, dtype=bool)
    rounds = 0
    if check_first and enough(conv):
        return iters, conv, rounds
    while not conv.all() and int(iters.max(initial=0)) < cap:
        idx = np.nonzero(~conv)[0]
        k = min(round_len, cap - int(iters.max(initial=0)))
        it, c = run(idx, k)
        iters[idx] += it
        conv[idx] = c
        rounds += 1
        if enough(conv):
            break
    return iters, conv, rounds


def local_residual(mat, F, Lam, G, rho, mu_ref, n=None, force=None, Fprev=None, nprev=None):
    """r_l of Section 2.1: the unit-cell L2 norm of the local optimality residual
    grad phi = W_F(F) - Lam + rho (F - G) at the local step's result, over mu_ref
    (read as a norm, like r_p and r_d).  For the LCE the two tangential components
    of phi_n at the director are included.  Arguments per voxel, (V, d, d)."""
    if n is None:
        g = mat.P(F) - Lam + rho * (F - G)
        s2 = np.einsum("vij,vij->v", g, g)
    else:
        P, Wn, _, _, _ = mat.derivatives(F, n)
        gF = P - Lam + rho * (F - G)
        gn = Wn - force
        if Fprev is not None:  # dissipation terms of the LCE time step
            gF = gF + mat.cF[:, None, None] * (F - Fprev)
            gn = gn + mat.cn[:, None] * (n - nprev)
        a, b = tangent_basis(n)
        s2 = (np.einsum("vij,vij->v", gF, gF) + np.sum(gn * a, axis=1) ** 2 + np.sum(gn * b, axis=1) ** 2)
    return float(np.sqrt(np.mean(s2))) / mu_ref


# --------------------------------------------------------------------------- Step 1 for the LCE (F and director n)


def frank_force(n_field: np.ndarray, kappa: np.ndarray) -> np.ndarray:
    """Explicit Frank force at every voxel from the director field of iterate i
    (eq. kin2: the gradient of the internal variable is taken from the previous
    iterate).  The discrete Frank energy kappa sum_edges |n(x + h e_j) - n(x)|^2 / h^2
    restricted to |n(x)| = 1 with the neighbours frozen is const - f . n(x) with

        f(x) = 2 kappa / h^2 * sum of the 2d neighbours' directors,

    which equals 2 kappa Delta_h n_i up to a multiple of n_i (the same tangential
    force, hence the same fixed points).  n_field (3, *grid); returns (V, 3)."""
    d = n_field.ndim - 1
    N = n_field.shape[-1]
    s = np.zeros_like(n_field)
    for ax in range(1, d + 1):
        s = s + np.roll(n_field, 1, axis=ax) + np.roll(n_field, -1, axis=ax)
    return (2.0 * N * N) * np.asarray(kappa)[:, None] * s.reshape(3, -1).T


def tangent_basis(n: np.ndarray):
    """Orthonormal (a, b) spanning the plane normal to each unit vector n (V, 3):
    Gram-Schmidt of the coordinate axis least aligned with n, b = n x a."""
    k = np.argmin(np.abs(n), axis=1)
    e = np.zeros_like(n)
    e[np.arange(n.shape[0]), k] = 1.0
    a = e - np.sum(e * n, axis=1)[:, None] * n
    a = a / np.linalg.norm(a, axis=1)[:, None]
    b = np.cross(n, a)
    return a, b


def retract(n, a, b, t1, t2):
    """Move on the unit sphere: normalise(n + t1 a + t2 b)."""
    v = n + t1[:, None] * a + t2[:, None] * b
    return v / np.linalg.norm(v, axis=1)[:, None]


def local_newton_lce(mat, F0, n_init, Lam, G, force, rho, step_tol=1e-10, cap=60, armijo=1e-4, small_step=1e-7,
                     Fprev=None, nprev=None, return_conv=False):
    """Step 1 (eqs. eq and kin with the Frank gradient treated explicitly, eq. kin2) for
    the LCE at every voxel: minimise over F and the unit director n

        phi(F, n) = W(F, n) - force . n - Lam : F + rho/2 |F - G|^2,

    force: the explicit Frank force from the previous director field (frank_force).  Newton on the 11 unknowns (F, t) with n = normalise(n + t1 a + t2 b),
    (a, b) a basis of the tangent plane at the current n: the reduced Hessian adds the
    sphere's curvature term -(n . phi_n) I, plus a shift 1e-6 mu I on that block.  Backtracking keeps J > 0 and the Armijo
    decrease; steepest descent when Newton's direction does not descend.  A voxel
    stops after a full step with max |step| <= step_tol; ``cap`` bounds this call's
    iterations (another call from the returned state continues the iteration).
    Fprev, nprev (V,3,3), (V,3): the previous time step's fields; with the material's
    dissipation weights cF = nu_F/dt, cn = nu_n/dt the objective gains Section 5.1's
    dt D((F - Fprev)/dt, (n - nprev)/dt) = cF/2 |F - Fprev|^2 + cn/2 |n - nprev|^2.
    F0, Lam, G (V,3,3); n_init, force (V,3).  Returns (F, n, iters), and with
    return_conv=True also the mask of voxels that met the convergence test."""
    if Fprev is None:
        Fprev = F0
    if nprev is None:
        nprev = n_init
    V = F0.shape[0]
    F = F0.copy()
    n = n_init.copy()
    iters = np.zeros(V, dtype=np.int64)
    active = np.ones(V, dtype=bool)
    conv = np.zeros(V, dtype=bool)

    def phi(sub, Fs, ns, Lam_s, G_s, f_s, Fp, np_):
        dF, dn = Fs - Fp, ns - np_
        return (sub.W(Fs, ns) - np.sum(f_s * ns, axis=1) - np.einsum("vij,vij->v", Lam_s, Fs)
                + 0.5 * rho * np.einsum("vij,vij->v", Fs - G_s, Fs - G_s)
                + 0.5 * sub.cF * np.einsum("vij,vij->v", dF, dF) + 0.5 * sub.cn * np.sum(dn * dn, axis=1))

    for _ in range(cap + 1):
        idx = np.nonzero(active & (iters < cap))[0]
        if idx.size == 0:
            break
        sub = mat.subset(idx)
        Fa, na = F[idx], n[idx]
        Lam_s, G_s, f_s = Lam[idx], G[idx], force[idx]
        Fp_s, np_s = Fprev[idx], nprev[idx]
        P, Wn, WFF, WFn, Wnn = sub.derivatives(Fa, na)
        gF = P - Lam_s + rho * (Fa - G_s) + sub.cF[:, None, None] * (Fa - Fp_s)
        gn = Wn - f_s + sub.cn[:, None] * (na - np_s)
        a, b = tangent_basis(na)
        E = np.stack([a, b], axis=2)                                       # (v, 3, 2)
        gt = np.einsum("vk,vka->va", gn, E)
        Htt = np.einsum("vka,vkp,vpb->vab", E, Wnn, E) - np.sum(na * gn, axis=1)[:, None, None] * np.eye(2)[None]
        HFt = np.einsum("vklp,vpb->vklb", WFn, E).reshape(-1, 9, 2)
        H = np.zeros((idx.size, 11, 11))
        H[:, :9, :9] = WFF.reshape(-1, 9, 9) + (rho + sub.cF)[:, None, None] * np.eye(9)[None]
        Htt = Htt + sub.cn[:, None, None] * np.eye(2)[None]
        H[:, :9, 9:] = HFt
        H[:, 9:, :9] = HFt.transpose(0, 2, 1)
        # Levenberg shift on the two director unknowns: keeps the step defined where W does
        # not depend on n (r = 1, alpha = 0); the converged point (gradient zero) is unchanged
        H[:, 9:, 9:] = Htt + 1e-6 * sub.mu[:, None, None] * np.eye(2)[None]
        g = np.concatenate([gF.reshape(-1, 9), gt], axis=1)
        delta = -np.linalg.solve(H, g[..., None])[..., 0]
        slope = np.sum(g * delta, axis=1)
        bad = ~(slope < 0.0) | ~np.all(np.isfinite(delta), axis=1)
        if np.any(bad):
            delta[bad] = -g[bad]
            slope[bad] = -np.sum(g[bad] * g[bad], axis=1)
        phi0 = phi(sub, Fa, na, Lam_s, G_s, f_s, Fp_s, np_s)
        size = np.max(np.abs(delta), axis=1)
        t = np.ones(idx.size)
        accepted = np.zeros(idx.size, dtype=bool)
        for _ls in range(60):
            pend = ~accepted
            if not np.any(pend):
                break
            Ft = Fa + t[:, None, None] * delta[:, :9].reshape(-1, 3, 3)
            nt = retract(na, a, b, t * delta[:, 9], t * delta[:, 10])
            J = np.linalg.det(Ft)
            ok = J > 0.0
            with np.errstate(invalid="ignore", divide="ignore"):
                ph = phi(sub, Ft, nt, Lam_s, G_s, f_s, Fp_s, np_s)
            dec = ph <= phi0 + armijo * t * slope
            acc = pend & ok & (dec | (t * size <= small_step))
            accepted |= acc
            t = np.where(pend & ~acc, 0.5 * t, t)
        t = np.where(accepted, t, 0.0)
        F[idx] = Fa + t[:, None, None] * delta[:, :9].reshape(-1, 3, 3)
        n[idx] = retract(na, a, b, t * delta[:, 9], t * delta[:, 10])
        iters[idx] += 1
        done = accepted & (t == 1.0) & (size <= step_tol)
        active[idx[done]] = False
        conv[idx[done]] = True
    return (F, n, iters, conv) if return_conv else (F, n, iters)


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0


def cofactor(F):
    """Cofactor matrix d(det F)/dF = det(F) F^{-T}, per voxel (V,3,3), from its polynomial form."""
    return 0.5 * np.einsum("kri,lsj,vrs,vij->vkl", _EPS, _EPS, F, F)


def d2det(F):
    """Second derivative of det F: d2J/dF_kl dF_rs = sum_ij eps_kri eps_lsj F_ij, shape (V,3,3,3,3)."""
    return np.einsum("kri,lsj,vij->vklrs", _EPS, _EPS, F)


def local_newton_lce_inc(mat, F0, n_init, Lam, G, force, rho, step_tol=1e-10, cap=60, big=0.25,
                         Fprev=None, nprev=None):
    """Step 1 for the incompressible LCE (Section 5.1: det F = 1 enforced in the local
    step by a Lagrange multiplier p; the director on the unit sphere as in
    local_newton_lce).  Newton on the stationarity of phi - p (det F - 1) in (F, t, p):
    the 12 x 12 system [[K, -a], [-a^T, 0]] (dx, dp) = (-g, det F - 1), with g the
    gradient of phi - p det F, K its Hessian in (F, t) (phi's plus -p d2det on the F
    block, the sphere's curvature term and the 1e-6 mu shift on the director block;
    (mu + rho) I is added where K is not positive definite) and a = (cof F, 0, 0).  p starts from the least-squares fit of cof F to phi's F-gradient.
    A step longer than `big` (max norm over F and t) is scaled to `big`; every step
    keeps det F > 0 by halving; no merit line search.  A voxel stops after a full step
    of size <= step_tol.  Returns (F, n, iters)."""
    V = F0.shape[0]
    F = F0.copy()
    n = n_init.copy()
    if Fprev is None:
        Fprev = F0
    if nprev is None:
        nprev = n_init
    iters = np.zeros(V, dtype=np.int64)
    active = np.ones(V, dtype=bool)
    p = np.full(V, np.nan)
    for _ in range(cap):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        sub = mat.subset(idx)
        Fa, na = F[idx], n[idx]
        Lam_s, G_s, f_s = Lam[idx], G[idx], force[idx]
        Fp_s, np_s = Fprev[idx], nprev[idx]
        P, Wn, WFF, WFn, Wnn = sub.derivatives(Fa, na)
        K9 = cofactor(Fa)
        J = np.einsum("vij,vij->v", Fa, K9) / 3.0
        gF0 = P - Lam_s + rho * (Fa - G_s) + sub.cF[:, None, None] * (Fa - Fp_s)
        pa = p[idx]
        fresh = np.isnan(pa)
        if np.any(fresh):
            pa[fresh] = (np.einsum("vij,vij->v", K9, gF0) / np.einsum("vij,vij->v", K9, K9))[fresh]
        gF = gF0 - pa[:, None, None] * K9
        gn = Wn - f_s + sub.cn[:, None] * (na - np_s)
        a, b = tangent_basis(na)
        E = np.stack([a, b], axis=2)
        gt = np.einsum("vk,vka->va", gn, E)
        Htt = (np.einsum("vka,vkp,vpb->vab", E, Wnn, E) - np.sum(na * gn, axis=1)[:, None, None] * np.eye(2)[None]
               + sub.cn[:, None, None] * np.eye(2)[None] + 1e-6 * sub.mu[:, None, None] * np.eye(2)[None])
        HFt = np.einsum("vklp,vpb->vklb", WFn, E).reshape(-1, 9, 2)
        KKT = np.zeros((idx.size, 12, 12))
        KKT[:, :9, :9] = ((WFF - pa[:, None, None, None, None] * d2det(Fa)).reshape(-1, 9, 9)
                          + (rho + sub.cF)[:, None, None] * np.eye(9)[None])
        KKT[:, :9, 9:11] = HFt
        KKT[:, 9:11, :9] = HFt.transpose(0, 2, 1)
        KKT[:, 9:11, 9:11] = Htt
        # a K that is not positive definite (the director near a maximum of W on the
        # sphere) gets the shift (mu + rho) I, so that the step descends on the constraint
        # manifold instead of converging to that stationary point
        notpd = np.linalg.eigvalsh(KKT[:, :11, :11])[:, 0] <= 0.0
        if np.any(notpd):
            KKT[notpd, :11, :11] += (sub.mu[notpd] + rho)[:, None, None] * np.eye(11)[None]
        KKT[:, :9, 11] = -K9.reshape(-1, 9)
        KKT[:, 11, :9] = -K9.reshape(-1, 9)
        rhs = np.concatenate([-gF.reshape(-1, 9), -gt, (J - 1.0)[:, None]], axis=1)
        sol = np.linalg.solve(KKT, rhs[..., None])[..., 0]
        dx, dp = sol[:, :11], sol[:, 11]
        size = np.max(np.abs(dx), axis=1)
        t = np.where(size > big, big / np.maximum(size, 1e-300), 1.0)
        for _h in range(40):
            Ft = Fa + t[:, None, None] * dx[:, :9].reshape(-1, 3, 3)
            bad = ~(np.linalg.det(Ft) > 0.0)
            if not np.any(bad):
                break
            t = np.where(bad, 0.5 * t, t)
        F[idx] = Fa + t[:, None, None] * dx[:, :9].reshape(-1, 3, 3)
        n[idx] = retract(na, a, b, t * dx[:, 9], t * dx[:, 10])
        p[idx] = pa + t * dp
        iters[idx] += 1
        done = (t == 1.0) & (size <= step_tol)
        active[idx[done]] = False
    return F, n, iters


# --------------------------------------------------------------------------- Steps 3 and 4


def multiplier_update(Lam, G_new, F, rho):
    """Step 3 (eq. update): Lambda_{i+1} = Lambda_i + rho (grad u_{i+1} - F_{i+1})."""
    return Lam + rho * (G_new - F)


# --------------------------------------------------------------------------- the iteration


def rms(T: np.ndarray) -> float:
    """Unit-cell L2 norm: sqrt(mean over voxels of the squared Frobenius norm)."""
    d = T.shape[0]
    return float(np.sqrt(np.sum(T * T) / T[0, 0].size))


def initial_state(mat, Fbar_d: np.ndarray, grid_shape, lambda0: str = "stress", n0=None):
    d = Fbar_d.shape[0]
    V = int(np.prod(grid_shape))
    Fv = np.broadcast_to(Fbar_d, (V, d, d)).copy()
    F = _to_field(Fv, grid_shape)
    if lambda0 == "stress":
        Lam = _to_field(mat.P(Fv) if n0 is None else mat.P(Fv, np.asarray(n0).reshape(3, -1).T), grid_shape)
    elif lambda0 == "zero":
        Lam = np.zeros_like(F)
    else:
        raise ValueError(lambda0)
    u = np.zeros((d,) + tuple(grid_shape))
    st = {"F": F, "Lam": Lam, "u": u}
    if n0 is not None:
        st["n"] = np.array(n0, dtype=np.float64).reshape((3,) + tuple(grid_shape))
    return st


def admm_solve(phase, params, Fbar, rho, tol, max_iter, model="neohookean", mu_ref=None,
               lambda0="stress", state=None, rho_policy="fixed", kappa=1.3, tau=10.0,
               rho_min=None, local_cap=50, step_tol=1e-10, n0=None, local_ratio=0.0, free=None,
               local_fraction=0.0, incompressible=False, local_round=1):
    """Run the ADMM iteration (Steps 1-4) until r_p <= tol and r_d <= tol, or max_iter.

    phase: uint8 grid (N,)*d; params: per-phase (mu, lam); Fbar: 3x3 (the upper-left
    d x d block is used).  Returns a dict with F, Lam, u (final state), iters,
    converged, history (list of (r_p, r_d, rho_used)), rho (next rho) and the
    homogenised first Piola-Kirchhoff stress <W_F(F)> (d x d).

    local_ratio = f > 0: approximate local steps with r_l <= f r_d (Section 2.1,
    "Approximate solution of the local problem"; Algorithm 1's inner loop; Section
    4.2's second strategy).  Step 1 of iteration i+1 runs Newton in rounds of
    ``local_round`` iterations at the points not yet converged and stops once the
    unit-cell L2 local residual r_l (local_residual) is <= f times the r_d of the
    latest check (Step 4 of iteration i); r_l is also tested before the first round.
    The first iteration has no r_d yet and solves exactly.  out["local_residual"]
    lists r_l after every Step 1, out["local_rounds"] the rounds each one took.

    free: optional (3, 3) boolean mask of components of <F> left free (mixed
    macroscopic control, Section 2.3; Section 5.3's UNI, PE and EB protocols): they
    join Step 2's minimisation, whose mean part gives <F>_free = <F - Lambda/rho>_free
    (the fluctuation Du~ has zero mean), so that <Lambda>_free = 0 after every
    multiplier update and <W_F(F)>_free -> 0 at convergence.  Fbar gives their
    starting values; out["Fbar"] holds the final macroscopic gradient (3 x 3).

    local_fraction = p > 0 (elastic laws): Section 4.2's first strategy.  Step 1 runs
    Newton in rounds of two iterations at the points not yet converged and, after
    each round, proceeds to Step 2 once at least p V points have met their pointwise
    test (a full Newton step <= step_tol).  out["local_rounds"] lists the rounds of
    every Step 1, out["local_converged"] the converged count after it.

    incompressible (model "lce"): the network of Section 5.1 with det F = 1 enforced in
    Step 1 by a multiplier (local_newton_lce_inc), whose local problem is always solved
    to the step tolerance (local_ratio does not apply); out["stress"] is then <Lambda>,
    which equals <W_F - p cof F> (+ the viscous part) once the iteration has converged.
    """
    phase = np.asarray(phase)
    d = phase.ndim
    grid = phase.shape
    lce = model == "lce"
    mat = make_lce(phase, params, n0, incompressible) if lce else make_material(model, phase, params)
    Fbar_d = np.array(np.asarray(Fbar, dtype=np.float64)[:d, :d])
    free_d = None if free is None else np.asarray(free, dtype=bool)[:d, :d]
    if mu_ref is None:
        mu_ref = float(np.mean(mat.mu))
    if rho_min is None:
        rho_min = mu_ref
    if state is None:
        st = initial_state(mat, Fbar_d, grid, lambda0, n0=n0 if lce else None)
    else:
        st = {k: np.array(v, dtype=np.float64, copy=True) for k, v in state.items()}
    F, Lam, u = st["F"], st["Lam"], st["u"]
    nd = st.get("n")
    G = Fbar_d.reshape((d, d) + (1,) * d) + grad_u(u)
    if lce:  # the previous time step of the dissipation terms: the state the solve starts from
        Fprev_v = _to_voxels(F).copy()
        nprev_v = nd.reshape(3, -1).T.copy()
    history = []
    local_res = []
    local_rounds = []
    local_conv = []
    converged = False
    it = 0
    V = int(np.prod(grid))
    for it in range(1, max_iter + 1):
        Lv, Gv = _to_voxels(Lam), _to_voxels(G)
        Fv = _to_voxels(F).copy()
        nv = nd.reshape(3, -1).T.copy() if lce else None
        force = frank_force(nd, mat.kappa) if lce else None
        # Step 1.  run(idx, k) advances the local Newton at voxels idx by k iterations.
        if lce and incompressible:
            def run(idx, k):
                sub = mat.subset(idx)
                Fv[idx], nv[idx], its = local_newton_lce_inc(sub, Fv[idx], nv[idx], Lv[idx], Gv[idx], force[idx],
                                                             rho, step_tol=step_tol, cap=k, Fprev=Fprev_v[idx],
                                                             nprev=nprev_v[idx])
                return its, its < k
        elif lce:
            def run(idx, k):
                sub = mat.subset(idx)
                Fv[idx], nv[idx], its, c = local_newton_lce(sub, Fv[idx], nv[idx], Lv[idx], Gv[idx], force[idx], rho,
                                                            step_tol=step_tol, cap=k, Fprev=Fprev_v[idx],
                                                            nprev=nprev_v[idx], return_conv=True)
                return its, c
        else:
            def run(idx, k):
                Fv[idx], its, c = local_newton(mat.subset(idx), Fv[idx], Lv[idx], Gv[idx], rho, step_tol=step_tol,
                                               cap=k, return_conv=True)
                return its, c

        def r_l():
            if lce:
                return local_residual(mat, Fv, Lv, Gv, rho, mu_ref, nv, force, Fprev_v, nprev_v)
            return local_residual(mat, Fv, Lv, Gv, rho, mu_ref)

        if local_ratio > 0.0 and history and not incompressible:
            rd_latest = history[-1][1]
            _, conv_v, rounds = local_step_rounds(run, V, local_cap, local_round,
                                                  lambda c: r_l() <= local_ratio * rd_latest, check_first=True)
        elif local_fraction > 0.0 and not lce:
            _, conv_v, rounds = local_step_rounds(run, V, local_cap, 2,
                                                  lambda c: np.count_nonzero(c) >= local_fraction * V,
                                                  check_first=False)
        else:
            _, conv_v, rounds = local_step_rounds(run, V, local_cap, local_cap, lambda c: False, check_first=False)
        local_rounds.append(rounds)
        local_conv.append(int(np.count_nonzero(conv_v)))
        local_res.append(r_l() if local_ratio > 0.0 else 0.0)
        if lce:
            nd = nv.T.reshape((3,) + tuple(grid))
        F = _to_field(Fv, grid)
        # Step 2 (with the free mean components of mixed control)
        uh, u = u_step(F, Lam, rho)
        if free_d is not None and free_d.any():
            Qbar = np.mean((F - Lam / rho).reshape(d, d, -1), axis=2)
            Fbar_d = np.where(free_d, Qbar, Fbar_d)
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
    if lce and incompressible:  # the pressure is not part of the state: <Lambda>
        stress = np.mean(_to_voxels(Lam), axis=0)
    elif lce:  # with the dissipation's viscous stress cF (F - Fprev)
        Fv = _to_voxels(F)
        stress = np.mean(mat.P(Fv, nd.reshape(3, -1).T) + mat.cF[:, None, None] * (Fv - Fprev_v), axis=0)
    else:
        stress = np.mean(mat.P(_to_voxels(F)), axis=0)
    out = {"F": F, "Lam": Lam, "u": u, "iters": it if max_iter > 0 else 0,
           "converged": converged, "history": history, "rho": rho,
           "stress": stress, "mu_ref": mu_ref, "local_residual": local_res, "local_rounds": local_rounds,
           "local_converged": local_conv}
    Fb3 = np.array(np.asarray(Fbar, dtype=np.float64))
    Fb3[:d, :d] = Fbar_d
    out["Fbar"] = Fb3
    if lce:
        out["n"] = nd
    return out


def homogenised_stress(phase, params, F, model="neohookean"):
    """<W_F(F)> over the cell (first Piola-Kirchhoff), shape (d, d)."""
    mat = make_material(model, phase, params)
    return np.mean(mat.P(_to_voxels(F)), axis=0)
