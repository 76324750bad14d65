"""Pins of the oracle's liquid crystal elastomer model (Section 5.1) and its local
solve, against facts independent of the oracle's derivative code."""
import numpy as np
import pytest
from scipy import optimize

import oracle
from oracle import admm as oadmm
from oracle.materials import LCE
from paper_2010_06697_gb300 import synth
from tests import energies as E

RNG = np.random.default_rng(99)
MU, LAM, R, ALPHA = 1.0, 20.0, 7.71, 0.06


def _unit(v):
    return v / np.linalg.norm(v)


def _mat(n0, r=R, alpha=ALPHA, kappa=0.0, V=1):
    return LCE(np.full(V, MU), np.full(V, LAM), np.full(V, r), np.full(V, alpha), np.full(V, kappa),
               np.broadcast_to(n0, (V, 3)).copy())


def test_lce_derivatives_match_complex_step():
    """W_F, and the derivatives in n along the unit sphere (the only ones the local
    solve uses: tangential gradient, Riemannian Hessian E^T W_nn E - (n.W_n) I, mixed
    block W_Fn E), equal complex-step / finite-difference derivatives of Section 5.1's
    energy typed separately (whose extension off |n| = 1 differs)."""
    for _ in range(5):
        F = np.eye(3) + 0.2 * RNG.uniform(-1, 1, (3, 3))
        n = _unit(RNG.standard_normal(3))
        n0 = _unit(RNG.standard_normal(3))
        m = _mat(n0)
        args = (MU, LAM, R, ALPHA, n0)
        assert abs(m.W(F[None], n[None])[0] - np.real(E.w_lce(F, n, *args))) < 1e-12
        P, Wn, WFF, WFn, Wnn = m.derivatives(F[None], n[None])
        gF, gn = E.lce_grad_cs(F, n, args)
        np.testing.assert_allclose(P[0], gF, atol=1e-11)
        a, b = oadmm.tangent_basis(n[None])
        Et = np.stack([a[0], b[0]], axis=1)                      # (3, 2)
        np.testing.assert_allclose(Et.T @ Wn[0], Et.T @ gn, atol=1e-11)
        eps = 1e-6
        for k in range(3):
            for l in range(3):
                dF = np.zeros((3, 3))
                dF[k, l] = eps
                gp, gnp = E.lce_grad_cs(F + dF, n, args)
                gm, gnm = E.lce_grad_cs(F - dF, n, args)
                np.testing.assert_allclose(WFF[0][:, :, k, l], (gp - gm) / (2 * eps), atol=1e-6)
                np.testing.assert_allclose(Et.T @ WFn[0][k, l, :], Et.T @ (gnp - gnm) / (2 * eps), atol=1e-6)
        # Riemannian Hessian in the tangent plane from second differences of W along the sphere
        def w_on_sphere(t):
            return np.real(E.w_lce(F, oadmm.retract(n[None], a, b, np.array([t[0]]), np.array([t[1]]))[0], *args))
        H_fd = np.zeros((2, 2))
        h = 1e-4
        for i in range(2):
            for j in range(2):
                ei, ej = np.eye(2)[i] * h, np.eye(2)[j] * h
                H_fd[i, j] = (w_on_sphere(ei + ej) - w_on_sphere(ei - ej) - w_on_sphere(-ei + ej)
                              + w_on_sphere(-ei - ej)) / (4 * h * h)
        H_or = Et.T @ Wnn[0] @ Et - np.dot(n, Wn[0]) * np.eye(2)
        np.testing.assert_allclose(H_or, H_fd, atol=1e-5)


def test_lce_ground_state_is_stress_free():
    """Section 5.1: F = R l0^{1/2} Q, n = R e gives W_el = 0; with n0 = e also W_ni = 0,
    and the homogeneous cell at that Fbar is an exact fixed point with zero stress."""
    e = _unit(np.array([0.6, 0.8, 0.0]))
    ell = R ** (-1 / 3) * (np.eye(3) + (R - 1) * np.outer(e, e))
    w, Q = np.linalg.eigh(ell)
    Fg = Q @ np.diag(np.sqrt(w)) @ Q.T
    th = 0.3
    Rot = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    m = _mat(e)
    assert abs(np.real(E.w_lce(Fg, e, MU, LAM, R, ALPHA, e))) < 1e-13
    assert abs(np.real(E.w_lce(Rot @ Fg, Rot @ e, MU, LAM, R, 0.0, e))) < 1e-13
    assert np.max(np.abs(m.P(Fg[None], e[None]))) < 1e-13
    n = 8
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.broadcast_to(e[:, None, None, None], (3, n, n, n)).copy()
    par = np.array([[MU, LAM, R, ALPHA, 4.0 / n ** 2]])
    r = oracle.admm_solve(ph, par, Fg, 10.0, 1e-12, 5, model="lce", n0=n0)
    assert r["converged"] and r["iters"] == 1
    assert np.max(np.abs(r["stress"])) < 1e-12
    assert np.max(np.abs(r["n"] - n0)) < 1e-12


def test_lce_reduces_to_neohookean():
    """r = 1, alpha = 0, kappa_F = 0: W no longer depends on n (Section 5.1) and the
    LCE iteration equals the neo-Hookean one."""
    n = 8
    ph = synth.inclusion_phase(n, 3, 2, radius=2)
    par_nh = synth.two_phase_params(1.0, 10.0)
    par = np.column_stack([par_nh, np.ones(2), np.zeros(2), np.zeros(2)])
    n0 = synth.director_grf(n, 3, corr=2.0)
    Fbar = np.diag([0.95, 1.02, 1.0])
    a = oracle.admm_solve(ph, par_nh, Fbar, 10.0, -1.0, 6)
    b = oracle.admm_solve(ph, par, Fbar, 10.0, -1.0, 6, model="lce", n0=n0)
    np.testing.assert_allclose(b["F"], a["F"], atol=1e-12)
    np.testing.assert_allclose(b["stress"], a["stress"], atol=1e-12)


def test_uniform_director_has_no_frank_torque():
    """A uniform director field: the Frank force is parallel to n (no tangential part)."""
    n = 6
    e = _unit(np.array([0.2, -0.5, 0.8]))
    field = np.broadcast_to(e[:, None, None, None], (3, n, n, n)).copy()
    f = oadmm.frank_force(field, np.full(n ** 3, 0.3))
    tang = f - np.sum(f * e[None], axis=1)[:, None] * e[None]
    assert np.max(np.abs(tang)) < 1e-12


def test_frank_force_is_tangentially_the_laplacian():
    """The neighbour-sum force equals 2 kappa Delta_h n (compact Laplacian, Section 2.3
    symbol, here by FFT) up to a multiple of n: same tangential component."""
    n = 8
    field = synth.director_grf(n, 5, corr=2.0)
    kap = 0.07
    f = oadmm.frank_force(field, np.full(n ** 3, kap))
    m = np.fft.fftfreq(n) * n
    s = -4.0 * n * n * np.sin(np.pi * m / n) ** 2
    sym = s[:, None, None] + s[None, :, None] + s[None, None, :]
    lap = np.fft.ifftn(np.fft.fftn(field, axes=(1, 2, 3)) * sym, axes=(1, 2, 3)).real
    g = 2 * kap * lap.reshape(3, -1).T
    nv = field.reshape(3, -1).T
    proj = lambda x: x - np.sum(x * nv, axis=1)[:, None] * nv
    np.testing.assert_allclose(proj(f), proj(g), atol=1e-9)


@pytest.mark.parametrize("trial", range(3))
def test_lce_local_solve_matches_brute_force(trial):
    """Step 1 for the LCE at one voxel: the oracle's (F, n) minimiser agrees with a
    derivative-free minimisation over F and the two spherical angles of n."""
    rng = np.random.default_rng(100 + trial)
    n0 = _unit(rng.standard_normal(3))
    n_init = _unit(n0 + 0.3 * rng.standard_normal(3))
    G = np.eye(3) + 0.08 * rng.uniform(-1, 1, (3, 3))
    Lam = 0.3 * rng.uniform(-1, 1, (3, 3))
    f = 0.5 * rng.standard_normal(3)
    rho = 10.0
    r_ = 2.5

    def phi(x):
        F = x[:9].reshape(3, 3)
        th, ps = x[9], x[10]
        nn = np.array([np.sin(th) * np.cos(ps), np.sin(th) * np.sin(ps), np.cos(th)])
        if np.linalg.det(F) <= 0:
            return np.inf
        return (float(np.real(E.w_lce(F, nn, MU, LAM, r_, ALPHA, n0))) - f @ nn - np.sum(Lam * F)
                + 0.5 * rho * np.sum((F - G) ** 2))

    m = _mat(n0, r=r_)
    Fn, nn, _ = oadmm.local_newton_lce(m, G[None].copy(), n_init[None], Lam[None], G[None], f[None], rho)
    th0 = np.arccos(np.clip(nn[0, 2], -1, 1))
    ps0 = np.arctan2(nn[0, 1], nn[0, 0])
    x_newton = np.concatenate([Fn[0].ravel(), [th0, ps0]])
    best = None
    for s in range(3):
        x0 = x_newton + 0.02 * rng.standard_normal(11)
        res = optimize.minimize(phi, x0, method="Nelder-Mead",
                                options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 60000, "maxfev": 120000})
        res = optimize.minimize(phi, res.x, method="Powell", options={"xtol": 1e-11, "ftol": 1e-15})
        if best is None or res.fun < best.fun:
            best = res
    assert phi(x_newton) <= best.fun + 1e-11
    np.testing.assert_allclose(Fn[0].ravel(), best.x[:9], atol=1e-5)
    nb = np.array([np.sin(best.x[9]) * np.cos(best.x[10]), np.sin(best.x[9]) * np.sin(best.x[10]), np.cos(best.x[9])])
    assert min(np.max(np.abs(nb - nn[0])), np.max(np.abs(nb + nn[0]))) < 1e-5


# ------------------------------------------------------------------ dissipation (one time step)

def test_lce_time_step_homogeneous_cell_matches_brute_force():
    """One implicit time step with Section 5.1's dissipation on a homogeneous cell: from
    a state (F_old, n_old), a new <F> makes F = <F> everywhere, the director minimises
    W(<F>, n) + cn/2 |n - n_old|^2 on the unit sphere (found here by multi-start
    Nelder-Mead over two angles, with the energy typed separately in tests/energies.py),
    and <S> = W_F(<F>, n*) + cF (<F> - F_old).  A uniform director has no Frank torque."""
    n = 4
    mu, lam, r, alpha, cF, cn = 1.0, 20.0, 4.0, 0.1, 5.6, 0.4
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.array([0.0, 1.0, 0.0])
    par = np.array([[mu, lam, r, alpha, (2.0 / n) ** 2, cF, cn]])
    n0f = np.broadcast_to(n0.reshape(3, 1, 1, 1), (3, n, n, n)).copy()
    F_old = np.diag([1.05, 0.97, 0.98])
    th = 0.4
    n_old = np.array([np.sin(th), np.cos(th), 0.0])
    V = n ** 3
    state = {"F": np.broadcast_to(F_old.reshape(3, 3, 1, 1, 1), (3, 3, n, n, n)).copy(),
             "Lam": np.zeros((3, 3, n, n, n)), "u": np.zeros((3, n, n, n)),
             "n": np.broadcast_to(n_old.reshape(3, 1, 1, 1), (3, n, n, n)).copy()}
    F_new = np.diag([1.12, 0.95, 0.96])
    res = oracle.admm_solve(ph, par, F_new, 10.0, 1e-11, 3000, model="lce", n0=n0f, state=state)
    assert res["converged"]

    def energy(angles):
        a, b = angles
        nn = np.array([np.sin(a) * np.cos(b), np.cos(a), np.sin(a) * np.sin(b)])
        w = E.w_lce(F_new, nn, mu, lam, r, alpha, n0)
        return w + 0.5 * cn * np.sum((nn - n_old) ** 2)

    best = min((optimize.minimize(energy, x0, method="Nelder-Mead",
                                  options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 20000})
                for x0 in ([0.1, 0.0], [0.5, 0.3], [1.2, -0.4], [2.0, 1.0])), key=lambda o: o.fun)
    a, b = best.x
    n_star = np.array([np.sin(a) * np.cos(b), np.cos(a), np.sin(a) * np.sin(b)])
    nv = res["n"].reshape(3, -1).T
    # the director is determined up to sign (n and -n are the same state)
    s = np.sign(nv @ n_star)[:, None]
    np.testing.assert_allclose(nv * s, np.broadcast_to(n_star, (V, 3)), atol=1e-6)
    np.testing.assert_allclose(res["F"].reshape(9, -1).T, np.broadcast_to(F_new.ravel(), (V, 9)), atol=1e-9)
    P_star, _ = E.lce_grad_cs(F_new, n_star, (mu, lam, r, alpha, n0))
    np.testing.assert_allclose(res["stress"], P_star + cF * (F_new - F_old), atol=1e-8)


# ------------------------------------------------------------------ incompressible network

def test_incompressible_uniaxial_stress_closed_form():
    """r = 1, alpha = 0 turns the incompressible LCE into incompressible neo-Hookean,
    W = mu/2 (|F|^2 - 3) with det F = 1.  Under uniaxial stress (<F_11> = s prescribed,
    every other component free: mixed control) the exact cell state is F =
    diag(s, s^-1/2, s^-1/2) with P_11 = mu (s - s^-2) and the other components zero."""
    n, mu, s = 4, 1.0, 1.15
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.broadcast_to(np.array([0.0, 1.0, 0.0]).reshape(3, 1, 1, 1), (3, n, n, n)).copy()
    par = np.array([[mu, 0.0, 1.0, 0.0, 0.0]])
    free = np.ones((3, 3), bool)
    free[0, 0] = False
    r = oracle.admm_solve(ph, par, np.diag([s, 1.0, 1.0]), 10.0, 1e-11, 3000, model="lce", n0=n0,
                          free=free, incompressible=True)
    assert r["converged"]
    q = s ** -0.5
    np.testing.assert_allclose(r["Fbar"], np.diag([s, q, q]), atol=1e-9)
    np.testing.assert_allclose(np.linalg.det(r["F"].reshape(9, -1).T.reshape(-1, 3, 3)), 1.0, atol=1e-12)
    np.testing.assert_allclose(r["stress"], np.diag([mu * (s - s ** -2), 0.0, 0.0]), atol=1e-9)


def test_incompressible_homogeneous_cell_director_and_reaction():
    """Homogeneous incompressible cell at an isochoric <F> (all components prescribed):
    F = <F> everywhere, the director minimises W(<F>, n) (brute force over the sphere,
    energy typed separately) and Lambda differs from W_F(<F>, n*) by a multiple of
    cof <F> only: the undetermined reaction pressure of the constraint."""
    n = 4
    mu, r_, alpha = 1.0, 4.0, 0.1
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.array([1.0, 0.0, 0.0])  # along the stretch: the director's stable minimum is nearby
    n0f = np.broadcast_to(n0.reshape(3, 1, 1, 1), (3, n, n, n)).copy()
    par = np.array([[mu, 0.0, r_, alpha, 0.0]])  # a uniform director has no Frank torque anyway
    s = 1.12
    Fb = np.diag([s, s ** -0.5, s ** -0.5])
    Fb[0, 1] = 0.05
    Fb[1, 2] = -0.03
    res = oracle.admm_solve(ph, par, Fb, 10.0, 1e-11, 3000, model="lce", n0=n0f, incompressible=True)
    assert res["converged"]
    np.testing.assert_allclose(res["F"].reshape(9, -1).T, np.broadcast_to(Fb.ravel(), (n ** 3, 9)), atol=1e-9)

    def w_inc(F, nn):  # incompressible network + non-ideality: the compressible form minus its volumetric terms
        lnJ = np.log(np.linalg.det(F))
        return E.w_lce(F, nn, mu, 0.0, r_, alpha, n0) + mu * lnJ

    # the director's minimum near n0 (local search in the tangent plane of n0)
    def nvec(c):
        v = n0 + c[0] * np.array([0.0, 1.0, 0.0]) + c[1] * np.array([0.0, 0.0, 1.0])
        return v / np.linalg.norm(v)

    best = optimize.minimize(lambda c: w_inc(Fb, nvec(c)), [0.0, 0.0], method="Nelder-Mead",
                             options={"xatol": 1e-12, "fatol": 1e-16, "maxiter": 20000})
    n_star = nvec(best.x)
    nv = res["n"].reshape(3, -1).T
    np.testing.assert_allclose(nv * np.sign(nv @ n_star)[:, None], np.broadcast_to(n_star, (n ** 3, 3)), atol=1e-6)
    # W_F of the incompressible energy by complex step (the compressible one minus
    # -mu F^-T), at the cell's director: it matches the brute-force minimiser above to
    # the search's accuracy, and W_F is not stationary in n, so the exact one is used
    n_cell = nv[0] * np.sign(nv[0] @ n_star)
    gF, _ = E.lce_grad_cs(Fb, n_cell, (mu, 0.0, r_, alpha, n0))
    WF = gF + mu * np.linalg.inv(Fb).T
    lam_mean = res["Lam"].reshape(9, -1).mean(axis=1).reshape(3, 3)
    cof = np.linalg.det(Fb) * np.linalg.inv(Fb).T
    d = lam_mean - WF
    p_fit = -np.sum(d * cof) / np.sum(cof * cof)
    np.testing.assert_allclose(d, -p_fit * cof, atol=1e-8)
