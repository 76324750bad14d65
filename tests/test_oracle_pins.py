"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the pin and the passage of the paper (Zhou & Bhattacharya) that
fixes it.  They run on the CPU (no GPU marker).
"""
import numpy as np
import pytest
from scipy import optimize

import oracle
from oracle import admm as oadmm
from oracle.materials import make_material
from paper_2010_06697_gb300 import synth
from tests import energies as E

RNG = np.random.default_rng(1234)


def _near_identity(d, amp, rng=RNG):
    return np.eye(d) + amp * rng.uniform(-1, 1, (d, d))


# ------------------------------------------------------------- P5: constitutive derivatives

@pytest.mark.parametrize("model", ["neohookean", "linear"])
@pytest.mark.parametrize("d", [2, 3])
def test_stress_and_tangent_match_numerical_derivatives(model, d):
    """W_F and W_FF of the oracle equal the complex-step / finite-difference derivatives
    of the energy written from Section 4.1 (independent route)."""
    mu, lam = 2.3, 3.7
    w = E.ENERGIES[model]
    for _ in range(5):
        F = _near_identity(d, 0.2)
        mat = make_material(model, np.zeros(1, np.uint8), np.array([[mu, lam]]))
        P = mat.P(F[None])[0]
        C = mat.C(F[None])[0]
        np.testing.assert_allclose(mat.W(F[None])[0], np.real(w(F, mu, lam)), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(P, E.stress_cs(w, F, mu, lam), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(C, E.tangent_fd(w, F, mu, lam), rtol=1e-7, atol=1e-7)


def test_plane_strain_3d_energy_reduces_to_2d():
    """The 3D compressible neo-Hookean at F = diag(F2, 1) equals the 2D Mooney-Rivlin form."""
    for _ in range(5):
        F2 = _near_identity(2, 0.2)
        F3 = np.eye(3)
        F3[:2, :2] = F2
        assert abs(E.w_neohooke_3d(F3, 1.3, 2.1) - E.w_mooney_rivlin_2d(F2, 1.3, 2.1)) < 1e-14


# ------------------------------------------------------------- P5: brute-force local problem

@pytest.mark.parametrize("model", ["neohookean", "linear"])
@pytest.mark.parametrize("d", [2, 3])
def test_local_newton_matches_brute_force_minimum(model, d):
    """Step 1 (eq. eq) at one voxel: the oracle's Newton minimiser agrees with a
    multi-start derivative-free minimisation of phi(F) = W - Lam:F + rho/2|F-G|^2."""
    rng = np.random.default_rng(7 + d)
    w = E.ENERGIES[model]
    for trial in range(3):
        mu, lam = rng.uniform(0.5, 10), rng.uniform(0.5, 15)
        rho = rng.uniform(2, 20)
        G = _near_identity(d, 0.15, rng)
        Lam = rng.uniform(-1, 1, (d, d))

        def phi(x):
            F = x.reshape(d, d)
            if np.linalg.det(F) <= 0:
                return np.inf
            return float(np.real(w(F, mu, lam))) - np.sum(Lam * F) + 0.5 * rho * np.sum((F - G) ** 2)

        best = None
        for s in range(4):
            x0 = (G + 0.05 * rng.standard_normal((d, d))).ravel()
            r = optimize.minimize(phi, x0, method="Nelder-Mead",
                                  options={"xatol": 1e-11, "fatol": 1e-15, "maxiter": 40000, "maxfev": 80000})
            r = optimize.minimize(phi, r.x, method="Powell", options={"xtol": 1e-12, "ftol": 1e-15})
            if best is None or r.fun < best.fun:
                best = r
        mat = make_material(model, np.zeros(1, np.uint8), np.array([[mu, lam]]))
        Fn, _ = oadmm.local_newton(mat, np.eye(d)[None].copy(), Lam[None], G[None], rho)
        assert phi(Fn[0].ravel()) <= best.fun + 1e-12
        np.testing.assert_allclose(Fn[0], best.x.reshape(d, d), atol=1e-6)
        # stationarity of eq. eq with the independent derivative
        res = E.stress_cs(w, Fn[0], mu, lam) - Lam - rho * (G - Fn[0])
        assert np.max(np.abs(res)) < 1e-11


# ------------------------------------------------------------- P4: Helmholtz projection

@pytest.mark.parametrize("d,n", [(2, 16), (3, 8), (2, 12), (3, 6)])
def test_poisson_recovers_manufactured_displacement(d, n):
    """Step 2 (eq. helmf, central-difference symbols): with Lambda = 0 and
    F = Fbar + D u* (real-space stencil), the projection returns D u~ = D u* exactly
    and u~ has no content on the null modes of D."""
    rng = np.random.default_rng(3)
    grid = (n,) * d
    u_star = rng.standard_normal((d,) + grid)
    Fbar = _near_identity(d, 0.1, rng)
    F = Fbar.reshape((d, d) + (1,) * d) + E.grad_stencil(u_star)
    uh, u = oadmm.u_step(F, np.zeros_like(F), 10.0)
    np.testing.assert_allclose(E.grad_stencil(u), E.grad_stencil(u_star), atol=1e-12)
    # null-mode content of u~ (m_j in {0, n/2} for all j) is zero
    U = np.fft.fftn(u, axes=tuple(range(1, d + 1)))
    m = np.fft.fftfreq(n) * n
    null1 = (m == 0) | (m == -n // 2)
    mask = np.ones(grid, dtype=bool)
    for a in range(d):
        shape = [1] * d
        shape[a] = n
        mask = mask & null1.reshape(shape)
    assert np.max(np.abs(U[:, mask])) < 1e-10


@pytest.mark.parametrize("d,n", [(2, 4), (2, 6), (3, 4)])
def test_poisson_equals_dense_least_squares(d, n):
    """Step 2 as the minimiser over u~ of ||Fbar + D u~ - F + Lambda/rho||^2 (Section 2.1),
    solved with an explicit dense matrix of the central-difference gradient."""
    rng = np.random.default_rng(11)
    grid = (n,) * d
    V = n ** d
    F = rng.standard_normal((d, d) + grid)
    Lam = rng.standard_normal((d, d) + grid)
    rho = 3.0
    # dense D: column (i, voxel) -> row (i, j, voxel)
    Dm = np.zeros((d * d * V, d * V))
    for i in range(d):
        for v in range(V):
            e = np.zeros((d,) + grid)
            e[i].reshape(-1)[v] = 1.0
            Dm[:, i * V + v] = E.grad_stencil(e).reshape(-1)
    rhs = (F - Lam / rho).reshape(-1)            # mean part is orthogonal to range(D)
    x, *_ = np.linalg.lstsq(Dm, rhs, rcond=None)
    _, u = oadmm.u_step(F, Lam, rho)
    np.testing.assert_allclose(E.grad_stencil(u).reshape(-1), Dm @ x, atol=1e-11)
    # normal equations D^T D u = D^T (F - Lam/rho) in real space
    lhs = -E.div_stencil(E.grad_stencil(u))
    rhs2 = -E.div_stencil(F - Lam / rho)
    np.testing.assert_allclose(lhs, rhs2, atol=1e-10)


# ------------------------------------------------------------- P1: affine exactness

@pytest.mark.parametrize("d,n", [(2, 16), (3, 8)])
def test_homogeneous_cell_is_fixed_point(d, n):
    """A single-phase cell at any Fbar: with Lambda_0 = W_F(Fbar) the affine state is an
    exact fixed point after one iteration; from Lambda_0 = 0 the iteration reaches it."""
    rng = np.random.default_rng(5)
    ph = np.zeros((n,) * d, np.uint8)
    par = np.array([[1.7, 2.9]])
    Fbar3 = np.eye(3)
    Fbar3[:d, :d] = _near_identity(d, 0.1, rng)
    Fb = Fbar3[:d, :d]
    P_ref = E.stress_cs(E.w_neohooke, Fb, 1.7, 2.9)
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, -1.0, 1)
    assert np.max(np.abs(r["F"] - Fb.reshape((d, d) + (1,) * d))) < 1e-14
    assert np.max(np.abs(r["u"])) < 1e-14
    assert np.max(np.abs(r["Lam"] - P_ref.reshape((d, d) + (1,) * d))) < 1e-12
    assert r["history"][0][0] < 1e-14 and r["history"][0][1] < 1e-13
    r0 = oracle.admm_solve(ph, par, Fbar3, 10.0, 1e-12, 300, lambda0="zero")
    assert r0["converged"]
    np.testing.assert_allclose(r0["stress"], P_ref, atol=1e-10)


# ------------------------------------------------------------- P2 / P3: laminates

def _laminate_exact(model, params, Fbar_d, f=0.5):
    """Exact laminate with normal e_1: F_A = Fbar + (1-f) a (x) e_1, F_B = Fbar - f a (x) e_1,
    traction continuity P_A(F_A) e_1 = P_B(F_B) e_1 (independent derivatives)."""
    d = Fbar_d.shape[0]
    w = E.ENERGIES[model]
    e1 = np.zeros(d)
    e1[0] = 1.0

    def FA(a):
        return Fbar_d + (1 - f) * np.outer(a, e1)

    def FB(a):
        return Fbar_d - f * np.outer(a, e1)

    def g(a):
        return (E.stress_cs(w, FA(a), *params[0]) - E.stress_cs(w, FB(a), *params[1])) @ e1

    a = np.zeros(d)
    for _ in range(12):                    # Newton on a finite-difference Jacobian
        J = np.zeros((d, d))
        for k in range(d):
            da = np.zeros(d)
            da[k] = 1e-6
            J[:, k] = (g(a + da) - g(a - da)) / 2e-6
        a = a - np.linalg.solve(J, g(a))
    PA = E.stress_cs(w, FA(a), *params[0])
    PB = E.stress_cs(w, FB(a), *params[1])
    return FA(a), FB(a), f * PA + (1 - f) * PB


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8)])
def test_linear_laminate_closed_form(d, n):
    """Linear two-phase laminate (Section 2.2 quadratic case): ADMM converges to the
    exact piecewise-constant solution and its effective stress."""
    rng = np.random.default_rng(21)
    ph = synth.laminate_phase(n, d)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.eye(3)
    Fbar3[:d, :d] = _near_identity(d, 0.05, rng)
    FA, FB, S = _laminate_exact("linear", par, Fbar3[:d, :d])
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, 1e-13, 2000, model="linear")
    assert r["converged"]
    np.testing.assert_allclose(r["stress"], S, atol=1e-10)
    F = r["F"]
    np.testing.assert_allclose(F[..., : n // 2], np.broadcast_to(FA.reshape((d, d) + (1,) * d), F[..., : n // 2].shape), atol=1e-10)
    np.testing.assert_allclose(F[..., n // 2:], np.broadcast_to(FB.reshape((d, d) + (1,) * d), F[..., n // 2:].shape), atol=1e-10)


def test_neohookean_laminate_config1():
    """2D 32x32 compressible neo-Hookean laminate, mu = 1 | 10, nu = 0.3, Fbar =
    diag(1.05, 1), rho = 10 (Section 4.1 energy): the ADMM stress after 300
    iterations equals the semi-analytic laminate stress."""
    ph = synth.laminate_phase(32, 2)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.diag([1.05, 1.0, 1.0])
    _, _, S = _laminate_exact("neohookean", par, Fbar3[:2, :2])
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, -1.0, 300)
    np.testing.assert_allclose(r["stress"], S, atol=1e-11)
    assert abs(S[0, 1]) < 1e-14 and abs(S[1, 0]) < 1e-14


def test_neohookean_laminate_3d_sheared():
    """3D neo-Hookean laminate with a general Fbar (shear included)."""
    rng = np.random.default_rng(2)
    ph = synth.laminate_phase(8, 3)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = _near_identity(3, 0.08, rng)
    _, _, S = _laminate_exact("neohookean", par, Fbar3)
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, 1e-12, 1000)
    assert r["converged"]
    np.testing.assert_allclose(r["stress"], S, atol=1e-9)


# ------------------------------------------------------------- P6: monotone residual (convex W)

@pytest.mark.parametrize("kind", ["laminate", "inclusion"])
def test_residual_energy_monotone_for_convex_energy(kind):
    """For convex W at fixed rho, E_i = rho r_p^2 + (mu_ref^2/rho) r_d^2 is
    non-increasing (ADMM theory quoted in Section 2.1, 'Convergence')."""
    d, n = 2, 16
    ph = synth.laminate_phase(n, d) if kind == "laminate" else synth.inclusion_phase(n, d, 3, radius=3)
    par = synth.two_phase_params(1.0, 10.0)
    rng = np.random.default_rng(9)
    Fbar3 = np.eye(3)
    Fbar3[:d, :d] = _near_identity(d, 0.05, rng)
    rho = 10.0
    r = oracle.admm_solve(ph, par, Fbar3, rho, 1e-12, 400, model="linear")
    mu = r["mu_ref"]
    Eh = np.array([rho * rp ** 2 + mu ** 2 / rho * rd ** 2 for rp, rd, _ in r["history"]])
    assert np.all(Eh[1:] <= Eh[:-1] * (1 + 1e-9) + 1e-26)
    assert Eh[-1] < 1e-20 * max(Eh[0], 1.0) or r["converged"]


# ------------------------------------------------------------- P7: per-iteration invariants

def test_invariants_every_iteration():
    """Appendix argument and Step 3: after every exact projection D^T Lambda = 0;
    <W_F(F)> = <Lambda> (local solve exact); <G> = Fbar."""
    d, n = 3, 8
    ph = synth.inclusion_phase(n, d, 1, radius=2)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.diag([0.9, 1.0, 1.0])
    Fb = Fbar3.reshape((3, 3) + (1,) * d)
    state = None
    mat = make_material("neohookean", ph, par)
    for it in range(6):
        r = oracle.admm_solve(ph, par, Fbar3, 10.0, -1.0, 1, state=state)
        state = {"F": r["F"], "Lam": r["Lam"], "u": r["u"]}
        Lam = r["Lam"]
        div = E.div_stencil(Lam)
        assert np.max(np.abs(div)) <= 1e-12 * np.max(np.abs(Lam)) * n
        P = mat.P(oadmm._to_voxels(r["F"])).mean(axis=0)
        np.testing.assert_allclose(P, Lam.reshape(3, 3, -1).mean(axis=2), atol=1e-11)
        G = Fb + E.grad_stencil(r["u"])
        np.testing.assert_allclose(G.reshape(3, 3, -1).mean(axis=2), Fbar3, atol=1e-14)


def test_adaptive_rho_rule():
    """Penalty update (He-Yang-Wang, Section 2.1): rho grows by kappa while r_p/r_d > tau
    and shrinks (not below rho_min) while r_d/r_p > tau."""
    ph = synth.laminate_phase(16, 2)
    par = synth.two_phase_params(1.0, 10.0)
    r = oracle.admm_solve(ph, par, np.diag([1.05, 1.0, 1.0]), 100.0, 1e-10, 300,
                          rho_policy="adaptive", kappa=1.3, tau=10.0)
    assert r["converged"]
    hist = r["history"]
    for (rp, rd, rho), (_, _, rho_next) in zip(hist[:-1], hist[1:]):
        if rp / rd > 10.0:
            assert rho_next == pytest.approx(1.3 * rho, rel=1e-15)
        elif rd / rp > 10.0:
            assert rho_next == pytest.approx(max(rho / 1.3, r["mu_ref"]), rel=1e-15)
        else:
            assert rho_next == rho
    assert any(h[2] != 100.0 for h in hist)
