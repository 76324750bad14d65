"""Pins of the inexact local step (Section 2.1, "Approximate solution of the local
problem"; Section 4.2, second strategy r_l <= f r_d) in the oracle.

The pins do not compare the oracle with itself only: the converged stress is held to
the closed-form laminate solutions (linear and neo-Hookean), which an inexact local
step must still reach because r_l -> 0 with r_d (the appendix bound on the
equilibrium error by the local and global residuals)."""
import numpy as np
import pytest

import oracle
from oracle import admm as oadmm
from paper_2010_06697_gb300 import synth
from tests.test_oracle_pins import _laminate_exact, _near_identity


@pytest.mark.parametrize("model,d,n", [("linear", 2, 16), ("neohookean", 3, 8)])
def test_inexact_local_steps_reach_laminate_closed_form(model, d, n):
    rng = np.random.default_rng(5)
    ph = synth.laminate_phase(n, d)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.eye(3)
    Fbar3[:d, :d] = _near_identity(d, 0.06, rng)
    _, _, S = _laminate_exact(model, par, Fbar3[:d, :d])
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, 1e-12, 3000, model=model, local_ratio=0.3)
    assert r["converged"]
    np.testing.assert_allclose(r["stress"], S, atol=1e-9)


def test_local_residual_bound_and_lag():
    """r_l of iteration i is at most f r_d of iteration i - 2 (the tolerance each
    voxel's Newton stops at, in the pointwise form); the first two iterations are
    exact local solves (r_l at the Newton floor)."""
    n, f = 10, 0.3
    ph = synth.inclusion_phase(n, 3, 1, radius=2)
    par = synth.two_phase_params(1.0, 10.0)
    r = oracle.admm_solve(ph, par, np.diag([0.92, 1.0, 1.03]), 10.0, 1e-9, 300, local_ratio=f)
    assert r["converged"]
    rd = np.array(r["history"])[:, 1]
    rl = np.array(r["local_residual"])
    assert rl[0] < 1e-9 and rl[1] < 1e-9
    assert np.all(rl[2:] <= f * rd[:-2] * (1 + 1e-12))
    # the relaxation is used: early local residuals are far above the exact floor
    assert np.max(rl[2:10]) > 1e-6


def test_local_residual_definition():
    """local_residual is the unit-cell L2 norm of W_F(F) - Lambda + rho (F - G) over
    mu_ref: an exact local minimiser gives ~0, a displaced F gives the norm of the
    gradient change, which for the linear law is (C + rho I) dF exactly."""
    n, d, rho, mu_ref = 6, 2, 7.0, 2.0
    ph = synth.laminate_phase(n, d)
    par = synth.two_phase_params(1.0, 10.0)
    mat = oracle.make_material("linear", ph, par)
    V = n ** d
    rng = np.random.default_rng(3)
    G = np.eye(d)[None] + 0.05 * rng.standard_normal((V, d, d))
    Lam = 0.1 * rng.standard_normal((V, d, d))
    F, _ = oadmm.local_newton(mat, G.copy(), Lam, G, rho)
    assert oadmm.local_residual(mat, F, Lam, G, rho, mu_ref) < 1e-12
    dF = 1e-3 * rng.standard_normal((V, d, d))
    mu = mat.mu.reshape(-1, 1, 1)
    lam = mat.lam.reshape(-1, 1, 1)
    tr = np.trace(dF, axis1=1, axis2=2).reshape(-1, 1, 1)
    dg = mu * (dF + dF.transpose(0, 2, 1)) + lam * tr * np.eye(d)[None] + rho * dF
    want = np.sqrt(np.mean(np.sum(dg * dg, axis=(1, 2)))) / mu_ref
    got = oadmm.local_residual(mat, F + dF, Lam, G, rho, mu_ref)
    assert abs(got - want) < 1e-9 * want


# ------------------------------------------------------------------ fraction-converged local steps

def test_fraction_cap_rule():
    """The cap rule on hand-counted Newton counts: bins of 2 iterations, cumulative."""
    iters = np.array([1, 1, 2, 3, 5, 7])
    conv = np.ones(6, bool)
    assert oadmm.fraction_cap(iters, conv, 0.5, 30, 30) == 2     # 3 of 6 within 2
    assert oadmm.fraction_cap(iters, conv, 0.8, 30, 30) == 6     # 5 of 6 within 6 (need 4.8)
    assert oadmm.fraction_cap(iters, conv, 1.0, 30, 30) == 8
    conv[5] = False                                               # the 7-step voxel hit the cap
    assert oadmm.fraction_cap(iters, conv, 0.9, 8, 30) == 10      # only 5 of 6 converged: cap + 2
    assert oadmm.fraction_cap(iters, conv, 0.9, 30, 30) == 30     # never above the configured cap


@pytest.mark.parametrize("model,d,n", [("linear", 2, 16), ("neohookean", 3, 8)])
def test_fraction_converged_steps_reach_laminate_closed_form(model, d, n):
    rng = np.random.default_rng(6)
    ph = synth.laminate_phase(n, d)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.eye(3)
    Fbar3[:d, :d] = _near_identity(d, 0.06, rng)
    _, _, S = _laminate_exact(model, par, Fbar3[:d, :d])
    r = oracle.admm_solve(ph, par, Fbar3, 10.0, 1e-12, 3000, model=model, local_fraction=0.5)
    assert r["converged"]
    np.testing.assert_allclose(r["stress"], S, atol=1e-9)
    caps = np.array(r["newton_caps"])
    assert caps[0] == caps[1] == 50 and np.all(caps >= 2) and np.all(caps % 2 == 0)
