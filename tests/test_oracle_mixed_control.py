"""Pins of mixed macroscopic control in the oracle (Section 2.3: some components of
<F> prescribed, the complementary components of <S> zero; Section 5.3's UNI, PE
and EB protocols leave the free components of <F> to the minimisation).

Each pin holds the result to something other than the oracle: a scalar equation
solved by root finding for a homogeneous cell, and the effective stiffness of the
exact laminate (built from the independent closed form of the laminate pins)."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2010_06697_gb300 import synth
from tests.test_oracle_pins import _laminate_exact

UNI = np.ones((3, 3), bool)
UNI[0, 0] = False                      # <F_11> prescribed, all other components free
PE = np.ones((3, 3), bool)
PE[0, 0] = PE[0, 1] = PE[1, 1] = False  # <F_11>, <F_12>, <F_22> prescribed
EB = PE.copy()                          # same prescribed set, <F_22> = <F_11>


def test_homogeneous_uniaxial_stress_neohookean():
    """One phase, UNI at stretch 1.1: F = diag(s, t, t) with P_22 = 0, i.e.
    mu t + (lam J (J - 1) - mu) / t = 0 with J = s t^2 (compressible neo-Hookean)."""
    mu, lam, s = 1.0, 1.5, 1.1
    ph = np.zeros((6, 6, 6), np.uint8)
    par = np.array([[mu, lam]])
    t = brentq(lambda t: mu * t + (lam * s * t * t * (s * t * t - 1.0) - mu) / t, 0.5, 1.2)
    r = oracle.admm_solve(ph, par, np.diag([s, 1.0, 1.0]), 10.0, 1e-12, 500, free=UNI)
    assert r["converged"]
    np.testing.assert_allclose(r["Fbar"], np.diag([s, t, t]), atol=1e-10)
    J = s * t * t
    P11 = mu * s + (lam * J * (J - 1.0) - mu) / s
    want = np.diag([P11, 0.0, 0.0])
    np.testing.assert_allclose(r["stress"], want, atol=1e-10)


def _c_eff(par, d=3):
    """Effective stiffness of the linear laminate: columns S(I + E_kl) - S(I)."""
    S0 = _laminate_exact("linear", par, np.eye(d))[2]
    C = np.zeros((d * d, d * d))
    for q in range(d * d):
        E = np.zeros(d * d)
        E[q] = 1.0
        C[:, q] = (_laminate_exact("linear", par, np.eye(d) + E.reshape(d, d))[2] - S0).ravel()
    return C


# Linear elasticity gives skew <H> no stiffness, so a mask freeing both F_ij and F_ji
# leaves a rotation undetermined; these masks free one of each pair.
UNI_LIN = np.zeros((3, 3), bool)
UNI_LIN[1, 1] = UNI_LIN[2, 2] = True
PE_LIN = np.zeros((3, 3), bool)
PE_LIN[2, 2] = PE_LIN[0, 2] = PE_LIN[1, 2] = True


@pytest.mark.parametrize("mask", ["UNI", "PE"])
def test_linear_laminate_mixed_control(mask):
    """Two-phase linear laminate (normal e_1), free components from the mask: the
    converged <F> solves the effective relation S_free(<H>) = 0 and <S> = C_eff <H>."""
    free = {"UNI": UNI_LIN, "PE": PE_LIN}[mask]
    par = synth.two_phase_params(1.0, 10.0)
    ph = synth.laminate_phase(8, 3)
    C = _c_eff(par)
    h = np.zeros(9)
    h[0] = 0.04
    pres, fr = ~free.ravel(), free.ravel()
    h[fr] = -np.linalg.solve(C[np.ix_(fr, fr)], C[np.ix_(fr, pres)] @ h[pres])
    Fb = np.eye(3)
    Fb[0, 0] += 0.04
    r = oracle.admm_solve(ph, par, Fb, 10.0, 1e-12, 4000, model="linear", free=free)
    assert r["converged"]
    np.testing.assert_allclose(r["Fbar"], np.eye(3) + h.reshape(3, 3), atol=1e-9)
    np.testing.assert_allclose(r["stress"].ravel(), C @ h, atol=1e-9)


def test_free_mean_multiplier_vanishes_every_iteration():
    """<Lambda>_free = 0 after each multiplier update (Step 2's mean part), so the
    free stress components vanish at convergence; the prescribed ones are kept."""
    n = 8
    ph = synth.inclusion_phase(n, 3, 3, radius=2)
    par = synth.two_phase_params(1.0, 10.0)
    Fb = np.diag([1.08, 1.08, 1.0])
    for iters in (1, 2, 5):
        r = oracle.admm_solve(ph, par, Fb, 10.0, -1.0, iters, free=EB)
        lam_mean = r["Lam"].reshape(3, 3, -1).mean(axis=2)
        assert np.max(np.abs(lam_mean[EB])) < 1e-12
        assert r["Fbar"][0, 0] == 1.08 and r["Fbar"][1, 1] == 1.08 and r["Fbar"][0, 1] == 0.0
    r = oracle.admm_solve(ph, par, Fb, 10.0, 1e-10, 2000, free=EB)
    assert r["converged"]
    assert np.max(np.abs(r["stress"][EB])) < 1e-8
    assert r["Fbar"][2, 2] < 1.0  # the sheet thins under equi-biaxial extension
