"""Mixed macroscopic control (rve_solve_mixed; Section 2.3 and the UNI / PE / EB
loadings of Section 5.3) on the GPU vs the FP64 oracle."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
PAR = synth.two_phase_params(1.0, 10.0)
UNI = np.ones((3, 3), bool)
UNI[0, 0] = False
PE = np.ones((3, 3), bool)
PE[0, 0] = PE[0, 1] = PE[1, 1] = False
EB = PE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def make(ph, precision="fp64", model="neohookean", par=PAR, n0=None, **opt):
    s = rve.Rve(ph.ndim, ph.shape[0], model, precision, **opt)
    s.set_material(ph, par, n0)
    return s


@pytest.mark.parametrize("mask_name,d,n", [("EB", 3, 12), ("UNI", 3, 16), ("PE2", 2, 24)])
def test_mixed_control_iterations_match_oracle(mask_name, d, n):
    if mask_name == "PE2":
        free = np.zeros((3, 3), bool)
        free[1, 1] = free[1, 0] = True
        Fbar = np.diag([1.06, 1.0, 1.0])
    else:
        free = {"EB": EB, "UNI": UNI}[mask_name]
        Fbar = np.diag([1.07, 1.07 if mask_name == "EB" else 1.0, 1.0])
    ph = synth.inclusion_phase(n, d, 5, radius=max(2, n // 6))
    s = make(ph, max_iter=6)
    info = s.solve(Fbar, 8.0, -1.0, free=free)
    ref = oracle.admm_solve(ph, PAR, Fbar, 8.0, -1.0, 6, free=free)
    assert info.iterations == 6
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert np.max(np.abs(st["u"] - ref["u"])) < TOL64
    assert np.max(np.abs(s.macro_gradient() - ref["Fbar"])) < 1e-12
    np.testing.assert_allclose(s.history()[:, :2], np.array(ref["history"])[:, :2], rtol=1e-9, atol=1e-14)
    assert rel(s.stress(), ref["stress"]) < TOL64


def test_uniaxial_stress_homogeneous_closed_form():
    """One neo-Hookean phase under UNI: <F> = diag(s, t, t) with P_22(t) = 0."""
    mu, lam, sx = 1.0, 1.5, 1.1
    ph = np.zeros((8, 8, 8), np.uint8)
    s = make(ph, par=np.array([[mu, lam]]), max_iter=500)
    info = s.solve(np.diag([sx, 1.0, 1.0]), 10.0, 1e-12, free=UNI)
    assert info.converged
    t = brentq(lambda t: mu * t + (lam * sx * t * t * (sx * t * t - 1.0) - mu) / t, 0.5, 1.2)
    np.testing.assert_allclose(s.macro_gradient(), np.diag([sx, t, t]), atol=1e-10)
    S = s.stress()
    assert np.max(np.abs(S[UNI])) < 1e-10


def test_mixed_precision_plane_stress_converges():
    """PE on a 32^3 inclusion cell in mixed precision: the free stress components
    vanish and <F> matches the FP64 solve."""
    ph = synth.inclusion_phase(32, 3, 0)
    Fbar = np.diag([1.08, 1.0, 1.0])
    s64 = make(ph, max_iter=2000)
    i64 = s64.solve(Fbar, 10.0, 1e-8, free=PE)
    smx = make(ph, precision="mixed", max_iter=2000)
    imx = smx.solve(Fbar, 10.0, 1e-8, free=PE)
    assert i64.converged and imx.converged
    S = smx.stress()
    assert np.max(np.abs(S[PE])) < 1e-6 * abs(S[0, 0])
    assert np.max(np.abs(smx.macro_gradient() - s64.macro_gradient())) < 1e-7


def test_mask_then_plain_solve_reuses_graphs_correctly():
    """A mixed-control solve, then a plain solve on the same handle from a reset
    state: the second equals a fresh handle's plain solve bit for bit."""
    ph = synth.inclusion_phase(16, 3, 2, radius=2)
    Fbar = np.diag([0.95, 1.0, 1.0])
    a = make(ph, max_iter=40)
    a.solve(Fbar, 10.0, -1.0, free=UNI)
    a.reset()
    a.solve(Fbar, 10.0, -1.0)
    b = make(ph, max_iter=40)
    b.solve(Fbar, 10.0, -1.0)
    for k in ("F", "Lam", "u"):
        assert np.array_equal(a.state()[k], b.state()[k])
    assert np.array_equal(a.macro_gradient(), Fbar)


def test_mask_outside_2d_block_rejected():
    ph = synth.laminate_phase(16, 2)
    s = make(ph, max_iter=5)
    free = np.zeros((3, 3), bool)
    free[2, 2] = True
    rc, _ = rve.rve_solve_mixed(s.h, np.eye(3), free, 10.0, 1e-8)
    assert rc == rve.RVE_E_INVALID_ARG


def test_lce_plane_stress_matches_oracle():
    """LCE cell under PE (the polydomain protocol), fixed iteration count."""
    n = 12
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 3, corr=2.5)
    par = np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2]])
    Fbar = np.diag([1.1, 1.0, 1.0])
    s = make(ph, model="lce", par=par, n0=n0, max_iter=8)
    s.solve(Fbar, 10.0, -1.0, free=PE)
    ref = oracle.admm_solve(ph, par, Fbar, 10.0, -1.0, 8, model="lce", n0=n0, free=PE)
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert np.max(np.abs(s.macro_gradient() - ref["Fbar"])) < 1e-12
