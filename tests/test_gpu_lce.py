"""Liquid crystal elastomer cells (Section 5.1) on the GPU vs the FP64 oracle.

The polydomain relaxation with the explicit Frank term is not run to a tolerance
(its residuals plateau while domains evolve); parity is checked element by element
after fixed iteration counts, plus the exact cases (ground state, neo-Hookean
reduction)."""
import numpy as np
import pytest

import oracle
from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
FBAR = np.diag([1.2, 0.91, 0.91])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def lce_params(n, r=7.71, alpha=0.06, wall=2.0):
    return np.array([[1.0, 20.0, r, alpha, (wall / n) ** 2]])


def run_gpu(ph, par, n0, Fbar, rho, tol, iters, precision="fp64", **opt):
    s = rve.Rve(3, ph.shape[0], "lce", precision, max_iter=iters, **opt)
    s.set_material(ph, par, n0)
    info = s.solve(Fbar, rho, tol)
    return s, info


@pytest.mark.parametrize("n,iters", [(8, 3), (12, 6), (16, 4)])
def test_lce_iterations_match_oracle(n, iters):
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, n, corr=3.0)
    par = lce_params(n)
    s, info = run_gpu(ph, par, n0, FBAR, 10.0, -1.0, iters)
    ref = oracle.admm_solve(ph, par, FBAR, 10.0, -1.0, iters, model="lce", n0=n0)
    assert info.iterations == iters
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert np.max(np.abs(st["u"] - ref["u"])) < TOL64
    np.testing.assert_allclose(s.history()[:, :2], np.array(ref["history"])[:, :2], rtol=1e-8, atol=1e-13)
    assert rel(s.stress(), ref["stress"]) < TOL64


def test_lce_two_phase_cell_matches_oracle():
    """Two LCE phases with different r, alpha, kappa on an inclusion map."""
    n = 12
    ph = synth.inclusion_phase(n, 3, 4, radius=2)
    n0 = synth.director_grf(n, 21, corr=2.5)
    par = np.array([[1.0, 20.0, 4.0, 0.1, 0.02], [2.0, 30.0, 2.0, 0.05, 0.01]])
    s, info = run_gpu(ph, par, n0, np.diag([1.1, 0.95, 0.97]), 10.0, -1.0, 5)
    ref = oracle.admm_solve(ph, par, np.diag([1.1, 0.95, 0.97]), 10.0, -1.0, 5, model="lce", n0=n0)
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert rel(s.stress(), ref["stress"]) < TOL64


def test_lce_ground_state_on_gpu():
    n = 8
    e = np.array([0.6, 0.8, 0.0])
    r = 7.71
    ell = r ** (-1 / 3) * (np.eye(3) + (r - 1) * np.outer(e, e))
    w, Q = np.linalg.eigh(ell)
    Fg = Q @ np.diag(np.sqrt(w)) @ Q.T
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.broadcast_to(e[:, None, None, None], (3, n, n, n)).copy()
    s, info = run_gpu(ph, lce_params(n), n0, Fg, 10.0, 1e-12, 5)
    assert info.converged and info.iterations == 1
    assert np.max(np.abs(s.stress())) < 1e-12


def test_lce_reduces_to_neohookean_on_gpu():
    n = 12
    ph = synth.inclusion_phase(n, 3, 2, radius=2)
    nh = synth.two_phase_params(1.0, 10.0)
    par = np.column_stack([nh, np.ones(2), np.zeros(2), np.zeros(2)])
    n0 = synth.director_grf(n, 3, corr=2.0)
    Fbar = np.diag([0.95, 1.02, 1.0])
    s, _ = run_gpu(ph, par, n0, Fbar, 10.0, -1.0, 6)
    a = rve.Rve(3, n, "neohookean", "fp64", max_iter=6)
    a.set_material(ph, nh)
    a.solve(Fbar, 10.0, -1.0)
    assert rel(s.get_field(rve.RVE_FIELD_F), a.get_field(rve.RVE_FIELD_F)) < 1e-12
    assert rel(s.stress(), a.stress()) < 1e-12


def test_lce_mixed_precision_tracks_fp64():
    """Float bulk (residuals in double): after 20 iterations the stress is within
    1e-4 of the FP64 path's."""
    n = 16
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 5, corr=3.0)
    par = lce_params(n)
    s64, _ = run_gpu(ph, par, n0, FBAR, 10.0, -1.0, 20)
    s32, info = run_gpu(ph, par, n0, FBAR, 10.0, -1.0, 20, precision="mixed")
    assert info.iterations == 20
    assert rel(s32.stress(), s64.stress()) < 1e-4
    n32 = s32.get_field(rve.RVE_FIELD_N)
    assert np.max(np.abs(np.sum(n32 ** 2, axis=0) - 1.0)) < 1e-5


# ------------------------------------------------------------------ time steps and loading paths

def lce_params_dt(n, cF=5.6, cn=0.0106):
    """Polydomain constants with Section 5.3's viscosities over its time step, normalised
    by mu: nu_F/(mu dt) = 2.65/23.63/0.02 = 5.6, nu_n/(mu dt) = 0.005/23.63/0.02 = 0.0106."""
    return np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2, cF, cn]])


def test_lce_time_step_matches_oracle():
    """One time step with dissipation from a warm state, fixed iteration count,
    element by element against the oracle (FP64)."""
    n = 12
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 9, corr=2.5)
    par = lce_params_dt(n)
    s, _ = run_gpu(ph, par, n0, FBAR, 10.0, -1.0, 5)
    warm = s.state()
    ref0 = oracle.admm_solve(ph, par, FBAR, 10.0, -1.0, 5, model="lce", n0=n0)
    F2 = FBAR.copy()
    F2[0, 0] += 0.02
    s.solve(F2, 10.0, -1.0)
    st = s.state()
    ref = oracle.admm_solve(ph, par, F2, 10.0, -1.0, 5, model="lce", n0=n0,
                            state={"F": ref0["F"], "Lam": ref0["Lam"], "u": ref0["u"], "n": ref0["n"]})
    assert rel(warm["F"], ref0["F"]) < TOL64
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert rel(s.stress(), ref["stress"]) < TOL64


def test_lce_plane_stress_path_matches_oracle():
    """A 3-step PE loading path (Section 5.3: <F_11> rising, <F_12> = 0, <F_22> = 1,
    the rest free) with dissipation through rve_solve_path, against the oracle's steps
    run one after another from each other's states: <S> and <F> of every step."""
    n = 12
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 10, corr=2.5)
    par = lce_params_dt(n)
    free = np.ones((3, 3), bool)
    free[0, 0] = free[0, 1] = free[1, 1] = False
    lam = [1.02, 1.04, 1.06]
    Fbars = np.stack([np.diag([l, 1.0, 1.0]) for l in lam])
    s = rve.Rve(3, n, "lce", "fp64", max_iter=6)
    s.set_material(ph, par, n0)
    S, Fo, infos = s.solve_path(Fbars, 10.0, -1.0, free=free)
    state, Fprev = None, None
    for k in range(3):
        Fb = Fbars[k].copy()
        if Fprev is not None:
            Fb[free] = Fprev[free]
        r = oracle.admm_solve(ph, par, Fb, 10.0, -1.0, 6, model="lce", n0=n0, free=free, state=state)
        state = {"F": r["F"], "Lam": r["Lam"], "u": r["u"], "n": r["n"]}
        Fprev = r["Fbar"]
        assert infos[k].iterations == 6
        assert rel(S[k], r["stress"]) < 1e-9
        assert np.max(np.abs(Fo[k] - r["Fbar"])) < 1e-11


# ------------------------------------------------------------------ incompressible network

def inc_params(n, r=4.0, alpha=0.1, wall=2.0, cF=0.0, cn=0.0):
    """Eighth entry 1: det F = 1 by the local step's multiplier (lambda unused)."""
    return np.array([[1.0, 0.0, r, alpha, (wall / n) ** 2, cF, cn, 1.0]])


def isochoric(s):
    return np.diag([s, s ** -0.5, s ** -0.5])


@pytest.mark.parametrize("n,iters,seed,cF,cn", [(8, 3, 13, 0.0, 0.0), (12, 5, 17, 0.0, 0.0),
                                                (12, 4, 9, 5.6, 0.0106)])
def test_incompressible_iterations_match_oracle(n, iters, seed, cF, cn):
    """Polydomain incompressible cell (with and without the dissipation terms), fixed
    iteration count, element by element against the oracle's KKT local step; every
    voxel's det F is 1 after each local step."""
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, seed, corr=3.0)
    par = inc_params(n, cF=cF, cn=cn)
    Fb = isochoric(1.1)
    s, info = run_gpu(ph, par, n0, Fb, 10.0, -1.0, iters)
    ref = oracle.admm_solve(ph, par, Fb, 10.0, -1.0, iters, model="lce", n0=n0, incompressible=True)
    assert info.iterations == iters
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert np.max(np.abs(st["u"] - ref["u"])) < TOL64
    np.testing.assert_allclose(s.history()[:, :2], np.array(ref["history"])[:, :2], rtol=1e-8, atol=1e-13)
    assert rel(s.stress(), ref["stress"]) < TOL64
    F = st["F"].reshape(9, -1).T.reshape(-1, 3, 3)
    assert np.max(np.abs(np.linalg.det(F) - 1.0)) < 1e-9


def test_incompressible_uniaxial_stress_on_gpu():
    """r = 1, alpha = 0: incompressible neo-Hookean.  Uniaxial stress by mixed control
    (<F_11> = s, the rest free): <F> = diag(s, s^-1/2, s^-1/2), <S_11> = mu (s - s^-2),
    every other component 0."""
    n, mu, s = 8, 1.0, 1.15
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = np.broadcast_to(np.array([0.0, 1.0, 0.0]).reshape(3, 1, 1, 1), (3, n, n, n)).copy()
    par = np.array([[mu, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    free = np.ones((3, 3), bool)
    free[0, 0] = False
    a = rve.Rve(3, n, "lce", "fp64", max_iter=3000)
    a.set_material(ph, par, n0)
    info = a.solve(np.diag([s, 1.0, 1.0]), 10.0, 1e-11, free=free)
    assert info.converged
    q = s ** -0.5
    np.testing.assert_allclose(a.macro_gradient(), np.diag([s, q, q]), atol=1e-9)
    np.testing.assert_allclose(a.stress(), np.diag([mu * (s - s ** -2), 0.0, 0.0]), atol=1e-9)


def test_incompressible_two_phase_matches_oracle():
    """Two incompressible phases with different r, alpha, kappa on an inclusion map."""
    n = 12
    ph = synth.inclusion_phase(n, 3, 4, radius=2)
    n0 = synth.director_grf(n, 21, corr=2.5)
    par = np.array([[1.0, 0.0, 4.0, 0.1, 0.02, 0.0, 0.0, 1.0], [2.0, 0.0, 2.0, 0.05, 0.01, 0.0, 0.0, 1.0]])
    Fb = isochoric(1.08)
    s, info = run_gpu(ph, par, n0, Fb, 10.0, -1.0, 5)
    ref = oracle.admm_solve(ph, par, Fb, 10.0, -1.0, 5, model="lce", n0=n0, incompressible=True)
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert np.max(np.abs(st["n"] - ref["n"])) < TOL64
    assert rel(s.stress(), ref["stress"]) < TOL64


def test_incompressible_mixed_precision_tracks_fp64():
    n = 16
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 5, corr=3.0)
    par = inc_params(n, r=7.71, alpha=0.06)
    Fb = isochoric(1.2)
    s64, _ = run_gpu(ph, par, n0, Fb, 10.0, -1.0, 20)
    s32, info = run_gpu(ph, par, n0, Fb, 10.0, -1.0, 20, precision="mixed")
    assert info.iterations == 20
    assert rel(s32.stress(), s64.stress()) < 1e-4


def test_incompressible_flag_checked():
    """The flag is 0 or 1 and the same in every phase."""
    n = 8
    ph = synth.inclusion_phase(n, 3, 4, radius=2)
    n0 = synth.director_grf(n, 21, corr=2.5)
    a = rve.Rve(3, n, "lce", "fp64", max_iter=5)
    bad_mix = np.array([[1.0, 0.0, 4.0, 0.1, 0.02, 0.0, 0.0, 1.0], [2.0, 0.0, 2.0, 0.05, 0.01, 0.0, 0.0, 0.0]])
    bad_val = np.array([[1.0, 0.0, 4.0, 0.1, 0.02, 0.0, 0.0, 0.5]] * 2)
    for par in (bad_mix, bad_val):
        with pytest.raises(rve.RveError):
            a.set_material(ph, par, n0)


def test_lce_plane_stress_path_mixed_tracks_fp64():
    """The same 3-step PE path with dissipation in the mixed scheme: <S> and <F> of every
    step within 1e-4 of the FP64 path (float bulk, fixed iteration counts)."""
    n = 12
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 10, corr=2.5)
    par = lce_params_dt(n)
    free = np.ones((3, 3), bool)
    free[0, 0] = free[0, 1] = free[1, 1] = False
    Fbars = np.stack([np.diag([l, 1.0, 1.0]) for l in (1.02, 1.04, 1.06)])
    out = {}
    for prec in ("fp64", "mixed"):
        s = rve.Rve(3, n, "lce", prec, max_iter=12)
        s.set_material(ph, par, n0)
        out[prec] = s.solve_path(Fbars, 10.0, -1.0, free=free)
    S64, F64, _ = out["fp64"]
    S32, F32, _ = out["mixed"]
    assert np.max(np.abs(S32 - S64)) < 1e-4 * max(1.0, np.max(np.abs(S64)))
    assert np.max(np.abs(F32 - F64)) < 1e-4
