"""The mixed-precision modes of the LCE (Section 5.1) and Bloch-wave (Section 2.4)
paths against the FP64 oracle itself (not only against the GPU's FP64 path), and
the 256^3 LCE workload's first iteration at sampled voxels.

Mixed mode runs the bulk of the iteration in float; after a fixed number of
iterations its fields differ from the FP64 oracle's by float rounding carried
through the iteration.  The tolerances below are the stated per-field tolerances
of the mixed modes (relative to each field's largest entry; stress relative):
F, Lambda 2e-5, directors 2e-5 absolute, stress 2e-5 for the LCE after 6
iterations; p 1e-4 and sigma 1e-5 for the float phase of the Bloch iteration."""
import numpy as np
import pytest

import oracle
from oracle import admm as oadmm
from oracle import bloch
from paper_2010_06697_gb300 import build, rve, synth

from .test_oracle_bloch import near_identity_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def lce_params(n):
    return np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2]])


def test_lce_mixed_matches_oracle_32():
    """32^3 polydomain cell (the 256^3 workload's constants), 6 iterations in the
    float bulk of RVE_MIXED against the FP64 oracle."""
    n, iters = 32, 6
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 2, corr=4.0)
    par = lce_params(n)
    Fbar = np.diag([1.2, 0.91, 0.91])
    s = rve.Rve(3, n, "lce", "mixed", max_iter=iters)
    s.set_material(ph, par, n0)
    info = s.solve(Fbar, 10.0, -1.0)
    assert info.iterations == iters and info.fp64_iterations == 0
    ref = oracle.admm_solve(ph, par, Fbar, 10.0, -1.0, iters, model="lce", n0=n0)
    st = s.state()
    errs = {"F": rel(st["F"], ref["F"]), "Lam": rel(st["Lam"], ref["Lam"]),
            "n": float(np.max(np.abs(st["n"] - ref["n"]))), "S": rel(s.stress(), ref["stress"])}
    assert errs["F"] < 2e-5 and errs["Lam"] < 2e-5 and errs["n"] < 2e-5 and errs["S"] < 2e-5, errs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_lce256_first_iteration_sampled(precision, tol):
    """The 256^3 LCE workload (bench launch shape, 16.8M voxels), one iteration: at
    2048 sampled voxels F_1 and n_1 equal the oracle's local solve (local_newton_lce)
    from the inputs alone -- F_0 = Fbar, Lambda_0 = W_F(Fbar; n_0), G_0 = Fbar and the
    explicit Frank force of n_0 (oracle.frank_force on the whole field)."""
    n = 256
    ph = np.zeros((n,) * 3, np.uint8)
    n0 = synth.director_grf(n, 0, corr=8.0)
    par = lce_params(n)
    Fbar = np.diag([1.2, 0.91, 0.91])
    s = rve.Rve(3, n, "lce", precision, max_iter=1)
    s.set_material(ph, par, n0)
    info = s.solve(Fbar, 10.0, -1.0)
    assert info.iterations == 1
    V = ph.size
    rng = np.random.default_rng(8)
    idx = rng.choice(V, 2048, replace=False)
    mat = oracle.make_lce(ph.reshape(-1)[idx], par, n0.reshape(3, -1)[:, idx])
    force = oadmm.frank_force(n0, np.full(V, par[0, 4]))[idx]
    n0s = n0.reshape(3, -1)[:, idx].T.copy()
    F0 = np.broadcast_to(Fbar, (idx.size, 3, 3)).copy()
    Lam0 = mat.P(F0, n0s)
    F1, n1, _ = oadmm.local_newton_lce(mat, F0, n0s, Lam0, F0.copy(), force, 10.0)
    Fg = s.get_field(rve.RVE_FIELD_F).reshape(9, V)[:, idx].T.reshape(-1, 3, 3)
    ng = s.get_field(rve.RVE_FIELD_N).reshape(3, V)[:, idx].T
    s.close()
    assert rel(Fg, F1) < tol, rel(Fg, F1)
    assert np.max(np.abs(ng - n1)) < tol, np.max(np.abs(ng - n1))


@pytest.mark.parametrize("d,n,k,iters", [(2, 64, (3, 4), 12), (3, 24, (2, 3, -4), 8)])
def test_bloch_float_phase_matches_oracle(d, n, k, iters):
    """RVE_FP32 (the float phase of the mixed Bloch iteration alone) after a fixed
    number of iterations against the FP64 oracle: p element by element and sigma."""
    ph = synth.inclusion_phase(n, d, 3, radius=max(1, n // 8))
    par = synth.two_phase_params(1.0, 4.0)
    F = near_identity_field(n, d, 5).astype(np.float32).astype(np.float64)
    p0 = synth.bloch_start(n, d, 11)
    s = rve.Rve(d, n, "neohookean", "fp32", max_iter=10)
    s.set_material(ph, par)
    s.set_field(rve.RVE_FIELD_F, F)
    rc, info, p, hist = rve.rve_bloch(s.h, k, p0, 10.0, -1.0, iters)
    assert info.iterations == iters and info.float_iterations == iters
    mu_ref = float(np.mean(par[ph.reshape(-1), 0]))
    ref = bloch.bloch_solve(bloch.tangent_field("neohookean", ph, par, F), p0, k, 10.0, -1.0, iters, mu_ref)
    assert rel(p, ref["p"]) < 1e-4, rel(p, ref["p"])
    assert abs(info.beta - ref["sigma"]) < 1e-5 * abs(ref["sigma"]), (info.beta, ref["sigma"])
