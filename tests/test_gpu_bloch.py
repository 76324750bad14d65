"""Bloch-wave ADMM (Section 2.4) on the GPU vs the FP64 oracle: element-wise parity
after fixed iteration counts, converged beta_k against the oracle and the dense
eigenvalue, closed forms, argument and state checks."""
import numpy as np
import pytest

from oracle import bloch
from paper_2010_06697_gb300 import build, rve, synth

from .test_oracle_bloch import dense_beta, near_identity_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def handle_with_state(d, n, model, ph, par, F):
    s = rve.Rve(d, n, model, "fp64", max_iter=10)
    s.set_material(ph, par)
    s.set_field(rve.RVE_FIELD_F, F)
    return s


def two_phase_case(d, n, seed=5):
    ph = synth.inclusion_phase(n, d, 3, radius=max(1, n // 8))
    par = synth.two_phase_params(1.0, 4.0)
    F = near_identity_field(n, d, seed)
    return ph, par, F


@pytest.mark.parametrize("d,n,k,iters", [(2, 12, (3, 4), 7), (2, 18, (2, -3), 5), (3, 8, (2, 3, -4), 4),
                                         (3, 6, (2, 1, 1), 3)])
def test_bloch_iterations_match_oracle(d, n, k, iters):
    ph, par, F = two_phase_case(d, n)
    mu_ref = float(np.mean(par[ph.reshape(-1), 0]))
    p0 = synth.bloch_start(n, d, 11)
    s = handle_with_state(d, n, "neohookean", ph, par, F)
    info, p, hist = s.bloch(k, 10.0, -1.0, iters, p0=p0)
    L = bloch.tangent_field("neohookean", ph, par, F)
    ref = bloch.bloch_solve(L, p0, k, 10.0, -1.0, iters, mu_ref)
    assert info.iterations == iters
    assert rel(p, ref["p"]) < 1e-10
    np.testing.assert_allclose(info.beta, ref["sigma"], rtol=1e-11)
    np.testing.assert_allclose(hist[:, :2], np.array(ref["history"]), rtol=1e-8, atol=1e-13)
    np.testing.assert_allclose(np.sum(np.abs(p) ** 2) / n ** d, 1.0, rtol=1e-12)


@pytest.mark.parametrize("d,n,k", [(2, 6, (3, -2)), (2, 6, (2, 1)), (3, 4, (2, 3, 1))])
def test_bloch_converged_beta_is_smallest_eigenvalue(d, n, k):
    ph = synth.inclusion_phase(n, d, 3, radius=1)
    par = synth.two_phase_params(1.0, 4.0)
    F = near_identity_field(n, d, 5)
    L = bloch.tangent_field("neohookean", ph, par, F)
    w, _, _ = dense_beta(L, n, d, k)
    s = handle_with_state(d, n, "neohookean", ph, par, F)
    info, p, _ = s.bloch(k, 10.0, 1e-10, 20000, p0=synth.bloch_start(n, d, 1))
    assert info.converged
    np.testing.assert_allclose(info.beta, w[0], rtol=1e-9)
    np.testing.assert_allclose(info.rayleigh, w[0], rtol=1e-9)


@pytest.mark.parametrize("d,n,k", [(2, 64, (2, 2)), (2, 48, (3, -5)), (3, 24, (2, 2, 3))])
def test_bloch_homogeneous_linear_closed_form(d, n, k):
    """Homogeneous isotropic linear elasticity: plane waves are eigenvectors with
    eigenvalues mu |q|^2 and (lam + 2 mu) |q|^2, q_j = N sin(2 pi (m_j + 1/k_j) / N),
    so beta_k = mu min_m |q(m)|^2."""
    mu, lam = 1.0, 1.5
    ph = np.zeros((n,) * d, np.uint8)
    F = np.broadcast_to(np.eye(d).reshape((d, d) + (1,) * d), (d, d) + (n,) * d).copy()
    s = handle_with_state(d, n, "linear", ph, np.array([[mu, lam]]), F)
    info, p, _ = s.bloch(k, 4.0, 1e-10, 20000, seed=3)
    m = np.arange(n)
    qmin = sum(np.min((n * np.sin(2 * np.pi * (m + 1.0 / k[j]) / n)) ** 2) for j in range(d))
    assert info.converged
    np.testing.assert_allclose(info.beta, mu * qmin, rtol=1e-9)
    np.testing.assert_allclose(info.rayleigh, mu * qmin, rtol=1e-9)


def test_bloch_after_solve_uses_resident_state():
    """beta_k of an equilibrium state from rve_solve (compressed two-phase cell) equals
    the oracle's beta for the same F field read back from the handle."""
    d, n, k = 2, 24, (2, 2)
    ph = synth.inclusion_phase(n, d, 7, radius=4)
    par = synth.two_phase_params(20.0, 1.0)
    s = rve.Rve(d, n, "neohookean", "fp64", max_iter=3000)
    s.set_material(ph, par)
    s.solve(np.diag([0.95, 0.95, 1.0]), 10.0, 1e-9)
    F = s.get_field(rve.RVE_FIELD_F)
    info, p, _ = s.bloch(k, 60.0, -1.0, 6, seed=2)
    mu_ref = float(np.mean(par[ph.reshape(-1), 0]))
    ref = bloch.bloch_solve(bloch.tangent_field("neohookean", ph, par, F), synth.bloch_start(n, d, 2), k, 60.0,
                            -1.0, 6, mu_ref)
    assert rel(p, ref["p"]) < 1e-10
    np.testing.assert_allclose(info.beta, ref["sigma"], rtol=1e-11)


def test_bloch_arguments_and_state_checked():
    d, n = 2, 8
    ph, par, F = two_phase_case(d, n)
    s = rve.Rve(d, n, "neohookean", "fp64", max_iter=10)
    s.set_material(ph, par)
    p0 = synth.bloch_start(n, d, 0)
    rc, *_ = rve.rve_bloch(s.h, (2, 2), p0, 10.0, 1e-8, 10)
    assert rc == rve.RVE_E_STATE  # no state yet
    s.set_field(rve.RVE_FIELD_F, F)
    for k in ((1, 1), (1, -1), (0, 2)):
        rc, *_ = rve.rve_bloch(s.h, k, p0, 10.0, 1e-8, 10)
        assert rc == rve.RVE_E_INVALID_ARG
    rc, *_ = rve.rve_bloch(s.h, (2, 2), np.zeros_like(p0), 10.0, 1e-8, 10)
    assert rc == rve.RVE_E_INVALID_ARG
    rc, *_ = rve.rve_bloch(s.h, (2, 2), p0, -1.0, 1e-8, 10)
    assert rc == rve.RVE_E_INVALID_ARG


def test_bloch_indefinite_tangent_reported():
    """A tangent with a negative eigenvalue below -rho makes L + rho I indefinite:
    RVE_E_NUMERICAL, no iterations."""
    d, n = 2, 8
    ph = np.zeros((n,) * d, np.uint8)
    par = np.array([[1.0, 50.0]])
    Fh = np.diag([0.35, 0.35])
    C = bloch.tangent_field("neohookean", np.zeros((1, 1), np.uint8), par, Fh.reshape(2, 2, 1, 1))[0]
    lam_min = np.linalg.eigvalsh(C.reshape(4, 4))[0]
    assert lam_min < -1.0  # the precondition, from the oracle's tangent
    F = np.broadcast_to(Fh.reshape(2, 2, 1, 1), (2, 2, n, n)).copy()
    s = handle_with_state(d, n, "neohookean", ph, par, F)
    rc, info, _, _ = rve.rve_bloch(s.h, (2, 2), synth.bloch_start(n, d, 0), 0.5 * abs(lam_min), 1e-8, 10)
    assert rc == rve.RVE_E_NUMERICAL


def test_beta22_changes_sign_under_compression():
    """Section 4.3's qualitative result on a synthetic cell (one soft disc, radius 0.4,
    mu_m / mu_i = 20, kappa / mu = 9.8): beta_(2,2) > 0 at <F> = I (L = W_FF(I) is
    positive definite there) and < 0 under strong equi-biaxial compression (0.88 I)."""
    n = 32
    ph = synth.disc_phase(n, 2, 0.4)
    par = np.array([[20.0, 196.0], [1.0, 9.8]])
    s = rve.Rve(2, n, "neohookean", "fp64", max_iter=20000)
    s.set_material(ph, par)
    betas = []
    for lam in (1.0, 0.88):
        assert s.solve(np.diag([lam, lam, 1.0]), 30.0, 1e-9).converged
        info, _, _ = s.bloch((2, 2), 200.0, 1e-6, 60000, seed=0)
        assert info.converged
        betas.append(info.beta)
    assert betas[0] > 0.0 > betas[1]


def test_bloch_full_size_matches_oracle():
    """At 512^2 (the Bloch bench's grid; multi-tile FFT lines, 1024-block reductions),
    on a synthetic near-identity F field of a two-phase neo-Hookean cell: p, sigma and
    the residual history after 5 iterations element by element against the oracle,
    and ||p|| = 1."""
    d, n, k, its = 2, 512, (3, 4), 5
    ph = synth.inclusion_phase(n, d, 5, radius=20)
    par = synth.two_phase_params(1.0, 4.0)
    F = near_identity_field(n, d, 9, amp=0.05)
    p0 = synth.bloch_start(n, d, 4)
    s = handle_with_state(d, n, "neohookean", ph, par, F)
    info, p, hist = s.bloch(k, 8.0, -1.0, its, p0=p0)
    mu_ref = float(np.mean(par[ph.reshape(-1), 0]))
    ref = bloch.bloch_solve(bloch.tangent_field("neohookean", ph, par, F), p0, k, 8.0, -1.0, its, mu_ref)
    assert info.iterations == its
    assert rel(p, ref["p"]) < 1e-10
    np.testing.assert_allclose(info.beta, ref["sigma"], rtol=1e-11)
    np.testing.assert_allclose(hist[:, :2], np.array(ref["history"]), rtol=1e-8, atol=1e-13)
    assert abs(np.sum(np.abs(p) ** 2) / n ** d - 1.0) < 1e-12


# ------------------------------------------------------------------ adaptive penalty

def test_bloch_adaptive_rho_matches_oracle():
    """Section 2.1's residual balancing on Steps 1'-4' (RVE_RHO_ADAPTIVE), from rho = 60 on
    a positive-definite tangent (F = I, floor mu_ref): p, sigma, residuals and the rho
    sequence after 30 iterations element by element against the oracle."""
    d, n, k, its = 2, 24, (3, 4), 30
    ph = synth.inclusion_phase(n, d, 5, radius=3)
    par = synth.two_phase_params(1.0, 4.0)
    F = np.broadcast_to(np.eye(d).reshape(d, d, 1, 1), (d, d, n, n)).copy()
    mu_ref = float(np.mean(par[ph.reshape(-1), 0]))
    p0 = synth.bloch_start(n, d, 2)
    s = rve.Rve(d, n, "neohookean", "fp64", max_iter=10, rho_policy="adaptive")
    s.set_material(ph, par)
    s.set_field(rve.RVE_FIELD_F, F)
    info, p, hist = s.bloch(k, 60.0, -1.0, its, p0=p0)
    ref = bloch.bloch_solve(bloch.tangent_field("neohookean", ph, par, F), p0, k, 60.0, -1.0, its, mu_ref,
                            rho_policy="adaptive")
    np.testing.assert_allclose(hist[:, 3], ref["rhos"], rtol=1e-14)
    assert len(set(np.round(hist[:, 3], 9))) > 3  # the rule acted
    assert rel(p, ref["p"]) < 1e-10
    np.testing.assert_allclose(info.beta, ref["sigma"], rtol=1e-11)
    np.testing.assert_allclose(hist[:, :2], np.array(ref["history"]), rtol=1e-8, atol=1e-13)


@pytest.mark.parametrize("d,n,k", [(2, 6, (3, -2)), (3, 4, (2, 3, 1))])
def test_bloch_adaptive_converges_to_smallest_eigenvalue(d, n, k):
    ph = synth.inclusion_phase(n, d, 3, radius=1)
    par = synth.two_phase_params(1.0, 4.0)
    F = near_identity_field(n, d, 5)
    L = bloch.tangent_field("neohookean", ph, par, F)
    w, _, _ = dense_beta(L, n, d, k)
    s = rve.Rve(d, n, "neohookean", "fp64", max_iter=10, rho_policy="adaptive")
    s.set_material(ph, par)
    s.set_field(rve.RVE_FIELD_F, F)
    info, _, _ = s.bloch(k, 60.0, 1e-10, 20000, p0=synth.bloch_start(n, d, 1))
    assert info.converged
    np.testing.assert_allclose(info.beta, w[0], rtol=1e-9)


def test_bloch_adaptive_is_faster_on_a_compressed_cell():
    """The compressed soft-disc cell (<F> = 0.92 I): the same beta_(2,2) in far fewer
    iterations than at the fixed starting penalty."""
    n = 32
    ph = synth.disc_phase(n, 2, 0.4)
    par = np.array([[20.0, 196.0], [1.0, 9.8]])
    out = {}
    for pol in ("fixed", "adaptive"):
        s = rve.Rve(2, n, "neohookean", "fp64", max_iter=20000, rho_policy=pol)
        s.set_material(ph, par)
        assert s.solve(np.diag([0.92, 0.92, 1.0]), 30.0, 1e-9).converged
        info, _, _ = s.bloch((2, 2), 200.0, 1e-7, 60000, seed=0)
        assert info.converged
        out[pol] = info
    np.testing.assert_allclose(out["adaptive"].beta, out["fixed"].beta, rtol=1e-5, atol=1e-6)
    assert out["adaptive"].iterations < out["fixed"].iterations / 3


def test_bloch_on_a_float_state_handle():
    """A handle in RVE_MIXED keeps a set F in float: the tangent is formed from the float F
    (promoted to double), so beta_k agrees with the FP64 handle's to float rounding of F."""
    d, n, k = 2, 16, (3, 4)
    ph, par, F = two_phase_case(d, n)
    out = []
    for prec in ("fp64", "mixed"):
        s = rve.Rve(d, n, "neohookean", prec, max_iter=10, rho_policy="adaptive")
        s.set_material(ph, par)
        s.set_field(rve.RVE_FIELD_F, F)
        info, _, _ = s.bloch(k, 20.0, 1e-9, 20000, seed=1)
        assert info.converged
        out.append(info.beta)
    np.testing.assert_allclose(out[1], out[0], rtol=1e-5)



# ------------------------------------------------------------------ float bulk

@pytest.mark.parametrize("d,n,k", [(2, 24, (3, 4)), (3, 12, (2, 3, -4))])
def test_bloch_mixed_matches_fp64(d, n, k):
    """RVE_MIXED: a float bulk, then FP64 to the tolerance; the same beta_k as the FP64
    handle on the same F (double in both: F is set through a double handle's field, then
    read back and set again, so both hold the float-representable values)."""
    ph, par, F = two_phase_case(d, n)
    F = F.astype(np.float32).astype(np.float64)  # exactly representable in both handles
    out = {}
    for prec in ("fp64", "mixed"):
        s = rve.Rve(d, n, "neohookean", prec, max_iter=10, rho_policy="adaptive")
        s.set_material(ph, par)
        s.set_field(rve.RVE_FIELD_F, F)
        info, p, hist = s.bloch(k, 40.0, 1e-10, 40000, seed=3)
        assert info.converged
        out[prec] = (info, p)
    im, i64 = out["mixed"][0], out["fp64"][0]
    assert 0 < im.float_iterations < im.iterations
    np.testing.assert_allclose(im.beta, i64.beta, rtol=1e-9)
    np.testing.assert_allclose(im.rayleigh, i64.rayleigh, rtol=1e-9)
    assert abs(np.sum(np.abs(out["mixed"][1]) ** 2) / n ** d - 1.0) < 1e-12


def test_bloch_fp32_stops_after_the_float_phase():
    d, n, k = 2, 24, (3, 4)
    ph, par, F = two_phase_case(d, n)
    F = F.astype(np.float32).astype(np.float64)
    s64 = handle_with_state(d, n, "neohookean", ph, par, F)
    i64, _, _ = s64.bloch(k, 10.0, 1e-10, 40000, seed=3)
    s = rve.Rve(d, n, "neohookean", "fp32", max_iter=10)
    s.set_material(ph, par)
    s.set_field(rve.RVE_FIELD_F, F)
    rc, info, p, hist = rve.rve_bloch(s.h, k, synth.bloch_start(n, d, 3), 10.0, 1e-10, 40000)
    assert rc in (rve.RVE_OK, rve.RVE_E_NOT_CONVERGED)
    assert info.float_iterations == info.iterations > 0
    np.testing.assert_allclose(info.beta, i64.beta, rtol=1e-4)
