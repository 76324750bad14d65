"""Pins of the Bloch-wave oracle (Section 2.4: the modulus of stability beta_k by
Steps 1'-4').

The reference value is the smallest eigenvalue of D^* L D assembled as a dense
matrix from the real-space definition of the Bloch central difference (shifts with
the phase factors exp(+-i omega_j h), no FFT, no symbol), so a wrong phase sign, a
wrong adjoint, a dropped multiplier term or a wrong normalisation in the oracle
changes beta and fails here."""
import numpy as np
import pytest
from scipy import linalg

from oracle import bloch
from paper_2010_06697_gb300 import synth

from . import energies as E


def dense_bloch_matrix(n, d, k):
    """Matrix of p -> D p on C-ordered voxels: rows (voxel, i, j), columns (voxel, i)."""
    V = n ** d
    h = 1.0 / n
    Dm = np.zeros((V * d * d, V * d), dtype=np.complex128)
    idx = np.arange(V).reshape((n,) * d)
    for v in range(V):
        pos = np.unravel_index(v, (n,) * d)
        for j in range(d):
            ax = d - 1 - j  # direction j is array axis d-1-j
            th = 2.0 * np.pi / k[j] * h
            up = list(pos)
            dn = list(pos)
            up[ax] = (pos[ax] + 1) % n
            dn[ax] = (pos[ax] - 1) % n
            vu, vd = idx[tuple(up)], idx[tuple(dn)]
            for i in range(d):
                row = v * d * d + i * d + j
                Dm[row, vu * d + i] += np.exp(1j * th) / (2 * h)
                Dm[row, vd * d + i] -= np.exp(-1j * th) / (2 * h)
    return Dm


def dense_beta(L, n, d, k):
    """Smallest eigenvalue and its vector of D^* L D (the 1/V of both mean-norms cancels)."""
    V = n ** d
    Dm = dense_bloch_matrix(n, d, k)
    Lb = linalg.block_diag(*[L[v].reshape(d * d, d * d) for v in range(V)])
    A = Dm.conj().T @ Lb @ Dm
    w, U = linalg.eigh(A)
    return w, U, A


def near_identity_field(n, d, seed, amp=0.08):
    u = synth.uniform(seed, 61, d * d * n ** d).reshape((d, d) + (n,) * d)
    return np.eye(d).reshape((d, d) + (1,) * d) + amp * (2.0 * u - 1.0)


def start_field(n, d, seed):
    return synth.bloch_start(n, d, seed)


CASES = [(2, 4, (2, 2), "homogeneous"), (2, 6, (3, -2), "two-phase"), (3, 4, (2, 3, 1), "two-phase"),
         (2, 6, (2, 1), "two-phase")]


@pytest.mark.parametrize("d,n,k,kind", CASES)
def test_beta_matches_dense_eigenvalue(d, n, k, kind):
    """Converged sigma and the Rayleigh quotient of p equal the smallest eigenvalue of the
    dense D^* L D; p is its eigenvector (residual of D^* L D p - beta p)."""
    if kind == "homogeneous":
        ph = np.zeros((n,) * d, np.uint8)
        F = np.broadcast_to(np.eye(d).reshape((d, d) + (1,) * d), (d, d) + (n,) * d).copy()
        par, model = np.array([[1.0, 1.5]]), "linear"
    else:
        ph = synth.inclusion_phase(n, d, 3, radius=1)
        F = near_identity_field(n, d, 5)
        par, model = synth.two_phase_params(1.0, 4.0), "neohookean"
    L = bloch.tangent_field(model, ph, par, F)
    w, U, A = dense_beta(L, n, d, k)
    r = bloch.bloch_solve(L, start_field(n, d, 1), k, 10.0, 1e-10, 20000, 1.0)
    assert r["converged"]
    np.testing.assert_allclose(r["sigma"], w[0], rtol=1e-9)
    np.testing.assert_allclose(r["rayleigh"], w[0], rtol=1e-9)
    pv = r["p"].reshape(d, -1).T.reshape(-1)  # (voxel, i) order
    res = A @ pv - w[0] * pv
    assert np.linalg.norm(res) <= 1e-6 * np.linalg.norm(A, 2) * np.linalg.norm(pv)


def test_unit_norm_and_fixed_point():
    """||p|| = 1 after every Step 2'; at convergence D p = G and g = L G."""
    d, n, k = 2, 6, (2, 3)
    ph = synth.inclusion_phase(n, d, 3, radius=1)
    par = synth.two_phase_params(1.0, 4.0)
    L = bloch.tangent_field("neohookean", ph, par, near_identity_field(n, d, 7))
    for it in (1, 2, 5):
        r = bloch.bloch_solve(L, start_field(n, d, 2), k, 10.0, -1.0, it, 1.0)
        assert abs(bloch.norm(r["p"]) - 1.0) < 1e-13
    r = bloch.bloch_solve(L, start_field(n, d, 2), k, 10.0, 1e-12, 20000, 1.0)
    assert r["converged"]
    Dp = bloch.bloch_grad(r["p"], k)
    assert bloch.norm(Dp - r["G"]) < 1e-10
    LG = np.einsum("vab,vb->va", L.reshape(-1, d * d, d * d), r["G"].reshape(d * d, -1).T).T
    assert np.max(np.abs(LG.reshape(r["g"].shape) - r["g"])) < 1e-8 * np.max(np.abs(r["g"]))


def test_tangent_matches_energy_second_derivative():
    """L = W_FF of the Section 4.1 energy: central differences of the complex-step W_F of
    the separately typed energy."""
    d = 2
    F = np.array([[1.05, 0.1], [-0.04, 0.93]])
    mu, lam = 1.3, 2.2
    L = bloch.tangent_field("neohookean", np.zeros((1, 1), np.uint8), np.array([[mu, lam]]),
                            F.reshape(d, d, 1, 1))[0]
    np.testing.assert_allclose(L, E.tangent_fd(E.w_neohooke, F, mu, lam), rtol=1e-6, atol=1e-8)


def test_step2_norm_root_is_unique_and_below_pole():
    """Step 2' returns sigma below rho min kappa with ||p(sigma)|| = 1, and ||p|| grows
    monotonically on that interval (so the root is the unique one the minimiser takes)."""
    rng = np.random.default_rng(3)
    n, d = 8, 2
    kappa = rng.uniform(0.5, 40.0, (n, n))
    b = rng.standard_normal((d, n, n)) + 1j * rng.standard_normal((d, n, n))
    sig, ph = bloch.constrained_step(b, kappa, 10.0, n * n)
    assert sig < 10.0 * kappa.min()
    np.testing.assert_allclose(np.sum(np.abs(ph) ** 2) / (n * n) ** 2, 1.0, rtol=1e-12)
    grid = np.linspace(sig - 50.0, 10.0 * kappa.min() - 1e-9, 50)
    norms = [np.sum(np.abs(10.0 * b / (10.0 * kappa - s)) ** 2) for s in grid]
    assert np.all(np.diff(norms) > 0)


@pytest.mark.parametrize("model", ["linear", "neohookean"])
@pytest.mark.parametrize("d,n,k", [(2, 8, (2, 3)), (2, 6, (-3, 2)), (3, 4, (2, 3, 5))])
def test_homogeneous_beta_closed_form(model, d, n, k):
    """Homogeneous isotropic cell at F = I (where the neo-Hookean tangent equals the linear
    one with the same mu, lambda): a Bloch wave p = e exp(2 pi i m.x) has D p = i e (x) s(m),
    and <Dp, L Dp> = e^H K(s) e with the acoustic tensor K = mu |s|^2 I + (mu + lam) s s^T,
    eigenvalues mu |s|^2 and (2 mu + lam) |s|^2.  So beta = mu min_m |s(m)|^2, with
    s_j(m) = N sin(2 pi (m_j + 1/k_j) / N); no dense matrix, no FFT."""
    mu, lam = 1.3, 0.7
    ph = np.zeros((n,) * d, np.uint8)
    F = np.broadcast_to(np.eye(d).reshape((d, d) + (1,) * d), (d, d) + (n,) * d).copy()
    L = bloch.tangent_field(model, ph, np.array([[mu, lam]]), F)
    m = np.arange(n)
    s2 = [(n * np.sin(2.0 * np.pi * (m + 1.0 / kj) / n)) ** 2 for kj in k]
    beta = mu * sum(float(np.min(q)) for q in s2)  # |s|^2 separates over the directions
    r = bloch.bloch_solve(L, start_field(n, d, 4), k, 2.0 * beta + 5.0, 1e-11, 20000, mu)
    assert r["converged"]
    np.testing.assert_allclose(r["sigma"], beta, rtol=1e-9)
    np.testing.assert_allclose(r["rayleigh"], beta, rtol=1e-9)


# ------------------------------------------------------------------ the pins bite

_orig_symbols = bloch.bloch_symbols


def _symbols_one_phase_flipped(n, dim, k):
    return _orig_symbols(n, dim, [-k[0]] + list(k[1:]))


def _step2_normalised_projection(b_hat, kappa, rho, nvox):
    """The unconstrained Step 2' followed by a normalisation (its fixed points are
    eigenvectors of the pencil (D^* L D, D^* D), not of D^* L D)."""
    ph = b_hat / kappa
    ph = ph / np.sqrt(np.sum(np.abs(ph) ** 2) / nvox ** 2)
    return float("nan"), ph


@pytest.mark.parametrize("name,fn", [("bloch_symbols", _symbols_one_phase_flipped),
                                     ("constrained_step", _step2_normalised_projection)])
def test_planted_mistakes_fail_the_dense_pin(monkeypatch, name, fn):
    d, n, k = 2, 6, (3, 4)  # omega = pi and -pi give the same Bloch waves: no k_j = +-2 here
    ph = synth.inclusion_phase(n, d, 3, radius=1)
    L = bloch.tangent_field("neohookean", ph, synth.two_phase_params(1.0, 4.0), near_identity_field(n, d, 5))
    w, _, _ = dense_beta(L, n, d, k)
    monkeypatch.setattr(bloch, name, fn)
    r = bloch.bloch_solve(L, start_field(n, d, 1), k, 10.0, 1e-10, 3000, 1.0)
    assert not (r["converged"] and abs(r["rayleigh"] - w[0]) <= 1e-9 * abs(w[0]))


@pytest.mark.parametrize("d,n,k", [(2, 6, (3, -2)), (3, 4, (2, 3, 1))])
def test_adaptive_rho_reaches_the_same_eigenvalue(d, n, k):
    """Section 2.1's residual balancing applied to Steps 1'-4' changes the path, not the
    fixed point: the converged sigma is the dense smallest eigenvalue, rho never drops
    below the floor and it changes by the factor kappa."""
    ph = synth.inclusion_phase(n, d, 3, radius=1)
    par = synth.two_phase_params(1.0, 4.0)
    L = bloch.tangent_field("neohookean", ph, par, near_identity_field(n, d, 5))
    w, _, _ = dense_beta(L, n, d, k)
    r = bloch.bloch_solve(L, start_field(n, d, 1), k, 60.0, 1e-10, 20000, 1.0, rho_policy="adaptive")
    assert r["converged"]
    np.testing.assert_allclose(r["sigma"], w[0], rtol=1e-9)
    floor = bloch.rho_floor(L, 1.0)
    rh = np.array(r["rhos"])
    assert np.all(rh >= floor * (1 - 1e-12))
    ratios = rh[1:] / rh[:-1]
    assert np.all(np.isclose(ratios, 1.0) | np.isclose(ratios, 1.3) | np.isclose(ratios, 1 / 1.3)
                  | np.isclose(rh[1:], floor))
    assert rh[-1] < 60.0
