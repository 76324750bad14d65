"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

FP64 mode must match the oracle within 1e-10 (relative to the field's largest
entry); mixed mode within 1e-5 relative on the homogenised stress.  Inputs come
from the seeded generators; no expected value comes from the CUDA path.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import admm as oadmm
from paper_2010_06697_gb300 import build, rve, synth
from tests import energies as E

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def cell(kind, d, n, seed=0):
    if kind == "laminate":
        return synth.laminate_phase(n, d)
    r = 6 if n >= 32 else max(1, n // 5)
    return synth.inclusion_phase(n, d, seed, radius=r)


PAR = synth.two_phase_params(1.0, 10.0)


def run_gpu(ph, par, Fbar, rho, tol, max_iter, model="neohookean", precision="fp64", **opt):
    s = rve.Rve(ph.ndim, ph.shape[0], model, precision, max_iter=max_iter, **opt)
    s.set_material(ph, par)
    info = s.solve(Fbar, rho, tol)
    return s, info


# ------------------------------------------------------------------ first iterations, many sizes

SIZES = [("laminate", 2, 32), ("inclusion", 2, 48), ("inclusion", 2, 6), ("inclusion", 2, 36),
         ("laminate", 3, 8), ("inclusion", 3, 12), ("inclusion", 3, 16), ("inclusion", 3, 24),
         ("inclusion", 3, 6), ("inclusion", 3, 18),
         ("inclusion", 3, 4), ("laminate", 2, 4), ("inclusion", 2, 512)]  # smallest and largest 2D grids


@pytest.mark.parametrize("kind,d,n", SIZES)
def test_first_iterations_match_oracle(kind, d, n):
    """Three FP64 iterations (Steps 1-4 each) from the fresh state: F, Lambda, u~,
    the residual history and <W_F(F)> agree with the oracle."""
    ph = cell(kind, d, n)
    Fbar = np.diag([0.93, 1.0, 1.04])
    Fbar[0, 1] = 0.02
    s, info = run_gpu(ph, PAR, Fbar, 7.0, -1.0, 3)
    ref = oracle.admm_solve(ph, PAR, Fbar, 7.0, -1.0, 3)
    assert info.iterations == 3
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert np.max(np.abs(st["u"] - ref["u"])) < TOL64 * max(1.0, np.max(np.abs(ref["u"])))
    hist = s.history()
    np.testing.assert_allclose(hist[:, :2], np.array(ref["history"])[:, :2], rtol=1e-9, atol=1e-14)
    assert rel(s.stress(), ref["stress"]) < TOL64


# ------------------------------------------------------------------ config 1: 2D laminate, 300 iterations

def test_config1_laminate_300_iterations():
    """2D 32x32 neo-Hookean laminate, mu = 1 | 10, nu = 0.3, Fbar = diag(1.05, 1),
    rho = 10, exactly 300 FP64 iterations: fields, history and stress vs the
    oracle, and the stress vs the semi-analytic laminate."""
    ph = synth.laminate_phase(32, 2)
    Fbar = np.diag([1.05, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 10.0, -1.0, 300)
    ref = oracle.admm_solve(ph, PAR, Fbar, 10.0, -1.0, 300)
    assert info.iterations == 300
    st = s.state()
    assert rel(st["F"], ref["F"]) < TOL64
    assert rel(st["Lam"], ref["Lam"]) < TOL64
    assert rel(s.stress(), ref["stress"]) < TOL64
    from tests.test_oracle_pins import _laminate_exact
    _, _, S = _laminate_exact("neohookean", PAR, Fbar[:2, :2])
    np.testing.assert_allclose(s.stress(), S, atol=1e-11)


# ------------------------------------------------------------------ converged solves

@pytest.mark.parametrize("d,n", [(3, 16), (2, 64)])
def test_converged_inclusion_cell_matches_oracle(d, n):
    """Inclusion cell in compression (Fbar = diag(0.9, 1, 1)), rho = 10, tol 1e-8:
    same iteration count and stress within 1e-10."""
    ph = cell("inclusion", d, n, seed=1)
    Fbar = np.diag([0.9, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 10.0, 1e-8, 1000)
    ref = oracle.admm_solve(ph, PAR, Fbar, 10.0, 1e-8, 1000)
    assert info.converged and ref["converged"]
    assert info.iterations == ref["iters"]
    assert rel(s.stress(), ref["stress"]) < TOL64
    assert rel(s.get_field(rve.RVE_FIELD_F), ref["F"]) < TOL64
    # <Lambda> = <W_F(F)> at an exact local solve
    assert rel(s.mean_lambda(), ref["stress"]) < 1e-9


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8)])
def test_linear_laminate_closed_form_on_gpu(d, n):
    from tests.test_oracle_pins import _laminate_exact
    ph = synth.laminate_phase(n, d)
    rng = np.random.default_rng(21)
    Fbar = np.eye(3)
    Fbar[:d, :d] += 0.05 * rng.uniform(-1, 1, (d, d))
    FA, FB, S = _laminate_exact("linear", PAR, Fbar[:d, :d])
    s, info = run_gpu(ph, PAR, Fbar, 10.0, 1e-13, 3000, model="linear")
    assert info.converged
    np.testing.assert_allclose(s.stress(), S, atol=1e-10)
    F = s.get_field(rve.RVE_FIELD_F)
    np.testing.assert_allclose(F[..., : n // 2].reshape(d, d, -1).mean(-1), FA, atol=1e-10)


def test_homogeneous_cell_affine_fixed_point():
    ph = np.zeros((8, 8, 8), np.uint8)
    par = np.array([[1.7, 2.9]])
    Fbar = np.array([[1.02, 0.03, 0.0], [-0.01, 0.97, 0.02], [0.0, 0.01, 1.05]])
    s, info = run_gpu(ph, par, Fbar, 10.0, 1e-14, 5)
    assert info.converged and info.iterations == 1
    P = E.stress_cs(E.w_neohooke, Fbar, 1.7, 2.9)
    np.testing.assert_allclose(s.stress(), P, atol=1e-12)
    np.testing.assert_allclose(s.get_field(rve.RVE_FIELD_U), 0.0, atol=1e-14)


# ------------------------------------------------------------------ state: warm start, checkpoint

def test_warm_start_load_steps_match_oracle():
    """Two load steps; the second starts from the first's state (Algorithm 1)."""
    ph = cell("inclusion", 3, 12, seed=2)
    F1 = np.diag([0.97, 1.0, 1.0])
    F2 = np.diag([0.94, 1.0, 1.0])
    s = rve.Rve(3, 12, "neohookean", "fp64", max_iter=400)
    s.set_material(ph, PAR)
    i1 = s.solve(F1, 10.0, 1e-9)
    i2 = s.solve(F2, 10.0, 1e-9)
    r1 = oracle.admm_solve(ph, PAR, F1, 10.0, 1e-9, 400)
    r2 = oracle.admm_solve(ph, PAR, F2, 10.0, 1e-9, 400, state={"F": r1["F"], "Lam": r1["Lam"], "u": r1["u"]})
    assert i1.iterations == r1["iters"] and i2.iterations == r2["iters"]
    assert rel(s.stress(), r2["stress"]) < TOL64


def test_checkpoint_resume_is_bit_exact():
    """Save (F, Lambda, u~) after 7 iterations, continue 9 more; a new handle
    restored from the snapshot reproduces the continuation bit for bit."""
    ph = cell("inclusion", 3, 16, seed=3)
    Fbar = np.diag([0.92, 1.0, 1.03])
    a = rve.Rve(3, 16, "neohookean", "fp64", max_iter=7)
    a.set_material(ph, PAR)
    a.solve(Fbar, 10.0, -1.0)
    snap = a.state()
    b = rve.Rve(3, 16, "neohookean", "fp64", max_iter=9)
    b.set_material(ph, PAR)
    b.set_state(snap)
    a2 = rve.Rve(3, 16, "neohookean", "fp64", max_iter=16)
    a2.set_material(ph, PAR)
    a2.solve(Fbar, 10.0, -1.0)
    b.solve(Fbar, 10.0, -1.0)
    for k in ("F", "Lam", "u"):
        assert np.array_equal(a2.state()[k], b.state()[k]), k


# ------------------------------------------------------------------ precision modes

def test_mixed_precision_stress_within_tolerance():
    """FP32 bulk with FP64 residuals, promoted to FP64 for the last iterations:
    converges to tol 1e-8 and <S> is within 1e-5 of the FP64 oracle."""
    ph = cell("inclusion", 3, 24, seed=4)
    Fbar = np.diag([0.9, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 10.0, 1e-8, 1000, precision="mixed")
    ref = oracle.admm_solve(ph, PAR, Fbar, 10.0, 1e-10, 1000)
    assert info.converged, info.as_dict()
    assert 0 < info.fp64_iterations < info.iterations
    assert rel(s.stress(), ref["stress"]) < 1e-5
    assert rel(s.get_field(rve.RVE_FIELD_F), ref["F"]) < 1e-4


def test_fp32_mode_reaches_its_floor():
    ph = cell("inclusion", 3, 16, seed=5)
    Fbar = np.diag([0.9, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 10.0, 1e-12, 1000, precision="fp32")
    ref = oracle.admm_solve(ph, PAR, Fbar, 10.0, 1e-10, 1000)
    assert not info.converged
    assert max(info.r_p, info.r_d) < 1e-4
    assert rel(s.stress(), ref["stress"]) < 1e-4


def test_adaptive_rho_decisions_match_oracle():
    """eq. rho-update: the sequence of penalties chosen on the GPU equals the oracle's."""
    ph = synth.laminate_phase(16, 2)
    Fbar = np.diag([1.05, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 100.0, 1e-10, 400, rho_policy="adaptive")
    ref = oracle.admm_solve(ph, PAR, Fbar, 100.0, 1e-10, 400, rho_policy="adaptive")
    hist = s.history()
    href = np.array(ref["history"])
    assert info.iterations == ref["iters"]
    np.testing.assert_array_equal(hist[:, 2], href[:, 2])
    assert len(set(href[:, 2])) > 1
    assert rel(s.stress(), ref["stress"]) < TOL64


# ------------------------------------------------------------------ errors

@pytest.mark.parametrize("nphase", [2, 5, 11])
def test_material_phase_counts_and_validation(nphase):
    """rve_set_material counts the voxels of each phase (mu_ref = volume average of mu,
    reported in the solve info) and rejects a phase id >= nphase wherever it sits: first
    voxel, inside or at the edge of an 8-voxel word, ragged tail."""
    n, d = 18, 3  # V = 5832: a multiple of 8; the 2D case below has V = 324 = 8*40 + 4
    for dim, nn in ((d, n), (2, n)):
        V = nn ** dim
        ph = (synth.splitmix64(3, 77, V) % np.uint64(nphase)).astype(np.uint8).reshape((nn,) * dim)
        par = np.array([[1.0 + p, 2.0] for p in range(nphase)])
        s = rve.Rve(dim, nn, "neohookean", "fp64", max_iter=1)
        s.set_material(ph, par)
        info = s.solve(np.diag([1.01, 1.0, 1.0]), 10.0, 1e-30)
        mu = par[ph.ravel(), 0]
        assert abs(info.mu_ref - mu.mean()) <= 1e-14 * mu.mean()
        for idx in (0, 5, 7, 8, V // 2 + 3, V - 4, V - 1):
            bad = ph.copy()
            bad.flat[idx] = nphase + idx % 3
            assert rve.rve_set_material(s.h, bad, par) == rve.RVE_E_INVALID_ARG, idx
        s.close()


def test_error_paths():
    s = rve.Rve(2, 16, "neohookean", "fp64", max_iter=10)
    rc, _ = rve.rve_solve(s.h, np.eye(3), 10.0, 1e-8)
    assert rc == rve.RVE_E_STATE
    ph = synth.laminate_phase(16, 2)
    assert rve.rve_set_material(s.h, ph + 5, PAR) == rve.RVE_E_INVALID_ARG
    s.set_material(ph, PAR)
    rc, _ = rve.rve_solve(s.h, np.diag([-1.0, 1.0, 1.0]), 10.0, 1e-8)
    assert rc == rve.RVE_E_INVALID_ARG
    rc, _ = rve.rve_solve(s.h, np.diag([np.nan, 1.0, 1.0]), 10.0, 1e-8)
    assert rc == rve.RVE_E_INVALID_ARG
    rc, _ = rve.rve_solve(s.h, np.eye(3), -1.0, 1e-8)
    assert rc == rve.RVE_E_INVALID_ARG
    rc, info = rve.rve_solve(s.h, np.diag([1.05, 1, 1]), 10.0, 1e-30)
    assert rc == rve.RVE_E_NOT_CONVERGED and info.iterations == 10
    bad = np.full((2, 2, 16, 16), np.inf)
    assert rve.rve_set_field(s.h, rve.RVE_FIELD_F, bad) == rve.RVE_E_INVALID_ARG


# ------------------------------------------------------------------ full size (128^3)

def _inclusions128():
    return synth.inclusion_phase(128, 3, 0)


def test_full_size_first_iteration_sampled():
    """128^3 inclusion cell, one FP64 iteration in the bench's launch shape:
    F_1 at sampled voxels equals the oracle's local solve from the inputs alone,
    and u~_1, Lambda_1 satisfy Step 2's normal equations and Step 3 exactly."""
    ph = _inclusions128()
    Fbar = np.diag([0.9, 1.0, 1.0])
    rho = 10.0
    s, info = run_gpu(ph, PAR, Fbar, rho, -1.0, 1)
    st = s.state()
    rng = np.random.default_rng(0)
    idx = rng.choice(ph.size, 4096, replace=False)
    mat = oracle.make_material("neohookean", ph.reshape(-1)[idx], PAR)
    F0 = np.broadcast_to(Fbar, (idx.size, 3, 3)).copy()
    Lam0 = mat.P(F0)
    F1, _ = oracle.local_newton(mat, F0, Lam0, F0.copy(), rho)
    F1_gpu = st["F"].reshape(3, 3, -1)[:, :, idx].transpose(2, 0, 1)
    assert rel(F1_gpu, F1) < TOL64
    # Step 2 normal equations D^T D u = D^T (F_1 - Lambda_0/rho) and Step 3
    Lam0_full = oracle.make_material("neohookean", ph, PAR).P(
        np.broadcast_to(Fbar, (ph.size, 3, 3)).copy()).transpose(1, 2, 0).reshape(3, 3, *ph.shape)
    Q = st["F"] - Lam0_full / rho
    lhs = E.div_stencil(E.grad_stencil(st["u"]))
    rhs = E.div_stencil(Q)
    assert np.max(np.abs(lhs - rhs)) < 1e-9 * np.max(np.abs(rhs))
    G = Fbar.reshape(3, 3, 1, 1, 1) + E.grad_stencil(st["u"])
    assert rel(st["Lam"], Lam0_full + rho * (G - st["F"])) < TOL64


def test_full_size_converged_stress_matches_stored_oracle_run():
    """128^3 inclusion cell to tol 1e-8: iteration count and <S> equal the stored
    oracle run (tests/golden/inclusions128.json, written by make_golden.py)."""
    path = os.path.join(HERE, "golden", "inclusions128.json")
    if not os.path.exists(path):
        pytest.skip("golden oracle run not present")
    g = json.load(open(path))
    ph = _inclusions128()
    assert abs(ph.mean() - g["phase_fraction"]) < 1e-12
    Fbar = np.array(g["recipe"]["Fbar"], float)
    s, info = run_gpu(ph, PAR, Fbar, g["recipe"]["rho"], g["recipe"]["tol"], 1000)
    assert info.converged and info.iterations == g["iters"]
    assert rel(s.stress(), np.array(g["stress"])) < TOL64
    m, im = run_gpu(ph, PAR, Fbar, g["recipe"]["rho"], g["recipe"]["tol"], 1000, precision="mixed")
    assert im.converged
    assert rel(m.stress(), np.array(g["stress"])) < 1e-5
    # the bench's configuration: the adaptive penalty from the same rho, FP64 and mixed
    a64, ia64 = run_gpu(ph, PAR, Fbar, g["recipe"]["rho"], g["recipe"]["tol"], 1000, rho_policy="adaptive")
    assert ia64.converged
    assert rel(a64.stress(), np.array(g["stress"])) < 1e-8
    am, iam = run_gpu(ph, PAR, Fbar, g["recipe"]["rho"], g["recipe"]["tol"], 1000, precision="mixed",
                      rho_policy="adaptive")
    assert iam.converged and iam.iterations < info.iterations
    assert rel(am.stress(), np.array(g["stress"])) < 1e-5


# ------------------------------------------------------------------ large sizes (256^3, maximum 512^3)

@pytest.mark.parametrize("n", [256, 512])
def test_large_first_iteration_sampled(n):
    """256^3 and the largest cell the library accepts, 512^3 (134M voxels), one FP64
    iteration with the fixed-length y/z kernels: at 2048 sampled voxels F_1 equals the
    oracle's local solve from the inputs alone, and u~_1, Lambda_1 satisfy Step 2's
    normal equations and Step 3 there (the stencils are gathered around each sampled
    voxel; each field is fetched, sampled and dropped in turn to bound host memory)."""
    ph = synth.inclusion_phase(n, 3, 1)
    Fbar = np.diag([0.9, 1.0, 1.0])
    rho = 10.0
    s, info = run_gpu(ph, PAR, Fbar, rho, -1.0, 1)
    assert info.iterations == 1
    V = ph.size
    rng = np.random.default_rng(3)
    idx = rng.choice(V, 2048, replace=False)
    z, y, x = np.unravel_index(idx, ph.shape)

    def at(dz=0, dy=0, dx=0):
        return np.ravel_multi_index(((z + dz) % n, (y + dy) % n, (x + dx) % n), ph.shape)

    off = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]  # e_1 (x), e_2 (y), e_3 (z) as (dz, dy, dx)
    plus = [at(*o) for o in off]
    minus = [at(-o[0], -o[1], -o[2]) for o in off]
    phf = ph.reshape(-1)
    mat_s = oracle.make_material("neohookean", phf[idx], PAR)
    F0 = np.broadcast_to(Fbar, (idx.size, 3, 3)).copy()
    F1, _ = oracle.local_newton(mat_s, F0, mat_s.P(F0), F0.copy(), rho)
    # Lambda_0 = W_F(Fbar) per phase
    P_phase = oracle.make_material("neohookean", np.arange(2, dtype=np.uint8), PAR).P(
        np.broadcast_to(Fbar, (2, 3, 3)).copy()).reshape(2, 9)
    Fg = s.get_field(rve.RVE_FIELD_F).reshape(9, V)
    F_c = Fg[:, idx].copy()
    F_p = [Fg[:, pts].copy() for pts in plus]
    F_m = [Fg[:, pts].copy() for pts in minus]
    del Fg
    assert rel(F_c.T.reshape(-1, 3, 3), F1) < TOL64
    U = s.get_field(rve.RVE_FIELD_U).reshape(3, V)
    half = n / 2.0
    G = np.zeros((3, 3, idx.size))
    for i in range(3):
        lhs = np.zeros(idx.size)
        rhs = np.zeros(idx.size)
        for j, (dz, dy, dx) in enumerate(off):
            lhs += (U[i, at(2 * dz, 2 * dy, 2 * dx)] - 2 * U[i, idx] + U[i, at(-2 * dz, -2 * dy, -2 * dx)]) * half * half
            qp = F_p[j][3 * i + j] - P_phase[phf[plus[j]], 3 * i + j] / rho
            qm = F_m[j][3 * i + j] - P_phase[phf[minus[j]], 3 * i + j] / rho
            rhs += (qp - qm) * half
            G[i, j] = Fbar[i, j] + (U[i, plus[j]] - U[i, minus[j]]) * half
        assert np.max(np.abs(lhs - rhs)) < 1e-9 * max(np.max(np.abs(rhs)), 1e-300)
    del U
    # Step 3: Lambda_1 = Lambda_0 + rho (Fbar + D u~_1 - F_1)
    Lg = s.get_field(rve.RVE_FIELD_LAMBDA).reshape(9, V)[:, idx].copy()
    for i in range(3):
        for j in range(3):
            want = P_phase[phf[idx], 3 * i + j] + rho * (G[i, j] - F_c[3 * i + j])
            assert np.max(np.abs(Lg[3 * i + j] - want)) < TOL64 * max(np.max(np.abs(want)), 1.0)
    s.close()


def test_float_path_fixed_length_kernels_match_double():
    """128^3, two iterations in float (fixed-length float y/z kernels) against the same
    two iterations in double: the fields agree to float accuracy."""
    ph = _inclusions128()
    Fbar = np.diag([0.9, 1.0, 1.0])
    s64, _ = run_gpu(ph, PAR, Fbar, 10.0, -1.0, 2)
    s32, _ = run_gpu(ph, PAR, Fbar, 10.0, -1.0, 2, precision="fp32")
    a, b = s32.state(), s64.state()
    assert rel(a["F"], b["F"]) < 2e-5
    assert rel(a["u"], b["u"]) < 2e-4
    assert rel(a["Lam"], b["Lam"]) < 2e-5


def test_mixed_adaptive_rho_freezes_for_the_polish():
    """RVE_MIXED with the adaptive penalty: the rule acts in the float bulk, rho stays at
    its value from the switch on (the double-word increment polish needs a constant rho),
    and the converged stress matches the FP64 solve's to the mixed tolerance."""
    n = 24
    ph = synth.inclusion_phase(n, 3, 1, radius=3)
    Fbar = np.diag([0.9, 1.0, 1.0])
    s, info = run_gpu(ph, PAR, Fbar, 100.0, 1e-8, 2000, precision="mixed", rho_policy="adaptive")
    s64, info64 = run_gpu(ph, PAR, Fbar, 100.0, 1e-8, 2000, rho_policy="adaptive")
    assert info.converged and info64.converged
    assert 0 < info.fp64_iterations < info.iterations
    hist = s.history()
    rhos = hist[:, 2]
    assert len(set(rhos[: info.iterations - info.fp64_iterations])) > 1  # the rule acted
    assert len(set(rhos[info.iterations - info.fp64_iterations:])) == 1  # frozen in the polish
    assert rel(s.stress(), s64.stress()) < 1e-5
