"""The lean per-RVE local kernels (fixed grids of 256^3 and 512^3, 134M voxels, and a
run-time grid, 96^3) against the FP64 oracle's local solve (Section 2.1, Step 1) at
sampled voxels, a whole mixed-precision solve on a run-time grid against the FP64 path,
and a batch mixing lean and tile-table members against the members solved alone.

RVE_MIXED on these grids runs the closed-form local step in the lean per-RVE kernel,
for the first local step of a solve (F_1 from Fbar) and fused with Steps 3-4 (F_2 from
G_1 = Fbar + D u~_1 and Lambda_1).  A one-iteration solve leaves (F_1, u~_1, Lambda_1);
a two-iteration solve from the same fresh state leaves F_2.  At 1024 sampled voxels:
  F_1 = argmin W(F) - Lambda_0 : F + rho/2 |F - Fbar|^2 with Lambda_0 = W_F(Fbar),
  Lambda_1 = Lambda_0 + rho (G_1 - F_1) (Step 3, G_1 from the GPU's u~_1 by the stencil),
  F_2 = argmin W(F) - Lambda_1 : F + rho/2 |F - G_1|^2, warm-started at F_1,
each to 2e-5 relative (the stated per-field tolerance of the float phase).  Fields are
fetched, sampled and dropped one at a time to bound host memory."""
import numpy as np
import pytest

import oracle
from paper_2010_06697_gb300 import build, rve, synth

from .test_gpu_batch import fbars, members

pytestmark = pytest.mark.gpu
TOL = 2e-5
PAR = synth.two_phase_params(1.0, 10.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def solve(ph, Fbar, rho, iters):
    s = rve.Rve(3, ph.shape[0], "neohookean", "mixed", max_iter=iters)
    s.set_material(ph, PAR)
    info = s.solve(Fbar, rho, -1.0)
    assert info.iterations == iters and info.fp64_iterations == 0, info.as_dict()
    return s


@pytest.mark.parametrize("n", [96, 256, 512])
def test_lean_local_steps_match_oracle_sampled(n):
    ph = synth.inclusion_phase(n, 3, 2)
    Fbar = np.diag([0.9, 1.0, 1.0])
    rho = 10.0
    V = ph.size
    rng = np.random.default_rng(5)
    idx = rng.choice(V, 1024, replace=False)
    z, y, x = np.unravel_index(idx, ph.shape)

    def at(dz, dy, dx):
        return np.ravel_multi_index(((z + dz) % n, (y + dy) % n, (x + dx) % n), ph.shape)

    off = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]  # x, y, z as (dz, dy, dx)
    plus = [at(*o) for o in off]
    minus = [at(-o[0], -o[1], -o[2]) for o in off]
    mat_s = oracle.make_material("neohookean", ph.reshape(-1)[idx], PAR)
    Fb = np.broadcast_to(Fbar, (idx.size, 3, 3)).copy()
    L0 = mat_s.P(Fb)

    s = solve(ph, Fbar, rho, 1)
    F1 = s.get_field(rve.RVE_FIELD_F).reshape(9, V)[:, idx].T.reshape(-1, 3, 3).copy()
    U = s.get_field(rve.RVE_FIELD_U).reshape(3, V)
    G1 = np.empty((idx.size, 3, 3))
    for i in range(3):
        for j in range(3):
            G1[:, i, j] = Fbar[i, j] + (U[i, plus[j]] - U[i, minus[j]]) * (n / 2.0)
    del U
    L1 = s.get_field(rve.RVE_FIELD_LAMBDA).reshape(9, V)[:, idx].T.reshape(-1, 3, 3).copy()
    s.close()

    F1_ref, _ = oracle.local_newton(mat_s, Fb, L0, Fb.copy(), rho)
    assert rel(F1, F1_ref) < TOL
    assert rel(L1, L0 + rho * (G1 - F1)) < TOL

    s = solve(ph, Fbar, rho, 2)
    F2 = s.get_field(rve.RVE_FIELD_F).reshape(9, V)[:, idx].T.reshape(-1, 3, 3).copy()
    s.close()
    F2_ref, _ = oracle.local_newton(mat_s, F1, L1, G1, rho)
    assert rel(F2, F2_ref) < TOL


def test_runtime_grid_mixed_solve_matches_fp64():
    """96^3 (a run-time grid: the float phase and the double-word polish both in the lean
    kernels) solved to tol 1e-8 in RVE_MIXED and in FP64 (the tile-table double kernels):
    both converge, their homogenised stresses agree to 1e-6, and so do the returned states
    F, Lambda and u~ (the mixed polish keeps u~ as float pairs and returns it in double)."""
    n = 96
    ph = synth.inclusion_phase(n, 3, 4)
    Fbar = np.diag([0.92, 1.0, 1.01])
    out = {}
    for prec in ("mixed", "fp64"):
        s = rve.Rve(3, n, "neohookean", prec, max_iter=2000)
        s.set_material(ph, PAR)
        info = s.solve(Fbar, 10.0, 1e-8)
        assert info.converged, (prec, info.as_dict())
        out[prec] = (info, s.stress(), {w: s.get_field(w) for w in (rve.RVE_FIELD_F, rve.RVE_FIELD_LAMBDA,
                                                                       rve.RVE_FIELD_U)})
        s.close()
    assert out["mixed"][0].fp64_iterations > 0
    assert rel(out["mixed"][1], out["fp64"][1]) < 1e-6
    for w, fm in out["mixed"][2].items():
        assert rel(fm, out["fp64"][2][w]) < 1e-6, w


def test_batch_with_lean_and_tile_members_bitwise():
    """A batch run of mixed sizes with lean members (64^3, 72^3: full local grids) and a
    tile-table member (12^3), mixed precision to tol 1e-8: every member's iterations and
    stress equal its alone solve bit for bit (the lean launch and the shared tile launch
    depend on each member alone)."""
    specs = [(3, 64, "inclusion", 21), (3, 12, "inclusion", 22), (3, 72, "laminate", 23)]
    Fb = fbars(len(specs), 70)
    alone = members(specs, "mixed")
    ref = []
    for s, F in zip(alone, Fb):
        info = s.solve(F, 10.0, 1e-8)
        assert info.converged
        ref.append((info.iterations, info.fp64_iterations, s.stress()))
        s.close()
    mix = members(specs, "mixed")
    infos = rve.Batch(mix).solve(Fb, np.full(len(specs), 10.0), 1e-8)
    for s, info, (it, it64, S) in zip(mix, infos, ref):
        assert info.iterations == it and info.fp64_iterations == it64
        assert np.array_equal(s.stress(), S)
        s.close()
