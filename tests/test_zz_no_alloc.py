"""rve_stress_noalloc: the homogenised stress for callers that cannot allocate
device memory (their device memory is owned by a pool they may not grow, or they
run in loops where cudaMalloc's possible device synchronisation is not allowed).
Its result must equal rve_stress and the FP64 oracle's <W_F(F)> on the same field,
call after call, although every call reuses the same static device scratch array.

This file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _call(dim, n, model, F_dev, ph_dev, par_dev, nphase, nparam, out):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    out.fill_(float("nan"))
    rc = rve.rve_stress_noalloc(dim, n, rve.MODELS[model], F_dev.data_ptr(), ph_dev.data_ptr(), par_dev.data_ptr(),
                                nphase, nparam, out.data_ptr(), stream)
    assert rc == rve.RVE_OK, rve.rve_strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(3, 3)


# 64^3 and 512^2 launch 256 blocks, more than the 128 threads of the last block's
# loop over block partials; the others launch 1 to 4 blocks
@pytest.mark.parametrize("dim,n,model", [(3, 16, "neohookean"), (2, 32, "neohookean"), (3, 12, "linear"),
                                         (3, 64, "neohookean"), (2, 512, "linear")])
def test_noalloc_stress_matches_rve_stress_and_oracle_twice(dim, n, model):
    import torch
    build.build()
    rve.lib()
    ph = synth.inclusion_phase(n, dim, 7, radius=3)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar = np.diag([0.93, 1.02, 1.0])
    Fbar[0, 1] = 0.03
    s = rve.Rve(dim, n, model, "fp64", max_iter=6)
    s.set_material(ph, par)
    s.solve(Fbar, 10.0, -1.0)
    S_ref = s.stress()
    F = s.get_field(rve.RVE_FIELD_F)
    s.close()
    S_orc = oracle.homogenised_stress(ph, par, F, model=model)
    # the caller's own device buffers (here provided by torch)
    F_dev = torch.from_numpy(np.ascontiguousarray(F).reshape(-1)).cuda()
    ph_dev = torch.from_numpy(np.ascontiguousarray(ph).reshape(-1)).cuda()
    par_dev = torch.from_numpy(np.ascontiguousarray(par).reshape(-1)).cuda()
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    for call in range(2):
        S = _call(dim, n, model, F_dev, ph_dev, par_dev, par.shape[0], par.shape[1], out)
        assert _rel(S[:dim, :dim], S_ref) < TOL, (call, S, S_ref)
        assert _rel(S[:dim, :dim], S_orc) < TOL, (call, S, S_orc)
        assert np.all(S[dim:, :] == 0.0) and np.all(S[:, dim:] == 0.0)


def test_noalloc_at_capacity_affine_field_closed_form():
    """256^3 (16,384 blocks, the capacity of the static scratch): an affine field
    F = Fbar everywhere gives <W_F> = sum over phases of (volume fraction) W_F(Fbar),
    written out here for the compressible neo-Hookean law of Section 4.1."""
    import torch
    rve.lib()
    n = 256
    ph = synth.inclusion_phase(n, 3, 0, radius=6)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar = np.array([[0.9, 0.02, 0.0], [0.0, 1.01, -0.01], [0.03, 0.0, 1.02]])
    J = np.linalg.det(Fbar)
    A = np.linalg.inv(Fbar).T
    want = np.zeros((3, 3))
    for p in range(2):
        mu, lam = par[p, 0], par[p, 1]
        want += np.mean(ph == p) * (mu * Fbar + (lam * J * (J - 1.0) - mu) * A)
    F_dev = torch.from_numpy(Fbar.reshape(9)).cuda().repeat_interleave(n ** 3)
    ph_dev = torch.from_numpy(ph.reshape(-1)).cuda()
    par_dev = torch.from_numpy(np.ascontiguousarray(par).reshape(-1)).cuda()
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    for _ in range(2):
        S = _call(3, n, "neohookean", F_dev, ph_dev, par_dev, 2, 2, out)
        assert _rel(S, want) < TOL, (S, want)
    del F_dev
    torch.cuda.empty_cache()


def test_noalloc_invalid_phase_gives_nan_then_recovers():
    """A phase byte equal to nphase (one past the table) makes the result NaN; the
    next call on valid data is correct again (the error flag is cleared per call).
    The kernel skips that voxel without reading the table, so nothing out of range
    is accessed."""
    import torch
    rve.lib()
    n = 16
    ph = synth.inclusion_phase(n, 3, 7, radius=3)
    par = synth.two_phase_params(1.0, 10.0)
    F = np.broadcast_to(np.diag([0.95, 1.0, 1.05]).reshape(3, 3, 1, 1, 1), (3, 3, n, n, n)).copy()
    F_dev = torch.from_numpy(F.reshape(-1)).cuda()
    par_dev = torch.from_numpy(np.ascontiguousarray(par).reshape(-1)).cuda()
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    bad = ph.reshape(-1).copy()
    bad[1234] = 2
    S = _call(3, n, "neohookean", F_dev, torch.from_numpy(bad).cuda(), par_dev, 2, 2, out)
    assert np.all(np.isnan(S[:3, :3]))
    S = _call(3, n, "neohookean", F_dev, torch.from_numpy(ph.reshape(-1)).cuda(), par_dev, 2, 2, out)
    assert _rel(S, oracle.homogenised_stress(ph, par, F)) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    rve.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    # 512^3 voxels exceed the 256^3 capacity of the static scratch: rejected before any launch
    assert rve.rve_stress_noalloc(3, 512, rve.RVE_NEOHOOKE, p, p, p, 2, 2, p) == rve.RVE_E_INVALID_ARG
    assert rve.rve_stress_noalloc(3, 16, rve.RVE_NEOHOOKE, 0, p, p, 2, 2, p) == rve.RVE_E_INVALID_ARG
