"""rve_stress_noalloc: the homogenised stress for callers that cannot allocate
device memory (their device memory is owned by a pool they may not grow, or they
run in loops where cudaMalloc's possible device synchronisation is not allowed).
Its result must equal rve_stress on the same field, call after call, although
every call reuses the same static device scratch array.

This file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dim,n,model", [(3, 16, "neohookean"), (2, 32, "neohookean"), (3, 12, "linear")])
def test_noalloc_stress_matches_rve_stress_twice(dim, n, model):
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
    # the caller's own device buffers (here provided by torch)
    F_dev = torch.from_numpy(np.ascontiguousarray(F).reshape(-1)).cuda()
    ph_dev = torch.from_numpy(np.ascontiguousarray(ph).reshape(-1)).cuda()
    par_dev = torch.from_numpy(np.ascontiguousarray(par).reshape(-1)).cuda()
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(float("nan"))
        rc = rve.rve_stress_noalloc(dim, n, rve.MODELS[model], F_dev.data_ptr(), ph_dev.data_ptr(),
                                    par_dev.data_ptr(), par.shape[0], par.shape[1], out.data_ptr(), stream)
        assert rc == rve.RVE_OK, rve.rve_strerror(rc)
        torch.cuda.synchronize()
        S = out.cpu().numpy().reshape(3, 3)
        assert _rel(S[:dim, :dim], S_ref) < TOL, (call, S, S_ref)
        assert np.all(S[dim:, :] == 0.0) and np.all(S[:, dim:] == 0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    rve.lib()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    # 512^3 voxels exceed the 256^3 capacity of the static scratch: rejected before any launch
    assert rve.rve_stress_noalloc(3, 512, rve.RVE_NEOHOOKE, p, p, p, 2, 2, p) == rve.RVE_E_INVALID_ARG
    assert rve.rve_stress_noalloc(3, 16, rve.RVE_NEOHOOKE, 0, p, p, 2, 2, p) == rve.RVE_E_INVALID_ARG
