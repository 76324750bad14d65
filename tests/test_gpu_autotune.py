"""FFT autotuner: the tuned geometry is used by later handles and keeps parity."""
import os

import numpy as np
import pytest

import oracle
from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
PAR = synth.two_phase_params(1.0, 10.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


@pytest.mark.parametrize("dim,n,precision", [(3, 24, "fp64"), (2, 96, "fp64"), (3, 48, "mixed")])
def test_autotuned_geometry_keeps_parity(dim, n, precision, tmp_path):
    import json
    cache = str(tmp_path / "fft.jsonl")
    ms = rve.rve_autotune(dim, n, precision, cache)
    assert ms > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["kind"] == "rve-fft-geometry" and rec["dim"] == dim and rec["n"] == n
    assert rve.rve_autotune_load(cache) == 1
    ph = synth.inclusion_phase(n, dim, 3, radius=3)
    Fbar = np.diag([0.95, 1.03, 1.0])
    s = rve.Rve(dim, n, "neohookean", "fp64", max_iter=3)
    s.set_material(ph, PAR)
    s.solve(Fbar, 10.0, -1.0)
    ref = oracle.admm_solve(ph, PAR, Fbar, 10.0, -1.0, 3)
    F = s.get_field(rve.RVE_FIELD_F)
    assert np.max(np.abs(F - ref["F"])) / np.max(np.abs(ref["F"])) < 1e-10
