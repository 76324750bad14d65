"""r_d of the float phase from the spectral solve (Parseval) against the u~ stencil.

In the float phase of RVE_MIXED on 3D grids of 128 and 256 (neo-Hookean law, exact
local steps) the z pass keeps the solved spectrum and sums |k|^2 |u^_{k+1} - u^_k|^2,
and the local pass takes r_d = (rho/mu) ||G_{k+1} - G_k|| from that sum (Section 2.1,
eq. check; the discrete Parseval identity of the central-difference gradient).  An
RVE_FP32 handle runs the same float kernels but forms r_d from the u~_k stencil.  r_d
does not feed back into the iterates at fixed rho (no switch within these
iterations), so both handles follow the same iterates bit for bit, r_p is identical,
and the two r_d agree to float rounding of the two summation orders."""
import numpy as np
import pytest

from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


@pytest.mark.parametrize("n", [128, 256])
def test_spectral_rd_equals_stencil_rd(n):
    iters = 12
    ph = synth.inclusion_phase(n, 3, 0)
    par = synth.two_phase_params(1.0, 10.0)
    Fbar = np.diag([0.9, 1.0, 1.0])
    out = {}
    for prec in ("mixed", "fp32"):
        s = rve.Rve(3, n, "neohookean", prec, max_iter=iters)
        s.set_material(ph, par)
        info = s.solve(Fbar, 10.0, -1.0)
        assert info.iterations == iters and info.fp64_iterations == 0, info.as_dict()
        out[prec] = (s.history()[:iters, :2].copy(), s.get_field(rve.RVE_FIELD_F))
        s.close()
    (hm, Fm), (hf, Ff) = out["mixed"], out["fp32"]
    assert np.array_equal(Fm, Ff)                  # same iterates
    assert np.array_equal(hm[:, 0], hf[:, 0])      # r_p from the same voxel sums
    assert hm[0, 1] == hf[0, 1]                    # first check of a solve: no kept spectrum yet
    np.testing.assert_allclose(hm[1:, 1], hf[1:, 1], rtol=2e-5)
    assert not np.array_equal(hm[1:, 1], hf[1:, 1])  # the spectral sums were used
