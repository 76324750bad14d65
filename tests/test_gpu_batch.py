"""Batched solves of uneven RVEs (one persistent launch per pass over a tile table):
each member's result is bitwise the same as solving it alone, and matches the oracle."""
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


def members(specs, precision, max_iter=600, **opt):
    out = []
    for dim, n, kind, seed in specs:
        model = "lce" if kind == "lce" else "neohookean"
        s = rve.Rve(dim, n, model, precision, max_iter=max_iter, **opt)
        if kind == "lce":
            ph = np.zeros((n,) * 3, np.uint8)
            s.set_material(ph, np.array([[1.0, 20.0, 4.0, 0.1, (2.0 / n) ** 2]]), synth.director_grf(n, seed, 3.0))
        else:
            ph = synth.laminate_phase(n, dim) if kind == "laminate" else synth.inclusion_phase(n, dim, seed, radius=3)
            s.set_material(ph, PAR)
        out.append(s)
    return out


def fbars(count, seed):
    return np.stack([synth.random_fbar(seed + i, 7, amp=0.06) for i in range(count)])


SPECS = [(3, 12, "inclusion", 1), (3, 16, "laminate", 2), (3, 24, "inclusion", 3), (2, 32, "inclusion", 4),
         (3, 18, "inclusion", 5), (2, 48, "laminate", 6), (3, 8, "inclusion", 7)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_members_equal_alone_solves_bitwise(precision):
    Fb = fbars(len(SPECS), 40)
    rho = np.full(len(SPECS), 10.0)
    alone = members(SPECS, precision)
    ref = []
    for s, F in zip(alone, Fb):
        info = s.solve(F, 10.0, 1e-8)
        ref.append((info.iterations, info.converged, s.state(), s.stress()))
    mix = members(SPECS, precision)
    b = rve.Batch(mix)
    infos = b.solve(Fb, rho, 1e-8)
    for s, info, (it, conv, st, S) in zip(mix, infos, ref):
        assert info.iterations == it and bool(info.converged) == conv
        st2 = s.state()
        for k in st:
            assert np.array_equal(st2[k], st[k]), (k, s.dim, s.n)
        assert np.array_equal(s.stress(), S)


def test_batch_mixed_adaptive_members_equal_alone_solves():
    """RVE_MIXED with the adaptive penalty in a batch: rho is frozen at each member's switch
    to double and the members take the increment polish; results equal the alone solves
    bitwise and converge."""
    specs = SPECS[:4]
    Fb = fbars(len(specs), 60)
    alone = members(specs, "mixed", rho_policy="adaptive")
    ref = []
    for s, F in zip(alone, Fb):
        info = s.solve(F, 30.0, 1e-8)
        ref.append((info.iterations, info.fp64_iterations, info.converged, s.stress()))
    mix = members(specs, "mixed", rho_policy="adaptive")
    infos = rve.Batch(mix).solve(Fb, np.full(len(specs), 30.0), 1e-8)
    for s, info, (it, it64, conv, S) in zip(mix, infos, ref):
        assert conv and info.converged
        assert info.iterations == it and info.fp64_iterations == it64
        assert np.array_equal(s.stress(), S)


def test_batch_with_lce_and_neohookean_groups():
    """Two model groups (neo-Hookean, LCE) in one batch, fixed iteration count."""
    specs = [(3, 12, "inclusion", 1), (3, 12, "lce", 2), (3, 16, "lce", 3), (3, 16, "laminate", 4)]
    Fb = fbars(len(specs), 50)
    alone = members(specs, "fp64", max_iter=7)
    ref = []
    for s, F in zip(alone, Fb):
        s.solve(F, 10.0, -1.0)
        ref.append(s.state())
    mix = members(specs, "fp64", max_iter=7)
    infos = rve.Batch(mix).solve(Fb, np.full(len(specs), 10.0), -1.0)
    for s, info, st in zip(mix, infos, ref):
        assert info.iterations == 7
        st2 = s.state()
        for k in st:
            assert np.array_equal(st2[k], st[k]), k


def test_batch_members_match_oracle():
    specs = [(3, 12, "inclusion", 11), (2, 24, "laminate", 12), (3, 16, "inclusion", 13)]
    Fb = fbars(len(specs), 60)
    mix = members(specs, "fp64", max_iter=6)
    infos = rve.Batch(mix).solve(Fb, np.array([10.0, 7.0, 12.0]), -1.0)
    for (dim, n, kind, seed), s, F, rho in zip(specs, mix, Fb, [10.0, 7.0, 12.0]):
        ph = synth.laminate_phase(n, dim) if kind == "laminate" else synth.inclusion_phase(n, dim, seed, radius=3)
        ref = oracle.admm_solve(ph, PAR, F, rho, -1.0, 6)
        F_gpu = s.get_field(rve.RVE_FIELD_F)
        assert np.max(np.abs(F_gpu - ref["F"])) / np.max(np.abs(ref["F"])) < 1e-10
        assert np.max(np.abs(s.stress() - ref["stress"])) / np.max(np.abs(ref["stress"])) < 1e-10


def test_batch_rejects_mixed_precision_and_duplicates():
    a = members([(3, 8, "inclusion", 1)], "fp64")[0]
    c = members([(3, 8, "inclusion", 1)], "mixed")[0]
    rc, _ = rve.rve_batch_create([a.h, c.h])
    assert rc == rve.RVE_E_INVALID_ARG
    rc, _ = rve.rve_batch_create([a.h, a.h])
    assert rc == rve.RVE_E_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uniform_batch_fixed_length_kernels_bitwise(precision):
    """Three 128^3 members (one grid size: the batched passes take the fixed-length FFT
    kernels, as a single handle does): bitwise equal to solving each alone."""
    specs = [(3, 128, "inclusion", 11), (3, 128, "laminate", 12), (3, 128, "inclusion", 13)]
    Fb = fbars(len(specs), 50)
    alone = members(specs, precision, max_iter=60)
    ref = []
    for s, F in zip(alone, Fb):
        s.solve(F, 10.0, -1.0)
        ref.append((s.state(), s.stress()))
        s.close()
    mix = members(specs, precision, max_iter=60)
    rve.Batch(mix).solve(Fb, np.full(len(specs), 10.0), -1.0)
    for s, (st, S) in zip(mix, ref):
        st2 = s.state()
        for k in st:
            assert np.array_equal(st2[k], st[k]), k
        assert np.array_equal(s.stress(), S)
