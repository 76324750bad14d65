"""The pins bite: each plausible mistake planted in the oracle (on the CPU, by
monkeypatching) makes at least one pin of tests/test_oracle_pins.py fail."""
import numpy as np
import pytest

from oracle import admm as oadmm
from oracle import materials as omat
from tests import test_oracle_pins as pins


def _transposed_gradient(uh):
    g = _orig_grad(uh)
    return np.swapaxes(g, 0, 1).copy()


_orig_grad = oadmm.grad_from_spectrum
_orig_u_step = oadmm.u_step
_orig_wavenumbers = oadmm.wavenumbers


def _u_step_no_multiplier(F, Lam, rho):
    return _orig_u_step(F, np.zeros_like(Lam), rho)


def _u_step_wrong_sign(F, Lam, rho):
    return _orig_u_step(F, -Lam, rho)


def _continuum_symbol(n, dim):
    m = np.fft.fftfreq(n) * n
    k = 2 * np.pi * m
    out = []
    for j in range(dim):
        shape = [1] * dim
        shape[dim - 1 - j] = n
        out.append(k.reshape(shape))
    return out


class _NHWrongTangent(omat.NeoHookean):
    def C(self, F):
        return super().C(F).transpose(0, 1, 2, 4, 3)


class _NHWrongStress(omat.NeoHookean):
    def P(self, F):
        A = np.linalg.inv(F).transpose(0, 2, 1)
        J = np.linalg.det(F)
        c = self.lam * J * (J - 1.0) + self.mu          # sign of the mu term flipped
        return self.mu[:, None, None] * F + c[:, None, None] * A


MUTATIONS = {
    "transposed_gradient": [("grad_from_spectrum", _transposed_gradient)],
    "u_step_drops_multiplier": [("u_step", _u_step_no_multiplier)],
    "u_step_multiplier_sign": [("u_step", _u_step_wrong_sign)],
    "continuum_symbol": [("wavenumbers", _continuum_symbol)],
}

PIN_CALLS = [
    lambda: pins.test_poisson_recovers_manufactured_displacement(2, 16),
    lambda: pins.test_poisson_equals_dense_least_squares(2, 4),
    lambda: pins.test_linear_laminate_closed_form(2, 16),
    lambda: pins.test_invariants_every_iteration(),
    lambda: pins.test_neohookean_laminate_3d_sheared(),
]


def _some_pin_fails():
    for call in PIN_CALLS:
        try:
            call()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_in_iteration_is_caught(name, monkeypatch):
    for attr, fn in MUTATIONS[name]:
        monkeypatch.setattr(oadmm, attr, fn)
    assert _some_pin_fails(), name


def test_multiplier_update_sign_is_caught(monkeypatch):
    """Lambda_{i+1} = Lambda_i - rho (G - F) instead of +: the laminate pin fails."""
    monkeypatch.setattr(oadmm, "multiplier_update", lambda Lam, G, F, rho: Lam - rho * (G - F))
    d, n = 2, 16
    ph = pins.synth.laminate_phase(n, d)
    par = pins.synth.two_phase_params(1.0, 10.0)
    Fbar3 = np.diag([1.05, 0.98, 1.0])
    _, _, S = pins._laminate_exact("linear", par, Fbar3[:d, :d])
    r = oadmm.admm_solve(ph, par, Fbar3, 10.0, 1e-13, 150, model="linear")
    assert not r["converged"]
    assert not np.allclose(r["stress"], S, atol=1e-10)


@pytest.mark.parametrize("cls", [_NHWrongTangent, _NHWrongStress])
def test_mutation_in_constitutive_law_is_caught(cls, monkeypatch):
    monkeypatch.setitem(omat.MODELS, "neohookean", cls)
    with pytest.raises(AssertionError):
        pins.test_stress_and_tangent_match_numerical_derivatives("neohookean", 3)
