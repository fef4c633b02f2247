"""Planted mistakes in the FP64 oracle (CPU only): each pin must fail on the mistake it is
there to catch.  The mistakes are swapped in with monkeypatch for one call and never touch
the CUDA path."""
import numpy as np
import pytest

from oracle import dual
from tests import test_oracle_pins as pins


def _fails(fn, *a):
    with pytest.raises(AssertionError):
        fn(*a)


def _nesterov_gradient_at_nu(P, h, st, beta, lhat):
    """Mistake: the Alg. 2 gradient taken at nu instead of eta."""
    th = st.theta
    res = dual.region_pass(P, h, st.nu, "smooth", beta=beta)
    st.zeta = st.zeta + res.grad / (th * lhat)
    st.nu = (1.0 - th) * st.nu + th * st.zeta
    st.theta = dual.next_theta(th)
    st.t += 1
    return res


def _plain_gradient_ascent(P, h, st, beta, lhat):
    """Mistake: no acceleration, nu += g / L_hat."""
    res = dual.region_pass(P, h, st.nu, "smooth", beta=beta)
    st.nu = st.nu + res.grad / lhat
    st.zeta = st.nu.copy()
    st.t += 1
    return res


def _nu_update_with_old_zeta(P, h, st, beta, lhat):
    """Mistake: nu = (1 - theta) nu + theta zeta uses zeta^(k) instead of zeta^(k+1)."""
    th = st.theta
    eta = (1.0 - th) * st.nu + th * st.zeta
    res = dual.region_pass(P, h, eta, "smooth", beta=beta)
    old = st.zeta
    st.zeta = st.zeta + res.grad / (th * lhat)
    st.nu = (1.0 - th) * st.nu + th * old
    st.theta = dual.next_theta(th)
    st.t += 1
    return res


@pytest.mark.parametrize("mistake", [_nesterov_gradient_at_nu, _plain_gradient_ascent, _nu_update_with_old_zeta])
def test_nesterov_hand_pin_catches(monkeypatch, mistake):
    monkeypatch.setattr(dual, "nesterov_step", mistake)
    _fails(pins.test_nesterov_three_steps_by_hand)


def test_rate_pin_catches_plain_gradient_ascent(monkeypatch):
    monkeypatch.setattr(dual, "nesterov_step", _plain_gradient_ascent)
    _fails(pins.test_nesterov_rate_of_the_accelerated_corollary)


@pytest.mark.parametrize("rule", [lambda a, t: a / (t + 1.0), lambda a, t: a, lambda a, t: a / np.sqrt(t + 2.0)])
def test_step_rule_pin_catches(monkeypatch, rule):
    orig = dual.step_size
    monkeypatch.setattr(dual, "step_size", lambda r, a, t: rule(a, t) if r == "sqrt" else orig(r, a, t))
    _fails(pins.test_subgradient_inv_sqrt_steps_by_hand)


def _lowest_only(lam, theta, tol):
    """Mistake: the lowest eigenvector alone, even inside a degenerate ground space."""
    w = np.zeros_like(lam)
    w[..., 0] = 1.0
    return w


def _all_below_mean(lam, theta, tol):
    """Mistake: a mixture over every eigenvalue below the mean."""
    m = lam <= lam.mean(axis=-1, keepdims=True)
    return m / m.sum(axis=-1, keepdims=True)


@pytest.mark.parametrize("mistake", [_lowest_only, _all_below_mean])
def test_ground_mixture_pin_catches(monkeypatch, mistake):
    monkeypatch.setattr(dual, "ground_weights", mistake)
    caught = 0
    for spectrum, mult in [((-1, -1, 1, 1), 2), ((-2, -2, -2, 0.5), 3), ((-1, 0, 0.5, 2), 1)]:
        try:
            pins.test_ground_mixture_is_the_normalised_ground_projector(spectrum, mult)
        except AssertionError:
            caught += 1
    assert caught >= 1


def test_embedding_sign_caught_by_hand_pins(monkeypatch):
    """Mistake: theta_e = h_e + sum_children 1 (x) nu (wrong sign of the child embedding)."""
    orig = dual.embed
    monkeypatch.setattr(dual, "embed", lambda op, pos, k, d=2: -orig(op, pos, k, d))
    _fails(pins.test_nesterov_three_steps_by_hand)
    _fails(pins.test_subgradient_inv_sqrt_steps_by_hand)


def test_partial_trace_transpose_caught(monkeypatch):
    """Mistake: the partial trace returned transposed (wrong for complex Hermitian states)."""
    orig = dual.partial_trace
    monkeypatch.setattr(dual, "partial_trace", lambda r, keep, k, d=2: np.swapaxes(orig(r, keep, k, d), -1, -2))
    _fails(pins.test_partial_trace_is_adjoint_of_embedding)
