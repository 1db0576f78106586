"""Pins of the oracle's S4 discretisation that do not lean on its own formula.

The oracle discretises every diagonal mode with the bilinear (trapezoidal) rule of
App. "Details on the implementation of the DysonNet block", Eq. discretization:
lam_bar = (1 + dt Lam / 2) / (1 - dt Lam / 2), B_bar = dt B / (1 - dt Lam / 2), and the
forward taps of one mode are B_bar lam_bar^r (r >= 0).  Every other tap pin reuses the
same discretisation, so two facts about the trapezoidal rule are checked here from
the taps alone, with expected values that come from the continuous system:

  * DC gain.  The discrete response sums to the continuous one for every step size:
    sum_{r >= 0} B_bar lam_bar^r = B_bar / (1 - lam_bar) = -B / Lam.  This fails if
    the 1 / (1 - dt Lam / 2) of B_bar is lost, or if lam_bar is taken from another rule
    while B_bar keeps the trapezoidal form.
  * Order of accuracy.  lam_bar is the (1,1) Pade approximant of exp(z), z = dt Lam, so
    lam_bar - exp(z) = z^3 / 12 + z^4 / 12 + O(z^5).  Zero-order hold (lam_bar = exp(z)),
    forward Euler (1 + z) or backward Euler (1 / (1 - z)) give other limits.

A mode is read back as complex numbers by running the oracle twice, with C = 1 and
C = -i (Re(-i x) = Im x).  The same checks are applied to deliberately edited copies
of the discretisation, computed here in numpy, and must reject every one of them.
"""
import cmath

import numpy as np
import pytest

import oracle
from synth import ModelDesc

_DESC = ModelDesc(L=1, d=1, s=1, w=0, dh=1, dout=1, periodic=0, fkind=0)


def _block(lam, dt, B, cf, cb):
    """S4 parameter block of one channel with one mode: lam, log dt, B, C_fwd, C_bwd."""
    lam, B, cf, cb = complex(lam), complex(B), complex(cf), complex(cb)
    return np.array([lam.real, lam.imag, np.log(dt), B.real, B.imag, cf.real, cf.imag, cb.real, cb.imag])


def _oracle_taps(lam, dt, B, cf, cb, N):
    return oracle.s4_taps(_DESC, _block(lam, dt, B, cf, cb), N, periodic=False)[:, 0]


def _edited_taps(rule):
    """Open-chain taps of one mode with a replaced discretisation `rule(z, dt, B)`."""

    def taps(lam, dt, B, cf, cb, N):
        lb, bb = rule(dt * complex(lam), dt, complex(B))
        g = np.zeros(2 * N - 1)
        for r in range(-(N - 1), N):
            c = cf if r >= 0 else cb
            g[r + N - 1] = (complex(c) * bb * lb ** abs(r)).real
        return g

    return taps


_RULES = {
    "trapezoidal (reference copy)": lambda z, dt, B: ((1 + z / 2) / (1 - z / 2), dt * B / (1 - z / 2)),
    "B_bar without 1/(1 - z/2)": lambda z, dt, B: ((1 + z / 2) / (1 - z / 2), dt * B),
    "zero-order-hold lam_bar, trapezoidal B_bar": lambda z, dt, B: (cmath.exp(z), dt * B / (1 - z / 2)),
    "zero-order hold": lambda z, dt, B: (cmath.exp(z), (cmath.exp(z) - 1) / (z / dt) * B),
    "forward Euler": lambda z, dt, B: (1 + z, dt * B),
    "backward Euler": lambda z, dt, B: (1 / (1 - z), dt * B / (1 - z)),
}

# Modes with Re Lam < 0: real, S4D-Lin-like and strongly oscillating.
_MODES = [(-0.5, 1.0), (-0.5 + 1j * np.pi, 0.3 - 0.7j), (-2.0 + 5.0j, -1.1 + 0.4j)]


def _forward_complex(taps, lam, dt, B, N):
    """B_bar lam_bar^r for r = 0..N-1 as complex numbers (forward direction only)."""
    re = taps(lam, dt, B, 1.0, 0.0, N)[N - 1:]
    im = taps(lam, dt, B, -1j, 0.0, N)[N - 1:]
    return re + 1j * im


def _dc_gain_error(taps):
    """max over modes and steps of |sum_r B_bar lam_bar^r - (-B/Lam)| / |B/Lam|."""
    worst = 0.0
    for lam, B in _MODES:
        for dt in (0.05, 0.2, 1.0, 3.0):
            N = 4000
            t = _forward_complex(taps, lam, dt, B, N)
            if not abs(t[-1]) < 1e-20 * abs(t[0]):
                return np.inf   # the response does not decay: no finite gain
            want = -complex(B) / complex(lam)
            worst = max(worst, abs(t.sum() - want) / abs(want))
    return worst


def _third_order_error(taps):
    """max over modes and small steps of |(lam_bar - e^z)/z^3 - (1 + z)/12| / |z|^2."""
    worst = 0.0
    for lam, B in _MODES:
        for dt in (2e-3, 5e-3, 1e-2):
            t = _forward_complex(taps, lam, dt, B, 3)
            lb = t[1] / t[0]
            z = dt * complex(lam)
            dev = (lb - cmath.exp(z)) / z**3 - (1 + z) / 12
            worst = max(worst, abs(dev) / abs(z) ** 2)
    return worst


def test_dc_gain_of_oracle_taps_equals_continuous_gain():
    assert _dc_gain_error(_oracle_taps) < 1e-11


def test_oracle_lam_bar_is_third_order_pade_of_exponential():
    # (lam_bar - e^z)/z^3 = 1/12 + z/12 + c z^2 + ..., |c| < 0.06; rounding adds < 1e-6 here.
    assert _third_order_error(_oracle_taps) < 0.5


def test_backward_direction_excludes_lag_zero_and_sums_to_the_same_gain():
    # r = 0 comes from the forward output only; the backward taps are B_bar lam_bar^|r|,
    # so the backward sum is the continuous gain minus the forward lag-0 tap B_bar.
    for lam, B in _MODES:
        dt, N = 0.2, 3000
        bwd_re = _oracle_taps(lam, dt, B, 0.0, 1.0, N)
        bwd_im = _oracle_taps(lam, dt, B, 0.0, -1j, N)
        bwd = bwd_re[:N] + 1j * bwd_im[:N]           # rows r = -(N-1) .. 0
        assert bwd[N - 1] == 0.0
        fwd = _forward_complex(_oracle_taps, lam, dt, B, N)
        want = -complex(B) / complex(lam) - fwd[0]
        assert abs(bwd.sum() - want) < 1e-11 * abs(want)


def test_reference_copy_of_the_rule_passes_the_same_checks():
    taps = _edited_taps(_RULES["trapezoidal (reference copy)"])
    assert _dc_gain_error(taps) < 1e-11
    assert _third_order_error(taps) < 0.5


@pytest.mark.parametrize("rule", [k for k in _RULES if k != "trapezoidal (reference copy)"])
def test_edited_rules_are_rejected(rule):
    taps = _edited_taps(_RULES[rule])
    dc, third = _dc_gain_error(taps), _third_order_error(taps)
    assert dc > 1e-6 or third > 10.0, (rule, dc, third)
