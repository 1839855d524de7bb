"""Pins of the strict-mode polynomial log/exp/sincos(2 pi u) against libm (numpy float64).

The toy model defines these functions as explicit FP32 polynomial evaluations
(so CPU and GPU agree bit for bit); here they are held to a stated error bound
against correctly rounded FP64 references, over the input ranges the model uses.
"""
import numpy as np

import oracle


def _ulp_err(approx32, exact64):
    exact32 = exact64.astype(np.float32)
    spacing = np.spacing(np.abs(exact32)).astype(np.float64)
    return np.abs(approx32.astype(np.float64) - exact64) / spacing


def _all_floats(lo, hi, stride):
    a = np.array([lo], np.float32).view(np.uint32)[0]
    b = np.array([hi], np.float32).view(np.uint32)[0]
    return np.arange(a, b, stride, dtype=np.uint32).view(np.float32)


def test_spec_log_error_bound():
    # arguments in use: uniforms in [2^-24, 1] and energies in [1e-2, 1e5] MeV
    x = _all_floats(2.0 ** -24, 2.0 ** 17, 97)
    y = oracle.spec_log(x)
    ref = np.log(x.astype(np.float64))
    nz = np.abs(ref) > 1e-3
    err = _ulp_err(y[nz], ref[nz])
    assert err.max() <= 2.0, err.max()
    # near 1 the absolute error matters
    assert np.max(np.abs(y[~nz] - ref[~nz])) < 2e-10
    assert oracle.spec_log(np.array([1.0]))[0] == 0.0
    assert oracle.spec_log(np.array([2.0]))[0] == np.float32(np.log(2.0))


def test_spec_exp_error_bound():
    small = _all_floats(1e-6, 1.0, 1013)
    x = np.concatenate([np.linspace(-87.0, 88.0, 2_000_003, dtype=np.float32), -small, small])
    y = oracle.spec_exp(x)
    ref = np.exp(x.astype(np.float64))
    normal = ref > 1.2e-38
    err = _ulp_err(y[normal], ref[normal])
    assert err.max() <= 2.0, err.max()
    assert oracle.spec_exp(np.array([0.0]))[0] == 1.0
    assert oracle.spec_exp(np.array([-100.0]))[0] == 0.0
    assert np.isinf(oracle.spec_exp(np.array([100.0]))[0])


def test_spec_sincos2pi_error_bound():
    u = np.concatenate([np.arange(1, 1 << 24, 7, dtype=np.float64) * 2.0 ** -24, [1.0]])
    u = u.astype(np.float32)
    s, c = oracle.spec_sincos2pi(u)
    a = 2 * np.pi * u.astype(np.float64)
    assert np.max(np.abs(s - np.sin(a))) < 3e-7
    assert np.max(np.abs(c - np.cos(a))) < 3e-7
    assert np.max(np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1)) < 1e-6
    # exact quadrant points
    s4, c4 = oracle.spec_sincos2pi(np.array([0.25, 0.5, 0.75, 1.0], np.float32))
    assert list(s4) == [1.0, 0.0, -1.0, 0.0]
    assert list(np.abs(c4)) == [0.0, 1.0, 0.0, 1.0]
    assert c4[1] == -1.0 and c4[3] == 1.0
