"""The device primitives against the oracle's own implementations, bit for bit: Philox on
a million counters and keys, the u01 map on its full input range, and the strict model's
log, exp and sincos(2 pi u) on every value the transport can feed them from a uniform
draw (all 2^24 outputs of u01) plus wide random samples.  The two sides are written
independently (the oracle in C, the device code in CUDA) from the same definitions."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _eval(what, x, out_shape, out_dtype):
    import torch
    from paper_2302_08252_gb300 import et
    out = torch.empty(out_shape, dtype=out_dtype, device="cuda")
    et.et_debug_eval(what, _dev(x), out)
    return out.cpu().numpy()


def test_philox_matches_oracle():
    import torch
    from paper_2302_08252_gb300 import et
    rng = np.random.Generator(np.random.Philox(key=11))
    for key in [(0, 0), (1, 0), (0xFFFFFFFF, 0xFFFFFFFF), tuple(rng.integers(0, 2**32, 2))]:
        ctr = rng.integers(0, 2**32, size=(1 << 18, 4), dtype=np.uint64).astype(np.uint32)
        ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
        inp = np.concatenate([ctr, np.tile(np.array(key, np.uint32), (len(ctr), 1))], axis=1)
        got = _eval(et.EVAL_PHILOX, inp, (len(ctr), 4), torch.int32).view(np.uint32)
        np.testing.assert_array_equal(got, oracle.philox(ctr, key))


def test_u01_and_strict_math_on_every_uniform():
    import torch
    from paper_2302_08252_gb300 import et
    # every 32-bit input in steps of 2^8 (u01 ignores the low 8 bits), i.e. all 2^24 outputs
    x = (np.arange(1 << 24, dtype=np.uint64) << 8).astype(np.uint32)
    u = _eval(et.EVAL_U01, x, (len(x),), torch.float32)
    ref = np.array([oracle.u01(int(v)) for v in x[:: 1 << 12]], dtype=np.float32)
    np.testing.assert_array_equal(u[:: 1 << 12], ref)
    np.testing.assert_array_equal(u, ((x >> 8).astype(np.float64) + 1.0).astype(np.float32) * np.float32(2.0 ** -24))
    got = _eval(et.EVAL_LOG, u, (len(u),), torch.float32)
    np.testing.assert_array_equal(got.view(np.uint32), oracle.spec_log(u).view(np.uint32))
    sc = _eval(et.EVAL_SINCOS2PI, u, (len(u), 2), torch.float32)
    s, c = oracle.spec_sincos2pi(u)
    np.testing.assert_array_equal(sc[:, 0].view(np.uint32), s.view(np.uint32))
    np.testing.assert_array_equal(sc[:, 1].view(np.uint32), c.view(np.uint32))


def test_strict_log_exp_on_wide_samples():
    import torch
    from paper_2302_08252_gb300 import et
    rng = np.random.Generator(np.random.Philox(key=12))
    # log: positive normal floats of every exponent, plus the energies the tables span
    bits = rng.integers(0x00800000, 0x7F800000, size=1 << 22, dtype=np.uint64).astype(np.uint32)
    e = np.exp(rng.uniform(np.log(1e-3), np.log(1e5), 1 << 20)).astype(np.float32)
    xs = np.concatenate([bits.view(np.float32), e, np.float32([1.0, 2.0, 0.5, 1e-3, 1e5])])
    got = _eval(et.EVAL_LOG, xs, (len(xs),), torch.float32)
    np.testing.assert_array_equal(got.view(np.uint32), oracle.spec_log(xs).view(np.uint32))
    # exp: the arguments the model forms (-a1 u in Compton sampling, u ln(T/k_c) in brems)
    # and the rest of the finite range
    ys = np.concatenate([rng.uniform(-20.0, 0.0, 1 << 21), rng.uniform(0.0, 20.0, 1 << 21),
                         rng.uniform(-87.0, 88.0, 1 << 20)]).astype(np.float32)
    ys = np.concatenate([ys, np.float32([0.0, -0.0, 1.0, -1.0])])
    got = _eval(et.EVAL_EXP, ys, (len(ys),), torch.float32)
    np.testing.assert_array_equal(got.view(np.uint32), oracle.spec_exp(ys).view(np.uint32))
