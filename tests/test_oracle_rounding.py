"""Pins of the oracle's age storage rounding (Section 5.7: fp32 math, cast on
store, round to nearest even). binary16 is checked exhaustively against
numpy's float32 -> float16 conversion, bfloat16 against torch's CPU
conversion, both independent implementations of IEEE round-to-nearest-even.
"""
import numpy as np
import pytest
import torch


def test_f16_rounding_exhaustive_against_numpy(oracle_mod):
    # every finite binary16 value as an age, plus the step added in float32
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float32)
    for dt in (0.1, 0.05, 0.25, 0.0333):
        ref = (h + np.float32(dt)).astype(np.float16).astype(np.float32)
        got = np.array([oracle_mod.age_next(float(a), dt, oracle_mod.AGE_F16) for a in h], dtype=np.float32)
        np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_f16_bits_random_floats_against_numpy(oracle_mod):
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(0, 70000, 20000).astype(np.float32),
        (rng.uniform(0, 1, 20000) * 2.0 ** rng.integers(-30, -10, 20000)).astype(np.float32),
        np.array([65504, 65519.99, 65520, 2.0 ** -24, 2.0 ** -25, 2.0 ** -25 * 1.0001, 0.0], dtype=np.float32),
    ])
    x = np.concatenate([x, -x])
    ref = x.astype(np.float16).view(np.uint16)
    got = np.array([oracle_mod.f16_bits(float(v)) for v in x], dtype=np.uint16)
    np.testing.assert_array_equal(got, ref)


def test_bf16_rounding_against_torch(oracle_mod):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(0, 200, 30000), rng.uniform(0, 1e-3, 5000),
                        np.arange(0, 1000, dtype=np.float64) / 8 + 1 / 512]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle_mod.bf16_bits(float(v)) for v in x], dtype=np.uint16)
    np.testing.assert_array_equal(got, ref)
    # bf16 ages: fp32 add then round (ulp 0.25 above 32 d freezes a 0.1 d step)
    a = np.float32(0)
    seq = []
    for _ in range(600):
        a = np.float32(oracle_mod.age_next(float(a), 0.1, oracle_mod.AGE_BF16))
        seq.append(a)
    tref = torch.zeros((), dtype=torch.bfloat16)
    for s in seq:
        tref = (tref.float() + torch.tensor(0.1, dtype=torch.float32)).to(torch.bfloat16)
        assert float(tref) == float(s)
    assert max(seq) == 32.0


def test_f32_age_is_one_single_add(oracle_mod):
    a = np.float32(0)
    for _ in range(3000):
        nxt = oracle_mod.age_next(float(a), 0.1, oracle_mod.AGE_F32)
        assert np.float32(nxt) == np.float32(a) + np.float32(0.1)
        a = np.float32(nxt)
