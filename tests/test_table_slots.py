"""The memoised probability tables of the step hold two (age, p) slots per
index rint(age / dt): enough for every fixed-step age sequence the storage
types produce. Checked here from the sequences themselves (FP32 add, then
round-to-nearest-even to the storage type, numpy's casts), independently of
the library: at most two distinct ages share an index, and FP16 / BF16
storage does produce shared indices, so the second slot is used."""
import numpy as np
import pytest
import torch


def age_sequence(dt: float, dtype: str, steps: int = 4096) -> np.ndarray:
    out = np.empty(steps, dtype=np.float32)
    v = np.float32(0.0)
    d = np.float32(dt)
    for n in range(steps):
        out[n] = v
        s = np.float32(v + d)
        if dtype == "f16":
            s = np.float32(np.float16(s))
        elif dtype == "bf16":
            s = np.float32(torch.tensor(float(s), dtype=torch.float32).to(torch.bfloat16).item())
        v = s
    return out


def index_of(ages: np.ndarray, dt: float) -> np.ndarray:
    inv = np.float32(1.0 / dt)
    return np.rint((ages * inv).astype(np.float32)).astype(np.int64)   # FP32 product, half to even


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dt", [0.1, 0.05, 0.25, 0.0333, 0.2])
def test_at_most_two_distinct_ages_per_index(dtype, dt):
    ages = age_sequence(dt, dtype)
    assert np.all(np.diff(ages) >= 0)                  # monotone: same-index ages are consecutive
    idx = index_of(ages, dt)
    distinct = {}
    for a, i in zip(ages.tolist(), idx.tolist()):
        distinct.setdefault(i, set()).add(a)
    assert max(len(v) for v in distinct.values()) <= 2


def test_reduced_precision_sequences_share_indices():
    shared = {}
    for dtype in ("f32", "f16", "bf16"):
        ages = age_sequence(0.1, dtype)
        idx = index_of(ages, 0.1)
        per = {}
        for a, i in zip(ages.tolist(), idx.tolist()):
            per.setdefault(i, set()).add(a)
        shared[dtype] = sum(1 for v in per.values() if len(v) == 2)
    assert shared["f32"] == 0
    assert shared["f16"] > 0 and shared["bf16"] > 0
