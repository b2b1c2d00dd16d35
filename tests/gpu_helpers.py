"""Helpers shared by the GPU parity tests: the lock-step trajectory protocol.

Lock-step: at every step the oracle is fed the GPU's own state, and its next
state is compared node by node with the GPU's next state. A node may differ
only where the Bernoulli decision was a near-tie (|u - p| < 1e-6, with p from
the oracle's double-precision hazard); such mismatches are counted and must
stay at or below 1e-6 of all Bernoulli decisions. Where no mismatch occurs
the GPU trajectory is, by induction, exactly the oracle's trajectory.
Ages must agree bit for bit wherever the state agrees.
"""
from __future__ import annotations

import numpy as np

import paper_2604_22092_gb300 as fs

TIE = 1e-6


def ages_as_float(A: np.ndarray, age_dtype: int) -> np.ndarray:
    if age_dtype == fs.FS_AGE_F32:
        return A.astype(np.float32)
    if age_dtype == fs.FS_AGE_F16:
        return A.view(np.float16).astype(np.float32)
    return (A.astype(np.uint32) << np.uint32(16)).view(np.float32)


def oracle_params(om, p) -> object:
    """oracle Params equal to a C-ABI fs_sim_params."""
    def lw(L):
        return om.Law(L.kind, L.k, L.a, L.b)
    return om.Params(p.model, p.age_dtype, lw(p.latent), lw(p.infectious), p.beta, p.dt, p.seed,
                     p.replicate, p.shed_mode, lw(p.shedding))


class LockstepReport:
    def __init__(self):
        self.mismatches = 0
        self.decisions = 0
        self.node_steps = 0
        self.near_ties = 0


def lockstep(om, g, params, sim, steps: int, report: LockstepReport | None = None):
    """Advance `sim` by `steps` single steps, checking each against the oracle."""
    rep = report or LockstepReport()
    prm = oracle_params(om, params)
    X, A, k = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
    for _ in range(steps):
        Af = ages_as_float(A, params.age_dtype)
        Xo, Ao, margin, _ = om.step(g.row_ptr, g.col_ind, prm, k, X, Af, want_margin=True)
        fs.fs_sim_step(sim)
        X2, A2, k2 = fs.fs_sim_get_state(sim, g.n, params.age_dtype)
        assert k2 == k + 1
        bad = X2 != Xo
        trials = np.isfinite(margin)
        rep.decisions += int(trials.sum())
        rep.node_steps += g.n
        rep.near_ties += int((np.abs(margin[trials]) < TIE).sum())
        if bad.any():
            assert (np.abs(margin[bad]) < TIE).all(), (
                f"step {k}: {int(bad.sum())} state mismatches outside the tie band; "
                f"nodes {np.flatnonzero(bad)[:10]}, margins {margin[bad][:10]}")
            rep.mismatches += int(bad.sum())
        ok = ~bad
        A2f = ages_as_float(A2, params.age_dtype)
        same = A2f[ok].view(np.uint32) == Ao[ok].view(np.uint32)
        assert same.all(), f"step {k}: age mismatch at nodes {np.flatnonzero(ok)[~same][:10]}"
        X, A, k = X2, A2, k2
    assert rep.mismatches <= max(1e-6 * rep.decisions, 0), (rep.mismatches, rep.decisions)
    return rep
