"""The allocation-free step (fs_step_noalloc) against the regular entry points.

fs_step_noalloc serves callers that cannot call cudaMalloc while stepping:
code running under CUDA stream capture, and applications whose device memory
belongs to their own pool. Its scratch lives in a fixed array inside the
library. This test drives it through the C ABI on caller-owned buffers for two
consecutive steps and checks that it produces exactly what fs_sim_step
produces (the tolerance of the step parity tests: bit-identical states and
ages), on a graph whose merge class uses that scratch, for each age storage
type (FP32, and FP16 and BF16 compared as their 16-bit patterns). It sits in a file that
pytest collects last, and must pass alone in a fresh process as well as after
the other tests.
"""
import math

import numpy as np
import pytest

import paper_2604_22092_gb300 as fs
import workloads as W

pytestmark = pytest.mark.gpu


def degree_sorted(g: W.Graph) -> W.Graph:
    """The same graph relabelled by ascending degree, so that the library's
    internal node order equals the caller's order (identity layout)."""
    order = np.argsort(g.degree, kind="stable")
    new = np.empty(g.n, dtype=np.int64)
    new[order] = np.arange(g.n)
    rows = np.repeat(np.arange(g.n), g.degree)
    keep = rows < g.col_ind
    return W.csr_from_edges(g.n, new[rows[keep]], new[g.col_ind[keep].astype(np.int64)])


def bitmap(X: np.ndarray) -> np.ndarray:
    words = (X.size >> 5) + 1
    bits = np.zeros(words * 32, dtype=np.uint64)
    bits[:X.size] = X == fs.FS_I
    return (bits.reshape(words, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


AGE_TORCH = {fs.FS_AGE_F32: "float32", fs.FS_AGE_F16: "float16", fs.FS_AGE_BF16: "bfloat16"}


@pytest.mark.parametrize("age_dtype", [fs.FS_AGE_F32, fs.FS_AGE_F16, fs.FS_AGE_BF16])
def test_noalloc_step_matches_sim_step_twice(age_dtype):
    import torch
    assert torch.cuda.is_available()
    g = degree_sorted(W.barabasi_albert(60_000, 5, seed=3))
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind)
    info = fs.fs_graph_info_get(gh)
    assert info["identity_layout"] == 1
    assert 0 < info["n_merge"] <= 65536 and info["merge_chunks"] > 1
    p = fs.sim_params(fs.FS_SEIR, fs.law("lognormal", math.log(6.0), 0.6), 0.25, 0.1, seed=17,
                      latent=fs.law("weibull", 2.0, 4.0), age_dtype=age_dtype)
    idx = W.index_nodes(g.n, 60, seed=5, allowed=W.non_hub_nodes(g))
    sh = fs.fs_sim_init(gh, p, idx)
    fs.fs_sim_run(sh, 150, want_counts=False)            # into the growth phase
    X0, A0, k0 = fs.fs_sim_get_state(sh, g.n, age_dtype)
    c0 = fs.fs_sim_run(sh, 0)[0].astype(np.int64)
    ref = []
    for _ in range(2):
        c = fs.fs_sim_step(sh).astype(np.int64)
        X, A, _ = fs.fs_sim_get_state(sh, g.n, age_dtype)
        ref.append((X, A, c))
    fs.fs_sim_destroy(sh)
    assert (ref[1][2] != c0).any(), "the window must contain transitions"

    dev = torch.device("cuda")
    dX = torch.from_numpy(X0.copy()).to(dev)
    # ages travel as their raw storage bits, then are viewed as the storage type
    dA = torch.from_numpy(A0.copy().view(np.int32 if A0.itemsize == 4 else np.int16)).to(dev)
    dA = dA.view(getattr(torch, AGE_TORCH[age_dtype]))
    bm = [torch.from_numpy(bitmap(X0).view(np.int32)).to(dev),
          torch.zeros((g.n >> 5) + 1, dtype=torch.int32, device=dev)]
    deltas = torch.zeros(5, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    prev = c0
    for t in range(2):
        k = k0 + t
        fs.fs_step_noalloc(gh, p, k, dX, dA, bm[t % 2], bm[(t + 1) % 2], deltas, stream)
        torch.cuda.synchronize()
        X_ref, A_ref, c_ref = ref[t]
        np.testing.assert_array_equal(dX.cpu().numpy(), X_ref)
        bits = np.uint32 if A_ref.itemsize == 4 else np.uint16
        got = dA.view(torch.int32 if A_ref.itemsize == 4 else torch.int16).cpu().numpy().view(bits)
        np.testing.assert_array_equal(got, A_ref.view(bits))
        np.testing.assert_array_equal(bm[(t + 1) % 2].cpu().numpy().view(np.uint32), bitmap(X_ref))
        d = deltas.cpu().numpy()
        assert d[4] == 0
        expect = prev.copy()
        expect[0] -= d[0]
        expect[1] += d[0] - d[1]
        expect[2] += d[1] - d[2]
        expect[3] += d[2]
        np.testing.assert_array_equal(expect, c_ref)
        prev = c_ref
    fs.fs_graph_destroy(gh)


def test_noalloc_rejects_graphs_beyond_its_scratch():
    import torch
    g = W.erdos_renyi(100_000, 40, seed=1)           # nearly every row in the merge class
    gh = fs.fs_graph_create(g.n, g.row_ptr, g.col_ind, opts=fs.graph_opts(thread_max_deg=31))
    assert fs.fs_graph_info_get(gh)["n_merge"] > 65536
    p = fs.sim_params(fs.FS_SIR, fs.law("exp", 0.2), 0.3, 0.1, seed=1)
    dev = torch.device("cuda")
    X = torch.zeros(g.n, dtype=torch.uint8, device=dev)
    A = torch.zeros(g.n, dtype=torch.float32, device=dev)
    b0 = torch.zeros((g.n >> 5) + 1, dtype=torch.int32, device=dev)
    b1 = torch.zeros_like(b0)
    d = torch.zeros(5, dtype=torch.int64, device=dev)
    with pytest.raises(fs.FsError) as e:
        fs.fs_step_noalloc(gh, p, 0, X, A, b0, b1, d)
    assert e.value.status == 1 and "65536" in str(e.value)
    fs.fs_graph_destroy(gh)
