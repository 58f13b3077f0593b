"""dupin_peel_noalloc: the entry point for callers that may not allocate device memory.

Services that reserve all GPU memory up front, latency-critical loops where an
allocation would synchronise the device, and plug-ins whose host process owns
the allocator cannot let a library call cudaMalloc.  This entry point keeps its
working state in one fixed device array instead.  The test calls it through
the C ABI and checks it against dupin_peel (same exact integer results), on
two calls in a row with different inputs, so state left in the shared array by
one call cannot leak into the next.  It lives in its own file so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_09311_gb300 import dupin, synth

    dupin.lib()
    return torch, dupin, synth


def _device_csr(torch, g):
    ptr, idx, w = g.symmetric_csr()
    d = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return d(ptr), d(idx), d(w), d(g.a)


def _run(torch, dupin, g, metric, k, eps, flags=0):
    n = g.n
    d_ptr, d_idx, d_w, d_a = _device_csr(torch, g)
    pr = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    mk = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    cap = n + 2
    trace = (torch.zeros(cap, dtype=torch.int64, device="cuda"), torch.zeros(cap, dtype=torch.int64, device="cuda"),
             torch.zeros(cap, dtype=torch.int64, device="cuda"), torch.zeros(cap, dtype=torch.int64, device="cuda"))
    p = dupin.make_params(metric, k, eps, flags=flags)
    r = dupin.peel_noalloc(n, d_ptr, d_idx, d_w, d_a, p, pr, mk, trace)
    torch.cuda.synchronize()
    R = r.n_rounds + 1
    fh, fl = trace[0].cpu().numpy(), trace[1].cpu().numpy().view(np.uint64)
    tf = [(int(fh[i]) << 64) + int(fl[i]) for i in range(R)]
    return r, pr.cpu().numpy(), mk.cpu().numpy(), tf, trace[2].cpu().numpy()[:R], trace[3].cpu().numpy()[:R]


def test_noalloc_matches_dupin_peel_twice(env):
    torch, dupin, synth = env
    g1 = synth.random_general(3000, 20000, seed=21)
    synth.with_weights(g1, "dw", seed=21, a_range=(0, 5))
    g2 = synth.bipartite_zipf(4000, 2000, 30000, 1.8, 1, 40, 40, 0.5, 10, seed=22)
    g2.c = synth.fd_weights(g2)
    cases = [(g1, "dw", 1, (1, 10), 0), (g2, "fd", 2, (1, 20), dupin.GPO)]
    for g, metric, k, eps, flags in cases:  # two calls in a row on different inputs
        dg = dupin.Graph.from_synth(g)
        ref = dupin.peel(dg, metric, k, eps, flags=flags)
        dg.free()
        r, pr, mk, tf, sz, pe = _run(torch, dupin, g, metric, k, eps, flags)
        assert np.array_equal(pr, ref.peel_round)
        assert np.array_equal(mk, ref.best_mask)
        assert tf == ref.trace_f
        assert np.array_equal(sz, ref.trace_size) and np.array_equal(pe, ref.trace_peeled)
        assert (r.n_rounds, r.best_round, r.best_size) == (ref.n_rounds, ref.best_round, ref.best_size)
        assert (int(r.best_f_hi) << 64) + int(r.best_f_lo) == ref.best_f
        assert r.n_min_rule == ref.n_min_rule


def test_noalloc_rejects_sizes_beyond_its_maximum(env):
    torch, dupin, synth = env
    n = dupin.NOALLOC_MAX_N + 1
    g = synth.random_general(n, 4 * n, seed=3)
    d_ptr, d_idx, _, _ = _device_csr(torch, g)
    pr = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel_noalloc(n, d_ptr, d_idx, None, None, dupin.make_params("dg", 1, (1, 10)), pr)
    assert e.value.code == dupin.ERR_INVALID_ARG
    assert str(dupin.NOALLOC_MAX_N) in str(e.value)


def test_noalloc_matches_the_oracle_at_its_maximum_size(env):
    """n = DUPIN_NOALLOC_MAX_N exactly, against the CPU oracle (not another CUDA
    path): a k = 1 peel (minimum rule) and an Algorithm 4 (LPO) peel."""
    import oracle

    torch, dupin, synth = env
    n = dupin.NOALLOC_MAX_N
    g = synth.random_general(n, 6 * n, seed=31)
    synth.with_weights(g, "dw", seed=31, a_range=(0, 4))
    og = oracle.Graph.from_synth(g, "dw")
    for k, eps, flags, oflags in ((1, (1, 10), 0, 0), (2, (1, 20), dupin.LPO, oracle.FLAG_LPO)):
        ref = oracle.peel_batch(og, k, eps, flags=oflags)
        r, pr, mk, tf, sz, pe = _run(torch, dupin, g, "dw", k, eps, flags)
        assert g.n == n
        assert np.array_equal(pr, ref.peel_round), (k, flags)
        assert np.array_equal(mk, ref.best_mask), (k, flags)
        assert tf == ref.trace_f
        assert np.array_equal(sz, ref.trace_size) and np.array_equal(pe, ref.trace_peeled)
        assert (r.n_rounds, r.best_round, r.best_size) == (ref.n_rounds, ref.best_round, ref.best_size)
        assert (int(r.best_f_hi) << 64) + int(r.best_f_lo) == ref.best_f
        assert r.n_min_rule == ref.n_min_rule
    og.close()


def test_noalloc_call_allocates_no_device_memory(env):
    """After the first call on the device (its one-time set-up), a call leaves
    the device's free memory exactly as it found it."""
    torch, dupin, synth = env
    g = synth.random_general(5000, 30000, seed=41)
    synth.with_weights(g, "dw", seed=41, a_range=(0, 3))
    n = g.n
    d_ptr, d_idx, d_w, d_a = _device_csr(torch, g)
    pr = torch.empty(n, dtype=torch.int32, device="cuda")
    mk = torch.empty(n, dtype=torch.uint8, device="cuda")
    p = dupin.make_params("dw", 1, (1, 10))
    dupin.peel_noalloc(n, d_ptr, d_idx, d_w, d_a, p, pr, mk)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        dupin.peel_noalloc(n, d_ptr, d_idx, d_w, d_a, p, pr, mk)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_a_malformed_csr(env):
    """A self-loop, an id out of range, decreasing offsets, an odd arc count and
    an asymmetric CSR are each INVALID_ARG (checked before any peel kernel)."""
    torch, dupin, synth = env
    Q = 1 << 32
    d = lambda x, t: torch.tensor(x, dtype=t, device="cuda")
    cases = {
        "self-loop": (2, [0, 1, 2], [0, 1]),
        "id out of range": (2, [0, 1, 2], [1, 5]),
        "decreasing offsets": (3, [0, 2, 1, 2], [1, 2]),
        "odd arc count": (3, [0, 1, 2, 3], [1, 0, 1]),
        "asymmetric": (3, [0, 1, 2, 4], [1, 2, 0, 1]),
    }
    for name, (n, rp, col) in cases.items():
        pr = torch.empty(n, dtype=torch.int32, device="cuda")
        w = d([Q] * len(col), torch.int64)
        with pytest.raises(dupin.DupinError) as e:
            dupin.peel_noalloc(n, d(rp, torch.int64), d(col, torch.int32), w, None,
                               dupin.make_params("dw", 1, (1, 10)), pr)
        assert e.value.code == dupin.ERR_INVALID_ARG, name
    # a symmetric path with unequal weights on an arc and its reverse
    pr = torch.empty(3, dtype=torch.int32, device="cuda")
    with pytest.raises(dupin.DupinError) as e:
        dupin.peel_noalloc(3, d([0, 1, 3, 4], torch.int64), d([1, 0, 2, 1], torch.int32),
                           d([Q, Q, 2 * Q, 3 * Q], torch.int64), None, dupin.make_params("dw", 1, (1, 10)), pr)
    assert e.value.code == dupin.ERR_INVALID_ARG
