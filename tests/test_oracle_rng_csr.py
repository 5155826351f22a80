"""Pins of the oracle's random numbers, connectivity, scaling law and memory
formulas against published vectors, closed forms and brute force."""
import math
import os

import numpy as np
import pytest

import oracle
import snn_inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_philox_known_answers():
    for r in _rows("philox4x32_10_kat.txt"):
        assert r[0] == "10"
        ctr = [int(x, 16) for x in r[1:5]]
        key = [int(x, 16) for x in r[5:7]]
        want = [int(x, 16) for x in r[7:11]]
        assert list(oracle.philox4x32_10(ctr, key)) == want


def test_bernoulli_threshold_closed_forms():
    assert oracle.bernoulli_threshold(0.0) == 0
    assert oracle.bernoulli_threshold(-1.0) == 0
    assert oracle.bernoulli_threshold(1.0) == 2**32
    assert oracle.bernoulli_threshold(2.0) == 2**32
    assert oracle.bernoulli_threshold(0.5) == 2**31
    # 20 Hz at dt = 0.1 ms: p = 0.002, 0.002 * 2^32 = 8589934.592
    assert oracle.bernoulli_threshold(0.002) == 8589935


def test_poisson_source_rate_within_3_sigma():
    n, steps, rate, dt = 1000, 1000, 20.0, 0.1
    spec = I.net([I.source_pop(n, rate)], [], dt=dt, steps=steps)
    net = oracle.from_spec(spec)
    net.step(steps)
    count, _ = net.counters(0)
    p = rate * dt * 1e-3
    mean, sd = n * steps * p, math.sqrt(n * steps * p * (1 - p))
    assert abs(count - mean) < 3 * sd


def test_source_draw_matches_generator_definition():
    # the source spike at (t, i) is word 0 of Philox(counter=(i, t, tag, 1), key=seed)
    seed, tag = 0x1234_5678_9ABC_DEF0, 7
    thr = oracle.bernoulli_threshold(0.3)
    for t, i in [(0, 0), (5, 17), (123456, 999)]:
        u = oracle.philox4x32_10([i, t, tag, 1], [seed & 0xFFFFFFFF, seed >> 32])[0]
        assert oracle.source_spike(seed, tag, t, i, 3000.0, 0.1) == int(u < thr)


def _brute_mask(seed, tag, n_pre, n_post, p):
    thr = oracle.bernoulli_threshold(p)
    mask = np.zeros((n_pre, n_post), dtype=bool)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n_pre):
        for j4 in range((n_post + 3) // 4):
            out = oracle.philox4x32_10([j4, i, tag, 3], key)
            for w in range(4):
                j = 4 * j4 + w
                if j < n_post:
                    mask[i, j] = out[w] < thr
    return mask


@pytest.mark.parametrize("n_pre,n_post,p", [(30, 50, 0.1), (7, 13, 0.5), (16, 4, 0.9), (5, 9, 0.0)])
def test_csr_matches_brute_force_mask(n_pre, n_post, p):
    seed, tag = 4242, 3
    rp, col = oracle.csr_bernoulli(seed, tag, n_pre, n_post, p)
    mask = _brute_mask(seed, tag, n_pre, n_post, p)
    want_rp = np.concatenate([[0], np.cumsum(mask.sum(1))])
    assert np.array_equal(rp, want_rp)
    assert np.array_equal(col, np.nonzero(mask)[1].astype(np.int32))


def test_csr_nnz_binomial_5_sigma_and_layout_invariants():
    n_pre, n_post, p = 200, 500, 0.1
    rp, col = oracle.csr_bernoulli(I.SEED, 0, n_pre, n_post, p)
    nnz = rp[-1]
    mean, sd = n_pre * n_post * p, math.sqrt(n_pre * n_post * p * (1 - p))
    assert abs(nnz - mean) < 5 * sd
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and len(col) == nnz
    for i in range(n_pre):
        r = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(r) > 0) and (len(r) == 0 or (r[0] >= 0 and r[-1] < n_post))


def test_gscale_tables_and_rewritten_form():
    for name, k1, k2, k3, nc, want in _rows("gscale_tables.txt"):
        k1, k2, k3, nc, want = map(float, (k1, k2, k3, nc, want))
        got = oracle.gscale(k1, k2, k3, nc)
        if math.isnan(want):
            assert got is None, name
            continue
        assert got == pytest.approx(want, rel=1e-7), name
        # Sec. 5.1 rewrites the law as (gScale - k3)(nConn + k2) = k1
        assert (got - k3) * (nc + k2) == pytest.approx(k1, rel=1e-12)
    # the benchmark workloads use k1 = 1, k2 = k3 = 0: gScale = 1 / nConn
    assert oracle.gscale(1.0, 0.0, 0.0, 0.1 * 100) == pytest.approx(0.1, rel=1e-15)


def test_memory_words_eq1_eq2_against_array_sizes():
    n_pre, n_post, p = 40, 70, 0.2
    rp, col = oracle.csr_bernoulli(7, 1, n_pre, n_post, p)
    w = np.zeros(len(col), np.float32)
    stored = len(rp) + len(col) + len(w) + 1          # + the nnz integer
    assert oracle.memory_words(len(col), n_pre, n_post, False) == stored
    assert oracle.memory_words(len(col), n_pre, n_post, True) == np.zeros((n_pre, n_post)).size
    # dense and sparse storage break even near p = 0.5 for large populations
    n = 10_000
    assert oracle.memory_words(int(0.49 * n * n), n, n, False) < oracle.memory_words(0, n, n, True)
    assert oracle.memory_words(int(0.51 * n * n), n, n, False) > oracle.memory_words(0, n, n, True)


def test_event_list_matches_row_concatenation():
    rp, col = oracle.csr_bernoulli(11, 2, 50, 80, 0.2)
    w = np.arange(len(col), dtype=np.float64) * 0.5
    spk = np.array([3, 4, 17, 49], np.int32)
    post, wv = oracle.event_list(rp, col, w, spk)
    want_post = np.concatenate([col[rp[i]:rp[i + 1]] for i in spk])
    want_w = np.concatenate([w[rp[i]:rp[i + 1]] for i in spk])
    assert np.array_equal(post, want_post) and np.array_equal(wv, want_w)
    post0, _ = oracle.event_list(rp, col, w, np.zeros(0, np.int32))
    assert len(post0) == 0


def test_dense_batch_oracle_matches_per_instance_delivery():
    # the batched dense definition (a matrix product) against the network
    # oracle's own dense delivery loop, one instance at a time
    import snn_inputs as I
    rng = np.random.default_rng(5)
    n_pre, n_post, B = 30, 17, 4
    W = rng.uniform(0, 1, (n_pre, n_post)).astype(np.float32).astype(np.float64)
    spikes = [np.sort(rng.choice(n_pre, k, replace=False)) for k in (0, 1, 7, 30)]
    scale = rng.uniform(0.5, 2.0, B)
    G0 = rng.uniform(0, 1, (B, n_post))
    G = oracle.dense_batch_deliver(W, spikes, scale, G0)
    for b in range(B):
        spec = I.net([I.source_pop(n_pre, 0.0), I.hh_pop(n_post)],
                     [I.proj(0, 1, "dense", 1.0, ("uniform", 0.0, 1.0), k=(0.0, 0.0, 1.0), user_scale=scale[b])],
                     dt=0.1, steps=1)
        pops = [dict(spec["pops"][0], v0=None), dict(spec["pops"][1], v0=None)]
        proj = dict(spec["projs"][0], w=W.ravel(), n_conn=n_pre)
        net = oracle.OracleNet(pops, [proj], 0.1, 4, 1)
        net.set(1, "g0", G0[b])
        net.deliver(0, spikes[b].astype(np.int32))
        assert np.allclose(net.get(1, "g0"), G[b], rtol=1e-14, atol=1e-14)


def test_dense_grad_update_brute_force_and_closed_forms():
    # D[i, j] = D0[i, j] + sum_t R[t, i] N[j, t]: element-by-element loops on a
    # small case, a K = 1 outer product, and all-ones operands (D0 + K)
    rng = np.random.default_rng(9)
    K, m, n = 5, 4, 3
    R = rng.normal(size=(K, m))
    N = rng.normal(size=(n, K))
    D0 = rng.normal(size=(m, n))
    D = oracle.dense_grad_update(R, N, D0)
    for i in range(m):
        for j in range(n):
            s = D0[i, j]
            for t in range(K):
                s += R[t, i] * N[j, t]
            assert D[i, j] == pytest.approx(s, rel=1e-13, abs=1e-13)
    r, v = rng.normal(size=(1, m)), rng.normal(size=(n, 1))
    assert np.allclose(oracle.dense_grad_update(r, v, np.zeros((m, n))), np.outer(r[0], v[:, 0]), rtol=1e-15, atol=0)
    assert np.array_equal(oracle.dense_grad_update(np.ones((7, m)), np.ones((n, 7)), D0), D0 + 7.0)
