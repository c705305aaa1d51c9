"""Batched sort (one graph launch for many independent sets) and its
autotuner: every set must equal its own oracle sort; the tuned options are
cached per device and batch shape."""
import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import gen
import oracle
import paper_1305_1157_gb300 as sss
from paper_1305_1157_gb300 import build as sbuild

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    sbuild.build()
    sss.load()


@pytest.fixture(autouse=True)
def keep_options():
    o = sss.sss_get_options()
    yield
    sss.sss_set_options(o)


def _dev(b):
    s = b.strings
    return (torch.from_numpy(s.chars).cuda(), torch.from_numpy(s.offsets.view(np.int64)).cuda(),
            torch.full((s.n,), -1, dtype=torch.int32, device="cuda"),
            torch.full((s.n,), -1, dtype=torch.int32, device="cuda"))


def _batched(b, device_set_begin=False):
    chars, offsets, perm, lcp = _dev(b)
    nsets = len(b.set_begin) - 1
    sb = torch.from_numpy(b.set_begin.view(np.int64)).cuda() if device_set_begin else b.set_begin
    sss.sss_sort_batched(chars, offsets, b.strings.n, sb, nsets, perm, lcp)
    torch.cuda.synchronize()
    return perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32)


def _verify_set(b, perm, lcp, j):
    lo, hi = int(b.set_begin[j]), int(b.set_begin[j + 1])
    s = gen.set_strings(b, j)
    code, bad = oracle.verify(s.chars, s.offsets, perm[lo:hi], lcp[lo:hi])
    return j, code, bad


def _verify_sets(b, perm, lcp, threads=1):
    """Every set against the oracle's check of the unique answer (linear in
    the set's bytes); sets are independent, so several run at once (the
    oracle's C code releases the interpreter lock)."""
    nsets = len(b.set_begin) - 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for j, code, bad in ex.map(lambda j: _verify_set(b, perm, lcp, j), range(nsets)):
            assert code == 0, (j, oracle.VERIFY_CODES[code], bad)


def test_batched_sets_10k_full_workload():
    w = gen.BATCH_WORKLOADS["sets-10k"]
    b = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"])
    perm, lcp = _batched(b)
    _verify_sets(b, perm, lcp)


def test_batched_sets_literal_full_workload():
    """The sets-literal batch: 10,000 sets with sizes log-uniform in
    [100, 1M] (1.09 G strings, about 51 GB of characters), so one graph
    launch mixes device-wide rounds of sets up to 1M strings with thousands
    of small sets.  Every set is checked against the oracle's verify."""
    w = gen.BATCH_WORKLOADS["sets-literal"]
    sizes, _ = gen.batch_sizes(w["num_sets"], w["lo"], w["hi"], w["seed"])
    n = int(sizes.sum())
    free, _ = torch.cuda.mem_get_info()
    need = 51 * 10**9 + 8 * n + 8 * n + sss.sss_workspace_size(n)
    if free < need * 1.05:
        pytest.skip(f"needs about {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    b = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"])
    assert b.strings.n == n and b.strings.total > 2**32  # characters beyond 4 GiB too
    try:
        perm, lcp = _batched(b)
    finally:
        torch.cuda.empty_cache()
        sss.sss_release()  # the ~97 GB workspace is not kept for the later tests
    _verify_sets(b, perm, lcp, threads=max(1, min(32, os.cpu_count() or 1)))
    st = sss.sss_get_last_stats()
    assert st.rounds >= 2


def test_batched_equals_per_set_sorts():
    b = gen.generate_batch(200, 100, 3000, 21)
    perm, lcp = _batched(b)
    chars, offsets, _, _ = _dev(b)
    for j in range(0, 200, 13):
        lo, hi = int(b.set_begin[j]), int(b.set_begin[j + 1])
        p1 = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
        l1 = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
        sss.sss_sort(chars, offsets[lo:hi], hi - lo, p1, l1)
        torch.cuda.synchronize()
        assert np.array_equal(p1.cpu().numpy().view(np.uint32), perm[lo:hi])
        assert np.array_equal(l1.cpu().numpy().view(np.uint32), lcp[lo:hi])


def test_batched_set_begin_in_device_memory():
    """set_begin may live on the device (read back once): the same output as
    with the host array, every set checked against the oracle; a bad device
    array is rejected before any sorting."""
    b = gen.generate_batch(150, 100, 20_000, 23)
    p_host, l_host = _batched(b)
    p_dev, l_dev = _batched(b, device_set_begin=True)
    assert np.array_equal(p_host, p_dev) and np.array_equal(l_host, l_dev)
    _verify_sets(b, p_dev, l_dev)
    chars, offsets, perm, lcp = _dev(b)
    bad = b.set_begin.astype(np.int64).copy()
    bad[3], bad[4] = bad[4], bad[3]  # decreasing
    with pytest.raises(sss.SSSError) as e:
        sss.sss_sort_batched(chars, offsets, b.strings.n, torch.from_numpy(bad).cuda(), 150, perm, lcp)
    assert e.value.code == -1


def test_autotune_picks_valid_options_and_caches_them(tmp_path):
    tune = gen.generate_batch(300, 100, 4000, 31)
    chars, offsets, perm, lcp = _dev(tune)
    cache = tmp_path / "autotune.jsonl"
    best, ms = sss.sss_autotune_batched(chars, offsets, tune.strings.n, tune.set_begin, 300, perm, lcp,
                                        str(cache))
    assert 5 <= best.k_max <= 10 and 32 <= best.base_threshold <= 128 and ms > 0
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["k_max"] == best.k_max and lines[0]["ms"] == pytest.approx(ms, rel=1e-3)
    # the tuned options are current; a second call is answered from the cache
    cur = sss.sss_get_options()
    assert (cur.k_max, cur.base_threshold, cur.medium_threshold, cur.chunk, cur.key_bytes) == \
        (best.k_max, best.base_threshold, best.medium_threshold, best.chunk, best.key_bytes)
    best2, ms2 = sss.sss_autotune_batched(chars, offsets, tune.strings.n, tune.set_begin, 300, perm, lcp,
                                          str(cache))
    assert (best2.k_max, best2.chunk, best2.key_bytes) == (best.k_max, best.chunk, best.key_bytes)
    assert ms2 == pytest.approx(ms, rel=1e-3) and best.key_bytes in (8, 16)
    assert len(cache.read_text().splitlines()) == 1
    # the tuned options sort another batch of the same shape exactly
    real = gen.generate_batch(300, 100, 4000, 32)
    p2, l2 = _batched(real)
    _verify_sets(real, p2, l2)
