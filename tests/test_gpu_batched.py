"""Batched sort (one graph launch for many independent sets) and its
autotuner: every set must equal its own oracle sort; the tuned options are
cached per device and batch shape."""
import json

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


def _batched(b):
    chars, offsets, perm, lcp = _dev(b)
    nsets = len(b.set_begin) - 1
    sss.sss_sort_batched(chars, offsets, b.strings.n, b.set_begin, nsets, perm, lcp)
    torch.cuda.synchronize()
    return perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32)


def _verify_sets(b, perm, lcp):
    for j in range(len(b.set_begin) - 1):
        lo, hi = int(b.set_begin[j]), int(b.set_begin[j + 1])
        s = gen.set_strings(b, j)
        code, bad = oracle.verify(s.chars, s.offsets, perm[lo:hi], lcp[lo:hi])
        assert code == 0, (j, oracle.VERIFY_CODES[code], bad)


def test_batched_sets_10k_full_workload():
    w = gen.BATCH_WORKLOADS["sets-10k"]
    b = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"])
    perm, lcp = _batched(b)
    _verify_sets(b, perm, lcp)


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
