"""The seeded input generators produce the shapes the workload recipes state
(lengths, alphabets, duplicate share, set sizes), deterministically."""
import re

import numpy as np

import gen


def _lengths(s):
    ends = np.append(s.offsets[1:], np.uint64(s.total)).astype(np.int64)
    return ends - s.offsets.astype(np.int64) - 1  # terminator excluded


def test_uniform_recipe():
    s = gen.generate(1, 50_000, 1)
    L = _lengths(s)
    assert L.min() >= 8 and L.max() <= 20
    body = s.chars[:s.total]
    letters = body[body != 0]
    assert letters.min() >= ord("a") and letters.max() <= ord("z")
    assert int((body == 0).sum()) == s.n  # one terminator per string, none inside


def test_url_recipe():
    s = gen.generate(2, 50_000, 2)
    L = _lengths(s)
    assert 50 <= (L.mean() + 1) <= 70  # mean about 60 B with the terminator
    pat = re.compile(rb"^https?://[a-z0-9.\-]+(/[a-z0-9]{3,12}){1,6}$")
    for i in range(0, s.n, 997):
        assert pat.match(s.get(i)), s.get(i)
    # hosts repeat (a 2,000-host pool drawn Zipf): far fewer distinct hosts than strings
    hosts = {s.get(i).split(b"/")[2] for i in range(0, s.n, 7)}
    assert len(hosts) <= 2000


def test_dna_recipe():
    s = gen.generate(3, 50_000, 3)
    L = _lengths(s)
    assert (L == 64).all()
    body = s.chars[:s.total]
    assert set(np.unique(body).tolist()) == {0, ord("A"), ord("C"), ord("G"), ord("T")}
    distinct = len({s.get(i) for i in range(s.n)})
    dup_share = 1 - distinct / s.n
    assert 0.07 <= dup_share <= 0.13  # about 10 % exact copies


def test_batch_recipe():
    b = gen.generate_batch(200, 100, 4000, 5)
    sizes = np.diff(b.set_begin.astype(np.int64))
    assert len(sizes) == 200 and sizes.min() >= 100 and sizes.max() <= 4000
    assert set(np.unique(b.kinds).tolist()) <= {1, 2, 3}
    assert b.set_begin[-1] == b.strings.n


def test_literal_batch_sizes():
    """The sets-literal batch: 10,000 sets, sizes log-uniform in [100, 1M]
    (mean (1M - 100) / ln(10^4), about 108.6k strings a set), kinds uniform."""
    w = gen.BATCH_WORKLOADS["sets-literal"]
    sizes, kinds = gen.batch_sizes(w["num_sets"], w["lo"], w["hi"], w["seed"])
    assert len(sizes) == 10_000 and sizes.min() >= 100 and sizes.max() <= 1_000_000
    assert int(sizes.sum()) == 1_092_616_105
    assert abs(sizes.mean() / ((1e6 - 100) / np.log(1e4)) - 1) < 0.03
    # log-uniform: each decade of sizes holds about a quarter of the sets
    dec = np.histogram(np.log10(sizes), bins=[2, 3, 4, 5, 6.0001])[0]
    assert (np.abs(dec / 10_000 - 0.25) < 0.03).all(), dec
    assert all(abs(int((kinds == k).sum()) / 10_000 - 1 / 3) < 0.03 for k in (1, 2, 3))
    assert sizes.max() < 2 ** 32 and int(sizes.sum()) < 2 ** 32 - 1


def test_generators_are_deterministic_and_thread_independent():
    for kind in (1, 2, 3):
        a = gen.generate(kind, 20_000, 11, threads=1)
        c = gen.generate(kind, 20_000, 11, threads=8)
        assert np.array_equal(a.chars, c.chars) and np.array_equal(a.offsets, c.offsets)
        d = gen.generate(kind, 20_000, 12)
        assert not np.array_equal(a.chars[:a.total], d.chars[:d.total])
