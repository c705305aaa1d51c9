"""Pins of the CPU oracle against facts that do not come from the oracle
itself: brute force over tiny inputs, Python's own sort (a library routine),
closed forms, the worked example of Fig. 1 and hand-worked fixtures."""
import itertools
import os
import random

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def py_sorted(items):
    """(perm, lcp) by Python's sort on (bytes, index) and a plain LCP loop."""
    perm = sorted(range(len(items)), key=lambda i: (items[i], i))
    lcp = [0] * len(items)
    for r in range(1, len(items)):
        a, b = items[perm[r - 1]], items[perm[r]]
        k = 0
        while k < min(len(a), len(b)) and a[k] == b[k]:
            k += 1
        lcp[r] = k
    return perm, lcp


def run_oracle(items):
    s = gen.from_list(items)
    perm, lcp = oracle.sort(s.chars, s.offsets)
    return list(map(int, perm)), list(map(int, lcp))


TINY = [b""] + [bytes(t) for L in range(1, 4) for t in itertools.product(b"ab", repeat=L)]


def test_bruteforce_all_short_sequences():
    # every sequence of up to 3 strings over {a,b} of length 0..3
    for m in range(0, 4):
        for seq in itertools.product(TINY, repeat=m):
            assert run_oracle(list(seq)) == py_sorted(list(seq))


def test_bruteforce_all_permutations_of_multiset():
    base = [b"ab", b"a", b"", b"ab", b"b", b"a", b"ba"]
    for seq in itertools.permutations(base):
        assert run_oracle(list(seq)) == py_sorted(list(seq))


def test_bruteforce_random_multisets_up_to_7():
    rng = random.Random(7)
    for _ in range(3000):
        seq = [rng.choice(TINY) for _ in range(rng.randint(0, 7))]
        assert run_oracle(seq) == py_sorted(seq)


def _random_strings(rng, n, maxlen, alphabet, prefixes):
    out = []
    for _ in range(n):
        p = rng.choice(prefixes)
        tail = bytes(rng.choice(alphabet) for _ in range(rng.randint(0, maxlen)))
        out.append(p + tail)
    for _ in range(n // 10):  # exact duplicates
        out[rng.randrange(n)] = out[rng.randrange(n)]
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_library_sort_midsize(seed):
    rng = random.Random(seed)
    alphabet = list(range(1, 256))  # includes 0x80..0xff: unsigned order
    prefixes = [b"", b"http://www.", b"\xff\xfe", b"a" * 40, b"ab" * 13]
    items = _random_strings(rng, 3000, 30, alphabet, prefixes)
    assert run_oracle(items) == py_sorted(items)


def test_small_alphabet_long_prefixes():
    rng = random.Random(11)
    items = _random_strings(rng, 2000, 12, [1, 2, 0x80], [b"x" * 1100, b"x" * 1100 + b"\x01" * 9, b""])
    assert run_oracle(items) == py_sorted(items)


def test_generated_workload_matches_library_sort():
    s = gen.workload("uniform-100k", n=20000)
    items = [s.get(i) for i in range(s.n)]
    perm, lcp = oracle.sort(s.chars, s.offsets)
    assert (list(map(int, perm)), list(map(int, lcp))) == py_sorted(items)


def test_verify_accepts_only_the_unique_answer():
    items = [b"b", b"a", b"a", b"ab", b"", b"abc", b"b"]
    s = gen.from_list(items)
    perm, lcp = oracle.sort(s.chars, s.offsets)
    assert oracle.verify(s.chars, s.offsets, perm, lcp) == (0, 0)
    # order violated
    p = perm.copy(); p[3], p[4] = p[4], p[3]
    assert oracle.verify(s.chars, s.offsets, p, None)[0] == 2
    # equal strings out of index order ("a" at 1 and 2)
    p = perm.copy(); i = list(p).index(1); j = list(p).index(2); p[i], p[j] = p[j], p[i]
    assert oracle.verify(s.chars, s.offsets, p, None)[0] == 3
    # not a permutation
    p = perm.copy(); p[0] = p[1]
    assert oracle.verify(s.chars, s.offsets, p, None)[0] == 1
    # lcp off by one
    l2 = lcp.copy(); l2[5] += 1
    assert oracle.verify(s.chars, s.offsets, perm, l2) == (4, 5)
    l2 = lcp.copy(); l2[0] = 1
    assert oracle.verify(s.chars, s.offsets, perm, l2) == (4, 0)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_dist_prefix_worked_example():
    rows = {r[0]: r[1:] for r in _read_golden("dist_prefix_example.txt")}
    items = [w.encode() for w in rows["strings"]]
    s = gen.from_list(items)
    perm, lcp = oracle.sort(s.chars, s.offsets)
    assert list(map(int, perm)) == list(map(int, rows["perm"]))
    assert list(map(int, lcp)) == list(map(int, rows["lcp"]))
    assert s.total == int(rows["N"][0])
    assert oracle.dist_prefix(s.chars, s.offsets, perm, lcp) == int(rows["D"][0])


def test_dist_prefix_all_duplicated_is_N():
    # fixed-length strings that all occur at least twice: D = N (Table 1,
    # Sinha DNA: D/N = 100 % with terminators counted)
    rng = random.Random(5)
    base = [bytes(rng.choice(b"ACGT") for _ in range(9)) for _ in range(300)]
    items = base + base + [rng.choice(base) for _ in range(100)]
    rng.shuffle(items)
    s = gen.from_list(items)
    perm, lcp = oracle.sort(s.chars, s.offsets)
    assert s.total == 10 * len(items)
    assert oracle.dist_prefix(s.chars, s.offsets, perm, lcp) == s.total


def test_dist_prefix_distinct_first_chars():
    # all first characters distinct: one character each decides the order
    items = [bytes([c]) * 5 for c in range(1, 200)]
    s = gen.from_list(items)
    perm, lcp = oracle.sort(s.chars, s.offsets)
    assert oracle.dist_prefix(s.chars, s.offsets, perm, lcp) == len(items)


def test_key_word_golden():
    for w, d, h in _read_golden("key_words.txt"):
        s = gen.from_list([w.encode()])
        assert oracle.key_word(s.chars, 0, int(d)) == int(h, 16), (w, d)


def test_key_word_order_is_prefix_order():
    # the point of the big-endian packing: comparing words compares the
    # 8-character windows as strings (bytes after a terminator are 0)
    rng = random.Random(3)
    items = _random_strings(rng, 400, 12, [1, 2, 0x7f, 0x80, 0xff], [b"", b"ab"])
    s = gen.from_list(items)
    for _ in range(3000):
        i, j = rng.randrange(len(items)), rng.randrange(len(items))
        d = rng.randint(0, min(len(items[i]), len(items[j])))
        ki = oracle.key_word(s.chars, int(s.offsets[i]), d)
        kj = oracle.key_word(s.chars, int(s.offsets[j]), d)
        wi, wj = items[i][d:d + 8], items[j][d:d + 8]
        assert (ki < kj) == (wi < wj) and (ki == kj) == (wi == wj)


def test_key_word_past_end_is_zero():
    s = gen.from_list([b"abc", b"defgh"])
    assert oracle.key_word(s.chars, 0, 5) == 0  # never reads the next string


def test_classify_fig1():
    rows = _read_golden("fig1_ternary_tree.txt")
    x = [int(v) for v in rows[0][1:]]
    for key, b in rows[1:]:
        assert oracle.classify(int(key), x) == int(b)


def test_classify_buckets_partition_the_key_space():
    # 2v+1 buckets in key order; odd buckets hold exactly the splitters
    rng = random.Random(9)
    x = sorted(rng.sample(range(1, 10 ** 6), 15))
    prev = 0
    for key in range(0, 10 ** 6, 997):
        b = oracle.classify(key, x)
        assert 0 <= b <= 2 * len(x) and b >= prev
        assert (b % 2 == 1) == (key in x)
        prev = b
    for i, xi in enumerate(x):
        assert oracle.classify(xi, x) == 2 * i + 1


def test_classify_lower_bound_with_duplicate_splitters():
    x = [5, 5, 7]
    assert [oracle.classify(k, x) for k in (4, 5, 6, 7, 8)] == [0, 1, 4, 5, 6]


def test_select_splitters_no_duplicates_is_every_second_sample():
    # without repeated samples the recursive choice takes the middle of each
    # range, i.e. every alpha-th (alpha = 2) sample of 2^(k+1) - 1 samples
    for k in range(1, 9):
        s = np.arange(1, 2 ** (k + 1), dtype=np.uint64) * 3
        level, ino = oracle.select_splitters(s, k)
        assert list(ino) == list(s[1::2])
        assert int(level[0]) == int(s[len(s) // 2])


def test_select_splitters_hand_example_with_duplicates():
    # sample 1 1 1 1 1 2 3 (indices 0..6), k = 2:
    #   root: middle index 3 -> x = 1; scanning left skips all of 0..2 (equal)
    #         -> left range empty; scanning right skips 4 -> right range 5..6
    #   left child: empty range -> repeats the parent's 1
    #   right child: middle of 5..6 is index 5 -> 2
    level, ino = oracle.select_splitters(np.array([1, 1, 1, 1, 1, 2, 3], dtype=np.uint64), 2)
    assert list(map(int, level)) == [1, 1, 2]
    assert list(map(int, ino)) == [1, 1, 2]


def test_select_splitters_all_equal():
    level, ino = oracle.select_splitters(np.full(15, 42, dtype=np.uint64), 3)
    assert set(map(int, ino)) == {42}


def test_select_splitters_inorder_sorted_and_from_sample():
    rng = random.Random(4)
    for _ in range(200):
        k = rng.randint(1, 7)
        cnt = 2 ** (k + 1) - 1
        s = np.array(sorted(rng.choice(range(6)) for _ in range(cnt)), dtype=np.uint64)
        level, ino = oracle.select_splitters(s, k)
        assert all(int(ino[i]) <= int(ino[i + 1]) for i in range(len(ino) - 1))
        assert set(map(int, ino)) <= set(map(int, s))


def test_cdf_uniform_parameters_give_identity():
    # equal increments: F(u) = u exactly (closed form)
    u = np.linspace(0, 1, 101)
    F = oracle.cdf_forward(np.zeros(64), u)
    assert np.allclose(F, u, atol=1e-12)


def test_cdf_monotone_and_normalised():
    rng = np.random.default_rng(0)
    theta = rng.normal(size=32)
    u = np.sort(rng.random(500))
    F = oracle.cdf_forward(theta, np.concatenate([[0.0], u, [1.0]]))
    assert F[0] == 0.0 and abs(F[-1] - 1.0) < 1e-12
    assert np.all(np.diff(F) >= -1e-15)


def test_cdf_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    M = 16
    theta = rng.normal(size=M)
    u = rng.random(50)
    y = np.sort(rng.random(50))
    g = oracle.cdf_grad(theta, u, y)
    h = 1e-6
    fd = np.zeros(M)
    for j in range(M):
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        fd[j] = (oracle.cdf_loss(tp, u, y) - oracle.cdf_loss(tm, u, y)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)


def _cut_depth(level):
    """Levels of a level-order tree that hold a node differing from its
    parent (a node repeats its parent's splitter exactly when its sample
    range was empty; a chosen splitter never equals its parent's, whose
    equal samples the child ranges skip)."""
    d = 1
    for i in range(2, len(level) + 1):
        if int(level[i - 1]) != int(level[(i >> 1) - 1]):
            d = max(d, i.bit_length())
    return d


def _in_order(level, d):
    """In-order sequence of the top d levels of a level-order tree."""
    out = [0] * (2 ** d - 1)
    for i in range(1, 2 ** d):
        lv = i.bit_length() - 1
        q = i - (1 << lv)
        out[(2 * q + 1) * (1 << (d - 1 - lv)) - 1] = int(level[i - 1])
    return out


def test_cut_tree_keeps_the_nonempty_buckets():
    # the splitter tree cut to the levels whose nodes still choose a new
    # splitter (the sample-driven tree depth) puts every key with the same
    # other keys, and in an equality bucket exactly when the full tree does
    rng = random.Random(9)
    for trial in range(300):
        k = rng.randint(2, 8)
        cnt = 2 ** (k + 1) - 1
        distinct = rng.choice([1, 2, 3, 5, 9, 17, 40, 1000])
        vals = [rng.randrange(1, 10 ** 6) for _ in range(distinct)]
        weights = [rng.random() ** 3 for _ in vals]
        s = np.array(sorted(rng.choices(vals, weights, k=cnt)), dtype=np.uint64)
        level, ino = oracle.select_splitters(s, k)
        d = _cut_depth(level)
        assert 1 <= d <= k
        cut = _in_order(level, d)
        assert cut == sorted(cut)
        assert set(cut) == set(map(int, ino))  # the same splitters, fewer repeats
        keys = sorted(set(vals) | {v + 1 for v in vals} | {v - 1 for v in vals} | {0, 2 ** 63})
        full_b = [oracle.classify(q, ino) for q in keys]
        cut_b = [oracle.classify(q, cut) for q in keys]
        for i in range(len(keys) - 1):
            assert (full_b[i] == full_b[i + 1]) == (cut_b[i] == cut_b[i + 1])
        assert [b & 1 for b in full_b] == [b & 1 for b in cut_b]


@pytest.mark.parametrize("threads", [1, 2, 5, 8])
def test_parallel_oracle_equals_the_sequential_one(threads):
    """The host-threaded baseline (sample-cut ranges, each sorted by the
    multikey quicksort) gives exactly oracle.sort's answer: on the three
    generator kinds, on input where most strings are equal (so one range
    holds a long run of equal strings and many sample strings coincide), and
    with empty strings."""
    rng = random.Random(threads)
    cases = [gen.generate(k, 30_000, 40 + k) for k in (1, 2, 3)]
    items = [b"dup"] * 20_000 + [b""] * 500 + [bytes(rng.choice(b"ab") for _ in range(rng.randint(0, 6)))
                                                for _ in range(9_000)]
    rng.shuffle(items)
    cases.append(gen.from_list(items))
    for s in cases:
        p1, l1 = oracle.sort(s.chars, s.offsets)
        p2, l2 = oracle.sort_parallel(s.chars, s.offsets, threads)
        assert np.array_equal(p1, p2) and np.array_equal(l1, l2)
