"""GPU parity of alphabet compression (App. A.2, "Practical Refinements"):
with the option on, strings over sigma' <= 15 characters are rewritten with
g characters per byte before the sort and the LCP array is converted back.
The output must equal the oracle's, bit for bit, for every alphabet size,
string length mix and sort form."""
import random

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


def to_dev(s):
    chars = torch.from_numpy(s.chars).cuda()
    offsets = torch.from_numpy(s.offsets.view(np.int64)).cuda()
    return chars, offsets


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_sort(s):
    chars, offsets = to_dev(s)
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    sss.sss_sort(chars, offsets, s.n, perm, lcp)
    torch.cuda.synchronize()
    return u32(perm), u32(lcp)


def assert_same(s, perm, lcp):
    ref_perm, ref_lcp = oracle.sort(s.chars, s.offsets)
    if not np.array_equal(perm, ref_perm):
        i = int(np.nonzero(perm != ref_perm)[0][0])
        raise AssertionError(f"perm differs first at rank {i}: gpu {perm[i]} oracle {ref_perm[i]}")
    if not np.array_equal(lcp, ref_lcp):
        i = int(np.nonzero(lcp != ref_lcp)[0][0])
        raise AssertionError(f"lcp differs first at rank {i}: gpu {lcp[i]} oracle {ref_lcp[i]}")


def expected_group(sigma):
    """Characters per byte: the largest g with (sigma + 1)^g <= 256, at most 8;
    1 (no rewrite) for sigma = 0 or sigma >= 16."""
    if sigma == 0 or sigma >= 16:
        return 1
    g = 0
    while g < 8 and (sigma + 1) ** (g + 1) <= 256:
        g += 1
    return g


def small_alphabet_strings(rng, sigma, n, maxlen):
    """n strings over sigma random byte values: random lengths 0..maxlen,
    shared prefixes cut from earlier strings, exact duplicates."""
    alpha = rng.sample(range(1, 256), sigma)
    out = []
    for _ in range(n):
        r = rng.random()
        if out and r < 0.3:
            b = rng.choice(out)
            out.append(b[:rng.randint(0, len(b))] + bytes(rng.choice(alpha) for _ in range(rng.randint(0, 6))))
        elif out and r < 0.4:
            out.append(rng.choice(out))
        else:
            out.append(bytes(rng.choice(alpha) for _ in range(rng.randint(0, maxlen))))
    return out


SORT_FORMS = [
    dict(graph=0, key_bytes=16),
    dict(graph=1, key_bytes=16),
    dict(graph=0, key_bytes=8, base_threshold=16, medium_threshold=16, k_max=2, chunk=2048),
    dict(graph=0, key_bytes=16, base_threshold=16, medium_threshold=8192, k_max=10, chunk=2048),
]


@pytest.mark.parametrize("sigma", [1, 2, 3, 4, 5, 6, 7, 15, 16, 40])
@pytest.mark.parametrize("form", range(len(SORT_FORMS)))
def test_every_alphabet_size(sigma, form):
    sss.sss_set_options(alphabet=1, **SORT_FORMS[form])
    rng = random.Random(1000 * sigma + form)
    items = small_alphabet_strings(rng, sigma, 30_000, 90)
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    st = sss.sss_get_last_stats()
    present = len(set(c for w in items for c in w))
    assert st.alphabet_symbols == present
    assert st.alphabet_group == expected_group(present)


@pytest.mark.parametrize("form", range(len(SORT_FORMS)))
def test_dna_workload(form):
    sss.sss_set_options(alphabet=1, **SORT_FORMS[form])
    s = gen.generate(3, 200_000, 71)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    st = sss.sss_get_last_stats()
    assert st.alphabet_symbols == 4 and st.alphabet_group == 3


EDGE_CASES = {
    "one": [b"x"],
    "one_empty": [b""],
    "all_empty": [b""] * 3000,  # sigma' = 0: nothing to rewrite
    "two_equal": [b"ab", b"ab"],
    "unary_lengths": [b"a" * L for L in range(0, 300)] * 3,  # sigma' = 1, g = 8
    "binary_long_prefix": [b"ab" * 700 + bytes([97 + i % 2]) * (i % 9) for i in range(3000)],
    "group_boundaries": [b"ACGT"[: (i % 4) + 1] * (i % 13) for i in range(5000)],
    "high_and_low_bytes": [bytes([0xff, 0x01, 0xff][: i % 4]) * (i % 11) for i in range(4000)],
    "differ_after_4k": [b"C" * 4100 + bytes([65 + (i * 7) % 3]) for i in range(300)],
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
@pytest.mark.parametrize("form", [0, 1, 2])
def test_edge_cases(name, form):
    sss.sss_set_options(alphabet=1, **SORT_FORMS[form])
    items = list(EDGE_CASES[name])
    random.Random(len(items)).shuffle(items)
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


def test_character_missing_from_the_sample():
    # the alphabet comes from every (n / 16384)-th string; a character that
    # occurs only elsewhere must send the packing pass back to the exact scan
    sss.sss_set_options(alphabet=1)
    rng = random.Random(81)
    items = [bytes(rng.choice(b"ACGT") for _ in range(rng.randint(0, 40))) for _ in range(100_000)]
    for i in (1, 4999, 77_777):  # not multiples of the sample step (6)
        items[i] = items[i][:5] + b"N" + items[i][5:]
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    st = sss.sss_get_last_stats()
    assert st.alphabet_symbols == 5 and st.alphabet_group == 3


def test_long_strings_missing_from_the_sample():
    # the packed buffer is sized from the sample's mean length; long strings
    # the sample did not see overflow it and force the exact sizes
    sss.sss_set_options(alphabet=1)
    rng = random.Random(82)
    items = [bytes(rng.choice(b"ab") for _ in range(rng.randint(0, 6))) for _ in range(100_000)]
    for j in range(200):
        i = 6 * j + 1
        items[i] = bytes(rng.choice(b"ab") for _ in range(100_000))
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    st = sss.sss_get_last_stats()
    assert st.alphabet_symbols == 2 and st.alphabet_group == 5


def test_profiled_run_times_the_alphabet_kernels():
    sss.sss_set_options(alphabet=1, profile=1)
    s = gen.generate(3, 100_000, 72)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    st = sss.sss_get_last_stats().as_dict()
    assert st["profile"]["alphabet"]["launches"] == 2  # sampled character scan, packing
    assert st["profile"]["alphabet"]["ms"] > 0.0
    tl = sss.sss_get_last_timeline()
    assert sum(1 for c, a, b in tl if c == "alphabet") == 2


def test_sort_host_and_batched_with_alphabet():
    sss.sss_set_options(alphabet=1)
    s = gen.generate(3, 50_000, 73)
    h_perm = np.empty(s.n, dtype=np.uint32)
    h_lcp = np.empty(s.n, dtype=np.uint32)
    sss.sss_sort_host(s.chars, len(s.chars), s.offsets, s.n, h_perm, h_lcp)
    assert_same(s, h_perm, h_lcp)
    # batched: sets of mixed alphabets share one rewrite (the union alphabet)
    sizes = [0, 1, 700, 2049, 5000]
    parts = [gen.generate(3, m, 740 + j) for j, m in enumerate(sizes)]
    items = [p.get(i) for p in parts for i in range(p.n)]
    b = gen.from_list(items)
    set_begin = np.zeros(len(sizes) + 1, dtype=np.uint64)
    set_begin[1:] = np.cumsum(sizes)
    chars, offsets = to_dev(b)
    perm = torch.full((b.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((b.n,), -1, dtype=torch.int32, device="cuda")
    sss.sss_sort_batched(chars, offsets, b.n, set_begin, len(sizes), perm, lcp)
    torch.cuda.synchronize()
    perm, lcp = u32(perm), u32(lcp)
    for j, p in enumerate(parts):
        lo, hi = int(set_begin[j]), int(set_begin[j + 1])
        rp, rl = oracle.sort(p.chars, p.offsets)
        assert np.array_equal(perm[lo:hi], rp), j
        assert np.array_equal(lcp[lo:hi], rl), j


def test_full_size_dna_20m_verified():
    # the unique answer at the full workload, checked by the oracle entry by entry
    sss.sss_set_options(alphabet=1, graph=1)
    s = gen.workload("dna-20m")
    perm, lcp = gpu_sort(s)
    code, bad = oracle.verify(s.chars, s.offsets, perm, lcp)
    assert code == 0, (oracle.VERIFY_CODES[code], bad)
    st = sss.sss_get_last_stats()
    assert st.alphabet_group == 3


def test_release_frees_and_sorting_resumes():
    # sss_release drops the workspace, the graph cache and the alphabet
    # buffers; the next calls allocate again and still sort correctly
    s = gen.generate(3, 30_000, 75)
    for graph in (0, 1):
        sss.sss_set_options(alphabet=1, graph=graph)
        perm, lcp = gpu_sort(s)
        assert_same(s, perm, lcp)
        sss.sss_release()
        perm, lcp = gpu_sort(s)
        assert_same(s, perm, lcp)
        assert sss.sss_get_last_stats().alphabet_group == 3
