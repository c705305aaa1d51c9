"""GPU parity: every step and the whole sort, through the C ABI, against the
CPU oracle on the same seeded inputs.  Integer work: results must be
bit-identical."""
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
    offsets = torch.from_numpy(s.offsets.view(np.int64)).cuda() if s.n else torch.zeros(1, dtype=torch.int64,
                                                                                        device="cuda")
    return chars, offsets


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_sort(s, learned=False):
    chars, offsets = to_dev(s)
    n = s.n
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    (sss.sss_sort_learned if learned else sss.sss_sort)(chars, offsets, n, perm, lcp)
    torch.cuda.synchronize()
    return u32(perm[:n]), u32(lcp[:n])


def assert_same(s, perm, lcp):
    ref_perm, ref_lcp = oracle.sort(s.chars, s.offsets)
    if not np.array_equal(perm, ref_perm):
        i = int(np.nonzero(perm != ref_perm)[0][0])
        raise AssertionError(f"perm differs first at rank {i}: gpu {perm[i]} oracle {ref_perm[i]}")
    if not np.array_equal(lcp, ref_lcp):
        i = int(np.nonzero(lcp != ref_lcp)[0][0])
        raise AssertionError(f"lcp differs first at rank {i}: gpu {lcp[i]} oracle {ref_lcp[i]}")


def rand_strings(rng, n, maxlen, alphabet, prefixes=(b"",), dup_frac=0.1):
    out = []
    for _ in range(n):
        p = rng.choice(prefixes)
        out.append(p + bytes(rng.choice(alphabet) for _ in range(rng.randint(0, maxlen))))
    for _ in range(int(n * dup_frac)):
        out[rng.randrange(n)] = out[rng.randrange(n)]
    return out


# ------------------------------------------------------------------ steps

def test_gather_keys_every_alignment_and_depth():
    rng = random.Random(1)
    items = rand_strings(rng, 600, 40, [1, 2, 0x61, 0x7f, 0x80, 0xfe, 0xff])
    s = gen.from_list(items)
    pairs = [(i, d) for i, w in enumerate(items) for d in range(0, len(w) + 1)]
    idx = np.array([p[0] for p in pairs], dtype=np.uint32)
    dep = np.array([p[1] for p in pairs], dtype=np.uint32)
    chars, offsets = to_dev(s)
    out = torch.zeros(len(pairs), dtype=torch.int64, device="cuda")
    sss.sss_gather_keys(chars, offsets, torch.from_numpy(idx).cuda(), torch.from_numpy(dep).cuda(), len(pairs), out)
    got = out.cpu().numpy().view(np.uint64)
    ref = np.array([oracle.key_word(s.chars, int(s.offsets[i]), int(d)) for i, d in pairs], dtype=np.uint64)
    assert np.array_equal(got, ref)
    assert len({int(o) % 16 for o in s.offsets}) == 16


@pytest.mark.parametrize("k", list(range(1, 11)))
def test_build_splitters_matches_oracle(k):
    rng = np.random.default_rng(k)
    full = 2 ** (k + 1) - 1
    for count, distinct in ((full, 1 << 40), (full, 3), (full, max(2, full // 4)), (1, 5), (max(1, full // 3), 7)):
        sample = rng.integers(0, distinct, size=count, dtype=np.uint64) * np.uint64(0x0101010101)
        level = torch.zeros(2 ** k - 1, dtype=torch.int64, device="cuda")
        ino = torch.zeros(2 ** k - 1, dtype=torch.int64, device="cuda")
        sss.sss_build_splitters(torch.from_numpy(sample.view(np.int64)).cuda(), count, k, level, ino)
        ref_level, ref_ino = oracle.select_splitters(np.sort(sample), k)
        assert np.array_equal(level.cpu().numpy().view(np.uint64), ref_level)
        assert np.array_equal(ino.cpu().numpy().view(np.uint64), ref_ino)
    # keys equal to the all-ones padding of the sorted sample: their run of
    # equal keys must end at the sample's end, not run on into the padding
    for count in (full, max(1, full - 2)):
        sample = rng.choice(np.array([0, 7, 2 ** 64 - 1], dtype=np.uint64), size=count)
        level = torch.zeros(2 ** k - 1, dtype=torch.int64, device="cuda")
        ino = torch.zeros(2 ** k - 1, dtype=torch.int64, device="cuda")
        sss.sss_build_splitters(torch.from_numpy(sample.view(np.int64)).cuda(), count, k, level, ino)
        ref_level, ref_ino = oracle.select_splitters(np.sort(sample), k)
        assert np.array_equal(level.cpu().numpy().view(np.uint64), ref_level)
        assert np.array_equal(ino.cpu().numpy().view(np.uint64), ref_ino)


def _classify_gpu(keys, level, ino, k):
    out = torch.zeros(len(keys), dtype=torch.int16, device="cuda")
    sss.sss_classify(torch.from_numpy(keys.view(np.int64)).cuda(), len(keys),
                     torch.from_numpy(level.view(np.int64)).cuda(), torch.from_numpy(ino.view(np.int64)).cuda(),
                     k, out)
    return out.cpu().numpy().view(np.uint16).astype(np.int64)


def test_classify_fig1():
    # Fig. 1: v = 3 splitters, buckets b_0..b_6
    x = np.array([10, 20, 30], dtype=np.uint64)
    level = np.array([20, 10, 30], dtype=np.uint64)
    keys = np.array([0, 9, 10, 11, 19, 20, 21, 29, 30, 31, 2 ** 64 - 1], dtype=np.uint64)
    assert list(_classify_gpu(keys, level, x, 2)) == [0, 0, 1, 2, 2, 3, 4, 4, 5, 6, 6]


@pytest.mark.parametrize("k", [1, 4, 10])
def test_classify_matches_oracle(k):
    rng = np.random.default_rng(100 + k)
    sample = rng.integers(0, 50, size=2 ** (k + 1) - 1, dtype=np.uint64) << np.uint64(56)
    level, ino = oracle.select_splitters(np.sort(sample), k)
    keys = np.concatenate([rng.integers(0, 51, size=3000, dtype=np.uint64) << np.uint64(56),
                           rng.integers(0, 2 ** 63, size=3000, dtype=np.uint64), ino])
    got = _classify_gpu(keys, level, ino, k)
    ref = np.array([oracle.classify(int(q), ino) for q in keys])
    assert np.array_equal(got, ref)


def _classify_equal_gpu(keys, level, k):
    kd = torch.from_numpy(keys.view(np.int64)).cuda()
    ld = torch.from_numpy(level.view(np.int64)).cuda()
    out = torch.zeros(len(keys), dtype=torch.int16, device="cuda")
    sss.sss_classify_equal(kd, len(keys), ld, k, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16).astype(np.int64)


def test_classify_equal_fig1():
    level = np.array([20, 10, 30], dtype=np.uint64)
    keys = np.array([0, 9, 10, 11, 19, 20, 21, 29, 30, 31, 2 ** 64 - 1], dtype=np.uint64)
    assert list(_classify_equal_gpu(keys, level, 2)) == [0, 0, 1, 2, 2, 3, 4, 4, 5, 6, 6]


@pytest.mark.parametrize("k", [1, 4, 10])
def test_classify_equal_matches_oracle(k):
    # distinct splitters: the pS5-Equal descent gives the oracle's buckets;
    # repeated splitters: every bucket is a valid one for its key (an odd
    # bucket holds keys equal to its splitter, an even one keys strictly
    # between its neighbours) and equal keys share a bucket
    rng = np.random.default_rng(200 + k)
    sample = np.unique(rng.integers(0, 2 ** 40, size=4 * 2 ** (k + 1), dtype=np.uint64))
    sample = rng.permutation(sample)[:2 ** (k + 1) - 1] << np.uint64(20)
    level, ino = oracle.select_splitters(np.sort(sample), k)
    keys = np.concatenate([rng.integers(0, 2 ** 60, size=3000, dtype=np.uint64), ino, ino + np.uint64(1)])
    got = _classify_equal_gpu(keys, level, k)
    ref = np.array([oracle.classify(int(q), ino) for q in keys])
    assert np.array_equal(got, ref)
    dup = rng.integers(0, 20, size=2 ** (k + 1) - 1, dtype=np.uint64) << np.uint64(56)
    level, ino = oracle.select_splitters(np.sort(dup), k)
    keys = np.concatenate([rng.integers(0, 21, size=3000, dtype=np.uint64) << np.uint64(56), ino])
    got = _classify_equal_gpu(keys, level, k)
    v = len(ino)
    for q, b in zip(keys.tolist(), got.tolist()):
        j = b >> 1
        if b & 1:
            assert ino[j] == q
        else:
            assert (j == 0 or ino[j - 1] < q) and (j == v or q < ino[j])
    first = {}
    for q, b in zip(keys.tolist(), got.tolist()):
        assert first.setdefault(q, b) == b


# ------------------------------------------------------------------ whole sort

def test_uniform_100k_full_workload():
    s = gen.workload("uniform-100k")
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


@pytest.mark.parametrize("key_bytes", [8, 16])
@pytest.mark.parametrize("kind,n,seed", [(2, 300_000, 12), (3, 200_000, 13), (1, 50_000, 14)])
def test_generated_kinds(kind, n, seed, key_bytes):
    sss.sss_set_options(key_bytes=key_bytes)
    s = gen.generate(kind, n, seed)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


# options that push small inputs through many distribution rounds, tiny
# trees and one-tile chunks
SMALL_OPTS = [
    # every bucket above 16 strings through device-wide rounds, tiny trees,
    # one-word keys
    dict(base_threshold=16, medium_threshold=16, k_max=2, chunk=2048, key_bytes=8),
    # small base case, everything else per-CTA rounds
    dict(base_threshold=16, medium_threshold=8192, k_max=10, chunk=2048, key_bytes=16),
    dict(base_threshold=100, medium_threshold=300, k_max=5, chunk=4096, key_bytes=8),
    # defaults
    dict(base_threshold=128, medium_threshold=8192, k_max=10, chunk=16384, key_bytes=16),
    # as above with two-word keys and one-word keys
    dict(base_threshold=16, medium_threshold=16, k_max=2, chunk=2048, key_bytes=16),
    dict(base_threshold=16, medium_threshold=8192, k_max=10, chunk=2048, key_bytes=8),
    # the pS5-Equal classifier
    dict(base_threshold=16, medium_threshold=16, k_max=3, chunk=2048, key_bytes=16, classifier=1),
    dict(base_threshold=128, medium_threshold=2048, k_max=10, chunk=32768, key_bytes=8, classifier=1),
    # radix classification of every device-wide segment whose sample keys
    # differ (F4), both key widths, and the entropy-driven choice
    dict(base_threshold=16, medium_threshold=16, k_max=3, chunk=2048, key_bytes=16, radix=2),
    dict(base_threshold=16, medium_threshold=16, k_max=6, chunk=2048, key_bytes=8, radix=2),
    dict(base_threshold=128, medium_threshold=1024, k_max=10, chunk=8192, key_bytes=16, radix=1),
]


@pytest.mark.parametrize("opts", SMALL_OPTS)
def test_options_sweep_urls(opts):
    sss.sss_set_options(**opts)
    s = gen.generate(2, 60_000, 21)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


@pytest.mark.parametrize("opts", SMALL_OPTS)
def test_options_sweep_dna(opts):
    sss.sss_set_options(**opts)
    s = gen.generate(3, 40_000, 22)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


EDGE_CASES = {
    "one": [b"x"],
    "two_equal": [b"ab", b"ab"],
    "two_empty": [b"", b""],
    "all_empty": [b""] * 5000,
    "all_equal": [b"same string here"] * 9000,
    "all_equal_8": [b"abcdefgh"] * 3000,
    "word_boundaries": [b"a" * L for L in range(0, 40)] * 50,
    "high_bytes": [bytes([0xff, 0x80, c]) for c in range(1, 256)] * 20 + [b"\x7f", b"\x80", b"\x01"],
    "long_prefix_1k": [b"p" * 1100 + bytes([65 + i % 26]) * (i % 5) for i in range(4000)],
    "differ_after_8k": [b"q" * 8200 + bytes([65 + (i * 7) % 26]) for i in range(300)],
    "prefix_chain": [b"z" * L for L in range(0, 600)],
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
@pytest.mark.parametrize("opts", [SMALL_OPTS[0], SMALL_OPTS[1], SMALL_OPTS[3], SMALL_OPTS[4], SMALL_OPTS[5],
                                  SMALL_OPTS[6], SMALL_OPTS[7], SMALL_OPTS[8], SMALL_OPTS[9]])
def test_edge_cases(name, opts):
    sss.sss_set_options(**opts)
    items = list(EDGE_CASES[name])
    random.Random(len(items)).shuffle(items)
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


def test_zero_strings():
    s = gen.from_list([])
    perm, lcp = gpu_sort(s)
    assert len(perm) == 0


def test_random_bytes_many_duplicates_ragged():
    rng = random.Random(5)
    items = rand_strings(rng, 70_001, 24, list(range(1, 256)), prefixes=(b"", b"http://", b"\xff" * 9), dup_frac=0.3)
    s = gen.from_list(items)
    sss.sss_set_options(base_threshold=64, medium_threshold=1000, k_max=6, chunk=2048)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


# ------------------------------------------------------------------ other entry points

def test_sort_host_buffers():
    s = gen.generate(2, 100_000, 31)
    perm = np.zeros(s.n, dtype=np.uint32)
    lcp = np.zeros(s.n, dtype=np.uint32)
    sss.sss_sort_host(s.chars, len(s.chars), s.offsets, s.n, perm, lcp)
    assert_same(s, perm, lcp)


def test_sort_with_caller_workspace():
    s = gen.generate(1, 80_000, 32)
    chars, offsets = to_dev(s)
    nbytes = sss.sss_workspace_size(s.n)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    perm = torch.empty(s.n, dtype=torch.int32, device="cuda")
    lcp = torch.empty(s.n, dtype=torch.int32, device="cuda")
    sss.sss_sort_ws(chars, offsets, s.n, perm, lcp, ws, nbytes)
    torch.cuda.synchronize()
    assert_same(s, u32(perm), u32(lcp))
    with pytest.raises(sss.SSSError) as e:
        sss.sss_sort_ws(chars, offsets, s.n, perm, lcp, ws, nbytes // 2)
    assert e.value.code == -2


@pytest.mark.parametrize("profile", [0, 1])  # graph launch / timed host-driven rounds
def test_batched_matches_per_set_oracle(profile):
    rng = random.Random(8)
    sizes = [0, 1, 2, 3, 17, 1000, 2047, 2048, 2049, 5000, 30000, 1, 0, 777]
    kinds = [rng.choice([1, 2, 3]) for _ in sizes]
    parts = [gen.generate(k, m, 900 + j) for j, (k, m) in enumerate(zip(kinds, sizes))]
    items = [p.get(i) for p in parts for i in range(p.n)]
    s = gen.from_list(items)
    set_begin = np.zeros(len(sizes) + 1, dtype=np.uint64)
    set_begin[1:] = np.cumsum(sizes)
    chars, offsets = to_dev(s)
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    sss.sss_set_options(base_threshold=32, medium_threshold=600, k_max=8, chunk=2048, profile=profile)
    sss.sss_sort_batched(chars, offsets, s.n, set_begin, len(sizes), perm, lcp)
    torch.cuda.synchronize()
    perm, lcp = u32(perm), u32(lcp)
    for j, p in enumerate(parts):
        b, e = int(set_begin[j]), int(set_begin[j + 1])
        rp, rl = oracle.sort(p.chars, p.offsets)
        assert np.array_equal(perm[b:e], rp), j
        assert np.array_equal(lcp[b:e], rl), j


def test_stats_report_rounds():
    s = gen.generate(2, 200_000, 41)
    gpu_sort(s)
    st = sss.sss_get_last_stats().as_dict()
    assert st["rounds"] >= 1
    assert st["round_active"][0] == s.n
    assert st["base_strings"] > 0


# ------------------------------------------------------------------ full sizes

@pytest.mark.parametrize("key_bytes,classifier", [(8, 0), (16, 0), (16, 1)])
@pytest.mark.parametrize("name", ["url-16m", "dna-20m"])
def test_full_size_workloads_verified(name, key_bytes, classifier):
    # the unique answer: permutation, strict (string, index) order of every
    # adjacent pair and every LCP entry, checked by the oracle one by one
    sss.sss_set_options(key_bytes=key_bytes, classifier=classifier)
    s = gen.workload(name)
    perm, lcp = gpu_sort(s)
    code, bad = oracle.verify(s.chars, s.offsets, perm, lcp)
    assert code == 0, (oracle.VERIFY_CODES[code], bad)


# ------------------------------------------------------------------ graph form

@pytest.mark.parametrize("opts", [SMALL_OPTS[0], SMALL_OPTS[1], SMALL_OPTS[3]])
@pytest.mark.parametrize("kind,n,seed", [(2, 200_000, 61), (3, 100_000, 62), (1, 100_000, 63)])
def test_graph_form_matches_oracle(opts, kind, n, seed):
    sss.sss_set_options(graph=1, **opts)
    s = gen.generate(kind, n, seed)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    # the cached graph is relaunched on the same buffers
    chars, offsets = to_dev(s)
    st = sss.sss_get_last_stats()
    assert st.rounds >= 1 and st.launches > 0


@pytest.mark.parametrize("name", ["all_equal", "long_prefix_1k", "two_empty", "one", "high_bytes"])
def test_graph_form_edge_cases(name):
    sss.sss_set_options(graph=1, base_threshold=16, medium_threshold=64, k_max=3, chunk=2048)
    items = list(EDGE_CASES[name])
    random.Random(len(items)).shuffle(items)
    s = gen.from_list(items)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)


def test_graph_relaunch_is_repeatable():
    sss.sss_set_options(graph=1)
    s = gen.generate(2, 300_000, 64)
    chars, offsets = to_dev(s)
    perm = torch.empty(s.n, dtype=torch.int32, device="cuda")
    lcp = torch.empty(s.n, dtype=torch.int32, device="cuda")
    ref_perm, ref_lcp = oracle.sort(s.chars, s.offsets)
    for _ in range(3):
        perm.fill_(-1)
        lcp.fill_(-1)
        sss.sss_sort(chars, offsets, s.n, perm, lcp)
        torch.cuda.synchronize()
        assert np.array_equal(u32(perm), ref_perm)
        assert np.array_equal(u32(lcp), ref_lcp)


def test_graph_form_learned():
    sss.sss_set_options(graph=1)
    s = gen.generate(2, 300_000, 65)
    perm, lcp = gpu_sort(s, learned=True)
    assert_same(s, perm, lcp)


def test_profiled_timeline():
    sss.sss_set_options(profile=1)
    s = gen.generate(2, 200_000, 71)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    tl = sss.sss_get_last_timeline()
    st = sss.sss_get_last_stats()
    assert tl and tl[0][1] == 0.0
    assert all(c in sss.K_CLASSES and 0.0 <= a <= b for c, a, b in tl)
    # every kernel class with timed launches appears in the timeline as often
    for i, c in enumerate(sss.K_CLASSES):
        if c != "scan":  # one timed entry covers the scan's two kernels
            assert sum(1 for x in tl if x[0] == c) == st.prof_launches[i], c


@pytest.mark.parametrize("key_bytes", [8, 16])
@pytest.mark.parametrize("group", [(1500, 97), (300, 53)])
def test_medium_rounds_step_over_shared_prefixes(key_bytes, group):
    # medium-sized groups whose strings share 100+ characters: the medium
    # round steps over them in place (gathering keys deeper) before it moves;
    # groups of 1500..2567 strings take the per-CTA round, groups of 300..883
    # the per-warp one
    rng = random.Random(17)
    items = []
    for gi in range(12):
        prefix = b"group%02d/" % gi + bytes(rng.choice(b"abcdef") for _ in range(100 + 7 * gi))
        for _ in range(group[0] + group[1] * gi):
            items.append(prefix + bytes(rng.choice(b"ab") for _ in range(rng.randint(0, 12))))
    rng.shuffle(items)
    s = gen.from_list(items)
    sss.sss_set_options(base_threshold=32, medium_threshold=8192, k_max=10, chunk=2048, key_bytes=key_bytes)
    perm, lcp = gpu_sort(s)
    assert_same(s, perm, lcp)
    assert sss.sss_get_last_stats().medium_refilled_strings > 0


@pytest.mark.parametrize("opts", [dict(key_bytes=16), dict(key_bytes=8), dict(key_bytes=16, graph=1)])
def test_offsets_beyond_4gib(opts):
    """Strings placed after more than 4 GiB of other bytes in one chars
    buffer (offsets >= 2^32, so every offset and address is 64-bit), mixed
    with strings before that point; compared element by element with the
    oracle on the same strings packed compactly (the answer does not depend
    on where the strings lie)."""
    pad = (1 << 32) + 4099  # odd, so the far strings start at every alignment
    s = gen.generate(2, 60_000, 81)
    cut = s.n // 3
    head_bytes = int(s.offsets[cut])
    if torch.cuda.mem_get_info()[0] < pad + 2 * len(s.chars) + (1 << 30):
        pytest.skip("needs about 5 GB of device memory")
    sss.sss_set_options(**opts)
    chars = torch.zeros(pad + len(s.chars), dtype=torch.uint8, device="cuda")
    body = torch.from_numpy(s.chars).cuda()
    chars[:head_bytes] = body[:head_bytes]          # the first third below 4 GiB
    chars[pad + head_bytes:] = body[head_bytes:]    # the rest beyond it
    off = s.offsets.astype(np.uint64).copy()
    off[cut:] += np.uint64(pad)
    assert int(off[cut]) >= 2**32
    offsets = torch.from_numpy(off.view(np.int64)).cuda()
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    sss.sss_sort(chars, offsets, s.n, perm, lcp)
    torch.cuda.synchronize()
    del chars, body
    torch.cuda.empty_cache()
    assert_same(s, u32(perm), u32(lcp))


@pytest.mark.parametrize("key_bytes", [8, 16])
def test_radix_classification_by_sample_entropy(key_bytes):
    """Option radix = 1 (App. A.2 adaptivity): letters a-z spread the sample's
    digits almost evenly, so device-wide segments take the digit.  Output
    identical to the oracle with and without radix rounds, on letters and on
    DNA (4 characters a byte position: its roots keep the tree)."""
    sss.sss_set_options(base_threshold=16, medium_threshold=64, k_max=10, chunk=2048, key_bytes=key_bytes, radix=1)
    s = gen.generate(1, 300_000, 61)
    perm, lcp = gpu_sort(s)
    assert sss.sss_get_last_stats().radix_segments > 0
    assert_same(s, perm, lcp)
    d = gen.generate(3, 200_000, 62)
    perm, lcp = gpu_sort(d)
    assert_same(d, perm, lcp)
    sss.sss_set_options(radix=0)
    perm0, lcp0 = gpu_sort(s)
    assert sss.sss_get_last_stats().radix_segments == 0
    assert_same(s, perm0, lcp0)


@pytest.mark.parametrize("radix", [1, 2])
def test_radix_graph_and_batched_forms(radix):
    """Radix rounds inside the graph form and the batched sort."""
    sss.sss_set_options(base_threshold=16, medium_threshold=16, k_max=8, chunk=2048, radix=radix, graph=1)
    for kind in (1, 2, 3):
        s = gen.generate(kind, 80_000, 70 + kind)
        perm, lcp = gpu_sort(s)
        assert_same(s, perm, lcp)
    b = gen.generate_batch(120, 100, 3000, 77)
    chars, offsets = to_dev(b.strings)
    perm = torch.full((b.strings.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((b.strings.n,), -1, dtype=torch.int32, device="cuda")
    sss.sss_sort_batched(chars, offsets, b.strings.n, b.set_begin, 120, perm, lcp)
    torch.cuda.synchronize()
    p, l = u32(perm), u32(lcp)
    for j in range(120):
        lo, hi = int(b.set_begin[j]), int(b.set_begin[j + 1])
        ss = gen.set_strings(b, j)
        code, bad = oracle.verify(ss.chars, ss.offsets, p[lo:hi], l[lo:hi])
        assert code == 0, (j, code, bad)
