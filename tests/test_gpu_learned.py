"""Learned bucket proposal: the GPU fit's loss and gradient against the CPU
oracle (FP64), bit-exact sorts with the proposal, and what training gains
over the untrained (uniform) model."""
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


def gpu_loss_grad(theta, u, y):
    t = torch.from_numpy(theta.astype(np.float32)).cuda()
    uu = torch.from_numpy(u.astype(np.float32)).cuda()
    yy = torch.from_numpy(y.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.zeros(len(theta), dtype=torch.float32, device="cuda")
    sss.sss_cdf_loss_grad(t, len(theta), uu, yy, len(u), loss, grad)
    torch.cuda.synchronize()
    return float(loss.item()), grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("M,S,seed", [(16, 50, 1), (64, 2047, 2), (4096, 2047, 3), (4096, 300, 4)])
def test_loss_and_gradient_match_oracle(M, S, seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=0.7, size=M).astype(np.float32)
    # clustered inputs, as key words of real data are
    u = np.sort(np.concatenate([rng.beta(0.3, 3.0, size=S // 2), rng.random(S - S // 2)])).astype(np.float32)
    y = ((np.arange(S) + 0.5) / S).astype(np.float32)
    loss, grad = gpu_loss_grad(theta, u, y)
    t64, u64, y64 = theta.astype(np.float64), u.astype(np.float64), y.astype(np.float64)
    ref_loss = oracle.cdf_loss(t64, u64, y64)
    ref_grad = oracle.cdf_grad(t64, u64, y64)
    assert loss == pytest.approx(ref_loss, rel=2e-4, abs=1e-7)
    scale = np.abs(ref_grad).max()
    assert np.allclose(grad, ref_grad, rtol=5e-3, atol=2e-3 * scale), np.abs(grad - ref_grad).max() / scale


def test_gradient_of_uniform_model_at_its_own_cdf_is_zero():
    # uniform parameters give F(u) = u; with targets y = u the loss and the
    # gradient vanish
    M, S = 256, 1000
    u = np.linspace(0.0005, 0.9995, S).astype(np.float32)
    loss, grad = gpu_loss_grad(np.zeros(M, dtype=np.float32), u, u)
    assert loss < 1e-12
    assert np.abs(grad).max() < 1e-6


def _learned_sort(s):
    chars = torch.from_numpy(s.chars).cuda()
    offsets = torch.from_numpy(s.offsets.view(np.int64)).cuda()
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    ls = sss.sss_sort_learned(chars, offsets, s.n, perm, lcp)
    torch.cuda.synchronize()
    # the call's own stats out-parameter agrees with the library's last stats
    st = sss.sss_get_last_stats()
    assert (ls.proposals, ls.misses, ls.models) == (st.learned_keys, st.learned_misses, st.learned_models)
    assert ls.miss_rate == pytest.approx(ls.misses / ls.proposals if ls.proposals else 0.0)
    return perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32)


def _assert_oracle(s, perm, lcp):
    ref_perm, ref_lcp = oracle.sort(s.chars, s.offsets)
    assert np.array_equal(perm, ref_perm)
    assert np.array_equal(lcp, ref_lcp)


@pytest.mark.parametrize("kind,n,seed", [(2, 400_000, 51), (3, 300_000, 52), (1, 200_000, 53)])
@pytest.mark.parametrize("opts", [{}, dict(base_threshold=16, medium_threshold=16, k_max=4, chunk=2048),
                                  dict(cdf_segments=64, cdf_steps=5)])
def test_learned_sort_is_bit_exact(kind, n, seed, opts):
    if opts:
        sss.sss_set_options(**opts)
    s = gen.generate(kind, n, seed)
    perm, lcp = _learned_sort(s)
    _assert_oracle(s, perm, lcp)
    st = sss.sss_get_last_stats()
    assert st.learned_misses <= st.learned_keys


def test_learned_edge_cases():
    sss.sss_set_options(base_threshold=16, medium_threshold=16, k_max=3, chunk=2048)
    items = ([b"same"] * 3000 + [b"x" * 300 + bytes([65 + i % 7]) for i in range(3000)] +
             [bytes([0xff, c]) for c in range(1, 256)] * 10 + [b""] * 100)
    random.Random(3).shuffle(items)
    s = gen.from_list(items)
    perm, lcp = _learned_sort(s)
    _assert_oracle(s, perm, lcp)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_training_lowers_the_miss_rate(kind):
    # keys shaped like the learned-proposal workload (URL generator) and the
    # other two kinds; cdf_steps = 0 is the untrained uniform model F(u) = u,
    # without which every key descends the tree (miss rate 1)
    s = gen.generate(kind, 2_000_000, 4)
    trained = max(1, sss.sss_get_options().cdf_steps)  # the default fit
    rates = {}
    for steps in (0, trained):
        sss.sss_set_options(cdf_steps=steps)
        perm, lcp = _learned_sort(s)
        st = sss.sss_get_last_stats()
        rates[steps] = st.learned_misses / st.learned_keys
    print("kind %d: miss rate untrained %.4f trained %.4f" % (kind, rates[0], rates[trained]))
    assert rates[trained] < rates[0]
    code, bad = oracle.verify(s.chars, s.offsets, perm, lcp)
    assert code == 0


def test_learned_full_size_url_64m_verified():
    # the 64M-string URL workload the learned proposal is measured on: the
    # unique answer, every entry checked by the oracle one by one
    s = gen.workload("url-64m")
    perm, lcp = _learned_sort(s)
    st = sss.sss_get_last_stats()
    assert st.learned_keys > 0 and st.learned_misses < st.learned_keys and st.learned_models >= 1
    code, bad = oracle.verify(s.chars, s.offsets, perm, lcp)
    assert code == 0, (oracle.VERIFY_CODES[code], bad)
