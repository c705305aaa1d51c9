"""sss_sort_noalloc: the sort for callers that cannot allocate device memory
(its scratch is a static device array of the library).  Its output must
equal sss_sort's, exactly (integer work), on consecutive calls that reuse the
same static scratch.  Kept in a file of its own, collected last."""
import numpy as np
import pytest

import gen
import paper_1305_1157_gb300 as sss
from paper_1305_1157_gb300 import build as sbuild

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_STRINGS = 1 << 16


@pytest.fixture(scope="module", autouse=True)
def built():
    sbuild.build()
    sss.load()


def _dev(s):
    return (torch.from_numpy(s.chars).cuda(), torch.from_numpy(s.offsets.view(np.int64)).cuda())


def _run(fn, s):
    chars, offsets = _dev(s)
    perm = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    lcp = torch.full((s.n,), -1, dtype=torch.int32, device="cuda")
    fn(chars, offsets, s.n, perm, lcp)
    torch.cuda.synchronize()
    return perm.cpu().numpy().view(np.uint32), lcp.cpu().numpy().view(np.uint32)


def test_noalloc_matches_sss_sort_on_two_calls_in_a_row():
    inputs = [gen.generate(2, MAX_STRINGS, 71), gen.generate(3, 40_000, 72)]
    got = [_run(sss.sss_sort_noalloc, s) for s in inputs]  # back to back on the shared scratch
    for s, (perm, lcp) in zip(inputs, got):
        ref_perm, ref_lcp = _run(sss.sss_sort, s)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(lcp, ref_lcp)


def test_noalloc_rejects_more_than_its_maximum():
    s = gen.generate(1, MAX_STRINGS + 1, 73)
    with pytest.raises(sss.SSSError) as e:
        _run(sss.sss_sort_noalloc, s)
    assert e.value.code == -5
