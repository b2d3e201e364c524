"""fw_reduce_noalloc: contact reduction for callers that may not allocate device memory.

Some programs cannot call cudaMalloc once they run: a control loop with a hard latency
budget (an allocation can stall the whole device), or a host whose memory pool owns the
GPU.  fw_reduce_noalloc serves them: the caller passes device input and output buffers and
the call's scratch is a fixed block inside the library.  This file checks, through the C
ABI, that it returns exactly what fw_reduce returns, on two calls in a row (the second one
finds the first call's data still in the shared scratch).  It runs last so that a run
stopping at the first failure has already run every other test, and it passes both alone
and after the others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2205_03532_b300 import scenes as S


def _candidates(seed, n, max_sample, clusters=9):
    rng = np.random.default_rng(seed)
    from paper_2205_03532_b300 import fw
    c = np.zeros(n, fw.CANDIDATE_DTYPE)
    c["sample"] = np.sort(rng.choice(max_sample, n, replace=False))
    dirs = rng.normal(size=(clusters, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    nn = dirs[rng.integers(0, clusters, n)] + 0.05 * rng.normal(size=(n, 3))
    c["n"] = nn / np.linalg.norm(nn, axis=1)[:, None]
    c["phi"] = rng.uniform(-2e-4, 1e-4, n)
    c["x"] = rng.uniform(-0.01, 0.01, (n, 3))
    return c


def _noalloc(w, cands, cap, spare=0):
    """fw_reduce_noalloc on device copies of cands; the output buffer holds `spare` more
    contacts than cap, filled with a 0xA5 byte pattern; returns (contacts, count, patches,
    the spare bytes after the call)."""
    import torch
    from paper_2205_03532_b300 import fw
    raw = torch.from_numpy(cands.view(np.uint8).copy()).cuda()
    out = torch.zeros((cap + spare) * fw.CONTACT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    out[cap * fw.CONTACT_DTYPE.itemsize:] = 0xA5
    counts = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    # the inputs were written on torch's stream; the call runs on the world's own stream
    torch.cuda.current_stream().synchronize()
    w.reduce_noalloc(raw, len(cands), out, cap, counts)
    w.sync()
    k, npatch = counts.cpu().tolist()
    host = out.cpu().numpy()
    res = host[: cap * fw.CONTACT_DTYPE.itemsize].view(fw.CONTACT_DTYPE)
    return res[: max(0, min(k, cap))].copy(), k, npatch, host[cap * fw.CONTACT_DTYPE.itemsize:]


def _same(a, b):
    for f in ("sample", "patch", "pair"):
        np.testing.assert_array_equal(a[f], b[f])
    for f in ("phi", "xa", "xb", "n"):
        np.testing.assert_array_equal(a[f], b[f])      # same device code: bit-identical


def test_noalloc_matches_fw_reduce_on_two_calls_in_a_row():
    from paper_2205_03532_b300 import fw
    w = fw.World(max_patches=128)
    inputs = [_candidates(1, 3000, 5000), _candidates(2, 2500, 60000, clusters=14)]
    for c in inputs:
        ref, ref_np = w.reduce(c)
        got, k, npatch, _ = _noalloc(w, c, cap=7 * 256)
        assert k == len(ref) and npatch == ref_np
        _same(got, ref)


def test_noalloc_reports_overflow_through_the_count():
    """With cap below the number of contacts the call writes the first cap contacts (the
    same as fw_reduce's first cap), reports the full count in counts[0] and writes nothing
    past entry cap - 1."""
    from paper_2205_03532_b300 import fw
    w = fw.World(max_patches=128)
    c = _candidates(4, 3000, 5000)
    ref, ref_np = w.reduce(c)
    cap = len(ref) // 3
    assert cap > 0
    got, k, npatch, spare = _noalloc(w, c, cap=cap, spare=64)
    assert k == len(ref) and npatch == ref_np
    _same(got, ref[:cap])
    assert np.all(spare == 0xA5)


def test_noalloc_rejects_bad_input():
    from paper_2205_03532_b300 import fw
    w = fw.World()
    c = _candidates(3, 100, 1000)
    c["sample"][[10, 11]] = c["sample"][[11, 10]]          # out of order: rejected on the device
    _, k, npatch, _ = _noalloc(w, c, cap=64)
    assert (k, npatch) == (-1, 0)
    big = np.zeros(70000, fw.CANDIDATE_DTYPE)                # beyond the fixed scratch: rejected on the host
    with pytest.raises(fw.FwError) as e:
        w.reduce_noalloc(1, len(big), 1, 1, 1)
    assert e.value.status == -1 and "65536" in str(e.value)
