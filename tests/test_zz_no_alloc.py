"""vqnqs_compress_rows_noalloc, the allocation-free variant of the (I, V)
compression for callers that cannot allocate device memory (for instance
while a stream is being captured into a CUDA graph): called through the C ABI
twice in a row, its output must match vqnqs_compress_rows on the same input.
New ids are dense but their assignment order is unspecified, so the test
compares what is unique: the count, the partition of the rows, and that every
row's id maps back to the row's own pair.  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _noalloc(lib, uid, code):
    R = uid.numel()
    dev = uid.device
    out = [torch.empty(R, dtype=torch.int32, device=dev) for _ in range(3)] + [torch.empty(1, dtype=torch.int32,
                                                                                          device=dev)]
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.vqnqs_compress_rows_noalloc(R, p(uid), p(code), p(out[0]), p(out[1]), p(out[2]), p(out[3]),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    return out


def _same_result(a, b, uid, code):
    (ia, ua, ca, na), (ib, ub, cb, nb) = a, b
    assert int(na.item()) == int(nb.item())
    ia, ib = ia.cpu().numpy(), ib.cpu().numpy()
    # same partition of the rows: a bijection between the two id sets
    pairs = set(zip(ia.tolist(), ib.tolist()))
    assert len(pairs) == int(na.item()) == len(set(ia.tolist())) == len(set(ib.tolist()))
    u, c = uid.cpu().numpy(), code.cpu().numpy()
    assert np.array_equal(ua.cpu().numpy()[ia], u) and np.array_equal(ca.cpu().numpy()[ia], c)
    assert np.array_equal(ub.cpu().numpy()[ib], u) and np.array_equal(cb.cpu().numpy()[ib], c)


def test_noalloc_matches_compress_rows_twice():
    from paper_2212_11296_gb300 import VQNQS, _lib
    from paper_2212_11296_gb300.api import lib
    m = VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))
    rng = np.random.default_rng(11)
    for R, n_uid, n_code in [(200000, 4000, 256), (_lib.NOALLOC_MAX_ROWS, 1 << 20, 300)]:
        uid = torch.as_tensor(rng.integers(0, n_uid, R).astype(np.int32)).cuda()
        code = torch.as_tensor(rng.integers(0, n_code, R).astype(np.int32)).cuda()
        ref = m.compress_rows(uid, code)
        first = _noalloc(lib(), uid, code)
        second = _noalloc(lib(), uid, code)
        torch.cuda.synchronize()
        _same_result(ref, first, uid, code)
        _same_result(ref, second, uid, code)


def test_noalloc_rejects_too_many_rows():
    from paper_2212_11296_gb300 import _lib
    from paper_2212_11296_gb300.api import lib
    z = ctypes.c_void_p(0)
    assert lib().vqnqs_compress_rows_noalloc(_lib.NOALLOC_MAX_ROWS + 1, z, z, z, z, z, z, z) == 1
