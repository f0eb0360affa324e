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


def _outputs(uid):
    R = uid.numel()
    return [torch.empty(R, dtype=torch.int32, device=uid.device) for _ in range(3)] + [
        torch.empty(1, dtype=torch.int32, device=uid.device)]


def _call(lib, uid, code, out):
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    return lib.vqnqs_compress_rows_noalloc(uid.numel(), p(uid), p(code), p(out[0]), p(out[1]), p(out[2]),
                                           p(out[3]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _noalloc(lib, uid, code):
    out = _outputs(uid)
    assert _call(lib, uid, code, out) == 0
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


def test_noalloc_allocates_nothing_and_replays_in_a_graph():
    """After a first eager call (which looks up the array's address), a call
    takes no device memory, neither from PyTorch's allocator nor from the
    driver, and a call captured into a CUDA graph gives the same result on
    replay, also on a second input copied into the captured buffers."""
    from paper_2212_11296_gb300 import VQNQS
    from paper_2212_11296_gb300.api import lib
    m = VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))
    rng = np.random.default_rng(12)
    R = 150000
    inputs = []
    for n_uid, n_code in [(3000, 256), (50000, 40)]:
        uid = torch.as_tensor(rng.integers(0, n_uid, R).astype(np.int32)).cuda()
        code = torch.as_tensor(rng.integers(0, n_code, R).astype(np.int32)).cuda()
        inputs.append((uid, code, m.compress_rows(uid, code)))
    uid, code = inputs[0][0].clone(), inputs[0][1].clone()
    out = _outputs(uid)
    assert _call(lib(), uid, code, out) == 0  # first call: address lookup, kernels loaded
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call(lib(), uid, code, out) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] >= free0
    _same_result(inputs[0][2], out, uid, code)

    for t in out:
        t.fill_(-7)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(g):
        rcs.append(_call(lib(), uid, code, out))
    assert rcs == [0]
    for u_in, c_in, ref in inputs:
        uid.copy_(u_in)
        code.copy_(c_in)
        for t in out:
            t.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        _same_result(ref, out, u_in, c_in)


def test_noalloc_rejects_too_many_rows():
    from paper_2212_11296_gb300 import _lib
    from paper_2212_11296_gb300.api import lib
    z = ctypes.c_void_p(0)
    assert lib().vqnqs_compress_rows_noalloc(_lib.NOALLOC_MAX_ROWS + 1, z, z, z, z, z, z, z) == 1
