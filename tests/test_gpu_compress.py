"""The standalone (I, V) compression (Sec. 3.2) through the C ABI: dense ids of
the distinct (row id, code) pairs, checked against numpy's unique on the host.
Which pair gets which id is unspecified, so the test compares what is unique
(the partition of the rows, the count) and checks the rest is valid."""
import numpy as np
import pytest
import torch

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def ctx():
    from paper_2212_11296_gb300 import VQNQS
    return VQNQS(4, True, 1.0, 1, 64, 2, 4, si.make_weights(16, 1, 64, 4))


@pytest.mark.parametrize("R,n_uid,n_code", [(0, 1, 1), (1, 5, 5), (1000, 30, 7), (300000, 5000, 256),
                                            (70000, 1 << 30, 65535)])
def test_compress_rows_partition(R, n_uid, n_code):
    m = ctx()
    rng = np.random.default_rng(R)
    uid = rng.integers(0, n_uid, R, dtype=np.int64).astype(np.int32)
    code = rng.integers(0, n_code, R, dtype=np.int64).astype(np.int32)
    new_id, rep_uid, rep_code, count = m.compress_rows(torch.as_tensor(uid).cuda(), torch.as_tensor(code).cuda())
    torch.cuda.synchronize()
    U = int(count.item())
    pairs = uid.astype(np.int64) * 65536 + code
    uniq, inv = np.unique(pairs, return_inverse=True)
    assert U == len(uniq)
    nid = new_id.cpu().numpy()
    assert np.all((nid >= 0) & (nid < max(U, 1))) if R else True
    if R:
        # same pair <-> same id
        first_id = np.full(len(uniq), -1)
        first_id[inv] = nid
        assert np.array_equal(first_id[inv], nid)
        assert len(np.unique(nid)) == U
        ru, rc = rep_uid.cpu().numpy(), rep_code.cpu().numpy()
        assert np.array_equal(ru[nid], uid) and np.array_equal(rc[nid], code)
    assert m.stats()["device_status"] == 0
