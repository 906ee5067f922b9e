"""wg_upper_hood_noalloc against wg_upper_hood_ex (GPU).

The no-allocation entry point keeps its bookkeeping in a fixed array inside
the library instead of a caller-provided workspace, for callers that cannot
allocate device memory. It must give the same corners as the workspace form,
and keep giving them on the next call, since every call reuses the array.
The file name sorts last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1203_5004_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    import __graft_entry__ as g
    g.build_library()
    from paper_1203_5004_gb300 import _lib
    return _lib, _lib.load()


@pytest.mark.parametrize("kind,n", [("uniform", 1 << 20), ("band", 3_000_001), ("duplicates", 5_000),
                                    ("uniform", 1 << 26), ("arc", 1 << 18), ("columns", 1)])
def test_noalloc_matches_workspace_form_twice(kind, n):
    L, lib = _lib()
    ps = inputs.make(kind, n, 17)
    pts = torch.from_numpy(ps.points()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    ws = torch.zeros(lib.wg_upper_hood_workspace_size(n), dtype=torch.uint8, device="cuda")
    ref = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    ref_cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    L.check(lib.wg_upper_hood_ex(pts.data_ptr(), n, ref.data_ptr(), ref_cnt.data_ptr(), ws.data_ptr(),
                                 ws.numel(), None, stream), "wg_upper_hood_ex")
    want = ref[: int(ref_cnt.item())].cpu().numpy()
    # exact: corner indices are integers, and the oracle agrees
    assert np.array_equal(want, oracle.upper_hull(ps.kx, ps.ky))
    for call in range(2):
        out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        L.check(lib.wg_upper_hood_noalloc(pts.data_ptr(), n, out.data_ptr(), cnt.data_ptr(), stream),
                "wg_upper_hood_noalloc")
        got = out[: int(cnt.item())].cpu().numpy()
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_rejects_bad_sizes():
    L, lib = _lib()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    assert lib.wg_upper_hood_noalloc(p, -1, p, p, None) == 1
    assert lib.wg_upper_hood_noalloc(p, 1 << 31, p, p, None) == 7
