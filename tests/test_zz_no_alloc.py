"""qr_factor_d_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory (it uses a fixed scratch array compiled into
the library instead of a caller buffer). Called through the C ABI and
compared with qr_factor_d on the same inputs, two calls in a row each.

Kept in its own file, named to be collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1102_5328_gb300 import inputs


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("m,n,nb,ib", [(512, 512, 128, 32), (700, 300, 64, 16), (333, 333, 96, 9)])
def test_noalloc_matches_qr_factor_d(q, m, n, nb, ib):
    L = q.lib()
    A_np = inputs.uniform_matrix(m, n, seed=m + 3 * n)
    t_elems, sbytes = q.qr_workspace(m, n, nb, ib)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    # reference: the entry point with a caller-owned scratch buffer
    A_ref = _dev(A_np)
    T_ref = torch.zeros(t_elems, dtype=torch.float64, device="cuda")
    scratch = torch.empty(sbytes, dtype=torch.uint8, device="cuda")
    assert L.qr_factor_d(m, n, _ptr(A_ref), m, nb, ib, _ptr(T_ref), _ptr(scratch), sbytes, sp) == 0
    for call in range(2):
        A = _dev(A_np)
        T = torch.zeros(t_elems, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert L.qr_factor_d_noalloc(m, n, _ptr(A), m, nb, ib, _ptr(T), _ptr(st), sp) == 0
        torch.cuda.synchronize()
        assert int(st.item()) == 0, call
        # every tile sees the same operation sequence, so the two agree
        # exactly (tolerance 0, as in the determinism test)
        assert torch.equal(A, A_ref), call
        assert torch.equal(T, T_ref), call


def test_noalloc_rejects_oversize(q):
    L = q.lib()
    A = torch.empty(1, dtype=torch.float64, device="cuda")
    # 4096 x 4096 needs 128 MiB of scratch, more than the fixed array; the
    # code (QR_NOALLOC_TOO_LARGE) differs from every argument error
    rc = L.qr_factor_d_noalloc(4096, 4096, _ptr(A), 4096, 128, 32, _ptr(A), None, None)
    assert rc == -100
    # a bad argument still reports its position
    assert L.qr_factor_d_noalloc(-1, 4, _ptr(A), 4, 128, 32, _ptr(A), None, None) == -1
