"""Host-side logic of the tile Cholesky, CPU only (no GPU call): the task
count of the DAG against a brute-force enumeration of its tasks, workspace
sizes, argument checks, and the NB table's closest-order lookup (Sec. 6.1's
interpolation applied to the Cholesky table; ties to the smaller order)."""
import ctypes
import os

import pytest

lib_mod = pytest.importorskip("paper_1102_5328_gb300._lib")


@pytest.fixture(scope="module")
def L():
    return lib_mod.load()


def _brute_count(NT):
    c = 0
    for k in range(NT):
        c += 1                                    # POTRF(k)
        c += sum(1 for i in range(k + 1, NT))     # TRSM(i, k)
        c += sum(1 for i in range(k + 1, NT))     # SYRK(i, k)
        c += sum(1 for i in range(k + 1, NT) for j in range(k + 1, i))  # GEMM(i, j, k)
    return c


@pytest.mark.parametrize("n,nb", [(1, 32), (64, 64), (65, 64), (1000, 128), (10000, 64), (777, 96)])
def test_task_count(L, n, nb):
    NT = (n + nb - 1) // nb
    assert L.chol_task_count_n(n, nb) == _brute_count(NT)


def test_workspace_and_arguments(L):
    b = ctypes.c_int64()
    assert L.chol_workspace(1000, 128, ctypes.byref(b)) == 0
    NT = 8
    assert b.value >= NT * NT * 128 * 128 * 8  # at least the tile copy
    assert L.chol_workspace(1000, 100, ctypes.byref(b)) == -2  # nb not a multiple of 16
    assert L.chol_workspace(1000, 272, ctypes.byref(b)) == -2  # nb above 256
    assert L.chol_workspace(-1, 64, ctypes.byref(b)) == -1
    A = ctypes.c_void_p(0)
    assert L.chol_factor_d(10, A, 10, 64, A, 0, None) == -2   # no matrix
    assert L.chol_factor_d(10, ctypes.c_void_p(8), 5, 64, A, 0, None) == -3   # lda < n
    assert L.chol_factor_d(10, ctypes.c_void_p(8), 10, 48, None, 0, None) == -5  # no scratch
    assert L.chol_factor_d(0, A, 1, 64, None, 0, None) == 0    # empty: nothing to do


def test_table_lookup(L, tmp_path):
    p = tmp_path / "chol.json"
    p.write_text('{\n  "factorization": "cholesky",\n  "entries": [\n'
                 '    {"n": 1000, "nb": 32, "gflops": 1.0},\n'
                 '    {"n": 2000, "nb": 64, "gflops": 1.0},\n'
                 '    {"n": 6000, "nb": 128, "gflops": 1.0}\n  ]\n}\n')
    assert L.chol_load_table(str(p).encode()) == 0
    nb = ctypes.c_int()
    for n, want in [(10, 32), (1400, 32), (1500, 32), (1501, 64), (3999, 64), (4000, 64), (4001, 128), (10 ** 6, 128)]:
        assert L.chol_lookup(n, ctypes.byref(nb)) == 0
        assert nb.value == want, (n, nb.value)
    # put the committed table back (later tests may look NB up)
    tuned = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1102_5328_gb300", "tuned",
                         "gb300_chol_fp64.json")
    if os.path.exists(tuned):
        assert L.chol_load_table(tuned.encode()) == 0
