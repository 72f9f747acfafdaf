"""Host-side logic of the tile LU, CPU only (no GPU call): the task count of
its DAG against a brute-force enumeration of the tasks, workspace sizes and
argument checks."""
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
        c += 1                                                      # GETRF(k)
        c += sum(1 for j in range(k + 1, NT))                       # GESSM(k, j)
        c += sum(1 for i in range(k + 1, NT))                       # TSTRF(i, k)
        c += sum(1 for i in range(k + 1, NT) for j in range(k + 1, NT))  # SSSSM(i, j, k)
    return c


@pytest.mark.parametrize("n,nb", [(1, 8), (64, 64), (65, 64), (1000, 64), (10000, 64), (777, 48), (100, 8)])
def test_task_count(L, n, nb):
    NT = (n + nb - 1) // nb
    assert L.lu_task_count_n(n, nb) == _brute_count(NT)
    assert L.lu_task_count_n(n, 0) == _brute_count((n + 63) // 64)


def test_workspace_and_arguments(L):
    pe, sb = ctypes.c_int64(), ctypes.c_int64()
    assert L.lu_workspace(1000, 64, ctypes.byref(pe), ctypes.byref(sb)) == 0
    NT = 16
    assert pe.value == NT * NT * 64
    assert sb.value >= NT * NT * 64 * 64 * 8  # at least the tile copy
    assert L.lu_workspace(1000, 0, ctypes.byref(pe), ctypes.byref(sb)) == 0 and pe.value == NT * NT * 64
    assert L.lu_workspace(1000, 72, ctypes.byref(pe), ctypes.byref(sb)) == -4  # nb above 64
    assert L.lu_workspace(1000, 4, ctypes.byref(pe), ctypes.byref(sb)) == -4   # nb below 8
    assert L.lu_workspace(-1, 64, ctypes.byref(pe), ctypes.byref(sb)) == -1
    assert L.lu_task_count_n(100, 100) == -1
    Z = ctypes.c_void_p(0)
    P = ctypes.c_void_p(8)
    assert L.lu_factor_d(10, Z, 10, 64, P, P, 1 << 20, None) == -2           # no matrix
    assert L.lu_factor_d(10, P, 5, 64, P, P, 1 << 20, None) == -3            # lda < n
    assert L.lu_factor_d(10, P, 10, 65, P, P, 1 << 20, None) == -4           # nb
    assert L.lu_factor_d(10, P, 10, 8, None, P, 1 << 20, None) == -5         # no pivot records
    assert L.lu_factor_d(10, P, 10, 8, P, None, 1 << 20, None) == -6         # no scratch
    assert L.lu_factor_d(10, P, 10, 8, P, P, 16, None) == -7                 # scratch too small
    assert L.lu_factor_d(0, Z, 1, 64, None, None, 0, None) == 0              # empty: nothing to do
    assert L.lu_status(None, ctypes.byref(ctypes.c_int()), None, None) == -1


def test_table_lookup(L, tmp_path):
    p = tmp_path / "lu.json"
    p.write_text('{\n  "factorization": "lu",\n  "entries": [\n'
                 '    {"n": 1000, "nb": 32, "gflops": 1.0},\n'
                 '    {"n": 2000, "nb": 48, "gflops": 1.0},\n'
                 '    {"n": 6000, "nb": 64, "gflops": 1.0}\n  ]\n}\n')
    try:
        assert L.lu_load_table(str(p).encode()) == 0
        nb = ctypes.c_int()
        for n, want in [(10, 32), (1500, 32), (1501, 48), (4000, 48), (4001, 64), (10 ** 6, 64)]:
            assert L.lu_lookup(n, ctypes.byref(nb)) == 0
            assert nb.value == want, (n, nb.value)
        pe, sb = ctypes.c_int64(), ctypes.c_int64()
        assert L.lu_workspace(1000, 0, ctypes.byref(pe), ctypes.byref(sb)) == 0 and pe.value == 32 * 32 * 32
        bad = tmp_path / "bad.json"
        bad.write_text('{"entries": [\n    {"n": 1000, "nb": 128, "gflops": 1.0}\n]}\n')
        assert L.lu_load_table(str(bad).encode()) == -1  # nb outside 8..64
    finally:
        L.lu_clear_table()
        nb = ctypes.c_int()
        assert L.lu_lookup(5000, ctypes.byref(nb)) == 0 and nb.value == 64  # built-in default
        path = os.path.join(os.path.dirname(lib_mod.__file__), "tuned", "gb300_lu_fp64.json")
        if os.path.exists(path):
            assert L.lu_load_table(path.encode()) == 0
