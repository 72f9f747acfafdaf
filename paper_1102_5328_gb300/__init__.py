"""GB300-native tile Householder QR with an empirical NB/IB autotuner.

The method is Agullo, Dongarra, Nath, Tomov, "A Fully Empirical Autotuned
Dense QR Factorization for Multicore Architectures" (tile QR, Sec. 2; the
empirical tuner, Secs. 5–6), re-designed for one GB300 GPU. The compute
path lives in the CUDA library ``libtileqr.so`` behind the C ABI of
``include/tileqr.h``; this package is its Python binding. PyTorch is used
only for device memory and streams.

Matrices are column-major: a torch tensor ``A`` of shape (m, n) with
``A.stride() == (1, lda)`` (see :func:`colmajor`).
"""
import ctypes
import json
import os

import torch

from . import _lib

QR_PREC_F64 = 0
QR_PREC_F32 = 1
QR_PREC_TF32 = 2
QR_PREC_BF16X3 = 3
QR_DEV_TIMEOUT = 1
QR_DEV_NONFINITE = 2
QR_DEV_NOT_SPD = 4
QR_DEV_SINGULAR = 8
QR_OPT_WAIT_TIMEOUT_US = 1
QR_OPT_CTAS_PER_SM = 2
QR_OPT_SPLIT = 3
QR_OPT_GRID_LIMIT = 4
QR_OPT_DROP_TASK = 5
QR_OPT_RECORD_EVENTS = 6
QR_OPT_ORDER = 7
QR_OPT_PANEL_WEIGHT = 8
QR_OPT_UNMQR_WEIGHT = 9
QR_OPT_LS_REFINE = 10
QR_OPT_GMRES_MAX = 11
QR_OPT_GMRES_TOL_EXP = 12
QR_OPT_SM_BUDGET = 13
QR_OPT_TUNE_IB_TOL = 14


_TUNED_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned")
_tables_loaded = False


def lib():
    """The loaded C library; on first use also installs the committed tuning
    results for this GPU (decision table of qr_tune, batched size classes)."""
    global _tables_loaded
    L = _lib.load()
    if not _tables_loaded:
        _tables_loaded = True
        for name in ("gb300_fp64.json", "gb300_fp32.json"):
            path = os.path.join(_TUNED_DIR, name)
            if os.path.exists(path):
                L.qr_load_table(path.encode())
        for name in ("gb300_fp64_costs.json", "gb300_fp32_costs.json"):
            path = os.path.join(_TUNED_DIR, name)
            if os.path.exists(path):
                with open(path) as f:
                    tab = json.load(f)
                prec = QR_PREC_F32 if tab.get("prec") == "fp32" else QR_PREC_F64
                for e in tab.get("entries", []):
                    c = (ctypes.c_double * 4)(*e["costs"])
                    L.qr_set_task_costs(prec, int(e["nb"]), int(e["ib"]), c)
        path = os.path.join(_TUNED_DIR, "gb300_chol_fp64.json")
        if os.path.exists(path):
            L.chol_load_table(path.encode())
        path = os.path.join(_TUNED_DIR, "gb300_lu_fp64.json")
        if os.path.exists(path):
            L.lu_load_table(path.encode())
        path = os.path.join(_TUNED_DIR, "gb300_batched_classes.json")
        if os.path.exists(path):
            with open(path) as f:
                cls = json.load(f)
            for prec_name, prec in (("f64", QR_PREC_F64), ("f32", QR_PREC_F32)):
                for m_hi, v in cls.get(prec_name, {}).items():
                    L.qr_batched_set_class(prec, int(m_hi), int(v["best"][0]), int(v["best"][1]))
    return L


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def colmajor(x):
    """Column-major copy (or view, when already column-major) of a 2-D tensor."""
    if x.dim() == 1:
        x = x[:, None]
    if x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0]):
        return x
    return x.t().contiguous().t()


def colmajor_empty(m, n, dtype, device="cuda"):
    return torch.empty((n, m), dtype=dtype, device=device).t()


def _prec(dtype):
    if dtype == torch.float64:
        return QR_PREC_F64
    if dtype == torch.float32:
        return QR_PREC_F32
    raise TypeError("dtype must be float64 or float32")


def qr_workspace(m, n, nb, ib, dtype=torch.float64):
    """(t_elems, scratch_bytes) for qr_factor."""
    t = ctypes.c_int64()
    s = ctypes.c_int64()
    _lib.check(lib().qr_workspace(m, n, nb, ib, _prec(dtype), ctypes.byref(t), ctypes.byref(s)), "qr_workspace")
    return t.value, s.value


class Factorization:
    """Result of qr_factor: A overwritten with R and the tile reflectors, the
    T factors, and the scratch buffer (which holds the device status word).
    p is the number of panel domains (1 = flat tree)."""

    def __init__(self, A, T, scratch, nb, ib, p=1):
        self.A, self.T, self.scratch, self.nb, self.ib, self.p = A, T, scratch, nb, ib, p
        self.m, self.n = A.shape

    def R(self):
        return torch.triu(self.A[: self.n, :])

    def status(self, stream=None):
        return qr_status(self.scratch, stream)


def qr_workspace_p(m, n, nb, ib, p, dtype=torch.float64):
    """(t_elems, scratch_bytes) for qr_factor with p panel domains."""
    t = ctypes.c_int64()
    s = ctypes.c_int64()
    _lib.check(lib().qr_workspace_p(m, n, nb, ib, p, _prec(dtype), ctypes.byref(t), ctypes.byref(s)),
               "qr_workspace_p")
    return t.value, s.value


def qr_factor(A, nb=0, ib=0, T=None, scratch=None, stream=None, p=None):
    """Tile QR of A (in place). ``nb = 0`` uses the tuned table (including
    its panel-domain count p for tall-skinny shapes); ``p > 1`` splits every
    panel into domains merged by a binary tree; p = 1 is the flat tree."""
    m, n = A.shape
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.stride(0) != 1:
        raise ValueError("A must be column-major (use colmajor())")
    lda = A.stride(1) if n > 1 else m
    if nb == 0:
        nb, ib, pt = qr_lookup_p(m, n, A.dtype)
        if p is None:
            p = pt
    if p is None:
        p = 1
    if p > 1:
        t_elems, sbytes = qr_workspace_p(m, n, nb, ib, p, A.dtype)
        if T is None or T.numel() < t_elems:
            T = torch.empty(max(t_elems, 1), dtype=A.dtype, device=A.device)
        if scratch is None or scratch.numel() < sbytes:
            scratch = torch.empty(sbytes, dtype=torch.uint8, device=A.device)
        f = lib().qr_factor_p_d if A.dtype == torch.float64 else lib().qr_factor_p_s
        _lib.check(f(m, n, ctypes.c_void_p(A.data_ptr()), lda, nb, ib, p, ctypes.c_void_p(T.data_ptr()),
                     ctypes.c_void_p(scratch.data_ptr()), sbytes, _stream_ptr(stream)), "qr_factor_p")
        return Factorization(A, T, scratch, nb, ib, p)
    t_elems, sbytes = qr_workspace(m, n, nb, ib, A.dtype)
    if T is None or T.numel() < t_elems:
        T = torch.empty(max(t_elems, 1), dtype=A.dtype, device=A.device)
    if scratch is None or scratch.numel() < sbytes:
        scratch = torch.empty(sbytes, dtype=torch.uint8, device=A.device)
    f = lib().qr_factor_d if A.dtype == torch.float64 else lib().qr_factor_s
    _lib.check(f(m, n, ctypes.c_void_p(A.data_ptr()), lda, nb, ib, ctypes.c_void_p(T.data_ptr()),
                 ctypes.c_void_p(scratch.data_ptr()), sbytes, _stream_ptr(stream)), "qr_factor")
    return Factorization(A, T, scratch, nb, ib)


def qr_factor_mixed(A, prec, nb=0, ib=0, p=None, T=None, scratch=None, stream=None):
    """FP32 tile QR of A (float32, in place) with the UNMQR/TSMQR products at
    precision ``prec`` (QR_PREC_F32, QR_PREC_TF32 or QR_PREC_BF16X3) through
    qr_factor_mixed_s; p panel domains (None: the tuned table's, else 1)."""
    m, n = A.shape
    if A.dtype != torch.float32 or not A.is_cuda or A.stride(0) != 1:
        raise ValueError("A must be a column-major float32 CUDA tensor")
    lda = A.stride(1) if n > 1 else m
    if nb == 0:
        nb, ib, pt = qr_lookup_p(m, n, torch.float32)
        if p is None:
            p = pt
    if p is None:
        p = 1
    t_elems, sbytes = qr_workspace_p(m, n, nb, ib, p, torch.float32) if p > 1 else \
        qr_workspace(m, n, nb, ib, torch.float32)
    if T is None or T.numel() < t_elems:
        T = torch.empty(max(t_elems, 1), dtype=torch.float32, device=A.device)
    if scratch is None or scratch.numel() < sbytes:
        scratch = torch.empty(sbytes, dtype=torch.uint8, device=A.device)
    _lib.check(lib().qr_factor_mixed_s(m, n, ctypes.c_void_p(A.data_ptr()), lda, nb, ib, p, prec,
                                       ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(scratch.data_ptr()), sbytes,
                                       _stream_ptr(stream)), "qr_factor_mixed_s")
    return Factorization(A, T, scratch, nb, ib, p)


def qr_apply_qt(fact, C, trans=True, stream=None, parallel=True):
    """C <- Q^T C (trans) or Q C, in place, with the factors of qr_factor.
    parallel=True uses the dependency-ordered persistent kernel
    (qr_apply_qt_ws_*), False the column-chunk kernel (qr_apply_qt_*)."""
    if C.stride(0) != 1:
        raise ValueError("C must be column-major (use colmajor())")
    if C.dtype != fact.A.dtype:
        raise TypeError("C must have the factorization's dtype")
    m, n = fact.m, fact.n
    nrhs = C.shape[1]
    ldc = C.stride(1) if nrhs > 1 else m
    f = lib().qr_apply_qt_d if C.dtype == torch.float64 else lib().qr_apply_qt_s
    lda = fact.A.stride(1) if n > 1 else m
    if getattr(fact, "p", 1) > 1:
        wb = ctypes.c_int64()
        _lib.check(lib().qr_apply_workspace_p(m, n, nrhs, fact.nb, fact.p, ctypes.byref(wb)), "qr_apply_workspace_p")
        ws = torch.empty(wb.value, dtype=torch.uint8, device=C.device)
        f = lib().qr_apply_qt_p_d if C.dtype == torch.float64 else lib().qr_apply_qt_p_s
        _lib.check(f(m, n, nrhs, ctypes.c_void_p(fact.A.data_ptr()), lda, fact.nb, fact.ib, fact.p,
                     ctypes.c_void_p(fact.T.data_ptr()), ctypes.c_void_p(C.data_ptr()), ldc, 1 if trans else 0,
                     ctypes.c_void_p(ws.data_ptr()), wb.value, _stream_ptr(stream)), "qr_apply_qt_p")
        return C
    if parallel:
        wb = ctypes.c_int64()
        _lib.check(lib().qr_apply_workspace(m, n, nrhs, fact.nb, ctypes.byref(wb)), "qr_apply_workspace")
        ws = torch.empty(wb.value, dtype=torch.uint8, device=C.device)
        f = lib().qr_apply_qt_ws_d if C.dtype == torch.float64 else lib().qr_apply_qt_ws_s
        _lib.check(f(m, n, nrhs, ctypes.c_void_p(fact.A.data_ptr()), lda, fact.nb, fact.ib,
                     ctypes.c_void_p(fact.T.data_ptr()), ctypes.c_void_p(C.data_ptr()), ldc, 1 if trans else 0,
                     ctypes.c_void_p(ws.data_ptr()), wb.value, _stream_ptr(stream)), "qr_apply_qt_ws")
        return C
    _lib.check(f(m, n, nrhs, ctypes.c_void_p(fact.A.data_ptr()), lda, fact.nb, fact.ib,
                 ctypes.c_void_p(fact.T.data_ptr()), ctypes.c_void_p(C.data_ptr()), ldc, 1 if trans else 0,
                 _stream_ptr(stream)), "qr_apply_qt")
    return C


def form_q(fact, stream=None, parallel=True):
    """Explicit thin Q (m x n) = Q [I; 0], on the GPU."""
    Q = colmajor_empty(fact.m, fact.n, fact.A.dtype, fact.A.device)
    Q.zero_()
    Q.diagonal().fill_(1)
    return qr_apply_qt(fact, Q, trans=False, stream=stream, parallel=parallel)


def qr_solve_ls(A, B, prec=QR_PREC_F64, nb=0, ib=0, max_iter=0, tol=2.0 ** -52, work=None, stream=None, p=0):
    """min ||A X - B|| (A, B FP64, column-major CUDA tensors; unchanged).
    ``nb = 0`` takes (nb, ib) from the tuned table of the factorization's
    precision, and p too when ``p = 0`` (the C library's p = 0 picks
    ceil(MT/NT) domains). prec: QR_PREC_F64, F32, TF32 or BF16X3. Returns
    (X, info) with info = (corrections, converged, device status, GMRES
    iterations)."""
    m, n = A.shape
    nrhs = B.shape[1]
    if A.dtype != torch.float64 or B.dtype != torch.float64:
        raise TypeError("A and B must be float64")
    if A.stride(0) != 1 or B.stride(0) != 1:
        raise ValueError("A and B must be column-major")
    if nb == 0:
        nb, ib, tp = qr_lookup_p(m, n, torch.float64 if prec == QR_PREC_F64 else torch.float32)
        p = p if p else tp
    wb = ctypes.c_int64()
    _lib.check(lib().qr_solve_ls_workspace(m, n, nrhs, prec, nb, ib, p, ctypes.byref(wb)), "qr_solve_ls_workspace")
    if work is None or work.numel() < wb.value:
        work = torch.empty(wb.value, dtype=torch.uint8, device=A.device)
    X = colmajor_empty(n, nrhs, torch.float64, A.device)
    info = (ctypes.c_int * 4)()
    lda = A.stride(1) if n > 1 else m
    ldb = B.stride(1) if nrhs > 1 else m
    ldx = X.stride(1) if nrhs > 1 else n
    _lib.check(lib().qr_solve_ls(m, n, nrhs, ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(B.data_ptr()), ldb,
                                 ctypes.c_void_p(X.data_ptr()), ldx, prec, nb, ib, p, max_iter, tol, info,
                                 ctypes.c_void_p(work.data_ptr()), wb.value, _stream_ptr(stream)), "qr_solve_ls")
    return X, tuple(info)


class BatchedPlan:
    """Device-side descriptors of a batched QR (qr_batched_plan + upload)."""

    def __init__(self, mats, force_nb=0, force_ib=0):
        count = len(mats)
        dtype = mats[0].dtype
        dev = mats[0].device
        ms = [int(a.shape[0]) for a in mats]
        ns = [int(a.shape[1]) for a in mats]
        I = ctypes.c_int * count
        nb, ib, order = I(), I(), I()
        toff = (ctypes.c_int64 * count)()
        ttot = ctypes.c_int64()
        _lib.check(lib().qr_batched_plan(count, I(*ms), I(*ns), _prec(dtype), force_nb, force_ib, nb, ib, order, toff,
                                         ctypes.byref(ttot)), "qr_batched_plan")
        self.count, self.dtype = count, dtype
        self.m = torch.tensor(ms, dtype=torch.int32, device=dev)
        self.n = torch.tensor(ns, dtype=torch.int32, device=dev)
        self.lda = torch.tensor([a.stride(1) if a.shape[1] > 1 else a.shape[0] for a in mats], dtype=torch.int32,
                                device=dev)
        self.ptrs = torch.tensor([a.data_ptr() for a in mats], dtype=torch.int64, device=dev)
        self.nb = torch.tensor(list(nb), dtype=torch.int32, device=dev)
        self.ib = torch.tensor(list(ib), dtype=torch.int32, device=dev)
        self.order = torch.tensor(list(order), dtype=torch.int32, device=dev)
        self.toff = torch.tensor(list(toff), dtype=torch.int64, device=dev)
        self.T = torch.zeros(ttot.value, dtype=dtype, device=dev)
        self.scratch = torch.zeros(256, dtype=torch.uint8, device=dev)
        self.h_nb, self.h_ib, self.h_toff = list(nb), list(ib), list(toff)

    def launch(self, stream=None):
        f = lib().qr_factor_batched_d if self.dtype == torch.float64 else lib().qr_factor_batched_s
        P = ctypes.c_void_p
        _lib.check(f(self.count, P(self.m.data_ptr()), P(self.n.data_ptr()), P(self.ptrs.data_ptr()),
                     P(self.lda.data_ptr()), P(self.T.data_ptr()), P(self.toff.data_ptr()), P(self.nb.data_ptr()),
                     P(self.ib.data_ptr()), P(self.order.data_ptr()), P(self.scratch.data_ptr()),
                     _stream_ptr(stream)), "qr_factor_batched")

    def status(self, stream=None):
        st = ctypes.c_int()
        _lib.check(lib().qr_batched_status(ctypes.c_void_p(self.scratch.data_ptr()), ctypes.byref(st),
                                           _stream_ptr(stream)), "qr_batched_status")
        return st.value

    def factorization(self, b, A):
        """Factorization view of matrix b (for qr_apply_qt / form_q)."""
        m, n = A.shape
        nbe = min(self.h_nb[b], m)
        T = self.T[self.h_toff[b]:]
        return Factorization(A, T, None, nbe, self.h_ib[b])


def qr_batched_set_class(dtype, m_hi, nb, ib):
    _lib.check(lib().qr_batched_set_class(_prec(dtype), m_hi, nb, ib), "qr_batched_set_class")


def qr_batched_clear_classes(dtype):
    _lib.check(lib().qr_batched_clear_classes(_prec(dtype)), "qr_batched_clear_classes")


def qr_status(scratch, stream=None):
    st = ctypes.c_int()
    _lib.check(lib().qr_status(ctypes.c_void_p(scratch.data_ptr()), ctypes.byref(st), _stream_ptr(stream)),
               "qr_status")
    return st.value


def qr_set_option(opt, value):
    _lib.check(lib().qr_set_option(opt, int(value)), "qr_set_option")


def qr_set_task_costs(dtype, nb, ib, costs=None):
    """Measured (GEQRT, UNMQR, TSQRT, TSMQR) costs for the list schedule of
    factorizations with this (nb, ib); None removes them."""
    c = None if costs is None else (ctypes.c_double * 4)(*[float(v) for v in costs])
    _lib.check(lib().qr_set_task_costs(_prec(dtype), nb, ib, c), "qr_set_task_costs")


def qr_set_trace(buf=None):
    """Per-task trace of the persistent kernels into ``buf`` (a CUDA int64
    tensor of shape (capacity, 4), see read_trace); None turns it off."""
    if buf is None:
        _lib.check(lib().qr_set_trace(None, 0), "qr_set_trace")
    else:
        if buf.dtype != torch.int64 or buf.dim() != 2 or buf.shape[1] != 4 or not buf.is_contiguous():
            raise ValueError("trace buffer must be a contiguous int64 tensor of shape (capacity, 4)")
        _lib.check(lib().qr_set_trace(ctypes.c_void_p(buf.data_ptr()), buf.shape[0]), "qr_set_trace")


def read_trace(buf, ntasks):
    """Records 0..ntasks-1 of a trace buffer as NumPy arrays: task, type,
    sm, t_take, t_ready, t_done (ns, relative to the earliest t_take)."""
    r = buf[:ntasks].cpu().numpy().view("uint64")
    task = (r[:, 0] & ((1 << 40) - 1)).astype("int64")
    typ = ((r[:, 0] >> 40) & 0xFF).astype("int64")
    sm = (r[:, 0] >> 48).astype("int64")
    t0 = r[:, 1].min()
    return (task, typ, sm, (r[:, 1] - t0).astype("int64"), (r[:, 2] - t0).astype("int64"),
            (r[:, 3] - t0).astype("int64"))


def qr_get_option(opt):
    return lib().qr_get_option(opt)


def qr_last_kernel_ms():
    ms = ctypes.c_float()
    _lib.check(lib().qr_last_kernel_ms(ctypes.byref(ms)), "qr_last_kernel_ms")
    return ms.value


def qr_peak_fp64(stream=None):
    g = ctypes.c_double()
    _lib.check(lib().qr_peak_fp64(ctypes.byref(g), _stream_ptr(stream)), "qr_peak_fp64")
    return g.value


def qr_task_count(m, n, nb, ib, dtype=torch.float64):
    return lib().qr_task_count(m, n, nb, ib, _prec(dtype))


def qr_lookup(m, n, dtype=torch.float64):
    """(nb, ib) from the loaded tuning table (built-in default otherwise)."""
    nb, ib = ctypes.c_int(), ctypes.c_int()
    _lib.check(lib().qr_lookup(m, n, _prec(dtype), ctypes.byref(nb), ctypes.byref(ib)), "qr_lookup")
    return nb.value, ib.value


def qr_lookup_sms(m, n, dtype=torch.float64, sms=0):
    """(nb, ib, p) tuned for m x n on an SM budget of ``sms`` SMs (0 = the
    whole GPU): the closest tuned budget, then the closest tuned shape."""
    nb, ib, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(lib().qr_lookup_sms(m, n, _prec(dtype), int(sms), ctypes.byref(nb), ctypes.byref(ib),
                                   ctypes.byref(p)), "qr_lookup_sms")
    return nb.value, ib.value, p.value


def qr_lookup_p(m, n, dtype=torch.float64):
    """(nb, ib, p) from the loaded tuning table (built-in default otherwise)."""
    nb, ib, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(lib().qr_lookup_p(m, n, _prec(dtype), ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p)),
               "qr_lookup_p")
    return nb.value, ib.value, p.value


def qr_flops(m, n):
    """Credited flops 2mn^2 - 2n^3/3 (= 4/3 N^3 when m = n, Sec. 2.2)."""
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


class CholFactorization:
    """Result of chol_factor: A with L in its lower triangle, the scratch
    buffer (which holds the device status) and the tile order used."""

    def __init__(self, A, scratch, nb):
        self.A, self.scratch, self.nb = A, scratch, nb

    def L(self):
        return torch.tril(self.A)

    def status(self, stream=None):
        """(QR_DEV_* bits, first column whose pivot was not positive or -1)."""
        st, col = ctypes.c_int(), ctypes.c_int64()
        _lib.check(lib().chol_status(ctypes.c_void_p(self.scratch.data_ptr()), ctypes.byref(st), ctypes.byref(col),
                                     _stream_ptr(stream)), "chol_status")
        return st.value, col.value


def chol_factor(A, nb=0, scratch=None, stream=None):
    """Tile Cholesky of the SPD matrix A (float64, column-major CUDA tensor;
    its lower triangle is read and overwritten with L). nb = 0 uses the
    Cholesky tuning table."""
    n = A.shape[0]
    if A.dtype != torch.float64 or not A.is_cuda or A.stride(0) != 1 or A.shape[1] != n:
        raise ValueError("A must be a square column-major float64 CUDA tensor")
    if nb == 0:
        nbv = ctypes.c_int()
        _lib.check(lib().chol_lookup(n, ctypes.byref(nbv)), "chol_lookup")
        nb = nbv.value
    b = ctypes.c_int64()
    _lib.check(lib().chol_workspace(n, nb, ctypes.byref(b)), "chol_workspace")
    if scratch is None or scratch.numel() < b.value:
        scratch = torch.empty(b.value, dtype=torch.uint8, device=A.device)
    lda = A.stride(1) if n > 1 else max(n, 1)
    _lib.check(lib().chol_factor_d(n, ctypes.c_void_p(A.data_ptr()), lda, nb, ctypes.c_void_p(scratch.data_ptr()),
                                   b.value, _stream_ptr(stream)), "chol_factor_d")
    return CholFactorization(A, scratch, nb)


class LUFactorization:
    """Result of lu_factor: A with U on and above its diagonal and the
    multipliers below, the pivot records (int32, tile (i, k) at
    piv[(k * NT + i) * nb + c]) and the scratch buffer (device status)."""

    def __init__(self, A, piv, scratch, nb):
        self.A, self.piv, self.scratch, self.nb = A, piv, scratch, nb

    def status(self, stream=None):
        """(QR_DEV_* bits, first column whose pivot was zero or -1)."""
        st, col = ctypes.c_int(), ctypes.c_int64()
        _lib.check(lib().lu_status(ctypes.c_void_p(self.scratch.data_ptr()), ctypes.byref(st), ctypes.byref(col),
                                   _stream_ptr(stream)), "lu_status")
        return st.value, col.value


def lu_workspace(n, nb=0):
    """(pivot-record elements, scratch bytes) for lu_factor."""
    pe, sb = ctypes.c_int64(), ctypes.c_int64()
    _lib.check(lib().lu_workspace(n, nb, ctypes.byref(pe), ctypes.byref(sb)), "lu_workspace")
    return pe.value, sb.value


def lu_factor(A, nb=0, piv=None, scratch=None, stream=None):
    """Tile LU with incremental pivoting of the square float64 column-major
    CUDA tensor A, in place. nb in [8, 64]; 0 takes the LU tuning table's
    (64 without one)."""
    n = A.shape[0]
    if A.dtype != torch.float64 or not A.is_cuda or A.stride(0) != 1 or A.shape[1] != n:
        raise ValueError("A must be a square column-major float64 CUDA tensor")
    if nb == 0:
        nbv = ctypes.c_int()
        _lib.check(lib().lu_lookup(n, ctypes.byref(nbv)), "lu_lookup")
        nb = nbv.value
    pe, sb = lu_workspace(n, nb)
    if piv is None or piv.numel() < pe:
        piv = torch.full((max(pe, 1),), -1, dtype=torch.int32, device=A.device)
    if scratch is None or scratch.numel() < sb:
        scratch = torch.empty(sb, dtype=torch.uint8, device=A.device)
    lda = A.stride(1) if n > 1 else max(n, 1)
    _lib.check(lib().lu_factor_d(n, ctypes.c_void_p(A.data_ptr()), lda, nb, ctypes.c_void_p(piv.data_ptr()),
                                 ctypes.c_void_p(scratch.data_ptr()), sb, _stream_ptr(stream)), "lu_factor_d")
    return LUFactorization(A, piv, scratch, nb)


def lu_tune(ns, heuristic=2, reps=6, table="", log="", stream=None):
    """The LU NB tuner (lu_tune); returns its wall-time figures."""
    L = lib()
    b = ctypes.c_int64()
    _lib.check(L.lu_tune_workspace(max(ns), ctypes.byref(b)), "lu_tune_workspace")
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    arr = (ctypes.c_int64 * len(ns))(*ns)
    secs = (ctypes.c_double * 4)()
    _lib.check(L.lu_tune(arr, len(ns), heuristic, reps, table.encode(), log.encode(), ctypes.c_void_p(work.data_ptr()),
                         b.value, secs, _stream_ptr(stream)), "lu_tune")
    return {"seconds": secs[0], "step1_seconds": secs[1], "step2_seconds": secs[2], "factorizations_timed": int(secs[3]),
            "heuristic": heuristic, "reps": reps, "ns": list(ns), "table": table, "log": log}


def chol_tune(ns, heuristic=2, reps=6, table="", log="", stream=None):
    """The Cholesky NB tuner (chol_tune); returns its wall-time figures."""
    L = lib()
    b = ctypes.c_int64()
    _lib.check(L.chol_tune_workspace(max(ns), ctypes.byref(b)), "chol_tune_workspace")
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    arr = (ctypes.c_int64 * len(ns))(*ns)
    secs = (ctypes.c_double * 4)()
    _lib.check(L.chol_tune(arr, len(ns), heuristic, reps, table.encode(), log.encode(), ctypes.c_void_p(work.data_ptr()),
                           b.value, secs, _stream_ptr(stream)), "chol_tune")
    return {"seconds": secs[0], "step1_seconds": secs[1], "step2_seconds": secs[2], "factorizations_timed": int(secs[3]),
            "heuristic": heuristic, "reps": reps, "ns": list(ns), "table": table, "log": log}
