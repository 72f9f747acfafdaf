"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pins of test_oracle.py and test_oracle_checkers.py catch each one:
in the factorization a dropped term, a wrong sign convention, a wrong index
and a wrong tau formula; in the accuracy checks a dropped factor 2 on the
off-diagonal terms of I - Q^T Q, a loop that skips the diagonal (of R, or of
Q^T Q), a missing square root and a wrong normalisation; in the Cholesky
factorization a dropped term, a wrong divisor and a transposed operand, and
in its residual a skipped diagonal term."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle as pins
from tests import test_oracle_checkers as cpins
from tests import test_chol_oracle as chpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "qr_oracle.c")

MUTANTS = {
    "dropped_pivot_term": ("      double w = a[0];\n      for (int64_t r = 0; r < len; ++r) w += v[r] * a[r + 1];\n      w *= t;\n      a[0] -= w;\n      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];\n    }\n  }\n  return 0;\n}\n\n/* C <- Q^T C",
                           "      double w = 0.0;\n      for (int64_t r = 0; r < len; ++r) w += v[r] * a[r + 1];\n      w *= t;\n      a[0] -= w;\n      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];\n    }\n  }\n  return 0;\n}\n\n/* C <- Q^T C"),
    "flipped_beta_sign": ("double beta = (a < 0.0) ? norm : -norm;", "double beta = (a < 0.0) ? -norm : norm;"),
    "shifted_row_index": ("      a[0] -= w;\n      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];\n    }\n  }\n  return 0;\n}\n\n/* C <- Q^T C",
                          "      a[0] -= w;\n      for (int64_t r = 0; r < len; ++r) a[r] -= w * v[r];\n    }\n  }\n  return 0;\n}\n\n/* C <- Q^T C"),
    "wrong_tau": ("double tau = (beta - a) / beta;", "double tau = (beta - a) / a;"),
    "fact_skips_diagonal": ("for (int64_t p = 0; p <= c; ++p) s -=", "for (int64_t p = 0; p < c; ++p) s -="),
    "fact_unsquared_norm": ("return (double)(sqrtl(num) / sqrtl(den));\n}\n\n/* ||I - Q^T Q||_F",
                            "return (double)(sqrtl(num) / den);\n}\n\n/* ||I - Q^T Q||_F"),
    "orth_dropped_offdiag_2x": ("acc += (i == j) ? s * s : 2.0L * s * s;", "acc += s * s;"),
    "orth_skips_diagonal": ("for (int64_t i = 0; i <= j; ++i) {\n      long double s = (i == j)",
                            "for (int64_t i = 0; i < j; ++i) {\n      long double s = (i == j)"),
    "orth_missing_sqrt": ("return (double)sqrtl(acc);", "return (double)acc;"),
    "potrf_drops_last_term": ("for (int64_t k = 0; k < j; ++k) d -=", "for (int64_t k = 0; k + 1 < j; ++k) d -="),
    "potrf_wrong_divisor": ("A[IDX(i, j, lda)] = s / ljj;", "A[IDX(i, j, lda)] = s / d;"),
    "potrf_transposed_operand": ("s -= A[IDX(i, k, lda)] * A[IDX(j, k, lda)];", "s -= A[IDX(k, i, lda)] * A[IDX(j, k, lda)];"),
    "chol_residual_skips_diagonal_term": ("for (int64_t k = 0; k <= kmax; ++k) s -=", "for (int64_t k = 0; k < kmax; ++k) s -="),
}

PIN_TESTS = [
    lambda: pins.test_closed_form_2x2(),
    lambda: pins.test_constructed_q0_r0(0),
    lambda: pins.test_rtr_equals_ata(),
    lambda: pins.test_against_long_double_mgs(8, 5),
    lambda: pins.test_backward_and_orthogonality(128, 128),
    lambda: cpins.test_fact_residual_exact_rational(7, 4, 1),
    lambda: cpins.test_fact_residual_single_entry(6, 6, 0),
    lambda: cpins.test_orth_residual_exact_rational(6, 3, 1),
    lambda: cpins.test_orth_residual_perturbed(6, 6, 0),
    lambda: cpins.test_orth_residual_scaled_columns(),
    lambda: chpins.test_closed_form_3x3(),
    lambda: chpins.test_exact_recovery(9, 1),
    lambda: chpins.test_against_lapack(40),
    lambda: chpins.test_residual_exact_rational(),
    lambda: chpins.test_single_entry_perturbation(),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    tmp = tempfile.mkdtemp()
    try:
        c = os.path.join(tmp, "m.c")
        so = os.path.join(tmp, "libm.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, c, "-lm"])
        saved = oracle._lib
        oracle._lib = None
        oracle.lib()  # sets argtypes on the real library
        real = oracle._lib
        mut = ctypes.CDLL(so)
        # copy signatures onto the mutant
        for sym in ["oracle_geqr2", "oracle_apply_qt", "oracle_apply_q", "oracle_form_q", "oracle_trsm_upper",
                    "oracle_mgs_ld", "oracle_fact_residual", "oracle_orth_residual", "oracle_ls_solve",
                    "oracle_ls_refine", "oracle_set_threads", "oracle_potrf", "oracle_chol_residual"]:
            getattr(mut, sym).argtypes = getattr(real, sym).argtypes
            getattr(mut, sym).restype = getattr(real, sym).restype
        oracle._lib = mut
        caught = 0
        try:
            for t in PIN_TESTS:
                try:
                    t()
                except AssertionError:
                    caught += 1
        finally:
            oracle._lib = saved
        assert caught >= 1, "no pin caught mutant " + name
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
