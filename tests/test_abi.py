"""The C ABI: library loads, exports every declared symbol, validates on the host.  CPU only.

These run no decode (no GPU here): they cover the boundary's host-side checks, which
run before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2605_10433_gb300 import build
    build.build()
    from paper_2605_10433_gb300 import _native
    return _native


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sagms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sagms_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    names = declared_functions()
    assert "sagms_decode" in names and "sagms_load_code" in names
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_alpha_star(native):
    import oracle
    assert "sm_103a" in native.sagms_version()
    for L0, dc in ((3.2958, 10), (5.0, 16), (2.0, 4)):
        assert abs(native.sagms_alpha_star(L0, dc) - oracle.alpha_star(L0, dc)) < 1e-12
    assert np.isnan(native.sagms_alpha_star(-1.0, 4))


@pytest.mark.parametrize("kw,ok", [
    (dict(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=1.1, max_iter=100), True),
    (dict(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=0.0, max_iter=100), True),   # default eta
    (dict(mode=2, alpha_min=0.3, alpha_max=0.95, eta_unsat=1.1, max_iter=100), False),  # a_max eta > 1
    (dict(mode=2, alpha_min=0.6, alpha_max=0.5, eta_unsat=1.1, max_iter=100), False),   # a_min > a_max
    (dict(mode=2, alpha_min=0.0, alpha_max=0.5, eta_unsat=1.1, max_iter=100), False),
    (dict(mode=2, alpha_min=2.0 ** -20, alpha_max=0.5, eta_unsat=1.1, max_iter=100), True),
    (dict(mode=2, alpha_min=2.0 ** -21, alpha_max=0.5, eta_unsat=1.1, max_iter=100), False),  # gain may round to 0
    (dict(mode=2, alpha_min=1e-7, max_iter=100, flags=16), False),                            # same, auto ceiling
    (dict(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=0.9, max_iter=100), False),   # eta < 1
    (dict(mode=1, alpha=0.75, max_iter=100), True),
    (dict(mode=1, alpha=0.0, max_iter=100), False),
    (dict(mode=1, alpha=1.5, max_iter=100), False),
    (dict(mode=0, max_iter=-1), False),
    (dict(mode=7, max_iter=10), False),
    (dict(mode=3, max_iter=10, flags=16), False),
    (dict(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=1.1, max_iter=100, flags=32), True),   # layered
    (dict(mode=0, max_iter=100, flags=32 | 1 | 2), True),
    (dict(mode=3, max_iter=10, flags=32), False),      # layered: MS family only
    (dict(mode=0, max_iter=10, flags=64), False),      # unknown flag
])
def test_param_validation(native, kw, ok):
    p = native.sagms_params(**kw)
    rc = native.sagms_check_params(p)
    assert (rc == 0) == ok, (kw, rc, native.sagms_last_error_string())
    if not ok:
        assert rc in (-1, -4) and native.sagms_last_error_string()


@pytest.mark.parametrize("rows,n,err", [
    ([[0, 1], [1, 1]], 2, -2),          # duplicate column
    ([[0, 5]], 3, -2),                  # column out of range
    ([list(range(33))], 33, -3),        # check degree > 32
])
def test_csr_validation(native, rows, n, err):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array([c for r in rows for c in r], dtype=np.int32)
    with pytest.raises(native.SagmsError) as ei:
        native.sagms_load_code(len(rows), n, rp, ci)
    assert ei.value.code == err


def test_csr_non_monotone_and_bad_sizes(native):
    with pytest.raises(native.SagmsError) as ei:
        native.sagms_load_code(2, 4, np.array([0, 3, 2], dtype=np.int32), np.array([0, 1, 2], dtype=np.int32))
    assert ei.value.code == -2
    with pytest.raises(native.SagmsError) as ei:
        native.sagms_load_code(0, 4, np.array([0], dtype=np.int32), np.array([], dtype=np.int32))
    assert ei.value.code == -1
    with pytest.raises(native.SagmsError) as ei:
        native.sagms_load_code(1025, 4, np.zeros(1026, dtype=np.int32), np.array([], dtype=np.int32))
    assert ei.value.code == -9
    # qubit degree 17 > 16
    rows = [[0] for _ in range(17)]
    rp = np.arange(18, dtype=np.int32)
    with pytest.raises(native.SagmsError) as ei:
        native.sagms_load_code(17, 1, rp, np.zeros(17, dtype=np.int32))
    assert ei.value.code == -3


def test_null_arguments_are_rejected(native):
    lib = native.lib()
    assert lib.sagms_decode(None, None, 0, None, None, None, None, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.sagms_load_code(1, 1, 0, None, None, ctypes.byref(h)) == -1
    p = native.sagms_params(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=1.1, max_iter=10)
    assert lib.sagms_decode_host(None, ctypes.byref(p), 10, None, None, None, None, None) == -1


def test_device_buffer_checks_come_before_any_launch(native):
    """sagms_decode refuses NULL or misaligned device buffers before it touches the code
    handle or CUDA (the pointers below are never dereferenced)."""
    lib = native.lib()
    p = native.sagms_params(mode=2, alpha_min=0.3, alpha_max=0.5, eta_unsat=1.1, max_iter=10)
    A, M = 0x10000, 0x10002            # a 4-byte aligned and a misaligned address
    ok = [A, A, A, A, A]
    assert lib.sagms_decode(None, ctypes.byref(p), 10, None, A, A, A, A, None) == -1
    assert "NULL device buffer" in native.sagms_last_error_string()
    for k in (0, 1, 2, 4):             # d_syn, d_L0, d_err, d_iters (d_conv holds bytes)
        args = list(ok)
        args[k] = M
        assert lib.sagms_decode(None, ctypes.byref(p), 10, *args, None) == -1
        assert "4-byte aligned" in native.sagms_last_error_string()
    args = list(ok)
    args[3] = A + 1                    # a byte buffer may start anywhere
    assert lib.sagms_decode(None, ctypes.byref(p), 10, *args, None) == -1
    assert "code is NULL" in native.sagms_last_error_string()


def test_monte_carlo_buffer_checks_come_before_any_launch(native):
    """The sampler's optional outputs and the logical check's buffers are checked for NULL and
    alignment before the code handle or CUDA is touched."""
    lib = native.lib()
    A, M = 0x10000, 0x10002
    assert lib.sagms_mc_sample(None, 1, 0.1, 4.0, 0, 10, M, None, None, None) == -1
    assert "aligned" in native.sagms_last_error_string()
    assert lib.sagms_mc_sample(None, 1, 0.1, 4.0, 0, 10, None, None, None, None) == -1
    assert "code is NULL" in native.sagms_last_error_string()   # all three outputs may be NULL
    assert lib.sagms_mc_check(None, 10, A, A, A, A, None, None, None) == -1
    assert "NULL device buffer" in native.sagms_last_error_string()
    assert lib.sagms_mc_check(None, 10, A, A, A, A, None, A + 4, None) == -1   # counters are 8-byte
    assert "misaligned" in native.sagms_last_error_string()
    assert lib.sagms_mc_check(None, 10, A, A, A + 1, A, None, A, None) == -1   # conv holds bytes
    assert "code is NULL" in native.sagms_last_error_string()


def test_oracle_source_shares_nothing_with_the_cuda_path():
    """The FP64 checker and the CUDA library include none of each other's files."""
    cu = open(os.path.join(ROOT, "paper_2605_10433_gb300", "csrc", "sagms.cu")).read()
    kern = open(os.path.join(ROOT, "paper_2605_10433_gb300", "csrc", "decode_kernel.cuh")).read()
    orc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "oracle" not in cu + kern
    assert "sagms.h" not in orc and "decode_kernel" not in orc
    for f in os.listdir(os.path.join(ROOT, "paper_2605_10433_gb300")):
        if f.endswith(".py"):
            s = open(os.path.join(ROOT, "paper_2605_10433_gb300", f)).read()
            assert "import oracle" not in s and "from oracle" not in s, f


def test_op_count_model_matches_eq15_and_table1():
    import json
    from paper_2605_10433_gb300 import roofline
    from paper_2605_10433_gb300 import inputs as I
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_printed_values.json")))["cn_op_counts_dc10"]
    assert roofline.CN_OPS["bp"](g["dc"]) == g["BP4"]
    assert roofline.CN_OPS["sms"](g["dc"]) == g["SMS"]
    assert roofline.CN_OPS["sagms"](g["dc"]) == g["SAGMS"]
    c = I.gb_code(1023, 5)
    # m (2 d_c + 3) + n (2 d_v + 1) + E + m at d_c = 10, d_v = 5
    assert roofline.ops_per_iteration("sagms", c.row_ptr, c.col_idx, c.n) == 1023 * 23 + 2046 * 11 + 10230 + 1023
    assert roofline.hbm_bytes_per_shot(c.m, c.n) == 128 + 4 + 256 + 1 + 4   # 393 B
    # on-chip bytes: r = 1 moves 12E + 4n (no old-message read), each further round 16E + 4n,
    # a shot that stops at its first check moves nothing
    E, n = c.nnz, c.n
    assert roofline.smem_bytes([0], E, n) == 0
    assert roofline.smem_bytes([1], E, n) == 12 * E + 4 * n
    assert roofline.smem_bytes([1, 3, 0], E, n) == (12 * E + 4 * n) + (12 * E + 4 * n + 2 * (16 * E + 4 * n))
    assert roofline.smem_peak_bytes(152, 2070) == 152 * 128 * 2070e6


def test_gf4_op_count_model():
    """The GF(4) iteration count on the CSS stack of GB(63, 5): m = n = 126, every row and every
    qubit of degree 10 (five X-type and five Z-type rows per qubit), E = 1260.  Per check the
    Eq. 15 rule; per qubit 2 d_v Pauli-total additions, d_v extrinsic subtractions, 3 decision
    comparisons and three commute LLRs of four transcendentals (weight 10) and four simple
    operations each; one anticommutation test per edge and one popcount step per check."""
    from paper_2605_10433_gb300 import roofline
    from paper_2605_10433_gb300 import inputs as I
    from paper_2605_10433_gb300.inputs import gf4 as I4
    g = I4.css_code(I.gb_code(63, 5))
    assert (g.m, g.n, g.nnz) == (126, 126, 1260)
    vn = 126 * (2 * 10 + 10 + 3 + 3 * (4 * 10 + 4))
    assert roofline.gf4_ops_per_iteration("sagms", g.row_ptr, g.col_idx, g.n) == 126 * 23 + vn + 1260 + 126
    assert roofline.gf4_ops_per_iteration("bp", g.row_ptr, g.col_idx, g.n) == 126 * 207 + vn + 1260 + 126
    assert roofline.gf4_ops_per_iteration("sms", g.row_ptr, g.col_idx, g.n) == 126 * 18 + vn + 1260 + 126


@pytest.mark.parametrize("rows,pauli,n,err", [
    ([[0, 1], [1, 2]], [1, 2, 3, 4], 3, "SAGMS_ERR_CSR"),        # Pauli code 4
    ([[0, 1], [1, 2]], [1, 0, 3, 1], 3, "SAGMS_ERR_CSR"),        # Pauli code 0 (identity entry)
    ([[0, 0], [1, 2]], [1, 1, 2, 2], 3, "SAGMS_ERR_CSR"),        # duplicate column
    ([[0, 5]], [1, 2], 3, "SAGMS_ERR_CSR"),                      # column out of range
    ([list(range(17))], [1] * 17, 20, "SAGMS_ERR_DEGREE"),       # check degree 17
])
def test_gf4_loader_refuses_bad_matrices_before_any_cuda_call(native, rows, pauli, n, err):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    ci = np.array([c for r in rows for c in r], dtype=np.int32)
    pa = np.array(pauli, dtype=np.uint8)
    out = ctypes.c_void_p()
    rc = native.lib().sagms_gf4_load_code(len(rows), n, int(rp[-1]), rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          pa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(out))
    code = {v: k for k, v in native.ERRORS.items()}[err.replace("SAGMS_", "")]
    assert rc == code and not out.value, native.sagms_last_error_string()


def test_gf4_decode_refuses_before_any_launch(native):
    p = native.sagms_params(2, 0.75, 0.3, 0.5, 1.1, 10, 0)
    lib = native.lib()
    err_arg = -1
    assert lib.sagms_gf4_decode(None, ctypes.byref(p), 10, 16, 16, 16, 16, 16, None) == err_arg
    assert lib.sagms_gf4_layout(None) == err_arg
    assert lib.sagms_gf4_load_code(600, 10, 0, None, None, None, None) == err_arg   # out is NULL
    out = ctypes.c_void_p()
    rp = np.zeros(601, dtype=np.int32)
    rc = lib.sagms_gf4_load_code(600, 10, 0, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, None,
                                 ctypes.byref(out))
    assert rc == err_arg and "512" in native.sagms_last_error_string()
