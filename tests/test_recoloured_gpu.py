"""Codes whose CSR order does not suit the column-indexed layout (rows with sorted columns,
random LDPC codes, permuted rows): the library assigns slots by edge colouring at load time
and every kernel uses that edge order, so the column-indexed kernel runs them and stays bit
for bit identical to the one-shot-per-CTA, two-slot and two-group kernels; the FP64 oracle
(which reads the CSR as given) checks the decoded results."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G
from tests.test_column_slots import _random_code, _sorted_rows
from tests.test_group_kernel_gpu import (KERNEL_GENERIC, KERNEL_GROUPS, KERNEL_QC, KERNEL_SLOTS, PARAMS, _decode_with_kernel,
                                         _same, _with)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sorted_gb(l, w):
    g = I.gb_code(l, w)
    return I.Code(m=g.m, n=g.n, row_ptr=g.row_ptr, col_idx=_sorted_rows(g.row_ptr, g.col_idx),
                  name=f"GB({l},{w}) sorted rows")


def _random(m, n, dv, dc, seed):
    rp, ci = _random_code(m, n, dv, dc, seed)
    return I.Code(m=m, n=n, row_ptr=rp, col_idx=ci, name=f"random ({dv},{dc}) m={m} seed={seed}")


CODES = {
    "gb1023-sorted": lambda: _sorted_gb(1023, 5),
    "gb255x4-sorted": lambda: _sorted_gb(255, 4),
    "random-1024x2048-(5,10)": lambda: _random(1024, 2048, 5, 10, 11),
    "random-512x1024-(4,8)": lambda: _random(512, 1024, 4, 8, 12),
    "random-128x256-(3,6)": lambda: _random(128, 256, 3, 6, 13),
    "random-700x1400-(3,6)": lambda: _random(700, 1400, 3, 6, 14),
}


@pytest.mark.parametrize("key", list(CODES))
def test_recoloured_code_runs_on_the_column_indexed_kernel(key):
    c = CODES[key]()
    dc = S.DeviceCode.from_code(c)
    assert "two-group-qc" in dc.kernels
    _, syn, L0, _ = I.workload(c, [0.01, 0.03, 0.06], 2001, seed=5)
    syn = syn.copy()
    syn[::17] = 0
    for mode in ("ms", "sms", "sagms"):
        p = PARAMS[mode]
        ref = _decode_with_kernel(c, KERNEL_GENERIC, syn, L0, p)
        for kernel in (KERNEL_SLOTS, KERNEL_GROUPS, KERNEL_QC):
            assert _same(_decode_with_kernel(c, kernel, syn, L0, p), ref), (mode, kernel)
    tr = _decode_with_kernel(c, KERNEL_GENERIC, syn[:12], L0[:12], PARAMS["sagms"], trace=True)["trace"]
    tq = _decode_with_kernel(c, KERNEL_QC, syn[:12], L0[:12], PARAMS["sagms"], trace=True)["trace"]
    assert np.array_equal(np.nan_to_num(tr, nan=7.0), np.nan_to_num(tq, nan=7.0))


@pytest.mark.parametrize("key", ["gb1023-sorted", "random-1024x2048-(5,10)", "random-128x256-(3,6)"])
def test_recoloured_code_oracle_parity(key):
    c = CODES[key]()
    dc = S.DeviceCode.from_code(c)
    S._native.sagms_set_plan(dc.handle, KERNEL_QC)
    _, syn, L0, _ = I.workload(c, [0.01, 0.03], 300, seed=6)
    G.compare(c, dc, syn, L0, PARAMS["sagms"])


def test_recoloured_code_per_qubit_priors():
    c = CODES["random-512x1024-(4,8)"]()
    rng = np.random.default_rng(21)
    _, syn = I.sample(c, 0.03, 801, seed=22)
    L0q = I.llr_prior(rng.uniform(0.005, 0.08, size=c.n)).astype(np.float32)
    L0q[rng.choice(c.n, size=c.n // 50, replace=False)] *= -1.0
    p = _with(PARAMS["sagms"], flags=S.FLAG_L0_PER_QUBIT)
    assert _same(_decode_with_kernel(c, KERNEL_QC, syn, L0q, p), _decode_with_kernel(c, KERNEL_GENERIC, syn, L0q, p))
    dc = S.DeviceCode.from_code(c)
    S._native.sagms_set_plan(dc.handle, KERNEL_QC)
    G.compare(c, dc, syn[:200], L0q, p)


def test_sorted_and_term_ordered_rows_decode_alike():
    """The same GB(1023, 5) matrix with two column orders: both run the column-indexed kernel,
    their edge orders differ only by a permutation of slots inside each half, so results agree
    on nearly every shot (a qubit's message sum may round differently)."""
    g = I.gb_code(1023, 5)
    a = S.DeviceCode.from_code(g)
    b = S.DeviceCode.from_code(_sorted_gb(1023, 5))
    _, syn, L0, _ = I.workload(g, [0.01, 0.03], 4000, seed=9)
    ra, rb = G.gpu_decode(a, syn, L0, PARAMS["sagms"]), G.gpu_decode(b, syn, L0, PARAMS["sagms"])
    same = (ra["err"] == rb["err"]).all(axis=1) & (ra["iters"] == rb["iters"])
    assert same.mean() > 0.995
    # each order on its own against the oracle, under the full acceptance
    sb = _sorted_gb(1023, 5)
    G.compare(g, a, syn, L0, PARAMS["sagms"], gpu=ra)
    G.compare(sb, b, syn, L0, PARAMS["sagms"], gpu=rb)
