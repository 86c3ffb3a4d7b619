"""Pins of the oracle's GF(4) shadow replay (``oracle.gf4.shadow``), applied by the GF(4) GPU
tests to every shot whose outcome differs from the oracle's: a plain binary32 GF(4) decoder
written for this test (``tests/fp32_gf4_decoder.py``) stays within the replay's rounding bound
in every mode, on the paper's CSS matrix and on random Pauli matrices with Y entries, and the
same decoder with one planted mistake breaks it."""
import numpy as np
import pytest

import oracle
from oracle import gf4 as O4
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.inputs import gf4 as I4

from tests import fp32_gf4_decoder as D

MODES = {"sagms": dict(mode=oracle.SAGMS), "sms": dict(mode=oracle.SMS, alpha=0.6), "bp": dict(mode=oracle.BP)}


def _ratio(dev, bnd):
    a = np.abs(dev)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(a == 0.0, 0.0, a / bnd)
    return float(np.nanmax(r)) if r.size else 0.0


def _random_pauli(m, n, seed):
    rng = np.random.default_rng(seed)
    rows = [sorted(rng.choice(n, size=int(rng.integers(2, 6)), replace=False).tolist()) for _ in range(m)]
    return I4.Gf4Code(m=m, n=n, row_ptr=np.cumsum([0] + [len(r) for r in rows]).astype(np.int32),
                      col_idx=np.array([c for r in rows for c in r], dtype=np.int32),
                      pauli=rng.integers(1, 4, size=sum(len(r) for r in rows)).astype(np.uint8))


def _syndromes(g, eps, shots, seed):
    rng = np.random.default_rng(seed)
    kind = np.where(rng.random((shots, g.n)) < eps, rng.integers(1, 4, size=(shots, g.n)), 0)
    s = np.zeros((shots, g.m), dtype=np.uint8)
    for i in range(g.m):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            c, t = g.col_idx[e], int(g.pauli[e])
            s[:, i] ^= (((kind[:, c] & 1) & (t >> 1)) ^ ((kind[:, c] >> 1) & (t & 1))).astype(np.uint8)
    return I.pack_bits(s)


@pytest.mark.parametrize("name", ["sagms", "sms", "bp"])
def test_binary32_gf4_decoder_stays_within_the_bound(name):
    kw = MODES[name]
    worst, rounds_seen = 0.0, 0
    for g, syn, eps in [(I4.css_code(I.gb_code(63, 3)), I4.depolarizing(I4.css_code(I.gb_code(63, 3)), 0.05, 6, 11)[2],
                         0.05),
                        (_random_pauli(30, 36, 4), _syndromes(_random_pauli(30, 36, 4), 0.06, 6, 12), 0.06)]:
        L0 = np.array([np.float32(I4.prior(eps))], dtype=np.float64)   # the binary32 prior both sides use
        for s in range(len(syn)):
            G, rounds = D.decode(g, syn[s], L0, max_iter=15, **kw)
            dev, bnd, _ = O4.shadow(g, syn[s], L0, G, rounds, **kw)
            worst = max(worst, _ratio(dev, bnd))
            rounds_seen += rounds
    assert rounds_seen > 20
    assert worst <= 1.0, f"{name}: binary32 GF(4) decoder at {worst:.3g} of the bound"


@pytest.mark.parametrize("mutant", D.MUTANTS)
def test_planted_gf4_mistake_breaks_the_bound(mutant):
    g = _random_pauli(30, 36, 7)
    syn = _syndromes(g, 0.06, 8, 13)
    L0 = np.array([np.float32(I4.prior(0.06))], dtype=np.float64)
    worst = 0.0
    for s in range(len(syn)):
        G, rounds = D.decode(g, syn[s], L0, max_iter=10, mutant=mutant, mode=oracle.SAGMS)
        if rounds == 0:
            continue
        dev, bnd, _ = O4.shadow(g, syn[s], L0, G, rounds, mode=oracle.SAGMS)
        worst = max(worst, _ratio(dev, bnd))
    assert worst > 10.0, f"{mutant}: planted mistake stays within the bound ({worst:.3g})"
