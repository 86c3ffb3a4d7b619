"""Pins of the oracle's shadow replay (``oracle.shadow``), the acceptance check the GPU
parity tests apply to every shot whose outcome differs from the FP64 oracle's.

The replay takes an implementation's binary32 posterior trace, re-evaluates each round of
Algorithm 1 in FP64 from that implementation's own previous posteriors, and bounds how far
binary32 rounding can move the result.  Pinned here, on the CPU, against things other than
the replay itself:
* MS in L0-normalised units is integer-valued, so the FP64 oracle's own trace is exact in
  binary32 and must replay with zero deviation;
* a plain binary32 decoder (``tests/fp32_decoder.py``, written for this test) must stay
  within the bound in every mode, on loopy codes, over many rounds;
* that decoder with one planted mistake of Eqs. 1-8 must break the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2605_10433_gb300 import inputs as I

from tests import fp32_decoder as D

MODES = {
    "sagms": dict(mode=oracle.SAGMS),
    "sms": dict(mode=oracle.SMS, alpha=0.75),
    "sms08": dict(mode=oracle.SMS, alpha=0.8),
    "ms": dict(mode=oracle.MS),
    "bp": dict(mode=oracle.BP),
}


def _shots(code, p, k, seed):
    _, syn, L0, _ = I.workload(code, [p], k, seed=seed)
    return syn, L0


def _ratio(dev, bnd):
    """Largest |dev| / bound; an exact zero deviation passes under a zero bound."""
    a = np.abs(dev)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(a == 0.0, 0.0, a / bnd)
    return float(np.max(r)) if r.size else 0.0


def test_ms_oracle_trace_replays_exactly():
    code = I.gb_code(63, 3)
    syn, L0 = _shots(code, 0.06, 24, 91)
    o = oracle.decode_code(code, syn, L0.astype(np.float64), mode=oracle.MS, max_iter=30, trace=True)
    for s in range(len(syn)):
        rounds = int(o["iters"][s])
        G = o["trace"][s, :rounds + 1].astype(np.float32)
        assert np.array_equal(G.astype(np.float64), o["trace"][s, :rounds + 1])   # integer-valued
        dev, bnd, flips = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, mode=oracle.MS)
        assert np.all(dev == 0.0) and np.all(flips == 0)


@pytest.mark.parametrize("name", ["sagms", "sms", "sms08", "ms", "bp"])
def test_binary32_decoder_stays_within_the_bound(name):
    code = I.gb_code(63, 3)
    syn, L0 = _shots(code, 0.05, 16, 17 + len(name))
    kw = MODES[name]
    worst = 0.0
    rounds_seen = 0
    for s in range(len(syn)):
        G, rounds, conv = D.decode(code, syn[s], L0[s:s + 1], max_iter=40, **kw)
        dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, **kw)
        worst = max(worst, _ratio(dev, bnd))
        rounds_seen += rounds
    assert rounds_seen > 60          # loopy trajectories, many rounds
    assert worst <= 1.0, f"{name}: binary32 decoder at {worst:.3g} of the rounding bound"


def test_binary32_decoder_per_qubit_priors():
    code = I.gb_code(127, 4)
    syn, _ = _shots(code, 0.03, 6, 5)
    rng = np.random.default_rng(8)
    q = rng.uniform(0.01, 0.05, code.n)
    L0q = np.log((1 - q) / q).astype(np.float32)
    worst = 0.0
    for s in range(len(syn)):
        G, rounds, _ = D.decode(code, syn[s], L0q, mode=oracle.SAGMS, max_iter=30, flags=oracle.FLAG_L0_PER_QUBIT)
        dev, bnd, _ = oracle.shadow_code(code, syn[s], L0q, G, rounds, mode=oracle.SAGMS,
                                         flags=oracle.FLAG_L0_PER_QUBIT)
        worst = max(worst, _ratio(dev, bnd))
    assert worst <= 1.0


@pytest.mark.parametrize("mutant", [m for m in D.MUTANTS if m != "layer_stale"])
def test_planted_mistake_breaks_the_bound(mutant):
    code = I.gb_code(63, 3)
    syn, L0 = _shots(code, 0.05, 8, 33)
    mode = oracle.BP if mutant == "bp_half" else oracle.SAGMS
    worst = 0.0
    for s in range(len(syn)):
        G, rounds, _ = D.decode(code, syn[s], L0[s:s + 1], mode=mode, max_iter=20, mutant=mutant)
        if rounds == 0:
            continue
        dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, mode=mode)
        worst = max(worst, _ratio(dev, bnd))
    assert worst > 10.0, f"{mutant}: planted mistake stays within the bound ({worst:.3g})"


@pytest.mark.parametrize("name", ["sagms", "sms08", "bp"])
@pytest.mark.parametrize("rebuild", [None, 1.0])
def test_layered_binary32_decoder_stays_within_the_bound(name, rebuild):
    """The layered schedule: in-place posterior updates, and (rebuild = 1) the posterior
    recomputed from the messages after every round with a posterior above 1."""
    code = I.gb_code(63, 3)
    syn, L0 = _shots(code, 0.05, 10, 71 + len(name))
    kw = MODES[name]
    worst = 0.0
    for s in range(len(syn)):
        G, rounds, _ = D.decode(code, syn[s], L0[s:s + 1], max_iter=25, flags=oracle.FLAG_LAYERED,
                                rebuild_above=rebuild, **kw)
        dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, flags=oracle.FLAG_LAYERED, **kw)
        worst = max(worst, _ratio(dev, bnd))
    assert worst <= 1.0, f"layered {name}: {worst:.3g} of the bound"


def test_layered_replay_rejects_flooding_and_stale_layers():
    """A flooding trace is not a layered one, and a layered decoder that reads the
    round-start posterior breaks the bound."""
    code = I.gb_code(63, 3)
    syn, L0 = _shots(code, 0.05, 8, 44)
    w_flood, w_stale = 0.0, 0.0
    for s in range(len(syn)):
        G, rounds, _ = D.decode(code, syn[s], L0[s:s + 1], max_iter=15)
        if rounds:
            dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, flags=oracle.FLAG_LAYERED)
            w_flood = max(w_flood, _ratio(dev, bnd))
        G, rounds, _ = D.decode(code, syn[s], L0[s:s + 1], max_iter=15, flags=oracle.FLAG_LAYERED,
                                mutant="layer_stale")
        if rounds:
            dev, bnd, _ = oracle.shadow_code(code, syn[s], L0[s:s + 1], G, rounds, flags=oracle.FLAG_LAYERED)
            w_stale = max(w_stale, _ratio(dev, bnd))
    assert w_flood > 10.0 and w_stale > 10.0
