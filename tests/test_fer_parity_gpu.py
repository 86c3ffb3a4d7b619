"""Frame-error-rate parity, every mode on every workload (max_iter 100): the GPU decoder and
the FP64 oracle (all host cores) decode the same seeded shots, 1e5 to 1e6 per point.  Per shot
the acceptance of tests/gpu_helpers.py applies (exact agreement, or a shadow-validated
mismatch: at most 0.01% near-ties and at most the workload's cap of amplified ones), and
each side's FER must lie in the other's 95% Wilson interval.

The matrix: GB(127,4) (depolarising p marginalised to 2p/3) in every mode; GB(255, w) for every
w in every mode; GB(1023,5) on the headline mix in every mode; and the serving workload's four
codes at its noise range, one point per code."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.stats import wilson_interval
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

MODES = {
    "sagms": S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=100),
    "sms": S.Params(mode="sms", alpha=0.75, max_iter=100),
    "ms": S.Params(mode="ms", max_iter=100),
    "bp": S.Params(mode="bp", max_iter=100),
}
CASES = ([((127, 4), p * 2 / 3, mode, 4000 + k) for k, (p, mode) in enumerate(
             [(0.04, "sagms"), (0.04, "sms"), (0.04, "ms"), (0.04, "bp"), (0.02, "sagms"), (0.01, "sagms")])]
         + [((255, w), 0.02, "sagms", 5000 + w) for w in (3, 4, 5, 6, 8)])
# config 3, the other modes: 1e5 shots per code and mode
CASES3 = [((255, w), 0.02, mode, 5100 + 10 * w + k) for w in (3, 4, 5, 6, 8)
          for k, mode in enumerate(("ms", "sms", "bp"))]
# config 4: GB(1023,5) on the headline mix p in {0.005, 0.01, 0.02} (shots interleaved)
CASES4 = [("sagms", 1_000_000, 6000), ("sms", 100_000, 6001), ("ms", 200_000, 6002), ("bp", 100_000, 6003)]
# the serving workload's codes (n = 126, 510, 1022, 2046), p over its range U[0.005, 0.03]
SERVING = [((63, 3), 7001), ((255, 4), 7002), ((511, 5), 7003), ((1023, 5), 7004)]
SERVING_P = [0.005, 0.01, 0.015, 0.02, 0.025, 0.03]
# Cap on amplified mismatches (fraction of shots) per workload and mode: about twice the
# measured count, rounded up (the measured values are in the design notes).
AMPLIFIED_CAP = {"sagms": 1e-3, "sms": 1e-2, "ms": 1e-3, "bp": 5e-3}


def _fer_check(r, shots):
    fails_g = int(round(r["fer_gpu"] * shots))
    fails_o = int(round(r["fer_oracle"] * shots))
    lo_o, hi_o = wilson_interval(fails_o, shots)
    lo_g, hi_g = wilson_interval(fails_g, shots)
    assert lo_o - 1e-12 <= r["fer_gpu"] <= hi_o + 1e-12
    assert lo_g - 1e-12 <= r["fer_oracle"] <= hi_g + 1e-12
    return lo_o, hi_o


def _line(tag, shots, r, lo, hi):
    print(f"{tag}: {shots} shots, FER gpu {r['fer_gpu']:.3e} oracle {r['fer_oracle']:.3e} [{lo:.3e}, {hi:.3e}], "
          f"mismatches {r['mismatch']} (near-tie {r['near_tie']}, amplified {r['amplified']}, "
          f"shadow worst {r['shadow_worst']:.3g})")


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("lw,q,mode,seed", CASES)
def test_million_shot_fer_parity(lw, q, mode, seed):
    """Config 2 (GB(127,4), depolarising p = 0.04, 0.02, 0.01 marginalised to q = 2p/3; every
    mode at p = 0.04) and config 3 (GB(255, w) for every w at q = 0.02)."""
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    shots = 1_000_000
    _, syn, L0, _ = I.workload(c, [q], shots, seed=seed)
    r = G.compare(c, dc, syn, L0, MODES[mode], max_amplified=AMPLIFIED_CAP[mode])
    lo, hi = _fer_check(r, shots)
    _line(f"GB{lw} q={q:.4f} {mode}", shots, r, lo, hi)


@pytest.mark.parametrize("lw,q,mode,seed", CASES3)
def test_config3_other_modes_fer_parity(lw, q, mode, seed):
    """Config 3 (GB(255, w), w in {3, 4, 5, 6, 8}, q = 0.02) in MS, SMS(0.75) and BP."""
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    shots = 100_000
    _, syn, L0, _ = I.workload(c, [q], shots, seed=seed)
    r = G.compare(c, dc, syn, L0, MODES[mode], max_amplified=AMPLIFIED_CAP[mode])
    lo, hi = _fer_check(r, shots)
    _line(f"GB{lw} q={q:.4f} {mode}", shots, r, lo, hi)


@pytest.mark.parametrize("mode,shots,seed", CASES4)
def test_large_code_fer_parity(mode, shots, seed):
    """Config 4: GB(1023,5), iid Z flips at p in {0.005, 0.01, 0.02}, max_iter 100."""
    c = I.gb_code(1023, 5)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02], shots, seed=seed)
    r = G.compare(c, dc, syn, L0, MODES[mode], max_amplified=AMPLIFIED_CAP[mode])
    lo, hi = _fer_check(r, shots)
    _line(f"GB(1023,5) {mode}", shots, r, lo, hi)


@pytest.mark.parametrize("lw,seed", SERVING)
def test_serving_codes_fer_parity(lw, seed):
    """The serving workload's codes with SAGMS at its noise range (p interleaved over
    0.005..0.03), 1e5 shots each."""
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    shots = 100_000
    _, syn, L0, _ = I.workload(c, SERVING_P, shots, seed=seed)
    r = G.compare(c, dc, syn, L0, MODES["sagms"], max_amplified=AMPLIFIED_CAP["sagms"])
    lo, hi = _fer_check(r, shots)
    _line(f"serving GB{lw} sagms", shots, r, lo, hi)
