"""Frame-error-rate parity at a million shots per point (configs 2 and 3, max_iter 100):
the GPU decoder and the FP64 oracle (all host cores) decode the same seeded shots.  Per shot
the usual acceptance of tests/gpu_helpers.py applies (exact agreement except for reported
FP32-undetermined shots and at most 0.01% near-ties), and each side's FER must lie in the
other's 95% Wilson interval."""
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
# config 4: GB(1023,5) on the headline mix p in {0.005, 0.01, 0.02} (shots interleaved)
CASES4 = [("sagms", 1_000_000, 6000), ("sms", 100_000, 6001), ("ms", 200_000, 6002)]


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
    r = G.compare(c, dc, syn, L0, MODES[mode])
    fails_g = int(round(r["fer_gpu"] * shots))
    fails_o = int(round(r["fer_oracle"] * shots))
    lo_o, hi_o = wilson_interval(fails_o, shots)
    lo_g, hi_g = wilson_interval(fails_g, shots)
    assert lo_o - 1e-12 <= r["fer_gpu"] <= hi_o + 1e-12
    assert lo_g - 1e-12 <= r["fer_oracle"] <= hi_g + 1e-12
    print(f"GB{lw} q={q:.4f} {mode}: {shots} shots, FER gpu {r['fer_gpu']:.3e} oracle {r['fer_oracle']:.3e} "
          f"[{lo_o:.3e}, {hi_o:.3e}], mismatches {r['mismatch']} (near-tie {r['near_tie']}, "
          f"undetermined {r['ill_conditioned']})")


@pytest.mark.parametrize("mode,shots,seed", CASES4)
def test_large_code_fer_parity(mode, shots, seed):
    """Config 4: GB(1023,5), iid Z flips at p in {0.005, 0.01, 0.02}, max_iter 100."""
    c = I.gb_code(1023, 5)
    dc = S.DeviceCode.from_code(c)
    _, syn, L0, _ = I.workload(c, [0.005, 0.01, 0.02], shots, seed=seed)
    r = G.compare(c, dc, syn, L0, MODES[mode])
    fails_o = int(round(r["fer_oracle"] * shots))
    fails_g = int(round(r["fer_gpu"] * shots))
    lo_o, hi_o = wilson_interval(fails_o, shots)
    lo_g, hi_g = wilson_interval(fails_g, shots)
    assert lo_o - 1e-12 <= r["fer_gpu"] <= hi_o + 1e-12
    assert lo_g - 1e-12 <= r["fer_oracle"] <= hi_g + 1e-12
    print(f"GB(1023,5) {mode}: {shots} shots, FER gpu {r['fer_gpu']:.3e} oracle {r['fer_oracle']:.3e} "
          f"[{lo_o:.3e}, {hi_o:.3e}], mismatches {r['mismatch']} (near-tie {r['near_tie']}, "
          f"undetermined {r['ill_conditioned']})")
