"""Channel mismatch (Sec. V-C, Fig. 2b and Fig. 3): the decoder assumes a depolarising
probability eps0 = 0.1 while the shots are drawn at eps in {0.01, 0.02}.  On the binary
(Z-flip) problem this is a per-shot prior L0 = ln((1 - q0)/q0) with q0 = 2 eps0 / 3 that
differs from the sampling probability q = 2 eps / 3.

* GPU against the FP64 oracle on the same mismatched shots, every mode the experiment
  compares (SAGMS, SMS(0.75), BP), under the acceptance of tests/gpu_helpers.py and the
  Wilson-interval FER check.
* The MS family is positively homogeneous in its messages, so its decisions do not depend on
  |L0| at all: SAGMS and SMS decode the mismatched shots exactly as the matched ones.  BP is
  not homogeneous, and its FER moves with the assumed eps0 -- the robustness argument of
  Sec. V-C, measured here on the GPU path.
"""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

EPS0 = 0.1
MODES = {
    "sagms": S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=100),
    "sms": S.Params(mode="sms", alpha=0.75, max_iter=100),
    "bp": S.Params(mode="bp", max_iter=100),
}
CASES = [((127, 4), 0.02, 100_000, 8101), ((127, 4), 0.01, 100_000, 8102), ((1023, 5), 0.02, 100_000, 8103)]


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shots(code, eps, shots, seed):
    q = float(I.depolarizing_to_z(eps))
    _, syn, L0, _ = I.workload(code, [q], shots, seed=seed)
    q0 = float(I.depolarizing_to_z(EPS0))
    L0_mis = np.full(shots, np.log((1 - q0) / q0), dtype=np.float32)
    return syn, L0, L0_mis


@pytest.mark.parametrize("lw,eps,shots,seed", CASES)
@pytest.mark.parametrize("mode", ["sagms", "sms", "bp"])
def test_mismatched_prior_fer_parity(lw, eps, shots, seed, mode):
    c = I.gb_code(*lw)
    dc = S.DeviceCode.from_code(c)
    syn, L0, L0_mis = _shots(c, eps, shots, seed)
    r = G.compare(c, dc, syn, L0_mis, MODES[mode])
    (lo, hi), pm = G.fer_check(r, shots)
    matched = G.gpu_decode(dc, syn, L0, MODES[mode])
    fer_matched = float((matched["conv"] == 0).mean())
    if mode != "bp":
        # homogeneous rule: the assumed eps0 changes nothing
        for k in ("err", "conv", "iters"):
            assert np.array_equal(matched[k], r["gpu"][k])
    print(f"mismatch GB{lw} eps={eps} eps0={EPS0} {mode}: FER gpu {r['fer_gpu']:.3e} oracle {r['fer_oracle']:.3e} "
          f"[{lo:.3e}, {hi:.3e}] McNemar p {pm:.3g} (matched prior: {fer_matched:.3e}); mismatches {r['mismatch']} "
          f"(near-tie {r['near_tie']}, amplified {r['amplified']})")
