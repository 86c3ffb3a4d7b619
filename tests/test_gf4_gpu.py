"""GPU parity of the quaternary (GF(4)) decoder against the GF(4) FP64 oracle, on the paper's own
decoding setting (Sec. II, Sec. V): the overcomplete stabilizer matrix of a GB code with l = 63,
w = 5 (X-type rows of H_X over Z-type rows of H_Z: m = 126 rows, check and qubit degree 10),
depolarising noise at eps, prior L0 = ln((1 - eps0)/(eps0/3)) with eps0 = eps (matched) or
eps0 = 0.1 (the mismatch of Fig. 2b / Fig. 3).  Modes: BP4, SMS(0.5), SAGMS(0.30, 0.50, 1.10).

Per point: each side's FER lies in the other's 95% Wilson interval; per-shot outputs
(x bits, z bits, conv, iters) are identical except for a capped fraction of shots, each traced
to its first differing decision; posterior traces agree to 1e-5 (normwise, LLR units) at every
check before the first differing decision within the first rounds.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_10433_gb300 as S
from oracle import gf4 as O4
from paper_2605_10433_gb300 import inputs as I
from paper_2605_10433_gb300.inputs import gf4 as I4
from paper_2605_10433_gb300.stats import wilson_interval

pytestmark = pytest.mark.gpu

MODES = {
    "bp": (S.Params(mode="bp", max_iter=100), oracle.BP),
    "sms": (S.Params(mode="sms", alpha=0.5, max_iter=100), oracle.SMS),
    "sagms": (S.Params(mode="sagms", alpha_min=0.30, alpha_max=0.50, eta_unsat=1.10, max_iter=100), oracle.SAGMS),
}
MISMATCH_CAP = 2e-3


@pytest.fixture(scope="module")
def setting():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = I4.css_code(I.gb_code(63, 5))
    return g, S.Gf4DeviceCode(g)


def _run(g, dc, syn, L0, p, mode_o, trace=False, threads=16):
    d_syn = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda()
    d_L0 = torch.from_numpy(np.ascontiguousarray(L0, dtype=np.float32)).cuda()
    out = S.gf4_decode(dc, d_syn, d_L0, p, trace=trace)
    torch.cuda.synchronize()
    gres = {"ex": out[0][:, 0].cpu().numpy().view(np.uint32), "ez": out[0][:, 1].cpu().numpy().view(np.uint32),
            "conv": out[1].cpu().numpy(), "iters": out[2].cpu().numpy()}
    if trace:
        gres["trace"] = out[3].cpu().numpy()
    o = O4.decode(g, syn, L0.astype(np.float64), mode=mode_o, alpha=p.alpha, alpha_min=p.alpha_min,
                  alpha_max=p.alpha_max, eta_unsat=p.eta_unsat, max_iter=p.max_iter, flags=p.flags, trace=trace,
                  threads=threads)
    return gres, o


def _same(a, b):
    return ((a["ex"] == b["ex"]).all(axis=1) & (a["ez"] == b["ez"]).all(axis=1) & (a["conv"] == b["conv"])
            & (a["iters"] == b["iters"]))


@pytest.mark.parametrize("eps,eps0", [(0.01, 0.01), (0.02, 0.02), (0.01, 0.1), (0.02, 0.1)])
@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_fer_parity(setting, mode, eps, eps0):
    g, dc = setting
    shots = 100_000
    _, _, syn = I4.depolarizing(g, eps, shots, seed=int(9000 + 1000 * eps + 100 * eps0))
    L0 = np.full(shots, I4.prior(eps0), dtype=np.float32)
    p, mo = MODES[mode]
    gr, o = _run(g, dc, syn, L0, p, mo)
    same = _same(gr, o)
    bad = np.nonzero(~same)[0]
    fer_g, fer_o = 1 - gr["conv"].mean(), 1 - o["conv"].mean()
    lo, hi = wilson_interval(int(round(fer_o * shots)), shots)
    lo_g, hi_g = wilson_interval(int(round(fer_g * shots)), shots)
    assert lo - 1e-12 <= fer_g <= hi + 1e-12
    assert lo_g - 1e-12 <= fer_o <= hi_g + 1e-12
    # classify the mismatches at their first differing decision (traced re-decode of both sides)
    near = 0
    for c0 in range(0, min(len(bad), 256), 64):
        idx = bad[c0:c0 + 64]
        gt, ot = _run(g, dc, syn[idx], L0[idx], p, mo, trace=True)
        for k, s in enumerate(idx):
            assert gt["iters"][k] == gr["iters"][s] and np.array_equal(gt["ex"][k], gr["ex"][s])
            last = min(int(gt["iters"][k]), int(ot["iters"][k]))
            for l in range(last + 1):
                a = np.concatenate([np.zeros((g.n, 1)), gt["trace"][k, l]], axis=1)
                b = np.concatenate([np.zeros((g.n, 1)), ot["trace"][k, l]], axis=1)
                if (np.argmin(a, axis=1) != np.argmin(b, axis=1)).any():
                    diff = np.argmin(a, axis=1) != np.argmin(b, axis=1)
                    srt = np.sort(b[diff], axis=1)
                    near += int(float((srt[:, 1] - srt[:, 0]).max()) < 1e-4)
                    break
    assert len(bad) <= MISMATCH_CAP * shots, f"{len(bad)} mismatching shots of {shots}"
    print(f"gf4 GB(63,5) CSS eps={eps} eps0={eps0} {mode}: FER gpu {fer_g:.3e} oracle {fer_o:.3e} "
          f"[{lo:.3e}, {hi:.3e}], mismatches {len(bad)} ({near} near-ties among the first 256), "
          f"mean iters {gr['iters'].mean():.2f}")


@pytest.mark.parametrize("mode", ["bp", "sms", "sagms"])
def test_gf4_posterior_traces(setting, mode):
    g, dc = setting
    _, _, syn = I4.depolarizing(g, 0.03, 64, seed=321)
    L0 = np.full(64, I4.prior(0.03), dtype=np.float32)
    p, mo = MODES[mode]
    p = S.Params(**{**p.__dict__, "max_iter": 30})
    gt, ot = _run(g, dc, syn, L0, p, mo, trace=True)
    worst = 0.0
    for s in range(64):
        last = min(int(gt["iters"][s]), int(ot["iters"][s]), 3)
        for l in range(last + 1):
            a = gt["trace"][s, l].astype(np.float64)
            b = ot["trace"][s, l]
            da = np.argmin(np.concatenate([np.zeros((g.n, 1)), a], axis=1), axis=1)
            db = np.argmin(np.concatenate([np.zeros((g.n, 1)), b], axis=1), axis=1)
            e = float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1.0))
            worst = max(worst, e)
            assert e <= 1e-5, f"shot {s} check {l}: normwise error {e:.3g}"
            if (da != db).any():
                break
    print(f"gf4 traces {mode}: normwise error {worst:.2e} over the first rounds")


def test_gf4_edge_cases(setting):
    g, dc = setting
    z = torch.zeros((50, g.mw), dtype=torch.int32, device="cuda")
    L0 = torch.full((50,), float(I4.prior(0.01)), dtype=torch.float32, device="cuda")
    L0[7] = float("nan")
    err, conv, iters = S.gf4_decode(dc, z, L0, MODES["sagms"][0])
    torch.cuda.synchronize()
    assert not err.any()
    c, it = conv.cpu().numpy(), iters.cpu().numpy()
    assert it[7] == -1 and c[7] == 0
    keep = np.arange(50) != 7
    assert (c[keep] == 1).all() and (it[keep] == 0).all()
    e0, _, _ = S.gf4_decode(dc, torch.zeros((0, g.mw), dtype=torch.int32, device="cuda"),
                            torch.zeros((0,), dtype=torch.float32, device="cuda"), MODES["bp"][0])
    assert e0.shape[0] == 0
