"""Mixed-code batched launches, CUDA graph replay and launch-plan autotuning (GPU).

Each shot's decode is independent of how it is scheduled, so every path here must give
bit-for-bit the results of separate sagms_decode calls (parity of those against the FP64
oracle is covered in test_parity_gpu.py)."""
import numpy as np
import pytest
import torch

import paper_2605_10433_gb300 as S
from paper_2605_10433_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jobs_spec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = []
    for k, (l, w, mode) in enumerate([(255, 3, "sagms"), (255, 4, "sagms"), (255, 5, "sms"), (255, 6, "sagms"),
                                      (255, 8, "sagms"), (63, 3, "bp"), (1023, 5, "ms"), (127, 4, "sagms")]):
        c = I.gb_code(l, w)
        dc = S.DeviceCode.from_code(c)
        shots = 3000 + 977 * k
        _, syn, L0, _ = I.workload(c, [0.01, 0.02, 0.04], shots, seed=900 + k)
        spec.append((dc, torch.from_numpy(syn.view(np.int32)).cuda(), torch.from_numpy(L0).cuda(),
                     S.Params(mode=mode, max_iter=100)))
    return spec


def _reference(spec):
    out = []
    for dc, syn, L0, p in spec:
        out.append(S.decode(dc, syn, L0, p))
    torch.cuda.synchronize()
    return out


def _same(job, ref):
    return all(torch.equal(a, b) for a, b in zip((job.err, job.conv, job.iters), ref))


def test_decode_multi_matches_separate_decodes(jobs_spec):
    ref = _reference(jobs_spec)
    jobs = [S.Job(dc, syn, L0, p) for dc, syn, L0, p in jobs_spec]
    S.decode_multi(jobs)
    torch.cuda.synchronize()
    for j, r in zip(jobs, ref):
        assert _same(j, r)


def test_graph_replays_and_follows_new_inputs(jobs_spec):
    ref = _reference(jobs_spec)
    jobs = [S.Job(dc, syn.clone(), L0.clone(), p) for dc, syn, L0, p in jobs_spec]
    g = S.Graph(jobs)
    for _ in range(2):
        for j in jobs:
            j.err.fill_(-1)
            j.iters.fill_(-7)
        g.launch()
        torch.cuda.synchronize()
        for j, r in zip(jobs, ref):
            assert _same(j, r)
    # new syndromes in the same buffers: the replay decodes them
    j0 = jobs[0]
    dc, _, _, p = jobs_spec[0]
    _, syn2, L02, _ = I.workload(I.gb_code(255, 3), [0.03], j0.syn.shape[0], seed=77)
    j0.syn.copy_(torch.from_numpy(syn2.view(np.int32)))
    j0.L0.copy_(torch.from_numpy(L02))
    g.launch()
    r2 = S.decode(dc, j0.syn, j0.L0, p)
    torch.cuda.synchronize()
    assert _same(j0, r2)
    g.close()


def test_every_launch_plan_gives_identical_results(jobs_spec):
    from paper_2605_10433_gb300 import _native
    dc, syn, L0, p = jobs_spec[4]
    ref = S.decode(dc, syn, L0, p)
    torch.cuda.synchronize()
    for kernel in (0, 1, 2, 3, 4):
        for cps in (0, 1, 2):
            for clg in (0, 1, 3, 4):
                _native.sagms_set_plan(dc.handle, kernel | (cps << 8) | (clg << 16))
                out = S.decode(dc, syn, L0, p)
                torch.cuda.synchronize()
                assert all(torch.equal(a, b) for a, b in zip(out, ref)), (kernel, cps, clg)
    _native.sagms_set_plan(dc.handle, 0)


def test_autotune_picks_a_plan_and_changes_no_result(jobs_spec, tmp_path, monkeypatch):
    dc, syn, L0, p = jobs_spec[1]
    ref = S.decode(dc, syn, L0, p)
    torch.cuda.synchronize()
    plan, rate = S.autotune(dc, syn, L0, p)
    info = S.decode_plan(plan)
    assert info["kernel"] in ("two-group-qc", "two-group", "two-slot", "one-shot-per-CTA") and rate > 0
    out = S.decode(dc, syn, L0, p)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(out, ref))
