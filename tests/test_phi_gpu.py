"""The BP rule's phi(x) = -ln tanh(x/2) as the decoder evaluates it (two series, one CUDA
expf or logf each), against an FP64 reference and against the library composition
log1pf(2 / expm1f(x)) it replaces: on a grid from 1e-30 through the split at x = 1 to the
underflow of e^-x its error stays within a few FP32 ulps; the ends (0, subnormals, +inf)
saturate as the BP rule needs."""
import numpy as np
import pytest
import torch

from paper_2605_10433_gb300 import _native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def dev_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grid():
    pts = list(np.logspace(-30, 2.3, 200001).astype(np.float32))
    pts += list(np.linspace(0.9, 1.1, 20001).astype(np.float32))
    one = np.float32(1.0)
    pts += [np.nextafter(one, np.float32(0)), one, np.nextafter(one, np.float32(2))]
    pts += list(np.linspace(80.0, 110.0, 3001).astype(np.float32))
    return np.unique(np.array(pts, dtype=np.float32))


def _reference(x):
    x64 = x.astype(np.float64)
    with np.errstate(divide="ignore", over="ignore"):
        small = -np.log(np.tanh(x64 / 2))
        large = 2.0 * np.arctanh(np.exp(-x64))
    return np.where(x64 < 1.0, small, large)


def _ulp_error(y, ref):
    ref32 = ref.astype(np.float32)
    err = np.abs(y.astype(np.float64) - ref)
    ulp = np.spacing(np.abs(ref32)).astype(np.float64)
    finite = np.isfinite(ref)
    out = np.zeros_like(ref)
    out[finite] = err[finite] / ulp[finite]
    out[~finite] = np.where(y[~finite] == ref32[~finite], 0.0, np.inf)
    return out


def test_phi_accuracy_against_fp64_and_the_library_composition():
    x = _grid()
    d = torch.from_numpy(x).cuda()
    mine = _native.sagms_phi(d, 0).cpu().numpy()
    lib = _native.sagms_phi(d, 1).cpu().numpy()
    ref = _reference(x)
    e_mine, e_lib = _ulp_error(mine, ref), _ulp_error(lib, ref)
    print(f"max ulp error: decoder phi {e_mine.max():.2f}, log1pf(2/expm1f(x)) {e_lib.max():.2f}")
    assert e_mine.max() <= 4.0
    assert e_mine.max() <= e_lib.max() + 2.0
    # the ends: phi(0) = +inf, phi(+inf) = 0; below 1e-37 both forms saturate (the library's
    # 2 / expm1f(x) overflows, the series' x/2 reaches the subnormals) at +inf or above 85,
    # where the second phi of the BP rule returns 0 either way
    ends = torch.tensor([0.0, 1e-45, 1e-40, 1e-38, np.inf], dtype=torch.float32).cuda()
    e = _native.sagms_phi(ends, 0).cpu().numpy()
    assert e[0] == np.inf and e[-1] == 0.0 and (e[1:4] > 85.0).all()
