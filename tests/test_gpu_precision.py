"""Half storage (FP16 / BF16 volumes and sinograms, FP32 arithmetic) against
the FP64 oracle, error stated per result.

Bound from the storage rounding: A and the test inputs are non-negative, so
an input rounding |dx| <= u |x| (unit roundoff u) gives |A dx| <= u A|x|
elementwise, and an output rounding adds u: relative L2 <= u per rounding
(+ the FP32 arithmetic, ~1e-5).  FP16 keeps 11 significant bits (u = 2^-11):
2^-11 one side, 2^-10 both -- within 1e-3.  BF16 keeps 8 (u = 2^-8 = 3.9e-3):
2^-8 one side, 2^-7 both; on piecewise-constant phantoms the input errors do
not average out (every voxel of a body rounds the same value), so BF16
storage cannot promise 1e-3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import PROJECTORS, TOL_F16, ragged, rel_l2

pytestmark = pytest.mark.gpu
T = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
# (input, output, bound)
ARITH = 2e-5
CASES = [("f16", "f16", 2.0 ** -10 + ARITH), ("f16", "f32", 2.0 ** -11 + ARITH),
         ("f32", "f16", 2.0 ** -11 + ARITH), ("bf16", "f32", 2.0 ** -8 + ARITH),
         ("bf16", "bf16", 2.0 ** -7 + ARITH)]


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


@pytest.mark.parametrize("tin,tout,bound", CASES)
@pytest.mark.parametrize("proj", PROJECTORS)
@pytest.mark.parametrize("kind", ["circ3d", "noncirc3d"])
def test_half_storage_forward_and_back(ct, report, kind, proj, tin, tout, bound):
    assert bound <= TOL_F16 or "bf16" in (tin, tout)
    spec = ragged(kind, "flat", seed=7)
    g = ct.Geometry.from_spec(spec)
    x = W.phantom(spec, seed=3)
    y_ref = oracle.forward(spec, proj, x)
    y = ct.forward(g, torch.as_tensor(x, dtype=T[tin]).cuda(), proj, out_dtype=T[tout])
    e_fwd = rel_l2(y.float().cpu().numpy(), y_ref)
    s = W.random_sino(spec, seed=3)[0]
    x_ref = oracle.back(spec, proj, s)
    xb = ct.back(g, torch.as_tensor(s, dtype=T[tin]).cuda(), proj, out_dtype=T[tout])
    e_back = rel_l2(xb.float().cpu().numpy(), x_ref)
    report(f"{kind} {proj} {tin}->{tout}: forward {e_fwd:.2e}, back {e_back:.2e}")
    assert e_fwd <= bound and e_back <= bound, (e_fwd, e_back)


def test_half_output_rounds_once(ct):
    """FP16 output equals the FP32 result rounded to FP16 (one rounding)."""
    spec = ragged("circ3d", "curved", seed=8)
    g = ct.Geometry.from_spec(spec)
    x = torch.as_tensor(W.phantom(spec, seed=4), dtype=torch.float32).cuda()
    for proj in PROJECTORS:
        y32 = ct.forward(g, x, proj)
        y16 = ct.forward(g, x, proj, out_dtype=torch.float16)
        assert torch.equal(y16, y32.half())
