"""kc_atomic_ceilings: the measured random-update rates the bench's roofline
uses as its atomic ceiling are positive and ordered as the memory they hit
(shared memory above L2-resident global memory above HBM-resident)."""
import pytest

import paper_1712_03254_gb300 as kc

pytestmark = pytest.mark.gpu


def test_atomic_ceilings_are_ordered():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = kc.atomic_ceilings()
    assert all(v > 0 for v in r.values())
    assert r["smem_add32_per_s"] > r["l2_or64_per_s"] > r["hbm_or64_per_s"]
    assert r["smem_or64_per_s"] > r["hbm_or64_per_s"]
