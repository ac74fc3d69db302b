"""The hardware probes behind the benchmark's roofline denominators: each
returns a finite positive rate of a plausible size, and the shared-memory load
rate exceeds the rate at which bulk copies fill shared memory from L2 (the
loads only read on-chip memory)."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def syk():
    import paper_2311_00639_b300 as p

    return p


def test_probe_rates(syk):
    import torch

    buf = torch.zeros(32 << 20, dtype=torch.uint8, device="cuda")
    lds = syk.probe_smem()
    stage = {r: syk.probe_staging(buf, r, 1024) for r in (-1, 0, 1, 2)}
    dfma = syk.probe_fp64()
    print(f"smem loads {lds / 1e12:.2f} TB/s, staging {[round(v / 1e12, 2) for v in stage.values()]} TB/s, "
          f"DFMA {dfma / 1e12:.3f} T/s")
    for v in (lds, dfma, *stage.values()):
        assert math.isfinite(v) and v > 0
    assert 1e12 < lds < 1e15
    assert all(1e11 < v < 1e15 for v in stage.values())
    assert lds > stage[0]
    assert 1e10 < dfma < 1e14
