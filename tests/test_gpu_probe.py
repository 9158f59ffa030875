"""The read-bandwidth probe behind the L2 roofline: a buffer far above L2
reads at about the measured HBM copy rate, one that fits in L2 reads faster."""

import json
import os

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def la():
    import torch
    from paper_1110_6231_gb300 import build
    build.build()
    import paper_1110_6231_gb300 as la
    assert torch.cuda.is_available()
    return la


def test_probe_hbm_and_l2_rates(la):
    import torch
    big = torch.ones(1 << 30, dtype=torch.int32, device="cuda")        # 4 GiB
    small = torch.ones(16 << 20, dtype=torch.int32, device="cuda")     # 64 MiB
    la.probe_read_gbps(big, 1)
    hbm = max(la.probe_read_gbps(big, 2) for _ in range(3))
    la.probe_read_gbps(small, 1)
    l2 = max(la.probe_read_gbps(small, 20) for _ in range(3))
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    ref = json.load(open(peaks)).get("hbm_gbs") if os.path.exists(peaks) else 6800.0
    assert 0.5 * ref < hbm < 1.5 * ref, (hbm, ref)
    assert l2 > 1.2 * hbm, (l2, hbm)
