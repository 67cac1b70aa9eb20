"""Failure detection without a GPU fault: a bounded device-side wait that runs
out is reported as SHT_ETIMEOUT by sht_sync_status, and the handle (and the
CUDA context) stay usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_1202_6522_gb300 import synthetic

from _util import fp64_bound, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_bounded_wait_reports_timeout_and_recovers():
    from paper_1202_6522_gb300 import build
    build.build()
    from paper_1202_6522_gb300 import SHT, _capi as C
    sht = SHT(15, 15, 16, 32)
    stream = torch.cuda.current_stream().cuda_stream
    assert C.sht_sync_status(sht._h, stream) == 0
    C.sht_selftest_timeout(sht._h, 20000, stream)   # 20 ms bound on a barrier nothing completes
    with pytest.raises(C.SHTError) as exc:
        C.sht_sync_status(sht._h, stream)
    assert exc.value.code == C.SHT_ETIMEOUT
    assert C.sht_sync_status(sht._h, stream) == 0   # reading the status cleared it
    a = synthetic.spectrum(15, seed=1)
    g = sht.synth_(torch.from_numpy(a).to(DEV))
    assert normwise(g.cpu().numpy(), oracle.synth(15, 15, 16, 32, a)) < fp64_bound(15)
