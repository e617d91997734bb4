"""Reporting of bounded device-side waits that give up (the status word behind
sfft4_sync_status), exercised from the host: a test hook sets the word as a wait that gave up
does, so no device wait has to run out on the GPU."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def test_sync_status_reports_timeout_once(s4):
    import torch
    from paper_2011_05698_gb300 import _lib
    p = s4.Plan(2**14, 16, 4, 0.5, seed=0, B1=64, precision="bf16x3")
    idx, val, nf, votes = p.execute(torch.zeros(2**14, dtype=torch.complex64, device="cuda"))
    p.sync_status()                       # a clean execute leaves the word clear
    p.inject_status(1)
    with pytest.raises(s4.Sfft4Error) as e:
        p.sync_status()
    assert e.value.code == _lib.SFFT4_ETIMEOUT
    p.sync_status()                       # reading it cleared it
    # an execute after the report runs normally and leaves the word clear
    p.execute(torch.zeros(2**14, dtype=torch.complex64, device="cuda"))
    p.sync_status()
    assert int(nf) == 0
    p.close()


def test_sync_status_of_a_batch_plan(s4):
    from paper_2011_05698_gb300 import _lib
    bp = s4.BatchPlan([2**16, 2**14], [20, 16], 16, 1.0, seed=1)
    bp.sync_status()
    _lib.load().sfft4_inject_status(bp._h, 1)
    with pytest.raises(s4.Sfft4Error) as e:
        bp.sync_status()
    assert e.value.code == _lib.SFFT4_ETIMEOUT
    bp.sync_status()
    bp.close()
