"""Failure detection without a GPU fault: the library's spin-waits are bounded, and a wait
that runs out sets the device status word's timeout bit and returns.  The self-test kernel
takes that path on purpose (a barrier nothing arrives on); the host must see
LX_ERR_DEVICE_STATUS at the next sync, the word must be cleared by reading it, and the
device must stay usable for the next batch."""
import numpy as np
import pytest

import oracle
from paper_2307_03452_gb300 import inputs, lx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def test_exhausted_wait_is_reported_and_the_device_stays_usable():
    lx.sync_status()  # start from a clear status word
    lx.selftest_timeout(1000)
    with pytest.raises(lx.LxError) as e:
        lx.sync_status()
    assert e.value.code == -9  # LX_ERR_DEVICE_STATUS
    lx.sync_status()  # cleared by the read
    basis, quartets = inputs.uniform_class((4, 4, 4, 4), 4, 61, cube=3.0, exps=(0.1, 5.0))
    out, off = lx.eri(basis, quartets, solid=True, path="split")
    ref, _ = oracle.eri(basis, quartets, solid=True)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10
