"""The device self-check: the approximate instructions whose exact values
the kernels rely on have them on this GPU (rcp.approx(1) = 1: the intensity
adjoint's fast path divides the transmittance by 1 - alpha = 1 for every
pair outside the cutoff and must leave its bits unchanged)."""
import pytest

pytestmark = pytest.mark.gpu


def test_device_selfcheck():
    import torch
    from paper_2506_21633_b300 import _lib as L
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.sdgr_device_selfcheck(flags.data_ptr())
    torch.cuda.synchronize()
    assert int(flags.item()) == L.SELFCHECK_ALL
