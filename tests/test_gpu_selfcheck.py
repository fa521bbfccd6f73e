"""The device self-check: the approximate instructions whose exact values
the kernels rely on have them on this GPU (rcp.approx(1) = 1: the intensity
adjoint's fast path divides the transmittance by 1 - alpha = 1 for every
pair outside the cutoff and must leave its bits unchanged).  And the
pipe-rate diagnostic behind the roofline gives rates a GPU can have."""
import pytest

pytestmark = pytest.mark.gpu


def test_device_selfcheck():
    import torch
    from paper_2506_21633_b300 import _lib as L
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.sdgr_device_selfcheck(flags.data_ptr())
    torch.cuda.synchronize()
    assert int(flags.item()) == L.SELFCHECK_ALL


def test_pipe_rates_plausible():
    """Per-SM rates in thread-instructions per cycle: fma at most the 128 FP32
    lanes and not far below them, the SFU kinds well below fma, the mixed
    streams between the two (an SFU instruction costs at least one slot)."""
    import torch
    from paper_2506_21633_b300 import _lib as L
    scratch = torch.empty(L.PIPE_RATES_SCRATCH, dtype=torch.uint8, device="cuda")
    r = L.sdgr_pipe_rates(scratch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert 64.0 <= r["ffma"] <= 128.5
    assert 4.0 <= r["ex2"] <= r["ffma"] / 2 and 4.0 <= r["rcp"] <= r["ffma"] / 2
    for k in ("ex2_in_ffma_stream", "rcp_in_ffma_stream"):
        assert 0.3 * r["ffma"] <= r[k] <= 1.02 * r["ffma"], (k, r)
    # a packed instruction does two FMAs: the FMA rate stays at most the
    # lanes' (two per instruction), the instruction rate about half of fma's
    assert 0.3 * r["ffma"] <= r["ffma2"] and 2 * r["ffma2"] <= 1.02 * r["ffma"] + 2.0, r
    # beside integer work, more FMAs per cycle go through packed than scalar
    # (half of each alternating stream is FMA instructions: one FMA or two)
    assert r["ffma_and_lop3"] <= 128.5 and r["ffma2_and_lop3"] <= 128.5, r
    assert r["ffma2_and_lop3"] >= r["ffma_and_lop3"] / 2, r
