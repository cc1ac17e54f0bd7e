"""Host-side checks of the binding (no GPU): caller output buffers are
validated before their raw pointers reach a kernel."""
import pytest
import torch

from paper_2509_26222_gb300 import native


def test_output_buffer_checks():
    ok = torch.empty(10, dtype=torch.float32)
    assert native._out_tensor(ok, 10, "cpu") is ok
    assert native._out_tensor(torch.empty(3, 4), 12, "cpu").numel() == 12
    with pytest.raises(ValueError):
        native._out_tensor(torch.empty(9), 10, "cpu")  # too small
    with pytest.raises(ValueError):
        native._out_tensor(torch.empty(10, dtype=torch.float64), 10, "cpu")  # wrong type
    with pytest.raises(ValueError):
        native._out_tensor(torch.empty(4, 6)[:, ::2], 12, "cpu")  # not contiguous
    with pytest.raises(ValueError):
        native._out_tensor([0.0] * 10, 10, "cpu")  # not a tensor
