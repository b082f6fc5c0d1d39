"""The binding of sg2v_sum_counts_noalloc checks torch tensors before the
call: the C entry point receives bare pointers and cannot see a buffer's
length or element type, so a float32 or too-short tensor would be read past
its end on the device.  These checks run on the CPU and launch nothing."""
import pytest
import torch

import paper_2009_11665_b300 as sg


def test_rejects_float32_values():
    with pytest.raises(ValueError, match="float64"):
        sg.sg2v_sum_counts_noalloc(torch.ones(8, dtype=torch.float32), 8, 1, torch.empty(1, dtype=torch.float64))


def test_rejects_short_values_and_totals():
    with pytest.raises(ValueError, match="needs 12"):
        sg.sg2v_sum_counts_noalloc(torch.ones(11, dtype=torch.float64), 4, 3, torch.empty(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="needs 3"):
        sg.sg2v_sum_counts_noalloc(torch.ones(12, dtype=torch.float64), 4, 3, torch.empty(2, dtype=torch.float64))


def test_rejects_host_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        sg.sg2v_sum_counts_noalloc(torch.ones(12, dtype=torch.float64), 4, 3, torch.empty(3, dtype=torch.float64))
