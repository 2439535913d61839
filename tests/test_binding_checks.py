"""Argument checks of the Python binding that need no GPU: the tensors'
type, shape, layout and GPU are checked before any address reaches the
library (a tensor on another GPU than the one the kernels run on would be
read through a foreign address).  CUDA tensors are imitated by a tensor
subclass that reports a CUDA device; only the checks run, nothing launches."""
import pytest
import torch

from paper_2201_11924_gb300 import simsense


class _OnGpu(torch.Tensor):
    gpu = 0

    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        return torch.device("cuda", type(self).gpu)


def _fake(shape, dtype, gpu):
    cls = type(f"OnGpu{gpu}", (_OnGpu,), {"gpu": gpu})
    return torch.zeros(shape, dtype=dtype).as_subclass(cls)


def test_a_tensor_on_the_kernels_gpu_passes():
    t = _fake((4, 6), torch.uint8, 1)
    assert simsense._dev_ptr(t, torch.uint8, (4, 6), "left", device=1).value == t.data_ptr()


def test_a_tensor_on_another_gpu_is_refused():
    with pytest.raises(ValueError, match=r"left is on cuda:1, but the kernels run on cuda:0"):
        simsense._dev_ptr(_fake((4, 6), torch.uint8, 1), torch.uint8, (4, 6), "left", device=0)


@pytest.mark.parametrize("t,why", [
    (torch.zeros((4, 6), dtype=torch.uint8), "CUDA tensor"),                    # host memory
    (_fake((4, 6), torch.int16, 0), "contiguous"),                               # dtype
    (_fake((6, 4), torch.uint8, 0), "contiguous"),                               # shape
    (_fake((6, 4), torch.uint8, 0).t(), "contiguous"),                           # strided view
    (None, "CUDA tensor"),
])
def test_type_shape_layout_and_host_tensors_are_refused(t, why):
    with pytest.raises(ValueError, match=why):
        simsense._dev_ptr(t, torch.uint8, (4, 6), "left", device=0)
