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


class _Fn:
    """A stand-in library function: records its calls, returns 0."""

    def __init__(self, log, name, effect=None):
        self.log, self.name, self.effect = log, name, effect

    def __call__(self, *args):
        self.log.append((self.name, args))
        if self.effect:
            self.effect(*args)
        return 0


class _FakeLib:
    """Stands in for libsimsense: creates report handle 0x1234, calls succeed."""

    def __init__(self):
        self.log = []
        self._batch_ready = False

    def __getattr__(self, name):
        if not name.startswith("simsense_"):
            raise AttributeError(name)

        def make_handle(out, *_):
            out._obj.value = 0x1234            # byref(handle) -> the handle itself

        fn = _Fn(self.log, name, make_handle if name in ("simsense_create", "simsense_batch_create") else None)
        setattr(self, name, fn)
        return fn


class _Stream:
    cuda_stream = 0


@pytest.fixture
def fake_lib(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(simsense, "_lib", lib)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 1)
    return lib


def test_handle_calls_pass_the_tensors_addresses_to_the_library(fake_lib):
    from paper_2201_11924_gb300 import configs
    wl = configs.SMALL_320
    m = simsense.SimSense.from_workload(wl)
    assert m.device == 1                             # the GPU current at creation
    l, r = _fake((wl.H, wl.W), torch.uint8, 1), _fake((wl.H, wl.W), torch.uint8, 1)
    d = _fake((wl.H, wl.W), torch.float32, 1)
    m.compute(l, r, d, stream=_Stream())
    name, args = fake_lib.log[-1]
    assert name == "simsense_compute"
    assert [a.value for a in args[1:4]] == [l.data_ptr(), r.data_ptr(), d.data_ptr()]
    with pytest.raises(ValueError, match="cuda:0, but the kernels run on cuda:1"):
        m.compute(_fake((wl.H, wl.W), torch.uint8, 0), r, d, stream=_Stream())
    m.close()
    assert fake_lib.log[-1][0] == "simsense_destroy"


def test_batch_calls_pass_the_tensors_addresses_to_the_library(fake_lib):
    from paper_2201_11924_gb300 import configs
    wls = [configs.SMALL_320, configs.SMALL_320.with_(D=96)]
    b = simsense.SimSenseBatch(wls)
    assert b.device == 1
    ls = [_fake((w.H, w.W), torch.uint8, 1) for w in wls]
    rs = [_fake((w.H, w.W), torch.uint8, 1) for w in wls]
    ds = [_fake((w.H, w.W), torch.float32, 1) for w in wls]
    b.compute(ls, rs, ds, stream=_Stream())
    name, args = fake_lib.log[-1]
    assert name == "simsense_batch_compute"
    assert [args[1][i] for i in range(2)] == [t.data_ptr() for t in ls]
    assert [args[3][i] for i in range(2)] == [t.data_ptr() for t in ds]
    with pytest.raises(ValueError, match=r"depth\[1\] is on cuda:0"):
        b.compute(ls, rs, [ds[0], _fake((wls[1].H, wls[1].W), torch.float32, 0)], stream=_Stream())
    b.close()
