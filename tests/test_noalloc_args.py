"""Argument checks of the allocation-free statistics entry point that run
before the C call (which sees bare device pointers and cannot check sizes or
devices), exercised on the CPU with stand-ins for device tensors."""
import pytest


class FakeDeviceTensor:
    """Just enough of a CUDA tensor for the argument checks."""

    is_cuda = True

    def __init__(self, n, device="cuda:0"):
        self.n = n
        self.device = device

    def numel(self):
        return self.n


def _check(*a):
    import paper_1705_04159_gb300 as bp
    return bp._check_noalloc_args(*a)


def test_accepts_buffers_that_fit():
    _check(FakeDeviceTensor(100 * 8), 100, 8, FakeDeviceTensor(8), FakeDeviceTensor(64))


@pytest.mark.parametrize("x,xbar,S", [(799, 8, 64), (800, 7, 64), (800, 8, 63)])
def test_rejects_buffers_too_small(x, xbar, S):
    with pytest.raises(ValueError, match="too small"):
        _check(FakeDeviceTensor(x), 100, 8, FakeDeviceTensor(xbar), FakeDeviceTensor(S))


def test_rejects_tensors_on_different_devices():
    with pytest.raises(ValueError, match="one device"):
        _check(FakeDeviceTensor(800), 100, 8, FakeDeviceTensor(8, "cuda:1"), FakeDeviceTensor(64))


def test_rejects_host_arrays():
    import numpy as np
    with pytest.raises(TypeError, match="device tensors"):
        _check(np.zeros(800, np.float32), 100, 8, FakeDeviceTensor(8), FakeDeviceTensor(64))


@pytest.mark.parametrize("R,K", [(0, 8), (100, 0)])
def test_rejects_empty_shapes(R, K):
    with pytest.raises(ValueError, match="positive"):
        _check(FakeDeviceTensor(800), R, K, FakeDeviceTensor(8), FakeDeviceTensor(64))
