"""Host-side plumbing of the autograd Function over the adjoint run: the
gradient it hands back to autograd (accumulated in FP64 on the host) takes
theta's dtype and device, and the field gradients pass through unchanged.
No GPU needed: the run is replaced by an object with its interface."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def make_function():
    from paper_1907_13088_gb300 import build

    build.build()
    from paper_1907_13088_gb300.adjoint import make_function as mf

    return mf


class FakeRun:
    """forward: E^N = 2 E0, B^N = 3 B0 (theta enters only the recorded call);
    backward: dL/dtheta = theta * 10 in FP64, dL/dE0 = 2 gE, dL/dB0 = 3 gB."""

    def __init__(self):
        self.calls = []

    def forward(self, th, E0, B0):
        self.calls.append(("forward", th.dtype, th.copy()))
        return 2.0 * E0, 3.0 * B0

    def backward(self, th, gE, gB, recompute):
        self.calls.append(("backward", recompute))
        return np.asarray(th, dtype=np.float64) * 10.0, 2.0 * gE, 3.0 * gB


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_theta_gradient_dtype_and_fields(make_function, dtype):
    run = FakeRun()
    th = torch.tensor([0.5, -1.25, 2.0], dtype=dtype, requires_grad=True)
    e0 = torch.ones((3, 4, 5), dtype=torch.float32, requires_grad=True)
    b0 = torch.ones((3, 4, 5), dtype=torch.float32, requires_grad=True)
    EN, BN = make_function().apply(th, e0, b0, run, True)
    (EN.sum() + 2.0 * BN.sum()).backward()
    assert run.calls[0][1] == np.float64 and run.calls[1] == ("backward", True)
    assert th.grad.dtype == dtype and th.grad.device == th.device
    np.testing.assert_allclose(th.grad.double().numpy(), [5.0, -12.5, 20.0])
    np.testing.assert_array_equal(e0.grad.numpy(), np.full((3, 4, 5), 2.0, np.float32))
    np.testing.assert_array_equal(b0.grad.numpy(), np.full((3, 4, 5), 6.0, np.float32))
