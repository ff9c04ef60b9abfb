"""The autograd wrapper's host logic (no GPU): log_z hands theta to the context's grad
call, returns its log Z, and its backward scales the kept gradient by the incoming one."""
import torch

import paper_2312_06484_gb300 as gp


class _FakeFilter:
    """Stands in for an AIRPF context: log Z_b = sum_d c_d theta_bd^2 (so the gradient is
    2 c theta), returned with the gradient the way AIRPF.grad returns them."""

    def __init__(self, c):
        self.c = c
        self.calls = []

    def grad(self, theta, y, *, chain0=0, iter=0):
        self.calls.append((chain0, iter, tuple(y.shape)))
        th = theta.detach().reshape(-1, self.c.numel()).double()
        return {"log_z": (self.c * th * th).sum(dim=1), "grad": 2 * self.c * th,
                "score": torch.zeros_like(th)}


def test_log_z_forward_and_backward_batch():
    c = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    f = _FakeFilter(c)
    th = torch.tensor([[0.3, 1.0, -2.0], [1.5, -0.5, 4.0]], dtype=torch.float64, requires_grad=True)
    y = torch.zeros(7, dtype=torch.float64)
    lz = gp.log_z(f, th, y, chain0=5, iter=9)
    assert f.calls == [(5, 9, (7,))]
    torch.testing.assert_close(lz, (c * th.detach() ** 2).sum(dim=1))
    w = torch.tensor([2.0, -1.0], dtype=torch.float64)
    (w * lz).sum().backward()
    torch.testing.assert_close(th.grad, w[:, None] * 2 * c * th.detach())


def test_log_z_single_filter_keeps_theta_shape_and_dtype():
    c = torch.tensor([1.0, 3.0], dtype=torch.float64)
    th = torch.tensor([0.5, -1.0], dtype=torch.float32, requires_grad=True)
    lz = gp.log_z(_FakeFilter(c), th, torch.zeros(3))
    lz.sum().backward()
    assert th.grad.shape == th.shape and th.grad.dtype == torch.float32
    torch.testing.assert_close(th.grad, (2 * c * th.detach().double()).float())
