"""Host logic of the autograd wrappers of the reverse-mode calls (no GPU):
backward returns grad_output times the gradient the forward sweep produced,
with one None per non-tensor argument."""
import numpy as np
import pytest


def test_adjoint_function_plumbing():
    torch = pytest.importorskip("torch")
    from paper_2510_18688_gb300 import sensitivity as S
    Fn = S._adjoint_fn("Quadratic", lambda q, a, b: (float(q @ q), 2.0 * q))
    q = torch.tensor([1.0, 2.0, -0.5], dtype=torch.float64, requires_grad=True)
    y = Fn.apply(q, "cfg", 7)
    (5.0 * y).backward()
    assert float(y.detach()) == pytest.approx(5.25)
    assert np.allclose(q.grad.numpy(), 5.0 * 2.0 * np.array([1.0, 2.0, -0.5]))
