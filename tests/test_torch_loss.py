"""The autograd plumbing of CrvpinnLoss, against a stand-in solver whose loss
and gradient are known in closed form (LOSS = sum c_i theta_i^2).  The GPU
parity of the loss and gradient themselves is in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

from paper_2604_20731_gb300.torch_loss import CrvpinnLoss, crvpinn_loss


class QuadraticSolver:
    """Has the four members CrvpinnLoss uses: nparams, set_theta, loss_grad, get."""

    def __init__(self, c):
        self.c = np.asarray(c, dtype=np.float64)
        self.theta = None
        self.sets = 0

    @property
    def nparams(self):
        return self.c.size

    def set_theta(self, theta):
        assert theta.dtype == np.float64 and theta.shape == self.c.shape
        self.theta = theta.copy()
        self.sets += 1

    def loss_grad(self):
        return float(np.sum(self.c * self.theta ** 2))

    def get(self, field):
        assert field == "GRAD"
        return 2.0 * self.c * self.theta


def test_backward_is_the_solver_gradient():
    rng = np.random.default_rng(0)
    fake = QuadraticSolver(rng.uniform(0.5, 2.0, 7))
    theta = torch.tensor(rng.normal(size=7), requires_grad=True)
    loss = crvpinn_loss(fake, theta)
    assert loss.item() == pytest.approx(float(np.sum(fake.c * theta.detach().numpy() ** 2)), rel=1e-15)
    (3.0 * loss).backward()
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * 2.0 * fake.c * theta.detach().numpy(), rtol=1e-15)
    assert fake.sets == 1


def test_gradcheck():
    fake = QuadraticSolver(np.linspace(0.5, 1.5, 5))
    theta = torch.randn(5, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: CrvpinnLoss.apply(t, fake), (theta,))


def test_float32_parameters_and_composition():
    fake = QuadraticSolver(np.ones(4))
    theta = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float32, requires_grad=True)
    out = crvpinn_loss(fake, theta) + theta.sum()
    out.backward()
    assert theta.grad.dtype == torch.float32
    np.testing.assert_allclose(theta.grad.numpy(), 2.0 * theta.detach().numpy() + 1.0, rtol=1e-6)


def test_wrong_size_is_refused():
    fake = QuadraticSolver(np.ones(4))
    with pytest.raises(ValueError):
        crvpinn_loss(fake, torch.zeros(5, requires_grad=True))
    with pytest.raises(ValueError):
        crvpinn_loss(fake, torch.zeros(2, 2, requires_grad=True))
