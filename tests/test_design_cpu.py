"""The design-side helpers of the differentiation path (plain tensor code that
maps a density rho to the solver's gamma): the cone density filter, the tanh
Heaviside projection and the masked design-to-gamma map, checked on CPU
against the properties that define them."""
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import autograd as A


def test_density_filter_keeps_constants_and_bounds():
    x = torch.full((6, 7, 8), 0.37, dtype=torch.float64)
    assert torch.allclose(A.density_filter(x, 2.0), x, rtol=0, atol=1e-15)
    g = torch.Generator().manual_seed(3)
    y = torch.rand((6, 7, 8), generator=g, dtype=torch.float64)
    fy = A.density_filter(y, 2.0)
    # a normalised average with non-negative weights stays within the range
    assert fy.min() >= y.min() - 1e-15 and fy.max() <= y.max() + 1e-15
    # linear in the field
    assert torch.allclose(A.density_filter(2 * y + x, 2.0), 2 * fy + x, atol=1e-14)


def test_cone_kernel_is_the_linear_cone():
    k = A.cone_kernel(2.0, 3, torch.float64)
    assert k.shape == (5, 5, 5)
    assert k[2, 2, 2] == 2.0 and k[2, 2, 3] == 1.0 and k[2, 2, 4] == 0.0
    assert torch.equal(k, k.flip(0)) and torch.equal(k, k.transpose(0, 2))


@pytest.mark.parametrize("beta,eta", [(8.0, 0.5), (4.0, 0.3), (16.0, 0.7)])
def test_heaviside_projection_fixes_the_ends_and_is_monotone(beta, eta):
    x = torch.linspace(0, 1, 101, dtype=torch.float64)
    p = A.heaviside_projection(x, beta, eta)
    assert abs(p[0].item()) < 1e-15 and abs(p[-1].item() - 1.0) < 1e-15
    assert (p[1:] >= p[:-1]).all()
    if eta == 0.5:
        assert abs(A.heaviside_projection(torch.tensor(0.5, dtype=torch.float64), beta, eta).item() - 0.5) < 1e-15


def test_design_to_gamma_keeps_fixed_nodes_and_has_the_right_gradient():
    g = torch.Generator().manual_seed(5)
    shape = (4, 5, 6)
    rho = torch.rand(shape, generator=g, dtype=torch.float64, requires_grad=True)
    mask = torch.rand(shape, generator=g) > 0.3
    fixed = torch.rand(shape, generator=g, dtype=torch.float64)
    gam = A.design_to_gamma(rho, mask, fixed, radius=1.5, beta=8.0, eta=0.5)
    assert torch.equal(gam[~mask], fixed[~mask])
    assert gam.min() >= 0 and gam.max() <= 1
    f = lambda r: A.design_to_gamma(r, mask, fixed, radius=1.5, beta=8.0, eta=0.5)
    assert torch.autograd.gradcheck(f, (rho,), eps=1e-6, atol=1e-8)
