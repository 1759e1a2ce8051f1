"""The seeded input recipes (no GPU): the Gaussian random field behind the variable
coefficients a = exp(g) has unit variance and the squared-exponential correlation of
length 1/16 on the unit square (statistics over 200 seeded fields of 64 x 64 cells); the
mixed-batch sizes are 2^m - 1 within the requested range; (eps, theta) are log-uniform
and uniform over their ranges; right-hand sides are uniform[-1, 1] and the loss vectors
standard normal."""
import numpy as np
import pytest

from paper_2102_12071_gb300 import inputs


@pytest.fixture(scope="module")
def fields():
    n = 63
    return n + 1, np.stack([np.log(inputs.grf_cells(10_000 + s, n).astype(np.float64)) for s in range(200)])


def test_grf_has_unit_variance_and_zero_mean(fields):
    _, g = fields
    assert abs(g.mean()) < 0.05
    assert abs(g.var() - 1.0) < 0.05


@pytest.mark.parametrize("lag", [1, 4, 8])
def test_grf_correlation_is_squared_exponential_of_length_one_sixteenth(fields, lag):
    m, g = fields
    expect = np.exp(-((lag / m) ** 2) / (2.0 * (1.0 / 16.0) ** 2))
    for axis in (1, 2):  # isotropic: rows and columns alike
        assert abs(np.mean(g * np.roll(g, lag, axis=axis)) - expect) < 0.03


def test_mixed_batch_sizes_are_admissible():
    sizes = inputs.grid_sizes_loguniform(7, 256)
    assert all(((s + 1) & s) == 0 and 63 <= s <= 2047 for s in sizes)
    assert len(set(sizes)) >= 5  # log-uniform over the range, not one size


def test_rotated_parameters_are_log_uniform_eps_and_uniform_theta():
    pairs = inputs.rotated_params(3, 4000)
    le = np.log10([e for e, _ in pairs])
    th = np.array([t for _, t in pairs])
    assert le.min() >= -3.0 and le.max() <= 0.0 and th.min() >= 0.0 and th.max() <= np.pi
    # uniform in log10(eps) and in theta: quartiles at a quarter of each range
    np.testing.assert_allclose(np.quantile(le, [0.25, 0.5, 0.75]), [-2.25, -1.5, -0.75], atol=0.08)
    np.testing.assert_allclose(np.quantile(th, [0.25, 0.5, 0.75]), np.pi * np.array([0.25, 0.5, 0.75]), atol=0.08)
    assert inputs.rotated_params(3, 4000) == pairs  # seeded: reproducible


def test_right_hand_sides_and_loss_vectors():
    b = inputs.rhs_uniform(1, 255)
    assert b.dtype == np.float32 and b.shape == (255, 255)
    assert b.min() >= -1.0 and b.max() <= 1.0 and abs(b.var() - 1.0 / 3.0) < 0.01
    z = inputs.gaussian_vectors(2, 8, 63)
    assert z.dtype == np.float32 and z.shape == (8, 63, 63)
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    assert np.array_equal(inputs.rhs_uniform(1, 255), b)  # reproducible


def test_sine_coefficient_of_the_variable_coefficient_experiment():
    """Sec. 6.3: a = sin(kappa pi x y) + 1.1 at cell centres, row = y, column = x."""
    n = 15
    a = inputs.sine_cells(n, 1.0)
    assert a.dtype == np.float32 and a.shape == (n + 1, n + 1)
    np.testing.assert_array_equal(a, a.T)  # symmetric in x and y
    # with kappa = 1 the argument kappa pi x y stays in (0, pi): a in (1.1, 2.1]
    assert a.min() > 1.1 and a.max() <= 2.1
    h = 1.0 / (n + 1)
    x, y = 5.5 * h, 2.5 * h  # cell (row 2, column 5)
    assert abs(float(a[2, 5]) - (np.sin(np.pi * x * y) + 1.1)) < 1e-7
    # kappa = 10 reaches the minimum 0.1 of the paper's coefficient range
    assert inputs.sine_cells(255, 10.0).min() < 0.11
