"""Seeded input generators: properties the recipes state."""
import numpy as np

from paper_1611_04214_gb300.inputs import three_phase_mixture


def test_three_phase_mixture_lies_in_the_triangle_of_the_roots():
    # Barycentric combinations of the three cube roots of unity fill their triangle: every point
    # satisfies the three half-plane conditions Re(z conj(z_i)) >= -1/2.
    u1, u2 = three_phase_mixture((64, 48), seed=3)
    assert u1.shape == (64, 48) and u2.shape == (64, 48)
    for t in (0.0, 2 * np.pi / 3, -2 * np.pi / 3):
        assert np.all(u1 * np.cos(t) + u2 * np.sin(t) >= -0.5 - 1e-12)


def test_three_phase_mixture_statistics_and_seeding():
    # Dirichlet(1, 1, 1) fractions have mean 1/3 each, so the mixture averages to the centroid 0;
    # the fraction of phase 1, p1 = (1 + 2 u1)/3 on the line u2 = 0 direction, has E[p1^2] = 1/6.
    u1, u2 = three_phase_mixture((400, 400), seed=11)
    assert abs(u1.mean()) < 5e-3 and abs(u2.mean()) < 5e-3
    p1 = (1.0 + 2.0 * u1) / 3.0          # barycentric coordinate of z_1 = (1, 0)
    assert abs(np.mean(p1 ** 2) - 1.0 / 6.0) < 3e-3
    a1, a2 = three_phase_mixture((10, 10), seed=11)
    b1, _ = three_phase_mixture((10, 10), seed=12)
    assert np.array_equal(a1, three_phase_mixture((10, 10), seed=11)[0]) and not np.array_equal(a1, b1)


def test_gaussian_noise_block_is_the_crop_of_the_full_field():
    from paper_1611_04214_gb300.inputs import gaussian_noise, gaussian_noise_block
    full = gaussian_noise((64, 48), 0.05, seed=0, mean=0.1)
    for rows, cols in ((32, 48), (10, 7), (1, 1)):
        assert np.array_equal(gaussian_noise_block((64, 48), rows, cols, 0.05, seed=0, mean=0.1), full[:rows, :cols])
    assert np.array_equal(gaussian_noise_block((64, 48), 9, 11, 0.05, seed=0, mean=0.1, row0=20, col0=30),
                          full[20:29, 30:41])
