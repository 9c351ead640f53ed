"""Pins of the seeded gauge-field generator (paper Sec. 4, Wilson plaquette action).

In two dimensions the U(1) plaquette action factorises over plaquettes, so in
infinite volume <Re U_p> = I_1(beta) / I_0(beta) exactly, and the Wilson-loop
area law gives l_sigma = [-1 / ln(I_1/I_0)]^(1/2).  The paper prints
l_sigma = 3.30 (beta = 6) and 4.35 (beta = 10); reproducing those pins the
sign and normalisation of the action, and the Metropolis average pins the
generator against the closed form.
"""
import json
import os

import numpy as np
import pytest
from scipy.special import i0, i1

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def plaquette_exact(beta):
    return i1(beta) / i0(beta)


def test_paper_correlation_lengths_from_closed_form():
    g = json.load(open(GOLDEN))["gauge_correlation_length"]
    for beta, key in ((6.0, "beta_6"), (10.0, "beta_10")):
        l_sigma = np.sqrt(-1.0 / np.log(plaquette_exact(beta)))
        assert round(l_sigma, 2) == pytest.approx(g[key], abs=1e-9)


@pytest.mark.parametrize("beta", [3.0, 6.0])
def test_metropolis_plaquette_matches_bessel_ratio(beta):
    L, therm, meas = 32, 100, 200
    theta = W.quenched_u1_angles(L, L, beta, therm, seed=21)
    rng = np.random.Generator(np.random.PCG64(22))
    samples = []
    for _ in range(meas):
        for mu in (0, 1):
            for parity in (0, 1):
                W._metropolis_half(theta, mu, parity, beta, 1.0, rng)
        samples.append(W.mean_plaquette(theta))
    samples = np.array(samples)
    # error from 20 bins of consecutive sweeps (autocorrelation-safe)
    bins = samples.reshape(20, -1).mean(axis=1)
    err = bins.std(ddof=1) / np.sqrt(len(bins))
    assert abs(samples.mean() - plaquette_exact(beta)) < 5 * err + 2e-4


def test_topological_charge_is_integer_and_deterministic():
    a = W.quenched_u1_angles(16, 16, 6.0, 50, seed=5)
    b = W.quenched_u1_angles(16, 16, 6.0, 50, seed=5)
    assert np.array_equal(a, b)
    q = W.topological_charge(a)
    assert abs(q - round(q)) < 1e-10


def test_cold_start_has_unit_plaquette():
    th = W.quenched_u1_angles(8, 8, 6.0, 0, seed=1)
    assert W.mean_plaquette(th) == 1.0
    assert W.topological_charge(th) == 0.0


def test_gaussian_field_normalisation():
    z = W.gaussian_field((200000,), 3)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z)) < 0.01


def test_noise_layout_length():
    n = W.setup_noise_len(16, 8, [(4, 4), (2, 2)], [3, 5])
    # level 1: 16x8 sites x 2 dof x (3+2); level 2: 4x2 sites x 6 dof x (5+2)
    assert n == 16 * 8 * 2 * 5 + 4 * 2 * 6 * 7
    assert W.setup_noise(16, 8, [(4, 4), (2, 2)], [3, 5], 1).shape == (n,)


def test_counter_uniforms_are_uniform_and_independent():
    """Philox4x32-10 uniforms of the counter-based generator: moments of U(0, 1),
    a flat histogram, no correlation between the two draws of a site, between
    neighbouring sites or between half-sweeps, and distinct seeds differ."""
    u, a = W.metropolis_uniforms(512, 512, 5, 3, 1, 0)
    n = u.size
    for v in (u, a):
        assert np.all((v >= 0) & (v < 1))
        assert abs(v.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
        assert abs(v.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
        h, _ = np.histogram(v, bins=64, range=(0, 1))
        chi2 = ((h - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 63 + 5 * np.sqrt(2 * 63)
    u2, _ = W.metropolis_uniforms(512, 512, 5, 3, 1, 1)
    u3, _ = W.metropolis_uniforms(512, 512, 6, 3, 1, 0)
    for x, y in ((u, a), (u.ravel()[:-1], u.ravel()[1:]), (u, u2), (u, u3)):
        assert abs(np.corrcoef(x.ravel(), y.ravel())[0, 1]) < 5 / np.sqrt(n)
    assert not np.array_equal(u, u3)
    # the 53-bit construction is exact: every value is a multiple of 2^-53
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)


def test_counter_metropolis_chunks_and_range():
    """Sweeps are functions of (seed, sweep): 6 sweeps at once equal 2 + 4 from
    the intermediate field; angles stay in [-pi, pi); Lx != Lt works."""
    full = W.quenched_u1_angles_counter(12, 8, 2.0, 6, 9)
    part = W.quenched_u1_angles_counter(12, 8, 2.0, 2, 9)
    part = W.quenched_u1_angles_counter(12, 8, 2.0, 4, 9, theta=part, first_sweep=2)
    assert np.array_equal(full, part)
    assert np.all((full >= -np.pi) & (full < np.pi))
    assert not np.array_equal(full, W.quenched_u1_angles_counter(12, 8, 2.0, 6, 10))


@pytest.mark.parametrize("beta", [3.0, 6.0])
def test_counter_metropolis_plaquette_matches_bessel_ratio(beta):
    L, therm, meas = 32, 100, 200
    theta = W.quenched_u1_angles_counter(L, L, beta, therm, seed=31)
    samples = []
    for k in range(meas):
        theta = W.quenched_u1_angles_counter(L, L, beta, 1, 31, theta=theta, first_sweep=therm + k)
        samples.append(W.mean_plaquette(theta))
    samples = np.array(samples)
    bins = samples.reshape(20, -1).mean(axis=1)
    err = bins.std(ddof=1) / np.sqrt(len(bins))
    assert abs(samples.mean() - plaquette_exact(beta)) < 5 * err + 2e-4
