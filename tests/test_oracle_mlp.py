"""Pins of the learned-upsampler oracle (oracle/mlp.py): gradients against
finite differences, features and targets against closed forms, and the
zero network against the plain Hermite boundary."""
import numpy as np
import pytest

from oracle import mlp
from flowcases import faces_from


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    K = 4
    p = mlp.init_params(1, K, scale=1.0)
    p["b1"] = rng.normal(0, 0.1, mlp.HIDDEN)  # move pre-activations off zero
    p["b2"] = rng.normal(0, 0.1, mlp.HIDDEN)
    X = rng.normal(0, 1, (7, mlp.NIN))
    X[:, mlp.NFEAT:] = 0.0
    T = rng.normal(0, 1, (7, 3 * K))
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, T)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 12, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)[0], T)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)), (name, idx, fd, an)


def test_features_of_a_linear_field():
    # sample features are the samples; in-face differences of a field linear
    # in space are its exact gradient, central and one-sided alike
    E, K, u_max = 8, 4, 0.05
    a = np.array([0.01, -0.02, 0.005])
    G = np.array([[1e-3, -2e-3, 5e-4], [3e-4, 1e-3, -1e-3], [-7e-4, 2e-4, 6e-4]])
    fn = lambda X, Y, Z, t: tuple(a[c] + G[c, 0] * X + G[c, 1] * Y + G[c, 2] * Z + 1e-4 * c * t for c in range(3))
    S = faces_from(fn, E, 5, K)
    X = mlp.features(S, 1, u_max)
    # face 2 (y = 0): p = x, q = z; row (f E + q) E + p
    f, q, pp = 2, 5, 3
    row = (f * E + q) * E + pp
    for k, jj in enumerate((0, 1, 2, 3)):
        assert np.allclose(X[row, 3 * k:3 * k + 3], S[jj, f, :, q, pp] / u_max, atol=1e-13)
    for k, jj in enumerate((1, 2)):
        gp = X[row, 12 + 6 * k:12 + 6 * k + 3] * u_max
        gq = X[row, 15 + 6 * k:15 + 6 * k + 3] * u_max
        assert np.allclose(gp, G[:, 0], atol=1e-15) and np.allclose(gq, G[:, 2], atol=1e-15)
    row_edge = (0 * E + 0) * E + (E - 1)  # face x-, q = z = 0, p = y = E - 1 (one-sided in both)
    gp = X[row_edge, 12:15] * u_max
    gq = X[row_edge, 15:18] * u_max
    assert np.allclose(gp, G[:, 1], atol=1e-15) and np.allclose(gq, G[:, 2], atol=1e-15)
    assert np.all(X[:, mlp.NFEAT:] == 0.0)


def test_targets_vanish_for_quadratic_time_series():
    # Catmull-Rom Hermite is exact on quadratics, so the residual to learn is zero
    E, K = 8, 4
    fn = lambda X, Y, Z, t: (0.01 + 1e-3 * t - 2e-5 * t * t + 0 * X, 2e-4 * t + 1e-3 * Y, -0.01 + 3e-6 * t * t + 0 * Z)
    fine = faces_from(fn, E, 6 * K + 1, 1)
    coarse = fine[::K]
    for j in (1, 2, 3):
        assert np.abs(mlp.targets(fine, coarse, j, K, 0.05)).max() < 1e-12
    # but not for a cubic in time: a non-trivial target exists
    fn3 = lambda X, Y, Z, t: (1e-6 * t ** 3 + 0 * X, 0 * Y, 0 * Z)
    fine3 = faces_from(fn3, E, 6 * K + 1, 1)
    assert np.abs(mlp.targets(fine3, fine3[::K], 2, K, 0.05)).max() > 1e-6


def test_residual_layout_from_the_output_bias():
    E, K, u_max = 8, 4, 0.05
    p = mlp.init_params(0, K)
    for k in p:
        p[k] = np.zeros_like(p[k])
    s, c = 2, 1
    p["b3"][3 * s + c] = 0.5
    S = np.zeros((6, 6, 3, E, E))
    R = mlp.residual_block(p, S, 1, K, u_max)
    assert np.allclose(R[:, c, s], 0.5 * u_max / mlp.OUT_DIV) and np.count_nonzero(R) == 6 * E * E


def test_zero_network_reproduces_hermite_boundary(orc):
    E, K, steps = 16, 4, 24
    from paper_0809_4958_gb300 import inputs
    modes = inputs.mode_table(4, 32, 1, 4, E)
    S = orc.face_samples(modes, E, K, 0, steps // K + 4)
    u0 = orc.volume_field(modes, E, 0.0)
    p = mlp.init_params(0, K)
    for k in p:
        p[k] = np.zeros_like(p[k])
    resid = np.stack([mlp.residual_block(p, S, j, K, 0.05) for j in range(steps // K)])
    herm = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_HERMITE), u0, S)
    mlpr = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_MLP), u0, S, resid=resid)
    assert herm.run(steps) == 0 and mlpr.run(steps) == 0
    assert np.array_equal(herm.f, mlpr.f)
    # a non-zero residual changes the boundary and hence the interior
    resid[1, 0, 0, 2] += 1e-3
    mlpr2 = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_MLP), u0, S, resid=resid)
    assert mlpr2.run(steps) == 0 and not np.array_equal(herm.f, mlpr2.f)


def test_exact_targets_reproduce_the_every_step_boundary(orc):
    # the targets, used as the residual of the boundary, must give back the
    # boundary of the run that sees a sample every step: same substep, face,
    # site and unit on both sides of the definition
    E, K, steps = 16, 4, 24
    from paper_0809_4958_gb300 import inputs
    modes = inputs.mode_table(4, 32, 1, 4, E)
    fine = orc.face_samples(modes, E, 1, 0, steps + 4 * K + 1)
    S = fine[::K]
    u0 = orc.volume_field(modes, E, 0.0)
    u_max = 0.05
    resid = np.zeros((steps // K, 6, 3, K, E, E))
    for j in range(steps // K):
        T = mlp.targets(fine, S, j, K, u_max)
        for s in range(K):
            for c in range(3):
                resid[j, :, c, s] = T[:, 3 * s + c].reshape(6, E, E) * (u_max / mlp.OUT_DIV)
    every = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=1, time_interp=orc.TIME_LINEAR), u0, fine)
    learned = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_MLP), u0, S, resid=resid)
    herm = orc.Sim(orc.BoxParams(E=E, tau=0.8, K=K, time_interp=orc.TIME_HERMITE), u0, S)
    assert every.run(steps) == 0 and learned.run(steps) == 0 and herm.run(steps) == 0
    u = every.fields()[1]
    assert np.max(np.abs(learned.fields()[1] - u)) <= 1e-15
    assert np.max(np.abs(herm.fields()[1] - u)) > 1e-7  # Hermite alone misses it
