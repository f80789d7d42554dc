"""Pins of the cost-model network reference (oracle/mlp.py) that do not use the reference itself:
finite differences, a hand-computed case, the closed form of Adam's first step, dead units."""
import numpy as np
import pytest

from oracle import mlp


def _instance(seed, batch=5):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.normal(0.0, 0.4, mlp.N_PARAMS)
    X = rng.normal(0.0, 1.0, (batch, mlp.N_IN))
    T = rng.normal(0.0, 1.0, batch)
    return theta, X, T


def test_layout_size():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 == 5313


def test_gradient_matches_central_differences():
    # pick an instance whose pre-activations stay clear of the relu kink
    for seed in range(20):
        theta, X, T = _instance(seed)
        _, (a1, _, a2, _) = mlp.forward(theta, X)
        if min(np.abs(a1).min(), np.abs(a2).min()) > 1e-3:
            break
    else:
        pytest.fail("no kink-free instance")
    g, L = mlp.gradient(theta, X, T)
    assert L == pytest.approx(mlp.loss(theta, X, T), rel=1e-14)
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.size):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd[k] = (mlp.loss(tp, X, T) - mlp.loss(tm, X, T)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_hand_computed_single_path():
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["W1"][0, 0] = 2.0
    p["b1"][0] = -1.0
    p["W2"][0, 0] = 3.0
    p["w3"][0] = 0.5
    p["b3"][0] = 0.25
    theta = mlp.pack(p)
    X = np.zeros((1, 16)); X[0, 0] = 1.5
    T = np.array([1.0])
    y, _ = mlp.forward(theta, X)
    assert y[0] == pytest.approx(3.25)           # relu(2*1.5-1)=2, relu(3*2)=6, 0.5*6+0.25
    g, L = mlp.gradient(theta, X, T)
    assert L == pytest.approx(2.25 ** 2)
    gp = mlp.unpack(g)
    assert gp["b3"][0] == pytest.approx(4.5)       # 2 * (3.25 - 1)
    assert gp["w3"][0] == pytest.approx(27.0)      # 4.5 * 6
    assert gp["b2"][0] == pytest.approx(2.25)      # 4.5 * 0.5
    assert gp["W2"][0, 0] == pytest.approx(4.5)    # 2.25 * 2
    assert gp["b1"][0] == pytest.approx(6.75)      # 2.25 * 3
    assert gp["W1"][0, 0] == pytest.approx(10.125)  # 6.75 * 1.5
    nz = np.count_nonzero(g)
    assert nz == 6


def test_adam_first_step_closed_form():
    rng = np.random.Generator(np.random.PCG64(3))
    theta = rng.normal(size=mlp.N_PARAMS)
    g = rng.normal(size=mlp.N_PARAMS)
    lr = 1e-2
    t1, m, v = mlp.adam_step(theta, np.zeros_like(g), np.zeros_like(g), g, 1, lr)
    np.testing.assert_allclose(t1, theta - lr * g / (np.abs(g) + mlp.EPS), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_dead_unit_has_zero_gradient():
    theta, X, T = _instance(7)
    p = mlp.unpack(theta.copy())
    p["b1"][5] = -1e6
    th = mlp.pack(p)
    g = mlp.unpack(mlp.gradient(th, X, T)[0])
    assert np.all(g["W1"][5] == 0.0) and g["b1"][5] == 0.0
    assert np.all(g["W2"][:, 5] == 0.0)


def test_adam_constant_gradient_every_step():
    """Adam with the same gradient g at every step: m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2
    (geometric sums from zero moments), so the bias-corrected mhat = g and vhat = g^2 at every t,
    and each step moves theta by -lr * g / (|g| + eps).  A wrong exponent in a bias correction, or
    a step count starting at 0, breaks this from t = 2 on."""
    rng = np.random.Generator(np.random.PCG64(11))
    theta0 = rng.normal(size=mlp.N_PARAMS)
    g = rng.normal(size=mlp.N_PARAMS)
    lr = 3e-3
    theta, m, v = theta0.copy(), np.zeros_like(g), np.zeros_like(g)
    for t in range(1, 6):
        theta, m, v = mlp.adam_step(theta, m, v, g, t, lr)
        np.testing.assert_allclose(theta, theta0 - t * lr * g / (np.abs(g) + mlp.EPS), rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)


def test_adam_three_steps_hand_computed():
    """One parameter, gradients 1, -2, 1/2, lr = 0.1, from theta = 0 and zero moments, worked out
    in exact fractions (b1 = 9/10, b2 = 999/1000):
      t = 1: m = 1/10, v = 1/1000; mhat = m / (1 - b1) = 1, vhat = v / (1 - b2) = 1;
             theta = -0.1 * 1 / (1 + 1e-8)
      t = 2: m = 9/10 * 1/10 - 2/10 = -11/100, v = 999/1000 * 1/1000 + 4/1000 = 4999/10^6;
             mhat = m / (1 - 81/100) = -11/19, vhat = v / (1 - 998001/10^6) = 4999/1999
      t = 3: m = 9/10 * (-11/100) + 1/20 = -49/1000, v = 999/1000 * 4999/10^6 + 1/4000
             = 5244001/10^9; mhat = m / (1 - 729/1000) = -49/271,
             vhat = v / (1 - 997002999/10^9) = 749143/428143
    theta_t = theta_{t-1} - 0.1 * mhat / (sqrt(vhat) + 1e-8)."""
    want_theta = [-0.09999999900000000999999990000000099999999,
                  -0.06338964652792491179449285107285070167998,
                  -0.04972058032617827440666908045065548322021]
    want_m = [1 / 10, -11 / 100, -49 / 1000]
    want_v = [1 / 1000, 4999 / 1e6, 5244001 / 1e9]
    theta, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for t, gt in enumerate((1.0, -2.0, 0.5), 1):
        theta, m, v = mlp.adam_step(theta, m, v, np.array([gt]), t, 0.1)
        assert m[0] == pytest.approx(want_m[t - 1], rel=1e-14)
        assert v[0] == pytest.approx(want_v[t - 1], rel=1e-13)
        assert theta[0] == pytest.approx(want_theta[t - 1], rel=1e-13, abs=1e-16)
