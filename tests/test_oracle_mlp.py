"""Pins for the selector-MLP oracle (multi-class classification, Section 5.4):
a hand-evaluated 2-unit network checks the log1p input transform, the
z-scoring, the ReLU and both affine layers."""
import math

import numpy as np


def test_hand_network(oracle):
    names = oracle.FEATURE_NAMES
    assert len(names) == 20
    f = np.zeros(20)
    f[names.index("nnz")] = 1000.0          # log feature
    f[names.index("density")] = 0.25         # raw feature
    f[names.index("gini")] = 0.5             # raw feature
    mu = np.zeros(20)
    sigma = np.ones(20)
    mu[names.index("gini")] = 0.1
    sigma[names.index("gini")] = 2.0
    W1 = np.zeros((2, 20))
    W1[0, names.index("nnz")] = 1.0
    W1[0, names.index("density")] = -4.0
    W1[1, names.index("gini")] = -1.0
    b1 = np.array([0.0, 0.1])
    W2 = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 3.0]])
    b2 = np.array([0.0, 0.5, 0.0])
    logits = oracle.mlp_forward(f, mu, sigma, W1, b1, W2, b2)
    h0 = max(math.log1p(1000.0) - 1.0, 0.0)
    h1 = max(-(0.5 - 0.1) / 2.0 + 0.1, 0.0)          # = 0 after ReLU
    assert h1 == 0.0
    want = np.array([h0, h1 + 0.5, -h0 + 3 * h1])
    assert np.allclose(logits, want, rtol=0, atol=1e-15)
    assert int(np.argmax(logits)) == 0


def test_log_features_are_the_count_like_ones(oracle):
    z = oracle.mlp_inputs(np.full(20, math.e - 1.0), np.zeros(20), np.ones(20))
    for k, name in enumerate(oracle.FEATURE_NAMES):
        want = 1.0 if name in oracle.LOG_FEATURES else math.e - 1.0
        assert abs(z[k] - want) < 1e-15, name
