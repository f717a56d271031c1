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


# ---------------------------------------------------------------------------
# Run-time mode (Section 5.3 steps 3-4): time head, conversion cost, gate
# ---------------------------------------------------------------------------

def test_time_head_hand_network(oracle):
    """A 2-unit hidden layer evaluated by hand: the time head reads the same
    ReLU layer as the classifier and adds its own bias per output (K label
    classes, then default CSR)."""
    names = oracle.FEATURE_NAMES
    f = np.zeros(20)
    f[names.index("max_row")] = math.e ** 2 - 1.0     # log1p -> 2
    f[names.index("diag_frac")] = 0.75                # raw
    mu, sigma = np.zeros(20), np.ones(20)
    sigma[names.index("diag_frac")] = 0.5             # z = 1.5
    W1 = np.zeros((2, 20))
    W1[0, names.index("max_row")] = 1.5               # 3.0
    W1[1, names.index("diag_frac")] = -2.0            # -3.0 + b1 -> ReLU 0
    b1 = np.array([-1.0, 0.5])
    W3 = np.array([[1.0, 10.0],                       # class 0
                   [-0.5, 4.0],                       # class 1
                   [0.25, -7.0]])                     # default CSR
    b3 = np.array([0.5, 3.0, 4.0])
    lt = oracle.time_head(f, mu, sigma, W1, b1, W3, b3)
    h0 = 2.0 * 1.5 - 1.0                              # 2.0
    h1 = max(-2.0 * 1.5 + 0.5, 0.0)                   # 0
    want = np.array([h0 + 0.5, -0.5 * h0 + 3.0, 0.25 * h0 + 4.0])
    assert h1 == 0.0
    assert np.allclose(lt, want, rtol=0, atol=1e-15)
    # the time head is not the classifier: W3 and b3 replace W2 and b2
    lg = oracle.mlp_forward(f, mu, sigma, W1, b1, W3, np.zeros(3))
    assert not np.allclose(lg, lt)


def test_conversion_cost_linear_and_clamped(oracle):
    assert oracle.conversion_cost_us((100.0, 2e-3, 5e-4), 1_000_000, 200_000) == 100.0 + 2000.0 + 100.0
    assert oracle.conversion_cost_us((-50.0, 0.0, 0.0), 10, 10) == 0.0     # never negative
    # nnz and m enter through their own coefficients
    assert oracle.conversion_cost_us((0.0, 1.0, 0.0), 7, 3) == 7.0
    assert oracle.conversion_cost_us((0.0, 0.0, 1.0), 7, 3) == 3.0


def test_gate_break_even(oracle):
    """Convert iff (t_cur - t_sel) * runs > select + pack (Section 5.3)."""
    g = oracle.gate
    # gain 10 us per product, overhead 1000 us: break-even at 100 products
    assert not g(60.0, 50.0, 400.0, 600.0, 99)
    assert not g(60.0, 50.0, 400.0, 600.0, 100)       # a tie keeps the format
    assert g(60.0, 50.0, 400.0, 600.0, 101)
    assert not g(60.0, 50.0, 0.0, 0.0, 0)             # no expected products
    assert g(60.0, 50.0, 0.0, 0.0, 1)                 # free switch of parameters
    # a slower selection never converts, however many products follow
    assert not g(50.0, 60.0, 0.0, 0.0, 10 ** 9)
    # both overhead terms count
    assert not g(60.0, 50.0, 1000.0, 0.0, 100)
    assert not g(60.0, 50.0, 0.0, 1000.0, 100)
    assert g(60.0, 50.0, 999.0, 0.0, 100)
