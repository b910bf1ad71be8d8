"""Pins of the oracle's learned-criterion pieces (O8): the FP64 network's
backward pass against central finite differences, its C forward pass against
the numpy one, the box-to-cube distance inside the features on hand-built
geometry, and the error labels' decay with distance."""
import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from paper_1005_5384_gb300 import workloads as W


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = M.init(7) + 0.05 * rng.standard_normal(M.NPARAM)
    X = rng.standard_normal((40, 12))
    t = rng.standard_normal(40)
    L, g = M.loss_and_grad(w, X, t)
    idx = rng.choice(M.NPARAM, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(M.NPARAM)
        e[k] = h
        fd = (M.loss_and_grad(w + e, X, t)[0] - M.loss_and_grad(w - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_c_forward_matches_numpy_forward():
    rng = np.random.default_rng(4)
    w = M.init(2)
    X = rng.standard_normal((25, 12))
    y, _ = M.forward(w, X)
    for k in range(25):
        assert O.mlp_forward_c(w, X[k]) == pytest.approx(y[k], rel=1e-12, abs=1e-12)


def test_network_layout_matches_hand_computation():
    """One hidden unit active per layer: y = w3 relu(W2 relu(W1 x + b1) + b2) + b3 by hand."""
    p = {k: np.zeros(s) for k, s in M.SIZES}
    p["W1"][5, 2] = 2.0            # unit 5 reads input 2
    p["b1"][5] = -1.0
    p["W2"][9, 5] = 3.0            # unit 9 reads hidden unit 5
    p["b2"][9] = 0.5
    p["w3"][9] = -4.0
    p["b3"][0] = 0.25
    w = M.pack(p)
    x = np.zeros(12)
    x[2] = 1.5                     # z1 = 2*1.5 - 1 = 2 ; z2 = 3*2 + 0.5 = 6.5 ; y = -26 + 0.25
    assert O.mlp_forward_c(w, x) == pytest.approx(-25.75, abs=1e-14)
    assert M.forward(w, x[None, :])[0][0] == pytest.approx(-25.75, abs=1e-14)
    x[2] = 0.25                    # z1 = -0.5 -> relu 0 -> z2 = 0.5 -> y = -2 + 0.25
    assert O.mlp_forward_c(w, x) == pytest.approx(-1.75, abs=1e-14)


def test_features_on_hand_built_geometry():
    """Two tight clusters in opposite octants of the root: the far cluster's
    cube lies at a known box distance from the near cluster's box."""
    a = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5], [0.5, 0.6, 0.5], [0.6, 0.6, 0.6]])
    b = np.array([[10.0, 10.0, 10.0], [10.2, 10.0, 10.0], [10.0, 10.2, 10.0], [10.2, 10.2, 10.2]])
    pos = np.vstack([a, b])
    m = np.array([1.0, 1, 1, 1, 2, 2, 2, 2])
    T = O.Tree(pos, m, n_leaf=4, n_group=4)
    ga = [g for g, c in enumerate(T.groups) if T.count[c] == 4 and T.bmax[c, 0] < 1][0]
    cb = [c for c in range(T.n_cells) if T.count[c] == 4 and T.bmin[c, 0] > 9][0]
    f = T.mlp_features(ga, cb)
    # cell b: box [10,10.2]^3 -> cube half side 0.1, l = 0.2
    # group a: box [0.5,0.6]^3 -> gap 9.4 on every axis -> d = 9.4 sqrt(3)
    d = 9.4 * np.sqrt(3.0)
    assert f[0] == pytest.approx(np.log2(0.2), rel=1e-12)
    assert f[1] == pytest.approx(np.log2(d), rel=1e-12)
    assert f[3] == pytest.approx(0.2 / d, rel=1e-12)
    assert f[4] == pytest.approx(np.log2(8.0), rel=1e-12)
    assert f[6] == pytest.approx(2.0, rel=1e-12)
    assert np.allclose(f[7:10], 0.05 / 0.2, rtol=1e-12)
    assert f[10] == pytest.approx(1.0, rel=1e-12)


def test_labels_fall_with_distance_as_expansion_error():
    """The label of accepting a fixed cell falls as (l/d)^3 relative to a fixed
    reference force (the first neglected term is the octupole)."""
    rng = np.random.default_rng(5)
    blob = rng.random((24, 3)) * 0.5
    labels = []
    ds = np.array([6.0, 12.0, 24.0, 48.0])
    for d in ds:
        probe = np.array([[d, d, d]])   # opposite octant of the root from the blob
        pos = np.vstack([blob, probe])
        m = np.append(np.full(24, 1.0), 1e-9)
        T = O.Tree(pos, m, n_leaf=1, n_group=1)
        g = [k for k, c in enumerate(T.groups) if T.count[c] == 1 and T.bmin[c, 0] > 5][0]
        c = [k for k in range(T.n_cells) if T.count[k] == 24][0]
        aref = np.zeros((25, 3))
        aref[:, 0] = 1.0                 # fixed reference magnitude
        F, L, P = T.mlp_samples([g], 100.0, 1e-6, aref)
        labels.append(L[list(P[:, 1]).index(c)])
    slope = np.polyfit(np.log(ds), np.log(labels), 1)[0]
    assert -5.4 < slope < -4.6               # (l/d)^3 * M/d^2 -> d^-5 absolute


def _one_unit(w1, b1, w2, b2, w3, b3):
    """Network with one active unit per layer: unit 5 of layer 1 reads input 2,
    unit 9 of layer 2 reads unit 5, the output reads unit 9."""
    p = {k: np.zeros(s) for k, s in M.SIZES}
    p["W1"][5, 2], p["b1"][5] = w1, b1
    p["W2"][9, 5], p["b2"][9] = w2, b2
    p["w3"][9], p["b3"][0] = w3, b3
    return M.pack(p)


def test_bf16_forward_equals_fp64_on_bf16_values():
    """Where every operand is a BF16 value the rounding changes nothing."""
    w = _one_unit(2.0, -1.0, 3.0, 0.5, -4.0, 0.25)
    for xv, y in ((1.5, -25.75), (0.25, -1.75)):
        x = np.zeros(12)
        x[2] = xv
        assert O.mlp_forward_bf16_c(w, x) == y == O.mlp_forward_c(w, x)


def test_bf16_forward_rounds_inputs_and_hidden_layer_by_hand():
    """BF16 keeps 8 significant bits: near 1 the spacing is 2^-7, so
    1 + 2^-9 rounds to 1, the midpoint 1 + 2^-8 rounds to the even 1, and the
    midpoint 1 + 3 * 2^-8 rounds to the even 1 + 2^-6."""
    w = _one_unit(1.0, 0.0, 1.0, 0.0, 1.0, 0.0)    # y = relu(relu(x))
    x = np.zeros(12)
    for xv, y in ((1 + 2.0 ** -9, 1.0), (1 + 2.0 ** -8, 1.0), (1 + 3 * 2.0 ** -8, 1 + 2.0 ** -6),
                  (1 + 2.0 ** -7, 1 + 2.0 ** -7)):
        x[2] = xv
        assert O.mlp_forward_bf16_c(w, x) == y, xv
        assert O.mlp_forward_c(w, x) == xv
    # the first hidden layer is rounded: z1 = 1 + 2^-9 -> 1; the second is not:
    # z2 = 1 + 2^-9 stays
    x[2] = 1.0
    assert O.mlp_forward_bf16_c(_one_unit(1.0, 2.0 ** -9, 1.0, 0.0, 1.0, 0.0), x) == 1.0
    assert O.mlp_forward_bf16_c(_one_unit(1.0, 0.0, 1.0, 2.0 ** -9, 1.0, 0.0), x) == 1 + 2.0 ** -9
    # 1/3 = 1.0101010|101... * 2^-2 rounds up to 1.0101011 * 2^-2 = 171 / 512
    x[2] = 1.0 / 3.0
    assert O.mlp_forward_bf16_c(w, x) == 171.0 / 512.0
